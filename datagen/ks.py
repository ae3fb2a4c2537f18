"""Kuramoto-Sivashinsky trajectories, u_t = -u u_x - u_xx - u_xxxx (Section 4, Eq. (ks)).

Periodic domain of length L, M Fourier modes, pseudospectral nonlinearity with
3/2 zero-padding dealiasing, ETDRK4 time stepping (Cox & Matthews 2002) whose
phi-function coefficients are evaluated by the contour-integral mean of
Kassam & Trefethen 2005 (Section 4.1 of the paper fixes L=22, M=64, dt=0.25).

Several independent trajectories can be integrated at once (``n_ens``): each
starts from its own seeded random state, is spun up, and its samples are
concatenated.  All trajectories sample the same chaotic attractor.
"""
import numpy as np


def etdrk4_coefficients(lin, h, n_contour=32):
    """ETDRK4 coefficients for the diagonal linear operator ``lin`` and step h.

    Returns (E, E2, Qc, f1, f2, f3) with E = exp(h lin), E2 = exp(h lin / 2) and
    the three phi-type weights of the fourth-order update.  Each weight is the
    mean of its analytic expression over n_contour points on a unit circle
    around h*lin, which avoids the cancellation of the closed forms near 0.
    """
    lin = np.asarray(lin, dtype=np.float64)
    E = np.exp(h * lin)
    E2 = np.exp(h * lin / 2)
    roots = np.exp(1j * np.pi * (np.arange(1, n_contour + 1) - 0.5) / n_contour)
    z = h * lin[:, None] + roots[None, :]
    Qc = h * np.real(np.mean((np.exp(z / 2) - 1) / z, axis=1))
    f1 = h * np.real(np.mean((-4 - z + np.exp(z) * (4 - 3 * z + z ** 2)) / z ** 3, axis=1))
    f2 = h * np.real(np.mean((2 + z + np.exp(z) * (-2 + z)) / z ** 3, axis=1))
    f3 = h * np.real(np.mean((-4 - 3 * z - z ** 2 + np.exp(z) * (4 - z)) / z ** 3, axis=1))
    return E, E2, Qc, f1, f2, f3


class _KS:
    def __init__(self, L=22.0, M=64, dt=0.25):
        self.M = M
        self.Mp = (3 * M) // 2                       # padded grid for dealiasing
        self.nk = M // 2                             # retained modes 0..M/2-1 (Nyquist dropped)
        self.q = 2 * np.pi / L * np.arange(self.nk)  # wavenumbers
        lin = self.q ** 2 - self.q ** 4              # -d_xx - d_xxxx in Fourier space
        self.coef = etdrk4_coefficients(lin, dt)
        # -1/2 d_x (u^2) in Fourier space
        self.g = -0.5j * self.q

    def to_spec(self, u):
        return np.fft.rfft(u, axis=-1)[..., : self.nk] / self.M

    def to_grid(self, v):
        full = np.zeros(v.shape[:-1] + (self.M // 2 + 1,), dtype=np.complex128)
        full[..., : self.nk] = v
        return np.fft.irfft(full, n=self.M, axis=-1) * self.M

    def nonlin(self, v):
        pad = np.zeros(v.shape[:-1] + (self.Mp // 2 + 1,), dtype=np.complex128)
        pad[..., : self.nk] = v
        u = np.fft.irfft(pad, n=self.Mp, axis=-1) * self.Mp
        w = np.fft.rfft(u * u, axis=-1)[..., : self.nk] / self.Mp
        return self.g * w

    def step(self, v):
        E, E2, Qc, f1, f2, f3 = self.coef
        Nv = self.nonlin(v)
        a = E2 * v + Qc * Nv
        Na = self.nonlin(a)
        b = E2 * v + Qc * Na
        Nb = self.nonlin(b)
        c = E2 * a + Qc * (2 * Nb - Nv)
        Nc = self.nonlin(c)
        return E * v + Nv * f1 + 2 * (Na + Nb) * f2 + Nc * f3


def ks_trajectory(n_samples, seed, n_ens=1, L=22.0, M=64, dt=0.25, spinup=1000.0,
                  sample_every=1.0, amplitude=0.1, ic="random"):
    """Grid values u(t_j, x_m) of KS trajectories, shape (n_samples, M), float64.

    ic="random": each of the ``n_ens`` trajectories starts from amplitude * xi
    with xi ~ N(0,1) per grid point (mean removed, since KS conserves the
    spatial mean).  ic="paper": the initial condition of Section 4.1, the
    leading four Fourier coefficients (wavenumbers 1..4) equal to 0.6 and the
    rest zero, in the convention u = sum_k c_k exp(i q_k x) + c.c.  The state is
    integrated for ``spinup`` time units and then sampled every
    ``sample_every`` time units.  Rows are ordered trajectory-major.
    """
    if n_samples % n_ens:
        raise ValueError("n_samples must be a multiple of n_ens")
    per = n_samples // n_ens
    ks = _KS(L, M, dt)
    if ic == "paper":
        v = np.zeros((n_ens, ks.nk), dtype=np.complex128)
        v[:, 1:5] = 0.6
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        u0 = amplitude * rng.standard_normal((n_ens, M))
        u0 -= u0.mean(axis=1, keepdims=True)
        v = ks.to_spec(u0)
    n_spin = int(round(spinup / dt))
    every = int(round(sample_every / dt))
    for _ in range(n_spin):
        v = ks.step(v)
    out = np.empty((n_ens, per, M))
    for j in range(per):
        out[:, j] = ks.to_grid(v)
        if j + 1 < per:
            for _ in range(every):
                v = ks.step(v)
    return out.reshape(n_samples, M)
