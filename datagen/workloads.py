"""Named synthetic workloads with the shapes of the paper's experiments.

Every workload is seeded; the recipe of each is stated in its docstring entry
of CONFIGS.  The bandwidth epsilon of the Gaussian kernel exp(-|x-y|^2/eps) is
the median of the pairwise squared distances (exact over all pairs for
N <= 20,000, else over 2^20 seeded pairs i != j); the paper's own rule (a
scaling-based calibration) gives eps=32 for its data, which the caller may pass
instead.
"""
import numpy as np
from .ks import ks_trajectory
from .embed import delay_embed_vsa, delay_embed_neighbours


def median_sq_distance(X, seed=0, exact_max=20000, n_pairs=1 << 20):
    """Median of |x_i - x_j|^2 over i<j (exact) or over seeded random pairs i != j."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    if N <= exact_max:
        from scipy.spatial.distance import pdist
        return float(np.median(pdist(X, "sqeuclidean")))
    rng = np.random.Generator(np.random.PCG64(seed + 0x5EED))
    i = rng.integers(0, N, n_pairs)
    j = rng.integers(0, N - 1, n_pairs)
    j = j + (j >= i)                                  # uniform over j != i
    diff = X[i] - X[j]
    return float(np.median(np.einsum("ij,ij->i", diff, diff)))


def _ks_points(n_times, seed, n_ens=1):
    return ks_trajectory(n_times, seed=seed, n_ens=n_ens)


def _vsa(n_times_total, J, seed, n_ens, neighbours, ic="random", spinup=1000.0):
    per = n_times_total // n_ens
    u = ks_trajectory(n_ens * (per + J - 1), seed=seed, n_ens=n_ens, ic=ic, spinup=spinup)
    u = u.reshape(n_ens, per + J - 1, -1)
    emb = delay_embed_neighbours if neighbours else delay_embed_vsa
    return np.concatenate([emb(u[e], J) for e in range(n_ens)], axis=0)


# name -> dict(recipe).  "method" is "greedy" (b=1) or "arpc".
CONFIGS = {
    # KS states (64 grid values), one trajectory, 1.0 t.u. apart after 1,000 t.u. spin-up.
    "ks2k": dict(N=2000, d=64, dtype="f64", method="greedy", r=128, b=1, k=32,
                 seed=1, ens=1, kind="ks"),
    # Same generator at scale: 100 independent trajectories x 2,000 samples each.
    "ks200k": dict(N=200000, d=64, dtype="f64", method="arpc", r=1024, b=64, k=64,
                   seed=2, ens=100, kind="ks"),
    # 8,192 times x 64 grid points, q=32 delays at x_{m-1}, x_m, x_{m+1}: d=96.
    "vsa524k": dict(N=524288, d=96, dtype="f32", method="arpc", r=2048, b=128, k=128,
                    seed=3, ens=1, kind="vsa_nb", q=32),
    # 31,250 times x 64 grid points, J=128 delays at one grid point: d=128.
    "vsa2m": dict(N=2000000, d=128, dtype="f32", method="arpc", r=2048, b=128, k=256,
                  seed=5, ens=10, kind="vsa", q=128),
    # Section 4.1 (first experiment): the paper's initial condition, 2,500 t.u. spin-up,
    # 575 samples, J = 64 delays at one grid point: 512 x 64 = 32,768 points; the
    # paper's bandwidth eps = 32 in exp(-|x-y|^2 / (eps J)), i.e. 2,048 here.
    "paper32k": dict(N=32768, d=64, dtype="f32", method="arpc", r=4096, b=64, k=64,
                     seed=6, ens=1, kind="vsa", q=64, ic="paper", spinup=2500.0, eps_fixed=32.0 * 64),
    # Section 4.2 (second experiment): 2,111 t.u. of samples -> 2,048 x 64 = 131,072 points.
    # Median-rule bandwidth: with eps = 32 J the kernel's numerical rank here is ~300, below
    # the ranks the paper sweeps (128 .. 16,384).
    "paper131k": dict(N=131072, d=64, dtype="f32", method="arpc", r=4096, b=64, k=64,
                      seed=7, ens=1, kind="vsa", q=64, ic="paper", spinup=2500.0),
}


def make_config(name, N=None, seed=None):
    """Build (X, eps, cfg) for a named workload; ``N`` truncates for smaller cases."""
    cfg = dict(CONFIGS[name])
    if seed is not None:
        cfg["seed"] = seed
    if cfg["kind"] == "ks":
        n = cfg["N"] if N is None else N
        ens = n // 2000 if n % 2000 == 0 else 1          # 2,000 samples per trajectory
        X = _ks_points(n, cfg["seed"], ens)
    else:
        M = 64
        times = cfg["N"] // M if N is None else -(-N // M)
        ens = cfg["ens"] if times % cfg["ens"] == 0 and times >= 100 * cfg["ens"] else 1
        X = _vsa(times, cfg["q"], cfg["seed"], ens, cfg["kind"] == "vsa_nb", cfg.get("ic", "random"),
                 cfg.get("spinup", 1000.0))
        if N is not None:
            X = X[:N]
    cfg["N"] = X.shape[0]
    X = np.ascontiguousarray(X, dtype=np.float64 if cfg["dtype"] == "f64" else np.float32)
    eps = cfg["eps_fixed"] if "eps_fixed" in cfg else median_sq_distance(X, seed=cfg["seed"])
    return X, eps, cfg


def gaussian_mixture(N, means, sigma, seed):
    """N points from an equal-weight isotropic Gaussian mixture with the given means."""
    rng = np.random.Generator(np.random.PCG64(seed))
    comp = rng.integers(0, means.shape[0], N)
    return means[comp] + sigma * rng.standard_normal((N, means.shape[1]))


def batched_problems(n_prob=64, seed=4, n_range=(5000, 100000), r_range=(128, 512)):
    """Independent problems of uneven N, d, eps and r.

    Per problem: N ~ U[n_range], d in {32, 64, 128}, 8-component isotropic
    Gaussian mixture whose means are 8 states of a KS sub-trajectory (d=32: every
    other grid value, d=64: the state, d=128: state followed by the next state),
    sigma = 0.1 x the RMS distance between means, eps = {0.25,0.5,1,2} x the
    median squared distance, r ~ U[r_range].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    u = ks_trajectory(n_prob * 9, seed=seed + 100, n_ens=n_prob)   # 9 states per problem
    u = u.reshape(n_prob, 9, -1)
    probs = []
    for p in range(n_prob):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(rng.choice([32, 64, 128]))
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        scale = float(rng.choice([0.25, 0.5, 1.0, 2.0]))
        states = u[p]
        if d == 32:
            means = states[:8, ::2]
        elif d == 64:
            means = states[:8]
        else:
            means = np.concatenate([states[:8], states[1:9]], axis=1)
        diff = means[:, None, :] - means[None, :, :]
        sep = np.sqrt(np.sum(diff ** 2) / (8 * 7))
        X = gaussian_mixture(N, means, 0.1 * sep, seed * 1000 + p)
        eps = scale * median_sq_distance(X, seed=p)
        probs.append(dict(X=X, eps=eps, N=N, d=d, r=r, k=16, b=min(64, r), seed=2000 + p))
    return probs
