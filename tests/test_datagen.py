"""Sanity of the seeded input generators (not part of the method)."""
import numpy as np

from datagen import etdrk4_coefficients, ks_trajectory, delay_embed_vsa, delay_embed_neighbours
from datagen import make_config, median_sq_distance


def test_etdrk4_coefficients_match_closed_forms():
    h = 0.25
    lin = np.array([-3.0, -1.0, 0.5, 2.0])
    E, E2, Q, f1, f2, f3 = etdrk4_coefficients(lin, h)
    z = h * lin
    assert np.allclose(E, np.exp(z)) and np.allclose(E2, np.exp(z / 2))
    assert np.allclose(Q, h * (np.exp(z / 2) - 1) / z, rtol=1e-12)
    assert np.allclose(f1, h * (-4 - z + np.exp(z) * (4 - 3 * z + z * z)) / z ** 3, rtol=1e-10)
    assert np.allclose(f2, h * (2 + z + np.exp(z) * (-2 + z)) / z ** 3, rtol=1e-10)
    assert np.allclose(f3, h * (-4 - 3 * z - z * z + np.exp(z) * (4 - z)) / z ** 3, rtol=1e-10)


def test_ks_trajectory_shape_seed_and_mean():
    u = ks_trajectory(50, seed=3, spinup=50.0)
    assert u.shape == (50, 64)
    assert np.allclose(u.mean(axis=1), 0.0, atol=1e-12)       # KS conserves the mean (0)
    assert np.array_equal(u, ks_trajectory(50, seed=3, spinup=50.0))
    assert 0.3 < u.std() < 3.0                                 # on the chaotic attractor


def test_delay_embeddings():
    u = np.arange(5 * 4, dtype=float).reshape(5, 4)           # u[t, m] = 4t + m
    X = delay_embed_vsa(u, 3)
    assert X.shape == (3 * 4, 3)
    assert X[0].tolist() == [u[2, 0], u[1, 0], u[0, 0]]
    assert X[5].tolist() == [u[3, 1], u[2, 1], u[1, 1]]
    Y = delay_embed_neighbours(u, 2)
    assert Y.shape == (4 * 4, 6)
    # point (t=1, m=0): neighbours m-1 = 3 (periodic), 0, 1
    assert Y[0].tolist() == [u[1, 3], u[0, 3], u[1, 0], u[0, 0], u[1, 1], u[0, 1]]


def test_median_rule_and_configs():
    X = np.array([[0.0], [1.0], [3.0]])                        # squared distances 1, 9, 4
    assert median_sq_distance(X) == 4.0
    X, eps, cfg = make_config("ks2k", N=300)
    assert X.shape == (300, 64) and X.dtype == np.float64 and eps > 0
    X, eps, cfg = make_config("vsa524k", N=640)
    assert X.shape == (640, 96) and X.dtype == np.float32
