"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package holds no arithmetic of the method itself (no kernel evaluation,
no pivoting, no normalisation).  It only produces point clouds X (N x d) with
the shapes and value distributions of the paper's workloads (Section 4: the
Kuramoto-Sivashinsky equation, Eq. (ks), its delay embeddings, Eq.
(data-kernel)) and the bandwidth epsilon for them.
"""
from .ks import ks_trajectory, etdrk4_coefficients
from .embed import delay_embed_vsa, delay_embed_neighbours
from .workloads import (median_sq_distance, make_config, CONFIGS, batched_problems,
                        gaussian_mixture)

__all__ = ["ks_trajectory", "etdrk4_coefficients", "delay_embed_vsa",
           "delay_embed_neighbours", "median_sq_distance", "make_config", "CONFIGS",
           "batched_problems", "gaussian_mixture"]
