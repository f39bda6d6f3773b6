"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the method: it only draws auxiliary-field
configurations s[tau, i] in {-1, +1} (int8, tau-major, shape (M, N)) with
numpy's PCG64 generator.  Three value structures stand in for the paper's
workloads (configurations at its finite-temperature critical point):

  uniform  -- independent +-1 with probability 1/2 each;
  domains  -- ferromagnetic domains with long imaginary-time correlation:
              the sign of a Gaussian field smoothed over `corr` sites in space
              and `corr_t` slices in time (periodic box filter);
  ordered  -- all +1 (the closed-form uniform-field case).
"""
import numpy as np


def uniform_field(seed, M, N):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.where(rng.random((M, N)) < 0.5, -1, 1).astype(np.int8)


def domain_field(seed, M, Lx, Ly, corr=3, corr_t=None):
    """Sign of a periodic box-smoothed Gaussian field on the (M, Ly, Lx) grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    corr_t = max(1, M // 4) if corr_t is None else corr_t
    g = rng.standard_normal((M, Ly, Lx))
    for axis, w in ((0, corr_t), (1, corr), (2, corr)):
        acc = np.zeros_like(g)
        for k in range(-(w // 2), w - w // 2):
            acc += np.roll(g, k, axis=axis)
        g = acc
    s = np.where(g >= 0.0, 1, -1).astype(np.int8)
    return s.reshape(M, Lx * Ly)


def ordered_field(M, N, value=1):
    return np.full((M, N), value, dtype=np.int8)


def batch_uniform(seed, B, M, N):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.where(rng.random((B, M, N)) < 0.5, -1, 1).astype(np.int8)
