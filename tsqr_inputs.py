"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds input generation only: it contains none of the
factorisation's arithmetic and imports neither the oracle nor the CUDA
library.  Every generator is a pure function of its seed (numpy PCG64).

Workloads (the matrix shapes of the paper's experiments are unnamed HDFS
matrices, Sec. V; these synthetic stand-ins have the shapes and spectra the
benchmark configurations name):

* ``gaussian(m, n, seed)``          -- i.i.d. N(0, 1).
* ``conditioned(m, n, kappa, seed)`` -- A = G diag(sigma) V^T with G i.i.d.
  N(0, 1/m), sigma log-spaced from 1 to 1/kappa, V a random orthogonal n x n
  matrix (the Q factor of a seeded Gaussian, taken from numpy's LAPACK QR).
* ``column_scaled(m, n, lo, seed)``  -- i.i.d. N(0, 1) times column factors
  log-spaced over [1, lo].
* ``power_spectrum(m, n, seed)``     -- A = G diag(j^-2) V^T (G ~ N(0, 1/m)).
"""
from __future__ import annotations

import numpy as np

# Seeds of the five benchmark configurations.
SEED_SMALL = 1301107101
SEED_SWEEP = 1301107102
SEED_MIXED = 1301107103
SEED_SVD = 1301107104
SEED_GRAD = 1301107105

_ROW_CHUNK = 1 << 20


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(m: int, n: int, seed: int, dtype=np.float64, rows: int | None = None) -> np.ndarray:
    """m x n i.i.d. N(0, 1), generated in FP64 row chunks then cast.  `rows`
    returns only the first rows of that matrix (a sample of the workload)."""
    rng = _rng(seed)
    mm = m if rows is None else min(m, rows)
    out = np.empty((mm, n), dtype=dtype)
    for r0 in range(0, mm, _ROW_CHUNK):
        r1 = min(mm, r0 + _ROW_CHUNK)
        out[r0:r1] = rng.standard_normal((r1 - r0, n))
    return out


def random_orthogonal(n: int, seed: int) -> np.ndarray:
    """Random orthogonal n x n: Q factor (numpy/LAPACK) of a seeded Gaussian,
    columns signed so that diag(R) > 0."""
    g = _rng(seed).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]


def log_spaced(n: int, hi: float, lo: float) -> np.ndarray:
    """n values log-spaced from hi down to lo (inclusive)."""
    if n == 1:
        return np.array([hi], dtype=np.float64)
    return np.logspace(np.log10(hi), np.log10(lo), n)


def _spectral(m: int, n: int, sigma: np.ndarray, seed: int, dtype, rows: int | None = None) -> np.ndarray:
    rng = _rng(seed)
    v = random_orthogonal(n, seed + 7919)
    mix = (sigma[:, None] * v.T)  # diag(sigma) V^T
    mm = m if rows is None else min(m, rows)
    out = np.empty((mm, n), dtype=dtype)
    scale = 1.0 / np.sqrt(m)
    for r0 in range(0, mm, _ROW_CHUNK):
        r1 = min(mm, r0 + _ROW_CHUNK)
        g = rng.standard_normal((r1 - r0, n)) * scale
        out[r0:r1] = g @ mix
    return out


def conditioned(m: int, n: int, kappa: float, seed: int, dtype=np.float64, rows: int | None = None) -> np.ndarray:
    """A = G diag(sigma) V^T, G ~ N(0, 1/m), sigma log-spaced 1 .. 1/kappa."""
    return _spectral(m, n, log_spaced(n, 1.0, 1.0 / kappa), seed, dtype, rows)


def power_spectrum(m: int, n: int, seed: int, dtype=np.float64, rows: int | None = None) -> np.ndarray:
    """A = G diag(j^-2) V^T, j = 1..n, G ~ N(0, 1/m)."""
    sigma = 1.0 / np.arange(1, n + 1, dtype=np.float64) ** 2
    return _spectral(m, n, sigma, seed, dtype, rows)


def column_scaled(m: int, n: int, lo: float, seed: int, dtype=np.float64) -> np.ndarray:
    """i.i.d. N(0, 1) times column factors log-spaced over [1, lo]."""
    c = log_spaced(n, 1.0, lo)
    rng = _rng(seed)
    out = np.empty((m, n), dtype=dtype)
    for r0 in range(0, m, _ROW_CHUNK):
        r1 = min(m, r0 + _ROW_CHUNK)
        out[r0:r1] = rng.standard_normal((r1 - r0, n)) * c[None, :]
    return out


def sigma_conditioned(n: int, kappa: float) -> np.ndarray:
    """The generated singular-value profile of ``conditioned`` (descending)."""
    return log_spaced(n, 1.0, 1.0 / kappa)


def sigma_power(n: int) -> np.ndarray:
    """The generated singular-value profile of ``power_spectrum``."""
    return 1.0 / np.arange(1, n + 1, dtype=np.float64) ** 2
