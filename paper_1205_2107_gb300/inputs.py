"""Seeded synthetic inputs for the tridiagonal eigensolver (shared by tests,
benchmark and oracle checks).

This module holds input recipes only -- none of the eigensolver's arithmetic.
Every generator returns NumPy float64 arrays (d of length n, e of length n-1)
and is deterministic for a given seed (NumPy PCG64 through ``default_rng``).

The matrix families follow the paper's test matrices (Sec. 2.3, "1-2-1" and
"Wilkinson" matrices; Sec. 4.1 fixes the tridiagonal to 1-2-1) plus the
workload shapes used to measure this library:
  * ``uniform``          d, e iid U(lo, hi)
  * ``toeplitz``         d = a, e = b (closed-form spectrum)
  * ``wilkinson_plus``   d_i = |i - (n+1)/2|, e = 1
  * ``glued_wilkinson``  copies of W21+ joined by a small glue value
  * ``clement``          d = 0, e_i = sqrt(i (n - i)) (integer spectrum)
  * ``normal``           d, e iid N(0, 1)
"""
from __future__ import annotations

import numpy as np


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0,
            elo: float | None = None, ehi: float | None = None):
    rng = np.random.default_rng(seed)
    d = rng.uniform(lo, hi, n)
    e = rng.uniform(lo if elo is None else elo, hi if ehi is None else ehi, max(n - 1, 0))
    return d, e


def normal(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))


def toeplitz(n: int, a: float = 2.0, b: float = -1.0):
    return np.full(n, float(a)), np.full(max(n - 1, 0), float(b))


def toeplitz_eigenvalues(n: int, a: float = 2.0, b: float = -1.0) -> np.ndarray:
    """Closed form lambda_k = a + 2 b cos(k pi / (n+1)), returned ascending."""
    k = np.arange(1, n + 1)
    return np.sort(a + 2.0 * b * np.cos(k * np.pi / (n + 1)))


def wilkinson_plus(n: int):
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.abs(i - (n + 1) / 2.0), np.ones(max(n - 1, 0))


def glued_wilkinson(copies: int, m: int = 21, glue: float = 1e-10):
    dw, ew = wilkinson_plus(m)
    d = np.tile(dw, copies)
    e = np.ones(copies * m - 1)
    for c in range(1, copies):
        e[c * m - 1] = glue
    return d, e


def clement(n: int):
    i = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(i * (n - i))


def clement_eigenvalues(n: int) -> np.ndarray:
    """-(n-1), -(n-3), ..., (n-3), (n-1)."""
    return np.arange(-(n - 1), n, 2, dtype=np.float64)


def batch_sizes(count: int = 4096, seed: int = 2107, nmin: int = 32, nmax: int = 2048) -> np.ndarray:
    """Sizes log-uniform in [nmin, nmax]: clip(round(exp(U(ln nmin, ln nmax))))."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count)))
    return np.clip(n, nmin, nmax).astype(np.int64)


def batched_uniform(sizes, seed: int = 2107):
    """Packed batch: d (sum n), e (sum n, last entry of each problem unused),
    offsets (batch+1)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    rng = np.random.default_rng(seed + 1)
    d = rng.uniform(-1.0, 1.0, int(off[-1]))
    e = rng.uniform(-1.0, 1.0, int(off[-1]))
    e[off[1:] - 1] = 0.0
    return d, e, off


def adjoint_case(batch: int = 256, n: int = 512, seed: int = 1206):
    """Batch of N(0,1) tridiagonals with loss weights w (batch, n) and
    C (batch, n, n) for loss = sum_i w_i lambda_i + sum_i (c_i^T z_i)^2."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((batch, n))
    e = rng.standard_normal((batch, n))
    e[:, -1] = 0.0
    w = rng.standard_normal((batch, n))
    C = rng.standard_normal((batch, n, n))
    return d, e, w, C


def large_uniform(n: int = 50000, seed: int = 50000):
    """d ~ U(0, 1), e ~ U(0, 1e-2)."""
    return uniform(n, seed, 0.0, 1.0, 0.0, 1e-2)
