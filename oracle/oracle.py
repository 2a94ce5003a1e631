"""CPU oracle for the symmetric tridiagonal eigenproblem (test infrastructure).

This module is TEST INFRASTRUCTURE: only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  The GPU library never calls
it and shares no code with it.

It wraps ``oracle.c`` (plain C, FP64; bisection with Sturm counts on T plus
classical inverse iteration with Gram-Schmidt inside clusters, and a dense
Jacobi solver for small n) through ctypes, and adds the dense reference
gradient of the eigen-decomposition in NumPy.

Paper passages (Petschow, Peise, Bientinesi, arXiv:1205.2107):
  * problem statement -- all or a subset of eigenpairs of a real symmetric
    tridiagonal T (Sec. 1.1; Sec. 2.3; Sec. 5);
  * accuracy goals -- residual O(n eps ||T||) and orthogonality O(n eps)
    (Sec. 2.3, Eqs. Tresnorm and Torthogo);
  * splitting threshold eps*||T|| (Sec. 3.1.1, footnote);
  * bisection and inverse iteration (Sec. 2.1 "BI"; Sec. 3.1, the inverse
    iteration equation), orfac = 1e-3 (Sec. 2.1 footnote), relative to each
    split block's norm;
  * every call first scales T by the power of two that brings G(T) into
    [1, 2) and scales the eigenvalues back (exact; see _scale_exponent).

The gradient (``adjoint``) is not in the paper: it is the standard first-order
perturbation of a symmetric eigen-decomposition, written out densely:
  dbar_j = sum_i wbar_i z_i(j)^2 + M_jj,
  ebar_j = 2 sum_i wbar_i z_i(j) z_i(j+1) + M_{j,j+1} + M_{j+1,j},
  M = Z (F o (Z^T Zbar)) Z^T,  F_ij = 1/(lambda_j - lambda_i) when
  |lambda_j - lambda_i| > tau, else 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, no fp contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_eigh.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_int64]
            lib.oracle_eigh.restype = ctypes.c_int
            lib.oracle_kth_eigenvalue.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int]
            lib.oracle_kth_eigenvalue.restype = ctypes.c_double
            lib.oracle_sturm_count.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
            lib.oracle_sturm_count.restype = ctypes.c_int
            lib.oracle_split.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip]
            lib.oracle_split.restype = ctypes.c_int
            lib.oracle_gershgorin_norm.argtypes = [ctypes.c_int, _dp, _dp]
            lib.oracle_gershgorin_norm.restype = ctypes.c_double
            lib.oracle_jacobi.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
            lib.oracle_jacobi.restype = ctypes.c_int
            lib.oracle_cluster_vectors.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp]
            lib.oracle_cluster_vectors.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _offdiag(d: np.ndarray, e) -> np.ndarray:
    n = d.shape[0]
    e = _f64(e)
    if e.shape[0] < max(n - 1, 0):
        raise ValueError("e needs n-1 entries")
    buf = np.zeros(max(n - 1, 1), dtype=np.float64)
    buf[: max(n - 1, 0)] = e[: max(n - 1, 0)]
    return buf


def _scale_exponent(d: np.ndarray, e: np.ndarray) -> int:
    """k such that 2^k G(T) lies in [1, 2) (0 when G(T) is 0 or not finite).

    Reading of the norm and scaling step (Sec. 3.1.1 takes the norm of T; the
    paper is silent on scaling): the oracle solves 2^k T and divides the
    eigenvalues by 2^k.  Scaling by a power of two is exact, leaves the
    eigenvectors unchanged, and keeps every e_i^2 of the Sturm recurrence in
    the normal range, which fails for T with entries below about 1e-154 (the
    squares underflow and the counts go wrong) or above about 1e154.
    """
    g = float(_load().oracle_gershgorin_norm(d.shape[0], _ptr(d), _ptr(e)))
    if g == 0.0 or not np.isfinite(g):
        return 0
    return 1 - int(np.frexp(g)[1])


def _normalised(d, e):
    """(2^k d, 2^k e padded to n-1 (at least 1), k) for the k of _scale_exponent."""
    d = _f64(d)
    eb = _offdiag(d, e)
    k = _scale_exponent(d, eb)
    if k == 0:
        return d, eb, 0
    return np.ldexp(d, k), np.ldexp(eb, k), k


def num_threads(nthreads: int = 0) -> int:
    """Threads the oracle uses for ``nthreads`` (0 = all online cores)."""
    return int(_load().oracle_num_threads(int(nthreads)))


def gershgorin_norm(d, e) -> float:
    """G(T) = max_i |d_i| + |e_{i-1}| + |e_i|, the norm the split threshold uses."""
    d = _f64(d)
    return float(_load().oracle_gershgorin_norm(d.shape[0], _ptr(d), _ptr(_offdiag(d, e))))


def split(d, e):
    """Split T where |e_i| <= eps*G(T).  Returns (split e, block starts incl. n)."""
    d = _f64(d)
    n = d.shape[0]
    eb = _offdiag(d, e)
    es = np.zeros_like(eb)
    starts = np.zeros(n + 1, dtype=np.int32)
    nb = _load().oracle_split(n, _ptr(d), _ptr(eb), _ptr(es),
                              starts.ctypes.data_as(_ip))
    return es[: max(n - 1, 0)], starts[: nb + 1].copy()


def sturm_count(d, e, x: float) -> int:
    """Number of eigenvalues of the split T strictly below x (Sturm count on T)."""
    d, eb, k = _normalised(d, e)
    return int(_load().oracle_sturm_count(d.shape[0], _ptr(d), _ptr(eb), float(np.ldexp(float(x), k))))


def kth_eigenvalue(d, e, k: int) -> float:
    """lambda_k (1-based, ascending) of the split T by bisection to full accuracy."""
    d, eb, s = _normalised(d, e)
    n = d.shape[0]
    if not 1 <= k <= n:
        raise ValueError("k out of range")
    return float(np.ldexp(_load().oracle_kth_eigenvalue(n, _ptr(d), _ptr(eb), int(k)), -s))


def eigvalsh_tridiagonal(d, e, il: int | None = None, iu: int | None = None,
                         nthreads: int = 0) -> np.ndarray:
    """Eigenvalues il..iu (1-based inclusive; default all), ascending."""
    d, eb, s = _normalised(d, e)
    n = d.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    k = max(iu - il + 1, 0)
    W = np.zeros(max(k, 1), dtype=np.float64)
    rc = _load().oracle_eigh(n, _ptr(d), _ptr(eb), il, iu, 0.0, int(nthreads), _ptr(W), None, 0)
    if rc != 0:
        raise ValueError("bad arguments")
    return np.ldexp(W[:k], -s)


def eigh_tridiagonal(d, e, il: int | None = None, iu: int | None = None,
                     orfac: float = 1e-3, nthreads: int = 0):
    """Eigenpairs il..iu: (W[k], Z[n, k]) with orthonormal columns of Z."""
    d, eb, s = _normalised(d, e)
    n = d.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    k = max(iu - il + 1, 0)
    W = np.zeros(max(k, 1), dtype=np.float64)
    Zf = np.zeros((max(k, 1), max(n, 1)), dtype=np.float64)  # row j = column j of Z
    rc = _load().oracle_eigh(n, _ptr(d), _ptr(eb), il, iu, float(orfac),
                             int(nthreads), _ptr(W), _ptr(Zf), max(n, 1))
    if rc != 0:
        raise ValueError("bad arguments")
    return np.ldexp(W[:k], -s), Zf[:k, :n].T.copy()


def cluster_vectors(d, e, mus) -> np.ndarray:
    """Inverse-iteration vectors (with Gram-Schmidt) for the given close values."""
    d, eb, s = _normalised(d, e)
    n = d.shape[0]
    mus = np.ldexp(_f64(mus), s)
    c = mus.shape[0]
    Zf = np.zeros((c, n), dtype=np.float64)
    rc = _load().oracle_cluster_vectors(n, _ptr(d), _ptr(eb), c, _ptr(mus), _ptr(Zf))
    if rc != 0:
        raise ValueError("bad arguments")
    return Zf.T.copy()


def jacobi(d, e):
    """Dense cyclic Jacobi on the (unsplit) T, n <= 512: (W ascending, V)."""
    d, eb, s = _normalised(d, e)
    n = d.shape[0]
    W = np.zeros(n, dtype=np.float64)
    V = np.zeros((n, n), dtype=np.float64)  # filled column-major
    rc = _load().oracle_jacobi(n, _ptr(d), _ptr(eb), _ptr(W), _ptr(V))
    if rc != 0:
        raise ValueError("jacobi: n must be in 1..512")
    return np.ldexp(W, -s), V.T.copy()


def tridiag_dense(d, e) -> np.ndarray:
    """The dense symmetric matrix with diagonal d and off-diagonal e."""
    d = _f64(d)
    n = d.shape[0]
    T = np.diag(d)
    if n > 1:
        e = _f64(e)[: n - 1]
        T += np.diag(e, 1) + np.diag(e, -1)
    return T


def adjoint(W, Z, Wbar=None, Zbar=None, tau: float = 0.0):
    """Reference gradient of a loss L(W, Z) w.r.t. (d, e) of T = Z diag(W) Z^T.

    Dense formula (plain NumPy): dbar_j = sum_i Wbar_i Z[j,i]^2 + M[j,j],
    ebar_j = 2 sum_i Wbar_i Z[j,i] Z[j+1,i] + M[j,j+1] + M[j+1,j] with
    M = Z (F o (Z^T Zbar)) Z^T and F[i,j] = 1/(W[j]-W[i]) if |W[j]-W[i]| > tau
    else 0 (so F[i,i] = 0).
    """
    W = _f64(W)
    Z = _f64(Z)
    n = Z.shape[0]
    dbar = np.zeros(n)
    ebar = np.zeros(max(n - 1, 0))
    if Wbar is not None:
        Wbar = _f64(Wbar)
        dbar += (Z * Z) @ Wbar
        if n > 1:
            ebar += 2.0 * (Z[:-1, :] * Z[1:, :]) @ Wbar
    if Zbar is not None:
        Zbar = _f64(Zbar)
        gap = W[None, :] - W[:, None]          # gap[i, j] = W[j] - W[i]
        with np.errstate(divide="ignore"):
            F = np.where(np.abs(gap) > tau, 1.0 / np.where(gap == 0, 1.0, gap), 0.0)
        np.fill_diagonal(F, 0.0)
        G = F * (Z.T @ Zbar)
        M = Z @ G @ Z.T
        dbar += np.diag(M)
        if n > 1:
            ebar += np.diag(M, 1) + np.diag(M, -1)
    return dbar, ebar
