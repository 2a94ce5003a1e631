"""CPU oracle for the dense stages around the tridiagonal eigensolver (test
infrastructure: only the test-suite and the benchmark's CPU legs use it; the
GPU library shares no code with it).

The paper's dense solvers reduce the problem to the tridiagonal one and back
(Sec. 1.2, the six stages of the generalized solver):
  1. Cholesky factorization B = L L^T;
  2. reduction to the standard problem, C = L^-1 A L^-T;
  3. reduction to tridiagonal form, C = Q T Q^T;
  4. the tridiagonal eigenproblem T Z = Z Lambda (oracle.eigh_tridiagonal);
  5. backtransformation Y = Q Z (eigenvectors of C);
  6. backtransformation X = L^-T Y (eigenvectors of the pair A, B).
Stages 3-5 alone solve the standard problem A Y = Y Lambda.

Each function is the textbook algorithm in plain NumPy, FP64, one column (or
row) at a time, with NumPy's vector and matrix products as its only library
steps; nothing is blocked or reordered:
  * tridiagonal_reduction -- Householder reflectors H_k = I - tau_k v_k v_k^T,
    k = 0 .. n-3, each annihilating column k below its subdiagonal, applied
    from both sides as the rank-2 update A <- A - v w^T - w v^T with
    p = tau A v, w = p - (tau/2)(p^T v) v;
  * apply_q -- Q Z = H_0 H_1 ... H_{n-3} Z, the reflectors applied from the
    last to the first;
  * cholesky -- the column-by-column (left-looking) factorization;
  * forward_substitution / back_substitution -- triangular solves by rows;
  * the drivers eigh_dense and eigh_generalized.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _tri


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, copy=True)


def householder_vector(x: np.ndarray):
    """(v, tau, beta) with (I - tau v v^T) x = beta e_1, v[0] = 1.

    beta = -sign(x_0) ||x|| (the sign that avoids cancellation in x_0 - beta);
    tau = 0 and beta = x_0 when x is already a multiple of e_1."""
    x = np.asarray(x, dtype=np.float64)
    m = x.shape[0]
    v = np.zeros(m)
    v[0] = 1.0
    if m == 0:
        return v, 0.0, 0.0
    sigma = float(x[1:] @ x[1:]) if m > 1 else 0.0
    alpha = float(x[0])
    if sigma == 0.0:
        return v, 0.0, alpha
    norm = np.sqrt(alpha * alpha + sigma)
    beta = -norm if alpha >= 0.0 else norm
    v[1:] = x[1:] / (alpha - beta)
    tau = (beta - alpha) / beta
    return v, tau, beta


def tridiagonal_reduction(A):
    """Householder reduction of a symmetric A (only its lower triangle is
    read) to T = Q^T A Q.  Returns (d, e, V, tau): T's diagonal and
    subdiagonal, and the reflectors: column k of V holds v_k in rows k+1..n-1
    (V[k+1, k] = 1), tau[k] its factor; Q = H_0 ... H_{n-3}."""
    A = _f64(A)
    n = A.shape[0]
    A = np.tril(A) + np.tril(A, -1).T  # symmetric from the lower triangle
    V = np.zeros((n, max(n - 2, 0)))
    tau = np.zeros(max(n - 2, 0))
    e = np.zeros(max(n - 1, 0))
    for k in range(n - 2):
        v, t, beta = householder_vector(A[k + 1:, k])
        V[k + 1:, k] = v
        tau[k] = t
        e[k] = beta
        # two-sided update of the trailing block A[k+1:, k+1:]
        S = A[k + 1:, k + 1:]
        p = t * (S @ v)
        w = p - (0.5 * t * float(p @ v)) * v
        S -= np.outer(v, w) + np.outer(w, v)
        A[k + 1:, k + 1:] = S
        A[k + 1:, k] = 0.0
        A[k, k + 1:] = 0.0
        A[k + 1, k] = A[k, k + 1] = beta
    if n >= 2:
        e[n - 2] = A[n - 1, n - 2]
    d = np.diag(A).copy()
    return d, e, V, tau


def apply_q(V, tau, Z):
    """Q Z for Q = H_0 H_1 ... H_{n-3} (H_k = I - tau_k v_k v_k^T): the
    reflectors from the last to the first."""
    Y = _f64(Z)
    for k in range(V.shape[1] - 1, -1, -1):
        v = V[k + 1:, k]
        Y[k + 1:, :] -= tau[k] * np.outer(v, v @ Y[k + 1:, :])
    return Y


def form_q(V, tau, n: int):
    """The orthogonal Q itself (Q applied to the identity)."""
    return apply_q(V, tau, np.eye(n))


def eigh_dense(A, il: int | None = None, iu: int | None = None):
    """Eigenpairs il..iu (1-based, inclusive) of the symmetric A: stage 3
    (reduction), stage 4 (oracle.eigh_tridiagonal), stage 5 (Y = Q Z)."""
    A = _f64(A)
    n = A.shape[0]
    d, e, V, tau = tridiagonal_reduction(A)
    W, Z = _tri.eigh_tridiagonal(d, e, il, iu)
    return W, apply_q(V, tau, Z)


def cholesky(B):
    """Lower-triangular L with L L^T = B (B symmetric positive definite; its
    lower triangle is read), column by column:
    L[j, j] = sqrt(B[j, j] - sum_k L[j, k]^2),
    L[i, j] = (B[i, j] - sum_k L[i, k] L[j, k]) / L[j, j]  (i > j)."""
    B = _f64(B)
    n = B.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        s = B[j, j] - float(L[j, :j] @ L[j, :j])
        if not s > 0.0:
            raise ValueError("matrix is not positive definite")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (B[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_substitution(L, Bm):
    """X with L X = Bm (L lower triangular), row by row."""
    L = np.asarray(L, dtype=np.float64)
    X = _f64(Bm)
    for i in range(L.shape[0]):
        X[i] = (X[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def back_substitution_transposed(L, Bm):
    """X with L^T X = Bm (L lower triangular), row by row from the last."""
    L = np.asarray(L, dtype=np.float64)
    X = _f64(Bm)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X


def reduce_generalized(A, L):
    """C = L^-1 A L^-T (stage 2): two triangular solves, the second on the
    transpose of the first's result, symmetrised from its lower triangle."""
    A = _f64(A)
    A = np.tril(A) + np.tril(A, -1).T
    M = forward_substitution(L, A)          # L^-1 A
    C = forward_substitution(L, M.T)        # L^-1 (L^-1 A)^T = L^-1 A L^-T
    return np.tril(C) + np.tril(C, -1).T


def eigh_generalized(A, B, il: int | None = None, iu: int | None = None):
    """Eigenpairs il..iu of A x = lambda B x (A symmetric, B symmetric
    positive definite), the six stages: L = cholesky(B),
    C = L^-1 A L^-T, (W, Y) = eigh_dense(C), X = L^-T Y."""
    L = cholesky(B)
    C = reduce_generalized(A, L)
    W, Y = eigh_dense(C, il, iu)
    return W, back_substitution_transposed(L, Y)
