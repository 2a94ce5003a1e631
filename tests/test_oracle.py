"""Pins for the CPU oracle: closed forms, invariants, brute force and library
routines that fix what the oracle must return (CPU only).

Tolerances are the accuracy goals of the paper's Eqs. Tresnorm / Torthogo
(Sec. 2.3) with the constants used throughout this repository:
|lambda - lambda_ref| <= 4 n eps ||T||, ||T z - lambda z|| <= 20 n eps ||T||,
max |Z^T Z - I| <= 20 n eps.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1205_2107_gb300 import inputs

EPS = 2.0 ** -53


def spectral_norm(W):
    return float(np.max(np.abs(W)))


def residual(d, e, W, Z):
    T = oracle.tridiag_dense(d, e)
    R = T @ Z - Z * W[None, :]
    return float(np.max(np.linalg.norm(R, axis=0)))


def orthogonality(Z):
    k = Z.shape[1]
    return float(np.max(np.abs(Z.T @ Z - np.eye(k))))


def check_pairs(d, e, W, Z, Wref=None, ref_err=0.0):
    """ref_err: rounding error of evaluating the reference values themselves."""
    n = len(d)
    tn = spectral_norm(oracle.eigvalsh_tridiagonal(d, e))
    if Wref is not None:
        assert np.max(np.abs(W - Wref)) <= 4 * n * EPS * tn + ref_err
    assert residual(d, e, W, Z) <= 20 * n * EPS * tn
    assert orthogonality(Z) <= 20 * n * EPS


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 300, 1000])
@pytest.mark.parametrize("a,b", [(2.0, -1.0), (2.0, 1.0), (-0.5, 3.0)])
def test_toeplitz_closed_form(n, a, b):
    d, e = inputs.toeplitz(n, a, b)
    W, Z = oracle.eigh_tridiagonal(d, e)
    ref = inputs.toeplitz_eigenvalues(n, a, b)
    # a + 2b cos(x) is itself evaluated with a few ulps of |a| + 2|b|
    check_pairs(d, e, W, Z, ref, ref_err=4 * EPS * (abs(a) + 2 * abs(b)))
    # eigenvectors: z_k(j) proportional to sin(j k pi/(n+1)) (times (-1)^j
    # when b > 0); ascending order maps to k = 1..n when b < 0
    if n >= 2 and b < 0:
        j = np.arange(1, n + 1)
        for k in [1, n // 2, n]:
            v = np.sin(j * k * np.pi / (n + 1))
            v /= np.linalg.norm(v)
            assert abs(abs(v @ Z[:, k - 1]) - 1.0) <= 1e-9


@pytest.mark.parametrize("n", [1, 2, 5, 6, 51, 200])
def test_clement_integer_spectrum(n):
    d, e = inputs.clement(n)
    W, Z = oracle.eigh_tridiagonal(d, e)
    check_pairs(d, e, W, Z, inputs.clement_eigenvalues(n))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_trace_and_frobenius(seed):
    d, e = inputs.uniform(400, seed)
    W = oracle.eigvalsh_tridiagonal(d, e)
    n = len(d)
    tn = spectral_norm(W)
    assert abs(W.sum() - d.sum()) <= n * n * EPS * tn
    frob = (d ** 2).sum() + 2 * (e ** 2).sum()
    assert abs((W ** 2).sum() - frob) <= 4 * n * n * EPS * tn * tn


def test_wilkinson_trace_exact():
    d, e = inputs.wilkinson_plus(2001)
    W = oracle.eigvalsh_tridiagonal(d, e)
    assert abs(W.sum() - 1001000.0) <= 2001 * 2001 * EPS * 1001
    # the top eigenvalues come in pairs that agree to far below eps
    assert abs(W[-1] - W[-2]) <= 8 * EPS * W[-1]


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (17, 3), (64, 4)])
def test_jacobi_against_library(n, seed):
    d, e = inputs.uniform(n, seed)
    W, V = oracle.jacobi(d, e)
    T = oracle.tridiag_dense(d, e)
    ref = np.linalg.eigvalsh(T)
    tn = max(spectral_norm(ref), 1e-300)
    assert np.max(np.abs(W - ref)) <= 4 * n * EPS * tn
    assert orthogonality(V) <= 20 * n * EPS
    assert np.max(np.linalg.norm(T @ V - V * W, axis=0)) <= 20 * n * EPS * tn


@pytest.mark.parametrize("n,seed", [(2, 5), (9, 6), (33, 7), (64, 8)])
def test_bisection_inverse_iteration_vs_jacobi(n, seed):
    d, e = inputs.normal(n, seed)
    W, Z = oracle.eigh_tridiagonal(d, e)
    Wj, Vj = oracle.jacobi(d, e)
    check_pairs(d, e, W, Z, Wj)
    # same invariant subspaces: singletons column by column (up to sign)
    tn = spectral_norm(Wj)
    for k in range(n):
        gap = min([abs(Wj[k] - Wj[j]) for j in range(n) if j != k] + [np.inf])
        if gap > 1e-6 * tn:
            assert abs(abs(Z[:, k] @ Vj[:, k]) - 1.0) <= 1e-8


def test_scipy_lapack_cross_check():
    d, e = inputs.uniform(300, 1205)
    W, Z = oracle.eigh_tridiagonal(d, e)
    Wl = scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True)
    tn = spectral_norm(Wl)
    assert np.max(np.abs(W - Wl)) <= 4 * 300 * EPS * tn


@pytest.mark.parametrize("maker", [lambda: inputs.uniform(500, 11), lambda: inputs.wilkinson_plus(301),
                                   lambda: inputs.glued_wilkinson(6)])
def test_sturm_index_bracket(maker):
    d, e = maker()
    n = len(d)
    W = oracle.eigvalsh_tridiagonal(d, e)
    delta = 4 * n * EPS * spectral_norm(W)
    for j in [1, 2, n // 3, n // 2, n - 1, n]:
        assert oracle.sturm_count(d, e, W[j - 1] - delta) <= j - 1 < oracle.sturm_count(d, e, W[j - 1] + delta)


@pytest.mark.parametrize("il,iu", [(1, 1), (3, 17), (100, 250), (250, 250), (1, 250)])
def test_subset_matches_full(il, iu):
    d, e = inputs.uniform(250, 99)
    Wa = oracle.eigvalsh_tridiagonal(d, e)
    W, Z = oracle.eigh_tridiagonal(d, e, il, iu)
    assert np.array_equal(W, Wa[il - 1:iu])
    assert Z.shape == (250, iu - il + 1)
    tn = spectral_norm(Wa)
    assert residual(d, e, W, Z) <= 20 * 250 * EPS * tn
    assert orthogonality(Z) <= 20 * 250 * EPS
    assert oracle.kth_eigenvalue(d, e, il) == W[0]


def test_split_blocks_are_independent():
    d, e = inputs.uniform(120, 3)
    e[[9, 40, 41, 99]] = 0.0
    e[70] = 1e-300  # below eps * G(T): also splits
    es, starts = oracle.split(d, e)
    assert list(starts) == [0, 10, 41, 42, 71, 100, 120]
    assert es[70] == 0.0
    W, Z = oracle.eigh_tridiagonal(d, e)
    ref = np.sort(np.concatenate([np.linalg.eigvalsh(oracle.tridiag_dense(d[s:t], es[s:t - 1]))
                                  for s, t in zip(starts[:-1], starts[1:])]))
    check_pairs(d, es, W, Z, ref)
    # every column lives in exactly one block
    for k in range(Z.shape[1]):
        nz = np.nonzero(Z[:, k])[0]
        blk = np.searchsorted(starts, nz, side="right")
        assert len(set(blk.tolist())) == 1


def test_split_subset_with_ties_across_blocks():
    # two identical blocks: every eigenvalue appears twice
    d1, e1 = inputs.uniform(30, 4)
    d = np.concatenate([d1, d1])
    e = np.concatenate([e1, [0.0], e1])
    Wa, Za = oracle.eigh_tridiagonal(d, e)
    assert np.all(np.diff(Wa) >= 0)
    W, Z = oracle.eigh_tridiagonal(d, e, 7, 20)
    assert np.array_equal(W, Wa[6:20])
    check_pairs(d, e, W, Z)


def test_cluster_members_separated_by_another_block():
    """A cluster of one block stays one cluster (re-orthogonalised together)
    when an eigenvalue of another block lies between its members in
    ascending order: the pair of W21+ near 9.2107 (gap 5.6e-11) with a 1x1
    block at its midpoint.  Inverse iteration alone leaves that pair about
    1e-7 from orthogonal."""
    d0, e0 = inputs.wilkinson_plus(21)
    W0 = np.linalg.eigvalsh(oracle.tridiag_dense(d0, e0))
    lo, hi = W0[17], W0[18]
    assert 0 < hi - lo < 1e-10
    d = np.append(d0, lo + (hi - lo) / 2)
    e = np.append(e0, 0.0)
    W, Z = oracle.eigh_tridiagonal(d, e)
    assert W[17] < W[18] < W[19] and W[18] == d[-1]
    check_pairs(d, e, W, Z, np.sort(np.append(W0, d[-1])))


@pytest.mark.parametrize("k", [-1000, -600, 600, 900])
def test_power_of_two_scaling_is_exact(k):
    """Eigenpairs of 2^k T are 2^k times those of T bit for bit (the oracle
    normalises ||T|| by an exact power of two), also where e_i^2 alone would
    underflow or overflow."""
    d, e = inputs.wilkinson_plus(21)
    W, Z = oracle.eigh_tridiagonal(d, e)
    Ws, Zs = oracle.eigh_tridiagonal(np.ldexp(d, k), np.ldexp(e, k))
    assert np.array_equal(Ws, np.ldexp(W, k)) and np.array_equal(Zs, Z)
    assert oracle.sturm_count(np.ldexp(d, k), np.ldexp(e, k), np.ldexp(W[10], k) * (1 + 1e-12)) == 11


def test_tiny_block_beside_a_normal_one():
    """A 1x1 block of magnitude 1e-239 next to a block of norm 1: its
    inverse iteration runs on the block scaled to norm 1, so the vector is a
    finite unit vector."""
    d = np.array([1.0, 2.23341364e-239, 0.0])
    e = np.array([0.0, 0.0])
    W, Z = oracle.eigh_tridiagonal(d, e)
    assert W.tolist() == [0.0, 2.23341364e-239, 1.0]
    assert np.array_equal(np.abs(Z), np.eye(3)[:, [2, 1, 0]])


@pytest.mark.parametrize("maker", [lambda: inputs.wilkinson_plus(201), lambda: inputs.glued_wilkinson(20),
                                   lambda: inputs.uniform(800, 1205), lambda: inputs.toeplitz(800)])
def test_clustered_vectors(maker):
    d, e = maker()
    W, Z = oracle.eigh_tridiagonal(d, e)
    check_pairs(d, e, W, Z, np.linalg.eigvalsh(oracle.tridiag_dense(d, e)))


def test_n0_and_n1():
    W, Z = oracle.eigh_tridiagonal(np.array([3.5]), np.array([]))
    assert W.tolist() == [3.5] and abs(Z[0, 0]) == 1.0
    W = oracle.eigvalsh_tridiagonal(np.zeros(0), np.zeros(0))
    assert W.shape == (0,)


def test_cluster_vectors_sampled():
    d, e = inputs.wilkinson_plus(401)
    W, Z = oracle.eigh_tridiagonal(d, e)
    V = oracle.cluster_vectors(d, e, W[-2:])
    # the top pair: same 2-D subspace
    P = Z[:, -2:].T @ V
    s = np.linalg.svd(P, compute_uv=False)
    assert np.min(s) >= 1 - 1e-10


# -------------------------------------------------------------------------
# gradient oracle: pinned by central finite differences through the solve


def _loss(d, e, w, C):
    W, Z = oracle.eigh_tridiagonal(d, e)
    return float(w @ W + np.sum(np.einsum("ji,ji->i", C, Z) ** 2))


def _fd_grad(d, e, w, C, h=1e-6):
    gd = np.zeros_like(d)
    ge = np.zeros_like(e)
    for j in range(len(d)):
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        gd[j] = (_loss(dp, e, w, C) - _loss(dm, e, w, C)) / (2 * h)
    for j in range(len(e)):
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        ge[j] = (_loss(d, ep, w, C) - _loss(d, em, w, C)) / (2 * h)
    return gd, ge


def _analytic(d, e, w, C, adjoint=oracle.adjoint):
    W, Z = oracle.eigh_tridiagonal(d, e)
    proj = np.einsum("ji,ji->i", C, Z)
    Zbar = 2.0 * C * proj[None, :]
    tau = 64 * EPS * spectral_norm(W)
    return adjoint(W, Z, w, Zbar, tau)


@pytest.mark.parametrize("n,seed", [(6, 1), (12, 2)])
def test_adjoint_against_finite_differences(n, seed):
    rng = np.random.default_rng(seed)
    d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    w, C = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, ge = _analytic(d, e, w, C)
    fd, fe = _fd_grad(d, e, w, C)
    scale = max(np.max(np.abs(fd)), np.max(np.abs(fe)))
    assert np.max(np.abs(gd - fd)) <= 1e-6 * scale
    assert np.max(np.abs(ge - fe)) <= 1e-6 * scale


def test_adjoint_eigenvalue_part_is_trace_derivative():
    # d(sum lambda)/dd_j = 1 and d(sum lambda)/de_j = 0 (trace invariant)
    d, e = inputs.normal(40, 3)
    W, Z = oracle.eigh_tridiagonal(d, e)
    gd, ge = oracle.adjoint(W, Z, np.ones(40), None)
    assert np.max(np.abs(gd - 1.0)) <= 1e-12
    assert np.max(np.abs(ge)) <= 1e-12


def test_fd_pin_catches_planted_mistakes():
    """The finite-difference pin rejects plausible slips in the gradient."""
    rng = np.random.default_rng(5)
    n = 8
    d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    w, C = rng.standard_normal(n), rng.standard_normal((n, n))
    fd, fe = _fd_grad(d, e, w, C)
    scale = max(np.max(np.abs(fd)), np.max(np.abs(fe)))

    def wrong_sign(W, Z, Wbar, Zbar, tau):  # F_ij = 1/(lambda_i - lambda_j)
        gd0, ge0 = oracle.adjoint(W, Z, Wbar, None, tau)
        gd1, ge1 = oracle.adjoint(W, Z, None, Zbar, tau)
        return gd0 - gd1, ge0 - ge1

    def dropped_offdiag(W, Z, Wbar, Zbar, tau):  # forgets M_{j+1,j}
        gd, ge = oracle.adjoint(W, Z, Wbar, Zbar, tau)
        gap = W[None, :] - W[:, None]
        F = np.where(np.abs(gap) > tau, 1.0 / np.where(gap == 0, 1, gap), 0.0)
        np.fill_diagonal(F, 0.0)
        M = Z @ (F * (Z.T @ Zbar)) @ Z.T
        return gd, ge - np.diag(M, -1)

    for bad in (wrong_sign, dropped_offdiag):
        gd, ge = _analytic(d, e, w, C, adjoint=bad)
        err = max(np.max(np.abs(gd - fd)), np.max(np.abs(ge - fe)))
        assert err > 1e-3 * scale
