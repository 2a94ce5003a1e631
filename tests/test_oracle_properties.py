"""Property-based pins for the CPU oracle (CPU only; needs hypothesis).

Random small tridiagonals drawn with the structures that break eigensolvers:
exact zeros in e (splits), repeated diagonal entries (ties), entries spread
over many binades, and whole-matrix scalings far from 1.  For each, the
oracle's eigenvalues must agree with LAPACK's (scipy's stebz/stemr route)
within 4 n eps ||T||, its Sturm counts must bracket them, its vectors must
meet the residual goal of Sec. 2.3 (Eq. Tresnorm), and each pair of vectors
the orthogonality that bisection + inverse iteration guarantees (clusters
re-orthogonalised to O(n eps), Eq. Torthogo; other pairs within the
Davis-Kahan bound of their gaps)."""
import numpy as np
import pytest
import scipy.linalg

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings, HealthCheck = hyp.given, hyp.settings, hyp.HealthCheck

EPS = 2.0 ** -53

_entry = st.one_of(
    st.just(0.0),
    st.sampled_from([1.0, -1.0, 0.5, 2.0]),
    st.floats(min_value=-4.0, max_value=4.0, allow_nan=False, allow_infinity=False),
    st.builds(lambda m, k: m * 2.0 ** k, st.floats(0.5, 1.0), st.integers(-30, 30)),
)


@st.composite
def tridiagonals(draw):
    n = draw(st.integers(1, 40))
    d = np.array(draw(st.lists(_entry, min_size=n, max_size=n)), dtype=np.float64)
    e = np.array(draw(st.lists(_entry, min_size=n - 1, max_size=n - 1)), dtype=np.float64)
    scale = 2.0 ** draw(st.sampled_from([0, 0, 0, -500, 500, -1000, 900]))
    return d * scale, e * scale


def _norm(d, e):
    return float(np.max(np.abs(np.linalg.eigvalsh(oracle.tridiag_dense(d, e))))) if len(d) else 0.0


@settings(max_examples=150, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(tridiagonals())
def test_eigenvalues_match_lapack(T):
    d, e = T
    n = len(d)
    W = oracle.eigvalsh_tridiagonal(d, e)
    Wl = scipy.linalg.eigvalsh_tridiagonal(d, e) if n > 1 else d.copy()
    tn = max(float(np.max(np.abs(Wl))), np.finfo(float).tiny)
    assert np.all(np.diff(W) >= 0)
    assert np.max(np.abs(W - Wl)) <= 4 * n * EPS * tn


@settings(max_examples=150, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(tridiagonals(), st.data())
def test_sturm_counts_bracket_each_eigenvalue(T, data):
    d, e = T
    n = len(d)
    W = oracle.eigvalsh_tridiagonal(d, e)
    j = data.draw(st.integers(0, n - 1))
    lam = W[j]
    tn = max(float(np.max(np.abs(W))), np.finfo(float).tiny)
    # the count treats a pivot within pivmin (a few safmin after scaling) of
    # zero as negative, so it is exact only outside that margin
    tol = 8 * n * EPS * tn + 16 * np.finfo(float).tiny
    # #{eigenvalues < x}: at most j below lam - tol, at least j + 1 below lam + tol
    assert oracle.sturm_count(d, e, lam - tol) <= j
    assert oracle.sturm_count(d, e, lam + tol) >= j + 1


def _pair_bounds(d, e, W, Z, res, orfac=1e-3):
    """Bound on |z_i^T z_j| for every pair of the oracle's columns, from the
    mathematics of bisection + inverse iteration on the split T (W, res in
    the units of the scaled T, whose norm is in [1, 2)):
      * columns of different blocks have disjoint supports: exactly 0;
      * members of one cluster (same block, consecutive in the block's order,
        gaps <= orfac ||T_b||) are re-orthogonalised: 20 n eps;
      * members of different clusters C, D of one block: the Davis-Kahan
        sin-theta theorem bounds the angle between span(Z_C) and the exact
        invariant subspace by ||R_C||_F / delta_C (R_C the residuals of C's
        columns, delta_C the distance from C's eigenvalues to the rest of
        the block's spectrum, less the eigenvalue error), so
        |z_i^T z_j| <= ||R_C|| / delta_C + ||R_D|| / delta_D + 20 n eps."""
    n = len(d)
    _, starts = oracle.split(d, e)
    row_block = np.searchsorted(starts, np.arange(n), side="right") - 1
    col_block = row_block[np.argmax(np.abs(Z), axis=0)]
    err = 2 * 4 * n * EPS * 2.0  # twice the eigenvalue tolerance at ||T|| < 2
    B = np.zeros((n, n))
    for b in np.unique(col_block):
        cols = np.flatnonzero(col_block == b)
        cols = cols[np.argsort(W[cols], kind="stable")]
        w = W[cols]
        tb = float(np.max(np.abs(w)))
        cl = np.concatenate([[0], np.cumsum(np.diff(w) > orfac * tb)])  # cluster id per member
        ncl = int(cl[-1]) + 1
        lo = np.array([w[cl == c][0] for c in range(ncl)])
        hi = np.array([w[cl == c][-1] for c in range(ncl)])
        delta = np.full(ncl, np.inf)
        delta[1:] = np.minimum(delta[1:], lo[1:] - hi[:-1])
        delta[:-1] = np.minimum(delta[:-1], lo[1:] - hi[:-1])
        rnorm = np.array([np.linalg.norm(res[cols[cl == c]]) for c in range(ncl)])
        sin_theta = np.where(np.isinf(delta), 0.0, rnorm / np.maximum(delta - err, 1e-300))
        for a, i in enumerate(cols):
            for c, j in enumerate(cols):
                if cl[a] == cl[c]:
                    B[i, j] = 20 * n * EPS
                else:
                    B[i, j] = sin_theta[cl[a]] + sin_theta[cl[c]] + 20 * n * EPS
    return B


@settings(max_examples=100, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(tridiagonals())
def test_vectors_meet_residual_and_orthogonality(T):
    d, e = T
    n = len(d)
    W, Z = oracle.eigh_tridiagonal(d, e)
    # residual of 2^k T with 2^k ||T|| in [1, 2) (exact scaling), so that the
    # check itself neither overflows nor underflows
    tn = _norm(d, e)
    k = 1 - int(np.frexp(tn)[1]) if tn > 0 else 0
    Ws = np.ldexp(W, k)
    A = oracle.tridiag_dense(np.ldexp(d, k), np.ldexp(e, k))
    res = np.linalg.norm(A @ Z - Z * Ws[None, :], axis=0)
    assert float(np.max(res)) <= 20 * n * EPS * max(np.ldexp(tn, k), 1.0)
    assert np.all(np.abs(np.linalg.norm(Z, axis=0) - 1.0) <= 20 * n * EPS)
    off = np.abs(Z.T @ Z - np.eye(n))
    bound = _pair_bounds(d, e, Ws, Z, res)
    bad = np.argwhere(off > bound)
    assert bad.size == 0, f"pairs {bad[:4].tolist()}: {off[tuple(bad[0])]:.3e} > {bound[tuple(bad[0])]:.3e}"


@settings(max_examples=100, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(tridiagonals(), st.data())
def test_subset_is_a_slice_of_the_full_solve(T, data):
    """Eigenvalues il..iu are exactly the slice of the full solve (the same
    bisection to full accuracy), and the subset's vectors meet the residual
    goal and are orthonormal within the subset's own clusters."""
    d, e = T
    n = len(d)
    il = data.draw(st.integers(1, n))
    iu = data.draw(st.integers(il, n))
    Wa = oracle.eigvalsh_tridiagonal(d, e)
    W, Z = oracle.eigh_tridiagonal(d, e, il, iu)
    assert np.array_equal(W, Wa[il - 1:iu])
    assert np.array_equal(oracle.eigvalsh_tridiagonal(d, e, il, iu), W)
    tn = _norm(d, e)
    k = 1 - int(np.frexp(tn)[1]) if tn > 0 else 0
    A = oracle.tridiag_dense(np.ldexp(d, k), np.ldexp(e, k))
    res = np.linalg.norm(A @ Z - Z * np.ldexp(W, k)[None, :], axis=0)
    assert float(np.max(res)) <= 20 * n * EPS * max(np.ldexp(tn, k), 1.0)
    assert np.all(np.abs(np.linalg.norm(Z, axis=0) - 1.0) <= 20 * n * EPS)


@settings(max_examples=200, deadline=None, derandomize=True)
@given(tridiagonals())
def test_gershgorin_norm_and_split_rule(T):
    """G(T) is the largest absolute row sum of the dense T (the infinity
    norm), and the split zeroes exactly the e_i with |e_i| <= eps G(T)
    (Sec. 3.1.1, footnote on numerical irreducibility), starting a block
    after each."""
    d, e = T
    n = len(d)
    A = oracle.tridiag_dense(d, e)
    g = oracle.gershgorin_norm(d, e)
    if n:
        with np.errstate(over="ignore"):
            rows = np.sum(np.abs(A), axis=1)
        assert g == np.max(rows) or np.isclose(g, np.max(rows), rtol=4 * EPS, atol=0)
    es, starts = oracle.split(d, e)
    cut = np.abs(e) <= EPS * g
    assert np.array_equal(es, np.where(cut, 0.0, e))
    assert starts.tolist() == [0] + [i + 1 for i in np.flatnonzero(cut)] + [n]


@settings(max_examples=100, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(tridiagonals())
def test_jacobi_matches_lapack(T):
    """The dense cyclic Jacobi solver (brute force for small n) on the same
    structured inputs: eigenvalues within 4 n eps ||T|| of LAPACK's,
    orthonormal vectors, residual within 20 n eps ||T||."""
    d, e = T
    n = len(d)
    W, V = oracle.jacobi(d, e)
    Wl = scipy.linalg.eigvalsh_tridiagonal(d, e) if n > 1 else d.copy()
    tn = max(float(np.max(np.abs(Wl))), np.finfo(float).tiny)
    # two approximations, each within a small multiple of eps ||T||: for tiny
    # n their difference can exceed 4 n eps ||T||, so the floor is 32 eps ||T||
    assert np.max(np.abs(np.sort(W) - Wl)) <= max(4 * n, 32) * EPS * tn
    assert float(np.max(np.abs(V.T @ V - np.eye(n)))) <= 20 * n * EPS
    k = 1 - int(np.frexp(tn)[1])
    A = oracle.tridiag_dense(np.ldexp(d, k), np.ldexp(e, k))
    R = A @ V - V * np.ldexp(W, k)[None, :]
    assert float(np.max(np.linalg.norm(R, axis=0))) <= 20 * n * EPS * 2.0
