"""Pins of the dense oracle (oracle/dense.py), CPU only: the stages around the
tridiagonal eigenproblem (paper Sec. 1.2) checked against facts that do not
come from the oracle itself -- orthogonality and the similarity Q^T A Q = T,
LAPACK's eigenvalues (numpy.linalg.eigvalsh / eigh, an independent library
routine), a matrix that is already tridiagonal, closed forms, NumPy's
Cholesky, and the generalized pencil's defining identities -- with planted
mistakes that the pins must catch."""
import numpy as np
import pytest

from oracle import dense

EPS = 2.0 ** -53


def sym(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return (X + X.T) / 2


def spd(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return X @ X.T + n * np.eye(n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 40, 120])
def test_reduction_is_an_orthogonal_similarity_to_a_tridiagonal(n):
    A = sym(n, n)
    d, e, V, tau = dense.tridiagonal_reduction(A)
    Q = dense.form_q(V, tau, n)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = np.linalg.norm(A, 2)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * n * EPS
    assert np.max(np.abs(Q.T @ A @ Q - T)) <= 10 * n * EPS * nrm
    # Q e_0 = e_0: the first row and column are never touched by a reflector
    assert np.array_equal(Q[:, 0], np.eye(n)[:, 0])


@pytest.mark.parametrize("n", [4, 33, 150])
def test_tridiagonal_eigenvalues_are_lapacks(n):
    A = sym(n, 100 + n)
    d, e, _, _ = dense.tridiagonal_reduction(A)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ref = np.linalg.eigvalsh(A)
    assert np.max(np.abs(np.linalg.eigvalsh(T) - ref)) <= 10 * n * EPS * np.max(np.abs(ref))


def test_an_already_tridiagonal_matrix_is_left_as_it_is():
    rng = np.random.default_rng(3)
    n = 30
    d0, e0 = rng.standard_normal(n), rng.standard_normal(n - 1)
    A = np.diag(d0) + np.diag(e0, 1) + np.diag(e0, -1)
    d, e, V, tau = dense.tridiagonal_reduction(A)
    assert np.array_equal(d, d0) and np.array_equal(e, e0) and np.all(tau == 0.0)


def test_householder_vector_maps_onto_the_first_axis():
    rng = np.random.default_rng(5)
    for m in (1, 2, 7):
        x = rng.standard_normal(m)
        v, t, beta = dense.householder_vector(x)
        y = x - t * v * (v @ x)
        assert abs(y[0] - beta) <= 4 * EPS * np.linalg.norm(x)
        assert np.max(np.abs(y[1:]), initial=0.0) <= 4 * EPS * np.linalg.norm(x)
        assert abs(abs(beta) - np.linalg.norm(x)) <= 4 * EPS * np.linalg.norm(x)


def test_dense_eigenpairs_closed_form():
    """A = c I + u u^T: eigenvalues c (n-1 times) and c + ||u||^2, the last
    one's vector u / ||u||."""
    rng = np.random.default_rng(7)
    n = 25
    u = rng.standard_normal(n)
    c = 1.5
    A = c * np.eye(n) + np.outer(u, u)
    W, Y = dense.eigh_dense(A)
    assert np.max(np.abs(W[:-1] - c)) <= 20 * n * EPS * (c + u @ u)
    assert abs(W[-1] - (c + u @ u)) <= 20 * n * EPS * (c + u @ u)
    assert abs(abs(Y[:, -1] @ u) / np.linalg.norm(u) - 1.0) <= 1e-10


@pytest.mark.parametrize("n", [1, 2, 64, 200])
def test_dense_eigenpairs_residual_orthogonality_and_lapack(n):
    A = sym(n, 200 + n)
    W, Y = dense.eigh_dense(A)
    nrm = np.max(np.abs(W))
    assert np.max(np.abs(W - np.linalg.eigvalsh(A))) <= 20 * n * EPS * nrm
    assert np.max(np.linalg.norm(A @ Y - Y * W, axis=0)) <= 20 * n * EPS * nrm
    assert np.max(np.abs(Y.T @ Y - np.eye(n))) <= 20 * n * EPS


def test_dense_subset_is_a_slice_of_all():
    A = sym(80, 9)
    W, Y = dense.eigh_dense(A)
    Ws, Ys = dense.eigh_dense(A, 11, 30)
    assert np.max(np.abs(Ws - W[10:30])) <= 100 * EPS * np.max(np.abs(W))
    assert np.max(np.linalg.norm(A @ Ys - Ys * Ws, axis=0)) <= 20 * 80 * EPS * np.max(np.abs(W))


def test_cholesky_is_numpys():
    for n in (1, 3, 50):
        B = spd(n, n)
        L = dense.cholesky(B)
        assert np.allclose(np.tril(L), L, atol=0.0)
        assert np.max(np.abs(L @ L.T - B)) <= 10 * n * EPS * np.linalg.norm(B, 2)
        assert np.max(np.abs(L - np.linalg.cholesky(B))) <= 100 * n * EPS * np.sqrt(np.linalg.norm(B, 2))
    with pytest.raises(ValueError):
        dense.cholesky(-np.eye(3))


def test_triangular_solves():
    rng = np.random.default_rng(11)
    L = np.tril(rng.standard_normal((20, 20))) + 20 * np.eye(20)
    Bm = rng.standard_normal((20, 4))
    X = dense.forward_substitution(L, Bm)
    assert np.max(np.abs(L @ X - Bm)) <= 1e-12
    X = dense.back_substitution_transposed(L, Bm)
    assert np.max(np.abs(L.T @ X - Bm)) <= 1e-12


@pytest.mark.parametrize("n", [1, 6, 90])
def test_generalized_pencil(n):
    A, B = sym(n, 300 + n), spd(n, 400 + n)
    W, X = dense.eigh_generalized(A, B)
    nrm = np.max(np.abs(W))
    # A X = B X Lambda and X^T B X = I: the pencil's defining identities
    assert np.max(np.abs(A @ X - (B @ X) * W)) <= 100 * n * EPS * max(nrm, 1.0) * np.linalg.norm(B, 2)
    assert np.max(np.abs(X.T @ B @ X - np.eye(n))) <= 100 * n * EPS
    # eigenvalues of the pencil from LAPACK via the symmetric L^-1 A L^-T of NumPy's own factor
    Ln = np.linalg.cholesky(B)
    Li = np.linalg.inv(Ln)
    ref = np.linalg.eigvalsh(Li @ A @ Li.T)
    assert np.max(np.abs(W - ref)) <= 1e-10 * max(nrm, 1.0)


def test_planted_mistakes_fail_the_pins():
    """A dropped correction term in the two-sided update, or a reflector
    applied in the wrong order, must fail the similarity or LAPACK pins."""
    n = 30
    A = sym(n, 31)
    ref = np.linalg.eigvalsh(A)

    # 1: w = p without the (tau/2)(p^T v) v correction
    B = np.array(A)
    for k in range(n - 2):
        v, t, beta = dense.householder_vector(B[k + 1:, k])
        S = B[k + 1:, k + 1:]
        p = t * (S @ v)
        S -= np.outer(v, p) + np.outer(p, v)
        B[k + 1:, k + 1:] = S
        B[k + 1:, k] = 0.0
        B[k, k + 1:] = 0.0
        B[k + 1, k] = B[k, k + 1] = beta
    assert np.max(np.abs(np.linalg.eigvalsh(np.tril(B) + np.tril(B, -1).T) - ref)) > 1e-6
    # 2: reflectors applied first-to-last in apply_q
    d, e, V, tau = dense.tridiagonal_reduction(A)
    Qbad = np.eye(n)
    for k in range(V.shape[1]):
        v = V[k + 1:, k]
        Qbad[k + 1:, :] -= tau[k] * np.outer(v, v @ Qbad[k + 1:, :])
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.max(np.abs(Qbad.T @ A @ Qbad - T)) > 1e-6
