"""GPU parity of the dense stages around the tridiagonal solver (paper Sec.
1.2, stages 3-5): Householder reduction to tridiagonal form (mrrr_sytrd),
the tridiagonal MRRR solve, and the backtransformation Y = Q Z
(mrrr_ormtr), against the CPU oracle (oracle/dense.py) and the accuracy
goals of the dense problem: eigenvalues within 20 n eps ||A|| of the
oracle's, residuals ||A y - lambda y|| within 20 n eps ||A||, |Y^T Y - I|
within 20 n eps."""
import numpy as np
import pytest
import torch

from oracle import dense as odense
from paper_1205_2107_gb300 import api
from tests import checks

pytestmark = pytest.mark.gpu

EPS = checks.EPS


def sym(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return (X + X.T) / 2


def clustered(n, seed):
    """Q diag(lambda) Q^T with lambda in a few tight groups (glued-like
    clusters for the tridiagonal stage)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.arange(1, n // 10 + 2, dtype=np.float64), 10)[:n] + 1e-12 * rng.standard_normal(n)
    return (Q * lam) @ Q.T


def graded(n, seed):
    rng = np.random.default_rng(seed)
    s = np.logspace(0, -8, n)
    X = sym(n, seed)
    return (s[:, None] * X) * s[None, :] + np.diag(s * s)


CASES = {"sym": sym, "clustered": clustered, "graded": graded}


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n", [1, 2, 3, 33, 64, 65, 200, 500])
@pytest.mark.parametrize("case", sorted(CASES))
def test_dense_eigenpairs_match_the_oracle(case, n):
    A = CASES[case](n, 1000 + n)
    A = (A + A.T) / 2
    At = dev(A)
    W, Y = api.eigh_dense(At)
    Wo, Yo = odense.eigh_dense(A)
    nrm = max(float(np.max(np.abs(Wo))), 1e-300)
    Wg = W.cpu().numpy()
    assert np.all(np.diff(Wg) >= 0)
    assert float(np.max(np.abs(Wg - Wo))) <= 20 * n * EPS * nrm
    R = At @ Y - Y * W[None, :]
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 20 * n * EPS * nrm
    assert checks.orthogonality(Y) <= 20 * n * EPS
    if n > 1:
        # subspaces per group of near-equal eigenvalues against the oracle's vectors
        for sin, bound in checks.subspace_errors(Y.cpu().numpy(), Yo, Wo, nrm, n):
            assert sin <= bound


@pytest.mark.parametrize("n", [2, 3, 40, 129, 300])
def test_reduction_is_an_orthogonal_similarity(n):
    A = sym(n, 7 + n)
    At = dev(A)
    d, e, tau, R = api.tridiagonalize(At)
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    Q = api.apply_q(R, tau, I)
    T = torch.diag(d) + torch.diag(e, 1) + torch.diag(e, -1)
    nrm = float(np.linalg.norm(A, 2))
    assert float((Q.t() @ Q - I).abs().max()) <= 20 * n * EPS
    assert float((Q.t() @ At @ Q - T).abs().max()) <= 20 * n * EPS * nrm
    # the oracle's reduction uses the same reflectors (beta = -sign(alpha) ||x||)
    do, eo, _, _ = odense.tridiagonal_reduction(A)
    assert float(np.max(np.abs(d.cpu().numpy() - do))) <= 20 * n * EPS * nrm
    assert float(np.max(np.abs(e.cpu().numpy() - eo))) <= 20 * n * EPS * nrm


def test_dense_subset_and_values_only():
    n = 300
    A = sym(n, 99)
    At = dev(A)
    Wall = api.eigh_dense(At, vectors=False)
    W, Y = api.eigh_dense(At, 50, 120)
    Wo = odense.eigh_dense(A)[0]
    nrm = float(np.max(np.abs(Wo)))
    assert float(np.max(np.abs(Wall.cpu().numpy() - Wo))) <= 20 * n * EPS * nrm
    assert float(np.max(np.abs(W.cpu().numpy() - Wo[49:120]))) <= 20 * n * EPS * nrm
    R = At @ Y - Y * W[None, :]
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 20 * n * EPS * nrm
    assert checks.orthogonality(Y) <= 20 * n * EPS


def test_dense_1000_against_the_oracle():
    n = 1000
    A = sym(n, 2024)
    At = dev(A)
    W, Y = api.eigh_dense(At)
    Wo = odense.eigh_dense(A)[0]
    nrm = float(np.max(np.abs(Wo)))
    assert float(np.max(np.abs(W.cpu().numpy() - Wo))) <= 20 * n * EPS * nrm
    R = At @ Y - Y * W[None, :]
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 20 * n * EPS * nrm
    assert checks.orthogonality(Y) <= 20 * n * EPS


def test_dense_is_deterministic():
    A = dev(sym(257, 5))
    W1, Y1 = api.eigh_dense(A)
    W2, Y2 = api.eigh_dense(A)
    assert torch.equal(W1, W2) and torch.equal(Y1, Y2)


# ---------------------------------------------------------------------------
# Generalized symmetric-definite problem A x = lambda B x (stages 1, 2, 6).

def spd(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return X @ X.T + n * np.eye(n)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 130, 400])
def test_cholesky_matches_the_oracle(n):
    B = spd(n, 50 + n)
    L = api.cholesky(dev(B))
    Lo = odense.cholesky(B)
    nb = float(np.linalg.norm(B, 2))
    assert float(np.max(np.abs(L.cpu().numpy() - Lo))) <= 20 * n * EPS * np.sqrt(nb)
    assert float((L @ L.t() - dev(B)).abs().max()) <= 20 * n * EPS * nb


def test_cholesky_reports_a_matrix_that_is_not_positive_definite():
    B = spd(100, 3)
    B[70, 70] = -1e6
    with pytest.raises(Exception) as err:
        api.cholesky(dev(B))
    assert "NOTSPD" in str(err.value)


@pytest.mark.parametrize("n", [1, 3, 64, 97, 300])
def test_generalized_eigenpairs_match_the_oracle(n):
    A, B = sym(n, 600 + n), spd(n, 700 + n)
    W, X = api.eigh_generalized(dev(A), dev(B))
    Wo, Xo = odense.eigh_generalized(A, B)
    nrm = max(float(np.max(np.abs(Wo))), 1.0)
    nb = float(np.linalg.norm(B, 2))
    Wg = W.cpu().numpy()
    assert np.all(np.diff(Wg) >= 0)
    # the pencil is well conditioned (B = X X^T + n I): eigenvalues to the
    # tolerance of the standard problem on C = L^-1 A L^-T
    assert float(np.max(np.abs(Wg - Wo))) <= 40 * n * EPS * nrm
    At, Bt = dev(A), dev(B)
    R = At @ X - (Bt @ X) * W[None, :]
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 40 * n * EPS * nrm * nb
    G = X.t() @ Bt @ X
    assert float((G - torch.eye(n, dtype=torch.float64, device="cuda")).abs().max()) <= 40 * n * EPS


def test_generalized_subset():
    n = 200
    A, B = sym(n, 11), spd(n, 12)
    W, X = api.eigh_generalized(dev(A), dev(B), 20, 60)
    Wo = odense.eigh_generalized(A, B)[0]
    nrm = float(np.max(np.abs(Wo)))
    assert float(np.max(np.abs(W.cpu().numpy() - Wo[19:60]))) <= 40 * n * EPS * nrm
    G = X.t() @ dev(B) @ X
    assert float((G - torch.eye(41, dtype=torch.float64, device="cuda")).abs().max()) <= 40 * n * EPS
