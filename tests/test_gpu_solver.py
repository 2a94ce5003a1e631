"""GPU parity: the CUDA MRRR solver against the CPU oracle, element by
element, on seeded inputs of the paper's matrix families (1-2-1 / Toeplitz,
Wilkinson, glued Wilkinson) and the workload shapes (uniform random, split
matrices, subsets), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import _lib, api, inputs
from tests import checks

pytestmark = pytest.mark.gpu

EPS = checks.EPS


def to_dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def solve(d, e, il=None, iu=None, plan=None, vectors=True):
    return api.eigh_tridiagonal(to_dev(d), to_dev(e if len(e) else np.zeros(1)), il, iu, plan=plan,
                                vectors=vectors)


def assert_parity(d, e, il=None, iu=None, plan=None, compare_vectors=True):
    n = len(d)
    il_ = 1 if il is None else il
    iu_ = n if iu is None else iu
    W, Z = solve(d, e, il, iu, plan)
    Wo, Zo = oracle.eigh_tridiagonal(d, e, il_, iu_)
    Wall = oracle.eigvalsh_tridiagonal(d, e)
    tn = float(np.max(np.abs(Wall))) if n else 0.0
    Wg = W.cpu().numpy()
    assert Wg.shape == Wo.shape
    assert np.all(np.diff(Wg) >= 0), "W not ascending"
    err = np.max(np.abs(Wg - Wo)) if n else 0.0
    assert err <= 4 * n * EPS * tn, f"eigenvalue error {err:.3e} > {4 * n * EPS * tn:.3e}"
    res = float(checks.residual_cols(to_dev(d), to_dev(np.append(e, 0.0)), W, Z).max())
    assert res <= 20 * n * EPS * tn, f"residual {res:.3e}"
    orth = checks.orthogonality(Z)
    assert orth <= 20 * n * EPS, f"orthogonality {orth:.3e}"
    if compare_vectors and n > 1:
        Zg = Z.cpu().numpy()
        if il_ == 1 and iu_ == n:
            errs = checks.subspace_errors(Zg, Zo, Wo, tn, n)
        else:  # groups formed on the whole spectrum, cut groups against the oracle's whole group
            errs = checks.subset_subspace_errors(Zg, il_, iu_, Wall, d, e, tn, n, Zo)
        for sin, bound in errs:
            assert sin <= bound, f"subspace angle {sin:.3e} > {bound:.3e}"
    return W, Z


FAMILIES = {
    "uniform": lambda n: inputs.uniform(n, 1000 + n),
    "normal": lambda n: inputs.normal(n, 2000 + n),
    "toeplitz": lambda n: inputs.toeplitz(n),
    "wilkinson": lambda n: inputs.wilkinson_plus(n),
    "clement": lambda n: inputs.clement(n),
    "neg_definite": lambda n: (-3.0 - np.abs(inputs.uniform(n, 7)[0]), 0.3 * inputs.uniform(n, 8)[1]),
    "repeated_d": lambda n: (np.full(n, 0.25), inputs.uniform(n, 9)[1]),
    "zeros_in_e": lambda n: (inputs.uniform(n, 10)[0], inputs.uniform(n, 10)[1] * (np.arange(max(n - 1, 0)) % 5 != 2)),
    "tiny_e": lambda n: (inputs.uniform(n, 11)[0], 1e-9 * inputs.uniform(n, 11)[1]),
}


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 200])
@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_small_families(family, n):
    d, e = FAMILIES[family](n)
    assert_parity(d, e)


def test_uniform_1000_all():
    d, e = inputs.uniform(1000, 1205)
    assert_parity(d, e)


def test_toeplitz_1000_closed_form():
    d, e = inputs.toeplitz(1000, 2.0, -1.0)
    W, Z = assert_parity(d, e)
    ref = inputs.toeplitz_eigenvalues(1000, 2.0, -1.0)
    assert np.max(np.abs(W.cpu().numpy() - ref)) <= 4 * 1000 * EPS * 4 + 16 * EPS
    j = np.arange(1, 1001)
    Zc = Z.cpu().numpy()
    for k in [1, 2, 500, 999, 1000]:
        v = np.sin(j * k * np.pi / 1001)
        v /= np.linalg.norm(v)
        assert abs(abs(v @ Zc[:, k - 1]) - 1) <= 1e-9


@pytest.mark.parametrize("il,iu", [(1, 1), (1, 100), (400, 600), (1000, 1000), (37, 37), (999, 1000)])
def test_subsets(il, iu):
    d, e = inputs.uniform(1000, 1205)
    assert_parity(d, e, il, iu)


def test_glued_wilkinson_420():
    d, e = inputs.glued_wilkinson(20)
    assert_parity(d, e)


@pytest.mark.parametrize("n", [201, 1001])
def test_wilkinson_plus(n):
    d, e = inputs.wilkinson_plus(n)
    assert_parity(d, e)


def test_split_all_and_subset_with_ties():
    d1, e1 = inputs.uniform(40, 4)
    d = np.concatenate([d1, d1, [0.5], d1[:13]])
    e = np.concatenate([e1, [0.0], e1, [0.0], [0.0], e1[:12]])
    assert_parity(d, e)
    assert_parity(d, e, 10, 60)
    assert_parity(d, e, 41, 41)


def test_diagonal_matrix():
    d = inputs.uniform(300, 5)[0]
    e = np.zeros(299)
    W, Z = assert_parity(d, e)
    assert np.array_equal(W.cpu().numpy(), np.sort(d))


def test_deterministic():
    d, e = inputs.uniform(700, 3)
    W1, Z1 = solve(d, e)
    W2, Z2 = solve(d, e)
    assert torch.equal(W1, W2) and torch.equal(Z1, Z2)


def test_eigenvalues_only_matches_vectors_run():
    d, e = inputs.uniform(500, 12)
    W1, _ = solve(d, e)
    W2 = solve(d, e, vectors=False)
    Wo = oracle.eigvalsh_tridiagonal(d, e)
    tn = np.max(np.abs(Wo))
    assert np.max(np.abs(W2.cpu().numpy() - Wo)) <= 4 * 500 * EPS * tn
    assert np.max(np.abs(W1.cpu().numpy() - W2.cpu().numpy())) <= 4 * 500 * EPS * tn


# ---------------------------------------------------------------------------
# error paths: host-side argument errors and device-side status codes


def test_bad_arguments():
    d = to_dev(np.ones(5))
    e = to_dev(np.ones(4))
    with pytest.raises(ValueError):
        api.eigh_tridiagonal(d, e, 0, 3)
    with pytest.raises(ValueError):
        api.eigh_tridiagonal(d, e, 3, 6)
    plan = api.default_plan()
    lib = _lib.load()
    W = torch.empty(5, dtype=torch.float64, device="cuda")
    rc = lib.mrrr_stein(plan.handle, 5, d.data_ptr(), e.data_ptr(), 1, 5, W.data_ptr(), None, 5, None, 0, None)
    assert rc == _lib.ERR_WORKSPACE
    rc = lib.mrrr_stein(plan.handle, -1, d.data_ptr(), e.data_ptr(), 1, 5, W.data_ptr(), None, 5, None, 0, None)
    assert rc == _lib.ERR_ARG


def test_nonfinite_input_is_reported():
    d, e = inputs.uniform(50, 1)
    d[17] = np.nan
    with pytest.raises(_lib.MrrrError) as ei:
        solve(d, e)
    assert ei.value.code == _lib.ERR_NONFINITE


def test_bisection_cap_reports_noconv():
    plan = api.Plan(max_bisect_steps=1)
    d, e = inputs.uniform(100, 2)
    with pytest.raises(_lib.MrrrError) as ei:
        solve(d, e, plan=plan)
    assert ei.value.code == _lib.ERR_NOCONV


def test_tiny_pool_grows_and_succeeds():
    plan = api.Plan(pool_rows=1, max_nodes=1)
    d, e = inputs.wilkinson_plus(301)
    assert_parity(d, e, plan=plan)
    assert plan.options["pool_rows"] > 1


@pytest.mark.parametrize("scale_exp", [-900, -300, 300, 900])
def test_extreme_scaling_is_exact(scale_exp):
    """Power-of-two scalings of T by 2^k scale W by exactly 2^k (the solver
    scales G(T) into [1, 2) internally) and leave Z unchanged."""
    d, e = inputs.uniform(300, 77)
    W0, Z0 = solve(d, e)
    f = 2.0 ** scale_exp
    W1, Z1 = solve(d * f, e * f)
    assert torch.equal(W1, W0 * f)
    assert torch.equal(Z1, Z0)


def test_graded_matrix():
    """Entries graded over many orders of magnitude (d_i = 10^(-i/10),
    e_i = sqrt(d_i d_{i+1}) / 2): parity with the oracle."""
    n = 150
    d = 10.0 ** (-np.arange(n) / 10.0)
    e = 0.5 * np.sqrt(d[:-1] * d[1:])
    assert_parity(d, e)


def test_two_by_two_subsets():
    d, e = np.array([1.0, 3.0]), np.array([2.0])
    for il, iu in [(1, 1), (2, 2), (1, 2)]:
        assert_parity(d, e, il, iu)


# Rayleigh-quotient corrections of singletons (option singleton_rq): the same
# parity bar as the full-bisection default, on the families with clusters
# (Wilkinson, glued) and without, all eigenpairs and a subset.
RQ_CASES = {
    "uniform_500": lambda: inputs.uniform(500, 77),
    "wilkinson_201": lambda: inputs.wilkinson_plus(201),
    "glued_x10": lambda: inputs.glued_wilkinson(10),
    "toeplitz_300": lambda: inputs.toeplitz(300),
    "clement_150": lambda: inputs.clement(150),
}


@pytest.mark.parametrize("steps", [-1, 1, 2])
@pytest.mark.parametrize("case", sorted(RQ_CASES))
def test_singleton_rayleigh_quotient_correction(case, steps):
    """-1: full bisection, no correction; 1 (the default), 2: corrections."""
    d, e = RQ_CASES[case]()
    plan = api.Plan(singleton_rq=steps)
    assert_parity(d, e, plan=plan)
    n = len(d)
    assert_parity(d, e, n // 4 + 1, n // 2, plan=plan)
    info = plan.info()
    assert info["status"] == 0


def test_singleton_rq_takes_one_more_factorization_per_step():
    d, e = inputs.uniform(400, 5)
    counts = []
    for steps in (-1, 1, 2):
        plan = api.Plan(singleton_rq=steps)
        solve(d, e, plan=plan)
        counts.append(plan.info()["twisted_solves"])
    # one correction: always a second factorization; two: a third unless
    # every lane of a warp had converged after the second
    assert counts[1] == 2 * counts[0] and 2 * counts[0] <= counts[2] <= 3 * counts[0]


def test_singleton_rq_options_are_checked():
    with pytest.raises(_lib.MrrrError):
        api.Plan(singleton_rq=5)
    with pytest.raises(_lib.MrrrError):
        api.Plan(singleton_rq=-2)
    # double-double vectors make their own correction: the FP64 option is ignored
    d, e = inputs.uniform(300, 6)
    plan = api.Plan(singleton_rq=2, vector_precision=2)
    assert_parity(d, e, plan=plan)
    assert plan.info()["twisted_solves"] == 2 * 300


@pytest.mark.parametrize("rtol", [2.0 ** -13, 2.0 ** -20])
@pytest.mark.parametrize("case", ["wilkinson_201", "glued_x10", "uniform_500"])
def test_fp32_prebisection_width(case, rtol):
    """The FP32 pre-bisection of the root intervals (option prebisect_rtol,
    2^-17 by default) only moves halvings between the FP32 and FP64 pipes:
    at its widest and narrowest setting the solve meets the same goals."""
    d, e = RQ_CASES[case]()
    plan = api.Plan(prebisect_rtol=rtol)
    assert_parity(d, e, plan=plan)
    assert plan.info()["status"] == 0
