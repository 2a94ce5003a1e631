"""GPU parity of the batched solver (mrrr_stein_batched): many independent
problems of uneven sizes in one set of launches, against the CPU oracle per
problem and against the single-problem path, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import api, inputs
from tests import checks

pytestmark = pytest.mark.gpu

EPS = checks.EPS


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def check_problem(d, e, W, Z, il, iu, compare_vectors=True):
    """Parity of one problem's (W, Z) with the oracle (tolerances of the
    accuracy goals: 4 n eps ||T||, 20 n eps ||T||, 20 n eps)."""
    n = len(d)
    eo = e[:max(n - 1, 0)]
    if compare_vectors:
        Wo, Zo = oracle.eigh_tridiagonal(d, eo, il, iu)
    else:  # eigenvalues only (inverse iteration on long chained clusters is slow)
        Wo, Zo = oracle.eigvalsh_tridiagonal(d, eo, il, iu), None
    tn = float(np.max(np.abs(oracle.eigvalsh_tridiagonal(d, eo)))) if n else 0.0
    Wg = W.cpu().numpy()
    assert Wg.shape == Wo.shape
    assert np.all(np.diff(Wg) >= 0)
    assert np.max(np.abs(Wg - Wo)) <= 4 * n * EPS * tn
    if Z is None:
        return
    res = float(checks.residual_cols(_dev(d), _dev(np.append(e[:max(n - 1, 0)], 0.0)), W, Z).max())
    assert res <= 20 * n * EPS * tn, f"residual {res:.3e}"
    assert checks.orthogonality(Z) <= 20 * n * EPS
    if compare_vectors and n > 1:
        if il == 1 and iu == n:
            errs = checks.subspace_errors(Z.cpu().numpy(), Zo, Wo, tn, n)
        else:
            Wall = oracle.eigvalsh_tridiagonal(d, eo)
            errs = checks.subset_subspace_errors(Z.cpu().numpy(), il, iu, Wall, d, eo, tn, n, Zo)
        for sin, bound in errs:
            assert sin <= bound, f"subspace angle {sin:.3e} > {bound:.3e}"


def solve_batch(sizes, seed, il=None, iu=None, vectors=True):
    d, e, off = inputs.batched_uniform(sizes, seed)
    lay = api.BatchLayout(sizes, "cuda", il, iu)
    out = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay, vectors=vectors)
    W, Z = out if vectors else (out, None)
    Ws, Zs = lay.unpack(W, Z) if vectors else (lay.unpack(W), [None] * len(sizes))
    probs = [(d[off[p]:off[p + 1]], e[off[p]:off[p + 1]]) for p in range(len(sizes))]
    return lay, probs, Ws, Zs


def test_ragged_batch_all_eigenpairs():
    sizes = [int(x) for x in inputs.batch_sizes(48, seed=3, nmin=1, nmax=300)]
    sizes[:4] = [1, 2, 3, 300]  # edge sizes in one launch
    lay, probs, Ws, Zs = solve_batch(sizes, 31)
    for (d, e), W, Z, n in zip(probs, Ws, Zs, sizes):
        check_problem(d, e, W, Z, 1, n)


def test_batch_subsets_per_problem():
    sizes = [50, 400, 7, 128, 129, 1000]
    il = [1, 200, 7, 1, 64, 990]
    iu = [50, 210, 7, 1, 65, 1000]
    lay, probs, Ws, Zs = solve_batch(sizes, 17, il, iu)
    for (d, e), W, Z, a, b in zip(probs, Ws, Zs, il, iu):
        check_problem(d, e, W, Z, a, b)


def test_batch_matches_single_problem_path():
    sizes = [64, 257, 33, 512]
    lay, probs, Ws, Zs = solve_batch(sizes, 99)
    for (d, e), W, Z in zip(probs, Ws, Zs):
        n = len(d)
        W1, Z1 = api.eigh_tridiagonal(_dev(d), _dev(e))
        tn = float(W1.abs().max())
        assert float((W - W1).abs().max()) <= 4 * n * EPS * tn
        # the same subspaces: |Z^T Z1| is a permutation-free orthogonal matrix block-diagonally
        M = (Z.t() @ Z1).abs()
        assert float((M.max(1).values - 1.0).abs().max()) <= 1e-7


def test_batch_with_split_problems_and_values_only():
    sizes = [40, 40, 40]
    d, e, off = inputs.batched_uniform(sizes, 5)
    e[off[0] + 10] = 0.0  # problem 0 splits into two blocks
    e[off[1]:off[2] - 1:4] = 1e-300  # problem 1 splits into many blocks
    lay = api.BatchLayout(sizes, "cuda")
    W = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay, vectors=False)
    W2, Z2 = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay)
    # with vectors the singletons' eigenvalues are Rayleigh quotients of the
    # vectors (default singleton_rq = 1), without them fully bisected values:
    # the same to a few ulps; with full bisection bit for bit
    tn = float(W2[:lay.k_total].abs().max())
    assert float((W[:lay.k_total] - W2[:lay.k_total]).abs().max()) <= 8 * EPS * tn
    W3, _ = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay, plan=api.Plan(singleton_rq=-1))
    assert torch.equal(W[:lay.k_total], W3[:lay.k_total])
    Ws, Zs = lay.unpack(W2, Z2)
    for p, (W_, Z_) in enumerate(zip(Ws, Zs)):
        check_problem(d[off[p]:off[p + 1]], e[off[p]:off[p + 1]], W_, Z_, 1, sizes[p])


def test_full_size_batch_4096_sampled():
    """4096 problems, sizes log-uniform in [32, 2048] (the batched workload):
    every problem checked for residual and orthogonality on the GPU, sampled
    problems against the oracle."""
    sizes = [int(x) for x in inputs.batch_sizes()]
    d, e, off = inputs.batched_uniform(sizes)
    lay = api.BatchLayout(sizes, "cuda")
    dt, et = _dev(d), _dev(e)
    W, Z = api.eigh_tridiagonal_batched(dt, et, lay)
    Ws, Zs = lay.unpack(W, Z)
    worst_res = worst_orth = 0.0
    for p in range(len(sizes)):
        n = sizes[p]
        Wp, Zp = Ws[p], Zs[p]
        tn = float(Wp.abs().max())
        ep = torch.cat([et[off[p]:off[p + 1] - 1], torch.zeros(1, dtype=torch.float64, device="cuda")])
        res = float(checks.residual_cols(dt[off[p]:off[p + 1]], ep, Wp, Zp).max()) / (n * EPS * tn)
        orth = checks.orthogonality(Zp) / (n * EPS)
        worst_res, worst_orth = max(worst_res, res), max(worst_orth, orth)
    assert worst_res <= 20 and worst_orth <= 20, (worst_res, worst_orth)
    # 64 seeded problems (and the largest) against the oracle's eigenvalues,
    # 8 of them also against the oracle's vectors (subspace angles)
    rng = np.random.default_rng(0)
    picks = sorted(set(rng.choice(len(sizes), 64, replace=False).tolist()) | {int(np.argmax(sizes))})
    with_vectors = set(rng.choice(picks, 8, replace=False).tolist())
    for p in picks:
        check_problem(d[off[p]:off[p + 1]], e[off[p]:off[p + 1]], Ws[p], Zs[p], 1, sizes[p],
                      compare_vectors=p in with_vectors)


def test_batch_with_empty_problems():
    """Problems of order 0 inside a batch produce nothing and disturb nothing."""
    sizes = [0, 5, 0, 17, 1, 0]
    d, e, off = inputs.batched_uniform(sizes, 23)
    lay = api.BatchLayout(sizes, "cuda")
    W, Z = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay)
    Ws, Zs = lay.unpack(W, Z)
    for p, n in enumerate(sizes):
        assert Ws[p].numel() == n and tuple(Zs[p].shape) == (n, n)
        if n:
            check_problem(d[off[p]:off[p + 1]], e[off[p]:off[p + 1]], Ws[p], Zs[p], 1, n)


def test_single_problem_of_order_zero():
    W, Z = api.eigh_tridiagonal(torch.zeros(0, dtype=torch.float64, device="cuda"),
                                torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert W.numel() == 0 and Z.numel() == 0


@pytest.mark.parametrize("width", [1, 4])
def test_batched_equals_plain_bitwise_under_a_fixed_schedule(width):
    """With a fixed multisection width (no pooling of points across
    intervals), an eigenpair's computation depends on its own problem alone:
    the batched solve and the single-problem solve give the same bits."""
    sizes = [64, 257, 33, 512, 1, 300]
    d, e, off = inputs.batched_uniform(sizes, 99)
    d[off[5]:off[6]] = inputs.glued_wilkinson(15)[0][:300]  # clustered problem in the batch
    e[off[5]:off[6] - 1] = inputs.glued_wilkinson(15)[1][:299]
    lay = api.BatchLayout(sizes, "cuda")
    plan = api.Plan(multisection_width=width)
    W, Z = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay, plan=plan)
    Ws, Zs = lay.unpack(W, Z)
    plan1 = api.Plan(multisection_width=width)
    for p, n in enumerate(sizes):
        W1, Z1 = api.eigh_tridiagonal(_dev(d[off[p]:off[p + 1]]), _dev(e[off[p]:off[p + 1]]), plan=plan1)
        assert torch.equal(Ws[p], W1), f"problem {p}: W differs"
        assert torch.equal(Zs[p], Z1), f"problem {p}: Z differs"
        check_problem(d[off[p]:off[p + 1]], e[off[p]:off[p + 1]], W1, Z1, 1, n, compare_vectors=n <= 300)


def test_one_lane_and_two_lane_vectors_are_bit_for_bit_alike():
    """A batch with more vectors than one wave of the GPU's lanes computes
    the first whole waves with one lane per vector and the rest with two
    (twisted_pair); each problem alone has fewer vectors than a wave and
    takes two lanes for all.  Under a fixed schedule the bits must agree."""
    sizes = [1000] * 24  # 24,000 eigenpairs: more than 608 x 32 slots
    d, e, off = inputs.batched_uniform(sizes, 123)
    lay = api.BatchLayout(sizes, "cuda")
    plan = api.Plan(multisection_width=4)
    W, Z = api.eigh_tridiagonal_batched(_dev(d), _dev(e), lay, plan=plan)
    Ws, Zs = lay.unpack(W, Z)
    plan1 = api.Plan(multisection_width=4)
    for p in (0, 5, 11, 17, 23):  # early problems in the one-lane waves, the last in the two-lane rest
        W1, Z1 = api.eigh_tridiagonal(_dev(d[off[p]:off[p + 1]]), _dev(e[off[p]:off[p + 1]]), plan=plan1)
        assert torch.equal(Ws[p], W1), f"problem {p}: W differs"
        assert torch.equal(Zs[p], Z1), f"problem {p}: Z differs"
