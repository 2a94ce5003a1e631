"""Index-range sharding on the GPU (paper Sec. 3.1.2: each process takes a
static share of the wanted eigenpairs; clusters spanning processes are
handled by the processes that hold their members).  The slices of N = 2, 3
and 4 equal parts are solved one after the other through mrrr_stein_slice,
as N GPUs would solve them, then put together and checked against the CPU
oracle: every eigenvalue, every residual, orthogonality over ALL columns
(across slices included), and subspaces per group of near-equal
eigenvalues.  Glued Wilkinson matrices put clusters of 20 and 200 equal
eigenvalues across the slice boundaries; W+ puts close pairs there."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import _lib, api, inputs
from tests import checks

pytestmark = pytest.mark.gpu

EPS = checks.EPS

CASES = {
    "uniform_1000": lambda: inputs.uniform(1000, 1205),
    "glued_x20": lambda: inputs.glued_wilkinson(20),
    "wilkinson_1001": lambda: inputs.wilkinson_plus(1001),
    "glued_x200": lambda: inputs.glued_wilkinson(200),
}


def solve_slices(d, e, il, iu, nslices, margin=32):
    dt = torch.as_tensor(d, device="cuda")
    et = torch.as_tensor(np.append(e, 0.0), device="cuda")
    plan = api.Plan()
    Ws, Zs, ranges = [], [], []
    for s in range(nslices):
        W, Z, ab = api.eigh_tridiagonal_slice(dt, et, il, iu, nslices, s, margin=margin, plan=plan)
        Ws.append(W)
        Zs.append(Z)
        ranges.append(ab)
    return dt, et, torch.cat(Ws), torch.cat(Zs, dim=1), ranges


@pytest.mark.parametrize("nslices", [2, 3, 4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_slices_together_match_the_oracle(case, nslices):
    d, e = CASES[case]()
    n = len(d)
    il, iu = 1, n
    dt, et, W, Z, ranges = solve_slices(d, e, il, iu, nslices)
    assert ranges[0][0] == il and ranges[-1][1] == iu
    assert all(b + 1 == c for (_, b), (c, _) in zip(ranges, ranges[1:]))
    Wall = oracle.eigvalsh_tridiagonal(d, e)
    tn = float(np.max(np.abs(Wall)))
    Wg = W.cpu().numpy()
    # ascending within each slice; across a boundary equal eigenvalues may
    # differ by an ulp in either order
    assert np.all(np.diff(Wg) >= -4 * EPS * tn)
    err = float(np.max(np.abs(Wg - Wall)))
    assert err <= 4 * n * EPS * tn, f"eigenvalue error {err / (n * EPS * tn):.2f} n eps ||T||"
    res = float(checks.residual_cols(dt, et, W, Z).max())
    assert res <= 20 * n * EPS * tn, f"residual {res / (n * EPS * tn):.2f} n eps ||T||"
    orth = checks.orthogonality(Z)  # every pair of columns, across slices included
    assert orth <= 20 * n * EPS, f"orthogonality {orth / (n * EPS):.2f} n eps"
    if n <= 1001:
        groups = checks.groups_by_gap(Wall, 1e-6 * tn)
        for bound, tol in checks.davis_kahan_errors(dt, et, W, Z, Wall, groups, tn, n):
            assert bound <= tol


def test_slices_of_a_subset_match_the_whole_subset():
    d, e = inputs.uniform(2000, 77)
    n = len(d)
    il, iu = 300, 1700
    dt, et, W, Z, ranges = solve_slices(d, e, il, iu, 4)
    assert (ranges[0][0], ranges[-1][1]) == (il, iu)
    W1, Z1 = api.eigh_tridiagonal(dt, et, il, iu)
    tn = float(np.max(np.abs(oracle.eigvalsh_tridiagonal(d, e))))
    assert float((W - W1).abs().max()) <= 4 * n * EPS * tn
    Wo = oracle.eigvalsh_tridiagonal(d, e, il, iu)
    assert float(np.max(np.abs(W.cpu().numpy() - Wo))) <= 4 * n * EPS * tn
    assert checks.orthogonality(Z) <= 20 * n * EPS
    assert float(checks.residual_cols(dt, et, W, Z).max()) <= 20 * n * EPS * tn


def test_a_cluster_across_the_boundary_is_computed_alike_by_both_slices():
    """Glued W21+ x200: groups of 200 equal eigenvalues.  With two slices and
    a margin wide enough, a group cut by the boundary is computed whole by
    both; the columns that one slice returns and the other computes in its
    margin are the same bits."""
    d, e = inputs.glued_wilkinson(200)
    n = len(d)
    dt = torch.as_tensor(d, device="cuda")
    et = torch.as_tensor(np.append(e, 0.0), device="cuda")
    plan = api.Plan()
    W0, Z0, (a0, b0) = api.eigh_tridiagonal_slice(dt, et, 1, n, 2, 0, margin=1024, plan=plan)
    W1, Z1, (a1, b1) = api.eigh_tridiagonal_slice(dt, et, 1, n, 2, 1, margin=1024, plan=plan)
    # the same columns through a three-way split whose middle slice straddles b0
    Wm, Zm, (am, bm) = api.eigh_tridiagonal_slice(dt, et, 1, n, 3, 1, margin=1024, plan=plan)
    assert am <= b0 < bm
    # the middle slice's columns against the two halves' columns, index by
    # index; the ordering pass may have swapped neighbours whose eigenvalues
    # are equal to the last bit, so a column may sit one place over
    Wref = torch.cat([W0[am - a0:], W1[:bm - b0]])
    Zref = torch.cat([Z0[:, am - a0:], Z1[:, :bm - b0]], dim=1)
    k = bm - am + 1
    for i in range(k):
        same = [j for j in (i - 1, i, i + 1) if 0 <= j < k and torch.equal(Zm[:, i], Zref[:, j])
                and bool(Wm[i] == Wref[j])]
        assert same, f"column {am + i} differs between the two splits"


def test_a_too_narrow_margin_is_reported_and_grown():
    d, e = inputs.glued_wilkinson(200)
    n = len(d)
    dt = torch.as_tensor(d, device="cuda")
    et = torch.as_tensor(np.append(e, 0.0), device="cuda")
    plan = api.Plan()
    # unchecked: the status word reports the margin
    W, Z, _ = api.eigh_tridiagonal_slice(dt, et, 1, n, 2, 0, margin=1, plan=plan, check=False)
    assert plan.info()["status"] == _lib.ERR_MARGIN
    # checked: the call grows the margin (8, 32, 128, 512) until the
    # boundary cluster fits
    W, Z, (a, b) = api.eigh_tridiagonal_slice(dt, et, 1, n, 2, 0, margin=8, plan=plan)
    assert plan.info()["status"] == _lib.OK
    Wo = oracle.eigvalsh_tridiagonal(d, e, a, b)
    assert float(np.max(np.abs(W.cpu().numpy() - Wo))) <= 4 * n * EPS * float(np.max(np.abs(Wo)))
