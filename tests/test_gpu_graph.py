"""The batched solver captured into a CUDA graph (use_graph) and the launch
autotuner: both must give the results of the directly launched solver."""
import numpy as np
import pytest
import torch

from paper_1205_2107_gb300 import api, inputs
from tests import checks

pytestmark = pytest.mark.gpu

EPS = checks.EPS


def _batch(count, seed, nmax=600):
    sizes = [int(x) for x in inputs.batch_sizes(count, seed=seed, nmin=16, nmax=nmax)]
    d, e, off = inputs.batched_uniform(sizes, seed)
    lay = api.BatchLayout(sizes, "cuda")
    return sizes, torch.as_tensor(d, device="cuda"), torch.as_tensor(e, device="cuda"), off, lay


def test_graph_replay_is_bitwise_equal_to_direct_launches():
    sizes, d, e, off, lay = _batch(64, 11)
    W0, Z0 = api.eigh_tridiagonal_batched(d, e, lay, plan=api.Plan(0))
    gplan = api.Plan(0, use_graph=1)
    W1, Z1 = api.eigh_tridiagonal_batched(d, e, lay, plan=gplan)  # capture + replay
    assert torch.equal(W0[:lay.k_total], W1[:lay.k_total])
    assert torch.equal(Z0[:lay.z_total], Z1[:lay.z_total])
    out = (W1, Z1)
    for _ in range(2):  # replays of the cached graph into the same buffers
        W1.fill_(0.0)
        api.eigh_tridiagonal_batched(d, e, lay, plan=gplan, out=out)
        assert torch.equal(W0[:lay.k_total], W1[:lay.k_total])
        assert torch.equal(Z0[:lay.z_total], Z1[:lay.z_total])
    info = gplan.info()
    assert info["status"] == 0 and info["levels"] >= 1


def test_graph_recaptures_for_new_inputs():
    sizes, d, e, off, lay = _batch(32, 12)
    gplan = api.Plan(0, use_graph=1)
    W1 = api.eigh_tridiagonal_batched(d, e, lay, plan=gplan, vectors=False)
    d2 = d * 0.5 + 0.1
    W2 = api.eigh_tridiagonal_batched(d2, e, lay, plan=gplan, vectors=False)
    R2 = api.eigh_tridiagonal_batched(d2, e, lay, plan=api.Plan(0), vectors=False)
    assert torch.equal(W2[:lay.k_total], R2[:lay.k_total])
    assert not torch.equal(W1[:lay.k_total], W2[:lay.k_total])


def test_autotune_keeps_results_valid():
    sizes, d, e, off, lay = _batch(96, 13, nmax=1000)
    plan = api.Plan(0)
    t = api.autotune_batched(d, e, lay, plan=plan)
    assert t["configs"] == 12 and t["best_ms"] <= t["default_ms"] + 1e-9
    assert t["engine_blocks_per_sm"] in (1, 2) and t["width_scale"] in (0.5, 1.0, 2.0)
    assert t["singleton_rq"] in (1, -1) and plan.options["singleton_rq"] == t["singleton_rq"]
    W, Z = api.eigh_tridiagonal_batched(d, e, lay, plan=plan)
    Ws, Zs = lay.unpack(W, Z)
    for p in range(0, len(sizes), 7):
        n = sizes[p]
        ep = torch.cat([e[off[p]:off[p + 1] - 1], torch.zeros(1, dtype=torch.float64, device="cuda")])
        tn = float(Ws[p].abs().max())
        assert float(checks.residual_cols(d[off[p]:off[p + 1]], ep, Ws[p], Zs[p]).max()) <= 20 * n * EPS * tn
        assert checks.orthogonality(Zs[p]) <= 20 * n * EPS


def test_single_problem_graph_replay_matches_direct():
    d, e = inputs.glued_wilkinson(20)
    dd = torch.as_tensor(d, device="cuda")
    ee = torch.as_tensor(np.append(e, 0.0), device="cuda")
    W0, Z0 = api.eigh_tridiagonal(dd, ee, plan=api.Plan(0))
    gplan = api.Plan(0, use_graph=1)
    for _ in range(3):  # capture, then replays (new output buffers: new signatures)
        W1, Z1 = api.eigh_tridiagonal(dd, ee, plan=gplan)
        assert torch.equal(W0, W1) and torch.equal(Z0, Z1)
    W2 = api.eigh_tridiagonal(dd, ee, 5, 40, plan=gplan, vectors=False)
    assert torch.equal(W2, api.eigh_tridiagonal(dd, ee, 5, 40, plan=api.Plan(0), vectors=False))
    # values only: fully bisected; with vectors: Rayleigh quotients, a few ulps apart
    assert float((W2 - W0[4:40]).abs().max()) <= 8 * 2.0 ** -53 * float(W0.abs().max())


def test_autotune_then_graph_recaptures():
    sizes, d, e, off, lay = _batch(48, 14, nmax=400)
    plan = api.Plan(0, use_graph=1)
    W0, Z0 = api.eigh_tridiagonal_batched(d, e, lay, plan=api.Plan(0))
    api.autotune_batched(d, e, lay, plan=plan)
    W1, Z1 = api.eigh_tridiagonal_batched(d, e, lay, plan=plan)
    # a different launch shape may change rounding inside the bisection, so
    # compare to the accuracy goals, not bit for bit
    tn = float(W0[:lay.k_total].abs().max())
    assert float((W1[:lay.k_total] - W0[:lay.k_total]).abs().max()) <= 4 * max(sizes) * EPS * tn
