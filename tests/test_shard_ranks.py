"""Index-range sharding on CPU (paper Sec. 3.1.2: the wanted eigenpairs are
divided statically among processes): two gloo ranks each take their slice of
il..iu, and the gather of W puts the slices back in index order.  The solve
of a slice is stood in for by the oracle on the host (the GPU path of a slice
is covered by tests/test_gpu_shard.py); the slice partition is the library's
own (mrrr_slice_range, host only), and the margin retry of the slice call is
driven by a stand-in status."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1205_2107_gb300 import _lib, api, inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _host_slice(d, e, il, iu, nslices, slice_, *, margin=32, vectors=True, plan=None, check=True):
    """Stand-in for api.eigh_tridiagonal_slice: the oracle's eigenpairs of
    the slice's indices, on the host."""
    import oracle
    a, b = api.slice_range(il, iu, nslices, slice_)
    W, Z = oracle.eigh_tridiagonal(d.numpy(), e.numpy()[:d.numel() - 1], a, b)
    return torch.tensor(W), torch.tensor(Z), (a, b)


def _rank(rank, world, port, q, il, iu):
    sys.path.insert(0, ROOT)
    from paper_1205_2107_gb300 import api as api_, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        api_.eigh_tridiagonal_slice = _host_slice
        d, e = inputs.glued_wilkinson(10)
        res = shard.eigh_tridiagonal_sharded(torch.tensor(d), torch.tensor(np.append(e, 0.0)), il, iu)
        q.put((rank, res.first, res.last, res.W_local.numpy(), res.W.numpy(), res.Z_local.shape))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("il,iu", [(None, None), (7, 150)])
def test_two_gloo_ranks_split_the_index_range_and_gather_w(il, iu):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, il, iu)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    d, e = inputs.glued_wilkinson(10)
    n = len(d)
    lo, hi = (1 if il is None else il), (n if iu is None else iu)
    # the slices partition lo..hi into two contiguous, equal (within one) parts
    (r0, a0, b0, W0, Wall0, zs0), (r1, a1, b1, W1, Wall1, zs1) = got
    assert (a0, b1) == (lo, hi) and b0 + 1 == a1 and abs((b0 - a0) - (b1 - a1)) <= 1
    assert zs0 == (n, b0 - a0 + 1) and zs1 == (n, b1 - a1 + 1)
    # every rank holds the gathered W, in index order, equal to the whole range
    ref = oracle.eigvalsh_tridiagonal(d, e, lo, hi)
    for Wall in (Wall0, Wall1):
        assert np.array_equal(Wall, np.concatenate([W0, W1]))
        assert np.max(np.abs(Wall - ref)) <= 4 * n * 2.0 ** -53 * np.max(np.abs(ref))


def test_slice_ranges_cover_the_range_exactly():
    for il, iu, ns in [(1, 1000, 4), (3, 9, 3), (1, 7, 7), (5, 5, 1), (10, 100, 6)]:
        parts = [api.slice_range(il, iu, ns, s) for s in range(ns)]
        assert parts[0][0] == il and parts[-1][1] == iu
        for (a, b), (c, _) in zip(parts, parts[1:]):
            assert c == b + 1
        sizes = [b - a + 1 for a, b in parts]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    for bad in [(1, 3, 4, 0), (1, 3, 2, 2), (1, 3, 0, 0), (4, 3, 1, 0), (0, 3, 1, 0)]:
        with pytest.raises(_lib.MrrrError):
            api.slice_range(*bad)


class _FakePlan:
    def __init__(self, statuses):
        self.statuses = list(statuses)
        self.options = {}

    def workspace(self, nbytes):
        return None

    def info(self):
        return {"status": self.statuses.pop(0), "pool_rows_used": 0, "nodes": 0}


class _FakeSliceCall:
    def __init__(self):
        self.margin = 32
        self.margins = []

    def grow_margin(self):
        self.margin *= 4

    def ws_bytes(self):
        return 256

    def __call__(self, ws, nbytes):
        self.margins.append(self.margin)
        return _lib.OK


def test_margin_retry_grows_the_margin_fourfold():
    call = _FakeSliceCall()
    plan = _FakePlan([_lib.ERR_MARGIN, _lib.ERR_MARGIN, _lib.OK])
    api._run_with_retry(plan, call, "mrrr_stein_slice", check=True)
    assert call.margins == [32, 128, 512]
    call = _FakeSliceCall()
    plan = _FakePlan([_lib.ERR_MARGIN] * 4)
    with pytest.raises(_lib.MrrrError):
        api._run_with_retry(plan, call, "mrrr_stein_slice", check=True)
