"""Host-side logic that needs no GPU: batch packing, the seeded input
generators, and the benchmark's oracle sampling."""
import os
import sys

import numpy as np
import pytest
import torch

from paper_1205_2107_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_layout_offsets_and_unpack():
    from paper_1205_2107_gb300.api import BatchLayout
    sizes = [3, 0, 5, 1]
    lay = BatchLayout(sizes, "cpu")
    assert lay.offsets_host == [0, 3, 3, 8, 9]
    assert lay.w_offsets_host == [0, 3, 3, 8, 9]
    assert lay.z_offsets_host == [0, 9, 9, 34, 35]
    assert lay.n_total == 9 and lay.k_total == 9 and lay.z_total == 35 and lay.n_max == 5 and lay.all
    W = torch.arange(9, dtype=torch.float64)
    Z = torch.arange(35, dtype=torch.float64)
    Ws, Zs = lay.unpack(W, Z)
    assert [w.numel() for w in Ws] == sizes
    # problem 2: column-major 5 x 5 block at offset 9; Z_p[i, j] = Z[9 + j * 5 + i]
    assert Zs[2][1, 3].item() == 9 + 3 * 5 + 1
    assert tuple(Zs[1].shape) == (0, 0)


def test_batch_layout_subsets():
    from paper_1205_2107_gb300.api import BatchLayout
    lay = BatchLayout([10, 4], "cpu", il=[2, 1], iu=[5, 4])
    assert lay.ks == [4, 4] and not lay.all
    assert lay.z_offsets_host == [0, 40, 56]
    assert lay.il.tolist() == [2, 1] and lay.iu.tolist() == [5, 4]


def test_generators_are_seeded_and_shaped():
    d1, e1 = inputs.uniform(100, 7)
    d2, e2 = inputs.uniform(100, 7)
    assert np.array_equal(d1, d2) and np.array_equal(e1, e2) and e1.shape == (99,)
    d, e = inputs.wilkinson_plus(21)
    assert d[0] == 10 and d[10] == 0 and np.all(e == 1.0)
    d, e = inputs.glued_wilkinson(3, glue=1e-10)
    assert d.shape == (63,) and e[20] == 1e-10 and e[41] == 1e-10 and e[19] == 1.0
    sizes = inputs.batch_sizes(4096)
    assert sizes.min() >= 32 and sizes.max() <= 2048 and len(sizes) == 4096
    d, e, off = inputs.batched_uniform([4, 0, 3], 1)
    assert off.tolist() == [0, 4, 4, 7] and e[3] == 0.0 and e[6] == 0.0
    d, e, w, C = inputs.adjoint_case(batch=2, n=8, seed=3)
    assert d.shape == (2, 8) and C.shape == (2, 8, 8) and np.all(e[:, -1] == 0.0)
    d, e = inputs.large_uniform(1000, 50000)
    assert d.min() >= 0 and d.max() <= 1 and e.min() >= 0 and e.max() <= 1e-2


def test_bench_oracle_windows():
    sys.path.insert(0, ROOT)
    import bench
    mats = [("a", *inputs.uniform(300, 1)), ("b", *inputs.uniform(200, 2))]
    jobs = bench.oracle_windows(mats, 3, offset=1)
    assert len(jobs) == 6
    for d, e, il, iu in jobs:
        assert 1 <= il <= iu <= len(d) and iu - il + 1 == bench.WINDOW
    done, secs = bench.oracle_sample(jobs[:2], 2)
    assert done == 2 * bench.WINDOW and secs > 0


def test_bench_records_the_host_cpu():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.host_cpu()
    assert isinstance(h["model"], str) and h["model"]
    assert h["nproc"] == os.cpu_count() and h["nproc"] >= 1


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """bench.py --impl reference: rank 0 prints one JSON line that carries the
    metric, the oracle sample as cpu_baseline, and an e2e with no copies;
    another rank prints nothing.  The window calibration is stubbed to one
    window per matrix, and the matrices to small ones, to keep this quick."""
    import argparse
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "workload_matrices",
                        lambda: [("a", *inputs.wilkinson_plus(301)), ("b", *inputs.glued_wilkinson(10))])
    monkeypatch.setattr(bench, "calibrated_windows", lambda mats, cores, secs: 1)
    args = argparse.Namespace(steps=2, warmup=1)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD


class _FakePlan:
    """Stands in for api.Plan in the retry loop: records option changes and
    reports the scripted statuses one solve after another."""

    def __init__(self, statuses):
        self.statuses = list(statuses)
        self.options = {}
        self.solves = 0

    def workspace(self, nbytes):
        return torch.empty(nbytes, dtype=torch.uint8)

    def info(self):
        st = self.statuses[min(self.solves, len(self.statuses)) - 1]
        return {"status": st, "pool_rows_used": 1000 * self.solves, "nodes": 50 * self.solves}

    def set_options(self, **options):
        self.options.update(options)


class _FakeCall:
    def __init__(self, plan):
        self.plan = plan

    def ws_bytes(self):
        return 64

    def __call__(self, ws, nbytes):
        self.plan.solves += 1
        return 0


def test_retry_grows_capacities_on_a_full_queue():
    from paper_1205_2107_gb300 import _lib, api
    plan = _FakePlan([_lib.ERR_QUEUE, _lib.OK])
    info = api._run_with_retry(plan, _FakeCall(plan), "solve", check=True)
    assert info["status"] == _lib.OK and plan.solves == 2
    # grown from what the failed solve reported: twice the rows + 1024, twice the nodes
    assert plan.options == {"pool_rows": 2 * 1000 + 1024, "max_nodes": 2 * 50}


def test_retry_gives_up_and_other_errors_raise_at_once():
    from paper_1205_2107_gb300 import _lib, api
    plan = _FakePlan([_lib.ERR_QUEUE] * 10)
    with pytest.raises(_lib.MrrrError) as ei:
        api._run_with_retry(plan, _FakeCall(plan), "solve", check=True)
    assert ei.value.code == _lib.ERR_QUEUE and plan.solves == 4
    plan = _FakePlan([_lib.ERR_NONFINITE])
    with pytest.raises(_lib.MrrrError) as ei:
        api._run_with_retry(plan, _FakeCall(plan), "solve", check=True)
    assert ei.value.code == _lib.ERR_NONFINITE and plan.solves == 1
    # unchecked: one solve, no status read
    plan = _FakePlan([_lib.ERR_QUEUE])
    assert api._run_with_retry(plan, _FakeCall(plan), "solve", check=False) is None and plan.solves == 1


def test_info_raises_when_the_status_read_fails(monkeypatch):
    """A failed synchronisation or status copy (ERR_CUDA from the host side)
    must not read as an OK solve; a device status, ERR_ARG included, is
    returned in the fields."""
    from paper_1205_2107_gb300 import _lib, api

    class FakeLib:
        def __init__(self, rc, status):
            self.rc, self.status = rc, status

        def mrrr_get_status(self, h, stream, out):
            if self.rc != _lib.ERR_CUDA:
                out._obj.status = self.status
            return self.rc

    plan = api.Plan.__new__(api.Plan)
    plan._h, plan.device = None, torch.device("cpu")
    monkeypatch.setattr(api, "_stream_handle", lambda dev: None)
    monkeypatch.setattr(_lib, "load", lambda *a, **k: FakeLib(_lib.ERR_CUDA, 0))
    with pytest.raises(_lib.MrrrError) as ei:
        plan.info()
    assert ei.value.code == _lib.ERR_CUDA
    monkeypatch.setattr(_lib, "load", lambda *a, **k: FakeLib(_lib.ERR_ARG, _lib.ERR_ARG))
    assert plan.info()["status"] == _lib.ERR_ARG
    plan._h = None  # nothing for __del__ to destroy



def test_call_objects_hold_no_reference_cycle(monkeypatch):
    """The per-call objects of the solver entries hold the plan (and with it
    its workspace) and the output tensors: dropping one must free it by
    reference counting, without waiting for the cyclic collector (a cycle
    kept several plans' workspaces alive at once)."""
    import gc
    import weakref

    from paper_1205_2107_gb300 import api

    monkeypatch.setattr(api, "slice_range", lambda il, iu, ns, s: (1, 4))
    t = torch.zeros(4, dtype=torch.float64)
    gc.disable()
    try:
        for make in (lambda: api._SteinCall(_FakePlan([]), 4, t, t, 1, 4, t, t),
                     lambda: api._SliceCall(_FakePlan([]), 4, t, t, 1, 4, 2, 0, 32, t, t),
                     lambda: api._BatchedCall(_FakePlan([]), 1, t, t, t, t, t, t, t, t, t, 4, 4, 4)):
            o = make()
            r = weakref.ref(o)
            del o
            assert r() is None
    finally:
        gc.enable()
