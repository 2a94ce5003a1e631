"""Command-line solve of one synthetic tridiagonal (for timing and profiling).

    python -m paper_1205_2107_gb300.cli --family wilkinson --n 4001 --repeat 3

Families are the seeded generators of ``inputs``: uniform (d, e iid
U[-1, 1]), normal, toeplitz (d = 2, e = -1), wilkinson (W+), glued (copies of
W21+ glued by 1e-10; --n is the number of copies), clement, large (d U[0,1],
e U[0, 1e-2]); batch (--n problems of sizes log-uniform in [32, 2048], one
batched solve); dense (an n x n symmetric matrix with N(0,1) entries: the
reduction to tridiagonal form, the tridiagonal solve and the
backtransformation; --generalized adds B = G G^T + n I).  Prints the stage
profile of the last solve as one JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import api, inputs

FAMILIES = {
    "uniform": lambda n, seed: inputs.uniform(n, seed),
    "normal": lambda n, seed: inputs.normal(n, seed),
    "toeplitz": lambda n, seed: inputs.toeplitz(n),
    "wilkinson": lambda n, seed: inputs.wilkinson_plus(n),
    "glued": lambda n, seed: inputs.glued_wilkinson(n),
    "clement": lambda n, seed: inputs.clement(n),
    "large": lambda n, seed: inputs.large_uniform(n, seed),
}


def run_batch(args, dev):
    """--n problems with sizes log-uniform in [32, 2048], d, e iid U[-1,1]."""
    sizes = [int(x) for x in inputs.batch_sizes(args.n, args.seed)]
    d, e, _ = inputs.batched_uniform(sizes, args.seed)
    lay = api.BatchLayout(sizes, dev)
    dd, ee = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    plan = api.Plan(dev)
    plan.set_timing(True)
    times = []
    for _ in range(args.repeat):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        api.eigh_tridiagonal_batched(dd, ee, lay, plan=plan, vectors=not args.values_only)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    info = plan.info()
    prof = plan.profile()
    print(json.dumps({"family": "batch", "problems": len(sizes), "n_total": lay.n_total, "ms": times,
                      "status": info["status"], "depth": info["depth"], "nodes": info["nodes"],
                      "launches": prof["launches"], "stages_ms": prof["stages"]}))
    if info["status"] != 0:
        raise SystemExit(f"solver status {info['status']}")


def run_dense(args, dev):
    """Dense symmetric A = (X + X^T) / 2, X iid N(0, 1) (seeded): stage times
    of one reduction, tridiagonal solve and backtransformation, then of the
    whole driver, each over --repeat runs (CUDA events)."""
    rng = np.random.default_rng(args.seed)
    X = rng.standard_normal((args.n, args.n))
    A = torch.tensor((X + X.T) / 2, device=dev)
    B = None
    if args.generalized:
        G = rng.standard_normal((args.n, args.n))
        B = torch.tensor(G @ G.T + args.n * np.eye(args.n), device=dev)
    plan = api.Plan(dev)

    def timed(fn):
        ms = []
        for _ in range(args.repeat):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            out = fn()
            ev1.record()
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return out, ms

    (d, e, tau, R), t_trd = timed(lambda: api.tridiagonalize(A, plan=plan))
    eo = torch.cat([e, e.new_zeros(1)])
    (W, Z), t_mrrr = timed(lambda: api.eigh_tridiagonal(d, eo, plan=plan))
    _, t_orm = timed(lambda: api.apply_q(R, tau, Z, plan=plan))
    rec = {"family": "dense", "n": args.n, "reduction_ms": t_trd, "tridiagonal_ms": t_mrrr,
           "backtransformation_ms": t_orm}
    if B is not None:
        _, rec["cholesky_ms"] = timed(lambda: api.cholesky(B, plan=plan))
        _, rec["generalized_ms"] = timed(lambda: api.eigh_generalized(A, B, plan=plan))
    else:
        _, rec["driver_ms"] = timed(lambda: api.eigh_dense(A, plan=plan))
    print(json.dumps(rec))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--family", choices=sorted(FAMILIES) + ["batch", "dense"], default="uniform")
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=1205)
    ap.add_argument("--il", type=int, default=None)
    ap.add_argument("--iu", type=int, default=None)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--values-only", action="store_true")
    ap.add_argument("--generalized", action="store_true", help="dense: the pencil (A, B) instead of A alone")
    args = ap.parse_args(argv)
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.family == "batch":
        return run_batch(args, dev)
    if args.family == "dense":
        return run_dense(args, dev)
    d, e = FAMILIES[args.family](args.n, args.seed)
    dd = torch.tensor(d, device=dev)
    ee = torch.tensor(np.append(e, 0.0), device=dev)
    plan = api.Plan(dev)
    plan.set_timing(True)
    times = []
    for _ in range(args.repeat):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        api.eigh_tridiagonal(dd, ee, args.il, args.iu, plan=plan, vectors=not args.values_only)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    info = plan.info()
    prof = plan.profile()
    print(json.dumps({"family": args.family, "n": len(d), "ms": times, "status": info["status"],
                      "depth": info["depth"], "nodes": info["nodes"], "launches": prof["launches"],
                      "stages_ms": prof["stages"]}))
    if info["status"] != 0:
        raise SystemExit(f"solver status {info['status']}")


if __name__ == "__main__":
    main()
