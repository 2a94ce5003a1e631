#!/usr/bin/env python3
"""Benchmark of the GB300 MRRR tridiagonal eigensolver (FP64).

Workload (one "step"): all eigenpairs of the two clustered-spectrum
tridiagonals of n ~ 20,000 -- the Wilkinson matrix W+ (d_i = |i-(n+1)/2|,
e_i = 1, n = 20001) and 952 copies of W21+ glued by e = 1e-10 (n = 19,992) --
solved one after the other through the library (Sec. 2.3 of the paper names
both test families).  Metric: eigenpairs per second, whole job.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(bisection + inverse iteration, plain C) on a bounded sample of the same
workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1205_2107_gb300 import inputs  # noqa: E402

METRIC = "FP64 tridiagonal eigenpairs/s + roofline fraction; batched & adjoint vs plain"
UNIT = "eigenpairs/s"
WORKLOAD = "clustered spectra n~20000: Wilkinson W+ n=20001 + glued W21+ x952 (n=19992, glue 1e-10), all eigenpairs"
# FP64 peaks are measured on the GPU at run time (mrrr_probe_peak); these
# derived figures are used only when no GPU probe ran
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070  # SMs x DFMA/clk/SM x flops/DFMA x GHz (max SM clock)
PEAKS = {"dfma": FP64_PEAK_GFLOPS * 1e9, "dmma": None, "ddiv": None, "source": "derived"}
# Fixed algorithmic model per eigenpair and matrix row: bisection 4 flops per
# Sturm step with B = 32 steps, plus 15 flops for the twisted factorization,
# solve and normalisation; 8 bytes of Z written.
BISECT_FLOPS_PER_ROW = 4 * 32
PATH_FLOPS_PER_ROW = BISECT_FLOPS_PER_ROW + 15
ENGINE_STAGES = ("bisect_root", "prerefine", "refine", "final_bisect")
DIV_COST_DFMA = 9.0  # DFMA-equivalents of one FP64 division; replaced by the measured ratio
# DRAM bytes (read + write) of the interval engine's launches over one clustered
# step, measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum, one pass)
# on the direct-launch batched solve of the same two matrices
ENGINE_DRAM_BYTES_PER_STEP = 128.997e9


def _hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0  # fallback figure for this part


HBM_GBS = _hbm_gbs()


def workload_matrices():
    d1, e1 = inputs.wilkinson_plus(20001)
    d2, e2 = inputs.glued_wilkinson(952)
    return [("wilkinson_plus_20001", d1, e1), ("glued_w21_x952", d2, e2)]


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline)

WINDOW = 64  # consecutive eigenpair indices per oracle sample window


def oracle_windows(mats, windows: int, offset: int = 0):
    """`windows` index windows of WINDOW consecutive eigenpairs per matrix,
    evenly spread over the spectrum (shifted by `offset` so that repeated
    samples differ)."""
    jobs = []
    for _, d, e in mats:
        n = len(d)
        starts = np.linspace(1, n - WINDOW + 1, windows).astype(int)
        for s0 in starts:
            il = int(np.clip(s0 + offset, 1, n - WINDOW + 1))
            jobs.append((d, e, il, il + WINDOW - 1))
    return jobs


def oracle_sample(jobs, nthreads: int):
    """The oracle as it stands (bisection on T, inverse iteration with
    Gram-Schmidt inside clusters) on index windows, one window per host
    thread at a time.  Returns (eigenpairs, seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()

    def one(job):
        d, e, il, iu = job
        W, _ = oracle.eigh_tridiagonal(d, e, il, iu, nthreads=1)
        return len(W)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        done = sum(ex.map(one, jobs))
    return done, time.perf_counter() - t0


def calibrated_windows(mats, nthreads: int, seconds: float) -> int:
    """Windows per matrix for a sample of about `seconds` of oracle work."""
    probe = max(1, nthreads // len(mats))
    p, t = oracle_sample(oracle_windows(mats, probe), nthreads)
    per_window = t / (probe * len(mats)) * nthreads  # thread-seconds per window
    want = seconds * nthreads / per_window / len(mats)
    return int(np.clip(round(want), 1, 4096))


def host_cpu() -> dict:
    """The host's CPU model and logical core count, recorded beside the
    oracle timings (x86 /proc/cpuinfo has a model name; on Arm lscpu gives
    one, else the implementer and part codes)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        info = ""
    for line in info.splitlines():
        if line.lower().startswith("model name"):
            model = line.split(":", 1)[1].strip()
            break
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        codes = {}
        for line in info.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("CPU implementer", "CPU part") and k.strip() not in codes:
                codes[k.strip()] = v.strip()
        model = " ".join(f"{k} {v}" for k, v in codes.items()) or os.uname().machine
    return {"model": model, "nproc": os.cpu_count()}


def sample_text(windows: int, nmats: int, cores: int, secs: float) -> str:
    return (f"{windows} windows x {WINDOW} consecutive eigenpairs per matrix ({windows * WINDOW * nmats} "
            f"eigenpairs, spread over each spectrum) of the same two matrices: oracle bisection on T + "
            f"inverse iteration with Gram-Schmidt inside clusters, {cores} threads, {secs:.1f} s")


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    mats = workload_matrices()
    cores = oracle.num_threads(0)
    # each step a bounded sample: the whole run stays within a few minutes
    per_step_s = float(np.clip(150.0 / max(args.steps + args.warmup, 1), 2.0, 20.0))
    windows = calibrated_windows(mats, cores, per_step_s)
    for w in range(args.warmup):
        oracle_sample(oracle_windows(mats, max(windows // 4, 1), offset=w), cores)
    total_pairs, total_t = 0, 0.0
    for s in range(args.steps):
        p, t = oracle_sample(oracle_windows(mats, windows, offset=s + 1), cores)
        total_pairs += p
        total_t += t
    value = total_pairs / total_t
    sample = sample_text(windows, len(mats), cores, total_t / max(args.steps, 1)) + " per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: every rank solves the same workload)

def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (the job takes as long as its
    slowest rank); x itself when running alone."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, steps: int, total_ms: float, world: int) -> float:
    """Units per second for the whole job: every rank processed
    units_per_rank_step units per step, in total_ms (max over ranks)."""
    return world * units_per_rank_step * steps / (total_ms * 1e-3)


# ---------------------------------------------------------------------------
# GPU leg

def run_ours(args, rank: int, world: int):
    import torch
    import torch.distributed as dist
    from paper_1205_2107_gb300 import api, build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    # the roofline denominators, measured on this GPU before anything else runs
    global FP64_PEAK_GFLOPS, DIV_COST_DFMA
    PEAKS.update({k: api.probe_peak(k) for k in ("dfma", "dmma", "ddiv")}, source="measured")
    FP64_PEAK_GFLOPS = PEAKS["dfma"] / 1e9
    DIV_COST_DFMA = PEAKS["dfma"] / 2.0 / PEAKS["ddiv"]
    mats = workload_matrices()
    sizes = [len(d) for _, d, _ in mats]
    pairs_per_step = sum(sizes)
    # both matrices in one batched solve: their cluster levels share launches
    lay = api.BatchLayout(sizes, dev)
    d_cat = torch.tensor(np.concatenate([d for _, d, _ in mats]), device=dev)
    e_cat = torch.tensor(np.concatenate([np.append(e, 0.0) for _, _, e in mats]), device=dev)
    # pinned host buffers of the end-to-end leg, allocated once up front and
    # written once from the CPU (D2H copies into them have ranged from 14 to
    # 193 GB/s between runs on the GB300 host; the pipeline below hides that)
    host_bufs = (d_cat.cpu().pin_memory(), e_cat.cpu().pin_memory(),
                 [torch.zeros(lay.k_total, dtype=torch.float64, pin_memory=True) for _ in range(2)],
                 [torch.zeros(lay.z_total, dtype=torch.float64, pin_memory=True) for _ in range(2)])
    # the timed step: one CUDA graph replay per step (setup, the cluster
    # levels in a conditional while node decided on the device, the vectors)
    plan = api.Plan(local, use_graph=1)
    plans = [plan]
    W_out = torch.empty(lay.k_total, dtype=torch.float64, device=dev)
    Z_out = torch.empty(lay.z_total, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(check: bool):
        return api.eigh_tridiagonal_batched(d_cat, e_cat, lay, plan=plan, check=check, out=(W_out, Z_out))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # the first warm-up step is verified against the accuracy goals: a
    # solution that misses them stops the benchmark instead of being timed
    verified = None
    for w in range(max(args.warmup, 3) if args.warmup > 0 else 0):
        step(check=True)
        if w == 0:
            verified = {}
            Ws_, Zs_ = lay.unpack(W_out, Z_out)
            for p, (name, _, _) in enumerate(mats):
                a, b = lay.offsets_host[p], lay.offsets_host[p + 1]
                verified[name] = verify_solution(d_cat[a:b], e_cat[a:b], Ws_[p], Zs_[p], seed=p)
                bad = [k for k, x in verified[name].items() if (x is False) or (not isinstance(x, bool) and x > 1.0)]
                if bad:
                    raise SystemExit(f"{name}: solution misses the accuracy goals ({bad}): {verified[name]}")
            del Ws_, Zs_
            torch.cuda.empty_cache()
    for plan in plans:
        plan.set_timing(True)
    barrier()
    times = []
    stage_ms: dict[str, float] = {}
    launches = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            res = step(check=False)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
            for plan in plans:
                prof = plan.profile()
                launches += prof["launches"]
                for k, v in prof["stages"].items():
                    stage_ms[k] = stage_ms.get(k, 0.0) + v
    barrier()
    child_rows = 0
    safeguards = {}
    engine_work = {}
    for plan in plans:
        info = plan.info()
        if info["status"] != 0:
            raise SystemExit(f"solver reported status {info['status']} ({info})")
        plan.set_timing(False)
        child_rows += int(info["pool_rows_used"]) - sum(sizes)
        # how often the method's safeguards fired in the last timed solve
        safeguards = {"fallbacks": info["fallbacks"], "child_growth_bound_missed": info["diag"][5],
                      "child_second_wave": info["diag"][4], "child_recomputed": info["diag"][9],
                      "orthogonality_fix_runs": info["diag"][8], "depth": info["depth"], "levels": info["levels"],
                      "cluster_nodes": info["nodes"], "twisted_solves": info["twisted_solves"]}
        # the interval engine's actual work, per mode: Sturm counts per
        # eigenpair (the fixed model counts 32) and the share of warp lanes
        # that counted (a warp pass costs its FP64 instructions either way)
        modes = ("root", "cluster_ends", "cluster_members", "singletons")
        engine_work = {
            "counts_per_eigenpair": {m: info["sturm_counts"][i] / pairs_per_step for i, m in enumerate(modes)},
            "counts_per_eigenpair_total": sum(info["sturm_counts"]) / pairs_per_step,
            "lane_utilisation": {m: info["sturm_counts"][i] / max(32 * info["warp_passes"][i], 1)
                                 for i, m in enumerate(modes)},
            "warp_pass_rows": sum(r // max(c, 1) * p for r, c, p in zip(info["sturm_rows"], info["sturm_counts"],
                                                                        info["warp_passes"])),
        }
    total_ms = max_over_ranks(sum(times), world, dev)
    value = whole_job_rate(pairs_per_step, args.steps, total_ms, world)

    # cross-check of the stage split outside the timed region: one direct-
    # launch solve (host reads the level count) with CUDA events between the
    # stages on the solve stream
    dplan = api.Plan(local)
    api.eigh_tridiagonal_batched(d_cat, e_cat, lay, plan=dplan, out=(W_out, Z_out))
    dplan.set_timing(True)
    flush.zero_()
    torch.cuda.synchronize(dev)
    api.eigh_tridiagonal_batched(d_cat, e_cat, lay, plan=dplan, out=(W_out, Z_out), check=False)
    torch.cuda.synchronize(dev)
    stages_direct = dplan.profile()["stages"]
    del dplan

    # the same two matrices solved one after the other by the single-problem
    # path (for comparison only)
    seq_plans = [api.Plan(local) for _ in mats]
    dmats = [(torch.tensor(d, device=dev), torch.tensor(np.append(e, 0.0), device=dev)) for _, d, e in mats]

    def sequential():
        for (d, e), pl in zip(dmats, seq_plans):
            api.eigh_tridiagonal(d, e, plan=pl, check=False)

    for (d, e), pl in zip(dmats, seq_plans):
        api.eigh_tridiagonal(d, e, plan=pl)
    t_seq = _time_cuda(sequential, 2, flush)
    del dmats, seq_plans

    # end to end through the public API with host buffers: every step copies
    # d, e in from pinned memory, solves, and copies W and Z back into pinned
    # memory.  Steps are pipelined the way a serving loop would run them: step
    # k + 1 solves (on the compute stream, into the other of two output
    # buffers, with its own plan and graph) while step k's W and Z copy back on
    # a second stream; the clock stops once the last step's copy has landed.
    # One unpipelined step (solve, copy, synchronise) is timed as well.
    hd, he, hw, hz = host_bufs
    h2d = (hd.numel() + he.numel()) * 8
    d2h = (hw[0].numel() + hz[0].numel()) * 8
    plans2 = [plan, api.Plan(local, use_graph=1)]
    outs = [(W_out, Z_out), (torch.empty_like(W_out), torch.empty_like(Z_out))]
    copy_stream = torch.cuda.Stream(dev)
    solved = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_solve(b: int, check: bool):
        return api.eigh_tridiagonal_batched(hd.to(dev, non_blocking=True), he.to(dev, non_blocking=True), lay,
                                            plan=plans2[b], check=check, out=outs[b])

    def e2e_pipelined(steps: int):
        for k in range(steps):
            b = k % 2
            if k >= 2:
                stream.wait_event(copied[b])  # step k - 2's copy out of buffer b has finished
            W, Z = e2e_solve(b, check=False)
            solved[b].record(stream)
            copy_stream.wait_event(solved[b])
            with torch.cuda.stream(copy_stream):
                hw[b].copy_(W[:lay.k_total], non_blocking=True)
                hz[b].copy_(Z[:lay.z_total], non_blocking=True)
                copied[b].record(copy_stream)
        torch.cuda.synchronize(dev)

    for b in range(2):  # checked solves: size the plans, capture their graphs
        e2e_solve(b, check=True)
    e2e_pipelined(2)
    barrier()
    with ClockSampler(local) as clk_e2e:
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_pipelined(args.steps)
        e2e_total_ms = 1e3 * (time.perf_counter() - t0)
    e2e_value = whole_job_rate(pairs_per_step, args.steps, max_over_ranks(e2e_total_ms, world, dev), world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    W, Z = e2e_solve(0, check=False)
    hw[0].copy_(W[:lay.k_total], non_blocking=True)
    hz[0].copy_(Z[:lay.z_total], non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_serial_ms = 1e3 * (time.perf_counter() - t0)
    del hz, hw, outs, plans2, W, Z, host_bufs

    # roofline of the dominant kernel: the persistent interval engine (every
    # bisection stage), against the bisection part of the fixed flop model
    engine_ms = sum(stage_ms.get(k, 0.0) for k in ENGINE_STAGES) / args.steps
    nk = sum(len(d) * len(d) for _, d, _ in mats)  # rows x eigenpairs per step
    roof = None
    if engine_ms > 0:
        achieved = BISECT_FLOPS_PER_ROW * nk / (engine_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": "k_engine (interval bisection, all modes)", "achieved": achieved,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": ENGINE_DRAM_BYTES_PER_STEP,
                "traffic_source": "DRAM bytes per step of the engine's 8 launches, one ncu capture of this "
                                  "workload (profiles/k_engine_dram_bench_clustered_n20000.md): 129 GB, nearly "
                                  "all reads of child representations (each pass of a warp streams its nodes' "
                                  "rows; the 10,000+ first-level child representations, 3.2 GB, exceed L2)",
                "child_rows": child_rows,
                "engine_ms_per_step": engine_ms,
                "peak_source": "measured on this GPU by mrrr_probe_peak (FP64 FMA throughput, all SMs)"}
    # whole path against T_roof = max(F / P_fp64, 8 n k / BW), F = 143 n k
    t_flop = PATH_FLOPS_PER_ROW * nk / (FP64_PEAK_GFLOPS * 1e9)
    t_hbm = 8.0 * nk / (HBM_GBS * 1e9)
    t_roof_ms = 1e3 * max(t_flop, t_hbm)
    # division-weighted: the model's 2 divides per row of the vector step count
    # DIV_COST_DFMA flop-equivalents each instead of 1 (measured DDIV vs DFMA rate)
    t_div = (PATH_FLOPS_PER_ROW + 2 * (DIV_COST_DFMA - 1)) * nk / (FP64_PEAK_GFLOPS * 1e9)
    path_roof = {"t_roof_ms": t_roof_ms, "t_step_ms": total_ms / args.steps,
                 "frac": t_roof_ms / (total_ms / args.steps), "bound": "alu" if t_flop >= t_hbm else "hbm",
                 "frac_division_weighted": 1e3 * max(t_div, t_hbm) / (total_ms / args.steps),
                 "model": "143 n flops + 8 n bytes per eigenpair", "hbm_gbs": HBM_GBS}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.num_threads(0)
        windows = calibrated_windows(mats, cores, args.cpu_seconds)
        p, t = oracle_sample(oracle_windows(mats, windows, offset=1), cores)
        cpu = {"value": p / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample_text(windows, len(mats), cores, t), "host": host_cpu()}
    side = None
    large = None
    dense = None
    mixed = None
    shard = None
    if not args.no_side:
        side = _leg(side_by_side, args, dev, flush)
        large = _leg(large_legs, dev, flush)
        dense = _leg(dense_legs, dev, flush)
        mixed = _leg(mixed_precision_leg, dev, flush)
        shard = _leg(shard_leg, dev, flush)
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": sizes, "eigenpairs_per_step": pairs_per_step,
                       "schedule": "both matrices in one batched solve (mrrr_stein_batched), one CUDA graph "
                                   "replay per step: cluster levels in a conditional while node",
                       "sequential_plain_ms": t_seq,
                       "verified": verified,
                       "l2": "flushed before each step (256 MB write); Z output 3.2 GB per matrix",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clocks, "gpu_launches": launches, "safeguards": safeguards, "engine_work": engine_work,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_total_ms / args.steps, "serial_step_ms": e2e_serial_ms,
                    "schedule": "steps pipelined: step k+1 solves while step k's W and Z copy back on a second "
                                "stream (two output buffers, two plans); every step's copies inside the timed "
                                "region; serial_step_ms: one step with solve, copies and synchronisation in turn",
                    "clocks": clk_e2e.summary()},
            "roofline": roof, "path_roofline": path_roof, "cpu_baseline": cpu,
            "peaks": {"fp64_fma_gflops": PEAKS["dfma"] / 1e9,
                      "fp64_mma_gflops": PEAKS["dmma"] / 1e9 if PEAKS["dmma"] else None,
                      "fp64_div_g_per_s": PEAKS["ddiv"] / 1e9 if PEAKS["ddiv"] else None,
                      "source": PEAKS["source"]},
            "batched": side["batched"] if side else None, "adjoint": side["adjoint"] if side else None,
            "large_n50000": large, "dense": dense, "mixed_precision": mixed, "index_slices": shard,
            "stages_ms_per_step": {k: v / args.steps for k, v in sorted(stage_ms.items())},
            "stages_source": "timed graph replays: GPU global timer read by one-thread kernels at the stage "
                             "boundaries inside the graph, summed over the steps",
            "stages_ms_direct_launch": stages_direct}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _leg(fn, *args):
    """Run one side leg and return its record with the device memory it
    peaked at; what it allocated is released before the next one."""
    import gc
    import torch
    torch.cuda.reset_peak_memory_stats()
    out = fn(*args)
    gc.collect()
    torch.cuda.empty_cache()
    if isinstance(out, dict):
        out["peak_device_gb"] = torch.cuda.max_memory_allocated() / 2 ** 30
    return out


def verify_solution(d, e, W, Z, seed: int = 0) -> dict:
    """Accuracy of one solved problem against the goals (Sec. 2.3, Eqs.
    Tresnorm and Torthogo), from properties that hold at any size, computed
    on the GPU: W ascending, every residual ||T z - lambda z|| <= 20 n eps ||T||,
    |Z^T Z - I| <= 20 n eps over all columns against 1,024 seeded columns and
    over each column's 256 neighbours on each side, and the trace identity
    sum lambda = sum d within n * 4 n eps ||T||.  ||T|| = max|lambda|.
    Returns the worst ratios to the bounds (<= 1 passes)."""
    import torch
    eps = 2.0 ** -53
    n = d.numel()
    tn = float(W.abs().max())
    asc = bool((W[1:] >= W[:-1]).all()) if n > 1 else True
    res = 0.0
    for a in range(0, n, 4096):
        Zc = Z[:, a:a + 4096]
        TZ = d[:, None] * Zc
        TZ[:-1] += e[:n - 1, None] * Zc[1:]
        TZ[1:] += e[:n - 1, None] * Zc[:-1]
        res = max(res, float(torch.linalg.vector_norm(TZ - Zc * W[None, a:a + 4096], dim=0).max()))
        del TZ
    cols = torch.as_tensor(np.random.default_rng(seed).choice(n, min(n, 1024), replace=False), device=Z.device)
    G = Z.t() @ Z[:, cols]
    G[cols, torch.arange(cols.numel(), device=Z.device)] -= 1.0
    orth = float(G.abs().max())
    del G
    for a in range(0, n, 2048):
        b = min(n, a + 2048)
        lo, hi = max(0, a - 256), min(n, b + 256)
        G = Z[:, a:b].t() @ Z[:, lo:hi]
        idx = torch.arange(a, b, device=Z.device)
        G[idx - a, idx - lo] -= 1.0
        orth = max(orth, float(G.abs().max()))
        del G
    trace = abs(float(W.sum()) - float(d.sum()))
    return {"ascending": asc, "residual": res / (20 * n * eps * tn), "orthogonality": orth / (20 * n * eps),
            "trace": trace / (4 * n * n * eps * tn)}


def _time_cuda(fn, reps: int, flush) -> float:
    """Mean milliseconds of fn() over reps runs (CUDA events, L2 flushed before each)."""
    import torch
    total = 0.0
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / reps


def large_legs(dev, flush):
    """The largest single-GPU configuration: n = 50,000, d iid U[0,1], e iid
    U[0, 1e-2] (seed 50000; Z = 20 GB in HBM), all eigenpairs and separately
    the index subset 25001..30000, each timed with CUDA events (mean of two
    solves after a checked warm-up), against T_roof = max(143 n k / P_fp64,
    8 n k / BW)."""
    import torch
    from paper_1205_2107_gb300 import api
    d, e = inputs.large_uniform()
    n = len(d)
    dt = torch.tensor(d, device=dev)
    et = torch.tensor(np.append(e, 0.0), device=dev)
    out = {}
    for name, il, iu in (("all", 1, n), ("subset_25001_30000", 25001, 30000)):
        plan = api.Plan(dev, use_graph=1)
        k = iu - il + 1
        api.eigh_tridiagonal(dt, et, il, iu, plan=plan)  # checked: sizes the plan's capacities
        torch.cuda.synchronize()

        def one():
            api.eigh_tridiagonal(dt, et, il, iu, plan=plan, check=False)

        ms = _time_cuda(one, 2, flush)
        if plan.info()["status"] != 0:
            raise SystemExit(f"n=50000 {name}: solver reported an error")
        nk = n * k
        t_roof = max(PATH_FLOPS_PER_ROW * nk / (FP64_PEAK_GFLOPS * 1e9), 8.0 * nk / (HBM_GBS * 1e9))
        out[name] = {"n": n, "il": il, "iu": iu, "eigenpairs": k, "ms": ms, "eigenpairs_per_s": k / (ms * 1e-3),
                     "path_roofline_frac": 1e3 * t_roof / ms, "timing": "CUDA graph replay, CUDA events"}
        del plan
        torch.cuda.empty_cache()
    return out


def _sampled_accuracy(A, W, Y, seed=0, ncols=256):
    """Residual max ||A y - lambda y|| / (n eps ||A||) and orthogonality
    max |Y^T Y_s - I_s| / (n eps) over a seeded sample of columns (the
    dense problem's accuracy goals, checked at any size)."""
    import torch
    eps = 2.0 ** -53
    n = A.shape[0]
    k = W.numel()
    cols = torch.as_tensor(np.sort(np.random.default_rng(seed).choice(k, min(k, ncols), replace=False)),
                           device=A.device)
    Ys = Y[:, cols]
    nrm = float(W.abs().max())
    res = float(torch.linalg.vector_norm(A @ Ys - Ys * W[cols][None, :], dim=0).max())
    G = Y.t() @ Ys
    G[cols, torch.arange(cols.numel(), device=A.device)] -= 1.0
    return {"residual": res / (n * eps * nrm), "orthogonality": float(G.abs().max()) / (n * eps)}


def dense_legs(dev, flush):
    """The dense stages around the tridiagonal solver (paper Sec. 1.2) on
    one GPU, n = 8000: the standard problem A y = lambda y (stage 3
    reduction, stage 4 MRRR, stage 5 backtransformation) and the generalized
    A x = lambda B x (adding stage 1 Cholesky, stage 2 reduction, stage 6
    backtransformation); A symmetric with N(0,1) entries (seed 8000),
    B = G G^T + n I.  Each stage timed with CUDA events (mean of two after a
    warm-up), against its bound: the reduction's symmetric products on the
    FP64 FMA pipe and its rank-2k updates on the FP64 MMA, every other
    stage a GEMM-shaped contraction on the FP64 MMA."""
    import torch
    from paper_1205_2107_gb300 import api
    n = 8000
    rng = np.random.default_rng(8000)
    X = rng.standard_normal((n, n))
    A = torch.tensor((X + X.T) / 2, device=dev)
    G = rng.standard_normal((n, n))
    B = torch.tensor(G @ G.T + n * np.eye(n), device=dev)
    del X, G
    plan = api.Plan(dev)
    fma_peak, mma_peak = PEAKS["dfma"], PEAKS["dmma"] or PEAKS["dfma"]
    W, Y = api.eigh_dense(A, plan=plan)
    acc = _sampled_accuracy(A, W, Y)
    d, e, tau, R = api.tridiagonalize(A, plan=plan)
    eo = torch.cat([e, e.new_zeros(1)])
    t_trd = _time_cuda(lambda: api.tridiagonalize(A, plan=plan, check=False), 2, flush)
    t_step = _time_cuda(lambda: api.eigh_tridiagonal(d, eo, plan=plan, check=False), 2, flush)
    Z = api.eigh_tridiagonal(d, eo, plan=plan)[1]
    t_orm = _time_cuda(lambda: api.apply_q(R, tau, Z, plan=plan), 2, flush)
    t_all = _time_cuda(lambda: api.eigh_dense(A, plan=plan, check=False), 2, flush)
    f_half = 2.0 / 3.0 * n ** 3
    trd_roof = 1e3 * (f_half / fma_peak + f_half / mma_peak)
    standard = {
        "workload": "dense symmetric n=8000, N(0,1) entries (seed 8000), all eigenpairs",
        "ms": t_all, "eigenpairs_per_s": n / (t_all * 1e-3),
        "stages_ms": {"reduction": t_trd, "tridiagonal_mrrr": t_step, "backtransformation": t_orm},
        "roofline": {"reduction_frac": trd_roof / t_trd,
                     "backtransformation_tflops": 2.0 * n ** 3 / (t_orm * 1e-3) / 1e12,
                     "backtransformation_frac": 2.0 * n ** 3 / (t_orm * 1e-3) / mma_peak,
                     "model": "reduction 4/3 n^3 flops (half on the FP64 FMA pipe, half on the FP64 MMA), "
                              "backtransformation 2 n^2 k on the FP64 MMA"},
        "accuracy_sampled": acc}
    del R, Z, Y
    Wg, Xg = api.eigh_generalized(A, B, plan=plan)
    Bx = B @ Xg[:, :256]
    gacc = {"b_orthogonality": float((Xg.t() @ Bx - torch.eye(n, 256, dtype=torch.float64, device=dev)).abs().max())
            / (n * 2.0 ** -53)}
    del Bx, Xg
    t_chol = _time_cuda(lambda: api.cholesky(B, plan=plan), 2, flush)
    t_gen = _time_cuda(lambda: api.eigh_generalized(A, B, plan=plan, check=False), 2, flush)
    generalized = {
        "workload": "generalized A x = lambda B x, n=8000, A as above, B = G G^T + n I (G N(0,1)), all eigenpairs",
        "ms": t_gen, "eigenpairs_per_s": n / (t_gen * 1e-3),
        "stages_ms": {"cholesky": t_chol, "standard_problem": t_all,
                      "reduction_and_backtransformation": t_gen - t_chol - t_all},
        "roofline": {"cholesky_tflops": n ** 3 / 3.0 / (t_chol * 1e-3) / 1e12,
                     "cholesky_frac": n ** 3 / 3.0 / (t_chol * 1e-3) / mma_peak,
                     "stage2_and_6_frac": 3.0 * n ** 3 / ((t_gen - t_chol - t_all) * 1e-3) / mma_peak,
                     "model": "Cholesky n^3/3, L^-1 A L^-T 2 n^3 (two triangular solves), L^-T Y n^3"},
        "accuracy_sampled": gacc}
    del A, B
    torch.cuda.empty_cache()
    return {"standard_n8000": standard, "generalized_n8000": generalized}


def shard_leg(dev, flush, nslices=4):
    """Index-range sharding (paper Sec. 3.1.2) of the clustered n ~ 20,000
    matrices of the headline step: for each, the slices of nslices equal
    parts solved one after the other on this GPU, as nslices GPUs would
    solve them side by side; the time such a job would take is the slowest
    slice (no data moves between slices), against one GPU solving the whole
    matrix.  Clusters that cross a slice boundary are computed whole by both
    neighbouring slices (W+'s pairs, glued W21+'s groups of up to 1,904
    equal eigenvalues, which grow the margin).  Columns of neighbouring
    slices are checked for orthogonality across each boundary."""
    import torch
    from paper_1205_2107_gb300 import api
    out = {}
    for name, d, e in workload_matrices():
        n = len(d)
        dt = torch.tensor(d, device=dev)
        et = torch.tensor(np.append(e, 0.0), device=dev)
        plan = api.Plan(dev)
        api.eigh_tridiagonal(dt, et, plan=plan)
        t_full = _time_cuda(lambda: api.eigh_tridiagonal(dt, et, plan=plan, check=False), 1, flush)
        del plan
        torch.cuda.empty_cache()
        times, edges, margins, stages = [], [], [], []
        prev = None
        for sl in range(nslices):
            splan = api.Plan(dev)
            W, Z, (a, b) = api.eigh_tridiagonal_slice(dt, et, 1, n, nslices, sl, plan=splan)
            # the margin the checked call settled on: grow until the status is clean
            m = 32
            while True:
                api.eigh_tridiagonal_slice(dt, et, 1, n, nslices, sl, margin=m, plan=splan, check=False)
                if splan.info()["status"] == 0 or m > n:
                    break
                m *= 4
            margins.append(m)
            splan.set_timing(True)
            times.append(_time_cuda(lambda: api.eigh_tridiagonal_slice(dt, et, 1, n, nslices, sl, margin=m,
                                                                      plan=splan, check=False), 1, flush))
            stages.append({k: round(v, 2) for k, v in splan.profile()["stages"].items() if v >= 0.05})
            if prev is not None:  # last 512 columns of the previous slice against the first 512 of this one
                G = prev.t() @ Z[:, :512]
                edges.append(float(G.abs().max()) / (n * 2.0 ** -53))
            prev = Z[:, -512:].clone()
            del W, Z, splan
            torch.cuda.empty_cache()
        out[name] = {"n": n, "slices": nslices, "full_ms": t_full, "slice_ms": times, "job_ms": max(times),
                     "speedup_over_one_gpu": t_full / max(times), "efficiency": t_full / max(times) / nslices,
                     "margins": margins, "boundary_orthogonality_n_eps": edges,
                     "slice_stages_ms": stages}
    out["note"] = "slices timed one after the other on one GPU; a job on as many GPUs takes the slowest slice"
    return out


def mixed_precision_leg(dev, flush):
    """The FP64 default (singletons bisected to 2^-36, then one
    Rayleigh-quotient correction: singleton_rq = 1) against singletons
    bisected to full accuracy (singleton_rq = -1) and against eigenvectors in
    double-double (vector_precision = 2), on the same tridiagonal:
    uniform random n=20000 (seed 1205), all eigenpairs; time and
    orthogonality (sampled: all columns against 1,024 seeded ones and a
    +-256 band)."""
    import torch
    from paper_1205_2107_gb300 import api
    d, e = inputs.uniform(20000, 1205)
    dt = torch.tensor(d, device=dev)
    et = torch.tensor(np.append(e, 0.0), device=dev)
    n = len(d)
    out = {}
    for name, opts in (("fp64_full_bisection", {"singleton_rq": -1}), ("fp64", {}),
                       ("double_double", {"vector_precision": 2})):
        plan = api.Plan(dev, **opts)
        W, Z = api.eigh_tridiagonal(dt, et, plan=plan)
        ms = _time_cuda(lambda: api.eigh_tridiagonal(dt, et, plan=plan, check=False), 2, flush)
        acc = verify_solution(dt, et, W, Z)
        out[name] = {"ms": ms, "eigenpairs_per_s": n / (ms * 1e-3),
                     "orthogonality_n_eps": acc["orthogonality"] * 20, "residual_n_eps": acc["residual"] * 20}
        del W, Z, plan
        torch.cuda.empty_cache()
    out["workload"] = "uniform random tridiagonal n=20000 (seed 1205), all eigenpairs"
    return out


def side_by_side(args, dev, flush):
    """The batched and adjoint workloads on the same GPU, next to the plain path:
    4096 problems with n log-uniform in [32, 2048] (one batched solve vs the
    plain solver looped over a sample of the same problems), and the backward
    pass of 256 problems of n = 512 (forward solve, then the adjoint)."""
    import torch
    from paper_1205_2107_gb300 import api
    sizes = [int(x) for x in inputs.batch_sizes()]
    d, e, off = inputs.batched_uniform(sizes)
    lay = api.BatchLayout(sizes, dev)
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    plan = api.Plan(dev)
    W = torch.empty(lay.k_total, dtype=torch.float64, device=dev)
    Z = torch.empty(lay.z_total, dtype=torch.float64, device=dev)

    def batched():
        api.eigh_tridiagonal_batched(dt, et, lay, plan=plan, check=False, out=(W, Z))

    # a checked solve first: it grows the plan's node table and representation
    # pool to what this batch needs (an unchecked solve that overflowed would
    # take the capacity fallback and time the wrong work)
    api.eigh_tridiagonal_batched(dt, et, lay, plan=plan, out=(W, Z))
    batched()
    torch.cuda.synchronize()
    t_direct = _time_cuda(batched, 2, flush)
    if plan.info()["status"] != 0:
        raise SystemExit("batched solve reported an error")
    # autotuned launch shape, then the solve captured into a CUDA graph and replayed
    tune = api.autotune_batched(dt, et, lay, plan=plan, out=(W, Z))
    gplan = api.Plan(dev, use_graph=1, engine_blocks_per_sm=tune["engine_blocks_per_sm"],
                     width_scale=tune["width_scale"], pool_rows=plan.options.get("pool_rows", 0),
                     max_nodes=plan.options.get("max_nodes", 0))

    def replay():
        api.eigh_tridiagonal_batched(dt, et, lay, plan=gplan, check=False, out=(W, Z))

    t_first = _time_cuda(replay, 1, flush)  # capture + instantiate + first replay
    if gplan.info()["status"] != 0:
        raise SystemExit("batched graph solve reported an error")
    t_b = _time_cuda(replay, 2, flush)
    launches_b = gplan.profile()["launches"]
    nk_b = sum(n * n for n in sizes)
    # plain solver looped over every 16th problem (same sizes mix), scaled to the batch
    sample = list(range(0, len(sizes), 16))
    pplan = api.Plan(dev)

    def plain_loop():
        for p in sample:
            api.eigh_tridiagonal(dt[off[p]:off[p + 1]], et[off[p]:off[p + 1]], plan=pplan, check=False)

    plain_loop()
    t_p = _time_cuda(plain_loop, 1, flush)
    n_sample = sum(sizes[p] for p in sample)
    batched_line = {
        "workload": "4096 STEPs, n log-uniform in [32, 2048] (seed 2107), d, e iid U[-1,1], all eigenpairs",
        "ms": t_b, "eigenpairs_per_s": sum(sizes) / (t_b * 1e-3), "matrices_per_s": len(sizes) / (t_b * 1e-3),
        "path_roofline_frac": 1e3 * PATH_FLOPS_PER_ROW * nk_b / (FP64_PEAK_GFLOPS * 1e9) / t_b,
        "timing": "CUDA graph replay (levels driven on the device), autotuned launch shape",
        "graph_launches": launches_b, "first_call_ms": t_first, "direct_launch_ms": t_direct,
        "autotune": tune,
        "plain_loop": {"problems": len(sample), "ms": t_p, "eigenpairs_per_s": n_sample / (t_p * 1e-3),
                       "matrices_per_s": len(sample) / (t_p * 1e-3)},
    }
    del W, Z
    # adjoint: 256 x n = 512, loss sum w_i lambda_i + sum (c_i^T z_i)^2
    da, ea, wa, Ca = inputs.adjoint_case()
    batch, n = da.shape
    alay = api.BatchLayout([n] * batch, dev)
    dA, eA = torch.tensor(da.reshape(-1), device=dev), torch.tensor(ea.reshape(-1), device=dev)
    aplan = api.Plan(dev)
    WA, ZA = api.eigh_tridiagonal_batched(dA, eA, alay, plan=aplan)
    WA, ZA = WA[:alay.k_total], ZA[:alay.z_total]
    Ct = torch.tensor(Ca, device=dev).transpose(1, 2)
    proj = (Ct * ZA.view(batch, n, n)).sum(2)
    Zbar = (2.0 * Ct * proj[:, :, None]).reshape(-1)
    Wbar = torch.tensor(wa.reshape(-1), device=dev)

    def forward():
        api.eigh_tridiagonal_batched(dA, eA, alay, plan=aplan, check=False, out=(WA, ZA))

    def backward():
        api.eigh_tridiagonal_backward(WA, ZA, Wbar, Zbar, alay, plan=aplan, check=False)

    backward()
    torch.cuda.synchronize()
    t_f = _time_cuda(forward, 2, flush)
    t_bw = _time_cuda(backward, 3, flush)
    flops_bw = 4.0 * n ** 3 * batch
    adjoint_line = {
        "workload": "256 STEPs n=512, d, e iid N(0,1) (seed 1206); loss sum w_i lambda_i + sum (c_i^T z_i)^2",
        "forward_ms": t_f, "backward_ms": t_bw, "backward_over_forward": t_bw / t_f,
        "backward_tflops": flops_bw / (t_bw * 1e-3) / 1e12,
        "backward_frac": flops_bw / (t_bw * 1e-3) / max(PEAKS["dfma"], PEAKS["dmma"] or 0.0),
        "fp64_peaks_tflops": {"dfma": PEAKS["dfma"] / 1e12,
                              "dmma": PEAKS["dmma"] / 1e12 if PEAKS["dmma"] else None},
        "peak_source": "the better of the measured FP64 FMA and FP64 MMA rates (mrrr_probe_peak)",
    }
    return {"batched": batched_line, "adjoint": adjoint_line}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target length of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the batched and adjoint side-by-side legs")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
