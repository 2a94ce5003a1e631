"""Python API over the C ABI: plans, workspaces and the solver calls.

PyTorch supplies device memory and the current CUDA stream; every step of the
solve runs in the CUDA library (libmrrr.so).  Inputs must be float64 CUDA
tensors; there is no CPU path.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_F64 = torch.float64

# Default gap threshold of the backward pass, relative to max|W| (the
# spectral norm of T): eigenvalue pairs closer than 64 eps ||T|| cannot be
# told apart by any FP64 solver, so their term F(i, j) = 1/(W_j - W_i) is
# dropped instead of amplifying rounding errors by 1/gap.
DEFAULT_TAU_REL = 64.0 * 2.0 ** -53


def _stream_handle(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


def _check_input(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != _F64:
        raise TypeError(f"{name} must be float64")
    return x.contiguous()


class Plan:
    """A solver plan (options + reusable device workspace) on one GPU.

    Options are the fields of ``mrrr_options`` (gap_tol, classify_rtol,
    max_depth, max_bisect_steps, engine_blocks_per_sm, threads_per_block,
    vec_blocks_per_sm, use_graph, max_nodes, pool_rows, cluster_rtol,
    root_perturb, width_scale, prebisect_rtol, multisection_width, root_side,
    vector_precision, singleton_rq); zero or absent means default, and a
    value out of range raises (MRRR_ERR_ARG) when the plan is created.  With
    ``use_graph=1`` a solve is captured once per call signature into a CUDA
    graph and replayed.
    """

    def __init__(self, device: torch.device | int | None = None, **options):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   (device if isinstance(device, int) else device.index or 0))
        self.options = dict(options)
        self._h = None
        self._ws = None
        self._create()

    def _create(self) -> None:
        lib = _lib.load()
        o = _lib.Options()
        lib.mrrr_options_default(ctypes.byref(o))
        for k, val in self.options.items():
            if not hasattr(o, k):
                raise ValueError(f"unknown option {k}")
            setattr(o, k, val)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(lib.mrrr_plan_create(ctypes.byref(h), ctypes.byref(o)), "mrrr_plan_create")
        self._h = h
        if getattr(self, "_timing", False):
            lib.mrrr_set_timing(h, 1)

    def _destroy(self) -> None:
        if self._h is not None and self._h.value:
            _lib.load().mrrr_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self._destroy()
        except Exception:
            pass

    def set_options(self, **options) -> None:
        self.options.update(options)
        self._destroy()
        self._create()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def workspace_size(self, batch: int, n_total: int, k_total: int, n_max: int) -> int:
        out = ctypes.c_size_t()
        _lib.check(_lib.load().mrrr_workspace_size(self._h, batch, n_total, k_total, n_max, ctypes.byref(out)),
                   "mrrr_workspace_size")
        return int(out.value)

    def workspace(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def set_timing(self, enable: bool) -> None:
        """Record CUDA events between the solver's stages (see profile())."""
        self._timing = bool(enable)
        _lib.load().mrrr_set_timing(self._h, int(enable))

    def profile(self) -> dict:
        """Kernel launches and per-stage milliseconds of the last solve."""
        prof = _lib.Profile()
        _lib.check(_lib.load().mrrr_get_profile(self._h, ctypes.byref(prof)), "mrrr_get_profile")
        return {"launches": int(prof.launches), "stages": prof.stages()}

    def info(self) -> dict:
        """Synchronise the current stream and return the last solve's status
        word and counters; raises MrrrError when the synchronisation or the
        status copy itself fails (ERR_CUDA, which the device never sets as a
        status: the fields are not written then)."""
        inf = _lib.Info()
        rc = _lib.load().mrrr_get_status(self._h, _stream_handle(self.device), ctypes.byref(inf))
        if rc == _lib.ERR_CUDA:
            raise _lib.MrrrError(rc, "mrrr_get_status")
        return inf.as_dict()


_default_plans: dict[int, Plan] = {}


def default_plan(device: torch.device | None = None) -> Plan:
    idx = torch.cuda.current_device() if device is None else (device.index or 0)
    if idx not in _default_plans:
        _default_plans[idx] = Plan(idx)
    return _default_plans[idx]


def _run_with_retry(plan: Plan, call, where: str, check: bool):
    """Run ``call(ws, ws_bytes)``; on a full node table or representation
    pool grow the plan's capacities to what the solve reported and rerun."""
    for attempt in range(4):
        ws_bytes = call.ws_bytes()
        ws = plan.workspace(ws_bytes)
        _lib.check(call(ws, ws_bytes), where)
        if not check:
            return None
        info = plan.info()
        st = info["status"]
        if st == _lib.ERR_MARGIN and hasattr(call, "grow_margin") and attempt < 3:
            call.grow_margin()
            continue
        if st == _lib.ERR_QUEUE and attempt < 3:
            need_rows = int(info["pool_rows_used"] * 2) + 1024
            need_nodes = int(max(info["nodes"], 16) * 2)
            plan.set_options(pool_rows=max(need_rows, plan.options.get("pool_rows", 0)),
                             max_nodes=max(need_nodes, plan.options.get("max_nodes", 0)))
            continue
        if st != _lib.OK:
            raise _lib.MrrrError(st, where)
        return info
    raise _lib.MrrrError(_lib.ERR_QUEUE, where)


class _SteinCall:
    def __init__(self, plan, n, d, e, il, iu, W, Zt):
        self.plan, self.n, self.d, self.e, self.il, self.iu, self.W, self.Zt = plan, n, d, e, il, iu, W, Zt

    def ws_bytes(self):
        return self.plan.workspace_size(1, self.n, self.iu - self.il + 1, self.n)

    def __call__(self, ws, ws_bytes):
        return _lib.load().mrrr_stein(self.plan.handle, self.n, _ptr(self.d), _ptr(self.e if self.n > 1 else self.d),
                                      self.il, self.iu, _ptr(self.W), _ptr(self.Zt), self.n, _ptr(ws), ws_bytes,
                                      _stream_handle(self.d.device))


def eigh_tridiagonal(d: torch.Tensor, e: torch.Tensor, il: int | None = None, iu: int | None = None, *,
                     vectors: bool = True, plan: Plan | None = None, check: bool = True):
    """Eigenpairs il..iu (1-based, inclusive; default all) of the symmetric
    tridiagonal matrix with diagonal d (n) and off-diagonal e (n-1).

    Returns (W, Z): W ascending (k,), Z (n, k) column-major (a transposed view
    of a contiguous (k, n) tensor), or W alone when ``vectors`` is False.
    With ``check`` the call synchronises and raises on device-side errors.
    """
    d = _check_input(d, "d")
    n = d.numel()
    e = _check_input(e, "e") if n > 1 else d
    if n > 1 and e.numel() < n - 1:
        raise ValueError("e needs n-1 entries")
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    if n == 0:
        W = torch.empty(0, dtype=_F64, device=d.device)
        return (W, torch.empty((0, 0), dtype=_F64, device=d.device)) if vectors else W
    if not (1 <= il <= iu <= n):
        raise ValueError("need 1 <= il <= iu <= n")
    k = iu - il + 1
    plan = plan or default_plan(d.device)
    W = torch.empty(k, dtype=_F64, device=d.device)
    Zt = torch.empty((k, n), dtype=_F64, device=d.device) if vectors else None
    _run_with_retry(plan, _SteinCall(plan, n, d, e, il, iu, W, Zt), "mrrr_stein", check)
    return (W, Zt.t()) if vectors else W


def slice_range(il: int, iu: int, nslices: int, slice_: int) -> tuple[int, int]:
    """Indices a..b (1-based, inclusive) of slice ``slice_`` of ``nslices``
    equal contiguous slices of il..iu (mrrr_slice_range; host only)."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _lib.check(_lib.load().mrrr_slice_range(int(il), int(iu), int(nslices), int(slice_), ctypes.byref(a),
                                            ctypes.byref(b)), "mrrr_slice_range")
    return int(a.value), int(b.value)


class _SliceCall:
    def __init__(self, plan, n, d, e, il, iu, nslices, slice_, margin, W, Zt):
        # explicit fields: no reference back to the call object itself, so it
        # (and the plan and tensors it holds) is freed as soon as it is dropped
        self.plan, self.n, self.d, self.e, self.il, self.iu = plan, n, d, e, il, iu
        self.nslices, self.slice_, self.margin, self.W, self.Zt = nslices, slice_, margin, W, Zt
        self.a, self.b = slice_range(il, iu, nslices, slice_)

    def grow_margin(self):
        self.margin *= 4

    def ws_bytes(self):
        lo, hi = max(1, self.a - self.margin), min(self.n, self.b + self.margin)
        return self.plan.workspace_size(1, self.n, hi - lo + 1, self.n)

    def __call__(self, ws, ws_bytes):
        return _lib.load().mrrr_stein_slice(
            self.plan.handle, self.n, _ptr(self.d), _ptr(self.e if self.n > 1 else self.d), self.il, self.iu,
            self.nslices, self.slice_, self.margin, _ptr(self.W), _ptr(self.Zt), self.n, _ptr(ws), ws_bytes,
            _stream_handle(self.d.device))


def eigh_tridiagonal_slice(d: torch.Tensor, e: torch.Tensor, il: int | None, iu: int | None, nslices: int,
                           slice_: int, *, margin: int = 32, vectors: bool = True, plan: Plan | None = None,
                           check: bool = True):
    """Eigenpairs of slice ``slice_`` of ``nslices`` equal slices of il..iu
    (mrrr_stein_slice): (W, Z, (a, b)) for the slice's indices a..b.  The
    slices of one range, solved separately (on different GPUs or one after
    the other), together form the solution of the range.  A cluster reaching
    past ``margin`` makes the call grow the margin fourfold and solve again
    (only when ``check``)."""
    d = _check_input(d, "d")
    n = d.numel()
    e = _check_input(e, "e") if n > 1 else d
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    if n == 0:
        W = torch.empty(0, dtype=_F64, device=d.device)
        return (W, torch.empty((0, 0), dtype=_F64, device=d.device), (1, 0)) if vectors else (W, (1, 0))
    a, b = slice_range(il, iu, nslices, slice_)
    k = b - a + 1
    plan = plan or default_plan(d.device)
    W = torch.empty(k, dtype=_F64, device=d.device)
    Zt = torch.empty((k, n), dtype=_F64, device=d.device) if vectors else None
    call = _SliceCall(plan, n, d, e, il, iu, nslices, slice_, int(margin), W, Zt)
    _run_with_retry(plan, call, "mrrr_stein_slice", check)
    return (W, Zt.t(), (a, b)) if vectors else (W, (a, b))


class _BatchedCall:
    def __init__(self, plan, batch, off, d, e, il, iu, W, w_off, Z, z_off, n_total, k_total, n_max):
        self.plan, self.batch, self.off, self.d, self.e, self.il, self.iu = plan, batch, off, d, e, il, iu
        self.W, self.w_off, self.Z, self.z_off = W, w_off, Z, z_off
        self.n_total, self.k_total, self.n_max = n_total, k_total, n_max

    def ws_bytes(self):
        return self.plan.workspace_size(self.batch, self.n_total, self.k_total, self.n_max)

    def __call__(self, ws, ws_bytes):
        return _lib.load().mrrr_stein_batched(
            self.plan.handle, self.batch, _ptr(self.off), _ptr(self.d), _ptr(self.e), _ptr(self.il), _ptr(self.iu),
            _ptr(self.W), _ptr(self.w_off), _ptr(self.Z), _ptr(self.z_off), self.n_total, self.k_total,
            self.n_max, _ptr(ws), ws_bytes, _stream_handle(self.d.device))


class BatchLayout:
    """Packing of a batch of problems: row offsets (d, e), W and Z offsets."""

    def __init__(self, sizes, device, il=None, iu=None):
        sizes = [int(s) for s in sizes]
        self.sizes = sizes
        self.batch = len(sizes)
        il = [1] * self.batch if il is None else [int(x) for x in il]
        iu = list(sizes) if iu is None else [int(x) for x in iu]
        if any(n < 0 for n in sizes):
            raise ValueError("problem sizes must be >= 0")
        if len(il) != self.batch or len(iu) != self.batch:
            raise ValueError("il and iu need one entry per problem")
        for p, (n, lo, hi) in enumerate(zip(sizes, il, iu)):
            if n > 0 and not 1 <= lo <= hi <= n:
                raise ValueError(f"problem {p}: need 1 <= il <= iu <= n (n={n}, il={lo}, iu={hi})")
        self.ks = [u - l + 1 if n > 0 else 0 for n, l, u in zip(sizes, il, iu)]
        off = [0]
        woff = [0]
        zoff = [0]
        for n, k in zip(sizes, self.ks):
            off.append(off[-1] + n)
            woff.append(woff[-1] + k)
            zoff.append(zoff[-1] + n * k)
        self.n_total, self.k_total, self.z_total = off[-1], woff[-1], zoff[-1]
        self.n_max = max(sizes) if sizes else 0
        self.offsets_host = off
        self.w_offsets_host = woff
        self.z_offsets_host = zoff
        self.offsets = torch.tensor(off, dtype=torch.int64, device=device)
        self.w_offsets = torch.tensor(woff, dtype=torch.int64, device=device)
        self.z_offsets = torch.tensor(zoff, dtype=torch.int64, device=device)
        self.all = il == [1] * self.batch and iu == list(sizes)
        self.il = None if self.all else torch.tensor(il, dtype=torch.int32, device=device)
        self.iu = None if self.all else torch.tensor(iu, dtype=torch.int32, device=device)

    def unpack(self, W, Z=None):
        Ws = [W[a:b] for a, b in zip(self.w_offsets_host[:-1], self.w_offsets_host[1:])]
        if Z is None:
            return Ws
        Zs = [Z[a:b].view(k, n).t() for a, b, n, k in zip(self.z_offsets_host[:-1], self.z_offsets_host[1:],
                                                          self.sizes, self.ks)]
        return Ws, Zs


def eigh_tridiagonal_batched(d: torch.Tensor, e: torch.Tensor, layout: BatchLayout, *, vectors: bool = True,
                             plan: Plan | None = None, check: bool = True, out=None):
    """Eigenpairs of a batch of problems packed by ``layout`` (see BatchLayout).

    d and e are packed with layout.offsets (e's last entry per problem is
    ignored).  Returns packed (W, Z): W[w_offsets[p]:...] ascending and Z's
    block of problem p column-major n_p x k_p at z_offsets[p].
    """
    d = _check_input(d, "d")
    e = _check_input(e, "e")
    if d.numel() < layout.n_total or e.numel() < layout.n_total:
        raise ValueError("d and e need n_total entries")
    plan = plan or default_plan(d.device)
    if out is None:
        W = torch.empty(max(layout.k_total, 1), dtype=_F64, device=d.device)
        Z = torch.empty(max(layout.z_total, 1), dtype=_F64, device=d.device) if vectors else None
    else:
        W, Z = out
    call = _BatchedCall(plan, layout.batch, layout.offsets, d, e, layout.il, layout.iu, W, layout.w_offsets,
                        Z, layout.z_offsets if vectors else None, layout.n_total, layout.k_total, layout.n_max)
    _run_with_retry(plan, call, "mrrr_stein_batched", check)
    return (W, Z) if vectors else W


def eigh_tridiagonal_backward(W: torch.Tensor, Z: torch.Tensor, Wbar: torch.Tensor | None,
                              Zbar: torch.Tensor | None, layout: BatchLayout, *,
                              tau_rel: float = DEFAULT_TAU_REL,
                              plan: Plan | None = None, check: bool = True):
    """Gradient (dbar, ebar) of a loss with respect to packed (d, e), given
    the packed all-eigenpair solution (W, Z) of ``layout`` and the loss
    gradients Wbar (like W) and Zbar (like Z); either may be None.

    dbar and ebar have the packing of d and e (ebar's last entry of each
    problem is 0).  F(i, j) = 1/(W_j - W_i) is dropped where the gap is at
    most tau_rel * max|W| of the problem (default 64 eps: numerically equal
    eigenvalues, whose individual vectors are not defined).
    """
    if not layout.all:
        raise ValueError("the backward pass needs all eigenpairs of every problem")
    W = _check_input(W, "W")
    Z = _check_input(Z, "Z")
    Wbar = _check_input(Wbar, "Wbar") if Wbar is not None else None
    Zbar = _check_input(Zbar, "Zbar") if Zbar is not None else None
    dev = W.device
    plan = plan or default_plan(dev)
    n_total = layout.n_total
    dbar = torch.empty(max(n_total, 1), dtype=_F64, device=dev)
    ebar = torch.empty(max(n_total, 1), dtype=_F64, device=dev)
    lib = _lib.load()
    nbytes = ctypes.c_size_t(0)
    _lib.check(lib.mrrr_backward_workspace_size(plan.handle, layout.batch, layout.z_total, ctypes.byref(nbytes)),
               "mrrr_backward_workspace_size")
    # own buffer: the solve's workspace keeps its status word for info()
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    rc = lib.mrrr_backward(plan.handle, layout.batch, _ptr(layout.offsets), _ptr(W), _ptr(Z), _ptr(Wbar),
                           _ptr(Zbar), float(tau_rel), layout.n_max, layout.z_total, _ptr(dbar), _ptr(ebar),
                           _ptr(ws), nbytes.value, _stream_handle(dev))
    _lib.check(rc, "mrrr_backward")
    if check:
        torch.cuda.synchronize(dev)
    return dbar[:n_total], ebar[:n_total]


def autotune_batched(d: torch.Tensor, e: torch.Tensor, layout: BatchLayout, *, plan: Plan | None = None,
                     out=None) -> dict:
    """Choose the batched solver's launch shape for this layout by timing
    the candidates (mrrr_autotune_batched); the choice stays on the plan.

    One checked solve runs first so that the plan's capacities fit the
    batch.  Returns the chosen engine_blocks_per_sm, width_scale and
    singleton_rq with the best and default times (ms).
    """
    d = _check_input(d, "d")
    e = _check_input(e, "e")
    plan = plan or default_plan(d.device)
    W, Z = eigh_tridiagonal_batched(d, e, layout, plan=plan, out=out)
    call = _BatchedCall(plan, layout.batch, layout.offsets, d, e, layout.il, layout.iu, W, layout.w_offsets, Z,
                        layout.z_offsets, layout.n_total, layout.k_total, layout.n_max)
    nbytes = call.ws_bytes()
    ws = plan.workspace(nbytes)
    t = _lib.Tuning()
    rc = _lib.load().mrrr_autotune_batched(
        plan.handle, layout.batch, _ptr(layout.offsets), _ptr(d), _ptr(e), _ptr(layout.il), _ptr(layout.iu),
        _ptr(W), _ptr(layout.w_offsets), _ptr(Z), _ptr(layout.z_offsets), layout.n_total, layout.k_total,
        layout.n_max, _ptr(ws), nbytes, _stream_handle(d.device), ctypes.byref(t))
    _lib.check(rc, "mrrr_autotune_batched")
    plan.options.update(engine_blocks_per_sm=int(t.engine_blocks_per_sm), width_scale=float(t.width_scale),
                        singleton_rq=int(t.singleton_rq))
    return {"engine_blocks_per_sm": int(t.engine_blocks_per_sm), "width_scale": float(t.width_scale),
            "singleton_rq": int(t.singleton_rq), "best_ms": float(t.best_ms), "default_ms": float(t.default_ms),
            "configs": int(t.configs)}


PEAK_KINDS = {"dfma": 0, "dmma": 1, "ddiv": 2, "ffma": 3, "dfma_one_lane": 4, "dfma_latency": 5,
              "ddiv_latency": 6}


def probe_peak(kind: str) -> float:
    """Measured peak rate of one unit of the current GPU (mrrr_probe_peak):
    'dfma' and 'dmma' in FP64 flop/s, 'ddiv' in divisions/s, 'ffma' in FP32
    flop/s, 'dfma_one_lane' in FP64 FMA warp instructions/s with one active
    lane per warp; 'dfma_latency' and 'ddiv_latency' in SM cycles per
    dependent step."""
    rate = ctypes.c_double(0.0)
    _lib.check(_lib.load().mrrr_probe_peak(PEAK_KINDS[kind], ctypes.byref(rate)), "mrrr_probe_peak")
    return float(rate.value)


# ---------------------------------------------------------------------------
# Dense symmetric eigenproblem (the paper's stages 3-5 around the tridiagonal
# solver).  A symmetric matrix is its own transpose, so a contiguous (n, n)
# tensor is passed as the column-major matrix itself.

def _dense_ws(plan: Plan, n: int, k: int) -> tuple[torch.Tensor, int]:
    nbytes = ctypes.c_size_t(0)
    _lib.check(_lib.load().mrrr_dense_workspace_size(plan.handle, n, k, ctypes.byref(nbytes)),
               "mrrr_dense_workspace_size")
    return plan.workspace(nbytes.value), int(nbytes.value)


def _dense_check(plan: Plan, ws: torch.Tensor, where: str, device) -> None:
    rc = _lib.load().mrrr_dense_status(_ptr(ws), _stream_handle(device))
    if rc != _lib.OK:
        raise _lib.MrrrError(rc, where)


def tridiagonalize(A: torch.Tensor, *, plan: Plan | None = None, check: bool = True):
    """Stage 3 (mrrr_sytrd): (d, e, tau, R) with T = tridiag(e, d, e) =
    Q^T A Q; R is A overwritten by the reflectors (below its subdiagonal),
    which apply_q reads."""
    A = _check_input(A, "A")
    n = A.shape[0]
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    R = A.clone()
    plan = plan or default_plan(A.device)
    d = torch.empty(max(n, 1), dtype=_F64, device=A.device)
    e = torch.empty(max(n - 1, 1), dtype=_F64, device=A.device)
    tau = torch.empty(max(n - 2, 1), dtype=_F64, device=A.device)
    ws, nbytes = _dense_ws(plan, n, 0)
    _lib.check(_lib.load().mrrr_sytrd(plan.handle, n, _ptr(R), n, _ptr(d), _ptr(e), _ptr(tau), _ptr(ws), nbytes,
                                      _stream_handle(A.device)), "mrrr_sytrd")
    if check:
        _dense_check(plan, ws, "mrrr_sytrd", A.device)
    return d[:n], e[:max(n - 1, 0)], tau[:max(n - 2, 0)], R


def apply_q(R: torch.Tensor, tau: torch.Tensor, Y: torch.Tensor, *, plan: Plan | None = None) -> torch.Tensor:
    """Stage 5 (mrrr_ormtr): Q Y for the Q of tridiagonalize; Y is (n, k)
    and is returned as a new column-major (n, k) view."""
    R = _check_input(R, "R")
    n = R.shape[0]
    k = Y.shape[1]
    plan = plan or default_plan(R.device)
    Yt = _check_input(Y, "Y").t().contiguous()  # (k, n) row-major = column-major Y
    ws, nbytes = _dense_ws(plan, n, min(k, n))
    _lib.check(_lib.load().mrrr_ormtr(plan.handle, n, k, _ptr(R), n, _ptr(tau), _ptr(Yt), n, _ptr(ws), nbytes,
                                      _stream_handle(R.device)), "mrrr_ormtr")
    return Yt.t()


def eigh_dense(A: torch.Tensor, il: int | None = None, iu: int | None = None, *, vectors: bool = True,
               plan: Plan | None = None, check: bool = True):
    """Eigenpairs il..iu (1-based, inclusive; default all) of the symmetric A
    (mrrr_dense_eigh: reduction, tridiagonal MRRR, backtransformation).
    Returns (W, Y) with Y (n, k) column-major, or W alone."""
    A = _check_input(A, "A")
    n = A.shape[0]
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    if n == 0:
        W = torch.empty(0, dtype=_F64, device=A.device)
        return (W, torch.empty((0, 0), dtype=_F64, device=A.device)) if vectors else W
    if not 1 <= il <= iu <= n:
        raise ValueError("need 1 <= il <= iu <= n")
    k = iu - il + 1
    plan = plan or default_plan(A.device)
    R = A.clone()
    W = torch.empty(k, dtype=_F64, device=A.device)
    Yt = torch.empty((k, n), dtype=_F64, device=A.device) if vectors else None
    for attempt in range(4):
        ws, nbytes = _dense_ws(plan, n, k)
        R.copy_(A)
        _lib.check(_lib.load().mrrr_dense_eigh(plan.handle, n, _ptr(R), n, il, iu, _ptr(W), _ptr(Yt), n, _ptr(ws),
                                               nbytes, _stream_handle(A.device)), "mrrr_dense_eigh")
        if not check:
            break
        _dense_check(plan, ws, "mrrr_dense_eigh", A.device)
        info = plan.info()
        if info["status"] == _lib.ERR_QUEUE and attempt < 3:
            plan.set_options(pool_rows=max(int(info["pool_rows_used"] * 2) + 1024, plan.options.get("pool_rows", 0)),
                             max_nodes=max(int(max(info["nodes"], 16) * 2), plan.options.get("max_nodes", 0)))
            continue
        if info["status"] != _lib.OK:
            raise _lib.MrrrError(info["status"], "mrrr_dense_eigh")
        break
    return (W, Yt.t()) if vectors else W


# ---------------------------------------------------------------------------
# Generalized symmetric-definite eigenproblem A x = lambda B x (the paper's
# six stages).

def _gen_ws(plan: Plan, n: int, k: int) -> tuple[torch.Tensor, int]:
    nbytes = ctypes.c_size_t(0)
    _lib.check(_lib.load().mrrr_gen_workspace_size(plan.handle, n, k, ctypes.byref(nbytes)),
               "mrrr_gen_workspace_size")
    return plan.workspace(nbytes.value), int(nbytes.value)


def cholesky(B: torch.Tensor, *, plan: Plan | None = None) -> torch.Tensor:
    """Stage 1 (mrrr_potrf): the lower-triangular L with L L^T = B."""
    B = _check_input(B, "B")
    n = B.shape[0]
    plan = plan or default_plan(B.device)
    Lt = B.clone()  # column-major storage of B (symmetric)
    ws, nbytes = _gen_ws(plan, n, 0)
    _lib.check(_lib.load().mrrr_potrf(plan.handle, n, _ptr(Lt), n, _ptr(ws), nbytes, _stream_handle(B.device)),
               "mrrr_potrf")
    rc = _lib.load().mrrr_dense_status(_ptr(ws), _stream_handle(B.device))
    if rc != _lib.OK:
        raise _lib.MrrrError(rc, "mrrr_potrf")
    return torch.tril(Lt.t())  # the column-major lower factor, as a row-major (n, n) tensor


def eigh_generalized(A: torch.Tensor, B: torch.Tensor, il: int | None = None, iu: int | None = None, *,
                     vectors: bool = True, plan: Plan | None = None, check: bool = True):
    """Eigenpairs il..iu of A x = lambda B x (A symmetric, B symmetric
    positive definite; mrrr_gen_eigh): (W, X) with X^T B X = I, X (n, k)
    column-major, or W alone."""
    A = _check_input(A, "A")
    B = _check_input(B, "B")
    n = A.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    if n == 0:
        W = torch.empty(0, dtype=_F64, device=A.device)
        return (W, torch.empty((0, 0), dtype=_F64, device=A.device)) if vectors else W
    if not 1 <= il <= iu <= n:
        raise ValueError("need 1 <= il <= iu <= n")
    k = iu - il + 1
    plan = plan or default_plan(A.device)
    W = torch.empty(k, dtype=_F64, device=A.device)
    Xt = torch.empty((k, n), dtype=_F64, device=A.device) if vectors else None
    for attempt in range(4):
        Ac, Bc = A.clone(), B.clone()
        ws, nbytes = _gen_ws(plan, n, k)
        _lib.check(_lib.load().mrrr_gen_eigh(plan.handle, n, _ptr(Ac), n, _ptr(Bc), n, il, iu, _ptr(W), _ptr(Xt), n,
                                             _ptr(ws), nbytes, _stream_handle(A.device)), "mrrr_gen_eigh")
        if not check:
            break
        rc = _lib.load().mrrr_gen_status(plan.handle, n, k, _ptr(ws), _stream_handle(A.device))
        if rc != _lib.OK:
            raise _lib.MrrrError(rc, "mrrr_gen_eigh")
        info = plan.info()
        if info["status"] == _lib.ERR_QUEUE and attempt < 3:
            plan.set_options(pool_rows=max(int(info["pool_rows_used"] * 2) + 1024, plan.options.get("pool_rows", 0)),
                             max_nodes=max(int(max(info["nodes"], 16) * 2), plan.options.get("max_nodes", 0)))
            continue
        if info["status"] != _lib.OK:
            raise _lib.MrrrError(info["status"], "mrrr_gen_eigh")
        break
    return (W, Xt.t()) if vectors else W
