// mrrr_api.cu -- the C ABI (include/mrrr.h): plans, workspace layout and the
// launch sequence of a solve.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "mrrr_launch.h"

// Everything a captured solve depends on: a replay is valid only for the
// same arguments, workspace and options.
struct GraphKey {
  mrrr::ProblemArgs a;
  const void *d, *e, *ws;
  void *W, *Z;
  int64_t n_total, k_total;
  int n_max;
  size_t ws_bytes;
  int64_t opt_version;
};

// Field by field: the structs have padding, whose bytes are not part of
// the key.
static bool same_key(const GraphKey& x, const GraphKey& y) {
  const mrrr::ProblemArgs &a = x.a, &b = y.a;
  return a.batch == b.batch && a.d_off == b.d_off && a.il == b.il && a.iu == b.iu && a.w_off == b.w_off &&
         a.z_off == b.z_off && a.n == b.n && a.il1 == b.il1 && a.iu1 == b.iu1 && a.ldz == b.ldz &&
         a.slice == b.slice && a.ol1 == b.ol1 && a.ou1 == b.ou1 && x.d == y.d &&
         x.e == y.e && x.ws == y.ws && x.W == y.W && x.Z == y.Z && x.n_total == y.n_total &&
         x.k_total == y.k_total && x.n_max == y.n_max && x.ws_bytes == y.ws_bytes && x.opt_version == y.opt_version;
}

struct mrrr_plan {
  mrrr_options opt;
  int device;
  int nsm;
  mrrr::Ctl* host_ctl;  // pinned, for the per-level count and the status
  void* last_ws;        // workspace of the last solve (for mrrr_get_status)
  mrrr::StageTimer timer;
  int64_t opt_version;  // bumped when the autotuner changes the options
  // CUDA graph of the last solve signature (use_graph)
  cudaStream_t cap_stream;
  cudaGraphExec_t exec;
  GraphKey key;
  bool have_graph;
  bool graph_conditional;  // the graph runs its levels in a conditional while node
  bool last_graph;         // the last solve was a graph replay (device-clock stage times)
  int64_t graph_launches;
  int64_t graph_part_launches[3];  // conditional graph: kernels before, per level, after the loop
};

namespace mrrr {

namespace {
thread_local StageTimer* g_timer = nullptr;
}

StageTimer* stage_timer() { return g_timer; }
void set_stage_timer(StageTimer* t) { g_timer = t; }

const char* const kStageNames[ST_COUNT] = {"prep",     "root",     "bisect_root", "rank",         "classify",
                                           "prerefine", "childrep", "refine",      "final_bisect", "vectors"};

int stage_index(const char* name) {
  for (int i = 0; i < ST_COUNT; ++i)
    if (std::strcmp(kStageNames[i], name) == 0) return i;
  return -1;
}

namespace {
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-clock stage mark: the time since the previous mark goes to stage id
// (id < 0: only the reference point is set).
__global__ void k_stage_mark(Ctl* c, int id) {
  const unsigned long long t = global_ns();
  if (id >= 0) c->stage_ns[id] += t - c->t_last;
  c->t_last = t;
}
}  // namespace

void StageTimer::begin(cudaStream_t s) {
  count = 0;
  launches = 0;
  nstages = 0;
  mark("start", s);
}

void StageTimer::mark(const char* what, cudaStream_t s) {
  if (device) {
    if (dev_ctl) {
      k_stage_mark<<<1, 1, 0, s>>>(dev_ctl, stage_index(what));
      ++launches;
    }
    return;
  }
  if (!on || count >= 256) return;
  if (!ev_ready) {
    for (int i = 0; i < 256; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
        return;
      }
    ev_ready = true;
  }
  name[count] = what;
  cudaEventRecord(ev[count], s);
  ++count;
}

void StageTimer::release() {
  if (ev_ready)
    for (int i = 0; i < 256; ++i) cudaEventDestroy(ev[i]);
  ev_ready = false;
}

void StageTimer::finish() {
  nstages = 0;
  if (device) {
    count = 0;
    return;
  }
  if (!on || count < 2) {
    count = 0;
    return;
  }
  cudaEventSynchronize(ev[count - 1]);
  const char* env = std::getenv("MRRR_TIMING");
  const bool each = env && std::strcmp(env, "2") == 0;  // every stage in launch order
  for (int i = 1; i < count; ++i) {
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[i - 1], ev[i]);
    if (each) std::fprintf(stderr, "[mrrr stage %3d] %-18s %10.3f ms\n", i, name[i], t);
    int k = 0;
    while (k < nstages && std::strcmp(stage_name[k], name[i]) != 0) ++k;
    if (k == nstages) {
      if (nstages >= 32) continue;
      stage_name[nstages] = name[i];
      stage_ms[nstages++] = 0.0;
    }
    stage_ms[k] += t;
  }
  if (std::getenv("MRRR_TIMING"))
    for (int k = 0; k < nstages; ++k) std::fprintf(stderr, "[mrrr timing] %-18s %10.3f ms\n", stage_name[k], stage_ms[k]);
  count = 0;
}

namespace {

constexpr size_t kAlign = 256;
constexpr int kSliceWidth = 4;  // multisection width of slice calls unless the options fix one

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t ctl, prob, blk, node, pool_dl, pool_ul, ilist, lwin, rgrid, sched_cnt, sched_claim, lo, hi, gap, wval, znrm2,
      snode, sj, spos, state, bflag, vscr;
  size_t total;
  int64_t max_blocks, max_nodes, max_slots, pool_rows, vscr_threads, vscr_rows;
};

// Threads of the eigenvector kernel (persistent; one vector at a time per
// thread): c CTAs of 128 on every SM -- the same number on each, so that
// every SM sub-partition holds c warps and the scheduler's ranks spread the
// 32-vector chunks evenly -- with c the number of chunk waves over the
// 4 nsm sub-partitions, at most vec_blocks_per_sm, and at most what fits in
// 32 GB of scratch (each thread owns 2 n_max doubles, 4 in double-double),
// but at least one.
int64_t vec_threads(const mrrr_plan* p, int64_t max_slots, int n_max) {
  const int64_t per_wave = (int64_t)p->nsm * 128;  // one warp per sub-partition
  const int64_t waves = (max_slots + per_wave - 1) / per_wave;
  const int64_t row_bytes = p->opt.vector_precision == 2 ? 32 : 16;  // scratch per row and thread
  const int64_t mem_c = ((int64_t)32 << 30) / (row_bytes * (int64_t)std::max(n_max, 1)) / per_wave;
  // at most 4: the eigenvector kernel runs 4 CTAs of 128 threads per SM
  const int64_t c = std::max<int64_t>(
      1, std::min<int64_t>({waves, (int64_t)std::min(4, std::max(1, p->opt.vec_blocks_per_sm)), mem_c}));
  return per_wave * c;
}

Layout make_layout(const mrrr_plan* p, int batch, int64_t n_total, int64_t k_total, int n_max) {
  Layout L{};
  const mrrr_options& o = p->opt;
  L.max_blocks = std::max<int64_t>(n_total, 1);
  L.max_slots = n_total + 2 * (int64_t)batch + 1;
  int64_t child_nodes = o.max_nodes > 0 ? o.max_nodes : std::max<int64_t>(k_total, 16);
  L.max_nodes = std::min<int64_t>(L.max_blocks + child_nodes, INT32_MAX - 1);
  int64_t pool_child = o.pool_rows;
  if (pool_child <= 0) {
    // automatic: room for many full-size child representations; a solve that
    // needs more reports MRRR_ERR_QUEUE and the needed rows in mrrr_info
    int64_t want = (std::max<int64_t>(k_total, 1) + 1) * std::max<int64_t>(n_max, 1);
    int64_t cap = std::max<int64_t>(256 * n_total, (int64_t)1 << 28);
    pool_child = std::min(want, cap);
  }
  L.pool_rows = n_total + pool_child;
  L.vscr_threads = vec_threads(p, L.max_slots, n_max);
  L.vscr_rows = std::max(n_max, 1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return at;
  };
  L.ctl = take(sizeof(Ctl));
  L.prob = take(sizeof(Problem) * (size_t)std::max(batch, 1));
  L.blk = take(sizeof(Block) * (size_t)L.max_blocks);
  L.node = take(sizeof(Node) * (size_t)L.max_nodes);
  L.pool_dl = take(sizeof(double2) * (size_t)L.pool_rows);
  L.pool_ul = take(sizeof(double2) * (size_t)L.pool_rows);
  L.ilist = take(sizeof(int64_t) * (size_t)L.max_slots);
  L.lwin = take(sizeof(int64_t) * 2 * (size_t)((L.max_slots + 31) / 32));
  L.rgrid = take(sizeof(int) * 2 * (size_t)std::max<int64_t>(n_total, 1));
  L.sched_cnt = take(sizeof(int) * (size_t)kSchedSlots);
  L.sched_claim = take(sizeof(int) * (size_t)L.max_slots);

  L.lo = take(sizeof(double) * (size_t)L.max_slots);
  L.hi = take(sizeof(double) * (size_t)L.max_slots);
  L.gap = take(sizeof(double) * (size_t)L.max_slots);
  L.wval = take(sizeof(double) * (size_t)L.max_slots);
  L.znrm2 = take(sizeof(double) * (size_t)L.max_slots);
  L.snode = take(sizeof(int) * (size_t)L.max_slots);
  L.sj = take(sizeof(int) * (size_t)L.max_slots);
  L.spos = take(sizeof(int) * (size_t)L.max_slots);
  L.state = take(sizeof(int) * (size_t)L.max_slots);
  L.bflag = take((size_t)L.max_slots);
  // the vector scratch: two interleaved arrays (L+, and s then U-) of
  // vscr_rows rows per thread; it also holds the FP32 copy of the root rows
  // (one float2 per row) during root bisection
  const size_t arrays = o.vector_precision == 2 ? 4 : 2;  // double-double: hi and lo of each
  L.vscr = take(sizeof(double) *
                std::max<size_t>(arrays * (size_t)L.vscr_threads * (size_t)L.vscr_rows, (size_t)n_total));
  L.total = off;
  return L;
}

Dev make_dev(const mrrr_plan* p, const Layout& L, void* ws, int batch, const double* d, const double* e,
             double* W, double* Z) {
  char* b = static_cast<char*>(ws);
  Dev v{};
  v.ctl = reinterpret_cast<Ctl*>(b + L.ctl);
  v.prob = reinterpret_cast<Problem*>(b + L.prob);
  v.blk = reinterpret_cast<Block*>(b + L.blk);
  v.node = reinterpret_cast<Node*>(b + L.node);
  v.rep_dl = reinterpret_cast<double2*>(b + L.pool_dl);
  v.rep_ul = reinterpret_cast<double2*>(b + L.pool_ul);
  v.ilist = reinterpret_cast<int64_t*>(b + L.ilist);
  v.lwin = reinterpret_cast<int64_t*>(b + L.lwin);
  v.rgrid = reinterpret_cast<int*>(b + L.rgrid);
  v.sched_cnt = reinterpret_cast<int*>(b + L.sched_cnt);
  v.sched_claim = reinterpret_cast<int*>(b + L.sched_claim);
  v.max_chunks = L.max_slots;
  v.nsm = p->nsm;

  v.max_list = L.max_slots;
  v.pool_cap = L.pool_rows;
  v.max_blocks = (int)std::min<int64_t>(L.max_blocks, INT32_MAX);
  v.max_nodes = (int)L.max_nodes;
  v.max_slots = L.max_slots;
  v.lo = reinterpret_cast<double*>(b + L.lo);
  v.hi = reinterpret_cast<double*>(b + L.hi);
  v.gap = reinterpret_cast<double*>(b + L.gap);
  v.wval = reinterpret_cast<double*>(b + L.wval);
  v.znrm2 = reinterpret_cast<double*>(b + L.znrm2);
  v.snode = reinterpret_cast<int*>(b + L.snode);
  v.sj = reinterpret_cast<int*>(b + L.sj);
  v.spos = reinterpret_cast<int*>(b + L.spos);
  v.state = reinterpret_cast<int*>(b + L.state);
  v.bflag = reinterpret_cast<unsigned char*>(b + L.bflag);
  v.pos_slot = nullptr;
  v.vscr = reinterpret_cast<double*>(b + L.vscr);
  v.vscr_threads = L.vscr_threads;
  v.vscr_rows = L.vscr_rows;
  v.d = d;
  v.e = e;
  v.W = W;
  v.Z = Z;
  v.batch = batch;
  const mrrr_options& o = p->opt;
  v.gap_tol = o.gap_tol;
  v.rtol = o.classify_rtol;
  v.rtol_cluster = o.cluster_rtol;
  v.root_perturb = o.root_perturb;
  v.max_depth = o.max_depth;
  v.max_bisect = o.max_bisect_steps;
  v.engine_ctas = o.engine_blocks_per_sm;
  v.width_scale = o.width_scale;
  v.fixed_width = o.multisection_width;
  v.root_side = o.root_side;
  v.vec_dd = o.vector_precision == 2;
  // double-double vectors take their own correction from a fully bisected value
  v.rq_steps = o.vector_precision == 2 || o.singleton_rq < 0 ? 0 : o.singleton_rq;
  v.root32_rtol = std::max(o.prebisect_rtol, o.classify_rtol);
  return v;
}

Grid make_grid(const mrrr_plan* p, int64_t max_slots, int n_max) {
  Grid g;
  g.nsm = p->nsm;
  g.tpb = std::max(32, std::min(1024, p->opt.threads_per_block));
  int64_t want = (max_slots + g.tpb - 1) / g.tpb;
  g.slot_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)p->nsm * 32));
  g.vec_blocks = (int)(vec_threads(p, max_slots, n_max) / 128);
  return g;
}

mrrr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA; }

// A slice of an index range (mrrr_stein_slice) must come out the same in
// every slice that computes it: a fixed multisection width (no pooling of
// points, whose runs depend on the list), the root shift on the side the
// whole range decides (root_side set by the entry point), and no neighbour
// orthogonality safeguard (its runs depend on which columns the call holds).
// Singletons are bisected to full accuracy, one factorization each: a
// slice's vector stage holds few vectors per SM sub-partition and is bound
// by the latency of each factorization, so a second one would not be hidden.
void slice_overrides(const mrrr_plan* p, const ProblemArgs& a, Dev& v) {
  if (!a.slice) return;
  v.fixed_width = p->opt.multisection_width > 0 ? p->opt.multisection_width : kSliceWidth;
  v.root_side = a.slice;  // 1 left, 2 right (set by mrrr_stein_slice)
  v.no_orth_fix = 1;
  v.rq_steps = 0;
}

// One solve enqueued on s.  device_levels: every level up to max_depth is
// enqueued without host synchronisation and the level kernels return at
// once after the tree is complete; otherwise the host reads the new-cluster
// count after each level and stops there.
mrrr_status solve(mrrr_plan* p, const ProblemArgs& a, const double* d, const double* e, double* W, double* Z,
                  int64_t n_total, int64_t k_total, int n_max, void* ws, size_t ws_bytes, cudaStream_t s,
                  bool device_levels = false) {
  Layout L = make_layout(p, a.batch, n_total, k_total, n_max);
  if (!ws || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  Dev v = make_dev(p, L, ws, a.batch, d, e, W, Z);
  slice_overrides(p, a, v);
  Grid g = make_grid(p, L.max_slots, n_max);
  p->last_ws = ws;
  p->last_graph = false;
  if (cudaMemsetAsync(v.ctl, 0, sizeof(Ctl), s) != cudaSuccess ||
      cudaMemsetAsync(v.sched_claim, 0, sizeof(int) * (size_t)v.max_chunks, s) != cudaSuccess)
    return MRRR_ERR_CUDA;
  // Clusters from an earlier solve on this workspace must not leak into this
  // one: the per-slot arrays are fully rewritten by the setup kernels.
  StageTimer* tm = &p->timer;
  const bool timing_was = tm->on;
  if (std::getenv("MRRR_TIMING") && !device_levels) tm->on = true;
  if (device_levels) tm->on = false;  // no event records inside a capture
  tm->device = false;
  set_stage_timer(tm);
  tm->begin(s);
  launch_setup(v, a, n_total, g, s);
  if (device_levels) {
    for (int level = 0; level <= p->opt.max_depth; ++level) {
      launch_level_classify(v, g, s);
      launch_level_children(v, g, s);
    }
  }
  for (int level = 0; !device_levels && level <= p->opt.max_depth; ++level) {
    launch_level_classify(v, g, s);
    if (cudaMemcpyAsync(p->host_ctl, v.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      tm->on = false;
      tm->finish();
      tm->on = timing_was;
      set_stage_timer(nullptr);
      return MRRR_ERR_CUDA;
    }
    if (p->host_ctl->status != 0 && p->host_ctl->status != MRRR_ERR_NOCONV) break;
    if (p->host_ctl->level_new == 0) break;
    launch_level_children(v, g, s);
  }
  launch_engine(v, 3, g, s);
  tm->mark("final_bisect", s);
  launch_vectors(v, g, s);
  tm->mark("vectors", s);
  tm->finish();
  set_stage_timer(nullptr);
  tm->on = timing_was;
  return cuda_status(cudaGetLastError());
}

// The solve as one CUDA graph whose cluster levels run in a conditional
// while node: setup, then the level body (classification, child
// representations, refinement) repeated on the device for as long as the
// last level made new clusters (k_level_end sets the condition), then the
// final bisection and the vectors.  No host synchronisation and no level is
// launched beyond the tree's depth.  Stage times come from device-clock
// marks.  Returns MRRR_ERR_NOTIMPL when the runtime refuses a conditional
// node (the caller then captures the unrolled form).
mrrr_status capture_conditional(mrrr_plan* p, const ProblemArgs& a, const double* d, const double* e, double* W,
                                double* Z, int64_t n_total, int64_t k_total, int n_max, void* ws,
                                cudaGraph_t* out) {
  *out = nullptr;
  Layout L = make_layout(p, a.batch, n_total, k_total, n_max);
  Dev v = make_dev(p, L, ws, a.batch, d, e, W, Z);
  slice_overrides(p, a, v);
  Grid g = make_grid(p, L.max_slots, n_max);
  cudaStream_t cs = p->cap_stream;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t graph = nullptr, tmp = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return MRRR_ERR_CUDA;
  StageTimer* tm = &p->timer;
  const bool timing_was = tm->on;
  tm->on = false;
  tm->device = true;
  tm->dev_ctl = v.ctl;
  set_stage_timer(tm);
  auto fail = [&](mrrr_status st) {
    cudaStreamCaptureStatus cst;
    if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaStreamEndCapture(cs, &tmp);
    }
    cudaGetLastError();
    cudaGraphDestroy(graph);
    tm->device = false;
    tm->on = timing_was;
    set_stage_timer(nullptr);
    return st;
  };
  // part 1: control block, setup, root bisection
  if (cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, mode) != cudaSuccess) return fail(MRRR_ERR_NOTIMPL);
  cudaMemsetAsync(v.ctl, 0, sizeof(Ctl), cs);
  cudaMemsetAsync(v.sched_claim, 0, sizeof(int) * (size_t)v.max_chunks, cs);
  tm->begin(cs);
  launch_setup(v, a, n_total, g, cs);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess)
    return fail(MRRR_ERR_CUDA);
  cudaGraphNode_t dep_copy[16];
  if (ndeps > 16) return fail(MRRR_ERR_NOTIMPL);
  for (size_t i = 0; i < ndeps; ++i) dep_copy[i] = deps[i];
  if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) return fail(MRRR_ERR_CUDA);
  p->graph_part_launches[0] = tm->launches;
  // part 2: the level loop
  cudaGraphConditionalHandle cond;
  if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(MRRR_ERR_NOTIMPL);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  if (cudaGraphAddNode(&loop, graph, dep_copy, nullptr, ndeps, &cp) != cudaSuccess) return fail(MRRR_ERR_NOTIMPL);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode) != cudaSuccess) return fail(MRRR_ERR_NOTIMPL);
  launch_level_classify(v, g, cs, cond, 1);
  launch_level_children(v, g, cs);
  if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) return fail(MRRR_ERR_NOTIMPL);
  p->graph_part_launches[1] = tm->launches - p->graph_part_launches[0];
  // part 3: singletons to full accuracy, vectors
  if (cudaStreamBeginCaptureToGraph(cs, graph, &loop, nullptr, 1, mode) != cudaSuccess) return fail(MRRR_ERR_NOTIMPL);
  launch_engine(v, 3, g, cs);
  tm->mark("final_bisect", cs);
  launch_vectors(v, g, cs);
  tm->mark("vectors", cs);
  if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) return fail(MRRR_ERR_CUDA);
  p->graph_part_launches[2] = tm->launches - p->graph_part_launches[0] - p->graph_part_launches[1];
  tm->device = false;
  tm->on = timing_was;
  set_stage_timer(nullptr);
  if (cudaGetLastError() != cudaSuccess) {
    cudaGraphDestroy(graph);
    return MRRR_ERR_CUDA;
  }
  *out = graph;
  return MRRR_OK;
}

// use_graph: capture the device-driven solve once per call signature on the
// plan's own stream, then replay the graph on the caller's stream.  The
// conditional-node form is tried first; where the runtime refuses it, every
// level up to max_depth is captured (levels past the tree's depth return at
// entry).
mrrr_status solve_graph(mrrr_plan* p, const ProblemArgs& a, const double* d, const double* e, double* W, double* Z,
                        int64_t n_total, int64_t k_total, int n_max, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (!ws || ws_bytes < make_layout(p, a.batch, n_total, k_total, n_max).total) return MRRR_ERR_WORKSPACE;
  GraphKey k{};
  k.a = a;
  k.d = d;
  k.e = e;
  k.ws = ws;
  k.W = W;
  k.Z = Z;
  k.n_total = n_total;
  k.k_total = k_total;
  k.n_max = n_max;
  k.ws_bytes = ws_bytes;
  k.opt_version = p->opt_version;
  if (!p->have_graph || !same_key(k, p->key)) {
    if (p->have_graph) {
      cudaGraphExecDestroy(p->exec);
      p->have_graph = false;
    }
    if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return MRRR_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    p->timer.launches = 0;
    mrrr_status st = capture_conditional(p, a, d, e, W, Z, n_total, k_total, n_max, ws, &graph);
    p->graph_conditional = st == MRRR_OK;
    if (st == MRRR_ERR_NOTIMPL) {
      p->timer.launches = 0;
      if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MRRR_ERR_CUDA;
      st = solve(p, a, d, e, W, Z, n_total, k_total, n_max, ws, ws_bytes, p->cap_stream, true);
      const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &graph);
      if (st == MRRR_OK && (ce != cudaSuccess || !graph)) st = MRRR_ERR_CUDA;
    }
    if (st != MRRR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    const cudaError_t ie = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return MRRR_ERR_CUDA;
    p->key = k;
    p->have_graph = true;
    p->graph_launches = p->timer.launches;
  }
  p->last_ws = ws;
  p->last_graph = true;
  p->timer.launches = p->graph_launches;
  p->timer.nstages = 0;
  return cuda_status(cudaGraphLaunch(p->exec, s));
}

mrrr_status dispatch(mrrr_plan* p, const ProblemArgs& a, const double* d, const double* e, double* W, double* Z,
                     int64_t n_total, int64_t k_total, int n_max, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (p->opt.use_graph) return solve_graph(p, a, d, e, W, Z, n_total, k_total, n_max, ws, ws_bytes, s);
  return solve(p, a, d, e, W, Z, n_total, k_total, n_max, ws, ws_bytes, s);
}

}  // namespace
}  // namespace mrrr

using namespace mrrr;

extern "C" {

mrrr_status mrrr_options_default(mrrr_options* opt) {
  if (!opt) return MRRR_ERR_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->gap_tol = 1e-4;
  opt->classify_rtol = 0x1p-20;
  opt->max_depth = 64;
  opt->max_bisect_steps = 256;
  opt->threads_per_block = 128;
  opt->vec_blocks_per_sm = 4;
  opt->cluster_rtol = 0x1p-40;
  opt->root_perturb = 64.0;
  opt->engine_blocks_per_sm = 2;
  opt->width_scale = 1.0;
  opt->prebisect_rtol = 0x1p-17;
  opt->vector_precision = 1;
  opt->singleton_rq = 1;
  return MRRR_OK;
}

mrrr_status mrrr_plan_create(mrrr_plan** plan, const mrrr_options* opt) {
  if (!plan) return MRRR_ERR_ARG;
  *plan = nullptr;
  mrrr_options o;
  mrrr_options_default(&o);
  if (opt) {
    if (opt->gap_tol > 0) o.gap_tol = opt->gap_tol;
    if (opt->classify_rtol > 0) o.classify_rtol = opt->classify_rtol;
    if (opt->max_depth > 0) o.max_depth = opt->max_depth;
    if (opt->max_bisect_steps > 0) o.max_bisect_steps = opt->max_bisect_steps;
    if (opt->threads_per_block > 0) o.threads_per_block = opt->threads_per_block;
    if (opt->vec_blocks_per_sm > 0) o.vec_blocks_per_sm = opt->vec_blocks_per_sm;
    if (opt->max_nodes > 0) o.max_nodes = opt->max_nodes;
    if (opt->pool_rows > 0) o.pool_rows = opt->pool_rows;
    if (opt->cluster_rtol > 0) o.cluster_rtol = opt->cluster_rtol;
    if (opt->root_perturb > 0) o.root_perturb = opt->root_perturb;
    if (opt->root_perturb < 0) o.root_perturb = 0.0;  // negative: no perturbation
    if (opt->use_graph > 0) o.use_graph = 1;
    if (opt->engine_blocks_per_sm > 0) o.engine_blocks_per_sm = std::min(opt->engine_blocks_per_sm, 2);
    if (opt->width_scale > 0) o.width_scale = opt->width_scale;
    if (opt->prebisect_rtol > 0) o.prebisect_rtol = std::max(opt->prebisect_rtol, 0x1p-20);
    if (opt->multisection_width > 0) o.multisection_width = opt->multisection_width;
    if (opt->root_side > 0) o.root_side = opt->root_side;
    if (opt->vector_precision > 0) o.vector_precision = opt->vector_precision;
    if (opt->singleton_rq != 0) o.singleton_rq = opt->singleton_rq;
  }
  const int mw = o.multisection_width;
  if (mw < 0 || mw > 32 || (mw & (mw - 1)) != 0 || o.root_side < 0 || o.root_side > 2 ||
      o.vector_precision < 0 || o.vector_precision > 2 || o.singleton_rq < -1 || o.singleton_rq > 4)
    return MRRR_ERR_ARG;
  if (o.gap_tol >= 1.0 || o.classify_rtol >= 0.25 || o.threads_per_block % 32 != 0) return MRRR_ERR_ARG;
  if (o.cluster_rtol >= 0.25 || o.prebisect_rtol >= 0.25 || !std::isfinite(o.root_perturb) ||
      !std::isfinite(o.width_scale))
    return MRRR_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRRR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MRRR_ERR_CUDA;
  mrrr_plan* p = new (std::nothrow) mrrr_plan();
  if (!p) return MRRR_ERR_CUDA;
  p->opt = o;
  p->device = dev;
  p->nsm = nsm;
  p->last_ws = nullptr;
  p->opt_version = 0;
  p->cap_stream = nullptr;
  p->exec = nullptr;
  p->have_graph = false;
  p->graph_conditional = false;
  p->last_graph = false;
  p->graph_launches = 0;
  if (cudaMallocHost(&p->host_ctl, sizeof(Ctl)) != cudaSuccess) {
    delete p;
    return MRRR_ERR_CUDA;
  }
  std::memset(p->host_ctl, 0, sizeof(Ctl));
  *plan = p;
  return MRRR_OK;
}

mrrr_status mrrr_plan_destroy(mrrr_plan* plan) {
  if (!plan) return MRRR_ERR_ARG;
  if (plan->have_graph) cudaGraphExecDestroy(plan->exec);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  plan->timer.release();
  cudaFreeHost(plan->host_ctl);
  delete plan;
  return MRRR_OK;
}

mrrr_status mrrr_workspace_size(const mrrr_plan* plan, int batch, int64_t n_total, int64_t k_total, int n_max,
                                size_t* bytes) {
  if (!plan || !bytes || batch < 0 || n_total < 0 || k_total < 0 || n_max < 0) return MRRR_ERR_ARG;
  *bytes = make_layout(plan, batch, n_total, k_total, n_max).total;
  return MRRR_OK;
}

mrrr_status mrrr_stein(mrrr_plan* plan, int n, const double* d, const double* e, int il, int iu, double* W,
                       double* Z, int64_t ldz, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!d || (n > 1 && !e) || !W || il < 1 || iu > n || il > iu || (Z && ldz < n)) return MRRR_ERR_ARG;
  ProblemArgs a{};
  a.batch = 1;
  a.n = n;
  a.il1 = il;
  a.iu1 = iu;
  a.ldz = Z ? ldz : n;
  // a 1x1 problem has no off-diagonal; any non-null pointer is never read
  const double* ee = (n > 1) ? e : d;
  return dispatch(plan, a, d, ee, W, Z, n, (int64_t)(iu - il + 1), n, workspace, ws_bytes,
                  static_cast<cudaStream_t>(stream));
}

mrrr_status mrrr_slice_range(int il, int iu, int nslices, int slice, int* a, int* b) {
  if (!a || !b || il < 1 || iu < il || nslices < 1 || slice < 0 || slice >= nslices || nslices > iu - il + 1)
    return MRRR_ERR_ARG;
  const int64_t k = (int64_t)iu - il + 1;
  *a = il + (int)((int64_t)slice * k / nslices);
  *b = il + (int)((int64_t)(slice + 1) * k / nslices) - 1;
  return MRRR_OK;
}

mrrr_status mrrr_stein_slice(mrrr_plan* plan, int n, const double* d, const double* e, int il, int iu, int nslices,
                             int slice, int margin, double* W, double* Z, int64_t ldz, void* workspace,
                             size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  int a = 0, b = 0;
  if (!d || (n > 1 && !e) || !W || il < 1 || iu > n || il > iu || (Z && ldz < n) || margin < 1 ||
      mrrr_slice_range(il, iu, nslices, slice, &a, &b) != MRRR_OK)
    return MRRR_ERR_ARG;
  ProblemArgs pa{};
  pa.batch = 1;
  pa.n = n;
  pa.il1 = std::max(1, a - margin);
  pa.iu1 = std::min(n, b + margin);
  pa.ol1 = a;
  pa.ou1 = b;
  // the root shift on the side the whole range il..iu chooses, for every slice
  pa.slice = (il + iu) <= (n + 1) ? 1 : 2;
  pa.ldz = Z ? ldz : n;
  const double* ee = (n > 1) ? e : d;
  return dispatch(plan, pa, d, ee, W, Z, n, (int64_t)(pa.iu1 - pa.il1 + 1), n, workspace, ws_bytes,
                  static_cast<cudaStream_t>(stream));
}

mrrr_status mrrr_stein_batched(mrrr_plan* plan, int batch, const int64_t* d_off, const double* d, const double* e,
                               const int* il, const int* iu, double* W, const int64_t* w_off, double* Z,
                               const int64_t* z_off, int64_t n_total, int64_t k_total, int n_max, void* workspace,
                               size_t ws_bytes, mrrr_stream stream) {
  if (!plan || batch < 0 || n_total < 0 || k_total < 0 || n_max < 0) return MRRR_ERR_ARG;
  if (batch == 0 || n_total == 0) return MRRR_OK;
  if (!d_off || !d || !e || !W || !w_off || (Z && !z_off)) return MRRR_ERR_ARG;
  ProblemArgs a{};
  a.batch = batch;
  a.d_off = d_off;
  a.il = il;
  a.iu = iu;
  a.w_off = w_off;
  a.z_off = z_off;
  return dispatch(plan, a, d, e, W, Z, n_total, k_total, n_max, workspace, ws_bytes,
                  static_cast<cudaStream_t>(stream));
}

mrrr_status mrrr_autotune_batched(mrrr_plan* plan, int batch, const int64_t* d_off, const double* d,
                                  const double* e, const int* il, const int* iu, double* W, const int64_t* w_off,
                                  double* Z, const int64_t* z_off, int64_t n_total, int64_t k_total, int n_max,
                                  void* workspace, size_t ws_bytes, mrrr_stream stream, mrrr_tuning* out) {
  if (!plan || !out || batch <= 0 || n_total <= 0 || k_total < 0 || n_max <= 0) return MRRR_ERR_ARG;
  if (!d_off || !d || !e || !W || !w_off || (Z && !z_off)) return MRRR_ERR_ARG;
  ProblemArgs a{};
  a.batch = batch;
  a.d_off = d_off;
  a.il = il;
  a.iu = iu;
  a.w_off = w_off;
  a.z_off = z_off;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  static const int kCtas[] = {2, 1};
  static const double kWidth[] = {1.0, 0.5, 2.0};
  // bisection steps before the vector stage: the default (singletons to
  // 2^-36, one Rayleigh-quotient correction) or full bisection (2 eps)
  static const int kRq[] = {1, -1};
  const mrrr_options saved = plan->opt;
  const bool timing = plan->timer.on;
  plan->timer.on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    plan->timer.on = timing;
    return MRRR_ERR_CUDA;
  }
  std::memset(out, 0, sizeof(*out));
  double best = INFINITY;
  mrrr_status st = MRRR_OK;
  int tried = 0;
  // one untimed solve first: the timed candidates then all run warm
  plan->opt.use_graph = 0;
  st = solve(plan, a, d, e, W, Z, n_total, k_total, n_max, workspace, ws_bytes, s, true);
  for (int k = 0; k < 12 && st == MRRR_OK; ++k) {
    const int ci = k / 6, wi = (k / 2) % 3, ri = k % 2;
    {
      if (plan->opt.vector_precision == 2 && ri == 1) continue;  // the option does not apply
      plan->opt.engine_blocks_per_sm = kCtas[ci];
      plan->opt.width_scale = kWidth[wi];
      plan->opt.singleton_rq = plan->opt.vector_precision == 2 ? saved.singleton_rq : kRq[ri];
      cudaEventRecord(e0, s);
      st = solve(plan, a, d, e, W, Z, n_total, k_total, n_max, workspace, ws_bytes, s, true);
      cudaEventRecord(e1, s);
      if (st != MRRR_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const mrrr_status dev = mrrr_get_status(plan, stream, nullptr);
      if (dev != MRRR_OK && dev != MRRR_ERR_NOCONV) {
        st = dev;
        break;
      }
      if (tried == 0) out->default_ms = ms;
      ++tried;
      if (ms < best) {
        best = ms;
        out->engine_blocks_per_sm = kCtas[ci];
        out->width_scale = kWidth[wi];
        out->singleton_rq = plan->opt.singleton_rq;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->opt = saved;
  plan->timer.on = timing;
  if (st != MRRR_OK) return st;
  plan->opt.engine_blocks_per_sm = out->engine_blocks_per_sm;
  plan->opt.width_scale = out->width_scale;
  plan->opt.singleton_rq = out->singleton_rq;
  ++plan->opt_version;
  out->best_ms = best;
  out->configs = tried;
  return MRRR_OK;
}

mrrr_status mrrr_get_status(mrrr_plan* plan, mrrr_stream stream, mrrr_info* out) {
  if (!plan) return MRRR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MRRR_ERR_CUDA;
  if (!plan->last_ws) {
    if (out) std::memset(out, 0, sizeof(*out));
    return MRRR_OK;
  }
  if (cudaMemcpy(plan->host_ctl, plan->last_ws, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MRRR_ERR_CUDA;
  const Ctl& c = *plan->host_ctl;
  if (out) {
    out->status = c.status;
    out->depth = c.depth;
    out->nodes = (int64_t)c.nodes - c.nblocks;
    out->pool_rows_used = c.pool_need;
    out->fallbacks = (int64_t)c.fallbacks;
    out->twisted_solves = (int64_t)c.twisted_solves;
    out->levels = c.levels;
    for (int i = 0; i < 12; ++i) out->diag[i] = (int64_t)c.diag[i];
    for (int i = 0; i < 4; ++i) {
      out->sturm_counts[i] = (int64_t)c.eng_counts[i];
      out->sturm_rows[i] = (int64_t)c.eng_rows[i];
      out->warp_passes[i] = (int64_t)c.eng_passes[i];
    }
  }
  return static_cast<mrrr_status>(c.status);
}

mrrr_status mrrr_set_timing(mrrr_plan* plan, int enable) {
  if (!plan) return MRRR_ERR_ARG;
  plan->timer.on = enable != 0;
  return MRRR_OK;
}

mrrr_status mrrr_get_profile(const mrrr_plan* plan, mrrr_profile* out) {
  if (!plan || !out) return MRRR_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  const StageTimer& t = plan->timer;
  out->launches = t.launches;
  if (plan->last_graph && plan->last_ws) {
    // graph replay: per-stage GPU time from the device-clock marks (the
    // caller has synchronised the stream the graph ran on)
    Ctl c;
    if (cudaMemcpy(&c, plan->last_ws, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return MRRR_ERR_CUDA;
    for (int k = 0; k < ST_COUNT; ++k) {
      std::strncpy(out->name[k], kStageNames[k], 23);
      out->ms[k] = (double)c.stage_ns[k] * 1e-6;
    }
    out->nstages = ST_COUNT;
    // kernels executed: the loop body ran once per level
    if (plan->graph_conditional)
      out->launches = plan->graph_part_launches[0] + (int64_t)c.levels * plan->graph_part_launches[1] +
                      plan->graph_part_launches[2];
    return MRRR_OK;
  }
  out->nstages = t.nstages;
  for (int k = 0; k < t.nstages && k < 32; ++k) {
    std::strncpy(out->name[k], t.stage_name[k], 23);
    out->ms[k] = t.stage_ms[k];
  }
  return MRRR_OK;
}

const char* mrrr_status_string(mrrr_status s) {
  switch (s) {
    case MRRR_OK: return "ok";
    case MRRR_ERR_ARG: return "invalid argument";
    case MRRR_ERR_WORKSPACE: return "workspace missing or too small";
    case MRRR_ERR_NONFINITE: return "non-finite input";
    case MRRR_ERR_NOCONV: return "iteration limit reached";
    case MRRR_ERR_QUEUE: return "cluster node table or representation pool full";
    case MRRR_ERR_TIMEOUT: return "bounded device wait gave up";
    case MRRR_ERR_CUDA: return "CUDA runtime error";
    case MRRR_ERR_NOTIMPL: return "not implemented";
    case MRRR_ERR_MARGIN: return "slice margin too small for a cluster at the slice boundary";
    case MRRR_ERR_NOTSPD: return "matrix not positive definite";
  }
  return "unknown status";
}

int mrrr_version(void) { return 100; }

}  // extern "C"
