// mrrr_engine.cu -- the interval engine: bisection of many eigenvalue
// intervals on shared representations (Sec. 3.1.1: every eigenvalue is
// approximated by bisection, O(n) flops each; the eigenvalues of a cluster
// are refined to high relative accuracy on the cluster's new RRR).
//
// Work is a list of chunks, each a contiguous range of slots of ONE node, in
// two kinds executed by one persistent kernel:
//   big chunks (nodes with many slots) -- a CTA streams the node's (D, LLD)
//     plane into shared memory with bulk asynchronous copies (cp.async.bulk,
//     completion on an mbarrier, bounded waits) and every thread counts
//     against the shared rows (broadcast reads); chunk sizes are chosen so
//     that the chunks fill about three CTAs per SM;
//   small chunks (nodes with few slots, e.g. the many two-eigenvalue
//     clusters of Wilkinson matrices) -- one warp per chunk reads the rows
//     straight from L1/L2 with register prefetch, so that many small nodes
//     run side by side.
// In both kinds an interval gets T threads when there are fewer intervals
// than threads: they evaluate T interior points per pass (multisection),
// which gains log2(T+1) bits per pass over the representation instead of one.
// The Sturm counts are the division-free recurrence of count_step().
//
// Modes:
//   ROOT       root representation of a block, from its Gershgorin bracket,
//              to the classification accuracy rtol;
//   PREREFINE  the two end members of a new cluster, in the PARENT's
//              representation, to the cluster accuracy (so that the child
//              shift can be placed right at the cluster's end);
//   REFINE     cluster members moved into the CHILD's coordinates
//              (lambda - sigma_c), the bracket confirmed by two counts and
//              widened until it holds, then bisected to rtol;
//   FINAL      singletons on their node's representation, to full relative
//              accuracy (the interval can no longer be split), so that one
//              twisted factorization gives the vector.
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {

namespace {

constexpr int kEngThreads = 128;
constexpr int kTileRows = 2048;  // 32 KiB per stage
constexpr int kStages = 2;
constexpr int kMaxChunkSlots = kEngThreads;
constexpr int kSmallNode = 24;   // nodes with at most this many slots run per warp
constexpr int kCtasPerSm = 3;
constexpr size_t kEngSmem = sizeof(double2) * kTileRows * kStages;

enum : int { MODE_ROOT = 0, MODE_PREREFINE = 1, MODE_REFINE = 2, MODE_FINAL = 3 };
enum : int { PH_BISECT = 0, PH_VERIFY = 1 };

__device__ __forceinline__ void node_range(const Dev& v, int mode, int& begin, int& end) {
  if (mode == MODE_ROOT) {
    begin = 0;
    end = v.ctl->nblocks;
  } else if (mode == MODE_FINAL) {
    begin = 0;
    end = min(v.ctl->nodes, v.max_nodes);
  } else {
    begin = v.ctl->level_begin;
    end = min(v.ctl->nodes, v.max_nodes);
  }
}

__device__ __forceinline__ bool node_eligible(const Dev& v, int mode, const Node& nd) {
  // PREREFINE uses the parent's representation: the node's own is built later
  if (nd.depth < 0 || (mode != MODE_PREREFINE && nd.rep < 0)) return false;
  return v.blk[nd.block].m > 1;
}

__global__ void k_reset_chunks(Dev v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    v.ctl->nchunks = 0;
    v.ctl->chunk_next = 0;
    v.ctl->nsmall = 0;
    v.ctl->small_next = 0;
    v.ctl->big_slots = 0;
  }
}

// Pass 1: total slots of the big nodes (sets the big chunk size).
template <int MODE>
__global__ void k_count_work(Dev v) {
  int begin, end;
  node_range(v, MODE, begin, end);
  long long local = 0;
  for (int64_t id = begin + gtid(); id < end; id += gstride()) {
    const Node nd = v.node[id];
    if (!node_eligible(v, MODE, nd)) continue;
    const int64_t size = nd.last - nd.first + 1;
    if (size > kSmallNode) local += size;
  }
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd((unsigned long long*)&v.ctl->big_slots, (unsigned long long)local);
}

// Pass 2: the chunks.  Big chunks from the front of the list, small ones
// (one per small node) from the back.
template <int MODE>
__global__ void k_make_chunks(Dev v, int nctas) {
  int begin, end;
  node_range(v, MODE, begin, end);
  const long long big = v.ctl->big_slots;
  int csize = (int)((big + nctas - 1) / nctas);
  csize = max(32, min(kMaxChunkSlots, csize));
  // the big chunks use at most big/32 + nodes entries from the front
  for (int64_t id = begin + gtid(); id < end; id += gstride()) {
    const Node nd = v.node[id];
    if (!node_eligible(v, MODE, nd)) continue;
    const int64_t size = nd.last - nd.first + 1;
    if (size <= kSmallNode) {
      const int k = atomicAdd(&v.ctl->nsmall, 1);
      const int64_t at = v.max_chunks - 1 - k;
      if (at < v.max_chunks / 2) {  // the back half holds the small chunks
        set_status(v.ctl, MRRR_ERR_QUEUE);
        continue;
      }
      v.chunks[at] = Chunk{(int)id, 0, nd.first, nd.last + 1};
      continue;
    }
    const int cnt = (int)((size + csize - 1) / csize);
    const int base = atomicAdd(&v.ctl->nchunks, cnt);
    if (base + cnt > v.max_chunks / 2) {
      set_status(v.ctl, MRRR_ERR_QUEUE);
      continue;
    }
    for (int c = 0; c < cnt; ++c) {
      const int64_t s0 = nd.first + (int64_t)c * csize;
      v.chunks[base + c] = Chunk{(int)id, 0, s0, min(nd.last + 1, s0 + csize)};
    }
  }
}

// Per-interval state.
struct IvState {
  double lo, hi, plo, phi, delta;
  int64_t slot;
  int j, phase, tries, steps, done, pad_;
};

template <int MODE>
__device__ __forceinline__ bool slot_wanted(const Dev& v, int64_t w, int node, const Node& nd) {
  if (MODE == MODE_FINAL) {
    const int st = v.state[w];
    return slot_final(st) && v.snode[w] == node && v.spos[w] >= 0;
  }
  if (MODE == MODE_PREREFINE && w != nd.first && w != nd.last) return false;
  return v.state[w] == SLOT_ACTIVE && v.snode[w] == node;
}

template <int MODE>
__device__ __forceinline__ void iv_init(const Dev& v, int64_t w, const Block& bk, const Node& nd, double pivmin,
                                        IvState& q) {
  q.slot = w;
  q.j = v.sj[w];
  q.steps = 0;
  q.tries = 0;
  q.done = 0;
  q.phase = PH_BISECT;
  if (MODE == MODE_ROOT) {
    q.lo = bk.gl;
    q.hi = bk.gu;
  } else if (MODE == MODE_REFINE) {
    q.plo = v.lo[w];
    q.phi = v.hi[w];
    q.delta = 16.0 * kEps * fmax(fabs(q.plo), fabs(q.phi)) + 4.0 * pivmin;
    q.lo = (q.plo - nd.sigma_rel) - q.delta;
    q.hi = (q.phi - nd.sigma_rel) + q.delta;
    q.phase = PH_VERIFY;
  } else {
    q.lo = v.lo[w];
    q.hi = v.hi[w];
  }
}

// Evaluation point of thread pt (of T) of an interval in this pass.
__device__ __forceinline__ bool iv_tau(const IvState& q, int T, int pt, double& tau) {
  if (q.phase == PH_VERIFY) {
    if (T >= 2) {
      tau = pt == 0 ? q.lo : q.hi;
      return pt < 2;
    }
    tau = (q.tries & 1) ? q.hi : q.lo;  // one end per pass: lo, then hi
    return true;
  }
  tau = q.lo + (q.hi - q.lo) * ((double)(pt + 1) / (double)(T + 1));
  return true;
}

// Update after a pass; neg(k) returns the count of point k of the interval.
// Returns true when the interval is finished.
template <int MODE, typename NegFn>
__device__ __forceinline__ bool iv_update(const Dev& v, const Node& nd, int T, double rtol, double atol, int maxsteps,
                                          IvState& q, NegFn neg) {
  if (q.phase == PH_VERIFY) {
    bool ok_lo, ok_hi, decided;
    if (T >= 2) {
      ok_lo = neg(0) <= q.j - 1;
      ok_hi = neg(1) >= q.j;
      decided = true;
    } else if ((q.tries & 1) == 0) {  // lower end just counted
      ok_lo = neg(0) <= q.j - 1;
      ok_hi = true;
      decided = !ok_lo;
      if (ok_lo) q.tries |= 1;  // next: upper end
    } else {
      ok_lo = true;
      ok_hi = neg(0) >= q.j;
      decided = true;
      q.tries &= ~1;
    }
    if (decided) {
      if (ok_lo && ok_hi) {
        q.phase = PH_BISECT;
        if (converged(q.lo, q.hi, rtol, atol)) return true;
      } else {
        q.tries = (q.tries & ~1) + 2;
        q.delta *= 4.0;
        q.lo = (q.plo - nd.sigma_rel) - q.delta;
        q.hi = (q.phi - nd.sigma_rel) + q.delta;
        if (q.tries > 48) {  // give up confirming; bisect what we have
          set_status(v.ctl, MRRR_ERR_NOCONV);
          diag(v.ctl, DIAG_REFINE_BRACKET);
          q.phase = PH_BISECT;
        }
      }
    }
    return false;
  }
  int k = 0;
  while (k < T && neg(k) < q.j) ++k;  // first point with count >= j
  const double nlo = k > 0 ? q.lo + (q.hi - q.lo) * ((double)k / (double)(T + 1)) : q.lo;
  const double nhi = k < T ? q.lo + (q.hi - q.lo) * ((double)(k + 1) / (double)(T + 1)) : q.hi;
  const bool stuck = !(nlo < nhi) || (nlo == q.lo && nhi == q.hi);
  q.lo = nlo;
  q.hi = nhi;
  ++q.steps;
  if (stuck || converged(q.lo, q.hi, rtol, atol) || q.steps >= maxsteps) {
    if (q.steps >= maxsteps && !stuck && !converged(q.lo, q.hi, rtol, atol)) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, MODE == MODE_ROOT ? DIAG_ROOT_BISECT : DIAG_REFINE_BISECT);
    }
    return true;
  }
  return false;
}

// Largest power of two T with T * n <= lanes.
__device__ __forceinline__ int points_per_interval(int n, int lanes) {
  int t = 1;
  while (t * 2 * n <= lanes) t *= 2;
  return t;
}

template <int MODE>
__device__ __forceinline__ double mode_rtol(const Dev& v) {
  return MODE == MODE_ROOT || MODE == MODE_REFINE ? v.rtol : MODE == MODE_FINAL ? 2.0 * kEps : v.rtol_cluster;
}

// ---------------------------------------------------------------------------
// Big chunks: one CTA, rows staged through shared memory.
template <int MODE>
__device__ void run_big_chunks(const Dev& v, double2* tiles, uint64_t* bars, uint32_t* parity, IvState* iv,
                               int* s_neg, int* s_misc) {
  const int tid = threadIdx.x;
  const double rtol = mode_rtol<MODE>(v);
  const int maxsteps = v.max_bisect;
  const int nchunks = min(v.ctl->nchunks, (int)(v.max_chunks / 2));
  int& s_chunk = s_misc[0];
  int& s_nact = s_misc[1];
  int& s_abort = s_misc[2];
  for (;;) {
    __syncthreads();  // readers of the previous chunk are done with tiles and state
    if (tid == 0) s_chunk = atomicAdd(&v.ctl->chunk_next, 1);
    __syncthreads();
    const int ci = s_chunk;
    if (ci >= nchunks || s_abort) break;
    const Chunk ch = v.chunks[ci];
    const Node nd = v.node[ch.node];
    const Block bk = v.blk[nd.block];
    const Node rn = MODE == MODE_PREREFINE ? v.node[nd.parent] : nd;  // representation used
    const int m = bk.m;
    const double2* dl = v.rep_dl + rn.rep;
    const double pivmin = rn.pivmin;
    const int pivexp = exp_field(pivmin);
    const double atol = 4.0 * pivmin;
    const int ntiles = (m + kTileRows - 1) / kTileRows;
    const bool resident = ntiles <= kStages;

    if (tid < 32) {  // warp 0 gathers the chunk's intervals
      int base = 0;
      for (int64_t w0 = ch.s0; w0 < ch.s1; w0 += 32) {
        const int64_t w = w0 + tid;
        const bool want = w < ch.s1 && slot_wanted<MODE>(v, w, ch.node, nd);
        const unsigned mask = __ballot_sync(0xffffffffu, want);
        if (want) {
          IvState& q = iv[base + __popc(mask & ((1u << tid) - 1u))];
          iv_init<MODE>(v, w, bk, nd, pivmin, q);
          if (q.phase == PH_BISECT && converged(q.lo, q.hi, rtol, atol)) {
            q.done = 1;
            v.lo[w] = q.lo;
            v.hi[w] = q.hi;
          }
        }
        base += __popc(mask);
      }
      if (tid == 0) s_nact = base;
    }
    __syncthreads();
    const int nact = s_nact;
    if (nact == 0) continue;
    const int T = points_per_interval(nact, kEngThreads);
    const int qi = tid / T, pt = tid % T;
    const bool mine = qi < nact;

    int pass = 0;
    const int max_passes = maxsteps + 2 * 26 + 8;
    for (;;) {
      double tau = 0.0;
      bool act = mine && !iv[qi].done;
      if (act) act = iv_tau(iv[qi], T, pt, tau);
      if (!__syncthreads_or(act) || pass >= max_passes || s_abort) break;
      if (tid == 0 && (!resident || pass == 0)) {
        fence_proxy_async();
        for (int t = 0; t < min(ntiles, kStages); ++t) {
          const int rows = min(kTileRows, m - t * kTileRows);
          mbar_expect_tx(&bars[t], (uint32_t)(rows * sizeof(double2)));
          tma_load_1d(tiles + t * kTileRows, dl + (int64_t)t * kTileRows, (uint32_t)(rows * sizeof(double2)),
                      &bars[t]);
        }
      }
      double a = -tau, b = 1.0;
      int neg = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int stg = t % kStages;
        if (!resident || pass == 0) {
          if (!mbar_wait(&bars[stg], parity[stg])) {
            if (atomicExch(&s_abort, 1) == 0) set_status(v.ctl, MRRR_ERR_TIMEOUT);
          }
          parity[stg] ^= 1u;
        }
        const double2* tl = tiles + stg * kTileRows;
        const int rows = min(kTileRows, m - t * kTileRows);
        if (act) {
#pragma unroll 4
          for (int i = 0; i < rows; ++i) {
            const double2 r = tl[i];
            count_step(r.x, r.y, tau, pivexp, pivmin, a, b, neg);
          }
        }
        if (!resident) {
          __syncthreads();  // every reader is done with this stage
          const int nt = t + kStages;
          if (tid == 0 && nt < ntiles) {
            fence_proxy_async();
            const int rows2 = min(kTileRows, m - nt * kTileRows);
            mbar_expect_tx(&bars[stg], (uint32_t)(rows2 * sizeof(double2)));
            tma_load_1d(tiles + stg * kTileRows, dl + (int64_t)nt * kTileRows,
                        (uint32_t)(rows2 * sizeof(double2)), &bars[stg]);
          }
        }
      }
      ++pass;
      s_neg[tid] = neg;
      __syncthreads();
      if (mine && pt == 0 && !iv[qi].done) {
        IvState& q = iv[qi];
        const int b0 = qi * T;
        if (iv_update<MODE>(v, nd, T, rtol, atol, maxsteps, q, [&](int k) { return s_neg[b0 + k]; })) {
          q.done = 1;
          v.lo[q.slot] = q.lo;
          v.hi[q.slot] = q.hi;
        }
      }
      __syncthreads();
    }
    // intervals left at the pass cap keep their current bracket
    if (mine && pt == 0 && !iv[qi].done) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      v.lo[iv[qi].slot] = iv[qi].lo;
      v.hi[iv[qi].slot] = iv[qi].hi;
    }
  }
}

// ---------------------------------------------------------------------------
// Small chunks: one warp, rows read from global memory (L1/L2) with a
// two-batch register prefetch.
constexpr int kPrefetch = 8;

__device__ __forceinline__ int warp_count(const double2* __restrict__ dl, int m, double tau, int pivexp,
                                          double pivmin, bool act) {
  double a = -tau, b = 1.0;
  int neg = 0;
  double2 cur[kPrefetch], nxt[kPrefetch];
#pragma unroll
  for (int u = 0; u < kPrefetch; ++u) cur[u] = u < m ? __ldg(dl + u) : make_double2(1.0, 0.0);
  for (int i0 = 0; i0 < m; i0 += kPrefetch) {
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int i = i0 + kPrefetch + u;
      nxt[u] = i < m ? __ldg(dl + i) : make_double2(1.0, 0.0);
    }
    if (act) {
#pragma unroll
      for (int u = 0; u < kPrefetch; ++u)
        if (i0 + u < m) count_step(cur[u].x, cur[u].y, tau, pivexp, pivmin, a, b, neg);
    }
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) cur[u] = nxt[u];
  }
  return neg;
}

template <int MODE>
__device__ void run_small_chunks(const Dev& v, const int& s_abort, int* s_neg) {
  const int lane = threadIdx.x & 31;
  int* wneg = s_neg + (threadIdx.x & ~31);  // this warp's 32 counts
  const double rtol = mode_rtol<MODE>(v);
  const int maxsteps = v.max_bisect;
  const int nsmall = min(v.ctl->nsmall, (int)(v.max_chunks - v.max_chunks / 2));
  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(&v.ctl->small_next, 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= nsmall || s_abort) break;
    const Chunk ch = v.chunks[v.max_chunks - 1 - c];
    const Node nd = v.node[ch.node];
    const Block bk = v.blk[nd.block];
    const Node rn = MODE == MODE_PREREFINE ? v.node[nd.parent] : nd;
    const int m = bk.m;
    const double2* dl = v.rep_dl + rn.rep;
    const double pivmin = rn.pivmin;
    const int pivexp = exp_field(pivmin);
    const double atol = 4.0 * pivmin;
    // compact the wanted slots (a small node has at most 32)
    const int64_t w = ch.s0 + lane;
    const bool want = w < ch.s1 && slot_wanted<MODE>(v, w, ch.node, nd);
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    const int nact = __popc(mask);
    if (nact == 0) continue;
    const int T = points_per_interval(nact, 32);
    const int qi = lane / T, pt = lane % T;
    const bool mine = qi < nact;
    // the slot of interval qi is the qi-th set bit of mask
    int64_t myslot = -1;
    {
      unsigned mm = mask;
      for (int k = 0; k < qi && mm; ++k) mm &= mm - 1;
      if (mine && mm) myslot = ch.s0 + (__ffs(mm) - 1);
    }
    IvState q{};
    if (mine) {
      iv_init<MODE>(v, myslot, bk, nd, pivmin, q);
      if (q.phase == PH_BISECT && converged(q.lo, q.hi, rtol, atol)) q.done = 1;
    }
    const int max_passes = maxsteps + 2 * 26 + 8;
    for (int pass = 0; pass < max_passes; ++pass) {
      double tau = 0.0;
      bool act = mine && !q.done;
      if (act) act = iv_tau(q, T, pt, tau);
      if (!__any_sync(0xffffffffu, act)) break;
      const int neg = warp_count(dl, m, tau, pivexp, pivmin, act);
      // every lane of an interval's group applies the same update
      const int b0 = qi * T;
      wneg[lane] = neg;
      __syncwarp();
      if (mine && !q.done) {
        if (iv_update<MODE>(v, nd, T, rtol, atol, maxsteps, q, [&](int k) { return wneg[b0 + k]; })) q.done = 1;
      }
      __syncwarp();
    }
    if (mine && pt == 0) {
      if (!q.done) set_status(v.ctl, MRRR_ERR_NOCONV);
      v.lo[myslot] = q.lo;
      v.hi[myslot] = q.hi;
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kEngThreads) k_engine(Dev v) {
  extern __shared__ __align__(128) unsigned char eng_smem[];
  double2* tiles = reinterpret_cast<double2*>(eng_smem);
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ IvState iv[kMaxChunkSlots];
  __shared__ int s_neg[kEngThreads];
  __shared__ int s_misc[4];
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
    s_misc[2] = 0;
  }
  __syncthreads();
  uint32_t parity[kStages];
  for (int st = 0; st < kStages; ++st) parity[st] = 0;
  run_big_chunks<MODE>(v, tiles, bars, parity, iv, s_neg, s_misc);
  run_small_chunks<MODE>(v, s_misc[2], s_neg);
  // a timed-out copy may still be in flight: wait (bounded) before exiting
  __syncthreads();
  if (tid == 0 && s_misc[2]) {
    for (int st = 0; st < kStages; ++st) mbar_wait(&bars[st], parity[st]);
  }
}

template <int MODE>
void launch_engine_mode(const Dev& v, const Grid& g, cudaStream_t s) {
  cudaFuncSetAttribute(k_engine<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEngSmem);
  const int nctas = g.nsm * kCtasPerSm;
  k_reset_chunks<<<1, 32, 0, s>>>(v);
  count_launch();
  k_count_work<MODE><<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  k_make_chunks<MODE><<<g.slot_blocks, 128, 0, s>>>(v, nctas);
  count_launch();
  k_engine<MODE><<<nctas, kEngThreads, kEngSmem, s>>>(v);
  count_launch();
}

}  // namespace

// Chunk list capacity: the front half holds big chunks (at most
// max_slots / 32 + max_nodes of them), the back half one chunk per small node.
int64_t engine_max_chunks(int64_t max_slots, int64_t max_nodes) {
  return 2 * (max_slots / 32 + max_nodes + 64);
}

void launch_engine(const Dev& v, int mode, const Grid& g, cudaStream_t s) {
  if (mode == 0)
    launch_engine_mode<MODE_ROOT>(v, g, s);
  else if (mode == 1)
    launch_engine_mode<MODE_PREREFINE>(v, g, s);
  else if (mode == 2)
    launch_engine_mode<MODE_REFINE>(v, g, s);
  else
    launch_engine_mode<MODE_FINAL>(v, g, s);
}

}  // namespace mrrr
