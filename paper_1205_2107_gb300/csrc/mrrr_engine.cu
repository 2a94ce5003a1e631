// mrrr_engine.cu -- the interval engine: bisection of many eigenvalue
// intervals on shared representations (Sec. 3.1.1: every eigenvalue is
// approximated by bisection, O(n) flops each; the eigenvalues of a cluster
// are refined to high relative accuracy on the cluster's new RRR).
//
// One launch works on one list of intervals (slot indices), built per mode
// by k_list and split into long intervals (many halvings to go) and short
// ones; the long ones run first.  The multisection width T (a power of two,
// 1..32) follows from each part's length and the number of resident lanes:
// with few intervals each gets T lanes that evaluate T interior points per
// pass over the representation (log2(T+1) bits per pass instead of one,
// which shortens the chain of dependent passes); with many intervals T = 1
// and no work is duplicated.  A warp holds 32/T lane groups and takes a
// chunk of 32/T consecutive list entries at a time, once all its groups are
// done, from the scheduler that spreads chunks over the SM sub-partitions
// (sched_next).  Every lane streams its node's (D, LLD) rows from L1/L2 with a
// register prefetch; the lanes of a group read the same rows.  The Sturm
// counts are the division-free recurrence of count_step().  Root intervals
// are first narrowed in FP32 (k_root32) and confirmed in FP64.
//
// Modes:
//   ROOT       root representation of a block, from the FP32 bracket (or,
//              if two FP64 counts reject it, the Gershgorin bracket), to the
//              classification accuracy rtol;
//   PREREFINE  the two end members of a new cluster, in the PARENT's
//              representation, to the cluster accuracy (so that the child
//              shift can be placed right at the cluster's end);
//   REFINE     cluster members moved into the CHILD's coordinates
//              (lambda - sigma_c), the bracket confirmed by two counts and
//              widened until it holds, then bisected to rtol;
//   FINAL      singletons on their node's representation, to full relative
//              accuracy (the interval can no longer be split), so that one
//              twisted factorization gives the vector (with Rayleigh-quotient
//              corrections in the vector stage: to 2^-36 only).
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {

namespace {

constexpr int kEngThreads = 256;
constexpr int kEngCtasPerSm = 2;
constexpr int kPrefetch = 8;

enum : int { MODE_ROOT = 0, MODE_PREREFINE = 1, MODE_REFINE = 2, MODE_FINAL = 3 };
enum : int { PH_BISECT = 0, PH_VERIFY = 1 };

// Whether slot w is worked on in this mode.
template <int MODE>
__device__ __forceinline__ bool slot_in_mode(const Dev& v, int64_t w, int level_begin) {
  const int st = v.state[w];
  if (MODE == MODE_FINAL) {
    if (!slot_final(st) || v.spos[w] < 0) return false;
  } else if (st != SLOT_ACTIVE) {
    return false;
  }
  const int nid = v.snode[w];
  if (nid < 0) return false;
  const Node& nd = v.node[nid];
  if (nd.depth < 0) return false;
  if (MODE == MODE_ROOT && nd.depth != 0) return false;
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && nid < level_begin) return false;
  // PREREFINE uses the parent's representation: the node's own is built later
  if (MODE != MODE_PREREFINE && nd.rep < 0) return false;
  if (v.blk[nd.block].m <= 1) return false;
  if (MODE == MODE_PREREFINE && w != nd.first && w != nd.last) return false;
  return true;
}

// Singletons whose vectors take Rayleigh-quotient corrections stop at 2^-36
// relative: one correction squares the relative error over the relative gap
// (>= 1e-4), which lands below eps.  Eigenvalues without vectors are bisected
// to full accuracy whatever the option.
constexpr double kRqRtol = 0x1p-36;

template <int MODE>
__device__ __forceinline__ double mode_rtol(const Dev& v) {
  if (MODE == MODE_FINAL) return v.rq_steps > 0 && v.Z ? kRqRtol : 2.0 * kEps;
  return MODE == MODE_ROOT || MODE == MODE_REFINE ? v.rtol : v.rtol_cluster;
}

constexpr double kLongBits = 12.0;  // bisection steps above which an interval is "long"

// Whether the interval of slot w still needs more than kLongBits halvings
// (estimated from its current bracket; ROOT brackets are always long).
template <int MODE>
__device__ __forceinline__ bool slot_is_long(const Dev& v, int64_t w) {
  if (MODE == MODE_ROOT) return true;
  double lo = v.lo[w], hi = v.hi[w];
  if (MODE == MODE_REFINE) {
    const double sig = v.node[v.snode[w]].sigma_rel;
    const double delta = 16.0 * kEps * fmax(fabs(lo), fabs(hi));
    lo = lo - sig - delta;
    hi = hi - sig + delta;
  }
  const double goal = mode_rtol<MODE>(v) * fmax(fabs(lo), fabs(hi));
  return hi - lo > ldexp(goal, (int)kLongBits);
}

// The work list: the wanted slots in slot order, long intervals from the
// front (nlist of them), short ones from the back (nlist2), built by a scan
// so that the list -- and with it which intervals share a warp -- is the same
// on every run.  Three launches: per 32-slot window the counts of its long
// and short entries, one CTA scanning them into offsets, then the writes.
template <int MODE>
__device__ __forceinline__ void window_flags(const Dev& v, int64_t w, int64_t nslots, int level_begin, bool& lng,
                                             bool& want) {
  want = w < nslots && slot_in_mode<MODE>(v, w, level_begin);
  lng = want && slot_is_long<MODE>(v, w);
}

template <int MODE>
__global__ void k_list_count(Dev v) {
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && v.ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nslots = v.ctl->nslots;
  const int level_begin = v.ctl->level_begin;
  const int64_t nwin = (nslots + 31) / 32;
  for (int64_t win = gtid() >> 5; win < nwin; win += gstride() >> 5) {
    bool lng, want;
    window_flags<MODE>(v, win * 32 + lane, nslots, level_begin, lng, want);
    const unsigned ml = __ballot_sync(0xffffffffu, lng);
    const unsigned ms = __ballot_sync(0xffffffffu, want && !lng);
    if (lane == 0) {
      v.lwin[2 * win] = __popc(ml);
      v.lwin[2 * win + 1] = __popc(ms);
    }
  }
}

constexpr int kScanThreads = 1024;

// Exclusive scan of the window counts (one CTA): each thread takes a
// contiguous run of windows, the per-thread sums are scanned in shared
// memory, then the offsets are written back in place.
__global__ void __launch_bounds__(kScanThreads) k_list_scan(Dev v, int mode) {
  if ((mode == MODE_PREREFINE || mode == MODE_REFINE) && v.ctl->done) {
    // levels enqueued past the end of the tree: an empty list, so that the
    // engine launch that follows does nothing
    if (threadIdx.x == 0) {
      v.ctl->nlist = 0;
      v.ctl->nlist2 = 0;
    }
    return;
  }
  __shared__ long long s_l[kScanThreads], s_s[kScanThreads];
  const int64_t nwin = (v.ctl->nslots + 31) / 32;
  const int64_t per = (nwin + kScanThreads - 1) / kScanThreads;
  const int64_t a = threadIdx.x * per, b = min(nwin, a + per);
  long long tl = 0, ts = 0;
  for (int64_t w = a; w < b; ++w) {
    tl += v.lwin[2 * w];
    ts += v.lwin[2 * w + 1];
  }
  s_l[threadIdx.x] = tl;
  s_s[threadIdx.x] = ts;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {  // inclusive Hillis-Steele scan
    long long xl = 0, xs = 0;
    if (threadIdx.x >= off) {
      xl = s_l[threadIdx.x - off];
      xs = s_s[threadIdx.x - off];
    }
    __syncthreads();
    s_l[threadIdx.x] += xl;
    s_s[threadIdx.x] += xs;
    __syncthreads();
  }
  long long ol = s_l[threadIdx.x] - tl, os = s_s[threadIdx.x] - ts;
  for (int64_t w = a; w < b; ++w) {
    const long long cl = v.lwin[2 * w], cs = v.lwin[2 * w + 1];
    v.lwin[2 * w] = ol;
    v.lwin[2 * w + 1] = os;
    ol += cl;
    os += cs;
  }
  if (threadIdx.x == kScanThreads - 1) {
    v.ctl->nlist = s_l[kScanThreads - 1];
    v.ctl->nlist2 = s_s[kScanThreads - 1];
    v.ctl->list_next = 0;
    v.ctl->list_next2 = 0;
  }
}

template <int MODE>
__global__ void k_list_write(Dev v) {
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && v.ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nslots = v.ctl->nslots;
  const int level_begin = v.ctl->level_begin;
  const int64_t nwin = (nslots + 31) / 32;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t win = gtid() >> 5; win < nwin; win += gstride() >> 5) {
    const int64_t w = win * 32 + lane;
    bool lng, want;
    window_flags<MODE>(v, w, nslots, level_begin, lng, want);
    const unsigned ml = __ballot_sync(0xffffffffu, lng);
    const unsigned ms = __ballot_sync(0xffffffffu, want && !lng);
    if (lng) {
      const long long at = v.lwin[2 * win] + __popc(ml & below);
      if (at < v.max_list) v.ilist[at] = w;
    } else if (want) {
      const long long at = v.lwin[2 * win + 1] + __popc(ms & below);
      if (at < v.max_list) v.ilist[v.max_list - 1 - at] = w;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 pre-bisection of the root intervals.  A root representation is
// definite (T - sigma I with sigma outside the spectrum), so rounding its
// entries to FP32 (relative perturbation 2^-24 each) moves every eigenvalue
// by a small relative amount.  The FP32 pipe issues about 60 times faster
// than the FP64 pipe on this part, so the first halvings of every root
// interval run on an FP32 copy of the rows, down to a relative width of
// root32_rtol (option prebisect_rtol, 2^-17 by default).  FP64 then
// confirms the bracket, widened by 4 root32_rtol relative and grown until
// two FP64 counts hold it, before bisecting to the classification accuracy.
// No FP32 result is trusted without that check.
constexpr float kPivmin32 = 0x1p-60f;

// FP32 rows of the root representations (D, LLD), in the eigenvector
// scratch, which is unused until the vectors are computed.
__device__ __forceinline__ float2* root32_rows(const Dev& v) { return reinterpret_cast<float2*>(v.vscr); }

__global__ void k_root32_copy(Dev v, int64_t n_total) {
  float2* r = root32_rows(v);
  for (int64_t i = gtid(); i < n_total; i += gstride()) {
    const double2 x = v.rep_dl[i];  // root representations occupy the first n_total pool rows
    r[i] = make_float2((float)x.x, (float)x.y);
  }
}

// One row of the division-free Sturm count of count_step() in FP32.
__device__ __forceinline__ void count_step32(float2 x, float tau, int pivexp, float& a, float& b, int& neg) {
  {
    float c = fmaf(x.x, b, a);
    int ci = __float_as_int(c);
    const int bi = __float_as_int(b);
    int cexp = (ci >> 23) & 0xff;
    if (cexp < pivexp) {
      c = bi < 0 ? kPivmin32 : -kPivmin32;
      ci = __float_as_int(c);
      cexp = pivexp;
    }
    neg += (ci ^ bi) < 0;
    const float an = fmaf(x.y, a, -tau * c);
    const int k = cexp - 127;
    b = __int_as_float((ci & 0x807fffff) | 0x3f800000);
    const int ai = __float_as_int(an);
    const int aexp = (ai >> 23) & 0xff;
    a = (aexp - k <= 0) ? 0.0f : (aexp - k >= 255 ? __int_as_float((ai & 0x80000000) | 0x7f000000)
                                                   : __int_as_float(ai - (k << 23)));
  }
}

// The FP32 count over m rows, kPrefetch rows loaded ahead into registers so
// that the loads stay off the recurrence's critical path.
__device__ __forceinline__ int negcount32(const float2* __restrict__ r, int m, float tau) {
  const int pivexp = (__float_as_int(kPivmin32) >> 23) & 0xff;
  float a = -tau, b = 1.0f;
  int neg = 0;
  float2 cur[kPrefetch], nxt[kPrefetch];
#pragma unroll
  for (int u = 0; u < kPrefetch; ++u) cur[u] = u < m ? __ldg(r + u) : make_float2(1.0f, 0.0f);
  for (int i0 = 0; i0 < m; i0 += kPrefetch) {
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int i = i0 + kPrefetch + u;
      nxt[u] = i < m ? __ldg(r + i) : make_float2(1.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u)
      if (i0 + u < m) count_step32(cur[u], tau, pivexp, a, b, neg);
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) cur[u] = nxt[u];
  }
  return neg;
}

// Per-interval state, replicated in every lane of the interval's group.
struct Iv {
  double lo, hi, plo, phi, delta, atol, pivmin;
  const double2* dl;
  int64_t slot;
  int j, m, phase, tries, steps, pivexp;
};

template <int MODE>
__device__ __forceinline__ void iv_load(const Dev& v, int64_t w, Iv& q) {
  const Node nd = v.node[v.snode[w]];
  const Block bk = v.blk[nd.block];
  const Node rn = MODE == MODE_PREREFINE ? v.node[nd.parent] : nd;  // representation used
  q.slot = w;
  q.j = v.sj[w];
  q.m = bk.m;
  q.dl = v.rep_dl + rn.rep;
  q.pivmin = rn.pivmin;
  q.pivexp = exp_field(rn.pivmin);
  q.atol = 4.0 * rn.pivmin;
  q.steps = 0;
  q.tries = 0;
  q.phase = PH_BISECT;
  if (MODE == MODE_ROOT) {
    // the FP32 bracket, widened, confirmed by two FP64 counts (and widened
    // further until they hold), inside the block's Gershgorin bracket
    q.plo = fmax(v.lo[w], bk.gl);
    q.phi = fmin(v.hi[w], bk.gu);
    q.delta = 4.0 * v.root32_rtol * fmax(fabs(q.plo), fabs(q.phi)) + (q.phi - q.plo) + 4.0 * rn.pivmin;
    q.lo = fmax(q.plo - q.delta, bk.gl);
    q.hi = fmin(q.phi + q.delta, bk.gu);
    q.phase = PH_VERIFY;
  } else if (MODE == MODE_REFINE) {
    // the parent bracket in child coordinates, widened by delta until two
    // counts confirm it
    q.plo = v.lo[w] - nd.sigma_rel;
    q.phi = v.hi[w] - nd.sigma_rel;
    q.delta = 16.0 * kEps * fmax(fabs(v.lo[w]), fabs(v.hi[w])) + 4.0 * rn.pivmin;
    q.lo = q.plo - q.delta;
    q.hi = q.phi + q.delta;
    q.phase = PH_VERIFY;
  } else {
    q.lo = v.lo[w];
    q.hi = v.hi[w];
  }
}

// Evaluation point of lane pos of a run of P lanes that share one bracket
// (one interval's T lanes, or the lanes of consecutive intervals of one node
// whose brackets coincide); false when the lane has no point this pass.
// Confirming a bracket needs its two ends: with P >= 2 both in one pass,
// with a single lane one end per pass (lower, then upper).
__device__ __forceinline__ bool iv_tau(const Iv& q, int P, int pos, double& tau) {
  if (q.phase == PH_VERIFY) {
    if (P >= 2) {
      tau = pos == 0 ? q.lo : q.hi;
      return pos < 2;
    }
    tau = (q.tries & 1) ? q.hi : q.lo;
    return true;
  }
  tau = q.lo + (q.hi - q.lo) * ((double)(pos + 1) / (double)(P + 1));
  return true;
}

// Update after a pass over a run of P points.  kfirst: index of the first
// point whose count is >= j (P when none); c_lo, c_hi: the counts at the
// run's points 0 and 1 (with P = 1, c_lo is the single count).  Returns true
// when the interval is finished.
template <int MODE>
__device__ __forceinline__ bool iv_update(const Dev& v, int P, double rtol, int maxsteps, int kfirst, int c_lo,
                                          int c_hi, Iv& q) {
  if (q.phase == PH_VERIFY) {
    bool ok_lo, ok_hi, decided;
    if (P >= 2) {
      ok_lo = c_lo <= q.j - 1;
      ok_hi = c_hi >= q.j;
      decided = true;
      q.tries &= ~1;
    } else if ((q.tries & 1) == 0) {  // lower end just counted
      ok_lo = c_lo <= q.j - 1;
      ok_hi = true;
      decided = !ok_lo;
      if (ok_lo) q.tries |= 1;  // next: upper end
    } else {
      ok_lo = true;
      ok_hi = c_lo >= q.j;
      decided = true;
      q.tries &= ~1;
    }
    if (decided) {
      if (ok_lo && ok_hi) {
        q.phase = PH_BISECT;
        if (converged(q.lo, q.hi, rtol, q.atol)) return true;
      } else {
        q.tries = (q.tries & ~1) + 2;
        q.delta *= 4.0;
        q.lo = q.plo - q.delta;
        q.hi = q.phi + q.delta;
        if (MODE == MODE_ROOT) {  // never beyond the confirmed Gershgorin bracket
          const Block& bk = v.blk[v.node[v.snode[q.slot]].block];
          q.lo = fmax(q.lo, bk.gl);
          q.hi = fmin(q.hi, bk.gu);
        }
        if (q.tries > 48) {  // give up confirming; bisect what we have
          set_status(v.ctl, MRRR_ERR_NOCONV);
          diag(v.ctl, DIAG_REFINE_BRACKET);
          q.phase = PH_BISECT;
        }
      }
    }
    return false;
  }
  const int k = kfirst;
  const double nlo = k > 0 ? q.lo + (q.hi - q.lo) * ((double)k / (double)(P + 1)) : q.lo;
  const double nhi = k < P ? q.lo + (q.hi - q.lo) * ((double)(k + 1) / (double)(P + 1)) : q.hi;
  const bool stuck = !(nlo < nhi) || (nlo == q.lo && nhi == q.hi);
  q.lo = nlo;
  q.hi = nhi;
  ++q.steps;
  if (stuck || converged(q.lo, q.hi, rtol, q.atol) || q.steps >= maxsteps) {
    if (q.steps >= maxsteps && !stuck && !converged(q.lo, q.hi, rtol, q.atol)) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, MODE == MODE_ROOT ? DIAG_ROOT_BISECT : DIAG_REFINE_BISECT);
    }
    return true;
  }
  return false;
}

// Sturm count of one lane over its m rows; the loop runs to m_all (the
// longest representation in the warp) so that the warp stays converged.
// Rows are prefetched kPrefetch at a time into registers.
__device__ __forceinline__ int lane_count(const double2* __restrict__ dl, int m, int m_all, double tau, int pivexp,
                                          double pivmin, bool act) {
  double a = -tau, b = 1.0;
  int neg = 0;
  const int mm = act ? m : 0;
  double2 cur[kPrefetch], nxt[kPrefetch];
#pragma unroll
  for (int u = 0; u < kPrefetch; ++u) cur[u] = u < mm ? __ldg(dl + u) : make_double2(1.0, 0.0);
  for (int i0 = 0; i0 < m_all; i0 += kPrefetch) {
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int i = i0 + kPrefetch + u;
      nxt[u] = i < mm ? __ldg(dl + i) : make_double2(1.0, 0.0);
    }
    if (i0 < mm) {
#pragma unroll
      for (int u = 0; u < kPrefetch; ++u)
        if (i0 + u < mm) count_step(cur[u].x, cur[u].y, tau, pivexp, pivmin, a, b, neg);
    }
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) cur[u] = nxt[u];
  }
  return neg;
}

// Multisection width for a list of nlist intervals: the largest power of
// two T <= 32 with T nlist <= lanes_total.  lanes_total is one warp per SM
// sub-partition (times width_scale): each sub-partition's FP64 unit takes
// about 64 cycles per warp instruction whatever the number of active lanes,
// and one warp's dependent count already keeps it busy, so more points per
// interval only pay while they fill sub-partitions that would otherwise idle.
__device__ __forceinline__ int width_for(long long nlist, long long lanes_total, int fixed) {
  if (fixed > 0) return fixed;
  int T = 1;
  while (T < 32 && 2LL * T * nlist <= lanes_total) T *= 2;
  return T;
}

// Starting brackets for the FP32 bisection: for every root block of at
// least kGridMinRows rows, FP32 counts at kGridPoints - 1 evenly spaced
// interior points of its Gershgorin bracket (one thread each), kept at
// 2 row0 of the block in an array of 2 ints per row of T (blocks never
// overlap).  The grid depends on the block alone, so an interval's starting
// bracket is the same whichever call, batch or slice computes it.  An interval then starts from the grid cell whose
// counts bracket its index instead of the whole Gershgorin bracket: about
// ten halvings fewer.  Counts that rounding made non-monotone can only give
// a wrong cell, which the FP64 check of the bracket widens as it would any
// FP32 result.
constexpr int kGridPoints = 1024;
constexpr int kGridMinRows = 512;

__device__ __forceinline__ float grid_point(float gl, float gu, int g) {
  return gl + (gu - gl) * ((float)g / (float)kGridPoints);
}

__device__ __forceinline__ int* grid_counts(const Dev& v, int64_t row0) { return v.rgrid + 2 * row0; }

__global__ void __launch_bounds__(kGridPoints) k_root32_grid(Dev v) {
  const float2* rows = root32_rows(v);
  const int nblocks = v.ctl->nblocks;
  for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const Block bk = v.blk[b];
    if (bk.m < kGridMinRows || bk.je < bk.js) continue;
    const int g = threadIdx.x + 1;
    if (g < kGridPoints)
      grid_counts(v, bk.row0)[g] =
          negcount32(rows + bk.row0, bk.m, grid_point((float)bk.gl, (float)bk.gu, g));
  }
}

// FP32 bisection of the root intervals from their blocks' Gershgorin
// brackets; the results go to lo/hi for the FP64 check.  Chunks spread over
// the SM sub-partitions by the scheduler, cut like the engine's lists: whole
// waves of chunks with one interval per lane, and a remainder whose few
// intervals take T lanes each (T points per pass, the first point whose
// count reaches j and the one before it bracket the eigenvalue).  With a
// fixed schedule (slices, options) every interval takes one lane, so that
// its bracket does not depend on the list it is in.
constexpr int kRoot32CtasPerSm = 4;

__global__ void __launch_bounds__(128) k_root32(Dev v) {
  const int lane = threadIdx.x & 31;
  const long long nlist = min(v.ctl->nlist, (long long)v.max_list);
  const float2* rows = root32_rows(v);
  const float width = (float)v.root32_rtol;
  const long long wave = (long long)v.nsm * 4 * 32;
  const bool fixed = v.fixed_width > 0;
  const long long nmain = fixed ? nlist : (nlist / wave) * wave;
  const int T_rest = fixed ? 1 : width_for(nlist - nmain, wave, 0);
  const long long g_rest = 32 / T_rest;
  const long long nch_main = (nmain + 31) / 32;
  const long long nchunks = nch_main + (nlist - nmain + g_rest - 1) / g_rest;
  const long long total_warps = (long long)gridDim.x * (blockDim.x / 32);
  const long long rank = sched_rank(v);
  bool first = true;
  for (;;) {
    const long long chunk = sched_next(v, nchunks, total_warps, rank, first);
    if (chunk < 0) break;
    const bool is_main = chunk < nch_main;
    const int T = is_main ? 1 : T_rest;
    const int pt = lane % T, lead = lane - pt;
    const long long item = is_main ? chunk * 32 + lane : nmain + (chunk - nch_main) * g_rest + lane / T;
    const bool mine = is_main ? item < nmain : item < nlist;
    int64_t w = 0, row0 = 0;
    int j = 0, m = 0;
    float lo = 0.f, hi = 0.f;
    if (mine) {
      w = v.ilist[item];
      const Block bk = v.blk[v.node[v.snode[w]].block];
      j = v.sj[w];
      m = bk.m;
      row0 = bk.row0;
      lo = (float)bk.gl;
      hi = (float)bk.gu;
      if (m >= kGridMinRows) {  // the grid cell whose counts bracket j
        const int* c = grid_counts(v, row0);
        int a = 1, z = kGridPoints;  // first point g in [1, kGridPoints) with count >= j, else kGridPoints
        while (a < z) {
          const int mid = (a + z) >> 1;
          if (c[mid] >= j)
            z = mid;
          else
            a = mid + 1;
        }
        const float gl = (float)bk.gl, gu = (float)bk.gu;
        lo = grid_point(gl, gu, a - 1);
        hi = a < kGridPoints ? grid_point(gl, gu, a) : gu;
      }
    }
    bool have = mine;
    for (int step = 0; step < 48; ++step) {
      if (have && hi - lo <= width * fmaxf(fabsf(lo), fabsf(hi))) have = false;
      const float tau = lo + (hi - lo) * ((float)(pt + 1) / (float)(T + 1));
      // the group stops when a point is not strictly inside its bracket
      bool inside = !have || (tau > lo && tau < hi);
      for (int o = 1; o < T; o <<= 1) inside &= __shfl_xor_sync(0xffffffffu, inside, o) != 0;
      if (!inside) have = false;
      if (!__any_sync(0xffffffffu, have)) break;
      const int cnt = have ? negcount32(rows + row0, m, tau) : 0;
      int kfirst = T;
      for (int k = T - 1; k >= 0; --k)
        if (__shfl_sync(0xffffffffu, cnt, lead + k) >= j) kfirst = k;
      if (have) {
        const float nlo = kfirst > 0 ? lo + (hi - lo) * ((float)kfirst / (float)(T + 1)) : lo;
        const float nhi = kfirst < T ? lo + (hi - lo) * ((float)(kfirst + 1) / (float)(T + 1)) : hi;
        lo = nlo;
        hi = nhi;
      }
    }
    if (mine && pt == 0) {
      v.lo[w] = (double)lo;
      v.hi[w] = (double)hi;
    }
  }
}

// How one engine launch cuts its list into chunks (one warp's intervals
// each): the long intervals first, then the short ones, each part with the
// width its own length allows.  Long intervals at width 1 are split into
// whole waves (every SM sub-partition gets the same number of full chunks)
// and a remainder that takes the width its own length allows: its few
// intervals then finish in fewer, wider passes on every sub-partition
// instead of a third (or later) full-length chunk on some of them.
struct ChunkPlan {
  long long nlong, nshort, nmain, nch_main, nch_long, nchunks;
  int T_rest, T_short;
};

__device__ __forceinline__ ChunkPlan chunk_plan(const Dev& v) {
  ChunkPlan c;
  c.nlong = min(v.ctl->nlist, (long long)v.max_list);
  c.nshort = min(v.ctl->nlist2, (long long)v.max_list - c.nlong);
  const long long lanes_total = (long long)((double)v.nsm * 4 * 32 * v.width_scale);
  const int T_long = width_for(c.nlong, lanes_total, v.fixed_width);
  const long long wave = (long long)v.nsm * 4 * 32;
  c.nmain = (T_long == 1 && v.fixed_width == 0) ? (c.nlong / wave) * wave : 0;
  c.T_rest = width_for(c.nlong - c.nmain, lanes_total, v.fixed_width);
  c.T_short = width_for(c.nshort, lanes_total, v.fixed_width);
  const long long g_rest = 32 / c.T_rest, g_short = 32 / c.T_short;
  c.nch_main = c.nmain / 32;
  c.nch_long = c.nch_main + (c.nlong - c.nmain + g_rest - 1) / g_rest;
  c.nchunks = c.nch_long + (c.nshort + g_short - 1) / g_short;
  return c;
}

// The order of the main chunks, in the second half of the list's window
// offsets (free once the list is written); the first half holds each
// chunk's estimate while the order is built.
__device__ __forceinline__ int64_t* chunk_perm(const Dev& v) { return v.lwin + (v.max_slots + 31) / 32; }

// Halvings an interval still needs in this mode (0..63), from its bracket.
template <int MODE>
__device__ __forceinline__ int halvings_left(const Dev& v, int64_t w) {
  double lo = v.lo[w], hi = v.hi[w];
  if (MODE == MODE_REFINE) {
    const double sig = v.node[v.snode[w]].sigma_rel;
    lo -= sig;
    hi -= sig;
  }
  const double goal = mode_rtol<MODE>(v) * fmax(fabs(lo), fabs(hi));
  const double wdt = hi - lo;
  if (!(wdt > goal) || !(goal > 0.0)) return 0;
  return max(0, min(63, ilogb(wdt) - ilogb(goal) + 1));
}

// Cluster modes only (whose chunks' lengths vary with the gaps inside
// their clusters): one CTA sorts the main chunks, four consecutive ones at a
// time (one SM's share of a wave, so that an SM's warps keep reading
// neighbouring representation rows), by the most halvings any of their
// intervals needs, longest first, and deals these quads to the SMs in a
// snake (wave 0 left to right, wave 1 right to left, ...), so that every SM
// pairs long work with short.  The engine's scheduler hands chunk position
// r to the warp of rank r, which sits on sub-partition r mod 4 of SM
// (r mod (4 x SMs)) / 4.  Only the placement of chunks changes: each
// chunk's intervals, and so the results, stay the same.
constexpr int kOrderThreads = 1024;

template <int MODE>
__host__ __device__ constexpr bool ordered_mode() {
  return MODE == MODE_PREREFINE || MODE == MODE_REFINE;
}

template <int MODE>
__global__ void __launch_bounds__(kOrderThreads) k_chunk_order(Dev v) {
  if (v.ctl->done) return;
  __shared__ unsigned long long hist[64];
  const ChunkPlan cp = chunk_plan(v);
  const long long nquad = cp.nch_main / 4;
  if (nquad <= 0) return;
  int64_t* est = v.lwin;
  int64_t* perm = chunk_perm(v);
  if (threadIdx.x < 64) hist[threadIdx.x] = 0;
  __syncthreads();
  for (long long qd = threadIdx.x; qd < nquad; qd += kOrderThreads) {
    int e = 0;
    for (int i = 0; i < 128; ++i) e = max(e, halvings_left<MODE>(v, v.ilist[qd * 128 + i]));
    est[qd] = e;
    atomicAdd(&hist[e], 1ull);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // start of each bucket, the largest first
    unsigned long long at = 0;
    for (int b = 63; b >= 0; --b) {
      const unsigned long long n = hist[b];
      hist[b] = at;
      at += n;
    }
  }
  __syncthreads();
  const long long nsm = v.nsm;
  for (long long qd = threadIdx.x; qd < nquad; qd += kOrderThreads) {
    const long long k = (long long)atomicAdd(&hist[est[qd]], 1ull);
    const long long wv = k / nsm, i = k % nsm;
    const long long sm = (wv & 1) ? nsm - 1 - i : i;
    for (int j = 0; j < 4; ++j) perm[wv * 4 * nsm + 4 * sm + j] = 4 * qd + j;
  }
}

// Phase 0 drains the long intervals (front of the list), phase 1 the short
// ones (back of the list), each with the width that its own length allows;
// a warp moves on to phase 1 as soon as the long list is exhausted for it.
//
// Pooled points: consecutive lane groups of a warp whose intervals lie on the
// same representation with the same bracket (cluster members refined from a
// common parent bracket) form a run, and the run's k T lanes evaluate k T
// points spread over that bracket.  A count at any point brackets every
// member at once, so k members sharing a bracket narrow it (k T + 1)-fold per
// pass instead of (T + 1)-fold each; each member then keeps the pair of
// neighbouring points that brackets its own index.  With a fixed width
// (options) runs are single groups: each interval's passes depend on nothing
// but itself.
template <int MODE>
__global__ void __launch_bounds__(kEngThreads, kEngCtasPerSm) k_engine(Dev v) {
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && v.ctl->done) return;
  const int lane = threadIdx.x & 31;
  const ChunkPlan cp = chunk_plan(v);
  const long long nlong = cp.nlong, nshort = cp.nshort, nmain = cp.nmain;
  const long long nch_main = cp.nch_main, nch_long = cp.nch_long, nchunks = cp.nchunks;
  const int T_rest = cp.T_rest, T_short = cp.T_short;
  const int64_t* perm = chunk_perm(v);
  const long long total_warps = (long long)gridDim.x * (blockDim.x / 32);
  const long long rank = sched_rank(v);
  const double rtol = mode_rtol<MODE>(v);
  const int maxsteps = v.max_bisect;
  const bool pool = v.fixed_width == 0 && MODE != MODE_ROOT && MODE != MODE_FINAL;
  const unsigned at_or_below = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  unsigned long long n_counts = 0, n_rows = 0, n_passes = 0;
  bool first = true;
  for (;;) {
    // the warp's next chunk (consecutive list entries: neighbouring slots, so
    // the same node or problem: the lanes share row lengths and often rows)
    const long long claimed = sched_next(v, nchunks, total_warps, rank, first);
    if (claimed < 0) break;
    // cluster modes: main chunks in the order k_chunk_order chose (longest
    // quads first, snaked over the SMs); everything else in list order
    const long long chunk = (ordered_mode<MODE>() && claimed < nch_main) ? perm[claimed] : claimed;
    const bool is_long = chunk < nch_long;
    const bool is_main = chunk < nch_main;
    const int T = is_main ? 1 : is_long ? T_rest : T_short;
    const int pt = lane % T;
    const int groups = 32 / T, grp = lane / T;
    const long long item = is_main   ? chunk * 32 + lane
                           : is_long ? nmain + (chunk - nch_main) * groups + grp
                                     : (chunk - nch_long) * groups + grp;
    const long long nlist = is_long ? nlong : nshort;
    Iv q{};
    bool have = false;
    if (item < nlist) {
      iv_load<MODE>(v, v.ilist[is_long ? item : v.max_list - 1 - item], q);
      if (q.phase == PH_BISECT && converged(q.lo, q.hi, rtol, q.atol)) {
        if (pt == 0) {  // already converged on entry
          v.lo[q.slot] = q.lo;
          v.hi[q.slot] = q.hi;
        }
      } else {
        have = true;
      }
    }
    while (__any_sync(0xffffffffu, have)) {
      // runs: a group joins the run of the group before it when both hold an
      // interval on the same rows, in the same phase, with the same bracket
      bool join = false;
      {
        const double plo = __shfl_up_sync(0xffffffffu, q.lo, T);
        const double phi = __shfl_up_sync(0xffffffffu, q.hi, T);
        const long long pdl = __shfl_up_sync(0xffffffffu, (long long)q.dl, T);
        const int pph = __shfl_up_sync(0xffffffffu, q.phase, T);
        const int phave = __shfl_up_sync(0xffffffffu, (int)have, T);
        join = pool && grp > 0 && have && phave && pdl == (long long)q.dl && pph == q.phase && plo == q.lo &&
               phi == q.hi;
      }
      const unsigned starts = __ballot_sync(0xffffffffu, pt == 0 && !join);
      const int run_lead = 31 - __clz(starts & at_or_below);
      const unsigned above = starts & ~at_or_below;
      const int P = (above ? __ffs(above) - 1 : 32) - run_lead;
      const int pos = lane - run_lead;
      double tau = 0.0;
      bool act = have;
      if (act) act = iv_tau(q, P, pos, tau);
      int m_all = act ? q.m : 0;
      for (int o = 16; o; o >>= 1) m_all = max(m_all, __shfl_xor_sync(0xffffffffu, m_all, o));
      const int neg = lane_count(q.dl, q.m, m_all, tau, q.pivexp, q.pivmin, act);
      {
        const unsigned am = __ballot_sync(0xffffffffu, act);
        n_counts += __popc(am);
        n_rows += (unsigned long long)__popc(am) * (unsigned long long)m_all;
        ++n_passes;
      }
      // each member's first point with count >= j, by bisection over the
      // run's points (P <= 32, six steps); the bracket found is valid even
      // if rounding made the counts non-monotone: count < j at point kfirst-1
      // and count >= j at point kfirst
      int klo = 0, khi = P;
      for (int it = 0; it < 6; ++it) {
        const int mid = (klo + khi) >> 1;
        const int c = __shfl_sync(0xffffffffu, neg, run_lead + min(mid, P - 1));
        if (klo < khi) {
          if (c >= q.j)
            khi = mid;
          else
            klo = mid + 1;
        }
      }
      const int c_lo = __shfl_sync(0xffffffffu, neg, run_lead);
      const int c_hi = __shfl_sync(0xffffffffu, neg, P >= 2 ? run_lead + 1 : run_lead);
      if (have && iv_update<MODE>(v, P, rtol, maxsteps, klo, c_lo, c_hi, q)) {
        if (pt == 0) {
          v.lo[q.slot] = q.lo;
          v.hi[q.slot] = q.hi;
        }
        have = false;
      }
    }
  }
  if (lane == 0 && n_passes) {
    atomicAdd(&v.ctl->eng_counts[MODE], n_counts);
    atomicAdd(&v.ctl->eng_rows[MODE], n_rows);
    atomicAdd(&v.ctl->eng_passes[MODE], n_passes);
  }
}

// Before the cluster stages: members of a new node whose brackets overlap
// take the union of their brackets, so that the engine can pool their points
// (the union contains each member's eigenvalue; REFINE confirms it in the
// child anyway).  PREREFINE works on the node's two ends only; REFINE on
// every member.  One thread per node of the current level.
template <int MODE>
__global__ void k_share_brackets(Dev v) {
  if (v.ctl->done) return;
  const int begin = v.ctl->level_begin;
  const int end = min(v.ctl->nodes, v.max_nodes);
  for (int64_t id = begin + gtid(); id < end; id += gstride()) {
    const Node nd = v.node[id];
    if (nd.depth < 0 || (MODE == MODE_REFINE && nd.rep < 0)) continue;
    if (MODE == MODE_PREREFINE) {
      const int64_t f = nd.first, l = nd.last;
      if (l > f && v.hi[f] >= v.lo[l]) {
        const double a = fmin(v.lo[f], v.lo[l]), b = fmax(v.hi[f], v.hi[l]);
        v.lo[f] = v.lo[l] = a;
        v.hi[f] = v.hi[l] = b;
      }
      continue;
    }
    int64_t s0 = nd.first;
    double a = v.lo[s0], b = v.hi[s0];
    for (int64_t w = nd.first + 1; w <= nd.last + 1; ++w) {
      const bool close = w > nd.last || v.lo[w] > b;
      if (close) {
        if (w - 1 > s0)
          for (int64_t t = s0; t < w; ++t) {
            v.lo[t] = a;
            v.hi[t] = b;
          }
        if (w <= nd.last) {
          s0 = w;
          a = v.lo[w];
          b = v.hi[w];
        }
      } else {
        a = fmin(a, v.lo[w]);
        b = fmax(b, v.hi[w]);
      }
    }
  }
}

template <int MODE>
void launch_engine_mode(const Dev& v, const Grid& g, cudaStream_t s, int64_t n_total) {
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && v.fixed_width == 0) {
    k_share_brackets<MODE><<<g.slot_blocks, 128, 0, s>>>(v);
    count_launch();
  }
  k_list_count<MODE><<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  k_list_scan<<<1, kScanThreads, 0, s>>>(v, MODE);
  count_launch();
  k_list_write<MODE><<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  if (MODE == MODE_ROOT) {
    k_root32_copy<<<g.slot_blocks, 256, 0, s>>>(v, n_total);
    count_launch();
    k_sched_reset<<<1, kSchedSlots, 0, s>>>(v);
    count_launch();
    k_root32_grid<<<g.slot_blocks, kGridPoints, 0, s>>>(v);
    count_launch();
    k_root32<<<g.nsm * kRoot32CtasPerSm, 128, 0, s>>>(v);
    count_launch();
  }
  if (ordered_mode<MODE>()) {
    k_chunk_order<MODE><<<1, kOrderThreads, 0, s>>>(v);
    count_launch();
  }
  k_sched_reset<<<1, kSchedSlots, 0, s>>>(v);
  count_launch();
  k_engine<MODE><<<g.nsm * max(1, min(kEngCtasPerSm, v.engine_ctas)), kEngThreads, 0, s>>>(v);
  count_launch();
}

}  // namespace

__global__ void k_sched_reset(Dev v) {
  for (int i = threadIdx.x; i < kSchedSlots; i += blockDim.x) v.sched_cnt[i] = 0;
  if (threadIdx.x == 0) {
    v.ctl->sched_gen += 1;
    v.ctl->sched_dyn = 0;
    v.ctl->sched_cleanup = 0;
  }
}

void launch_engine(const Dev& v, int mode, const Grid& g, cudaStream_t s, int64_t n_total) {
  if (mode == 0)
    launch_engine_mode<MODE_ROOT>(v, g, s, n_total);
  else if (mode == 1)
    launch_engine_mode<MODE_PREREFINE>(v, g, s, n_total);
  else if (mode == 2)
    launch_engine_mode<MODE_REFINE>(v, g, s, n_total);
  else
    launch_engine_mode<MODE_FINAL>(v, g, s, n_total);
}

}  // namespace mrrr
