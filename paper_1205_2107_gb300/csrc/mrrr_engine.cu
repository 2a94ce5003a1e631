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
// and no work is duplicated.  A warp holds 32/T lane groups and takes 32/T
// consecutive list entries at a time (atomic counter) once all its groups
// are done.  Every lane streams its node's (D, LLD) rows from L1/L2 with a
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
//              twisted factorization gives the vector.
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

__global__ void k_list_reset(Dev v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    v.ctl->nlist = 0;
    v.ctl->list_next = 0;
    v.ctl->nlist2 = 0;
    v.ctl->list_next2 = 0;
  }
}

template <int MODE>
__device__ __forceinline__ double mode_rtol(const Dev& v) {
  return MODE == MODE_ROOT || MODE == MODE_REFINE ? v.rtol : MODE == MODE_FINAL ? 2.0 * kEps : v.rtol_cluster;
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

// Compaction of the wanted slots into the list (warp-aggregated appends):
// long intervals from the front (nlist), short ones from the back (nlist2).
template <int MODE>
__global__ void k_list(Dev v) {
  if ((MODE == MODE_PREREFINE || MODE == MODE_REFINE) && v.ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nslots = v.ctl->nslots;
  const int level_begin = v.ctl->level_begin;
  for (int64_t w0 = gtid() - lane; w0 < nslots; w0 += gstride()) {
    const int64_t w = w0 + lane;
    const bool want = w < nslots && slot_in_mode<MODE>(v, w, level_begin);
    const bool lng = want && slot_is_long<MODE>(v, w);
    const unsigned ml = __ballot_sync(0xffffffffu, lng);
    const unsigned ms = __ballot_sync(0xffffffffu, want && !lng);
    if (!(ml | ms)) continue;
    unsigned long long bl = 0, bs = 0;
    if (lane == 0 && ml) bl = atomicAdd((unsigned long long*)&v.ctl->nlist, (unsigned long long)__popc(ml));
    if (lane == 0 && ms) bs = atomicAdd((unsigned long long*)&v.ctl->nlist2, (unsigned long long)__popc(ms));
    bl = __shfl_sync(0xffffffffu, bl, 0);
    bs = __shfl_sync(0xffffffffu, bs, 0);
    const unsigned below = (1u << lane) - 1u;
    if (lng) {
      const long long at = (long long)bl + __popc(ml & below);
      if (at < v.max_list) v.ilist[at] = w;
    } else if (want) {
      const long long at = (long long)bs + __popc(ms & below);
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
// kRoot32Width.  FP64 then confirms the bracket, widened by kRoot32Margin
// relative and grown until two FP64 counts hold it, before bisecting to the
// classification accuracy.  No FP32 result is trusted without that check.
constexpr float kRoot32Width = 0x1p-13f;
constexpr double kRoot32Margin = 0x1p-11;
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

// The division-free Sturm count of count_step() in FP32.
__device__ __forceinline__ int negcount32(const float2* __restrict__ r, int m, float tau) {
  const int pivexp = (__float_as_int(kPivmin32) >> 23) & 0xff;
  float a = -tau, b = 1.0f;
  int neg = 0;
  for (int i = 0; i < m; ++i) {
    const float2 x = r[i];
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
  return neg;
}

// One thread per root interval of the list: FP32 bisection from the block's
// Gershgorin bracket; the result goes to lo/hi for the FP64 check.
__global__ void k_root32(Dev v) {
  const long long nlist = min(v.ctl->nlist, (long long)v.max_list);
  const float2* rows = root32_rows(v);
  for (long long it = gtid(); it < nlist; it += gstride()) {
    const int64_t w = v.ilist[it];
    const Node nd = v.node[v.snode[w]];
    const Block bk = v.blk[nd.block];
    const int j = v.sj[w];
    float lo = (float)bk.gl, hi = (float)bk.gu;
    for (int step = 0; step < 48; ++step) {
      if (hi - lo <= kRoot32Width * fmaxf(fabsf(lo), fabsf(hi))) break;
      const float mid = 0.5f * (lo + hi);
      if (!(mid > lo && mid < hi)) break;
      if (negcount32(rows + bk.row0, bk.m, mid) >= j)
        hi = mid;
      else
        lo = mid;
    }
    v.lo[w] = (double)lo;
    v.hi[w] = (double)hi;
  }
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
    q.delta = kRoot32Margin * fmax(fabs(q.plo), fabs(q.phi)) + (q.phi - q.plo) + 4.0 * rn.pivmin;
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

// Evaluation point of lane pt (of T) of an interval in this pass; false when
// the lane has no point this pass.
__device__ __forceinline__ bool iv_tau(const Iv& q, int T, int pt, double& tau) {
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

// Update after a pass.  kfirst: index of the first point whose count is
// >= j (T when none); c0, c1: the counts of points 0 and 1.  Returns true
// when the interval is finished.
template <int MODE>
__device__ __forceinline__ bool iv_update(const Dev& v, int T, double rtol, int maxsteps, int kfirst, int c0,
                                          int c1, Iv& q) {
  if (q.phase == PH_VERIFY) {
    bool ok_lo, ok_hi, decided;
    if (T >= 2) {
      ok_lo = c0 <= q.j - 1;
      ok_hi = c1 >= q.j;
      decided = true;
    } else if ((q.tries & 1) == 0) {  // lower end just counted
      ok_lo = c0 <= q.j - 1;
      ok_hi = true;
      decided = !ok_lo;
      if (ok_lo) q.tries |= 1;  // next: upper end
    } else {
      ok_lo = true;
      ok_hi = c0 >= q.j;
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
  const double nlo = k > 0 ? q.lo + (q.hi - q.lo) * ((double)k / (double)(T + 1)) : q.lo;
  const double nhi = k < T ? q.lo + (q.hi - q.lo) * ((double)(k + 1) / (double)(T + 1)) : q.hi;
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
// two T <= 32 with 2 T nlist <= lanes_total.
__device__ __forceinline__ int width_for(long long nlist, long long lanes_total) {
  int T = 1;
  while (T < 32 && 2LL * T * nlist <= lanes_total) T *= 2;
  return T;
}

// Phase 0 drains the long intervals (front of the list), phase 1 the short
// ones (back of the list), each with the width that its own length allows;
// a warp moves on to phase 1 as soon as the long list is exhausted for it.
template <int MODE>
__global__ void __launch_bounds__(kEngThreads, kEngCtasPerSm) k_engine(Dev v) {
  const int lane = threadIdx.x & 31;
  const long long nlong = min(v.ctl->nlist, (long long)v.max_list);
  const long long nshort = min(v.ctl->nlist2, (long long)v.max_list - nlong);
  const long long lanes_total = (long long)((double)gridDim.x * blockDim.x * v.width_scale);
  const double rtol = mode_rtol<MODE>(v);
  const int maxsteps = v.max_bisect;
  for (int phase = 0; phase < 2; ++phase) {
    const long long nlist = phase == 0 ? nlong : nshort;
    if (nlist == 0) continue;
    unsigned long long* next = phase == 0 ? (unsigned long long*)&v.ctl->list_next
                                          : (unsigned long long*)&v.ctl->list_next2;
    const int T = width_for(nlist, lanes_total);
    const int pt = lane % T, leader = lane - pt;
    const unsigned gbits = T == 32 ? 0xffffffffu : (((1u << T) - 1u) << leader);
    const int groups = 32 / T, grp = lane / T;
    Iv q{};
    bool have = false, exhausted = false;
    for (;;) {
      // when every group of the warp is done, the warp takes the next
      // `groups` consecutive list entries (neighbouring slots: the same node
      // or problem, so the lanes share row lengths and often rows); an
      // interval already converged on entry is finished at once
      while (!exhausted && !__any_sync(0xffffffffu, have)) {
        long long base = 0;
        if (lane == 0) base = (long long)atomicAdd(next, (unsigned long long)groups);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nlist) {
          exhausted = true;
          break;
        }
        const long long item = base + grp;
        if (item < nlist) {
          iv_load<MODE>(v, v.ilist[phase == 0 ? item : v.max_list - 1 - item], q);
          if (q.phase == PH_BISECT && converged(q.lo, q.hi, rtol, q.atol)) {
            if (pt == 0) {
              v.lo[q.slot] = q.lo;
              v.hi[q.slot] = q.hi;
            }
          } else {
            have = true;
          }
        }
      }
      if (!__any_sync(0xffffffffu, have)) break;
      double tau = 0.0;
      bool act = have;
      if (act) act = iv_tau(q, T, pt, tau);
      int m_all = act ? q.m : 0;
      for (int o = 16; o; o >>= 1) m_all = max(m_all, __shfl_xor_sync(0xffffffffu, m_all, o));
      const int neg = lane_count(q.dl, q.m, m_all, tau, q.pivexp, q.pivmin, act);
      // the group's counts: first point with count >= j, and points 0 and 1
      const unsigned ge = __ballot_sync(0xffffffffu, act && neg >= q.j) & gbits;
      const int kfirst = ge ? (__ffs(ge) - 1 - leader) : T;
      const int c0 = __shfl_sync(0xffffffffu, neg, leader);
      const int c1 = __shfl_sync(0xffffffffu, neg, T >= 2 ? leader + 1 : leader);
      if (have && iv_update<MODE>(v, T, rtol, maxsteps, kfirst, c0, c1, q)) {
        if (pt == 0) {
          v.lo[q.slot] = q.lo;
          v.hi[q.slot] = q.hi;
        }
        have = false;
      }
    }
  }
}

template <int MODE>
void launch_engine_mode(const Dev& v, const Grid& g, cudaStream_t s, int64_t n_total) {
  k_list_reset<<<1, 32, 0, s>>>(v);
  count_launch();
  k_list<MODE><<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  if (MODE == MODE_ROOT) {
    k_root32_copy<<<g.slot_blocks, 256, 0, s>>>(v, n_total);
    count_launch();
    k_root32<<<g.slot_blocks, 128, 0, s>>>(v);
    count_launch();
  }
  k_engine<MODE><<<g.nsm * max(1, min(kEngCtasPerSm, v.engine_ctas)), kEngThreads, 0, s>>>(v);
  count_launch();
}

}  // namespace

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
