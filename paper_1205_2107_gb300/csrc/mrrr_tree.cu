// mrrr_tree.cu -- one level of the representation tree (paper Sec. 3.1.1):
// classification of the eigenvalues of each node into singletons and
// clusters by relative gap (singleton iff relgap > tol, tol = max(gap_tol,
// 1/m) with gap_tol = 1e-4 by default, gaps and magnitudes in the node's
// shifted coordinates), a child representation
// Lc Dc Lc^T = L D L^T - sigma_c I for every cluster (stationary qd
// transform, sigma_c at an end of the cluster), and refinement of the
// cluster's eigenvalues with respect to the child by bisection.
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {

namespace {

__global__ void k_level_start(Dev v) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !v.ctl->done) {
    v.ctl->level_begin = v.ctl->nodes;
    v.ctl->level_new = 0;
    v.ctl->cand_top = 0;
  }
}

// After a level's classification: the tree is complete when the level made
// no new cluster (or a fatal error was recorded); the kernels of all later
// levels then return at entry, so the levels can be enqueued without the
// host reading the count in between.  The current level is ctl->levels (the
// levels finished so far), so one captured level can be replayed by a graph
// loop; inside a CUDA graph's conditional while node (use_cond) this kernel
// also sets the loop's condition: one more level while the tree is not done.
__global__ void k_level_end(Dev v, cudaGraphConditionalHandle cond, int use_cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (!v.ctl->done) {
      const int level = v.ctl->levels;
      v.ctl->levels = level + 1;
      const int st = v.ctl->status;
      if (v.ctl->level_new == 0 || (st != 0 && st != MRRR_ERR_NOCONV) || level + 1 > v.max_depth) v.ctl->done = 1;
    }
    if (use_cond) cudaGraphSetConditional(cond, v.ctl->done ? 0u : 1u);
  }
}

// Boundary flags: a cluster ends after slot w when the (lower bound of the)
// absolute gap to w+1 is at least tol times the larger magnitude of the two.
// tol = max(gap_tol, 1 / m) for a block of order m.  Eq. errorangle bounds
// the error angle of a singleton's vector by O(m eps / relgap); measured, it
// behaves like c eps / relgap with c of a few units whatever m is, while the
// orthogonality goal is 20 m eps.  So relgap has to exceed about 1/m for
// small blocks, and large blocks can accept smaller gaps than the paper's
// 1e-3 (fewer, shallower cluster levels): the floor gap_tol defaults to 1e-4.
constexpr double kSmallBlockTol = 1.0;

__global__ void k_classify_flags(Dev v) {
  if (v.ctl->done) return;
  const int level = v.ctl->levels;
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid(); w < nslots; w += gstride()) {
    if (v.state[w] != SLOT_ACTIVE) continue;
    const Node& nd = v.node[v.snode[w]];
    if (nd.depth != level) continue;
    unsigned char f = 1;
    if (w != nd.last) {
      double lo0 = v.lo[w], hi0 = v.hi[w], lo1 = v.lo[w + 1], hi1 = v.hi[w + 1];
      double gap = lo1 - hi0;
      double mag = fmax(fmax(fabs(lo0), fabs(hi0)), fmax(fabs(lo1), fabs(hi1)));
      const double tol = fmax(v.gap_tol, kSmallBlockTol / (double)v.blk[nd.block].m);
      f = gap >= tol * mag;
    }
    v.bflag[w] = f;
  }
}

// Runs between boundaries: length 1 = singleton, otherwise a new child node.
__global__ void k_classify_runs(Dev v) {
  if (v.ctl->done) return;
  const int level = v.ctl->levels;
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid(); w < nslots; w += gstride()) {
    if (v.state[w] != SLOT_ACTIVE) continue;
    const int nid = v.snode[w];
    const Node nd = v.node[nid];
    if (nd.depth != level) continue;
    if (w != nd.first && !v.bflag[w - 1]) continue;  // not a run start
    int64_t e = w;
    while (e < nd.last && !v.bflag[e]) ++e;
    const double gl = (w == nd.first) ? nd.gapl : v.lo[w] - v.hi[w - 1];
    const double gr = (e == nd.last) ? nd.gapr : v.lo[e + 1] - v.hi[e];
    if (level == 0) {
      // a slice computes its indices plus a margin on each side; a root
      // cluster that holds returned indices must lie inside the computed
      // range (not touch an end that is not an end of the spectrum), or its
      // neighbouring slice may group it differently
      const Block& bk = v.blk[nd.block];
      if (v.prob[bk.prob].slice && ((w == nd.first && bk.js > 1) || (e == nd.last && bk.je < bk.m))) {
        bool returned = false;
        for (int64_t t = w; t <= e && !returned; ++t) returned = v.spos[t] >= 0;
        if (returned) set_status(v.ctl, MRRR_ERR_MARGIN);
      }
    }
    if (e == w) {
      v.state[w] = SLOT_SINGLETON;
      v.gap[w] = fmin(gl, gr);
      continue;
    }
    int id = -1;
    if (level + 1 <= v.max_depth) {
      id = atomicAdd(&v.ctl->nodes, 1);
      if (id >= v.max_nodes) {
        set_status(v.ctl, MRRR_ERR_QUEUE);
        id = -1;
      }
    }
    if (id < 0) {  // fallback: vectors at this node, treated as singletons
      for (int64_t t = w; t <= e; ++t) {
        double a = (t == w) ? gl : v.lo[t] - v.hi[t - 1];
        double b = (t == e) ? gr : v.lo[t + 1] - v.hi[t];
        v.state[t] = SLOT_FALLBACK;
        v.gap[t] = fmax(fmin(a, b), 0.0);
      }
      atomicAdd(&v.ctl->fallbacks, (unsigned long long)(e - w + 1));
      diag(v.ctl, level + 1 <= v.max_depth ? DIAG_CAPACITY : DIAG_DEPTH, (unsigned long long)(e - w + 1));
      continue;
    }
    Node c;
    c.block = nd.block;
    c.depth = level + 1;
    c.first = w;
    c.last = e;
    c.parent = nid;
    c.pad_ = 0;
    c.rep = -1;
    c.sigma_rel = 0.0;
    c.sigma_abs = nd.sigma_abs;
    c.gapl = gl;
    c.gapr = gr;
    c.pivmin = nd.pivmin;
    c.spdiam = nd.spdiam;
    v.node[id] = c;
    for (int64_t t = w; t <= e; ++t) v.snode[t] = id;
    atomicAdd(&v.ctl->level_new, 1);
    atomicMax(&v.ctl->depth, level + 1);
  }
}

// Stationary qd transform (dstqds) of the parent representation with shift
// sigma (paper Sec. 3.1.1: Lc Dc Lc^T = L D L^T - sigma_c I, computed in a
// mixed relatively stable way):
//   s_1 = -sigma, D+_i = D_i + s_i, L+_i = LD_i / D+_i,
//   s_{i+1} = L+_i l_i s_i - sigma.
// growth_only: returns max |D+_i| without storing (infinite when a pivot is
// not finite); otherwise writes the child rows and returns
// max(|D+_i|, |LLD+_i|).
// growth_d receives max |D+_i| (infinite when a pivot is not finite) in both
// forms.
template <bool kStore>
__device__ double dstqds_child(const double2* __restrict__ pdl, const double2* __restrict__ pul,
                               double2* __restrict__ cdl, double2* __restrict__ cul, int m, double sigma,
                               double pivmin, double* growth_d = nullptr) {
  double s = -sigma;
  double gd = 0.0, growth = 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const RepRow r = rep_row(pdl, pul, i);
    double dp = r.D + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    const double lp = r.LD / dp;
    s = fma(lp, r.l * s, -sigma);
    gd = fmax(gd, fabs(dp));
    if (kStore) {
      const double ldp = lp * dp;
      const double lldp = lp * ldp;
      rep_store(cdl, cul, i, RepRow{dp, lldp, lp, ldp});
      growth = fmax(growth, fabs(lldp));
    }
  }
  double dp = pdl[m - 1].x + s;
  if (fabs(dp) < pivmin) dp = -pivmin;
  if (kStore) rep_store(cdl, cul, m - 1, RepRow{dp, 0.0, 0.0, 0.0});
  gd = fmax(gd, fabs(dp));
  if (!isfinite(gd)) gd = INFINITY;
  growth = fmax(growth, gd);
  if (!isfinite(growth)) growth = INFINITY;
  if (growth_d) *growth_d = gd;
  return kStore ? growth : gd;
}

// The transform of dstqds_child with the stores predicated on `store`: every
// lane of a warp runs the same instructions whether it stores or not (two
// template instances in one warp would run one after the other).  Returns
// max(|D+_i|, |LLD+_i|); growth_d receives max|D+_i| (infinite when a pivot
// is not finite).
__device__ double dstqds_child_pred(const double2* __restrict__ pdl, const double2* __restrict__ pul,
                                    double2* __restrict__ cdl, double2* __restrict__ cul, int m, double sigma,
                                    double pivmin, bool store, double* growth_d) {
  double s = -sigma;
  double gd = 0.0, growth = 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const RepRow r = rep_row(pdl, pul, i);
    double dp = r.D + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    const double lp = r.LD / dp;
    s = fma(lp, r.l * s, -sigma);
    gd = fmax(gd, fabs(dp));
    const double ldp = lp * dp;
    const double lldp = lp * ldp;
    if (store) rep_store(cdl, cul, i, RepRow{dp, lldp, lp, ldp});
    growth = fmax(growth, fabs(lldp));
  }
  double dp = pdl[m - 1].x + s;
  if (fabs(dp) < pivmin) dp = -pivmin;
  if (store) rep_store(cdl, cul, m - 1, RepRow{dp, 0.0, 0.0, 0.0});
  gd = fmax(gd, fabs(dp));
  if (!isfinite(gd)) gd = INFINITY;
  growth = fmax(growth, gd);
  if (!isfinite(growth)) growth = INFINITY;
  *growth_d = gd;
  return growth;
}

// Candidate shift t (0 .. 19: ten per side) of a cluster: even t the left
// end lo_f - delta, odd t the right end hi_l + delta, delta = 4 eps |end| 4^(t/2)
// (+ 4 pivmin).
__device__ __forceinline__ double child_shift(int t, double lo_f, double hi_l, double pivmin) {
  const int side = t & 1, k = t >> 1;
  const double ref = side == 0 ? lo_f : hi_l;
  const double delta = 4.0 * kEps * fabs(ref) * (double)(1LL << (2 * k)) + 4.0 * pivmin;
  return side == 0 ? lo_f - delta : hi_l + delta;
}

__device__ __forceinline__ void set_child(Dev& v, int64_t id, Node c, const Node& p, int64_t base, double sigma,
                                          double R) {
  c.rep = base;
  c.sigma_rel = sigma;
  c.sigma_abs = p.sigma_abs + sigma;
  c.pivmin = pivmin_for(R);
  c.pad_ = 0;
  v.node[id] = c;
}

// Child representations, first wave.  The candidate shifts are tried in
// ladder order 0, 1, 2, 3, 4, 8, 9, 18, 19 (child_shift); the first whose
// element growth max|D+| is at most 8 spdiam is taken, else the one with the
// smallest growth (counted in the diagnostics).  A group of L lanes per new
// node (L from the number of nodes of the level: up to two warps per SM
// sub-partition, so that the extra lanes cost no time) evaluates the first
// min(L, 9) candidates in one pass over the parent's rows.  Each transform
// is a sequential recurrence, so a level with few clusters is bound by the
// latency of one pass: trying every candidate at once replaces up to three
// passes (first candidate, the others, the winner again with stores) by one.
// Candidate 0 always stores into the node's rows of the pool.  When the pool
// has room, every other candidate of the group stores into rows of its own
// there and the winner's rows become the child (the others stay unused);
// else, when the eigenvector scratch (idle while the tree is built) has
// room, the other candidates store there and the warp copies a winner's
// rows into the node's rows; otherwise a winner other than candidate 0 is
// computed once more with stores.  A node whose
// evaluated candidates all fail before the whole ladder was tried goes to
// the second wave (k_childrep).  Nodes whose rows do not fit take the
// fallback (their vectors at the parent).  The choice is the same whatever
// L is, so the child representation is too.
constexpr int kLadder = 9;
__constant__ int kLadderCands[kLadder] = {0, 1, 2, 3, 4, 8, 9, 18, 19};

__device__ __forceinline__ void child_fallback(Dev& v, int64_t id, Node c) {
  set_status(v.ctl, MRRR_ERR_QUEUE);
  // vectors of these slots are taken at the parent node
  for (int64_t t = c.first; t <= c.last; ++t) {
    v.state[t] = SLOT_FALLBACK;
    v.snode[t] = c.parent;
    double a = (t == c.first) ? c.gapl : v.lo[t] - v.hi[t - 1];
    double b = (t == c.last) ? c.gapr : v.lo[t + 1] - v.hi[t];
    v.gap[t] = fmax(fmin(a, b), 0.0);
  }
  atomicAdd(&v.ctl->fallbacks, (unsigned long long)(c.last - c.first + 1));
  diag(v.ctl, DIAG_CAPACITY, (unsigned long long)(c.last - c.first + 1));
  c.rep = -1;
  c.depth = -1;  // inert
  v.node[id] = c;
}

__global__ void k_childrep_first(Dev v) {
  if (v.ctl->done) return;
  const int begin = v.ctl->level_begin;
  const int end = min(v.ctl->nodes, v.max_nodes);
  const int N = end - begin;
  if (N <= 0) return;
  const long long lanes = (long long)v.nsm * 4 * 32 * 2;
  int L = 1;
  while (L < 16 && (long long)N * L * 2 <= lanes) L *= 2;
  const int ncand = min(L, kLadder);
  const int lane = threadIdx.x & 31;
  const int gl = lane % L, leader = lane - gl, per_warp = 32 / L;
  const unsigned gbits = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << leader);
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t id0 = begin + warp * per_warp; id0 < end; id0 += nwarps * per_warp) {
    const int64_t id = id0 + lane / L;
    const bool mine = id < end;
    Node c{};
    Node p{};
    int m = 0;
    int64_t base = -1, sbase = -1;
    bool multi = false;
    if (mine) {
      c = v.node[id];
      p = v.node[c.parent];
      m = v.blk[c.block].m;
      if (gl == 0) {
        // rows for every candidate when the pool keeps half its room free
        multi = ncand > 1 && v.ctl->pool_top + (int64_t)N * ncand * m <= v.pool_cap / 2;
        const int64_t rows = (int64_t)(multi ? ncand : 1) * m;
        base = (int64_t)atomicAdd((unsigned long long*)&v.ctl->pool_top, (unsigned long long)rows);
        atomicMax((unsigned long long*)&v.ctl->pool_need, (unsigned long long)(base + rows));
        if (base + rows > v.pool_cap) base = -1;
        if (!multi && ncand > 1 && base >= 0) {  // candidates 1.. in the scratch
          const int64_t srows = (int64_t)(ncand - 1) * m;
          const int64_t at = (int64_t)atomicAdd((unsigned long long*)&v.ctl->cand_top, (unsigned long long)srows);
          if (at + srows <= cand_capacity(v)) sbase = at;
        }
      }
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    sbase = __shfl_sync(0xffffffffu, sbase, leader);
    multi = __shfl_sync(0xffffffffu, (int)multi, leader) != 0;
    const bool live = mine && base >= 0;
    if (mine && base < 0 && gl == 0) child_fallback(v, id, c);
    const bool cand = live && gl < ncand;
    const int t = cand ? kLadderCands[gl] : 0;
    double sigma = 0.0, gd = INFINITY, R = 0.0;
    const bool scratch = !multi && sbase >= 0 && gl > 0;
    const bool stored = cand && (multi || gl == 0 || scratch);
    if (cand) {
      sigma = child_shift(t, v.lo[c.first], v.hi[c.last], p.pivmin);
      double2* odl = v.rep_dl + base + (multi ? (int64_t)gl * m : 0);
      double2* oul = v.rep_ul + base + (multi ? (int64_t)gl * m : 0);
      if (scratch) {
        odl = cand_dl(v) + sbase + (int64_t)(gl - 1) * m;
        oul = cand_ul(v) + sbase + (int64_t)(gl - 1) * m;
      }
      R = dstqds_child_pred(v.rep_dl + p.rep, v.rep_ul + p.rep, odl, oul, m, sigma, p.pivmin, stored, &gd);
    }
    const bool ok = cand && gd <= 8.0 * c.spdiam;
    const unsigned okmask = __ballot_sync(0xffffffffu, ok) & gbits;
    // smallest growth in the group, lowest candidate on ties
    double bg = gd;
    int bl = gl;
    for (int o = L / 2; o; o >>= 1) {
      const double og = __shfl_xor_sync(0xffffffffu, bg, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (og < bg || (og == bg && ol < bl)) bg = og, bl = ol;
    }
    int win = okmask ? __ffs(okmask) - 1 - leader : (ncand == kLadder ? bl : -1);
    const double gd0 = __shfl_sync(0xffffffffu, gd, leader);
    const double sig_w = __shfl_sync(0xffffffffu, sigma, leader + max(win, 0));
    const double R_w = __shfl_sync(0xffffffffu, R, leader + max(win, 0));
    // winners stored in the scratch: the whole warp copies their rows into
    // the node's rows of the pool, one group after the other
    {
      const bool cp = live && gl == 0 && !multi && sbase >= 0 && win > 0;
      __syncwarp();  // the candidates' stores are visible to the whole warp
      unsigned todo = __ballot_sync(0xffffffffu, cp);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t dst = __shfl_sync(0xffffffffu, base, src);
        const int mm = __shfl_sync(0xffffffffu, m, src);
        const int64_t from = __shfl_sync(0xffffffffu, sbase, src) +
                             (int64_t)(__shfl_sync(0xffffffffu, win, src) - 1) * mm;
        const double2* sdl = cand_dl(v) + from;
        const double2* sul = cand_ul(v) + from;
        for (int i = lane; i < mm; i += 32) {
          v.rep_dl[dst + i] = sdl[i];
          v.rep_ul[dst + i] = sul[i];
        }
      }
      __syncwarp();
    }
    if (!live || gl != 0) continue;
    if (win < 0) {  // second wave: the rest of the ladder
      c.rep = base;
      c.pad_ = 1;
      c.sigma_rel = gd0;  // growth of the first candidate, for the second wave
      c.pivmin = R;       // and its largest entry (candidate 0's rows stay at base)
      v.node[id] = c;
      diag(v.ctl, DIAG_CHILD_WAVE2);
      continue;
    }
    if (!okmask) diag(v.ctl, DIAG_CHILD_GROWTH);
    if (multi || win == 0 || sbase >= 0) {
      set_child(v, id, c, p, base + (multi ? (int64_t)win * m : 0), sig_w, R_w);
    } else {
      const double Rr = dstqds_child<true>(v.rep_dl + p.rep, v.rep_ul + p.rep, v.rep_dl + base, v.rep_ul + base, m,
                                           sig_w, p.pivmin);
      set_child(v, id, c, p, base, sig_w, Rr);
      diag(v.ctl, DIAG_CHILD_RESTORE);
    }
  }
}

// Phase 2, for nodes whose first candidate failed: a group of 8 lanes per
// node (4 nodes per warp) evaluates 8 further candidates spread over the
// ladder of child_shift; the first candidate in ladder order whose growth
// max|D+| is at most 8 spdiam is taken, else the one with the smallest
// growth among these and the first candidate (counted in the diagnostics).
// Every candidate stores into rows of its own -- in the pool when it has
// room (the winner's rows become the child), else in the eigenvector
// scratch (the warp copies the winner's rows over the node's) -- in one
// pass; when neither has room the pass measures growth only and the chosen
// transform is computed again with stores into the rows reserved in phase 1
// (which hold candidate 0's).
constexpr int kPhase2Group = 8;
__constant__ int kPhase2Cands[kPhase2Group] = {1, 2, 3, 4, 8, 9, 18, 19};

__global__ void k_childrep(Dev v) {
  if (v.ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int sub = lane / kPhase2Group, gl = lane % kPhase2Group, leader = sub * kPhase2Group;
  const int per_warp = 32 / kPhase2Group;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  const int begin = v.ctl->level_begin;
  const int end = min(v.ctl->nodes, v.max_nodes);
  for (int64_t id0 = begin + warp * per_warp; id0 < end; id0 += nwarps * per_warp) {
    const int64_t id = id0 + sub;
    Node c{};
    bool mine = id < end;
    if (mine) {
      c = v.node[id];
      mine = c.pad_ == 1;
    }
    double g = INFINITY, sigma = 0.0, Rc = 0.0;
    int cand = 0;
    Node p{};
    int64_t base = -1, sbase = -1;
    if (mine && gl == 0) {
      const int m = v.blk[c.block].m;
      const int64_t rows = (int64_t)kPhase2Group * m;
      if (v.ctl->pool_top + rows <= v.pool_cap / 2) {
        base = (int64_t)atomicAdd((unsigned long long*)&v.ctl->pool_top, (unsigned long long)rows);
        atomicMax((unsigned long long*)&v.ctl->pool_need, (unsigned long long)(base + rows));
        if (base + rows > v.pool_cap) base = -1;
      }
      if (base < 0) {  // else in the eigenvector scratch
        const int64_t at = (int64_t)atomicAdd((unsigned long long*)&v.ctl->cand_top, (unsigned long long)rows);
        if (at + rows <= cand_capacity(v)) sbase = at;
      }
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    sbase = __shfl_sync(0xffffffffu, sbase, leader);
    int m = 0;
    if (mine) {
      p = v.node[c.parent];
      m = v.blk[c.block].m;
      cand = kPhase2Cands[gl];
      sigma = child_shift(cand, v.lo[c.first], v.hi[c.last], p.pivmin);
      double2* odl = base >= 0 ? v.rep_dl + base + (int64_t)gl * m : cand_dl(v) + max(sbase, (int64_t)0) + (int64_t)gl * m;
      double2* oul = base >= 0 ? v.rep_ul + base + (int64_t)gl * m : cand_ul(v) + max(sbase, (int64_t)0) + (int64_t)gl * m;
      Rc = dstqds_child_pred(v.rep_dl + p.rep, v.rep_ul + p.rep, odl, oul, m, sigma, p.pivmin,
                             base >= 0 || sbase >= 0, &g);
    }
    const unsigned gbits = 0xffu << leader;
    const bool ok = mine && g <= 8.0 * c.spdiam;
    const unsigned okmask = __ballot_sync(0xffffffffu, ok) & gbits;
    // smallest growth in the group, lowest candidate on ties
    double bg = g;
    int bc = cand;
    for (int o = kPhase2Group / 2; o; o >>= 1) {
      const double og = __shfl_xor_sync(0xffffffffu, bg, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (og < bg || (og == bg && oc < bc)) bg = og, bc = oc;
    }
    // the lane (within the group) of the pick, -1 for candidate 0
    int pl;
    if (okmask) {
      pl = __ffs(okmask) - 1 - leader;
    } else {
      // the first candidate's growth was kept in sigma_rel by phase 1
      const int pick = c.sigma_rel <= bg ? 0 : bc;
      pl = -1;
      for (int k = 0; k < kPhase2Group; ++k)
        if (kPhase2Cands[k] == pick) pl = k;
    }
    const double R_pick = __shfl_sync(0xffffffffu, Rc, leader + max(pl, 0));
    // winners stored in the scratch: the whole warp copies their rows over
    // the node's rows (which held candidate 0), one node after the other
    {
      const bool cp = mine && gl == 0 && base < 0 && sbase >= 0 && pl >= 0;
      __syncwarp();  // the candidates' stores are visible to the whole warp
      unsigned todo = __ballot_sync(0xffffffffu, cp);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t dst = __shfl_sync(0xffffffffu, c.rep, src);
        const int mm = __shfl_sync(0xffffffffu, m, src);
        const int64_t from = __shfl_sync(0xffffffffu, sbase, src) + (int64_t)__shfl_sync(0xffffffffu, pl, src) * mm;
        for (int i = lane; i < mm; i += 32) {
          v.rep_dl[dst + i] = cand_dl(v)[from + i];
          v.rep_ul[dst + i] = cand_ul(v)[from + i];
        }
      }
      __syncwarp();
    }
    if (!mine || gl != 0) continue;
    if (!okmask) diag(v.ctl, DIAG_CHILD_GROWTH);
    const int pick = pl < 0 ? 0 : kPhase2Cands[pl];
    const double sig = child_shift(pick, v.lo[c.first], v.hi[c.last], p.pivmin);
    if (pl < 0) {  // candidate 0: its rows and largest entry from phase 1
      set_child(v, id, c, p, c.rep, sig, c.pivmin);
    } else if (base >= 0) {
      set_child(v, id, c, p, base + (int64_t)pl * m, sig, R_pick);
    } else if (sbase >= 0) {  // copied over the node's rows above
      set_child(v, id, c, p, c.rep, sig, R_pick);
    } else {
      const double R = dstqds_child<true>(v.rep_dl + p.rep, v.rep_ul + p.rep, v.rep_dl + c.rep, v.rep_ul + c.rep, m,
                                          sig, p.pivmin);
      set_child(v, id, c, p, c.rep, sig, R);
      diag(v.ctl, DIAG_CHILD_RESTORE);
    }
  }
}

}  // namespace

void launch_level_classify(const Dev& v, const Grid& g, cudaStream_t s, cudaGraphConditionalHandle cond,
                           int use_cond) {
  k_level_start<<<1, 32, 0, s>>>(v);
  count_launch();
  k_classify_flags<<<g.slot_blocks, g.tpb, 0, s>>>(v);
  count_launch();
  k_classify_runs<<<g.slot_blocks, g.tpb, 0, s>>>(v);
  count_launch();
  k_level_end<<<1, 32, 0, s>>>(v, cond, use_cond);
  count_launch();
  mark_stage("classify", s);
}

void launch_level_children(const Dev& v, const Grid& g, cudaStream_t s) {
  launch_engine(v, 1, g, s);
  mark_stage("prerefine", s);
  k_childrep_first<<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  k_childrep<<<g.slot_blocks, 128, 0, s>>>(v);
  count_launch();
  mark_stage("childrep", s);
  launch_engine(v, 2, g, s);
  mark_stage("refine", s);
}

}  // namespace mrrr
