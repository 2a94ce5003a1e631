// mrrr_tree.cu -- one level of the representation tree (paper Sec. 3.1.1):
// classification of the eigenvalues of each node into singletons and
// clusters by relative gap (singleton iff relgap > tol, tol = 1e-3, gaps and
// magnitudes in the node's shifted coordinates), a child representation
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
  }
}

// After a level's classification: the tree is complete when the level made
// no new cluster (or a fatal error was recorded); the kernels of all later
// levels then return at entry, so the levels can be enqueued without the
// host reading the count in between.
__global__ void k_level_end(Dev v, int level) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !v.ctl->done) {
    v.ctl->levels = level + 1;
    const int st = v.ctl->status;
    if (v.ctl->level_new == 0 || (st != 0 && st != MRRR_ERR_NOCONV)) v.ctl->done = 1;
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

__global__ void k_classify_flags(Dev v, int level) {
  if (v.ctl->done) return;
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
__global__ void k_classify_runs(Dev v, int level) {
  if (v.ctl->done) return;
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

constexpr int kShiftTries = 10;  // per side

// Candidate shift t (0 .. 2 kShiftTries - 1) of a cluster: even t the left
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

// Child representations, phase 1: one thread per new node reserves its rows
// in the representation pool and builds the transform for the first
// candidate shift (the left end of the cluster, smallest offset) with the
// stores done in the same pass.  It is kept when its element growth max|D+|
// is at most 8 spdiam; otherwise the node is marked for phase 2.  Nodes
// whose rows do not fit take the fallback (their vectors at the parent).
__global__ void k_childrep_first(Dev v) {
  if (v.ctl->done) return;
  const int begin = v.ctl->level_begin;
  const int end = min(v.ctl->nodes, v.max_nodes);
  for (int64_t id = begin + gtid(); id < end; id += gstride()) {
    Node c = v.node[id];
    const Node p = v.node[c.parent];
    const int m = v.blk[c.block].m;
    const int64_t base =
        (int64_t)atomicAdd((unsigned long long*)&v.ctl->pool_top, (unsigned long long)m);
    atomicMax((unsigned long long*)&v.ctl->pool_need, (unsigned long long)(base + m));
    if (base + m > v.pool_cap) {
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
      continue;
    }
    const double sigma = child_shift(0, v.lo[c.first], v.hi[c.last], p.pivmin);
    double gd;
    const double R = dstqds_child<true>(v.rep_dl + p.rep, v.rep_ul + p.rep, v.rep_dl + base, v.rep_ul + base, m,
                                        sigma, p.pivmin, &gd);
    if (gd <= 8.0 * c.spdiam) {
      set_child(v, id, c, p, base, sigma, R);
    } else {
      c.rep = base;
      c.pad_ = 1;           // phase 2
      c.sigma_rel = gd;     // growth of the first candidate, for phase 2
      v.node[id] = c;
    }
  }
}

// Phase 2, for nodes whose first candidate failed: a group of 8 lanes per
// node (4 nodes per warp) evaluates 8 further candidates spread over the
// ladder of child_shift (growth only); the first candidate in ladder order
// whose growth max|D+| is at most 8 spdiam is taken, else the one with the
// smallest growth among these and the first candidate (counted in the
// diagnostics).  The chosen transform is then recomputed with stores into
// the rows reserved in phase 1.
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
    double g = INFINITY, sigma = 0.0;
    int cand = 0;
    Node p{};
    if (mine) {
      p = v.node[c.parent];
      const int m = v.blk[c.block].m;
      cand = kPhase2Cands[gl];
      sigma = child_shift(cand, v.lo[c.first], v.hi[c.last], p.pivmin);
      g = dstqds_child<false>(v.rep_dl + p.rep, v.rep_ul + p.rep, nullptr, nullptr, m, sigma, p.pivmin);
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
    if (!mine || gl != 0) continue;
    const int m = v.blk[c.block].m;
    int pick;
    if (okmask) {
      pick = kPhase2Cands[__ffs(okmask) - 1 - leader];
    } else {
      // the first candidate's growth was kept in sigma_rel by phase 1
      pick = c.sigma_rel <= bg ? 0 : bc;
      diag(v.ctl, DIAG_CHILD_GROWTH);
    }
    const double sig = child_shift(pick, v.lo[c.first], v.hi[c.last], p.pivmin);
    const double R =
        dstqds_child<true>(v.rep_dl + p.rep, v.rep_ul + p.rep, v.rep_dl + c.rep, v.rep_ul + c.rep, m, sig, p.pivmin);
    set_child(v, id, c, p, c.rep, sig, R);
  }
}

}  // namespace

void launch_level_classify(const Dev& v, int level, const Grid& g, cudaStream_t s) {
  k_level_start<<<1, 32, 0, s>>>(v);
  count_launch();
  k_classify_flags<<<g.slot_blocks, g.tpb, 0, s>>>(v, level);
  count_launch();
  k_classify_runs<<<g.slot_blocks, g.tpb, 0, s>>>(v, level);
  count_launch();
  k_level_end<<<1, 32, 0, s>>>(v, level);
  count_launch();
}

void launch_level_children(const Dev& v, int level, const Grid& g, cudaStream_t s) {
  (void)level;
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
