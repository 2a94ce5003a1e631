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
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    v.ctl->level_begin = v.ctl->nodes;
    v.ctl->level_new = 0;
  }
}

// Boundary flags: a cluster ends after slot w when the (lower bound of the)
// absolute gap to w+1 is at least tol times the larger magnitude of the two.
__global__ void k_classify_flags(Dev v, int level) {
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
      f = gap >= v.gap_tol * mag;
    }
    v.bflag[w] = f;
  }
}

// Runs between boundaries: length 1 = singleton, otherwise a new child node.
__global__ void k_classify_runs(Dev v, int level) {
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

// One thread per slot of a new cluster: refine its interval in the PARENT's
// representation to the cluster accuracy, so that the child shift can be
// placed right at the cluster's end.
__global__ void k_prerefine(Dev v) {
  const int begin = v.ctl->level_begin;
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid(); w < nslots; w += gstride()) {
    if (v.state[w] != SLOT_ACTIVE) continue;
    const int nid = v.snode[w];
    if (nid < begin) continue;
    const Node c = v.node[nid];
    const Node p = v.node[c.parent];
    const int m = v.blk[c.block].m;
    double lo = v.lo[w], hi = v.hi[w];
    int it = bisect_interval(v.pool + p.rep, m, v.sj[w], p.pivmin, v.rtol_cluster, 4.0 * p.pivmin,
                             v.max_bisect, lo, hi);
    if (it >= v.max_bisect) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, DIAG_REFINE_BISECT);
    }
    v.lo[w] = lo;
    v.hi[w] = hi;
  }
}

// Stationary qd transform (dstqds) of the parent representation with shift
// sigma, written as the child representation:
//   s_1 = -sigma, D+_i = D_i + s_i, L+_i = LD_i / D+_i,
//   s_{i+1} = L+_i l_i s_i - sigma.
// Returns max |D+_i| (infinite when a pivot is not finite).
__device__ double dstqds_child(const RepRow* __restrict__ par, RepRow* __restrict__ out, int m,
                               double sigma, double pivmin) {
  double s = -sigma;
  double growth = 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const RepRow r = par[i];
    double dp = r.D + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    double lp = r.LD / dp;
    s = fma(lp, r.l * s, -sigma);
    double ldp = lp * dp;
    out[i] = RepRow{dp, lp * ldp, lp, ldp};
    growth = fmax(growth, fabs(dp));
  }
  double dp = par[m - 1].D + s;
  if (fabs(dp) < pivmin) dp = -pivmin;
  out[m - 1] = RepRow{dp, 0.0, 0.0, 0.0};
  growth = fmax(growth, fabs(dp));
  if (!isfinite(growth)) growth = INFINITY;
  return growth;
}

// One thread per new node: choose sigma_c at the left or right end of the
// cluster, moved outward geometrically until the element growth
// max|D+| <= 8 * spdiam; if no candidate qualifies the smallest growth seen
// is kept and the cluster is counted as a fallback.
__global__ void k_childrep(Dev v) {
  const int begin = v.ctl->level_begin;
  const int end = min(v.ctl->nodes, v.max_nodes);
  for (int64_t id = begin + gtid(); id < end; id += gstride()) {
    Node c = v.node[id];
    const Node p = v.node[c.parent];
    const int m = v.blk[c.block].m;
    int64_t base = atomicAdd((unsigned long long*)&v.ctl->pool_top, (unsigned long long)m);
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
      c.rep = p.rep;
      c.depth = -1;  // inert
      v.node[id] = c;
      continue;
    }
    const RepRow* par = v.pool + p.rep;
    RepRow* out = v.pool + base;
    const double lo_f = v.lo[c.first], hi_l = v.hi[c.last];
    const double bound = 8.0 * c.spdiam;
    double best_g = INFINITY, best_sigma = lo_f;
    double sigma = lo_f;
    bool ok = false;
    for (int t = 0; t < 10 && !ok; ++t) {
      for (int side = 0; side < 2 && !ok; ++side) {
        double ref = side == 0 ? lo_f : hi_l;
        double delta = 4.0 * kEps * fabs(ref) * (double)(1LL << (2 * t)) + 4.0 * c.pivmin;
        sigma = side == 0 ? lo_f - delta : hi_l + delta;
        double g = dstqds_child(par, out, m, sigma, c.pivmin);
        if (g < best_g) best_g = g, best_sigma = sigma;
        ok = g <= bound;
      }
    }
    if (!ok) {
      sigma = best_sigma;
      dstqds_child(par, out, m, sigma, c.pivmin);
      diag(v.ctl, DIAG_CHILD_GROWTH);
    }
    c.rep = base;
    c.sigma_rel = sigma;
    c.sigma_abs = p.sigma_abs + sigma;
    v.node[id] = c;
  }
}

// One thread per slot of a new node: move its interval into the child's
// coordinates, widen it until Sturm counts on the child confirm the bracket,
// then bisect to the classification accuracy.
__global__ void k_refine(Dev v) {
  const int begin = v.ctl->level_begin;
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid(); w < nslots; w += gstride()) {
    if (v.state[w] != SLOT_ACTIVE) continue;
    const int nid = v.snode[w];
    if (nid < begin) continue;
    const Node c = v.node[nid];
    if (c.depth < 0) continue;
    const int m = v.blk[c.block].m;
    const RepRow* rep = v.pool + c.rep;
    const int j = v.sj[w];
    const double plo = v.lo[w], phi = v.hi[w];
    double delta = 16.0 * kEps * fmax(fabs(plo), fabs(phi)) + 4.0 * c.pivmin;
    double lo = 0.0, hi = 0.0;
    bool ok = false;
    for (int t = 0; t < 24 && !ok; ++t) {
      lo = (plo - c.sigma_rel) - delta;
      hi = (phi - c.sigma_rel) + delta;
      ok = negcount(rep, m, lo, c.pivmin) <= j - 1 && negcount(rep, m, hi, c.pivmin) >= j;
      delta *= 4.0;
    }
    if (!ok) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, DIAG_REFINE_BRACKET);
    }
    int it = bisect_interval(rep, m, j, c.pivmin, v.rtol_cluster, 4.0 * c.pivmin, v.max_bisect, lo, hi);
    if (it >= v.max_bisect) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, DIAG_REFINE_BISECT);
    }
    v.lo[w] = lo;
    v.hi[w] = hi;
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
}

void launch_level_children(const Dev& v, int level, const Grid& g, cudaStream_t s) {
  (void)level;
  k_prerefine<<<g.slot_blocks, g.tpb, 0, s>>>(v);
  count_launch();
  mark_stage("prerefine", s);
  k_childrep<<<g.slot_blocks, 32, 0, s>>>(v);
  count_launch();
  mark_stage("childrep", s);
  k_refine<<<g.slot_blocks, g.tpb, 0, s>>>(v);
  count_launch();
  mark_stage("refine", s);
}

}  // namespace mrrr
