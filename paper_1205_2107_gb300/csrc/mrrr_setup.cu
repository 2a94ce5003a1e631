// mrrr_setup.cu -- problem table, norm and scaling, splitting into blocks,
// root representations and root bisection (Sec. 3.1.1: first a root
// representation RRR0 of the shifted matrix, then bisection for an
// approximation of every wanted eigenvalue; splitting follows the footnote
// on numerical irreducibility: off-diagonals below eps*||T|| are zero).
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {

namespace {

constexpr double kPivmin = 0x1p-900;  // zero-pivot guard while the root is built

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a counter-based 64-bit mixing function.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Top 53 bits as a double in [-1, 1).
__device__ __forceinline__ double uniform_pm1(uint64_t z) {
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

__device__ __forceinline__ double scaled_d(const Dev& v, const Problem& p, int64_t i) {
  return v.d[p.row0 + i] * p.scale;
}
__device__ __forceinline__ double scaled_e(const Dev& v, const Problem& p, int64_t i) {
  return v.e[p.row0 + i] * p.scale;
}

// ---------------------------------------------------------------------------
// Problem table.
__global__ void k_problems(Dev v, ProblemArgs a) {
  for (int64_t p = gtid(); p < a.batch; p += gstride()) {
    Problem q{};
    int n, il, iu;
    if (a.d_off == nullptr) {
      q.row0 = 0;
      n = a.n;
      il = a.il1;
      iu = a.iu1;
      q.wout = 0;
      q.zout = 0;
      q.ldz = a.ldz;
    } else {
      q.row0 = a.d_off[p];
      int64_t nn = a.d_off[p + 1] - a.d_off[p];
      n = (nn >= 0 && nn <= INT32_MAX) ? (int)nn : -1;
      il = a.il ? a.il[p] : 1;
      iu = a.iu ? a.iu[p] : n;
      q.wout = a.w_off ? a.w_off[p] : 0;
      q.zout = a.z_off ? a.z_off[p] : 0;
      q.ldz = n > 0 ? n : 1;
    }
    bool ok = n >= 0 && n <= v.vscr_rows && (n == 0 || (il >= 1 && il <= iu && iu <= n));
    if (!ok) {
      set_status(v.ctl, MRRR_ERR_ARG);
      n = 0;
    }
    int ol = il, ou = iu;
    if (a.d_off == nullptr && a.slice) {
      ol = a.ol1;
      ou = a.ou1;
      if (n && (ol < il || ou > iu || ol > ou)) {
        set_status(v.ctl, MRRR_ERR_ARG);
        n = 0;
      }
    }
    q.n = n;
    q.il = n ? il : 1;
    q.iu = n ? iu : 0;
    q.ol = n ? ol : 1;
    q.ou = n ? ou : 0;
    q.slice = a.d_off == nullptr ? a.slice : 0;
    q.k = n ? ou - ol + 1 : 0;
    q.scale = 1.0;
    v.prob[p] = q;
  }
}

// ---------------------------------------------------------------------------
// One warp per problem: finiteness, G(T) = max_i |d_i|+|e_{i-1}|+|e_i|, the
// power-of-two scale with G(T)*scale in [1,2), and the number of blocks.
__global__ void k_prep(Dev v) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5;
  const int64_t nwarps = gstride() >> 5;
  for (int64_t p = warp; p < v.batch; p += nwarps) {
    Problem q = v.prob[p];
    double g = 0.0;
    bool bad = false;
    for (int64_t i = lane; i < q.n; i += 32) {
      double di = v.d[q.row0 + i];
      double r = fabs(di);
      bad |= !isfinite(di);
      if (i > 0) r += fabs(v.e[q.row0 + i - 1]);
      if (i + 1 < q.n) {
        double ei = v.e[q.row0 + i];
        bad |= !isfinite(ei);
        r += fabs(ei);
      }
      g = fmax(g, r);
    }
    for (int o = 16; o; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    bad = __any_sync(0xffffffffu, bad);
    double thresh = kEps * g;
    int splits = 0;
    if (!bad) {
      for (int64_t i0 = 0; i0 < q.n - 1; i0 += 32) {
        int64_t i = i0 + lane;
        bool sp = (i < q.n - 1) && fabs(v.e[q.row0 + i]) <= thresh;
        splits += __popc(__ballot_sync(0xffffffffu, sp));
      }
    }
    if (lane == 0) {
      if (bad) {
        set_status(v.ctl, MRRR_ERR_NONFINITE);
        q.n = 0;
        q.k = 0;
      }
      int ex = 0;
      if (g > 0.0 && !bad) {
        frexp(g, &ex);  // g = f * 2^ex, f in [0.5, 1)
        q.scale = ldexp(1.0, 1 - ex);
      } else {
        q.scale = 1.0;
      }
      q.thresh = thresh;
      q.nblocks = q.n ? 1 + splits : 0;
      if (q.n == 0)
        q.nslots = 0;
      else if (q.nblocks == 1)
        q.nslots = min(q.n, q.iu + 1) - max(1, q.il - 1) + 1;
      else
        q.nslots = q.n;
      v.prob[p] = q;
    }
  }
}

// ---------------------------------------------------------------------------
// Single CTA: exclusive prefix sums of blocks and slots over the problems.
__global__ void k_scan(Dev v, int64_t n_total) {
  __shared__ int64_t sb[32], ss[32];
  __shared__ int64_t carry_b, carry_s;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  if (t == 0) carry_b = carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < v.batch; base += blockDim.x) {
    int64_t p = base + t;
    int64_t nb = 0, ns = 0;
    if (p < v.batch) {
      nb = v.prob[p].nblocks;
      ns = v.prob[p].nslots;
    }
    int64_t xb = nb, xs = ns;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      int64_t yb = __shfl_up_sync(0xffffffffu, xb, o);
      int64_t ys = __shfl_up_sync(0xffffffffu, xs, o);
      if (lane >= o) xb += yb, xs += ys;
    }
    if (lane == 31) sb[wid] = xb, ss[wid] = xs;
    __syncthreads();
    if (wid == 0) {
      int64_t wb = lane < nw ? sb[lane] : 0, ws = lane < nw ? ss[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t yb = __shfl_up_sync(0xffffffffu, wb, o);
        int64_t ys = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) wb += yb, ws += ys;
      }
      if (lane < nw) sb[lane] = wb, ss[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    int64_t offb = carry_b + (wid ? sb[wid - 1] : 0) + xb - nb;
    int64_t offs = carry_s + (wid ? ss[wid - 1] : 0) + xs - ns;
    if (p < v.batch) {
      v.prob[p].block0 = (int)offb;
      v.prob[p].slot0 = offs;
    }
    __syncthreads();
    if (t == 0) carry_b += sb[nw - 1], carry_s += ss[nw - 1];
    __syncthreads();
  }
  if (t == 0) {
    Ctl* c = v.ctl;
    if (carry_b > v.max_blocks || carry_s > v.max_slots || carry_b > v.max_nodes) {
      set_status(c, MRRR_ERR_WORKSPACE);
      carry_b = 0;
      carry_s = 0;
    }
    c->nblocks = (int)carry_b;
    c->nslots = carry_s;
    c->nodes = (int)carry_b;
    c->pool_top = n_total;
    c->pool_need = n_total;
  }
}

// ---------------------------------------------------------------------------
// One warp per problem: enumerate the blocks (row ranges between splits) and
// initialise their slots.
__global__ void k_blocks(Dev v) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5;
  const int64_t nwarps = gstride() >> 5;
  if (v.ctl->nblocks == 0) return;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t p = warp; p < v.batch; p += nwarps) {
    const Problem q = v.prob[p];
    if (q.n == 0) continue;
    int nb = 0;        // blocks emitted so far
    int64_t start = 0; // start row (local) of the next block
    for (int64_t i0 = 0; i0 < q.n; i0 += 32) {
      int64_t i = i0 + lane;
      bool end = (i == q.n - 1) || (i < q.n - 1 && fabs(v.e[q.row0 + i]) <= q.thresh);
      unsigned mask = __ballot_sync(0xffffffffu, end);
      if (end) {
        int rank = __popc(mask & lt);
        unsigned prev = mask & lt;
        int64_t s0 = prev ? (i0 + 31 - __clz(prev)) + 1 : start;
        int b = q.block0 + nb + rank;
        Block bk;
        bk.row0 = q.row0 + s0;
        bk.m = (int)(i - s0 + 1);
        bk.prob = (int)p;
        if (q.nblocks == 1) {
          bk.js = max(1, q.il - 1);
          bk.je = min(q.n, q.iu + 1);
          bk.slot0 = q.slot0;
        } else {
          bk.js = 1;
          bk.je = bk.m;
          bk.slot0 = q.slot0 + s0;
        }
        bk.gl = bk.gu = 0.0;
        v.blk[b] = bk;
        if (q.nblocks > 1) {  // slots of this block (one lane each block)
          for (int j = bk.js; j <= bk.je; ++j) {
            int64_t w = bk.slot0 + (j - bk.js);
            v.snode[w] = b;
            v.sj[w] = j;
            v.spos[w] = -1;  // set by the rank pass
            v.state[w] = bk.m == 1 ? SLOT_TRIVIAL : SLOT_ACTIVE;
          }
        }
      }
      if (mask) {
        int last = 31 - __clz(mask);
        start = i0 + last + 1;
        nb += __popc(mask);
      }
    }
    if (q.nblocks == 1) {  // slots of the single block, all lanes
      const int b = q.block0;
      const int js = max(1, q.il - 1), je = min(q.n, q.iu + 1);
      for (int j = js + lane; j <= je; j += 32) {
        int64_t w = q.slot0 + (j - js);
        v.snode[w] = b;
        v.sj[w] = j;
        v.spos[w] = (j >= q.ol && j <= q.ou) ? j - q.ol : -1;
        v.state[w] = q.n == 1 ? SLOT_TRIVIAL : SLOT_ACTIVE;
      }
    }
  }
}

// L D L^T = T_b - sigma I of a block by the recurrence D_1 = d_1 - sigma,
// l_i = e_i / D_i, D_{i+1} = d_{i+1} - sigma - l_i e_i (store = write the
// rows).  Returns whether every pivot has the sign of a definite
// factorization (positive for a shift left of the spectrum, negative right
// of it) and is finite.
__device__ bool root_factor(const Dev& v, const Problem& q, int64_t lr0, int m, double sigma, bool left,
                            bool store, double2* dl, double2* ul) {
  double Dcur = scaled_d(v, q, lr0) - sigma;
  for (int i = 0; i < m - 1; ++i) {
    if (!(left ? Dcur > kPivmin : Dcur < -kPivmin) || !isfinite(Dcur)) return false;
    const double ei = scaled_e(v, q, lr0 + i);
    const double l = ei / Dcur;
    const double LD = l * Dcur;
    const double LLD = l * LD;
    if (store) rep_store(dl, ul, i, RepRow{Dcur, LLD, l, LD});
    Dcur = (scaled_d(v, q, lr0 + i + 1) - sigma) - LLD;
  }
  if (!(left ? Dcur > kPivmin : Dcur < -kPivmin) || !isfinite(Dcur)) return false;
  if (store) rep_store(dl, ul, m - 1, RepRow{Dcur, 0.0, 0.0, 0.0});
  return true;
}

constexpr int kRootTries = 12;

// Shift t of the root ladder: the Gershgorin end, pushed outward by
// 4^t 4 eps spdiam (t = 1..10), then by 5% of spdiam.
__device__ __forceinline__ double root_shift(int t, double gl, double gu, double spdiam, bool left) {
  double delta = (t == 0) ? 0.0 : spdiam * kEps * 4.0 * (double)(1LL << (2 * t));
  if (t == kRootTries - 1) delta = 0.05 * spdiam + kPivmin;
  return left ? gl - delta : gu + delta;
}

// One warp per block: Gershgorin bounds (lanes over rows), the root shift
// sigma at the end of the spectrum nearer the wanted indices, and
// L0 D0 L0^T = T - sigma I, definite.  Lane 0 factors at the first shift of
// the ladder with stores while lanes 1..11 test the others; if the first
// fails, the first that holds is factored again with stores.  The seeded
// perturbation, the norm of the rows and the bracket counts also run across
// the lanes.  When the eigenvector scratch has room for 11 rows per row of
// T, lanes 1..11 store their factorizations there too and the warp copies a
// winner other than lane 0's into place: the block then costs one
// sequential pass over its rows; otherwise the winner is factored again.
__global__ void k_root(Dev v) {
  const int nblocks = v.ctl->nblocks;
  const int lane = threadIdx.x & 31;
  for (int64_t b = gtid() >> 5; b < nblocks; b += gstride() >> 5) {
    Block bk = v.blk[b];
    const Problem q = v.prob[bk.prob];
    const int m = bk.m;
    const int64_t lr0 = bk.row0 - q.row0;  // local row of the block start
    double2* dl = v.rep_dl + bk.row0;
    double2* ul = v.rep_ul + bk.row0;
    Node nd;
    nd.block = (int)b;
    nd.depth = 0;
    nd.first = bk.slot0;
    nd.last = bk.slot0 + (bk.je - bk.js);
    nd.parent = -1;
    nd.pad_ = 0;
    nd.rep = bk.row0;
    nd.gapl = INFINITY;
    nd.gapr = INFINITY;
    nd.pivmin = kPivmin;
    if (m == 1) {
      if (lane == 0) {
        double d0 = scaled_d(v, q, lr0);
        rep_store(dl, ul, 0, RepRow{0.0, 0.0, 0.0, 0.0});
        nd.sigma_rel = nd.sigma_abs = d0;
        nd.spdiam = 0.0;
        bk.gl = bk.gu = 0.0;
        v.blk[b] = bk;
        v.node[b] = nd;
        v.lo[bk.slot0] = v.hi[bk.slot0] = 0.0;
      }
      continue;
    }
    double gl = INFINITY, gu = -INFINITY;
    for (int i = lane; i < m; i += 32) {
      double r = 0.0;
      if (i > 0) r += fabs(scaled_e(v, q, lr0 + i - 1));
      if (i + 1 < m) r += fabs(scaled_e(v, q, lr0 + i));
      double di = scaled_d(v, q, lr0 + i);
      gl = fmin(gl, di - r);
      gu = fmax(gu, di + r);
    }
    for (int o = 16; o; o >>= 1) {
      gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
      gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
    }
    const double spdiam = gu - gl;
    const double gmax = fmax(fabs(gl), fabs(gu));
    // wanted range in the lower half, unless the side is fixed by the options
    const bool left = v.root_side == 1 ? true : v.root_side == 2 ? false : (bk.js + bk.je) <= (m + 1);
    bool ok_t = false;
    // candidate rows of lanes 1..11 in the scratch, at 11 rows per row of T
    const bool spare = (int64_t)(kRootTries - 1) * (bk.row0 + m) <= cand_capacity(v);
    const int64_t srow = (int64_t)(kRootTries - 1) * bk.row0 + (int64_t)(lane - 1) * m;
    if (lane < kRootTries) {
      const bool own = lane == 0;
      ok_t = root_factor(v, q, lr0, m, root_shift(lane, gl, gu, spdiam, left), left, own || spare,
                         own ? dl : cand_dl(v) + srow, own ? ul : cand_ul(v) + srow);
    }
    const unsigned okm = __ballot_sync(0xffffffffu, ok_t);
    const int t = okm ? __ffs(okm) - 1 : kRootTries - 1;
    const double sigma = root_shift(t, gl, gu, spdiam, left);
    if (okm && t > 0 && spare) {  // the winner's rows from the scratch
      __syncwarp();
      const int64_t from = (int64_t)(kRootTries - 1) * bk.row0 + (int64_t)(t - 1) * m;
      for (int i = lane; i < m; i += 32) {
        dl[i] = cand_dl(v)[from + i];
        ul[i] = cand_ul(v)[from + i];
      }
      __syncwarp();
    } else if (t > 0 && lane == 0) {
      root_factor(v, q, lr0, m, sigma, left, true, dl, ul);
    }
    if (!okm && lane == 0) {
      set_status(v.ctl, MRRR_ERR_NOCONV);
      diag(v.ctl, DIAG_ROOT_SHIFT);
    }
    __syncwarp();
    // Seeded random relative perturbation of the root representation by a
    // few ulps (D_i and l_i times 1 + pert*eps*u, u in [-1,1) from a
    // counter-based generator on the row within the problem, so that a
    // problem gets the same representation alone or in a batch), which breaks
    // the exact coincidence of eigenvalues of identical glued blocks
    // (Dhillon, Parlett and Voemel, "Glued matrices and the MRRR algorithm",
    // 2005).  Rows are independent: lanes over rows.
    double R = 0.0;
    const double amp = v.root_perturb > 0.0 ? fmin(v.root_perturb, m / 8.0) * kEps : 0.0;
    // at most m/8 ulps: the eigenvalue budget 4 m eps ||T|| is tight for
    // small blocks, and glued copies only matter for large ones
    for (int i = lane; i < m; i += 32) {
      RepRow r = rep_row(dl, ul, i);
      if (amp > 0.0) {
        const uint64_t row = (uint64_t)(lr0 + i);
        const double u1 = uniform_pm1(splitmix64(2 * row));
        const double u2 = uniform_pm1(splitmix64(2 * row + 1));
        r.D *= 1.0 + amp * u1;
        r.l *= 1.0 + amp * u2;
        r.LD = r.l * r.D;
        r.LLD = r.l * r.LD;
        rep_store(dl, ul, i, r);
      }
      R = fmax(R, fmax(fabs(r.D), fabs(r.LLD)));
    }
    for (int o = 16; o; o >>= 1) R = fmax(R, __shfl_xor_sync(0xffffffffu, R, o));
    __syncwarp();
    nd.pivmin = pivmin_for(R);
    // initial bracket in root coordinates, checked with Sturm counts: lane 0
    // moves the lower end down, lane 1 the upper end up
    const double pad = 4.0 * kEps * m * (gmax + spdiam) + 4.0 * kPivmin;
    const double lo0 = gl - sigma - pad, hi0 = gu - sigma + pad;
    double x = lane == 0 ? lo0 : hi0;
    if (lane < 2) {
      const double step = hi0 - lo0;
      for (int k = 0; k < 60; ++k) {
        const int c = negcount(dl, m, x, nd.pivmin);
        if (lane == 0 ? c == 0 : c == m) break;
        x += (lane == 0 ? -step : step) * (double)(1LL << k);
      }
    }
    const double lo = __shfl_sync(0xffffffffu, x, 0), hi = __shfl_sync(0xffffffffu, x, 1);
    if (lane == 0) {
      bk.gl = lo;
      bk.gu = hi;
      nd.sigma_rel = nd.sigma_abs = sigma;
      nd.spdiam = spdiam;
      v.blk[b] = bk;
      v.node[b] = nd;
    }
  }
}

// ---------------------------------------------------------------------------
// Problems split into several blocks: the output column of each slot is its
// rank among the problem's eigenvalues (by interval midpoint in absolute
// scaled coordinates; ties by slot order, i.e. by block), shifted by il-1.
__device__ __forceinline__ double slot_key(const Dev& v, int64_t w) {
  const Node& nd = v.node[v.snode[w]];
  return nd.sigma_abs + 0.5 * (v.lo[w] + v.hi[w]);
}

__global__ void k_rank(Dev v) {
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid(); w < nslots; w += gstride()) {
    const int p = v.blk[v.snode[w]].prob;
    const Problem q = v.prob[p];
    if (q.nblocks <= 1) continue;
    const double key = slot_key(v, w);
    int64_t rank = 0;
    for (int64_t u = q.slot0; u < q.slot0 + q.nslots; ++u) {
      double ku = slot_key(v, u);
      rank += (ku < key) || (ku == key && u < w);
    }
    int64_t pos = rank - (q.ol - 1);
    v.spos[w] = (pos >= 0 && pos < q.k) ? (int)pos : -1;
  }
}

}  // namespace

void launch_setup(const Dev& v, const ProblemArgs& a, int64_t n_total, const Grid& g, cudaStream_t s) {
  const int pb = (int)std::min<int64_t>((a.batch + 127) / 128, (int64_t)g.nsm * 8);
  k_problems<<<std::max(pb, 1), 128, 0, s>>>(v, a);
  count_launch();
  const int wb = (int)std::min<int64_t>((a.batch * 32 + 127) / 128, (int64_t)g.nsm * 16);
  k_prep<<<std::max(wb, 1), 128, 0, s>>>(v);
  count_launch();
  k_scan<<<1, 1024, 0, s>>>(v, n_total);
  count_launch();
  k_blocks<<<std::max(wb, 1), 128, 0, s>>>(v);
  count_launch();
  mark_stage("prep", s);
  k_root<<<std::max(wb, 1), 128, 0, s>>>(v);
  count_launch();
  mark_stage("root", s);
  launch_engine(v, 0, g, s, n_total);
  mark_stage("bisect_root", s);
  k_rank<<<g.slot_blocks, g.tpb, 0, s>>>(v);
  count_launch();
  mark_stage("rank", s);
}

}  // namespace mrrr
