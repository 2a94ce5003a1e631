// mrrr_vec.cu -- eigenvectors of singletons by one twisted factorization each
// on the node's representation (Sec. 3.1.1: a singleton's vector is computed
// in isolation from its representation, with the error bound of the
// eigenvector-angle inequality), the normalisation of the columns of Z, an
// orthogonality safeguard between neighbouring columns, and the ordering of
// split problems.
//
// The eigenvalue comes in bisected to full relative accuracy (the interval
// engine's FINAL mode), so a single twisted factorization suffices.
// Twisted factorization of L D L^T - lambda I at twist index r:
//   stationary (top-down)   s_1 = -lambda, D+_i = D_i + s_i,
//                           L+_i = LD_i / D+_i, s_{i+1} = L+_i l_i s_i - lambda
//   progressive (bottom-up) p_m = D_m - lambda, D-_{i+1} = LLD_i + p_{i+1},
//                           U-_i = LD_i / D-_{i+1},
//                           p_i = p_{i+1} D_i / D-_{i+1} - lambda
//   twist                   gamma_r = s_r + p_r + lambda, r = argmin |gamma_r|
//   solve N_r z = gamma_r e_r with z_r = 1:
//                           z_i = -L+_i z_{i+1} (i < r), z_{i+1} = -U-_i z_i (i >= r)
// The residual of (L D L^T - lambda I) z is |gamma_r| / ||z||.
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {

namespace {

constexpr int kRowAhead = 4;  // representation rows loaded ahead of the qd recurrences

// A: L+ (stride as), B: s then U- (stride bs), z: output (stride zs; may alias A).
// Returns the Sturm count (negative pivots of the stationary part).  The
// representation rows are read kRowAhead rows ahead of the recurrences, whose
// dependent chains (a division per row) do not wait on the loads.
__device__ int twisted_solve(const double2* __restrict__ dl, const double2* __restrict__ ul, int m, double lam,
                             double pivmin,
                             double* A, int64_t as, double* B, int64_t bs, double* z, int64_t zs,
                             int& r, double& gamma, double& norm2) {
  int negc = 0;
  double s = -lam;
  double2 pd[kRowAhead], pu[kRowAhead];
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    pd[u] = u < m - 1 ? __ldg(dl + u) : make_double2(0.0, 0.0);
    pu[u] = u < m - 1 ? __ldg(ul + u) : make_double2(0.0, 0.0);
  }
  for (int i0 = 0; i0 < m - 1; i0 += kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 + u;
      const double2 xd = pd[u], xu = pu[u];
      const int inext = i + kRowAhead;
      pd[u] = inext < m - 1 ? __ldg(dl + inext) : make_double2(0.0, 0.0);
      pu[u] = inext < m - 1 ? __ldg(ul + inext) : make_double2(0.0, 0.0);
      if (i < m - 1) {
        double dp = xd.x + s;
        if (fabs(dp) < pivmin) dp = -pivmin;
        negc += (dp < 0.0);
        const double lp = xu.y / dp;  // LD / D+
        A[i * as] = lp;
        B[i * bs] = s;
        s = fma(lp, xu.x * s, -lam);  // L+ l s - lambda
      }
    }
  }
  {
    double dp = dl[m - 1].x + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    negc += (dp < 0.0);
    B[(int64_t)(m - 1) * bs] = s;
  }
  double p = dl[m - 1].x - lam;
  double g = s + p + lam;
  double best = fabs(g);
  r = m - 1;
  gamma = g;
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    const int i = m - 2 - u;
    pd[u] = i >= 0 ? __ldg(dl + i) : make_double2(0.0, 0.0);
    pu[u] = i >= 0 ? __ldg(ul + i) : make_double2(0.0, 0.0);
  }
  for (int i0 = m - 2; i0 >= 0; i0 -= kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 - u;
      const double2 xd = pd[u], xu = pu[u];
      const int inext = i - kRowAhead;
      pd[u] = inext >= 0 ? __ldg(dl + inext) : make_double2(0.0, 0.0);
      pu[u] = inext >= 0 ? __ldg(ul + inext) : make_double2(0.0, 0.0);
      if (i >= 0) {
        double dm = xd.y + p;  // LLD + p
        if (fabs(dm) < pivmin) dm = -pivmin;
        const double t = xd.x / dm;  // D / D-
        const double um = xu.x * t;  // l D / D-
        p = fma(p, t, -lam);
        g = B[i * bs] + p + lam;
        if (fabs(g) <= best) {
          best = fabs(g);
          r = i;
          gamma = g;
        }
        B[i * bs] = um;
      }
    }
  }
  double zi = 1.0, n2 = 1.0;
  z[(int64_t)r * zs] = 1.0;
  for (int i = r - 1; i >= 0; --i) {
    zi = -A[i * as] * zi;
    z[i * zs] = zi;
    n2 = fma(zi, zi, n2);
  }
  zi = 1.0;
  for (int i = r; i < m - 1; ++i) {
    zi = -B[i * bs] * zi;
    z[(int64_t)(i + 1) * zs] = zi;
    n2 = fma(zi, zi, n2);
  }
  norm2 = n2;
  return negc;
}

__global__ void k_vectors(Dev v) {
  const int64_t tid = gtid(), nthr = gstride();
  const int64_t nslots = v.ctl->nslots;
  double* B = v.vscr + tid;
  unsigned long long iters = 0;
  for (int64_t w = tid; w < nslots; w += nthr) {
    const int st = v.state[w];
    if (st != SLOT_SINGLETON && st != SLOT_FALLBACK && st != SLOT_TRIVIAL) continue;
    const int pos = v.spos[w];
    if (pos < 0) continue;
    const Node nd = v.node[v.snode[w]];
    const Block bk = v.blk[nd.block];
    const Problem q = v.prob[bk.prob];
    const int m = bk.m;
    double* zc = v.Z ? v.Z + q.zout + (int64_t)pos * q.ldz + (bk.row0 - q.row0) : nullptr;
    if (st == SLOT_TRIVIAL || m == 1) {
      v.W[q.wout + pos] = nd.sigma_abs / q.scale;
      if (zc) zc[0] = 1.0;
      v.znrm2[w] = 1.0;
      continue;
    }
    if (!zc) {  // eigenvalues only: the bisected value is final
      v.W[q.wout + pos] = (nd.sigma_abs + 0.5 * (v.lo[w] + v.hi[w])) / q.scale;
      continue;
    }
    double* A = zc;
    const int64_t as = 1;
    const double2* rdl = v.rep_dl + nd.rep;
    const double2* rul = v.rep_ul + nd.rep;
    // the eigenvalue was bisected to full relative accuracy on this
    // representation: one twisted factorization gives the vector
    const double lam = 0.5 * (v.lo[w] + v.hi[w]);
    int r;
    double gamma, n2;
    twisted_solve(rdl, rul, m, lam, nd.pivmin, A, as, B, nthr, A, as, r, gamma, n2);
    ++iters;
    const double lam_out = lam;
    if (!isfinite(n2)) set_status(v.ctl, MRRR_ERR_NOCONV);
    v.W[q.wout + pos] = (nd.sigma_abs + lam_out) / q.scale;
    v.wval[w] = lam_out;
    v.znrm2[w] = n2;
    if (!zc) continue;
  }
  if (iters) atomicAdd(&v.ctl->twisted_solves, iters);
}

// One CTA per output slot: scale the column to unit norm and clear the rows
// outside its block (problems that split).
__global__ void k_normalize(Dev v) {
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = blockIdx.x; w < nslots; w += gridDim.x) {
    const int st = v.state[w];
    if (st != SLOT_SINGLETON && st != SLOT_FALLBACK && st != SLOT_TRIVIAL) continue;
    const int pos = v.spos[w];
    if (pos < 0) continue;
    const Node& nd = v.node[v.snode[w]];
    const Block& bk = v.blk[nd.block];
    const Problem& q = v.prob[bk.prob];
    double* col = v.Z + q.zout + (int64_t)pos * q.ldz;
    const double sc = 1.0 / sqrt(v.znrm2[w]);
    const int64_t r0 = bk.row0 - q.row0, r1 = r0 + bk.m;
    if (q.nblocks > 1) {
      for (int64_t i = threadIdx.x; i < q.n; i += blockDim.x)
        col[i] = (i >= r0 && i < r1) ? col[i] * sc : 0.0;
    } else {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) col[i] *= sc;
    }
  }
}

// Orthogonality safeguard.  A singleton computed on a representation with
// large element growth can carry an error of c eps / relgap along its
// nearest neighbours with c well above one; the inner products with the next
// kOrthNeighbors columns of the same block find such pairs, and runs of
// linked columns are re-orthogonalised (modified Gram-Schmidt, twice, in
// eigenvalue order), which removes exactly that component: the residual of a
// changed column grows by at most |z_i^T z_j| |lambda_j - lambda_i|.
constexpr int kOrthNeighbors = 8;
constexpr double kOrthFixTol = 10.0;  // link when |z_i^T z_j| > 10 m eps (block order m)

__device__ __forceinline__ const double* slot_column(const Dev& v, int64_t w, const Block& bk, const Problem& q) {
  return v.Z + q.zout + (int64_t)v.spos[w] * q.ldz + (bk.row0 - q.row0);
}

__device__ __forceinline__ bool slot_has_column(const Dev& v, int64_t w) {
  const int st = v.state[w];
  return (st == SLOT_SINGLETON || st == SLOT_FALLBACK || st == SLOT_TRIVIAL) && v.spos[w] >= 0;
}

__device__ __forceinline__ double warp_dot(const double* a, const double* b, int m, int lane) {
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s = fma(a[i], b[i], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One warp per slot: link[w] = largest k <= kOrthNeighbors with
// |z_w^T z_{w+k}| above the threshold (0 if none).  The per-slot index array
// sj (no longer needed once the eigenvalues are final) holds the links.
__global__ void k_orth_links(Dev v) {
  const int lane = threadIdx.x & 31;
  const int64_t nslots = v.ctl->nslots;
  for (int64_t w = gtid() >> 5; w < nslots; w += gstride() >> 5) {
    int link = 0;
    if (slot_has_column(v, w)) {
      const Block bk = v.blk[v.node[v.snode[w]].block];
      const Problem q = v.prob[bk.prob];
      const int64_t last = bk.slot0 + (bk.je - bk.js);
      const double thr = kOrthFixTol * bk.m * kEps;
      const double* zw = slot_column(v, w, bk, q);
      for (int k = 1; k <= kOrthNeighbors && w + k <= last; ++k) {
        if (!slot_has_column(v, w + k)) continue;
        const double dot = warp_dot(zw, slot_column(v, w + k, bk, q), bk.m, lane);
        if (fabs(dot) > thr) link = k;
      }
    }
    if (lane == 0) v.sj[w] = link;
  }
}

// One warp per block: runs of linked slots, each re-orthogonalised in order.
__global__ void k_orth_fix(Dev v) {
  const int lane = threadIdx.x & 31;
  const int nblocks = v.ctl->nblocks;
  for (int64_t b = gtid() >> 5; b < nblocks; b += gstride() >> 5) {
    const Block bk = v.blk[b];
    if (bk.m < 2 || bk.je < bk.js) continue;
    const Problem q = v.prob[bk.prob];
    const int64_t s0 = bk.slot0, s1 = bk.slot0 + (bk.je - bk.js);
    const int m = bk.m;
    int64_t w = s0;
    while (w <= s1) {
      // next linked slot at or after w, 32 slots per step
      const int64_t t0 = w + lane;
      const unsigned msk = __ballot_sync(0xffffffffu, t0 <= s1 && v.sj[t0] != 0);
      if (!msk) {
        w += 32;
        continue;
      }
      const int64_t start = w + __ffs(msk) - 1;
      int64_t reach = start + v.sj[start];
      for (int64_t t = start + 1; t <= reach && t <= s1; ++t) reach = max(reach, t + (int64_t)v.sj[t]);
      reach = min(reach, s1);
      if (lane == 0) diag(v.ctl, DIAG_ORTH_FIX);
      for (int64_t c = start + 1; c <= reach; ++c) {
        if (!slot_has_column(v, c)) continue;
        double* zc = const_cast<double*>(slot_column(v, c, bk, q));
        for (int pass = 0; pass < 2; ++pass) {
          for (int64_t p = start; p < c; ++p) {
            if (!slot_has_column(v, p)) continue;
            const double* zp = slot_column(v, p, bk, q);
            const double dot = warp_dot(zc, zp, m, lane);
            for (int i = lane; i < m; i += 32) zc[i] = fma(-dot, zp[i], zc[i]);
            __syncwarp();
          }
        }
        const double n2 = warp_dot(zc, zc, m, lane);
        const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
        for (int i = lane; i < m; i += 32) zc[i] *= sc;
        __syncwarp();
      }
      w = reach + 1;
    }
  }
}

// Split problems: columns were placed by the rank of interval midpoints;
// near-ties across blocks may leave W slightly out of order.  Odd-even
// transposition passes (one CTA per problem) restore ascending W, moving the
// columns of Z along.
__global__ void k_fix_order(Dev v) {
  __shared__ int swapped;
  for (int64_t p = blockIdx.x; p < v.batch; p += gridDim.x) {
    const Problem q = v.prob[p];
    if (q.nblocks <= 1 || q.k < 2) continue;
    double* W = v.W + q.wout;
    int quiet = 0;
    for (int pass = 0; pass < 2 * q.k + 2 && quiet < 2; ++pass) {
      if (threadIdx.x == 0) swapped = 0;
      __syncthreads();
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int64_t i = (pass & 1) + 2 * (int64_t)wid; i + 1 < q.k; i += 2 * (int64_t)nw) {
        double a = W[i], b = W[i + 1];
        if (a > b) {
          if (lane == 0) {
            W[i] = b;
            W[i + 1] = a;
            swapped = 1;
          }
          if (v.Z) {
            double* ca = v.Z + q.zout + i * q.ldz;
            double* cb = ca + q.ldz;
            for (int64_t r = lane; r < q.n; r += 32) {
              double t = ca[r];
              ca[r] = cb[r];
              cb[r] = t;
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
      quiet = swapped ? 0 : quiet + 1;
      __syncthreads();
    }
  }
}

}  // namespace

void launch_vectors(const Dev& v, const Grid& g, cudaStream_t s) {
  k_vectors<<<g.vec_blocks, 128, 0, s>>>(v);
  count_launch();
  if (v.Z) {
    k_normalize<<<g.nsm * 16, 256, 0, s>>>(v);
    count_launch();
    k_orth_links<<<g.nsm * 16, 256, 0, s>>>(v);
    count_launch();
    k_orth_fix<<<g.nsm * 4, 128, 0, s>>>(v);
    count_launch();
  }
  k_fix_order<<<g.nsm, 256, 0, s>>>(v);
  count_launch();
}

}  // namespace mrrr
