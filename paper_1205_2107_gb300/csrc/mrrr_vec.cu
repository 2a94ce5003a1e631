// mrrr_vec.cu -- eigenvectors of singletons by one twisted factorization each
// on the node's representation (Sec. 3.1.1: a singleton's vector is computed
// in isolation from its representation, with the error bound of the
// eigenvector-angle inequality), the normalisation of the columns of Z, an
// orthogonality safeguard between neighbouring columns, and the ordering of
// split problems.
//
// The eigenvalue comes in bisected to full relative accuracy (the interval
// engine's FINAL mode), so a single twisted factorization suffices; with
// Rayleigh-quotient corrections (option singleton_rq) it comes in to 2^-36
// and each correction takes one more factorization.
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

constexpr int kRowAhead = 4;    // representation and scratch rows loaded ahead of the recurrences
constexpr int kVecWarps = 4;    // 128 threads per CTA
constexpr int kVecCtasPerSm = 4;  // what the register cap (128) lets reside: every SM full
constexpr int kStageRows = 16;  // rows of z staged per lane before a coalesced flush
constexpr int kPairAhead = 8;   // scratch rows loaded ahead in the two-lane form's gamma and solve sweeps

// The 32 vectors of a warp are computed in row lockstep: every sweep runs over
// the rows in the same order for all lanes (a lane idles on rows outside its
// range), so the interleaved scratch (row i of thread t at i * nthr + t) is
// read and written in whole 256-byte rows, and z leaves through a shared
// staging tile: kStageRows rows of all 32 lanes, flushed column by column as
// 128-byte runs of consecutive rows.
struct VecLane {
  const double2* dl;  // (D, LLD) rows of the node's representation
  const double2* ul;  // (l, LD) rows
  double* zc;         // column of Z (rows of the block), nullptr when idle
  double lam;         // eigenvalue in the node's coordinates
  double pivmin;
  int m;              // rows of the block (0 when idle)
};

// Rows [c0, c0 + kStageRows) of each lane's column, restricted to the lane's
// range [lo, hi], from stage[row - c0][lane] to Z: two columns per step, 16
// lanes per column.
__device__ __forceinline__ void flush_stage(double (*stage)[33], int c0, double* zc, int lo, int hi, int lane) {
  __syncwarp();
  const int half = lane >> 4, rr = lane & 15;
  for (int L0 = 0; L0 < 32; L0 += 2) {
    const int L = L0 + half;
    const long long zp = __shfl_sync(0xffffffffu, (long long)zc, L);
    const int l = __shfl_sync(0xffffffffu, lo, L), h = __shfl_sync(0xffffffffu, hi, L);
    const int row = c0 + rr;
    if (zp && row >= l && row <= h) reinterpret_cast<double*>(zp)[row] = stage[rr][L];
  }
  __syncwarp();
}

// Twisted factorization of L D L^T - lam I for the warp's vectors and the
// solve, with z written to the lanes' columns of Z.  A (L+) and B (s, then
// U-) are the lane's interleaved scratch rows (stride nthr).  Returns, per
// lane, the twist index r, gamma_r and ||z||^2.
__device__ void twisted_warp(const VecLane& q, double* __restrict__ A, double* __restrict__ B, int64_t nthr,
                             double (*stage)[33], int lane, int& r_out, double& gamma_out, double& norm2_out) {
  const bool act = q.m > 0;
  const int m = q.m;
  int M = m;
  for (int o = 16; o; o >>= 1) M = max(M, __shfl_xor_sync(0xffffffffu, M, o));
  const double lam = q.lam, pivmin = q.pivmin;
  // stationary transform, top-down: D+_i = D_i + s_i, L+_i = LD_i / D+_i,
  // s_{i+1} = L+_i l_i s_i - lam; L+ to A, s to B
  double s = -lam;
  double2 pd[kRowAhead], pu[kRowAhead];
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    pd[u] = u < m - 1 ? __ldg(q.dl + u) : make_double2(0.0, 0.0);
    pu[u] = u < m - 1 ? __ldg(q.ul + u) : make_double2(0.0, 0.0);
  }
  for (int i0 = 0; i0 < M - 1; i0 += kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 + u;
      const double2 xd = pd[u], xu = pu[u];
      const int inext = i + kRowAhead;
      pd[u] = inext < m - 1 ? __ldg(q.dl + inext) : make_double2(0.0, 0.0);
      pu[u] = inext < m - 1 ? __ldg(q.ul + inext) : make_double2(0.0, 0.0);
      if (i < m - 1) {
        double dp = xd.x + s;
        if (fabs(dp) < pivmin) dp = -pivmin;
        const double lp = xu.y / dp;  // LD / D+
        A[i * nthr] = lp;
        B[i * nthr] = s;
        s = fma(lp, xu.x * s, -lam);  // L+ l s - lambda
      }
    }
  }
  double p = 0.0, g = 0.0, best = INFINITY, gamma = 0.0;
  int r = 0;
  if (act) {
    p = q.dl[m - 1].x - lam;
    g = s + p + lam;
    best = fabs(g);
    r = m - 1;
    gamma = g;
  }
  // progressive transform, bottom-up over the rows M-2 .. 0 (a lane joins at
  // its own m-2): D-_{i+1} = LLD_i + p_{i+1}, U-_i = LD_i / D-_{i+1},
  // p_i = p_{i+1} D_i / D-_{i+1} - lam; gamma_i = s_i + p_i + lam; U- to B
  double sb[kRowAhead];
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    const int i = M - 2 - u;
    const bool ok = i >= 0 && i <= m - 2;
    pd[u] = ok ? __ldg(q.dl + i) : make_double2(0.0, 0.0);
    pu[u] = ok ? __ldg(q.ul + i) : make_double2(0.0, 0.0);
    sb[u] = ok ? B[i * nthr] : 0.0;
  }
  for (int i0 = M - 2; i0 >= 0; i0 -= kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 - u;
      const double2 xd = pd[u], xu = pu[u];
      const double si = sb[u];
      const int inext = i - kRowAhead;
      const bool ok = inext >= 0 && inext <= m - 2;
      pd[u] = ok ? __ldg(q.dl + inext) : make_double2(0.0, 0.0);
      pu[u] = ok ? __ldg(q.ul + inext) : make_double2(0.0, 0.0);
      sb[u] = ok ? B[inext * nthr] : 0.0;
      if (i >= 0 && i <= m - 2) {
        double dm = xd.y + p;  // LLD + p
        if (fabs(dm) < pivmin) dm = -pivmin;
        const double t = xd.x / dm;  // D / D-
        const double um = xu.x * t;  // l D / D-
        p = fma(p, t, -lam);
        g = si + p + lam;
        if (fabs(g) <= best) {
          best = fabs(g);
          r = i;
          gamma = g;
        }
        B[i * nthr] = um;
      }
    }
  }
  // solve N_r z = gamma_r e_r with z_r = 1: upward z_i = -L+_i z_{i+1}
  // (i < r), downward z_{i+1} = -U-_i z_i (i >= r)
  if (act) q.zc[r] = 1.0;
  // ||z||^2 = (1 + upper part) + lower part, each part summed away from r
  // (the order the two-lane form of twisted_pair uses as well)
  double up = 0.0, down = 0.0;
  int R = act ? r : 0;
  for (int o = 16; o; o >>= 1) R = max(R, __shfl_xor_sync(0xffffffffu, R, o));
  double z = 1.0;
  double ab[kRowAhead];
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    const int i = R - 1 - u;
    ab[u] = (act && i >= 0 && i < r) ? A[i * nthr] : 0.0;
  }
  for (int i0 = R - 1; i0 >= 0; i0 -= kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 - u;
      const double a = ab[u];
      const int inext = i - kRowAhead;
      ab[u] = (act && inext >= 0 && inext < r) ? A[inext * nthr] : 0.0;
      if (i >= 0) {
        if (act && i < r) {
          z = -a * z;
          up = fma(z, z, up);
          stage[i & (kStageRows - 1)][lane] = z;
        }
        if ((i & (kStageRows - 1)) == 0) flush_stage(stage, i, q.zc, 0, r - 1, lane);
      }
    }
  }
  int Rmin = act ? r : INT32_MAX;
  for (int o = 16; o; o >>= 1) Rmin = min(Rmin, __shfl_xor_sync(0xffffffffu, Rmin, o));
  z = 1.0;
  // rows j = i + 1 from Rmin + 1 to M - 1; lane active for r < j <= m - 1
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    const int i = Rmin + u;
    ab[u] = (act && i >= r && i <= m - 2) ? B[i * nthr] : 0.0;
  }
  for (int i0 = Rmin; i0 <= M - 2; i0 += kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int i = i0 + u;
      const double b = ab[u];
      const int inext = i + kRowAhead;
      ab[u] = (act && inext >= r && inext <= m - 2) ? B[inext * nthr] : 0.0;
      if (i <= M - 2) {
        const int j = i + 1;
        if (act && i >= r && i <= m - 2) {
          z = -b * z;
          down = fma(z, z, down);
          stage[j & (kStageRows - 1)][lane] = z;
        }
        if ((j & (kStageRows - 1)) == kStageRows - 1 || j == M - 1)
          flush_stage(stage, j & ~(kStageRows - 1), q.zc, r + 1, m - 1, lane);
      }
    }
  }
  r_out = r;
  gamma_out = gamma;
  norm2_out = (1.0 + up) + down;
}

// The same twisted factorization with two lanes per vector (lane pairs
// 2k, 2k+1 of the warp), for vectors too few to fill the GPU, where the
// recurrences' latency, not the FP64 pipe, sets the time.  Both lanes run
// one instruction stream on different rows:
//   1. the even ("top") lane the stationary transform top-down (L+ and s
//      into its scratch), the odd ("bottom") lane the progressive transform
//      bottom-up (U- and p into its scratch) -- one recurrence each,
//      x = a + s, q = b / x, out = c1 q, s <- c2 s q - lam, with
//      (a, b, c1, c2) = (D, LD, 1, l) top and (LLD, D, l, 1) bottom;
//   2. gamma_i = s_i + p_i + lam over the lower half of the rows (top) and
//      the upper half (bottom), each reading its own and its partner's
//      scratch, and r = argmin |gamma_i| (lowest index on ties);
//   3. the solve from z_r = 1, upward with L+ (top) and downward with U-
//      (bottom), z stored directly.
// Every value is computed by the same operations in the same order as in
// twisted_warp, so the vector, gamma_r and ||z||^2 come out bit for bit the
// same.  Returns r, gamma_r and ||z||^2 in both lanes.
__device__ __noinline__ void twisted_pair(const VecLane& q, double* __restrict__ A, double* __restrict__ B, int64_t nthr,
                             int lane, int& r_out, double& gamma_out, double& norm2_out) {
  const bool top = (lane & 1) == 0;
  const bool act = q.m > 0;
  const int m = q.m;
  int M = m;
  for (int o = 16; o; o >>= 1) M = max(M, __shfl_xor_sync(0xffffffffu, M, o));
  const double lam = q.lam, pivmin = q.pivmin;
  // partner's scratch columns (the pair's threads are neighbours)
  const double* Bp = top ? B + 1 : B - 1;
  // 1. the two transforms, row i = k (top) or m - 2 - k (bottom)
  double s = top ? -lam : (act ? q.dl[m - 1].x - lam : 0.0);
  if (act && !top) B[(int64_t)(m - 1) * nthr] = s;  // p_{m-1}
  double2 pd[kRowAhead], pu[kRowAhead];
#pragma unroll
  for (int u = 0; u < kRowAhead; ++u) {
    const int i = top ? u : m - 2 - u;
    const bool ok = act && u < m - 1;
    pd[u] = ok ? __ldg(q.dl + i) : make_double2(0.0, 0.0);
    pu[u] = ok ? __ldg(q.ul + i) : make_double2(0.0, 0.0);
  }
  for (int k0 = 0; k0 < M - 1; k0 += kRowAhead) {
#pragma unroll
    for (int u = 0; u < kRowAhead; ++u) {
      const int k = k0 + u;
      const double2 xd = pd[u], xu = pu[u];
      const int knext = k + kRowAhead;
      const bool oknext = act && knext < m - 1;
      const int inext = top ? knext : m - 2 - knext;
      pd[u] = oknext ? __ldg(q.dl + inext) : make_double2(0.0, 0.0);
      pu[u] = oknext ? __ldg(q.ul + inext) : make_double2(0.0, 0.0);
      if (act && k < m - 1) {
        const int i = top ? k : m - 2 - k;
        const double a = top ? xd.x : xd.y;   // D | LLD
        const double b = top ? xu.y : xd.x;   // LD | D
        double x = a + s;
        if (fabs(x) < pivmin) x = -pivmin;
        const double qq = b / x;
        A[(int64_t)i * nthr] = top ? qq : xu.x * qq;  // L+ | U- = l D / D-
        const double s_new = top ? fma(qq, xu.x * s, -lam) : fma(s, qq, -lam);
        B[(int64_t)i * nthr] = top ? s : s_new;       // s_i | p_i
        s = s_new;
      }
    }
  }
  if (act && top) B[(int64_t)(m - 1) * nthr] = s;  // s_{m-1}
  __syncwarp();  // the partner's stores are visible
  // 2. gamma over the two halves; r = argmin |gamma|, lowest index on ties
  const int h = m / 2;
  const int lo = top ? 0 : h, hi = top ? h : m;
  int H = act ? hi - lo : 0;
  for (int o = 16; o; o >>= 1) H = max(H, __shfl_xor_sync(0xffffffffu, H, o));
  double best = INFINITY, gamma = 0.0;
  int r = m;
  double so[kPairAhead], sp[kPairAhead];  // own and partner rows, loaded ahead
#pragma unroll
  for (int u = 0; u < kPairAhead; ++u) {
    const bool ok = act && lo + u < hi;
    so[u] = ok ? B[(int64_t)(lo + u) * nthr] : 0.0;
    sp[u] = ok ? Bp[(int64_t)(lo + u) * nthr] : 0.0;
  }
  for (int j0 = 0; j0 < H; j0 += kPairAhead) {
#pragma unroll
    for (int u = 0; u < kPairAhead; ++u) {
      const int i = lo + j0 + u;
      const double own = so[u], other = sp[u];
      const int inext = i + kPairAhead;
      const bool ok = act && inext < hi;
      so[u] = ok ? B[(int64_t)inext * nthr] : 0.0;
      sp[u] = ok ? Bp[(int64_t)inext * nthr] : 0.0;
      if (act && i < hi) {
        const double g = (top ? own + other : other + own) + lam;  // (s_i + p_i) + lam
        const double ag = fabs(g);
        if (ag < best || (ag == best && i < r)) {
          best = ag;
          r = i;
          gamma = g;
        }
      }
    }
  }
  {
    const double ob = __shfl_xor_sync(0xffffffffu, best, 1);
    const int orr = __shfl_xor_sync(0xffffffffu, r, 1);
    const double og = __shfl_xor_sync(0xffffffffu, gamma, 1);
    if (ob < best || (ob == best && orr < r)) {
      best = ob;
      r = orr;
      gamma = og;
    }
  }
  if (act && r >= m) r = m - 1;  // no comparable gamma: the last row, as the one-lane form starts
  // 3. the solve: upward (top) rows r-1 .. 0 with L+, downward (bottom)
  // rows r+1 .. m-1 with U-
  if (act && top) q.zc[r] = 1.0;
  const int len = act ? (top ? r : m - 1 - r) : 0;
  int L = len;
  for (int o = 16; o; o >>= 1) L = max(L, __shfl_xor_sync(0xffffffffu, L, o));
  double z = 1.0, acc = 0.0;
  double av[kPairAhead];  // L+ / U- rows, loaded ahead
#pragma unroll
  for (int u = 0; u < kPairAhead; ++u) av[u] = u < len ? A[(int64_t)(top ? r - 1 - u : r + u) * nthr] : 0.0;
  for (int j0 = 0; j0 < L; j0 += kPairAhead) {
#pragma unroll
    for (int u = 0; u < kPairAhead; ++u) {
      const int j = j0 + u;
      const double a = av[u];
      const int jn = j + kPairAhead;
      av[u] = jn < len ? A[(int64_t)(top ? r - 1 - jn : r + jn) * nthr] : 0.0;
      if (j < len) {
        const int i = top ? r - 1 - j : r + j;  // scratch row
        z = -a * z;
        acc = fma(z, z, acc);
        q.zc[top ? i : i + 1] = z;
      }
    }
  }
  const double oacc = __shfl_xor_sync(0xffffffffu, acc, 1);
  const double upp = top ? acc : oacc, dwn = top ? oacc : acc;
  r_out = r;
  gamma_out = gamma;
  norm2_out = (1.0 + upp) + dwn;
}

template <bool RQ>
__global__ void __launch_bounds__(kVecWarps * 32, 4) k_vectors(Dev v) {
  __shared__ double stage_all[kVecWarps][kStageRows][33];
  const int lane = threadIdx.x & 31;
  double (*stage)[33] = stage_all[threadIdx.x >> 5];
  const int64_t nslots = v.ctl->nslots;
  // The grid fills every SM (kVecCtasPerSm CTAs, all resident), and the
  // warps that work are the first vscr_threads / (32 x 4 SMs) on each SM
  // sub-partition by the scheduler's rank: the same number on every
  // sub-partition however the hardware placed the CTAs.  A working warp's
  // scratch columns follow from its rank.
  const long long rank = sched_rank(v);
  const int64_t nthr = v.vscr_threads;  // scratch columns (the row stride)
  if (rank >= nthr / 32) return;
  const int64_t col = rank * 32 + lane;
  double* B = v.vscr + col;
  double* A = v.vscr + v.vscr_threads * v.vscr_rows + col;
  unsigned long long iters = 0;
  // chunks spread over the SM sub-partitions by the scheduler; every lane of
  // a warp works on the same chunk (warp-wide sweeps).  Whole waves (every
  // sub-partition the same number) of chunks of 32 consecutive slots, one
  // per lane; the slots past them in chunks of 16, two lanes per slot
  // (twisted_pair), which halves the length of the chunks that run where
  // the others have finished -- and of all chunks when the vectors are too
  // few for one wave.
  const long long wave = (long long)v.nsm * 4 * 32;
  const long long nmain = (nslots / wave) * wave;
  const long long nch_main = nmain / 32;
  const long long nchunks = nch_main + (nslots - nmain + 15) / 16;
  bool first = true;
  for (;;) {
    const long long chunk = sched_next(v, nchunks, nthr / 32, rank, first);
    if (chunk < 0) break;
    const bool pair = chunk >= nch_main;
    const bool lead = !pair || (lane & 1) == 0;  // the lane that writes a slot's results
    const int64_t w = pair ? nmain + (chunk - nch_main) * 16 + (lane >> 1) : chunk * 32 + lane;
    VecLane q{};
    int st = w < nslots ? v.state[w] : 0;
    const bool has = (st == SLOT_SINGLETON || st == SLOT_FALLBACK || st == SLOT_TRIVIAL) && v.spos[w] >= 0;
    Node nd{};
    Problem pr{};
    int pos = 0;
    if (has) {
      pos = v.spos[w];
      nd = v.node[v.snode[w]];
      const Block bk = v.blk[nd.block];
      pr = v.prob[bk.prob];
      const int m = bk.m;
      double* zc = v.Z ? v.Z + pr.zout + (int64_t)pos * pr.ldz + (bk.row0 - pr.row0) : nullptr;
      if (st == SLOT_TRIVIAL || m == 1) {
        if (lead) {
          v.W[pr.wout + pos] = nd.sigma_abs / pr.scale;
          if (zc) zc[0] = 1.0;
          v.znrm2[w] = 1.0;
        }
      } else if (!zc) {  // eigenvalues only: the bisected value is final
        if (lead) v.W[pr.wout + pos] = (nd.sigma_abs + 0.5 * (v.lo[w] + v.hi[w])) / pr.scale;
      } else {
        // the eigenvalue was bisected to full relative accuracy on this
        // representation: one twisted factorization gives the vector
        q.dl = v.rep_dl + nd.rep;
        q.ul = v.rep_ul + nd.rep;
        q.zc = zc;
        q.lam = 0.5 * (v.lo[w] + v.hi[w]);
        q.pivmin = nd.pivmin;
        q.m = m;
      }
    }
    if (!__any_sync(0xffffffffu, q.m > 0)) continue;
    int r;
    double gamma, n2;
    // Rayleigh-quotient corrections (rq_steps > 0): z^T (L D L^T - lam I) z =
    // gamma_r z_r with z_r = 1, so lam + gamma_r / ||z||^2 is the Rayleigh
    // quotient of the last vector; each new value, kept inside the
    // bisection bracket, gets a new twisted factorization, and the last
    // one's quotient is the eigenvalue.  After the second factorization
    // the warp stops early once no lane's correction exceeds 2 eps |lam|
    // (converged: a further factorization would repeat the vector).
    const double blo = (RQ && q.m > 0) ? v.lo[w] : 0.0;
    const double bhi = (RQ && q.m > 0) ? v.hi[w] : 0.0;
    int nfact = 0;
    for (int it = 0;; ++it) {
      if (pair)
        twisted_pair(q, A, B, nthr, lane, r, gamma, n2);
      else
        twisted_warp(q, A, B, nthr, stage, lane, r, gamma, n2);
      ++nfact;
      if (!RQ) break;
      bool small = true;
      if (q.m > 0) {
        const double nl = fmin(fmax(q.lam + gamma / n2, blo), bhi);
        small = fabs(nl - q.lam) <= 2.0 * kEps * fabs(q.lam);
        q.lam = nl;
      }
      if (it >= v.rq_steps || (it >= 1 && __all_sync(0xffffffffu, small))) break;
    }
    if (q.m > 0 && lead) {
      iters += nfact;
      if (!isfinite(n2)) set_status(v.ctl, MRRR_ERR_NOCONV);
      v.W[pr.wout + pos] = (nd.sigma_abs + q.lam) / pr.scale;
      v.wval[w] = q.lam;
      v.znrm2[w] = n2;
    }
  }
  if (iters) atomicAdd(&v.ctl->twisted_solves, iters);
}

// ---------------------------------------------------------------------------
// Double-double eigenvectors (vector_precision = 2).  A value is an
// unevaluated sum hi + lo with |lo| <= ulp(hi)/2, about 106 bits.  The
// building blocks are the classical error-free transformations: Knuth's
// two-sum (s + e = a + b exactly), the FMA two-product (p + e = a b exactly,
// e = fma(a, b, -p)), Dekker's renormalisation; division takes one FP64
// quotient, its remainder computed exactly with two-products, and one
// correction (a Newton step).  Accuracy about 2^-104 relative per operation.
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_renorm(double s, double e) {  // |s| >= |e|
  const double h = s + e;
  return dd{h, e - (h - s)};
}
__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return dd{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const dd s = dd_two_sum(x.hi, y.hi);
  const dd t = dd_two_sum(x.lo, y.lo);
  const dd u = dd_renorm(s.hi, s.lo + t.hi);
  return dd_renorm(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const double p = x.hi * y.hi;
  const double e = fma(x.hi, y.hi, -p);
  return dd_renorm(p, e + (x.hi * y.lo + x.lo * y.hi));
}
__device__ __forceinline__ dd dd_mul_d(dd x, double b) {
  const double p = x.hi * b;
  const double e = fma(x.hi, b, -p);
  return dd_renorm(p, e + x.lo * b);
}
__device__ __forceinline__ dd dd_div(dd x, dd y) {
  const double q1 = x.hi / y.hi;
  const dd r = dd_sub(x, dd_mul_d(y, q1));  // remainder x - q1 y
  const double q2 = r.hi / y.hi;
  return dd_renorm(q1, q2);
}
__device__ __forceinline__ dd dd_from(double a) { return dd{a, 0.0}; }

// One double-double twisted factorization of L D L^T - lam I (the rows of
// the representation, FP64, define it exactly: LD and LLD are recomputed
// from l and D) and the solve: returns the twist r, gamma_r and ||z||^2; with
// zc the vector (rounded to FP64) is written.  Scratch: four interleaved
// arrays (L+ hi/lo, then s and U- hi/lo) of stride nthr.
__device__ void twisted_dd(const double2* __restrict__ dl, const double2* __restrict__ ul, int m, dd lam,
                           double pivmin, double* Ah, double* Al, double* Bh, double* Bl, int64_t nthr, double* zc,
                           int& r_out, dd& gamma_out, dd& norm2_out) {
  // stationary, top-down: D+ = D + s, L+ = l D / D+, s' = L+ l s - lam
  dd s = dd_neg(lam);
  for (int i = 0; i < m - 1; ++i) {
    const double D = dl[i].x, l = ul[i].x;
    dd dp = dd_add(dd_from(D), s);
    if (fabs(dp.hi) < pivmin) dp = dd_from(-pivmin);
    const dd ld = dd_mul_d(dd_from(l), D);
    const dd lp = dd_div(ld, dp);
    Ah[i * nthr] = lp.hi;
    Al[i * nthr] = lp.lo;
    Bh[i * nthr] = s.hi;
    Bl[i * nthr] = s.lo;
    s = dd_sub(dd_mul(dd_mul_d(lp, l), s), lam);
  }
  // progressive, bottom-up: D- = l^2 D + p, t = D / D-, U- = l t, p' = p t - lam
  dd p = dd_sub(dd_from(dl[m - 1].x), lam);
  dd g = dd_add(dd_add(s, p), lam);
  double best = fabs(g.hi);
  int r = m - 1;
  dd gamma = g;
  for (int i = m - 2; i >= 0; --i) {
    const double D = dl[i].x, l = ul[i].x;
    const dd lld = dd_mul_d(dd_mul_d(dd_from(l), l), D);
    dd dm = dd_add(lld, p);
    if (fabs(dm.hi) < pivmin) dm = dd_from(-pivmin);
    const dd t = dd_div(dd_from(D), dm);
    const dd um = dd_mul_d(t, l);
    p = dd_sub(dd_mul(p, t), lam);
    g = dd_add(dd_add(dd{Bh[i * nthr], Bl[i * nthr]}, p), lam);
    if (fabs(g.hi) <= best) {
      best = fabs(g.hi);
      r = i;
      gamma = g;
    }
    Bh[i * nthr] = um.hi;
    Bl[i * nthr] = um.lo;
  }
  // solve with z_r = 1
  dd n2 = dd_from(1.0), z = dd_from(1.0);
  if (zc) zc[r] = 1.0;
  for (int i = r - 1; i >= 0; --i) {
    z = dd_neg(dd_mul(dd{Ah[i * nthr], Al[i * nthr]}, z));
    n2 = dd_add(n2, dd_mul(z, z));
    if (zc) zc[i] = z.hi + z.lo;
  }
  z = dd_from(1.0);
  for (int i = r; i < m - 1; ++i) {
    z = dd_neg(dd_mul(dd{Bh[i * nthr], Bl[i * nthr]}, z));
    n2 = dd_add(n2, dd_mul(z, z));
    if (zc) zc[i + 1] = z.hi + z.lo;
  }
  r_out = r;
  gamma_out = gamma;
  norm2_out = n2;
}

// Eigenvectors in double-double: per singleton, a twisted factorization at
// the bisected value (FP64, full accuracy), the Rayleigh-quotient correction
// lam += gamma_r / ||z||^2 (Eq. errorangle's residual |gamma_r| / ||z||, in
// double-double), then the twisted factorization and solve at the corrected
// value; the vector is rounded to FP64 and normalised by k_normalize.  One
// thread per vector, chunks of 32 slots from the scheduler.
__global__ void __launch_bounds__(128) k_vectors_dd(Dev v) {
  const int lane = threadIdx.x & 31;
  const int64_t tid = gtid(), nthr = gstride();
  const int64_t nslots = v.ctl->nslots;
  const int64_t plane = v.vscr_threads * v.vscr_rows;
  double* Ah = v.vscr + tid;
  double* Al = Ah + plane;
  double* Bh = Al + plane;
  double* Bl = Bh + plane;
  unsigned long long iters = 0;
  const long long nchunks = (nslots + 31) / 32;
  const long long rank = sched_rank(v);
  bool first = true;
  for (;;) {
    const long long chunk = sched_next(v, nchunks, nthr / 32, rank, first);
    if (chunk < 0) break;
    const int64_t w = chunk * 32 + lane;
    if (w >= nslots) continue;
    const int st = v.state[w];
    if ((st != SLOT_SINGLETON && st != SLOT_FALLBACK && st != SLOT_TRIVIAL) || v.spos[w] < 0) continue;
    const int pos = v.spos[w];
    const Node nd = v.node[v.snode[w]];
    const Block bk = v.blk[nd.block];
    const Problem pr = v.prob[bk.prob];
    const int m = bk.m;
    double* zc = v.Z ? v.Z + pr.zout + (int64_t)pos * pr.ldz + (bk.row0 - pr.row0) : nullptr;
    if (st == SLOT_TRIVIAL || m == 1) {
      v.W[pr.wout + pos] = nd.sigma_abs / pr.scale;
      if (zc) zc[0] = 1.0;
      v.znrm2[w] = 1.0;
      continue;
    }
    const double2* rdl = v.rep_dl + nd.rep;
    const double2* rul = v.rep_ul + nd.rep;
    dd lam = dd_from(0.5 * (v.lo[w] + v.hi[w]));
    int r;
    dd gamma, n2;
    twisted_dd(rdl, rul, m, lam, nd.pivmin, Ah, Al, Bh, Bl, nthr, nullptr, r, gamma, n2);
    const dd corr = dd_div(gamma, n2);
    // the correction stays inside the bisection bracket (else keep the value)
    const dd lam2 = dd_add(lam, corr);
    if (lam2.hi >= v.lo[w] && lam2.hi <= v.hi[w]) lam = lam2;
    twisted_dd(rdl, rul, m, lam, nd.pivmin, Ah, Al, Bh, Bl, nthr, zc, r, gamma, n2);
    iters += 2;
    if (!isfinite(n2.hi)) set_status(v.ctl, MRRR_ERR_NOCONV);
    const dd wabs = dd_add(dd_from(nd.sigma_abs), lam);
    v.W[pr.wout + pos] = (wabs.hi + wabs.lo) / pr.scale;
    v.wval[w] = lam.hi;
    v.znrm2[w] = n2.hi + n2.lo;
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

// One warp per slot: link[w] = largest k <= kOrthNeighbors with
// |z_w^T z_{w+k}| above the threshold (0 if none).  The warp reads its
// column once and the kOrthNeighbors following ones side by side (one
// accumulator per neighbour, lanes over rows); the per-slot index array sj
// (no longer needed once the eigenvalues are final) holds the links.
__global__ void __launch_bounds__(256) k_orth_links(Dev v) {
  const int lane = threadIdx.x & 31;
  const int64_t nslots = v.ctl->nslots;
  if (gtid() == 0) v.ctl->orth_runs = 0;
  for (int64_t w = gtid() >> 5; w < nslots; w += gstride() >> 5) {
    int link = 0;
    if (slot_has_column(v, w)) {
      const Block bk = v.blk[v.node[v.snode[w]].block];
      const Problem q = v.prob[bk.prob];
      const int64_t last = bk.slot0 + (bk.je - bk.js);
      const double thr = kOrthFixTol * bk.m * kEps;
      const double* zw = slot_column(v, w, bk, q);
      const double* zk[kOrthNeighbors];
#pragma unroll
      for (int k = 0; k < kOrthNeighbors; ++k) {
        const int64_t t = w + 1 + k;
        zk[k] = (t <= last && slot_has_column(v, t)) ? slot_column(v, t, bk, q) : nullptr;
      }
      double acc[kOrthNeighbors];
#pragma unroll
      for (int k = 0; k < kOrthNeighbors; ++k) acc[k] = 0.0;
      for (int i = lane; i < bk.m; i += 32) {
        const double a = zw[i];
#pragma unroll
        for (int k = 0; k < kOrthNeighbors; ++k)
          if (zk[k]) acc[k] = fma(a, zk[k][i], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < kOrthNeighbors; ++k) {
        double s = acc[k];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (zk[k] && fabs(s) > thr) link = k + 1;
      }
    }
    if (lane == 0) v.sj[w] = link;
  }
}

// One warp per block: the runs of linked slots (a slot and every slot its
// link reaches, closed under reaching), appended to the run list as
// (first slot, last slot) pairs in the engine's work list, free by now.
__global__ void k_orth_runs(Dev v) {
  const int lane = threadIdx.x & 31;
  const int nblocks = v.ctl->nblocks;
  for (int64_t b = gtid() >> 5; b < nblocks; b += gstride() >> 5) {
    const Block bk = v.blk[b];
    if (bk.m < 2 || bk.je < bk.js) continue;
    const int64_t s0 = bk.slot0, s1 = bk.slot0 + (bk.je - bk.js);
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
      if (lane == 0) {
        const long long r = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&v.ctl->orth_runs), 1ULL);
        if (2 * r + 1 < v.max_list) {
          v.ilist[2 * r] = start;
          v.ilist[2 * r + 1] = reach;
        }
        diag(v.ctl, DIAG_ORTH_FIX);
      }
      w = reach + 1;
    }
  }
}

constexpr int kFixThreads = 256;

// CTA-wide sum (all threads get it); red holds kFixThreads / 32 doubles.
__device__ __forceinline__ double cta_sum(double x, double* red) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < kFixThreads / 32; ++k) s += red[k];
  return s;
}

// One CTA per run: each column after the run's first is re-orthogonalised
// against the earlier ones, in eigenvalue order (modified Gram-Schmidt,
// twice), then normalised.
__global__ void __launch_bounds__(kFixThreads) k_orth_fix(Dev v) {
  __shared__ double red[kFixThreads / 32];
  const long long nruns = min(v.ctl->orth_runs, (long long)(v.max_list / 2));
  for (long long r = blockIdx.x; r < nruns; r += gridDim.x) {
    const int64_t start = v.ilist[2 * r], reach = v.ilist[2 * r + 1];
    const Block bk = v.blk[v.node[v.snode[start]].block];
    const Problem q = v.prob[bk.prob];
    const int m = bk.m;
    for (int64_t c = start + 1; c <= reach; ++c) {
      if (!slot_has_column(v, c)) continue;
      double* zc = const_cast<double*>(slot_column(v, c, bk, q));
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t p = start; p < c; ++p) {
          if (!slot_has_column(v, p)) continue;
          const double* zp = slot_column(v, p, bk, q);
          double part = 0.0;
          for (int i = threadIdx.x; i < m; i += kFixThreads) part = fma(zc[i], zp[i], part);
          const double dot = cta_sum(part, red);
          for (int i = threadIdx.x; i < m; i += kFixThreads) zc[i] = fma(-dot, zp[i], zc[i]);
        }
      }
      double part = 0.0;
      for (int i = threadIdx.x; i < m; i += kFixThreads) part = fma(zc[i], zc[i], part);
      const double n2 = cta_sum(part, red);
      const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
      for (int i = threadIdx.x; i < m; i += kFixThreads) zc[i] *= sc;
      __syncthreads();
    }
  }
}

// W ascending: in split problems columns were placed by the rank of interval
// midpoints, and near-ties across blocks may leave W slightly out of order;
// in any problem, eigenvalues equal to the last bit that were finished on
// different nodes (sigma_abs + local value, each rounded) can come out one or
// two ulps out of order.  One CTA per problem: a sweep over all of W finds
// whether any neighbours are out of order (the usual answer is no).  If so,
// and the running maximum of W exceeds no entry by more than kTieUlps ulps,
// the entries are rounding ties: each takes the running maximum (it moves by
// at most those few ulps, its column stays).  Otherwise odd-even
// transposition passes with every thread on its own pairs swap the values
// and queue the swapped pairs, whose columns of Z the warps then swap; the
// passes stop after two without a swap.
constexpr int kSwapQueue = 512;
constexpr double kTieUlps = 16.0;

__device__ __forceinline__ bool is_tie(double run, double w) {
  const double def = run - w;
  return !isnan(w) && (def <= kTieUlps * kEps * fmax(fabs(run), fabs(w)) || def <= 1e-300);
}

__global__ void __launch_bounds__(kFixThreads) k_fix_order(Dev v) {
  __shared__ int nq;
  __shared__ int64_t queue[kSwapQueue];
  __shared__ double cmax[kFixThreads];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int nw = kFixThreads / 32;
  for (int64_t p = blockIdx.x; p < v.batch; p += gridDim.x) {
    const Problem q = v.prob[p];
    if (q.k < 2) continue;
    double* W = v.W + q.wout;
    int bad = 0;
    for (int64_t i = threadIdx.x; i + 1 < q.k; i += kFixThreads) bad |= W[i] > W[i + 1];
    if (!__syncthreads_or(bad)) continue;
    // rounding ties only?  Thread t takes a contiguous chunk; the running
    // maximum enters it as the maximum of the chunks before.
    const int64_t per = (q.k + kFixThreads - 1) / kFixThreads;
    const int64_t a = min((int64_t)threadIdx.x * per, (int64_t)q.k), b = min(a + per, (int64_t)q.k);
    double m = -INFINITY;
    for (int64_t i = a; i < b; ++i) m = fmax(m, W[i]);
    cmax[threadIdx.x] = m;
    __syncthreads();
    double run = -INFINITY;
    for (int t = 0; t < (int)threadIdx.x; ++t) run = fmax(run, cmax[t]);
    const double run0 = run;
    int ties = 1;
    for (int64_t i = a; i < b; ++i) {
      run = fmax(run, W[i]);
      ties &= is_tie(run, W[i]);
    }
    if (__syncthreads_and(ties)) {
      run = run0;
      for (int64_t i = a; i < b; ++i) {
        run = fmax(run, W[i]);
        W[i] = run;
      }
      __syncthreads();
      continue;
    }
    int quiet = 0;
    for (int pass = 0; pass < 2 * q.k + 2 && quiet < 2; ++pass) {
      int swapped = 0;
      for (int64_t base = (pass & 1); base + 1 < q.k; base += 2 * (int64_t)kSwapQueue) {
        // a round of up to kSwapQueue pairs: swap values, queue the pairs
        if (threadIdx.x == 0) nq = 0;
        __syncthreads();
        for (int u = 0; u < kSwapQueue / kFixThreads; ++u) {
          const int64_t i = base + 2 * ((int64_t)u * kFixThreads + threadIdx.x);
          if (i + 1 < q.k) {
            const double a = W[i], b = W[i + 1];
            if (a > b) {
              W[i] = b;
              W[i + 1] = a;
              queue[atomicAdd(&nq, 1)] = i;
            }
          }
        }
        __syncthreads();
        const int cnt = nq;
        swapped |= cnt > 0;
        if (v.Z) {
          for (int t = wid; t < cnt; t += nw) {
            double* ca = v.Z + q.zout + queue[t] * q.ldz;
            double* cb = ca + q.ldz;
            for (int64_t r = lane; r < q.n; r += 32) {
              const double x = ca[r];
              ca[r] = cb[r];
              cb[r] = x;
            }
          }
        }
        __syncthreads();
      }
      quiet = swapped ? 0 : quiet + 1;
    }
  }
}

}  // namespace

void launch_vectors(const Dev& v, const Grid& g, cudaStream_t s) {
  k_sched_reset<<<1, kSchedSlots, 0, s>>>(v);
  count_launch();
  if (v.vec_dd)
    k_vectors_dd<<<g.vec_blocks, 128, 0, s>>>(v);
  else if (v.rq_steps > 0)
    k_vectors<true><<<g.nsm * kVecCtasPerSm, kVecWarps * 32, 0, s>>>(v);
  else
    k_vectors<false><<<g.nsm * kVecCtasPerSm, kVecWarps * 32, 0, s>>>(v);
  count_launch();
  if (v.Z) {
    k_normalize<<<g.nsm * 16, 256, 0, s>>>(v);
    count_launch();
    if (!v.no_orth_fix) {
      k_orth_links<<<g.nsm * 16, 256, 0, s>>>(v);
      count_launch();
      k_orth_runs<<<g.nsm, 128, 0, s>>>(v);
      count_launch();
      k_orth_fix<<<g.nsm * 2, kFixThreads, 0, s>>>(v);
      count_launch();
    }
  }
  k_fix_order<<<g.nsm, kFixThreads, 0, s>>>(v);
  count_launch();
}

}  // namespace mrrr
