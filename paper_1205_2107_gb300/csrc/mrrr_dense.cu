// mrrr_dense.cu -- the dense stages around the tridiagonal eigensolver
// (paper Sec. 1.2): stage 3, reduction of a symmetric A to tridiagonal form
// T = Q^T A Q by Householder reflectors, and stage 5, the backtransformation
// Y = Q Z of the tridiagonal eigenvectors (the generalized stages 1, 2 and 6
// are in mrrr_dense_gen.cu).  All FP64.
//
// Reduction (blocked, lower triangle): panels of kNb columns.  For column j
// of a panel, with V and W the panel's reflectors and update vectors so far:
//   a = A(j:n, j) - V W(j,:)^T - W V(j,:)^T            (column brought up to date)
//   (v, tau, beta) with (I - tau v v^T) a(j+1:n) = beta e_1, v_1 = 1
//   y = A22 v - V (W^T v) - W (V^T v)                 (A22 = A(j+1:n, j+1:n), lower)
//   w = tau y - (tau^2 / 2)(y^T v) v
// and after the panel the trailing lower triangle takes the rank-2k update
// A22 -= V W^T + W V^T on the FP64 tensor cores.  The symmetric product
// A22 v reads each lower 64x64 tile once and applies it and its transpose;
// partial sums go to a workspace and are reduced in a fixed order, so the
// result is deterministic.  On this part the FP64 units bound both halves:
// the symmetric product does 2 flops per 8 bytes, below the machine balance.
//
// Backtransformation (blocked): the panels' reflectors in compact WY form,
// H_j0 ... H_j0+k-1 = I - V T V^T, applied to Y from the last panel to the
// first: Y(j0+1:n, :) -= V (T (V^T Y(j0+1:n, :))), three GEMMs per panel.
#include <algorithm>
#include <cmath>

#include "mrrr_dense.cuh"

namespace mrrr {
namespace dense {

// ---------------------------------------------------------------------------
// FP64 tensor-core GEMM: C = alpha op(A) op(B) + beta C, column-major C.
// mma.sync m8n8k4 f64 fragments (PTX ISA): A one element (row lane/4,
// column lane%4), B one element (row lane%4, column lane/4), C/D two
// elements (row lane/4, columns 2(lane%4) + {0, 1}).
constexpr int kTM = 64, kTN = 64, kTK = 32, kKS = kTK + 4;
constexpr int kGemmThreads = 128;  // 4 warps, 2 x 2, each 32 x 32

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// As(rr, kk) = A(m0 + rr, k0 + kk), zero outside; stored K-contiguous.
__device__ __forceinline__ void load_a(double* As, const GemmArgs& g, int m0, int k0, int kend) {
  if (g.a_cs == 1) {  // K contiguous in memory
    for (int idx = threadIdx.x; idx < kTM * kTK; idx += blockDim.x) {
      const int rr = idx / kTK, kk = idx % kTK, i = m0 + rr, p = k0 + kk;
      As[rr * kKS + kk] = (i < g.m && p < kend) ? g.A[(int64_t)i * g.a_rs + p] : 0.0;
    }
  } else {  // rows contiguous (or general strides)
    for (int idx = threadIdx.x; idx < kTM * kTK; idx += blockDim.x) {
      const int kk = idx / kTM, rr = idx % kTM, i = m0 + rr, p = k0 + kk;
      As[rr * kKS + kk] = (i < g.m && p < kend) ? g.A[(int64_t)i * g.a_rs + (int64_t)p * g.a_cs] : 0.0;
    }
  }
}

// Bs(cc, kk) = B(k0 + kk, n0 + cc), zero outside; stored K-contiguous.
__device__ __forceinline__ void load_b(double* Bs, const GemmArgs& g, int n0, int k0, int kend) {
  if (g.b_rs == 1) {  // K contiguous in memory
    for (int idx = threadIdx.x; idx < kTN * kTK; idx += blockDim.x) {
      const int cc = idx / kTK, kk = idx % kTK, j = n0 + cc, p = k0 + kk;
      Bs[cc * kKS + kk] = (j < g.n && p < kend) ? g.B[p + (int64_t)j * g.b_cs] : 0.0;
    }
  } else {
    for (int idx = threadIdx.x; idx < kTN * kTK; idx += blockDim.x) {
      const int kk = idx / kTN, cc = idx % kTN, j = n0 + cc, p = k0 + kk;
      Bs[cc * kKS + kk] = (j < g.n && p < kend) ? g.B[(int64_t)p * g.b_rs + (int64_t)j * g.b_cs] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g) {
  __shared__ double As[kTM * kKS];
  __shared__ double Bs[kTN * kKS];
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  if (g.lower && n0 > m0 + kTM - 1) return;  // tile entirely above the diagonal
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int r = lane >> 2, c = lane & 3;
  double acc[4][4][2] = {};
  int kbeg = 0, kend = g.k;
  double* C = g.C;
  if (g.kchunk > 0) {
    kbeg = blockIdx.z * g.kchunk;
    kend = min(g.k, kbeg + g.kchunk);
    C += (int64_t)blockIdx.z * g.cstride;
  }
  for (int k0 = kbeg; k0 < kend; k0 += kTK) {
    load_a(As, g, m0, k0, kend);
    load_b(Bs, g, n0, k0, kend);
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < kTK; kq += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = As[(wm + 8 * i + r) * kKS + kq + c];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = Bs[(wn + 8 * j + r) * kKS + kq + c];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
    }
    __syncthreads();
  }
  const int c2 = c * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm + 8 * i + r, col = n0 + wn + 8 * j + c2 + h;
        if (row < g.m && col < g.n && (!g.lower || row >= col)) {
          double* p = C + row + (int64_t)col * g.ldc;
          *p = g.beta == 0.0 ? g.alpha * acc[i][j][h] : fma(g.alpha, acc[i][j][h], g.beta * *p);
        }
      }
}

void gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.m <= 0 || g.n <= 0) return;
  GemmArgs h = g;
  h.kchunk = 0;
  dim3 grid((g.m + kTM - 1) / kTM, (g.n + kTN - 1) / kTN);
  k_gemm<<<grid, kGemmThreads, 0, s>>>(h);
  count_launch();
}

namespace {
// C(i, j) = alpha sum_z P_z(i, j) + beta C(i, j), z in order.
__global__ void k_splitk_reduce(const double* P, int nsplit, int64_t pstride, int m, int n, double alpha,
                                double beta, double* C, int64_t ldc) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / m), i = (int)(idx % m);
    double sacc = 0.0;
    for (int z = 0; z < nsplit; ++z) sacc += P[z * pstride + i + (int64_t)j * m];
    double* c = C + i + (int64_t)j * ldc;
    *c = beta == 0.0 ? alpha * sacc : fma(alpha, sacc, beta * *c);
  }
}
}  // namespace

void gemm_splitk(GemmArgs g, double* partials, int max_split, int nsm, cudaStream_t s) {
  if (g.m <= 0 || g.n <= 0) return;
  const int64_t tiles = (int64_t)((g.m + kTM - 1) / kTM) * ((g.n + kTN - 1) / kTN);
  // enough CTAs for four per SM, K chunks of at least 256
  int64_t split = std::min<int64_t>({(int64_t)max_split, (4LL * nsm + tiles - 1) / tiles, (g.k + 255) / 256});
  if (split <= 1 || g.lower) {
    gemm(g, s);
    return;
  }
  const int kchunk = (int)(((g.k + split - 1) / split + kTK - 1) / kTK * kTK);
  split = (g.k + kchunk - 1) / kchunk;
  GemmArgs h = g;
  h.C = partials;
  h.ldc = g.m;
  h.alpha = 1.0;
  h.beta = 0.0;
  h.kchunk = kchunk;
  h.cstride = (int64_t)g.m * g.n;
  dim3 grid((g.m + kTM - 1) / kTM, (g.n + kTN - 1) / kTN, (unsigned)split);
  k_gemm<<<grid, kGemmThreads, 0, s>>>(h);
  const int64_t tot = (int64_t)g.m * g.n;
  k_splitk_reduce<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(8192, (tot + 255) / 256)), 256, 0, s>>>(
      partials, (int)split, h.cstride, g.m, g.n, g.alpha, g.beta, g.C, g.ldc);
  count_launch(2);
}

// Column-major operands: op(X) = X (ld) or X^T.
GemmArgs gemm_args(int m, int n, int k, double alpha, const double* A, int64_t lda, bool ta, const double* B,
                   int64_t ldb, bool tb, double beta, double* C, int64_t ldc, bool lower) {
  GemmArgs g{};
  g.m = m;
  g.n = n;
  g.k = k;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  if (!ta) {  // A(i, p) = A[i + p lda]
    g.a_rs = 1;
    g.a_cs = lda;
  } else {  // A(i, p) = A[p + i lda]
    g.a_rs = lda;
    g.a_cs = 1;
  }
  g.B = B;
  if (!tb) {  // B(p, j) = B[p + j ldb]
    g.b_rs = 1;
    g.b_cs = ldb;
  } else {  // B(p, j) = B[j + p ldb]
    g.b_rs = ldb;
    g.b_cs = 1;
  }
  g.C = C;
  g.ldc = ldc;
  g.lower = lower ? 1 : 0;
  return g;
}


// ---------------------------------------------------------------------------
// Reduction to tridiagonal form (stage 3).

namespace {

__device__ __forceinline__ double block_sum(double x, double* red) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0 (and warp 0)
}

__host__ __device__ __forceinline__ int row_ctas(int rows) { return (rows + kRowCta - 1) / kRowCta; }

// Column j (the panel's i-th) brought up to date with the panel's earlier
// reflectors, rows j .. n-1; per-CTA sums of squares of rows j+2 .. n-1.
__global__ void __launch_bounds__(kRowCta) k_trd_col(TrdArgs t, int j, int i) {
  __shared__ double red[kRowCta / 32];
  const int r = j + blockIdx.x * kRowCta + threadIdx.x;
  const int64_t n = t.n;
  double sq = 0.0;
  if (r < t.n) {
    double a = t.A[r + (int64_t)j * t.lda];
    for (int c = 0; c < i; ++c)
      a -= t.V[r + c * n] * t.W[j + c * n] + t.W[r + c * n] * t.V[j + c * n];
    t.A[r + (int64_t)j * t.lda] = a;
    if (r >= j + 2) sq = a * a;
  }
  const double tot = block_sum(sq, red);
  if (threadIdx.x == 0) t.colpart[blockIdx.x] = tot;
}

// The reflector of column j: beta, tau, v (v_{j+1} = 1) from the column and
// the sums of squares; v into V(:, i) and below the subdiagonal of A, beta
// onto the subdiagonal; per-CTA partial products W^T v and V^T v with the
// panel's earlier columns.
__global__ void __launch_bounds__(kRowCta) k_trd_vec(TrdArgs t, int j, int i) {
  __shared__ double red[kRowCta / 32];
  __shared__ double s_sc[3];
  const int64_t n = t.n;
  if (threadIdx.x < 32) {
    const int nb1 = row_ctas(t.n - j);
    double sg = 0.0;
    for (int b = threadIdx.x; b < nb1; b += 32) sg += t.colpart[b];
    for (int o = 16; o; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
    if (threadIdx.x == 0) {
      const double alpha = t.A[(j + 1) + (int64_t)j * t.lda];
      double beta = alpha, tau = 0.0, scale = 0.0;
      if (sg > 0.0) {
        const double nrm = sqrt(alpha * alpha + sg);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      s_sc[0] = beta;
      s_sc[1] = tau;
      s_sc[2] = scale;
      if (blockIdx.x == 0) {
        t.d[j] = t.A[j + (int64_t)j * t.lda];
        t.e[j] = beta;
        t.tau[j] = tau;
        if (!isfinite(beta) || !isfinite(tau)) atomicCAS(&t.ctl->status, 0, (int)MRRR_ERR_NONFINITE);
      }
    }
  }
  __syncthreads();
  const int r = j + 1 + blockIdx.x * kRowCta + threadIdx.x;
  double v = 0.0;
  if (r < t.n) {
    v = r == j + 1 ? 1.0 : t.A[r + (int64_t)j * t.lda] * s_sc[2];
    t.V[r + i * n] = v;
    t.A[r + (int64_t)j * t.lda] = r == j + 1 ? s_sc[0] : v;
  }
  for (int c = 0; c < i; ++c) {
    const double x = r < t.n ? t.W[r + c * n] * v : 0.0;
    const double z = r < t.n ? t.V[r + c * n] * v : 0.0;
    const double sx = block_sum(x, red);
    if (threadIdx.x == 0) t.dotpart[blockIdx.x * 2 * kNb + c] = sx;
    const double sz = block_sum(z, red);
    if (threadIdx.x == 0) t.dotpart[blockIdx.x * 2 * kNb + kNb + c] = sz;
  }
}

constexpr int kSymvTile = 64;

// y = A22 v (A22 = A(j+1:n, j+1:n), lower triangle stored), tile by tile:
// tile (I, J), J <= I, adds tile v_J to rows of block I and tile^T v_I to
// rows of block J, into P(I, J, :) and P(J, I, :); a diagonal tile applies
// its lower triangle both ways.  All 256 threads work: thread (q, t) sums a
// quarter (16 entries) of row t and of column t, then the quarters are
// added in a fixed order.  Four CTAs per SM.
__global__ void __launch_bounds__(256, 4) k_trd_symv(TrdArgs t, int j, int i) {
  __shared__ double tile[kSymvTile][kSymvTile + 1];
  __shared__ double vi[kSymvTile], vj[kSymvTile];
  __shared__ double rpart[4][kSymvTile], cpart[4][kSymvTile];
  const int m = t.n - j - 1;
  const int T = (m + kSymvTile - 1) / kSymvTile;
  const int64_t b = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((int64_t)(I + 1) * (I + 2) / 2 <= b) ++I;
  while ((int64_t)I * (I + 1) / 2 > b) --I;
  const int J = (int)(b - (int64_t)I * (I + 1) / 2);
  const int r0 = j + 1 + I * kSymvTile, c0 = j + 1 + J * kSymvTile;
  const int64_t n = t.n;
  const bool diag = I == J;
  for (int idx = threadIdx.x; idx < kSymvTile * kSymvTile; idx += blockDim.x) {
    const int cc = idx / kSymvTile, rr = idx % kSymvTile;  // rows contiguous in memory
    const int row = r0 + rr, col = c0 + cc;
    double x = 0.0;
    if (row < t.n && col < t.n && (!diag || rr >= cc)) x = t.A[row + (int64_t)col * t.lda];
    tile[rr][cc] = x;
  }
  if (threadIdx.x < kSymvTile) {
    const int row = r0 + threadIdx.x, col = c0 + threadIdx.x;
    vi[threadIdx.x] = row < t.n ? t.V[row + i * n] : 0.0;
    vj[threadIdx.x] = col < t.n ? t.V[col + i * n] : 0.0;
  }
  __syncthreads();
  const int tt = threadIdx.x & (kSymvTile - 1), q = threadIdx.x >> 6;
  const int k0 = q * (kSymvTile / 4);
  double rs = 0.0, cs = 0.0;
#pragma unroll 4
  for (int k = k0; k < k0 + kSymvTile / 4; ++k) {
    rs = fma(tile[tt][k], vj[k], rs);     // row tt of the tile
    cs = fma(tile[k][tt], diag ? vj[k] : vi[k], cs);  // column tt (on the diagonal: row tt of the upper half)
  }
  rpart[q][tt] = rs;
  cpart[q][tt] = cs;
  __syncthreads();
  double* P = t.P;
  if (threadIdx.x < kSymvTile) {
    const double r = ((rpart[0][tt] + rpart[1][tt]) + rpart[2][tt]) + rpart[3][tt];
    const double c = ((cpart[0][tt] + cpart[1][tt]) + cpart[2][tt]) + cpart[3][tt];
    if (diag) {
      P[((int64_t)I * T + J) * kSymvTile + tt] = r + c - tile[tt][tt] * vj[tt];
    } else {
      P[((int64_t)I * T + J) * kSymvTile + tt] = r;
      P[((int64_t)J * T + I) * kSymvTile + tt] = c;
    }
  }
}

// w = tau (A22 v - V (W^T v) - W (V^T v)); per-CTA partial w^T v.
__global__ void __launch_bounds__(kRowCta) k_trd_w(TrdArgs t, int j, int i) {
  __shared__ double red[kRowCta / 32];
  __shared__ double xz[2 * kNb];
  const int64_t n = t.n;
  const int m = t.n - j - 1;
  const int T = (m + kSymvTile - 1) / kSymvTile;
  const int nb3 = row_ctas(m);
  if (threadIdx.x < 2 * i) {
    const int c = threadIdx.x < i ? threadIdx.x : kNb + threadIdx.x - i;
    double sacc = 0.0;
    for (int b = 0; b < nb3; ++b) sacc += t.dotpart[b * 2 * kNb + c];
    xz[c] = sacc;
  }
  __syncthreads();
  const int q = blockIdx.x * kRowCta + threadIdx.x;
  const int r = j + 1 + q;
  const double tau = t.tau[j];
  double wv = 0.0;
  if (q < m) {
    const int I = q / kSymvTile, rr = q % kSymvTile;
    double y = 0.0;
    for (int J = 0; J < T; ++J) y += t.P[((int64_t)I * T + J) * kSymvTile + rr];
    for (int c = 0; c < i; ++c) y -= t.V[r + c * n] * xz[c] + t.W[r + c * n] * xz[kNb + c];
    const double w = tau * y;
    t.W[r + i * n] = w;
    wv = w * t.V[r + i * n];
  }
  const double tot = block_sum(wv, red);
  if (threadIdx.x == 0) t.wvpart[blockIdx.x] = tot;
}

// w -= (tau / 2) (w^T v) v.
__global__ void __launch_bounds__(kRowCta) k_trd_wfix(TrdArgs t, int j, int i) {
  __shared__ double s_c;
  const int64_t n = t.n;
  const int m = t.n - j - 1;
  if (threadIdx.x < 32) {
    const int nb = row_ctas(m);
    double sacc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) sacc += t.wvpart[b];
    for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
    if (threadIdx.x == 0) s_c = 0.5 * t.tau[j] * sacc;
  }
  __syncthreads();
  const int r = j + 1 + blockIdx.x * kRowCta + threadIdx.x;
  if (r < t.n) t.W[r + i * n] -= s_c * t.V[r + i * n];
}

// Columns c0 .. c1-1 of an n-row column-major panel to zero.
__global__ void k_zero_cols(double* X, int n, int c0, int c1) {
  const int64_t tot = (int64_t)n * (c1 - c0);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)c0 * n + idx] = 0.0;
}

__global__ void k_copy_block(const double* src, double* dst, int64_t count) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[idx] = src[idx];
}

// The last diagonal and subdiagonal entries (untouched by any reflector).
__global__ void k_trd_tail(TrdArgs t) {
  const int n = t.n;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (n == 1) {
    t.d[0] = t.A[0];
    return;
  }
  t.d[n - 2] = t.A[(n - 2) + (int64_t)(n - 2) * t.lda];
  t.d[n - 1] = t.A[(n - 1) + (int64_t)(n - 1) * t.lda];
  t.e[n - 2] = t.A[(n - 1) + (int64_t)(n - 2) * t.lda];
  for (int k = 0; k < n; ++k)
    if (!isfinite(t.d[k])) atomicCAS(&t.ctl->status, 0, (int)MRRR_ERR_NONFINITE);
}

}  // namespace

size_t trd_scratch_doubles(int n) {
  const int64_t T = (std::max(n - 1, 1) + kSymvTile - 1) / kSymvTile;
  const int64_t rc = (std::max(n, 1) + kRowCta - 1) / kRowCta;
  return (size_t)(3 * (int64_t)n * kNb + T * T * kSymvTile + rc * (2 + 2 * kNb));
}

TrdArgs trd_args(int n, double* A, int64_t lda, double* d, double* e, double* tau, double* scratch, DenseCtl* ctl) {
  TrdArgs t{};
  t.n = n;
  t.A = A;
  t.lda = lda;
  t.d = d;
  t.e = e;
  t.tau = tau;
  const int64_t T = (std::max(n - 1, 1) + kSymvTile - 1) / kSymvTile;
  const int64_t rc = (std::max(n, 1) + kRowCta - 1) / kRowCta;
  double* p = scratch;
  t.V = p;
  p += (int64_t)n * kNb;
  t.W = p;
  p += 2 * (int64_t)n * kNb;  // W, then the copy of V used by the trailing update
  t.P = p;
  p += T * T * kSymvTile;
  t.colpart = p;
  p += rc;
  t.wvpart = p;
  p += rc;
  t.dotpart = p;
  t.ctl = ctl;
  return t;
}

void launch_trd(const TrdArgs& t, cudaStream_t s) {
  const int n = t.n;
  for (int j0 = 0; j0 < n - 2; j0 += kNb) {
    const int ncols = std::min(kNb, n - 2 - j0);
    for (int i = 0; i < ncols; ++i) {
      const int j = j0 + i;
      const int m = n - j - 1;
      const int T = (m + kSymvTile - 1) / kSymvTile;
      k_trd_col<<<row_ctas(n - j), kRowCta, 0, s>>>(t, j, i);
      k_trd_vec<<<row_ctas(m), kRowCta, 0, s>>>(t, j, i);
      k_trd_symv<<<(unsigned)((int64_t)T * (T + 1) / 2), 256, 0, s>>>(t, j, i);
      k_trd_w<<<row_ctas(m), kRowCta, 0, s>>>(t, j, i);
      k_trd_wfix<<<row_ctas(m), kRowCta, 0, s>>>(t, j, i);
      count_launch(5);
    }
    // trailing update of the lower triangle, A22 -= V W^T + W V^T, as one
    // GEMM of depth 2 kNb: V, W and a copy of V lie side by side (n x 3 kNb),
    // so [V W] and [W V] are both column ranges of it
    const int j1 = j0 + ncols, m2 = n - j1;
    double* C = t.A + j1 + (int64_t)j1 * t.lda;
    if (ncols < kNb) {  // a partial last panel: the unused columns must not contribute
      k_zero_cols<<<(unsigned)std::max(1, (n * (kNb - ncols) + 255) / 256), 256, 0, s>>>(t.V, n, ncols, kNb);
      k_zero_cols<<<(unsigned)std::max(1, (n * (kNb - ncols) + 255) / 256), 256, 0, s>>>(t.W, n, ncols, kNb);
      count_launch(2);
    }
    k_copy_block<<<(unsigned)std::max(1, std::min(8192, (n * kNb + 255) / 256)), 256, 0, s>>>(t.V, t.W + (int64_t)n * kNb,
                                                                                           (int64_t)n * kNb);
    count_launch();
    gemm(gemm_args(m2, m2, 2 * kNb, -1.0, t.V + j1, n, false, t.W + j1, n, true, 1.0, C, t.lda, true), s);
  }
  if (n >= 1) {
    k_trd_tail<<<1, 32, 0, s>>>(t);
    count_launch();
  }
}


// ---------------------------------------------------------------------------
// Backtransformation Y = Q Y (stage 5).

namespace {

// The panel's reflectors as a unit lower trapezoidal Vp (rows j0+1 .. n-1,
// column i = reflector j0+i: zero above row i, one at row i, then the
// stored v below the subdiagonal of A).
__global__ void k_orm_vp(const double* __restrict__ A, int64_t lda, int n, int j0, int nbp, double* Vp) {
  const int rows = n - j0 - 1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)rows * nbp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / rows), r = (int)(idx % rows);
    double x = 0.0;
    if (r == i) x = 1.0;
    else if (r > i) x = A[(j0 + 1 + r) + (int64_t)(j0 + i) * lda];
    Vp[r + (int64_t)i * n] = x;
  }
}
// T of the compact WY form I - Vp T Vp^T = H_j0 ... H_j0+nbp-1 (upper
// triangular, leading dimension kNbBt, in global memory), from
// S = Vp^T Vp: T(i, i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) S(0:i, i),
// column by column.  One CTA of kNbBt threads.
__global__ void __launch_bounds__(kNbBt) k_orm_t(const double* __restrict__ S, const double* __restrict__ tau,
                                                 int nbp, double* T) {
  const int c = threadIdx.x;
  for (int i = 0; i < nbp; ++i) {
    double x = 0.0;
    if (c < i) {
      for (int l = c; l < i; ++l) x = fma(T[c + l * kNbBt], S[l + i * kNbBt], x);
      x = -tau[i] * x;
    }
    __syncthreads();
    if (c < nbp) T[c + i * kNbBt] = c < i ? x : (c == i ? tau[i] : 0.0);
    __syncthreads();
  }
}

}  // namespace

// Split factor the backtransformation's scratch is sized for: enough CTAs
// for four per SM on up to 160 SMs when the k columns alone give too few.
int orm_max_split(int k) {
  const int64_t tiles = 2LL * ((std::max(k, 1) + 63) / 64);
  return (int)std::max<int64_t>(1, std::min<int64_t>(8, (4LL * 160 + tiles - 1) / tiles));
}

size_t orm_scratch_doubles(int n, int k) {
  const int64_t kk = std::max(k, kNbBt);
  return (size_t)((int64_t)n * kNbBt + 2LL * kNbBt * kNbBt + 2LL * kNbBt * kk + (int64_t)orm_max_split(k) * kNbBt * kk);
}

void launch_orm(int n, int k, const double* A, int64_t lda, const double* tau, double* Y, int64_t ldy,
                double* scratch, int nsm, cudaStream_t s) {
  if (n <= 2 || k <= 0) return;
  const int64_t kk = std::max(k, kNbBt);
  double* Vp = scratch;
  double* S = Vp + (int64_t)n * kNbBt;
  double* T = S + kNbBt * kNbBt;
  double* G = T + kNbBt * kNbBt;
  double* G2 = G + kNbBt * kk;
  double* part = G2 + kNbBt * kk;
  const int msplit = orm_max_split(k);
  const int npanels = (n - 2 + kNbBt - 1) / kNbBt;
  for (int p = npanels - 1; p >= 0; --p) {
    const int j0 = p * kNbBt, nbp = std::min(kNbBt, n - 2 - j0), rows = n - j0 - 1;
    double* Ysub = Y + (j0 + 1);
    k_orm_vp<<<std::max(1, std::min(8192, (rows * nbp + 255) / 256)), 256, 0, s>>>(A, lda, n, j0, nbp, Vp);
    gemm_splitk(gemm_args(nbp, nbp, rows, 1.0, Vp, n, true, Vp, n, false, 0.0, S, kNbBt), part, msplit, nsm, s);
    k_orm_t<<<1, kNbBt, 0, s>>>(S, tau + j0, nbp, T);
    gemm_splitk(gemm_args(nbp, k, rows, 1.0, Vp, n, true, Ysub, ldy, false, 0.0, G, kNbBt), part, msplit, nsm, s);
    gemm(gemm_args(nbp, k, nbp, 1.0, T, kNbBt, false, G, kNbBt, false, 0.0, G2, kNbBt), s);
    gemm(gemm_args(rows, k, nbp, -1.0, Vp, n, false, G2, kNbBt, false, 1.0, Ysub, ldy), s);
    count_launch(2);
  }
}

}  // namespace dense
}  // namespace mrrr

// ---------------------------------------------------------------------------
// C ABI of the dense symmetric eigenproblem.

namespace {

using namespace mrrr::dense;

constexpr size_t kDAlign = 256;
size_t dalign(size_t x) { return (x + kDAlign - 1) / kDAlign * kDAlign; }

struct DenseLayout {
  size_t ctl, d, e, tau, scratch, step, total;
  size_t step_bytes;
};

DenseLayout dense_layout(const mrrr_plan* plan, int n, int k) {
  DenseLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = dalign(off + std::max<size_t>(bytes, 1));
    return at;
  };
  L.ctl = take(sizeof(DenseCtl));
  L.d = take(sizeof(double) * (size_t)std::max(n, 1));
  L.e = take(sizeof(double) * (size_t)std::max(n, 1));
  L.tau = take(sizeof(double) * (size_t)std::max(n, 1));
  // the reduction's scratch is free once T is formed: the backtransformation reuses it
  L.scratch = take(sizeof(double) * std::max(trd_scratch_doubles(n), orm_scratch_doubles(n, k)));
  size_t sb = 0;
  if (plan) mrrr_workspace_size(plan, 1, n, k, n, &sb);
  L.step_bytes = sb;
  L.step = take(sb);
  L.total = off;
  return L;
}

}  // namespace

extern "C" {

mrrr_status mrrr_dense_workspace_size(const mrrr_plan* plan, int n, int k, size_t* bytes) {
  if (!plan || !bytes || n < 0 || k < 0 || k > n) return MRRR_ERR_ARG;
  *bytes = dense_layout(plan, n, k).total;
  return MRRR_OK;
}

mrrr_status mrrr_sytrd(mrrr_plan* plan, int n, double* A, int64_t lda, double* d, double* e, double* tau,
                       void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!A || lda < n || !d || (n > 1 && !e) || (n > 2 && !tau)) return MRRR_ERR_ARG;
  const DenseLayout L = dense_layout(plan, n, 0);
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DenseCtl* ctl = reinterpret_cast<DenseCtl*>(w + L.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(DenseCtl), s) != cudaSuccess) return MRRR_ERR_CUDA;
  // e and tau of length 0 are never written: point them at the workspace
  double* ee = n > 1 ? e : reinterpret_cast<double*>(w + L.e);
  double* tt = n > 2 ? tau : reinterpret_cast<double*>(w + L.tau);
  launch_trd(trd_args(n, A, lda, d, ee, tt, reinterpret_cast<double*>(w + L.scratch), ctl), s);
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

mrrr_status mrrr_ormtr(mrrr_plan* plan, int n, int k, const double* A, int64_t lda, const double* tau, double* Y,
                       int64_t ldy, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0 || k < 0) return MRRR_ERR_ARG;
  if (n == 0 || k == 0) return MRRR_OK;
  if (!A || lda < n || (n > 2 && !tau) || !Y || ldy < n) return MRRR_ERR_ARG;
  const DenseLayout L = dense_layout(plan, n, std::min(k, n));
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MRRR_ERR_CUDA;
  launch_orm(n, k, A, lda, tau, Y, ldy, reinterpret_cast<double*>(w + L.scratch), nsm,
             static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

mrrr_status mrrr_dense_eigh(mrrr_plan* plan, int n, double* A, int64_t lda, int il, int iu, double* W, double* Y,
                            int64_t ldy, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!A || lda < n || !W || il < 1 || iu > n || il > iu || (Y && ldy < n)) return MRRR_ERR_ARG;
  const int k = iu - il + 1;
  const DenseLayout L = dense_layout(plan, n, k);
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  double* d = reinterpret_cast<double*>(w + L.d);
  double* e = reinterpret_cast<double*>(w + L.e);
  double* tau = reinterpret_cast<double*>(w + L.tau);
  mrrr_status st = mrrr_sytrd(plan, n, A, lda, d, e, tau, workspace, ws_bytes, stream);
  if (st != MRRR_OK) return st;
  // stage 4: the tridiagonal eigenpairs, Z written straight into Y
  st = mrrr_stein(plan, n, d, e, il, iu, W, Y, ldy, w + L.step, L.step_bytes, stream);
  if (st != MRRR_OK || !Y) return st;
  return mrrr_ormtr(plan, n, k, A, lda, tau, Y, ldy, workspace, ws_bytes, stream);
}

mrrr_status mrrr_dense_status(const void* workspace, mrrr_stream stream) {
  if (!workspace) return MRRR_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MRRR_ERR_CUDA;
  DenseCtl c{};
  if (cudaMemcpy(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return MRRR_ERR_CUDA;
  return static_cast<mrrr_status>(c.status);
}

}  // extern "C"
