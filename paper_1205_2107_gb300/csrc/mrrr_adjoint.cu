// mrrr_adjoint.cu -- backward pass: gradient of a loss L(W, Z) with respect
// to the tridiagonal (d, e), for a batch of problems solved for all
// eigenpairs.  Not in the paper: first-order perturbation theory of
// T = Z diag(W) Z^T.  With Tbar = Z (diag(Wbar) + F o (Z^T Zbar)) Z^T,
// F(a,b) = 1/(W_b - W_a) for |W_b - W_a| > tau (else 0, and 0 on the
// diagonal):
//   dbar_j = Tbar(j,j),   ebar_j = Tbar(j,j+1) + Tbar(j+1,j).
//
// Without Zbar only the eigenvalue part remains, one fused pass over Z:
//   dbar_j = sum_i Wbar_i Z(j,i)^2,  ebar_j = 2 sum_i Wbar_i Z(j,i) Z(j+1,i).
// With Zbar, S = H + H^T for H = diag(Wbar) + F o G, G = Z^T Zbar, i.e.
//   S = F o (G - G^T) + 2 diag(Wbar)       (F is antisymmetric),
// and with Q = Z S (row j of Q is z_j^T S, z_j = row j of Z):
//   dbar_j = z_j^T H z_j = (1/2) sum_a Q(j,a) Z(j,a),
//   ebar_j = z_j^T S z_{j+1} = sum_a Q(j,a) Z(j+1,a).
// G and Q are dense contractions of 2 n^3 flops each: they run on the FP64
// tensor cores (mma.sync m8n8k4 f64, the double-precision MMA of sm_103a)
// with the epilogues fused: the first GEMM stores G, one elementwise pass
// forms S in place, the second GEMM reduces Q against Z row by row and never
// stores Q.  Every reduction runs in a fixed order (no atomics): the result
// is deterministic.
#include <algorithm>
#include <cmath>

#include "mrrr_launch.h"

namespace mrrr {
namespace {

constexpr int kTM = 64;        // CTA tile rows (M)
constexpr int kTN = 64;        // CTA tile columns (N)
constexpr int kTK = 32;        // K per shared-memory stage
constexpr int kKS = kTK + 4;   // padded row stride of the K-contiguous tiles (doubles)
constexpr int kGemmThreads = 128;  // 4 warps, 2 x 2, each 32 x 32

// Problem geometry from the row offsets: n_p and the start of its n_p x n_p
// blocks (sum of n_q^2 over q < p, precomputed into zoff).
struct AdjArgs {
  int batch;
  const int64_t* d_off;
  int64_t* zoff;        // workspace, batch + 1 entries
  const double* W;
  const double* Z;
  const double* Wbar;
  const double* Zbar;
  double tau_rel;
  double* S;  // workspace, sum n_p^2 doubles
  double* dbar;
  double* ebar;
};

// zoff[p] = sum_{q<p} (d_off[q+1]-d_off[q])^2, one CTA.
__global__ void k_adj_offsets(AdjArgs a) {
  __shared__ int64_t s_part[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int per = (a.batch + nt - 1) / nt;
  const int p0 = min(a.batch, t * per), p1 = min(a.batch, p0 + per);
  int64_t sum = 0;
  for (int p = p0; p < p1; ++p) {
    const int64_t n = a.d_off[p + 1] - a.d_off[p];
    sum += n * n;
  }
  s_part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < nt; ++i) {
      const int64_t v = s_part[i];
      s_part[i] = run;
      run += v;
    }
    a.zoff[a.batch] = run;
  }
  __syncthreads();
  int64_t run = s_part[t];
  for (int p = p0; p < p1; ++p) {
    a.zoff[p] = run;
    const int64_t n = a.d_off[p + 1] - a.d_off[p];
    run += n * n;
  }
}

// Eigenvalue part only (Zbar absent): one thread per row j, columns i in
// order; consecutive threads read consecutive rows (coalesced).
__global__ void k_adj_values(AdjArgs a) {
  const int p = blockIdx.y;
  const int64_t r0 = a.d_off[p];
  const int n = (int)(a.d_off[p + 1] - r0);
  const double* Z = a.Z + a.zoff[p];
  const double* Wb = a.Wbar ? a.Wbar + r0 : nullptr;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double sd = 0.0, se = 0.0;
    if (Wb) {
      for (int i = 0; i < n; ++i) {
        const double w = Wb[i];
        const double zj = Z[(int64_t)i * n + j];
        const double wz = w * zj;
        sd = fma(wz, zj, sd);
        if (j + 1 < n) se = fma(wz, Z[(int64_t)i * n + j + 1], se);
      }
    }
    a.dbar[r0 + j] = sd;
    a.ebar[r0 + j] = j + 1 < n ? 2.0 * se : 0.0;
  }
}

// ---------------------------------------------------------------------------
// FP64 MMA: D(8x8) += A(8x4) B(4x8).  Fragments (PTX ISA, mma.m8n8k4 .f64):
// A: one element, row lane/4, column lane%4; B: one element, row lane%4,
// column lane/4; C/D: two elements, row lane/4, columns 2(lane%4) + {0,1}.
__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// One K stage: the warp's 32 x 32 block of C += As(m, k) Bs(n, k) over kTK,
// both tiles stored K-contiguous with row stride kKS.
__device__ __forceinline__ void mma_stage(const double* As, const double* Bs, int wm, int wn, int lane,
                                          double (&acc)[4][4][2]) {
  const int r = lane >> 2, c = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < kTK; k0 += 4) {
    double af[4], bf[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) af[i] = As[(wm + 8 * i + r) * kKS + k0 + c];
#pragma unroll
    for (int j = 0; j < 4; ++j) bf[j] = Bs[(wn + 8 * j + r) * kKS + k0 + c];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
  }
}

// Tile loaders into K-contiguous shared tiles T(row, k), rows r0.., k k0..:
// src(row, k) = base[row * ld + k] (K contiguous in memory) or
// base[k * ld + row] (rows contiguous in memory); zero outside [0, n).
__device__ __forceinline__ void load_kcontig(double* T, const double* base, int64_t ld, int n, int r0, int k0,
                                             int rows) {
  for (int idx = threadIdx.x; idx < rows * kTK; idx += blockDim.x) {
    const int rr = idx / kTK, kk = idx % kTK;
    const int row = r0 + rr, k = k0 + kk;
    T[rr * kKS + kk] = (row < n && k < n) ? base[(int64_t)row * ld + k] : 0.0;
  }
}
__device__ __forceinline__ void load_rcontig(double* T, const double* base, int64_t ld, int n, int r0, int k0,
                                             int rows) {
  for (int idx = threadIdx.x; idx < rows * kTK; idx += blockDim.x) {
    const int kk = idx / rows, rr = idx % rows;
    const int row = r0 + rr, k = k0 + kk;
    T[rr * kKS + kk] = (row < n && k < n) ? base[(int64_t)k * ld + row] : 0.0;
  }
}

// GEMM 1: G(a, b) = sum_j Z(j, a) Zbar(j, b), tile (blockIdx.x, blockIdx.y)
// of problem blockIdx.z, stored into S (row-major, n x n).
__global__ void __launch_bounds__(kGemmThreads) k_adj_gemm_g(AdjArgs a) {
  __shared__ double As[kTM * kKS];
  __shared__ double Bs[kTN * kKS];
  const int p = blockIdx.z;
  const int64_t r0 = a.d_off[p];
  const int n = (int)(a.d_off[p + 1] - r0);
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  if (m0 >= n || n0 >= n) return;
  const double* Z = a.Z + a.zoff[p];
  const double* Zb = a.Zbar + a.zoff[p];
  double* G = a.S + a.zoff[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  double acc[4][4][2] = {};
  for (int k0 = 0; k0 < n; k0 += kTK) {
    // A(a, j) = Z(j, a) = Z[a * n + j]: K-contiguous; B(b, j) = Zbar[b * n + j]
    load_kcontig(As, Z, n, n, m0, k0, kTM);
    load_kcontig(Bs, Zb, n, n, n0, k0, kTN);
    __syncthreads();
    mma_stage(As, Bs, wm, wn, lane, acc);
    __syncthreads();
  }
  const int r = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm + 8 * i + r, col = n0 + wn + 8 * j + c2 + h;
        if (row < n && col < n) G[(int64_t)row * n + col] = acc[i][j][h];
      }
}

// S = F o (G - G^T) + 2 diag(Wbar) in place: one thread per pair a <= b.
__global__ void k_adj_sym(AdjArgs a) {
  const int p = blockIdx.y;
  const int64_t r0 = a.d_off[p];
  const int n = (int)(a.d_off[p + 1] - r0);
  double* S = a.S + a.zoff[p];
  const double* W = a.W + r0;
  const double wmax = n ? fmax(fabs(W[0]), fabs(W[n - 1])) : 0.0;
  const double tau = a.tau_rel * wmax;
  const int64_t pairs = (int64_t)n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < pairs; t += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(t / n), ib = (int)(t % n);
    if (ib < ia) continue;
    if (ia == ib) {
      S[(int64_t)ia * n + ia] = a.Wbar ? 2.0 * a.Wbar[r0 + ia] : 0.0;
      continue;
    }
    const double gap = W[ib] - W[ia];
    const double f = fabs(gap) > tau ? 1.0 / gap : 0.0;  // F(a, b); F(b, a) = -f
    const double gab = S[(int64_t)ia * n + ib], gba = S[(int64_t)ib * n + ia];
    const double s = f * (gab - gba);
    S[(int64_t)ia * n + ib] = s;
    S[(int64_t)ib * n + ia] = s;
  }
}

// GEMM 2, rows j0..j0+63 of Q = Z S over all columns a, reduced on the fly:
//   dbar_j = 1/2 sum_a Q(j,a) Z(j,a),  ebar_j = sum_a Q(j,a) Z(j+1,a).
// One CTA per row tile (blockIdx.x) of problem blockIdx.y; column tiles in
// order, so the sums are deterministic.
__global__ void __launch_bounds__(kGemmThreads) k_adj_gemm_q(AdjArgs a) {
  __shared__ double As[kTM * kKS];
  __shared__ double Bs[kTN * kKS];
  __shared__ double s_d[kTM][2], s_e[kTM][2];  // per row, per warp column half
  const int p = blockIdx.y;
  const int64_t r0 = a.d_off[p];
  const int n = (int)(a.d_off[p + 1] - r0);
  const int m0 = blockIdx.x * kTM;
  if (m0 >= n) return;
  const double* Z = a.Z + a.zoff[p];
  const double* S = a.S + a.zoff[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int r = lane >> 2, c2 = (lane & 3) * 2;
  double rd[4] = {}, re[4] = {};  // this thread's partial sums of rows m0 + wm + 8i + r
  for (int n0 = 0; n0 < n; n0 += kTN) {
    double acc[4][4][2] = {};
    for (int k0 = 0; k0 < n; k0 += kTK) {
      // A(j, b) = Z(j, b) = Z[b * n + j]: rows contiguous; B(a, b) = S(b, a) = S[a * n + b] (S symmetric)
      load_rcontig(As, Z, n, n, m0, k0, kTM);
      load_kcontig(Bs, S, n, n, n0, k0, kTN);
      __syncthreads();
      mma_stage(As, Bs, wm, wn, lane, acc);
      __syncthreads();
    }
    // fused reduction against Z: rows j = m0+wm+8i+r, columns a = n0+wn+8jj+c2+h
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = m0 + wm + 8 * i + r;
      if (j >= n) continue;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = n0 + wn + 8 * jj + c2 + h;
          if (col >= n) continue;
          const double q = acc[i][jj][h];
          rd[i] = fma(q, Z[(int64_t)col * n + j], rd[i]);
          if (j + 1 < n) re[i] = fma(q, Z[(int64_t)col * n + j + 1], re[i]);
        }
    }
  }
  // reduce over the 4 lanes that share a row, then over the two warps of a row
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double d = rd[i], e = re[i];
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    e += __shfl_xor_sync(0xffffffffu, e, 2);
    if ((lane & 3) == 0) {
      s_d[wm + 8 * i + r][warp & 1] = d;
      s_e[wm + 8 * i + r][warp & 1] = e;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kTM; t += blockDim.x) {
    const int j = m0 + t;
    if (j >= n) continue;
    a.dbar[r0 + j] = 0.5 * (s_d[t][0] + s_d[t][1]);
    a.ebar[r0 + j] = j + 1 < n ? s_e[t][0] + s_e[t][1] : 0.0;
  }
}

}  // namespace
}  // namespace mrrr

using namespace mrrr;

extern "C" {

mrrr_status mrrr_backward_workspace_size(const mrrr_plan* plan, int batch, int64_t z_total, size_t* bytes) {
  if (!plan || !bytes || batch < 0 || z_total < 0) return MRRR_ERR_ARG;
  const size_t off = ((size_t)(batch + 1) * sizeof(int64_t) + 255) / 256 * 256;
  *bytes = off + (size_t)z_total * sizeof(double) + 256;
  return MRRR_OK;
}

mrrr_status mrrr_backward(mrrr_plan* plan, int batch, const int64_t* d_off, const double* W, const double* Z,
                          const double* Wbar, const double* Zbar, double tau_rel, int n_max, int64_t z_total,
                          double* dbar, double* ebar, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || batch < 0 || n_max < 0 || z_total < 0 || !(tau_rel >= 0.0)) return MRRR_ERR_ARG;
  if (batch > 65535) return MRRR_ERR_ARG;  // one grid z (or y) index per problem
  if (batch == 0 || n_max == 0) return MRRR_OK;
  if (!d_off || !W || !Z || !dbar || !ebar) return MRRR_ERR_ARG;
  size_t need = 0;
  mrrr_backward_workspace_size(plan, batch, z_total, &need);
  if (!workspace || ws_bytes < need) return MRRR_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* b = static_cast<unsigned char*>(workspace);
  const size_t off = ((size_t)(batch + 1) * sizeof(int64_t) + 255) / 256 * 256;
  AdjArgs a{batch, d_off, reinterpret_cast<int64_t*>(b), W, Z, Wbar, Zbar, tau_rel,
            reinterpret_cast<double*>(b + off), dbar, ebar};
  k_adj_offsets<<<1, 1024, 0, s>>>(a);
  if (!Zbar) {
    const int rows = (n_max + 127) / 128;
    k_adj_values<<<dim3(rows, batch), 128, 0, s>>>(a);
  } else {
    const int tiles = (n_max + kTM - 1) / kTM;
    k_adj_gemm_g<<<dim3(tiles, tiles, batch), kGemmThreads, 0, s>>>(a);
    const int64_t pairs = (int64_t)n_max * n_max;
    const int sblocks = (int)std::min<int64_t>((pairs + 255) / 256, 1024);
    k_adj_sym<<<dim3(sblocks, batch), 256, 0, s>>>(a);
    k_adj_gemm_q<<<dim3(tiles, batch), kGemmThreads, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

}  // extern "C"
