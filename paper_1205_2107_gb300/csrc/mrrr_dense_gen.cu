// mrrr_dense_gen.cu -- the generalized symmetric-definite eigenproblem
// A x = lambda B x around the standard one (paper Sec. 1.2, stages 1, 2, 6):
//   1. Cholesky factorization B = L L^T;
//   2. reduction to the standard problem C = L^-1 A L^-T;
//   (3-5. eigenpairs C y = lambda y: mrrr_dense_eigh)
//   6. backtransformation x = L^-T y.
// All blocked by 64 (the tile of the FP64 tensor-core GEMM): a diagonal
// block is factored or inverted by one CTA, everything else is GEMM.
//   Cholesky, block column J: L_JJ from A_JJ (one CTA), L_JJ^-1 (one CTA),
//     L_IJ = A_IJ L_JJ^-T (GEMM), trailing A -= L_.J L_.J^T (lower GEMM).
//   L X = B, block row I in order: B_I -= L_I,<I X_<I (GEMM), X_I = L_II^-1 B_I.
//   L^T X = B, block row I in reverse: B_I -= L_>I,I^T X_>I, X_I = L_II^-T B_I.
//   C = L^-1 (L^-1 A)^T (A symmetric, both triangles given).
#include <algorithm>
#include <cmath>

#include "mrrr_dense.cuh"

namespace mrrr {
namespace dense {
namespace {

constexpr int kB = 64;  // block of the triangular algorithms
constexpr int kSplit = 8;  // split-K factor the scratch is sized for

// Unblocked Cholesky of the diagonal block A(k0:k0+bs, k0:k0+bs) in shared
// memory, right-looking; a pivot that is not positive (or not finite) sets
// MRRR_ERR_NOTSPD and leaves the block as it is.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_potf2(double* A, int64_t lda, int k0, int bs, DenseCtl* ctl) {
  __shared__ double a[kB][kB + 1];
  __shared__ int bad;
  for (int idx = threadIdx.x; idx < bs * bs; idx += blockDim.x) {
    const int c = idx / bs, r = idx % bs;
    a[r][c] = A[(k0 + r) + (int64_t)(k0 + c) * lda];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    if (threadIdx.x == 0) {
      const double p = a[j][j];
      if (!(p > 0.0) || !isfinite(p)) {
        bad = 1;
      } else {
        a[j][j] = sqrt(p);
      }
    }
    __syncthreads();
    if (bad) break;
    const double ljj = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < bs; i += blockDim.x) a[i][j] /= ljj;
    __syncthreads();
    const int m = bs - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = j + 1 + idx / m, kk = j + 1 + idx % m;
      if (i >= kk) a[i][kk] -= a[i][j] * a[kk][j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicCAS(&ctl->status, 0, (int)MRRR_ERR_NOTSPD);
    return;
  }
  for (int idx = threadIdx.x; idx < bs * bs; idx += blockDim.x) {
    const int c = idx / bs, r = idx % bs;
    if (r >= c) A[(k0 + r) + (int64_t)(k0 + c) * lda] = a[r][c];
  }
}

// Inverse of the lower-triangular diagonal block L(k0:k0+bs, k0:k0+bs), one
// CTA per block (blockIdx.x = block index), thread c solving L x = e_c by
// forward substitution; written to Linv + block * kB * kB (column-major,
// leading dimension kB, zero above the diagonal and outside bs).
__global__ void __launch_bounds__(kB) k_trinv(const double* L, int64_t ldl, int n, double* Linv) {
  __shared__ double l[kB][kB + 1];
  const int k0 = blockIdx.x * kB, bs = min(kB, n - k0);
  for (int idx = threadIdx.x; idx < bs * bs; idx += blockDim.x) {
    const int c = idx / bs, r = idx % bs;
    l[r][c] = r >= c ? L[(k0 + r) + (int64_t)(k0 + c) * ldl] : 0.0;
  }
  __syncthreads();
  double* out = Linv + (int64_t)blockIdx.x * kB * kB;
  const int c = threadIdx.x;
  double x[kB];
#pragma unroll 1
  for (int r = 0; r < kB; ++r) x[r] = 0.0;
  if (c < bs) {
    for (int r = c; r < bs; ++r) {
      double sacc = r == c ? 1.0 : 0.0;
      for (int q = c; q < r; ++q) sacc -= l[r][q] * x[q];
      x[r] = sacc / l[r][r];
    }
  }
  for (int r = 0; r < kB; ++r) out[r + (int64_t)c * kB] = (c < bs && r < bs) ? x[r] : 0.0;
}

// dst(r, j) = src(r, j) for r < rows, j < cols (column-major).
__global__ void k_copy(const double* src, int64_t lds, double* dst, int64_t ldd, int rows, int cols) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / rows), r = (int)(idx % rows);
    dst[r + (int64_t)j * ldd] = src[r + (int64_t)j * lds];
  }
}

// dst = src^T (n x n, column-major).
__global__ void k_transpose(const double* src, int64_t lds, double* dst, int64_t ldd, int n) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = bx + threadIdx.x, c = by + k;
    if (r < n && c < n) t[k][threadIdx.x] = src[r + (int64_t)c * lds];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = by + threadIdx.x, c = bx + k;
    if (r < n && c < n) dst[r + (int64_t)c * ldd] = t[threadIdx.x][k];
  }
}

void copy(const double* src, int64_t lds, double* dst, int64_t ldd, int rows, int cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  const int64_t tot = (int64_t)rows * cols;
  k_copy<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(8192, (tot + 255) / 256)), 256, 0, s>>>(src, lds, dst,
                                                                                                 ldd, rows, cols);
  count_launch();
}

}  // namespace

size_t gen_scratch_doubles(int n, int k) {
  const int64_t nbk = (n + kB - 1) / kB;
  const int64_t w = std::max({n, k, 1});
  return (size_t)(nbk * kB * kB + (int64_t)kB * w * (1 + kSplit) + (int64_t)n * n);
}

// B (n x n) <- L L^T, lower; scratch: Linv blocks, a kB x n panel buffer.
void launch_potrf(int n, double* B, int64_t ldb, double* scratch, DenseCtl* ctl, cudaStream_t s) {
  const int nbk = (n + kB - 1) / kB;
  double* Linv = scratch;
  double* P = Linv + (int64_t)nbk * kB * kB;  // n x kB (column-major, ld n)
  for (int J = 0; J < nbk; ++J) {
    const int k0 = J * kB, bs = std::min(kB, n - k0), r1 = k0 + bs, rows = n - r1;
    k_potf2<<<1, 256, 0, s>>>(B, ldb, k0, bs, ctl);
    count_launch();
    if (rows <= 0) break;
    // L_JJ^-1 of this block alone (a one-block inverse at the block's offset)
    k_trinv<<<1, kB, 0, s>>>(B + k0 + (int64_t)k0 * ldb, ldb, bs, Linv);
    count_launch();
    // L_IJ = A_IJ L_JJ^-T into the panel buffer, then back into B
    gemm(gemm_args(rows, bs, bs, 1.0, B + r1 + (int64_t)k0 * ldb, ldb, false, Linv, kB, true, 0.0, P, n), s);
    copy(P, n, B + r1 + (int64_t)k0 * ldb, ldb, rows, bs, s);
    // trailing lower triangle: A -= L_.J L_.J^T
    gemm(gemm_args(rows, rows, bs, -1.0, P, n, false, P, n, true, 1.0, B + r1 + (int64_t)r1 * ldb, ldb, true), s);
  }
}

// X <- L^-1 X (trans = false) or L^-T X (trans = true), X n x k.
void launch_trsm(int n, int k, const double* L, int64_t ldl, double* X, int64_t ldx, bool trans, double* scratch,
                 int nsm, cudaStream_t s) {
  const int nbk = (n + kB - 1) / kB;
  double* Linv = scratch;
  double* T = Linv + (int64_t)nbk * kB * kB;  // kB x k
  double* part = T + (int64_t)kB * std::max({n, k, 1});  // split-K partials, kSplit x kB x k
  k_trinv<<<nbk, kB, 0, s>>>(L, ldl, n, Linv);
  count_launch();
  for (int step = 0; step < nbk; ++step) {
    const int I = trans ? nbk - 1 - step : step;
    const int r0 = I * kB, bs = std::min(kB, n - r0), r1 = r0 + bs;
    const double* Li = Linv + (int64_t)I * kB * kB;
    // the update of block row I has only kB rows: split its depth over CTAs
    if (!trans && r0 > 0)
      gemm_splitk(gemm_args(bs, k, r0, -1.0, L + r0, ldl, false, X, ldx, false, 1.0, X + r0, ldx), part, kSplit,
                  nsm, s);
    if (trans && r1 < n)
      gemm_splitk(gemm_args(bs, k, n - r1, -1.0, L + r1 + (int64_t)r0 * ldl, ldl, true, X + r1, ldx, false, 1.0,
                            X + r0, ldx),
                  part, kSplit, nsm, s);
    gemm(gemm_args(bs, k, bs, 1.0, Li, kB, trans, X + r0, ldx, false, 0.0, T, kB), s);
    copy(T, kB, X + r0, ldx, bs, k, s);
  }
}

// A (full symmetric) <- L^-1 A L^-T.
void launch_sygst(int n, double* A, int64_t lda, const double* L, int64_t ldl, double* scratch, int nsm,
                  cudaStream_t s) {
  const int nbk = (n + kB - 1) / kB;
  double* M = scratch + (int64_t)nbk * kB * kB + (int64_t)kB * std::max(n, 1) * (1 + kSplit);  // n x n
  launch_trsm(n, n, L, ldl, A, lda, false, scratch, nsm, s);  // A <- L^-1 A
  dim3 tb(32, 8), tg((n + 31) / 32, (n + 31) / 32);
  k_transpose<<<tg, tb, 0, s>>>(A, lda, M, n, n);          // M = (L^-1 A)^T = A L^-T
  count_launch();
  launch_trsm(n, n, L, ldl, M, n, false, scratch, nsm, s); // M <- L^-1 A L^-T
  copy(M, n, A, lda, n, n, s);
}

}  // namespace dense
}  // namespace mrrr

// ---------------------------------------------------------------------------
// C ABI of the generalized problem.

using namespace mrrr::dense;

namespace {

size_t galign(size_t x) { return (x + 255) / 256 * 256; }

int device_sms() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return nsm;
}

struct GenLayout {
  size_t ctl, scratch, dense, total, dense_bytes;
};

GenLayout gen_layout(const mrrr_plan* plan, int n, int k) {
  GenLayout L{};
  L.ctl = 0;
  L.scratch = galign(sizeof(DenseCtl));
  L.dense = galign(L.scratch + sizeof(double) * gen_scratch_doubles(n, k));
  size_t db = 0;
  mrrr_dense_workspace_size(plan, n, k, &db);
  L.dense_bytes = db;
  L.total = galign(L.dense + db);
  return L;
}

}  // namespace

extern "C" {

mrrr_status mrrr_gen_workspace_size(const mrrr_plan* plan, int n, int k, size_t* bytes) {
  if (!plan || !bytes || n < 0 || k < 0 || k > n) return MRRR_ERR_ARG;
  *bytes = gen_layout(plan, n, k).total;
  return MRRR_OK;
}

mrrr_status mrrr_potrf(mrrr_plan* plan, int n, double* B, int64_t ldb, void* workspace, size_t ws_bytes,
                       mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!B || ldb < n) return MRRR_ERR_ARG;
  const GenLayout L = gen_layout(plan, n, 0);
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DenseCtl* ctl = reinterpret_cast<DenseCtl*>(w + L.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(DenseCtl), s) != cudaSuccess) return MRRR_ERR_CUDA;
  launch_potrf(n, B, ldb, reinterpret_cast<double*>(w + L.scratch), ctl, s);
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

mrrr_status mrrr_sygst(mrrr_plan* plan, int n, double* A, int64_t lda, const double* Lf, int64_t ldl,
                       void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!A || lda < n || !Lf || ldl < n) return MRRR_ERR_ARG;
  const GenLayout L = gen_layout(plan, n, 0);
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  const int nsm = device_sms();
  if (nsm <= 0) return MRRR_ERR_CUDA;
  launch_sygst(n, A, lda, Lf, ldl, reinterpret_cast<double*>(w + L.scratch), nsm, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

mrrr_status mrrr_trsm_lt(mrrr_plan* plan, int n, int k, const double* Lf, int64_t ldl, double* X, int64_t ldx,
                         void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0 || k < 0) return MRRR_ERR_ARG;
  if (n == 0 || k == 0) return MRRR_OK;
  if (!Lf || ldl < n || !X || ldx < n) return MRRR_ERR_ARG;
  const GenLayout L = gen_layout(plan, n, std::min(k, n));
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  const int nsm = device_sms();
  if (nsm <= 0) return MRRR_ERR_CUDA;
  launch_trsm(n, k, Lf, ldl, X, ldx, true, reinterpret_cast<double*>(w + L.scratch), nsm,
              static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? MRRR_OK : MRRR_ERR_CUDA;
}

mrrr_status mrrr_gen_eigh(mrrr_plan* plan, int n, double* A, int64_t lda, double* B, int64_t ldb, int il, int iu,
                          double* W, double* X, int64_t ldx, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  if (!plan || n < 0) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!A || lda < n || !B || ldb < n || !W || il < 1 || iu > n || il > iu || (X && ldx < n)) return MRRR_ERR_ARG;
  const int k = iu - il + 1;
  const GenLayout L = gen_layout(plan, n, k);
  if (!workspace || ws_bytes < L.total) return MRRR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  mrrr_status st = mrrr_potrf(plan, n, B, ldb, workspace, ws_bytes, stream);  // stage 1
  if (st != MRRR_OK) return st;
  st = mrrr_sygst(plan, n, A, lda, B, ldb, workspace, ws_bytes, stream);  // stage 2
  if (st != MRRR_OK) return st;
  // stages 3-5 on C (its device status word is the dense workspace's own)
  st = mrrr_dense_eigh(plan, n, A, lda, il, iu, W, X, ldx, w + L.dense, L.dense_bytes, stream);
  if (st != MRRR_OK || !X) return st;
  return mrrr_trsm_lt(plan, n, k, B, ldb, X, ldx, workspace, ws_bytes, stream);  // stage 6
}

mrrr_status mrrr_gen_status(const mrrr_plan* plan, int n, int k, const void* workspace, mrrr_stream stream) {
  if (!plan || !workspace || n < 0 || k < 0 || k > n) return MRRR_ERR_ARG;
  const GenLayout L = gen_layout(plan, n, k);
  const mrrr_status a = mrrr_dense_status(workspace, stream);
  if (a != MRRR_OK) return a;
  return mrrr_dense_status(static_cast<const char*>(workspace) + L.dense, stream);
}

}  // extern "C"
