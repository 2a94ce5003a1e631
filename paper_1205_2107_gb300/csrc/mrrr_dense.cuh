// mrrr_dense.cuh -- shared pieces of the dense stages (mrrr_dense.cu,
// mrrr_dense_gen.cu): the FP64 tensor-core GEMM and the device status word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mrrr_launch.h"

namespace mrrr {
namespace dense {

// C(i, j) = alpha sum_p A(i, p) B(p, j) + beta C(i, j) for i < m, j < n,
// with A(i, p) = A[i a_rs + p a_cs], B(p, j) = B[p b_rs + j b_cs] and
// C(i, j) = C[i + j ldc].  lower: only i >= j is written (tiles above the
// diagonal are skipped).
struct GemmArgs {
  int m, n, k;
  int lower;
  const double* A;
  int64_t a_rs, a_cs;
  const double* B;
  int64_t b_rs, b_cs;
  double* C;
  int64_t ldc;
  double alpha, beta;
  int kchunk;       // split-K: CTA z of grid.z sums k in [z kchunk, (z+1) kchunk) (0: all)
  int64_t cstride;  //   into C + z cstride (the partials, reduced by gemm_splitk)
};

void gemm(const GemmArgs& g, cudaStream_t s);
// C = alpha op(A) op(B) + beta C with K split over CTAs when the output has
// too few tiles to fill the GPU: partial products into `partials` (room for
// max_split m x n blocks), then summed in a fixed order.
void gemm_splitk(GemmArgs g, double* partials, int max_split, int nsm, cudaStream_t s);

// op(A), op(B) of column-major matrices (ta / tb: transposed).
GemmArgs gemm_args(int m, int n, int k, double alpha, const double* A, int64_t lda, bool ta, const double* B,
                   int64_t ldb, bool tb, double beta, double* C, int64_t ldc, bool lower = false);

constexpr int kNb = 32;      // panel width of the reduction to tridiagonal form
constexpr int kNbBt = 128;   // reflectors per panel of the backtransformation
constexpr int kRowCta = 256; // threads of the row-parallel kernels

// Device status of a dense call (first error wins), in the workspace.
struct DenseCtl {
  int status;
  int pad_;
};

// Reduction to tridiagonal form: A (n x n, column-major, lower triangle
// read and overwritten by the reflectors), d, e, tau outputs, scratch.
struct TrdArgs {
  int n;
  double* A;
  int64_t lda;
  double* d;
  double* e;
  double* tau;
  double* V;        // panel reflectors, n x kNb
  double* W;        // panel update vectors, n x kNb
  double* P;        // symmetric-product partials, T x T x 64
  double* colpart;  // per-CTA sums of squares
  double* wvpart;   // per-CTA partial w^T v
  double* dotpart;  // per-CTA W^T v and V^T v, 2 kNb each
  DenseCtl* ctl;
};
size_t trd_scratch_doubles(int n);
TrdArgs trd_args(int n, double* A, int64_t lda, double* d, double* e, double* tau, double* scratch, DenseCtl* ctl);
void launch_trd(const TrdArgs& t, cudaStream_t s);

// Y (n x k, column-major) <- Q Y with Q = H_0 ... H_{n-3} from the reflectors
// below the subdiagonal of the reduced A and tau.
size_t orm_scratch_doubles(int n, int k);
void launch_orm(int n, int k, const double* A, int64_t lda, const double* tau, double* Y, int64_t ldy,
                double* scratch, int nsm, cudaStream_t s);

}  // namespace dense
}  // namespace mrrr
