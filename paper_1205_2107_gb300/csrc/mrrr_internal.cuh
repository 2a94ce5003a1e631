// mrrr_internal.cuh -- device data structures and the qd building blocks of
// the MRRR solver (FP64, sm_103a).
//
// Notation follows the paper's Sec. 3.1.1: a representation (RRR) of a
// shifted block is L D L^T with L unit lower bidiagonal (subdiagonal l_i) and
// D diagonal.  Each row i of a representation stores
//   D_i, LLD_i = l_i^2 D_i, l_i, LD_i = l_i D_i          (32 bytes, RepRow)
// so that the Sturm count (D, LLD), the stationary and progressive qd
// transforms (D, l, LD, LLD) read one contiguous record per row.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mrrr.h"

namespace mrrr {

constexpr double kEps = 0x1p-53;          // unit roundoff of IEEE double
constexpr double kSafmin = 0x1p-1022;     // smallest normal double

// Slot states
enum : int {
  SLOT_ACTIVE = 1,     // interval being refined / classified
  SLOT_SINGLETON = 2,  // well separated at its node: gets a vector
  SLOT_TRIVIAL = 3,    // 1x1 block: eigenvalue d, vector e_row
  SLOT_FALLBACK = 4,   // cluster beyond the depth limit, treated as singleton
};

struct Problem {
  int64_t row0;   // first row in the packed d / e
  int n;
  int il, iu;     // requested range (1-based, inclusive)
  int nblocks;
  int block0;     // first block index
  int k;          // iu - il + 1
  int64_t slot0;  // first slot of the problem
  int nslots;
  int64_t wout;   // W output offset
  int64_t zout;   // Z output offset (elements)
  int64_t ldz;
  double scale;   // T is handled as scale * T (a power of two)
  double thresh;  // split threshold eps * G(T) (unscaled units)
};

struct Block {
  int64_t row0;   // global row of the first row
  int m;          // order of the block
  int prob;       // problem index
  int js, je;     // local indices (1-based) with a slot: js..je
  int64_t slot0;  // slot of local index js
  double gl, gu;  // Gershgorin bounds of the scaled block
};

struct Node {
  int block;
  int depth;
  int64_t first, last;  // slot range (inclusive)
  int parent;           // -1 for a root
  int pad_;
  int64_t rep;          // first RepRow of this node's representation
  double sigma_rel;     // shift relative to the parent's coordinates
  double sigma_abs;     // eigenvalue of scaled T = sigma_abs + local value
  double gapl, gapr;    // absolute gaps to the left / right of the slot range
  double pivmin;        // zero-pivot guard of this representation
  double spdiam;        // width of the block's spectrum (shift invariant)
};

struct RepRow {
  double D, LLD, l, LD;
};

// Device control block (first bytes of the workspace).
struct Ctl {
  int status;             // first error (mrrr_status), 0 = OK
  int nblocks;
  int64_t nslots;
  int nodes;              // nodes allocated (roots = blocks, then children)
  int level_new;          // clusters created by the current level
  int level_begin;        // first node id created by the current level
  int depth;              // deepest level reached
  int64_t pool_top;       // rows of the pool in use (roots + children)
  int64_t pool_need;      // rows requested (may exceed the capacity)
  unsigned long long fallbacks;
  unsigned long long rq_iters;
  int levels;
  int pad_;
  unsigned long long diag[8];  // per-site event counters (see mrrr_info.diag)
};

// Indices of Ctl::diag (mirrored in mrrr_info.diag).
enum : int {
  DIAG_ROOT_SHIFT = 0,     // root shift retries exhausted (blocks)
  DIAG_ROOT_BISECT = 1,    // root bisection hit its step cap (intervals)
  DIAG_REFINE_BRACKET = 2, // child bracket could not be confirmed (intervals)
  DIAG_REFINE_BISECT = 3,  // child bisection hit its step cap (intervals)
  DIAG_RQ = 4,             // Rayleigh-quotient iteration cap (vectors)
  DIAG_CHILD_GROWTH = 5,   // no child shift met the growth bound (clusters)
  DIAG_DEPTH = 6,          // depth-limit fallback (eigenvalues)
  DIAG_CAPACITY = 7,       // node table / pool full fallback (eigenvalues)
};

// Device views of the workspace, passed by value to kernels.
struct Dev {
  Ctl* ctl;
  Problem* prob;
  Block* blk;
  Node* node;
  RepRow* pool;
  int64_t pool_cap;   // rows
  int max_blocks;
  int max_nodes;
  int64_t max_slots;
  // slots (structure of arrays)
  double* lo;
  double* hi;
  double* gap;        // absolute gap of a singleton (for the RQI stop test)
  double* wval;       // final eigenvalue (scaled, absolute)
  double* znrm2;      // squared norm of the unnormalised vector
  int* snode;
  int* sj;            // local index j (1-based) within its block
  int* spos;          // output column, -1 = computed but not returned
  int* state;
  unsigned char* bflag;  // boundary after this slot (classification)
  int64_t* pos_slot;  // output position -> slot (per problem: wout + pos)
  // eigenvector scratch (interleaved by thread)
  double* vscr;
  int64_t vscr_threads;
  int64_t vscr_rows;
  // problem inputs / outputs
  const double* d;
  const double* e;
  double* W;
  double* Z;
  int batch;
  // options
  double gap_tol;
  double rtol;          // root classification accuracy
  double rtol_cluster;  // accuracy of cluster eigenvalues (shift placement, children)
  double root_perturb;  // root perturbation size in ulps
  int max_depth;
  int max_bisect;
  int max_rq;
};

__device__ __forceinline__ void set_status(Ctl* c, int code) {
  atomicCAS(&c->status, 0, code);
}

__device__ __forceinline__ void diag(Ctl* c, int site, unsigned long long k = 1) {
  atomicAdd(&c->diag[site], k);
}

// ---------------------------------------------------------------------------
// Sturm count on a representation (Sec. 3.1.1: bisection on the RRR).  The
// number of negative pivots D+_i of the stationary transform
//   L+ D+ L+^T = L D L^T - tau I,
//   s_1 = -tau,  D+_i = D_i + s_i,  s_{i+1} = LLD_i s_i / D+_i - tau,
// equals the number of eigenvalues of L D L^T below tau (Sylvester's law of
// inertia).  Pivots with |D+_i| < pivmin are replaced by -pivmin.
__device__ __forceinline__ int negcount_div(const RepRow* __restrict__ rep, int m, double tau,
                                            double pivmin) {
  int cnt = 0;
  double s = -tau;
  for (int i = 0; i < m - 1; ++i) {
    const double2 dl = *reinterpret_cast<const double2*>(&rep[i].D);  // D, LLD
    double dp = dl.x + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    cnt += (dp < 0.0);
    s = fma(dl.y, s / dp, -tau);
  }
  double dp = rep[m - 1].D + s;
  if (fabs(dp) < pivmin) dp = -pivmin;
  cnt += (dp < 0.0);
  return cnt;
}

__device__ __forceinline__ int negcount(const RepRow* __restrict__ rep, int m, double tau, double pivmin) {
  return negcount_div(rep, m, tau, pivmin);
}

__device__ __forceinline__ bool converged(double lo, double hi, double rtol, double atol) {
  double w = hi - lo;
  return w <= fmax(rtol * fmax(fabs(lo), fabs(hi)), atol);
}

// Bisection of [lo, hi] (count(lo) <= j-1 < count(hi) on entry) until the
// width is below rtol relative (atol absolute).  Returns steps taken.
__device__ __forceinline__ int bisect_interval(const RepRow* __restrict__ rep, int m, int j,
                                               double pivmin, double rtol, double atol, int maxit,
                                               double& lo, double& hi) {
  int it = 0;
  for (; it < maxit; ++it) {
    if (converged(lo, hi, rtol, atol)) break;
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (negcount(rep, m, mid, pivmin) >= j)
      hi = mid;
    else
      lo = mid;
  }
  return it;
}

// Grid helpers
__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

}  // namespace mrrr
