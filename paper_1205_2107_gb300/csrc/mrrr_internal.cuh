// mrrr_internal.cuh -- device data structures and the qd building blocks of
// the MRRR solver (FP64, sm_103a).
//
// Notation follows the paper's Sec. 3.1.1: a representation (RRR) of a
// shifted block is L D L^T with L unit lower bidiagonal (subdiagonal l_i) and
// D diagonal.  A representation of m rows is stored as two planes of
// 16-byte records in the representation pool:
//   dl[i] = (D_i, LLD_i = l_i^2 D_i)   -- all a Sturm count reads
//   ul[i] = (l_i, LD_i = l_i D_i)      -- the rest of the qd transforms
// so a Sturm count streams exactly 16 bytes per row into shared memory.
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


__device__ __forceinline__ bool slot_final(int st) {
  return st == SLOT_SINGLETON || st == SLOT_FALLBACK;
}


struct Problem {
  int64_t row0;   // first row in the packed d / e
  int n;
  int il, iu;     // range of eigenvalues computed (1-based, inclusive)
  int ol, ou;     // range returned (within il..iu; equal to it except for a slice)
  int slice;      // a slice of a larger index range (mrrr_stein_slice)
  int pad_;
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

struct RepRow {  // one row of a representation, unpacked
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
  unsigned long long twisted_solves;
  int levels;
  int pad_;
  unsigned long long diag[12];  // per-site event counters (see mrrr_info.diag)
  long long nlist;        // long intervals in the engine's work list (front)
  long long list_next;    // next long entry to hand out
  long long nlist2;       // short intervals (back of the list)
  long long list_next2;   // next short entry to hand out
  int done;               // the tree is complete: later levels' kernels exit at once
  int pad4_;
  unsigned long long eng_counts[4];  // interval engine, per mode: Sturm counts evaluated (lanes)
  unsigned long long eng_rows[4];    //   rows those counts ran over
  unsigned long long eng_passes[4];  //   warp passes (each costs its FP64 instructions whatever
                                     //   the number of active lanes)
  int sched_gen;                     // chunk scheduler: launch generation (claim stamps)
  int pad5_;
  unsigned long long sched_dyn;      //   chunks handed out past the ranked ones
  unsigned long long sched_cleanup;  //   sweep over ranked chunks nobody claimed
  unsigned long long stage_ns[16];  // per-stage GPU time from device-clock marks (graph solves)
  unsigned long long t_last;        // global timer at the last mark
  long long orth_runs;              // runs of linked eigenvectors found by the safeguard
  long long cand_top;               // rows of candidate child transforms in the scratch (per level)
};

// Indices of Ctl::diag (mirrored in mrrr_info.diag).
enum : int {
  DIAG_ROOT_SHIFT = 0,     // root shift retries exhausted (blocks)
  DIAG_ROOT_BISECT = 1,    // root bisection hit its step cap (intervals)
  DIAG_REFINE_BRACKET = 2, // child bracket could not be confirmed (intervals)
  DIAG_REFINE_BISECT = 3,  // child bisection hit its step cap (intervals)
  DIAG_CHILD_WAVE2 = 4,    // clusters whose first candidate shifts all failed (second wave)
  DIAG_CHILD_GROWTH = 5,   // no child shift met the growth bound (clusters)
  DIAG_DEPTH = 6,          // depth-limit fallback (eigenvalues)
  DIAG_CAPACITY = 7,       // node table / pool full fallback (eigenvalues)
  DIAG_ORTH_FIX = 8,       // runs of neighbouring vectors re-orthogonalised
  DIAG_CHILD_RESTORE = 9,  // child transforms computed again with stores
  DIAG_SPARE10 = 10,
  DIAG_SPARE11 = 11,
};

// Device views of the workspace, passed by value to kernels.
struct Dev {
  Ctl* ctl;
  Problem* prob;
  Block* blk;
  Node* node;
  double2* rep_dl;    // (D, LLD) plane of the representation pool
  double2* rep_ul;    // (l, LD) plane
  int64_t pool_cap;   // rows
  int64_t* ilist;     // work list of the interval engine (slot indices)
  int64_t max_list;
  int64_t* lwin;      // per 32-slot window: offsets of its long and short entries in the list
  int* rgrid;         // FP32 root counts on a grid per block (2 ints per row of T)
  int* sched_cnt;     // chunk scheduler: warps seen per SM sub-partition (kSchedSlots)
  int* sched_claim;   //   per chunk: generation of the launch that claimed it
  int64_t max_chunks;
  int nsm;            // SMs of the device

  int max_blocks;
  int max_nodes;
  int64_t max_slots;
  // slots (structure of arrays)
  double* lo;
  double* hi;
  double* gap;        // absolute gap of a singleton or fallback slot to its neighbours
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
  double root32_rtol;   // relative width of the FP32 pre-bisection of root intervals
  int max_depth;
  int max_bisect;
  int engine_ctas;      // engine CTAs per SM (1 or 2)
  double width_scale;   // multiplies the resident lanes when choosing the multisection width
  int fixed_width;      // 0: width from the list length, brackets pooled; else fixed width, no pooling
  int no_orth_fix;      // skip the neighbour orthogonality safeguard (slices)
  int vec_dd;           // eigenvectors in double-double arithmetic
  int rq_steps;         // Rayleigh-quotient corrections of singletons (0: full bisection)
  int root_side;        // 0 nearer the wanted range, 1 left, 2 right
};

__device__ __forceinline__ void set_status(Ctl* c, int code) {
  atomicCAS(&c->status, 0, code);
}

__device__ __forceinline__ void diag(Ctl* c, int site, unsigned long long k = 1) {
  atomicAdd(&c->diag[site], k);
}

__device__ __forceinline__ RepRow rep_row(const double2* __restrict__ dl, const double2* __restrict__ ul, int64_t i) {
  const double2 a = dl[i], b = ul[i];
  return RepRow{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void rep_store(double2* dl, double2* ul, int64_t i, const RepRow& r) {
  dl[i] = make_double2(r.D, r.LLD);
  ul[i] = make_double2(r.l, r.LD);
}

// Zero-pivot guard of a representation whose entries are bounded by R (the
// problem is scaled so that G(T) is in [1,2)): pivots below pivmin are
// replaced by -pivmin.  pivmin = 2^-900 max(1, R)^2 keeps every quotient of
// the Sturm recurrence finite; as an exponent field for the integer test of
// the division-free count.
__device__ __forceinline__ double pivmin_for(double R) {
  double r = fmin(fmax(R, 1.0), 0x1p60);
  return 0x1p-900 * r * r;
}
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// ---------------------------------------------------------------------------
// Sturm count on a representation (Sec. 3.1.1: bisection on the RRR).  The
// number of negative pivots D+_i of the stationary transform
//   L+ D+ L+^T = L D L^T - tau I,
//   s_1 = -tau,  D+_i = D_i + s_i,  s_{i+1} = LLD_i s_i / D+_i - tau,
// equals the number of eigenvalues of L D L^T below tau (Sylvester's law of
// inertia).  Pivots with |D+_i| < pivmin are replaced by -pivmin.
//
// Division-free form used by the kernels: with s_i = a/b,
//   c = D_i b + a            (= D+_i b; sign(D+_i) = sign(c) sign(b))
//   a' = LLD_i a - tau c,  b' = c          (so s_{i+1} = a'/b')
// and (a', b') rescaled by the power of two that brings |b'| into [1,2)
// (integer operations on the exponent field; a' flushes to 0 below the
// normal range).  Three FP64 operations per row instead of a division; the
// rounding differs from the quotient form by a relative perturbation of tau
// of one ulp per row, i.e. a diagonal perturbation of size eps|tau| (so the
// count keeps the relative accuracy of the representation).
__device__ __forceinline__ void count_step(double D, double LLD, double tau, int pivexp, double pivmin,
                                           double& a, double& b, int& neg) {
  double c = fma(D, b, a);
  int chi = __double2hiint(c);
  const int bhi = __double2hiint(b);
  int cexp = (chi >> 20) & 0x7ff;
  if (cexp < pivexp) {  // |D+| < pivmin (|b| in [1,2)): counts as negative
    c = bhi < 0 ? pivmin : -pivmin;
    chi = __double2hiint(c);
    cexp = pivexp;
  }
  neg += (chi ^ bhi) < 0;
  const double an = fma(LLD, a, -tau * c);
  const int k = cexp - 1023;
  b = __hiloint2double((chi & 0x800fffff) | 0x3ff00000, __double2loint(c));
  const int ahi = __double2hiint(an);
  const int aexp = (ahi >> 20) & 0x7ff;
  a = (aexp - k <= 0) ? 0.0 : __hiloint2double(ahi - (k << 20), __double2loint(an));
}

__device__ __forceinline__ int negcount(const double2* __restrict__ dl, int m, double tau, double pivmin) {
  const int pivexp = exp_field(pivmin);
  double a = -tau, b = 1.0;
  int neg = 0;
  for (int i = 0; i < m; ++i) {
    const double2 r = dl[i];
    count_step(r.x, r.y, tau, pivexp, pivmin, a, b, neg);
  }
  return neg;
}

__device__ __forceinline__ bool converged(double lo, double hi, double rtol, double atol) {
  double w = hi - lo;
  return w <= fmax(rtol * fmax(fabs(lo), fabs(hi)), atol);
}

// Bisection of [lo, hi] (count(lo) <= j-1 < count(hi) on entry) until the
// width is below rtol relative (atol absolute).  Returns steps taken.
__device__ __forceinline__ int bisect_interval(const double2* __restrict__ dl, int m, int j, double pivmin,
                                               double rtol, double atol, int maxit, double& lo, double& hi) {
  int it = 0;
  for (; it < maxit; ++it) {
    if (converged(lo, hi, rtol, atol)) break;
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (negcount(dl, m, mid, pivmin) >= j)
      hi = mid;
    else
      lo = mid;
  }
  return it;
}

// ---------------------------------------------------------------------------
// Chunk scheduler of the persistent kernels (interval engine, eigenvectors).
// Each SM sub-partition's FP64 unit takes about 64 cycles per warp
// instruction whatever the number of active lanes, so a launch whose list has
// c chunks of one warp's work each should put them on c different
// sub-partitions (then on each a second one, ...).  The hardware places CTAs
// and warps as it likes (with two CTAs per SM, CTA b is not on SM b mod nsm),
// so each warp reads where it runs (%smid, %warpid mod 4), counts itself on
// that sub-partition (k-th warp there), and gets the rank
//   k * (4 nsmid) + 4 smid + subpartition,
// i.e. ranks 0 .. 4 nsmid - 1 are one warp on each sub-partition.  A warp
// first takes the chunk of its rank, then chunks past the number of warps
// from a counter, then sweeps the ranked chunks that no warp claimed (ranks
// of SMs that ran fewer warps).  Every chunk carries the generation of the
// launch that claimed it (atomic exchange), so each is done exactly once.
constexpr int kSchedSlots = 1024;  // sub-partition counters (4 per SM id)

__device__ __forceinline__ long long sched_rank(const Dev& v) {
  const int lane = threadIdx.x & 31;
  long long rank = 0;
  if (lane == 0) {
    unsigned smid, wid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    const unsigned slot = (smid * 4u + (wid & 3u)) % (unsigned)kSchedSlots;
    const int k = atomicAdd(&v.sched_cnt[slot], 1);
    rank = (long long)k * (4LL * (long long)nsmid) + (long long)slot;
  }
  return __shfl_sync(0xffffffffu, rank, 0);
}

__device__ __forceinline__ bool sched_claim(const Dev& v, long long c, int gen) {
  return atomicExch(&v.sched_claim[c], gen) != gen;
}

// Next chunk for this warp (warp-uniform), or -1 when none is left.
__device__ __forceinline__ long long sched_next(const Dev& v, long long nchunks, long long total_warps,
                                                long long rank, bool& first) {
  const int lane = threadIdx.x & 31;
  long long c = -1;
  if (lane == 0) {
    const int gen = v.ctl->sched_gen;
    if (first && rank < nchunks && sched_claim(v, rank, gen)) c = rank;
    const long long ranked = min(nchunks, total_warps);
    while (c < 0) {
      const long long d = total_warps + (long long)atomicAdd(&v.ctl->sched_dyn, 1ull);
      if (d < nchunks) {
        if (sched_claim(v, d, gen)) c = d;
        continue;
      }
      const long long r = (long long)atomicAdd(&v.ctl->sched_cleanup, 1ull);
      if (r >= ranked) break;
      if (sched_claim(v, r, gen)) c = r;
    }
  }
  first = false;
  return __shfl_sync(0xffffffffu, c, 0);
}

// Candidate representation rows in the eigenvector scratch, which is idle
// while the root representations and the tree are built: two planes of
// double2 (the pool's layout), each half of the scratch.
__device__ __forceinline__ int64_t cand_capacity(const Dev& v) {
  return (int64_t)((size_t)v.vscr_threads * (size_t)v.vscr_rows * (v.vec_dd ? 4 : 2) / 4);
}
__device__ __forceinline__ double2* cand_dl(const Dev& v) { return reinterpret_cast<double2*>(v.vscr); }
__device__ __forceinline__ double2* cand_ul(const Dev& v) {
  return reinterpret_cast<double2*>(v.vscr) + cand_capacity(v);
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

// Before each scheduled launch (one CTA of kSchedSlots threads): counters to
// zero, a new generation for the claims.
__global__ void k_sched_reset(Dev v);
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

}  // namespace mrrr
