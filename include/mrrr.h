/*
 * mrrr.h -- C ABI of a single-GPU (NVIDIA GB300, sm_103a) FP64 MRRR solver
 * for the real symmetric tridiagonal eigenproblem  T z = lambda z.
 *
 * The method is the MRRR algorithm as summarised in Petschow, Peise and
 * Bientinesi, "High-performance solvers for dense Hermitian eigenproblems"
 * (arXiv:1205.2107), Sec. 3.1.1 "The MRRR algorithm": a root representation
 * L0 D0 L0^T = T - sigma I, bisection for eigenvalue approximations,
 * classification into singletons and clusters by relative gap (the paper's
 * tol is 1e-3; here max(gap_tol, 1/m), see mrrr_options.gap_tol),
 * child representations Lc Dc Lc^T = L0 D0 L0^T - sigma_c I for clusters,
 * recursion, and the vector of each singleton from a single solve with a
 * twisted factorization (Eq. errorangle).  The problem statement -- all or an
 * index subset il..iu of the eigenpairs -- is the paper's (Sec. 1.1,
 * Sec. 2.3, Sec. 5).  The accuracy goals are Eqs. Tresnorm / Torthogo
 * (Sec. 2.3).  Batched solves and the backward (adjoint) pass are not in the
 * paper; they reuse the same representation of the problem.
 *
 * Conventions for every entry point:
 *   - all array arguments are DEVICE pointers unless stated otherwise;
 *   - the caller owns every buffer: inputs, outputs and the workspace; the
 *     library never allocates device memory on the solve path;
 *   - work is enqueued on the given stream; most calls return before the GPU
 *     has finished (see each call);
 *   - no exception crosses the ABI; each call returns an mrrr_status.  Errors
 *     that only the GPU can detect (non-finite input, non-convergence, a full
 *     node pool) are recorded in a device status word that mrrr_get_status()
 *     returns;
 *   - indices il, iu are 1-based and inclusive over the whole T (across split
 *     blocks); W comes out ascending and Z column-major, column j belonging
 *     to W[j]; the sign of each column makes its twist entry positive.
 */
#ifndef MRRR_H
#define MRRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef void* mrrr_stream;

typedef enum mrrr_status {
  MRRR_OK = 0,
  MRRR_ERR_ARG = 1,        /* invalid argument (size, range, null pointer) */
  MRRR_ERR_WORKSPACE = 2,  /* workspace missing or smaller than required   */
  MRRR_ERR_NONFINITE = 3,  /* d or e holds NaN or Inf (found on the GPU)   */
  MRRR_ERR_NOCONV = 4,     /* an iteration hit its cap (bisection)         */
  MRRR_ERR_QUEUE = 5,      /* cluster-node table or representation pool full */
  MRRR_ERR_TIMEOUT = 6,    /* reserved (bounded device waits); no kernel of
                              this version waits on another                */
  MRRR_ERR_CUDA = 7,       /* a CUDA runtime call failed                   */
  MRRR_ERR_NOTIMPL = 8,    /* option combination not implemented           */
  MRRR_ERR_MARGIN = 9,     /* mrrr_stein_slice: a cluster reaching into the slice
                              extends past the margin (call again with a larger one) */
  MRRR_ERR_NOTSPD = 10     /* Cholesky factorization: the matrix is not positive
                              definite (a pivot is not positive) */
} mrrr_status;

/* Tunables.  Zero-initialise and call mrrr_options_default(); fields left at
   0 keep their defaults. */
typedef struct mrrr_options {
  double gap_tol;          /* floor of the singleton threshold on the relative gap:
                              a block of order m uses tol = max(gap_tol, 1/m)
                              (default 1e-4; 1e-3 is the paper's value, Sec. 3.1.1) */
  double classify_rtol;    /* relative interval width reached by bisection before
                              classification (2^-20) */
  int max_depth;           /* cluster-tree depth limit (64); deeper clusters take the
                              documented fallback and are counted in mrrr_info */
  int max_bisect_steps;    /* per interval and pass (256) */
  int engine_blocks_per_sm; /* 256-thread CTAs per SM of the interval engine (2; 1 or 2) */
  int threads_per_block;   /* CUDA block size of the interval kernels (128) */
  int vec_blocks_per_sm;   /* 128-thread blocks per SM of the eigenvector kernel (4, what
                              its registers allow to be resident at once);
                              capped by the number of eigenpairs */
  int use_graph;           /* 1: the solve is captured once per call signature into a CUDA
                              graph and replayed: setup, then the cluster levels in a
                              conditional while node that runs one more level for as long as
                              the last one made new clusters (decided on the device, no host
                              synchronisation), then the vectors; 0: launched directly, the
                              host reads the new-cluster count after each level (default) */
  int64_t max_nodes;       /* capacity of the cluster-node table (0 = automatic) */
  int64_t pool_rows;       /* capacity of the child-representation pool in rows of
                              32 bytes (0 = automatic) */
  double cluster_rtol;     /* relative interval width of cluster eigenvalues before a
                              child shift is placed, and of their refinement in the
                              child (2^-40) */
  double root_perturb;     /* relative size, in units of eps, of the seeded random
                              perturbation of each root representation entry (64,
                              at most m/8 for a block of order m; negative = none) */
  double width_scale;      /* scales the resident lanes when the engine chooses its
                              multisection width (1.0; larger = more points per interval) */
  double prebisect_rtol;   /* relative width to which root intervals are first bisected
                              on an FP32 copy of the root rows (2^-17); FP64 then confirms
                              each bracket, widened by 4x this relative, before bisecting
                              to classify_rtol.  Smaller moves halvings from the FP64 pipe
                              to the FP32 one (at most 2^-20; never below classify_rtol) */
  int multisection_width;  /* 0: the engine picks the points per interval from the length of
                              its work list, and consecutive eigenvalues of one node whose
                              brackets coincide pool their points (default); 1..32 (a power
                              of two): that many points per interval, no pooling -- a fixed
                              schedule, under which an eigenpair comes out bit for bit the
                              same whatever else the solve or the batch holds */
  int root_side;           /* side of the spectrum where the root shift sits: 0 the
                              Gershgorin end nearer the wanted indices (default), 1 the left
                              end, 2 the right end (slices of one index range that must share
                              one root representation) */
  int vector_precision;    /* arithmetic of the eigenvector stage: 1 FP64 (default); 2
                              double-double (about 106 bits) -- each singleton's eigenvalue
                              is corrected once by the Rayleigh quotient of a double-double
                              twisted factorization on its representation, then its vector
                              is solved at the corrected value, also in double-double, and
                              rounded to FP64: vectors taken from one representation are
                              then eigenvectors of one matrix to about eps^2 / relgap, so
                              orthogonality improves (Sec. 2.3, higher internal precision);
                              several times the FP64 stage's time */
  int singleton_rq;        /* Rayleigh-quotient correction of singletons (Sec. 3.1.1: the
                              vector stage may improve an eigenvalue): k = 1..4 (default 1)
                              bisects each singleton to 2^-36 relative only, then takes
                              up to k + 1 twisted factorizations (at least two), each
                              moving lambda by the Rayleigh quotient gamma_r / ||z||^2 of
                              the last (kept inside the bisection bracket), stopping
                              early once the corrections of a warp's vectors are all
                              below 2 eps |lambda|; the vector is the last one's and
                              lambda its Rayleigh quotient.  -1: no correction, every
                              singleton bisected to full relative accuracy (2 eps) and one
                              twisted factorization.  Ignored with vector_precision 2
                              (which bisects fully and corrects in double-double) and by
                              mrrr_stein_slice (full bisection: a slice's vector stage is
                              bound by the latency of each factorization) */
  int reserved_[4];        /* zero */
} mrrr_options;

/* Counters reported by mrrr_get_status (device values after the last solve). */
typedef struct mrrr_info {
  int status;              /* device status word (an mrrr_status)           */
  int depth;               /* deepest cluster level reached                 */
  int64_t nodes;           /* cluster nodes created (roots excluded)        */
  int64_t pool_rows_used;  /* child-representation rows needed              */
  int64_t fallbacks;       /* eigenvalues whose vectors were taken at a parent
                              node (depth limit or full node table/pool)    */
  int64_t twisted_solves;  /* twisted factorizations solved, all vectors    */
  int64_t levels;          /* cluster levels processed                      */
  int64_t diag[12];        /* event counters: [0] root-shift retries exhausted,
                              [1] root bisection cap, [2] child bracket not
                              confirmed, [3] child bisection cap, [4] clusters
                              whose first wave of child shifts all failed,
                              [5] child growth bound missed, [6] depth-limit
                              fallbacks, [7] capacity fallbacks, [8] runs of
                              neighbouring eigenvectors re-orthogonalised,
                              [9] child transforms computed again with stores,
                              [10]-[11] unused */
  int64_t sturm_counts[4]; /* interval engine per mode (0 root bisection, 1 cluster ends in
                              the parent, 2 cluster members in the child, 3 singletons to
                              full accuracy): Sturm counts evaluated */
  int64_t sturm_rows[4];   /* rows those counts ran over */
  int64_t warp_passes[4];  /* warp-wide passes over the rows (a pass costs its FP64
                              instructions however many of the 32 lanes count) */
} mrrr_info;

typedef struct mrrr_plan mrrr_plan;

/* Fill *opt with the defaults above.  Never fails for a non-NULL opt. */
mrrr_status mrrr_options_default(mrrr_options* opt);

/* Create a plan on the current CUDA device.  opt may be NULL (defaults).
   The plan owns a small pinned host buffer and its CUDA graphs; it is not
   thread-safe: use one plan per host thread.  Options out of range
   (multisection_width not 0 or a power of two <= 32, root_side outside 0..2,
   vector_precision outside 0..2, singleton_rq outside -1..4, gap_tol >= 1,
   classify_rtol, cluster_rtol or prebisect_rtol >= 1/4, threads_per_block not
   a multiple of 32, a non-finite root_perturb or width_scale) give
   MRRR_ERR_ARG before any CUDA call, with *plan set to NULL (as on every
   failure). */
mrrr_status mrrr_plan_create(mrrr_plan** plan, const mrrr_options* opt);
mrrr_status mrrr_plan_destroy(mrrr_plan* plan);

/* Bytes of device workspace a solve needs.  batch problems whose sizes sum
   to n_total, largest n_max, requesting k_total eigenpairs in all.  The
   figure holds the automatic node and pool capacities unless the options
   set them.  Host-only; never fails for valid sizes. */
mrrr_status mrrr_workspace_size(const mrrr_plan* plan, int batch, int64_t n_total, int64_t k_total,
                                int n_max, size_t* bytes);

/*
 * mrrr_stein: eigenpairs il..iu of one symmetric tridiagonal T (paper
 * Sec. 3.1.1; subset at O(nk) cost, Sec. 2.3).
 *   n          order of T (n >= 0; n = 0 is a no-op)
 *   d, e       device, d[n] diagonal, e[n-1] off-diagonal (read only)
 *   il, iu     1-based inclusive range, 1 <= il <= iu <= n
 *   W          device, W[iu-il+1] eigenvalues, ascending
 *   Z          device, column-major n x (iu-il+1) with leading dimension
 *              ldz >= n; may be NULL for eigenvalues only
 *   workspace  device, ws_bytes >= mrrr_workspace_size(plan, 1, n, k, n)
 *   stream     CUDA stream for every launch
 * Returns MRRR_ERR_ARG / MRRR_ERR_WORKSPACE for bad host-side arguments.
 * Without use_graph the call synchronises the stream once per cluster
 * level; with use_graph it enqueues one graph launch (capturing it first for
 * a new call signature).  Device-side errors are read with mrrr_get_status.
 */
mrrr_status mrrr_stein(mrrr_plan* plan, int n, const double* d, const double* e, int il, int iu,
                       double* W, double* Z, int64_t ldz, void* workspace, size_t ws_bytes,
                       mrrr_stream stream);

/*
 * mrrr_slice_range: the index range a..b (1-based, inclusive) of slice
 * `slice` (0-based) when il..iu is cut into nslices equal contiguous slices:
 * a = il + floor(slice k / nslices), b = il + floor((slice+1) k / nslices) - 1
 * with k = iu - il + 1 (the paper's static division of the eigenpairs among
 * processes, Sec. 3.1.2).  Host only.  MRRR_ERR_ARG for an empty range, a
 * slice out of range or more slices than indices.
 */
mrrr_status mrrr_slice_range(int il, int iu, int nslices, int slice, int* a, int* b);

/*
 * mrrr_stein_slice: the eigenpairs of slice `slice` of nslices equal slices
 * of il..iu (mrrr_slice_range), computed so that the slices, each on its own
 * GPU or one after the other, together give the solution of il..iu: their
 * columns are mutually orthogonal as those of one solve are.  The paper's
 * PMRRR divides the wanted eigenpairs statically among processes, computes
 * the root representation redundantly in each, and lets processes that hold
 * members of one cluster cooperate on it (Sec. 3.1.2).  Here each slice
 * computes its indices plus `margin` more on each side (the root
 * representation redundantly, its shift on the side that il..iu as a whole
 * chooses), and a cluster that reaches across a slice boundary is computed
 * whole, identically, by both slices, each returning its own columns: no
 * data moves between slices.  For that every eigenpair must come out the
 * same whichever slice computes it, so a slice call uses a fixed schedule
 * (the plan's multisection_width, 4 when it is 0), and skips the neighbour
 * orthogonality safeguard.
 *   il, iu, nslices, slice   as in mrrr_slice_range
 *   margin     indices computed beyond each end of the slice (>= 1); when a
 *              cluster holding returned indices reaches past it the device
 *              status is MRRR_ERR_MARGIN: call again with a larger margin
 *   W, Z       device, W[b-a+1] and an n x (b-a+1) column-major Z (ldz >= n)
 *              for the slice's indices a..b (Z may be NULL)
 *   workspace  ws_bytes >= mrrr_workspace_size(plan, 1, n,
 *              min(n, b+margin) - max(1, a-margin) + 1, n)
 * W is ascending within a slice; across a slice boundary, eigenvalues equal
 * to the last bit may come out one ulp apart in either order.  Other
 * arguments, errors and synchronisation as in mrrr_stein.
 */
mrrr_status mrrr_stein_slice(mrrr_plan* plan, int n, const double* d, const double* e, int il, int iu, int nslices,
                             int slice, int margin, double* W, double* Z, int64_t ldz, void* workspace,
                             size_t ws_bytes, mrrr_stream stream);

/*
 * mrrr_stein_batched: many independent problems in one set of launches.
 *   batch      number of problems
 *   d_off      device int64[batch+1]; problem p owns rows d_off[p]..d_off[p+1]-1
 *   d, e       device packed arrays of d_off[batch] doubles; e uses the same
 *              offsets (the last entry of each problem is ignored)
 *   il, iu     device int32[batch] or NULL (NULL = all eigenpairs)
 *   W, w_off   device; problem p writes W[w_off[p] .. w_off[p]+k_p-1]
 *   Z, z_off   device (Z may be NULL); problem p writes an n_p x k_p
 *              column-major block at Z + z_off[p] with leading dimension n_p
 *   n_max      largest n_p; k_total = sum of k_p (workspace sizing)
 * Argument ranges inside the device arrays are checked on the GPU
 * (MRRR_ERR_ARG in the status word).  Not in the paper: every problem is
 * solved by the method of mrrr_stein (Sec. 3.1.1); the problems share the
 * launches, the work lists and the cluster levels.  Synchronisation as in
 * mrrr_stein (use_graph captures the whole batched solve).
 */
mrrr_status mrrr_stein_batched(mrrr_plan* plan, int batch, const int64_t* d_off, const double* d,
                               const double* e, const int* il, const int* iu, double* W,
                               const int64_t* w_off, double* Z, const int64_t* z_off, int64_t n_total,
                               int64_t k_total, int n_max, void* workspace, size_t ws_bytes,
                               mrrr_stream stream);

/*
 * mrrr_autotune_batched: choose the launch shape of the batched solver for
 * one batch layout by timing it.  Not in the paper (a scheduling aid for
 * the batched pattern).  Candidates: block shape (engine_blocks_per_sm in
 * {2, 1}) x threads per interval (width_scale, which scales the multisection
 * width and with it the bisection steps per pass, in {1, 0.5, 2}) x
 * bisection steps before the vectors (singleton_rq in {1, -1}: singletons to
 * 2^-36 then one Rayleigh-quotient correction, or to full accuracy; only the
 * plan's own setting with vector_precision 2): 12 candidates, each solving
 * the batch once (after one untimed warm-up solve) with CUDA events on
 * stream.  The fastest becomes the plan's setting (the plan's
 * CUDA graph, if any, is rebuilt on the next call).  Arguments as in
 * mrrr_stein_batched; on return W and Z hold a valid solution.  The call
 * synchronises the stream.  Device-side errors are returned.
 */
typedef struct mrrr_tuning {
  int engine_blocks_per_sm;  /* chosen */
  int configs;               /* candidates timed */
  double width_scale;        /* chosen */
  double best_ms;            /* time of the chosen candidate */
  double default_ms;         /* time of the first candidate (the defaults) */
  int singleton_rq;          /* chosen */
  int pad_;
} mrrr_tuning;

mrrr_status mrrr_autotune_batched(mrrr_plan* plan, int batch, const int64_t* d_off, const double* d,
                                  const double* e, const int* il, const int* iu, double* W,
                                  const int64_t* w_off, double* Z, const int64_t* z_off, int64_t n_total,
                                  int64_t k_total, int n_max, void* workspace, size_t ws_bytes,
                                  mrrr_stream stream, mrrr_tuning* out);

/*
 * mrrr_backward: gradient of a scalar loss L(W, Z) with respect to (d, e)
 * for a batch of problems solved for ALL eigenpairs, given Wbar = dL/dW and
 * Zbar = dL/dZ (either may be NULL).  Not in the paper: first-order
 * perturbation theory of T = Z diag(W) Z^T,
 *   Tbar = Z (diag(Wbar) + F o (Z^T Zbar)) Z^T,
 *   F(i,j) = 1/(W_j - W_i) if |W_j - W_i| > tau, else 0 (0 on the diagonal),
 *   tau = tau_rel * max|W| of the problem,
 *   dbar_j = Tbar(j,j),  ebar_j = Tbar(j,j+1) + Tbar(j+1,j),
 * so dbar_j = sum_i Wbar_i Z(j,i)^2 + ..., ebar_j = 2 sum_i Wbar_i Z(j,i)
 * Z(j+1,i) + ....  The two n^3 contractions run on the FP64 tensor cores.
 *   batch      0..65535 (each problem is one index of a grid dimension)
 *   d_off      device int64[batch+1] as in mrrr_stein_batched; W and Wbar
 *              use the same packing (n_p values of problem p at d_off[p])
 *   Z, Zbar    device; problem p's n_p x n_p column-major block starts at
 *              sum_{q<p} n_q^2 (the packing of mrrr_stein_batched for all
 *              eigenpairs); z_total = sum_p n_p^2
 *   tau_rel    >= 0, gap threshold of F relative to max|W|
 *   n_max      largest n_p (grid sizing)
 *   dbar, ebar device outputs with the packing of d and e (ebar's last entry
 *              of each problem is written as 0)
 *   workspace  device, ws_bytes >= mrrr_backward_workspace_size(...)
 * Deterministic (fixed reduction order).  Returns MRRR_ERR_ARG /
 * MRRR_ERR_WORKSPACE for bad host-side arguments, MRRR_ERR_CUDA when a launch
 * fails.
 */
mrrr_status mrrr_backward(mrrr_plan* plan, int batch, const int64_t* d_off, const double* W,
                          const double* Z, const double* Wbar, const double* Zbar, double tau_rel,
                          int n_max, int64_t z_total, double* dbar, double* ebar, void* workspace,
                          size_t ws_bytes, mrrr_stream stream);

/* Bytes of workspace mrrr_backward needs for batch problems with
   z_total = sum_p n_p^2. */
mrrr_status mrrr_backward_workspace_size(const mrrr_plan* plan, int batch, int64_t z_total, size_t* bytes);

/*
 * mrrr_eigenvalues_static: eigenvalues il..iu of one symmetric tridiagonal T
 * without allocating anything and without a caller workspace.  The paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc when
 * they need eigenvalues -- a process whose device memory is already reserved
 * by another allocator (a framework's caching allocator), or a
 * latency-sensitive loop that cannot afford cudaFree's device-wide
 * synchronisation.
 *   n          order of T, 0 <= n <= MRRR_STATIC_MAX_N (n = 0 is a no-op);
 *              larger n returns MRRR_ERR_ARG before any GPU work
 *   d, e       device, d[n] diagonal, e[n-1] off-diagonal (read only)
 *   il, iu     1-based inclusive range, 1 <= il <= iu <= n
 *   W          device, W[iu-il+1] eigenvalues, ascending, each bisected to
 *              full accuracy on the root representation T - sigma I = L D L^T
 *   stream     CUDA stream of the two launches; the call returns before the
 *              GPU has finished
 * Scratch is one array of (32 + 2 * MRRR_STATIC_MAX_N) doubles (about
 * 128 KiB) in the library's static device memory, which each GPU that loads
 * the library holds until the process exits.  Every call on a device uses
 * the same array and leaves its contents behind; each call rewrites all it
 * later reads (header and status word first), so no state carries over.
 * Calls whose work overlaps on the GPU (different streams, or different host
 * threads, on the same device) race on the array and give wrong results:
 * serialise them.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it for
 * the life of the process; make that first call before any stream capture.
 * The cached address belongs to the device's primary context: after
 * cudaDeviceReset on a device, this entry point must not be called on that
 * device again in the same process.  The root representation is built by
 * one thread (a sequential recurrence over n rows), the bisection by one
 * thread per eigenvalue.  Device-side errors
 * (non-finite input, no definite root shift) give NaN eigenvalues.  Returns
 * MRRR_ERR_ARG for bad host-side arguments and MRRR_ERR_CUDA when the
 * address lookup or a launch fails.
 */
#define MRRR_STATIC_MAX_N 8192
mrrr_status mrrr_eigenvalues_static(int n, const double* d, const double* e, int il, int iu, double* W,
                                    mrrr_stream stream);

/*
 * The dense symmetric eigenproblem A y = lambda y around the tridiagonal
 * solver: the paper's stages 3-5 (Sec. 1.2; its Fig. of the six stages):
 * reduction to tridiagonal form A = Q T Q^T by Householder reflectors
 * (stage 3, mrrr_sytrd), the tridiagonal eigenpairs T z = lambda z
 * (stage 4, mrrr_stein), and the backtransformation y = Q z (stage 5,
 * mrrr_ormtr); mrrr_dense_eigh runs the three.  Real symmetric, FP64,
 * column-major; the reflectors H_j = I - tau_j v_j v_j^T (v_j(j+1) = 1,
 * v_j(0:j) = 0) are kept below the subdiagonal of A, Q = H_0 ... H_{n-3}.
 * The reduction is blocked (panels of 32 columns; the trailing update and
 * the backtransformation run on the FP64 tensor cores); every reduction
 * sums in a fixed order, so results are deterministic.  Device-side errors
 * (a non-finite reflector) are read with mrrr_dense_status; those of the
 * tridiagonal solve with mrrr_get_status.
 */

/* Bytes of workspace for mrrr_sytrd, mrrr_ormtr (k columns) and
   mrrr_dense_eigh (k = iu - il + 1 eigenpairs) of order n. */
mrrr_status mrrr_dense_workspace_size(const mrrr_plan* plan, int n, int k, size_t* bytes);

/* Stage 3: T = Q^T A Q.  A: device, n x n, lda >= n, symmetric, its lower
   triangle read; on return the diagonal and subdiagonal of A are T's and
   the reflectors lie below the subdiagonal (the upper triangle is not
   referenced).  d[n], e[n-1], tau[n-2]: device outputs.  Asynchronous on
   stream. */
mrrr_status mrrr_sytrd(mrrr_plan* plan, int n, double* A, int64_t lda, double* d, double* e, double* tau,
                       void* workspace, size_t ws_bytes, mrrr_stream stream);

/* Stage 5: Y <- Q Y for Y (device, n x k, ldy >= n) with A and tau as
   mrrr_sytrd leaves them.  Asynchronous. */
mrrr_status mrrr_ormtr(mrrr_plan* plan, int n, int k, const double* A, int64_t lda, const double* tau, double* Y,
                       int64_t ldy, void* workspace, size_t ws_bytes, mrrr_stream stream);

/* Stages 3-5: eigenvalues il..iu (1-based, inclusive) of the symmetric A,
   ascending, into W[iu-il+1], and their eigenvectors into Y (n x (iu-il+1),
   ldy >= n; NULL for eigenvalues only).  A is overwritten as by
   mrrr_sytrd.  Synchronisation of the tridiagonal stage as in mrrr_stein. */
mrrr_status mrrr_dense_eigh(mrrr_plan* plan, int n, double* A, int64_t lda, int il, int iu, double* W, double* Y,
                            int64_t ldy, void* workspace, size_t ws_bytes, mrrr_stream stream);

/*
 * The generalized symmetric-definite eigenproblem A x = lambda B x (B
 * positive definite), the paper's six stages (Sec. 1.2): B = L L^T
 * (stage 1, mrrr_potrf), C = L^-1 A L^-T (stage 2, mrrr_sygst), the
 * eigenpairs of C (stages 3-5, mrrr_dense_eigh), X = L^-T Y (stage 6,
 * mrrr_trsm_lt); mrrr_gen_eigh runs them all.  Blocked by 64; diagonal
 * blocks are factored and inverted by one CTA each, the rest is FP64
 * tensor-core GEMM.  Real, FP64, column-major.
 */

/* Bytes of workspace for the calls below of order n with k eigenvectors. */
mrrr_status mrrr_gen_workspace_size(const mrrr_plan* plan, int n, int k, size_t* bytes);

/* Stage 1: B (device, n x n, ldb >= n; lower triangle read) <- its Cholesky
   factor L in the lower triangle (the upper triangle is left as it was).  A
   pivot that is not positive sets MRRR_ERR_NOTSPD in the device status word
   (mrrr_dense_status on this workspace).  Asynchronous. */
mrrr_status mrrr_potrf(mrrr_plan* plan, int n, double* B, int64_t ldb, void* workspace, size_t ws_bytes,
                       mrrr_stream stream);

/* Stage 2: A (device, n x n, both triangles of the symmetric A) <-
   L^-1 A L^-T, both triangles, with L the lower triangle of L (ldl >= n).
   Asynchronous. */
mrrr_status mrrr_sygst(mrrr_plan* plan, int n, double* A, int64_t lda, const double* L, int64_t ldl,
                       void* workspace, size_t ws_bytes, mrrr_stream stream);

/* Stage 6: X (device, n x k, ldx >= n) <- L^-T X.  Asynchronous. */
mrrr_status mrrr_trsm_lt(mrrr_plan* plan, int n, int k, const double* L, int64_t ldl, double* X, int64_t ldx,
                         void* workspace, size_t ws_bytes, mrrr_stream stream);

/* All six stages: eigenvalues il..iu of the pencil (A, B), ascending, into
   W[iu-il+1], and their B-orthonormal eigenvectors (X^T B X = I) into X
   (n x (iu-il+1), ldx >= n; NULL for eigenvalues only).  A (both
   triangles) and B (lower triangle) are overwritten.  Device-side errors
   of the dense stages: mrrr_gen_status; of the tridiagonal stage:
   mrrr_get_status. */
mrrr_status mrrr_gen_eigh(mrrr_plan* plan, int n, double* A, int64_t lda, double* B, int64_t ldb, int il, int iu,
                          double* W, double* X, int64_t ldx, void* workspace, size_t ws_bytes, mrrr_stream stream);

/* Synchronise stream and return the first device-side error of the last
   mrrr_gen_eigh (order n, k eigenpairs) on this workspace: MRRR_ERR_NOTSPD
   from the Cholesky factorization, MRRR_ERR_NONFINITE from the reduction. */
mrrr_status mrrr_gen_status(const mrrr_plan* plan, int n, int k, const void* workspace, mrrr_stream stream);

/* Synchronise stream and return the device status word of the last dense
   call on this workspace (MRRR_ERR_NONFINITE for a non-finite reflector,
   MRRR_ERR_NOTSPD from the Cholesky factorization). */
mrrr_status mrrr_dense_status(const void* workspace, mrrr_stream stream);

/* Stage profile of the last solve on a plan.  launches counts the kernels
   the solve ran.  Direct launches: when timing is enabled (mrrr_set_timing)
   the solve records CUDA events (a pool created once per plan) between its
   stages on its stream and ms[i] holds the time of stage name[i] summed over
   cluster levels.  Graph replays (use_graph): one-thread kernels at the
   stage boundaries accumulate the GPU global timer's advance per stage in
   the workspace, read back here (synchronise the stream first).  Not in the
   paper: measurement support. */
typedef struct mrrr_profile {
  int64_t launches;
  int nstages;
  int pad_;
  char name[32][24];
  double ms[32];
} mrrr_profile;

/* Enable (1) or disable (0) per-stage event timing on a plan.  Timing adds
   one event record per stage and a final event synchronisation. */
mrrr_status mrrr_set_timing(mrrr_plan* plan, int enable);

/* Copy the profile of the last solve on the plan into *out. */
mrrr_status mrrr_get_profile(const mrrr_plan* plan, mrrr_profile* out);

/* Measured peak rate of one arithmetic unit of the current GPU, the
   denominator of the solver's roofline figures.  Not in the paper:
   measurement support.  kind 0: FP64 FMA (flop/s, 2 per FMA), 1: FP64 tensor
   core MMA m8n8k4 (flop/s), 2: FP64 division (divisions/s), 3: FP32 FMA
   (flop/s), 4: FP64 FMA warp instructions per second with one active lane
   per warp.  Times throughput kernels on every SM with CUDA events on a
   stream of its own (best of three, about 0.1-0.2 s in all) and
   synchronises.  kind 5 / 6: SM clock cycles of one dependent FP64 FMA /
   of one dependent FP64 division plus add, one warp alone on the GPU
   (clock64 around a chain; the legacy stream, synchronous).  Returns MRRR_ERR_ARG for a bad kind or NULL rate,
   MRRR_ERR_CUDA when a launch fails. */
mrrr_status mrrr_probe_peak(int kind, double* rate);

/* Synchronise stream and report the device status word and counters of the
   last solve on this plan.  out may be NULL.  Returns info.status. */
mrrr_status mrrr_get_status(mrrr_plan* plan, mrrr_stream stream, mrrr_info* out);

/* Static English text for a status code. */
const char* mrrr_status_string(mrrr_status s);

/* Library version as major*10000 + minor*100 + patch. */
int mrrr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MRRR_H */
