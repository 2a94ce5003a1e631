/*
 * oracle.c -- plain, slow CPU reference for the real symmetric tridiagonal
 * eigenproblem (STEP) T z = lambda z, in IEEE double precision.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU solver is
 * checked against.  Nothing in the product path may link or call it; only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header or constant table with the CUDA library.
 *
 * What it computes and where the paper defines it (Petschow, Peise,
 * Bientinesi, "High-performance solvers for dense Hermitian eigenproblems"):
 *   - the problem: all or a subset il..iu of the eigenpairs of a symmetric
 *     tridiagonal T, eigenvalues ascending (Sec. 1.1, Sec. 2.3 "The
 *     Tridiagonal Eigenproblem", Sec. 5 Conclusions);
 *   - splitting: off-diagonals below eps*||T|| are treated as zero, which
 *     decouples T into independent blocks (Sec. 3.1.1, footnote on numerical
 *     irreducibility); ||T|| is taken as the Gershgorin bound
 *     G(T) = max_i (|d_i| + |e_{i-1}| + |e_i|);
 *   - eigenvalues: bisection with Sturm counts on T itself (Sec. 3.1.1 names
 *     bisection; Sec. 2.1 names the bisection + inverse iteration solver);
 *   - eigenvectors: classical inverse iteration (T - lambda I) z' = s z
 *     (Sec. 3.1, the inverse-iteration equation) with modified Gram-Schmidt
 *     re-orthogonalisation inside clusters, clusters being runs of one
 *     block's eigenvalues closer than orfac*||T_b||, orfac = 1e-3 by default
 *     (Sec. 2.1, footnote on the orfac parameter).  This is the paper's "BI"
 *     method: slow but simple and independent of MRRR;
 *   - a dense cyclic Jacobi solver for small n (brute force, used to pin the
 *     two methods above).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - zero pivots in the Sturm recurrence: |q_i| < pivmin is replaced by
 *     -pivmin, pivmin = safmin * max(1, max_i e_i^2) (Kahan's rule);
 *   - bisection stops when the midpoint equals an endpoint in floating point
 *     or the width is at most 2 eps max(|lo|,|hi|);
 *   - ties between equal eigenvalues of different blocks are ordered by block;
 *   - inverse iteration is done block by block with the block's own norm
 *     ||T_b|| = max |eigenvalue of T_b| (reorthogonalisation threshold,
 *     zero-pivot perturbation eps*||T_b||, growth test), on the block scaled
 *     by the power of two that brings ||T_b|| into [1, 2);
 *   - inverse-iteration start vectors come from a splitmix64 stream seeded by
 *     the eigenvalue's position, so results are deterministic.
 *
 * Built with -ffp-contract=off so that x86 and Arm hosts round identically.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_EPS (0x1p-53)
#define ORACLE_SAFMIN (0x1p-1022)

/* ------------------------------------------------------------------------ */
/* A tiny parallel-for over [0, count) with dynamic chunks.                 */

typedef void (*task_fn)(void* ctx, int64_t item);

typedef struct {
  task_fn fn;
  void* ctx;
  int64_t count;
  int64_t chunk;
  int64_t next; /* updated with __atomic builtins */
} pfor_t;

static void* pfor_worker(void* arg) {
  pfor_t* p = (pfor_t*)arg;
  for (;;) {
    int64_t start = __atomic_fetch_add(&p->next, p->chunk, __ATOMIC_RELAXED);
    if (start >= p->count) break;
    int64_t stop = start + p->chunk < p->count ? start + p->chunk : p->count;
    for (int64_t i = start; i < stop; ++i) p->fn(p->ctx, i);
  }
  return NULL;
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void parallel_for(int nthreads, int64_t count, int64_t chunk, task_fn fn, void* ctx) {
  pfor_t p = {fn, ctx, count, chunk > 0 ? chunk : 1, 0};
  int t = resolve_threads(nthreads);
  if (t > 256) t = 256;
  if (t <= 1 || count <= 1) {
    pfor_worker(&p);
    return;
  }
  pthread_t th[256];
  int started = 0;
  for (int i = 0; i < t - 1; ++i)
    if (pthread_create(&th[i], NULL, pfor_worker, &p) == 0) ++started;
  pfor_worker(&p);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

int oracle_num_threads(int nthreads) { return resolve_threads(nthreads); }

/* ------------------------------------------------------------------------ */
/* Splitting (Sec. 3.1.1 footnote: off-diagonals below eps*||T|| are zero). */

double oracle_gershgorin_norm(int n, const double* d, const double* e) {
  double g = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = fabs(d[i]);
    if (i > 0) r += fabs(e[i - 1]);
    if (i + 1 < n) r += fabs(e[i]);
    if (r > g) g = r;
  }
  return g;
}

/* Writes the split off-diagonal (zeros where T splits) into es[n-1] and the
   block start rows into starts[0..nb]; returns nb. */
int oracle_split(int n, const double* d, const double* e, double* es, int* starts) {
  double thresh = ORACLE_EPS * oracle_gershgorin_norm(n, d, e);
  int nb = 0;
  if (n <= 0) {
    starts[0] = 0;
    return 0;
  }
  starts[nb++] = 0;
  for (int i = 0; i + 1 < n; ++i) {
    if (fabs(e[i]) <= thresh) {
      es[i] = 0.0;
      starts[nb++] = i + 1;
    } else {
      es[i] = e[i];
    }
  }
  starts[nb] = n;
  return nb;
}

/* ------------------------------------------------------------------------ */
/* Sturm count on a block of T: number of eigenvalues strictly below x.     */
/* q_1 = d_1 - x,  q_i = d_i - x - e_{i-1}^2 / q_{i-1};  count = #{q_i < 0}. */

static int sturm_count_block(int m, const double* d, const double* e2, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

typedef struct {
  int m;
  const double* d;
  double* e2; /* owned, m-1 entries (squares of the split off-diagonal) */
  double pivmin;
  double gl, gu; /* bracket with count(gl) = 0, count(gu) = m */
} block_t;

static void block_init(block_t* b, int m, const double* d, const double* es) {
  b->m = m;
  b->d = d;
  b->e2 = (double*)malloc(sizeof(double) * (m > 1 ? m - 1 : 1));
  double emax2 = 0.0;
  for (int i = 0; i + 1 < m; ++i) {
    b->e2[i] = es[i] * es[i];
    if (b->e2[i] > emax2) emax2 = b->e2[i];
  }
  b->pivmin = ORACLE_SAFMIN * (emax2 > 1.0 ? emax2 : 1.0);
  double gl = INFINITY, gu = -INFINITY;
  for (int i = 0; i < m; ++i) {
    double r = 0.0;
    if (i > 0) r += fabs(es[i - 1]);
    if (i + 1 < m) r += fabs(es[i]);
    if (d[i] - r < gl) gl = d[i] - r;
    if (d[i] + r > gu) gu = d[i] + r;
  }
  double w = (gu - gl) + fabs(gl) + fabs(gu) + 1.0;
  double pad = 4.0 * ORACLE_EPS * m * w + 2.0 * b->pivmin;
  gl -= pad;
  gu += pad;
  /* The Gershgorin bracket must hold in floating point; widen until it does
     (bounded). */
  for (int t = 0; t < 64 && sturm_count_block(m, d, b->e2, gl, b->pivmin) > 0; ++t) gl -= (gu - gl);
  for (int t = 0; t < 64 && sturm_count_block(m, d, b->e2, gu, b->pivmin) < m; ++t) gu += (gu - gl);
  b->gl = gl;
  b->gu = gu;
}

static void block_free(block_t* b) { free(b->e2); }

/* k-th smallest eigenvalue (1-based) of the block by bisection. */
static double block_bisect(const block_t* b, int k) {
  if (b->m == 1) return b->d[0]; /* a 1x1 block is its own eigenvalue */
  double lo = b->gl, hi = b->gu;
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= 2.0 * ORACLE_EPS * fmax(fabs(lo), fabs(hi))) break;
    if (sturm_count_block(b->m, b->d, b->e2, mid, b->pivmin) >= k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* Public: number of eigenvalues of the split T strictly below x. */
int oracle_sturm_count(int n, const double* d, const double* e, double x) {
  if (n <= 0) return 0;
  double* es = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  int* starts = (int*)malloc(sizeof(int) * (n + 1));
  int nb = oracle_split(n, d, e, es, starts);
  int total = 0;
  for (int b = 0; b < nb; ++b) {
    block_t blk;
    int s = starts[b], m = starts[b + 1] - starts[b];
    block_init(&blk, m, d + s, es + s);
    total += sturm_count_block(m, d + s, blk.e2, x, blk.pivmin);
    block_free(&blk);
  }
  free(es);
  free(starts);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Eigenvalues of all blocks, merged in ascending order.                    */

typedef struct {
  double value;
  int block;
  int local; /* 1-based index within the block */
} eig_t;

typedef struct {
  const block_t* blocks;
  const int* starts;
  const int64_t* item_block; /* item -> block */
  const int64_t* item_local; /* item -> 1-based local index */
  eig_t* out;
} bisect_ctx;

static void bisect_task(void* vctx, int64_t item) {
  bisect_ctx* c = (bisect_ctx*)vctx;
  int b = (int)c->item_block[item];
  int k = (int)c->item_local[item];
  c->out[item].value = block_bisect(&c->blocks[b], k);
  c->out[item].block = b;
  c->out[item].local = k;
}

/* a selected eigenvalue by (block, index within the block), for clustering */
typedef struct {
  int block;
  int local;
  int64_t pos; /* output position */
} member_t;

static int member_cmp(const void* pa, const void* pb) {
  const member_t* a = (const member_t*)pa;
  const member_t* b = (const member_t*)pb;
  if (a->block != b->block) return a->block < b->block ? -1 : 1;
  return a->local < b->local ? -1 : (a->local > b->local);
}

static int eig_cmp(const void* pa, const void* pb) {
  const eig_t* a = (const eig_t*)pa;
  const eig_t* b = (const eig_t*)pb;
  if (a->value < b->value) return -1;
  if (a->value > b->value) return 1;
  if (a->block != b->block) return a->block < b->block ? -1 : 1;
  return a->local < b->local ? -1 : (a->local > b->local);
}

/* ------------------------------------------------------------------------ */
/* Inverse iteration on a block: (T_b - mu I) y = x by Gaussian elimination */
/* with partial pivoting (textbook banded LU: U gets two superdiagonals).   */

typedef struct {
  int m;
  double *u0, *u1, *u2, *mult;
  unsigned char* swap;
} lu_t;

static void lu_alloc(lu_t* f, int m) {
  f->m = m;
  f->u0 = (double*)malloc(sizeof(double) * m);
  f->u1 = (double*)malloc(sizeof(double) * m);
  f->u2 = (double*)malloc(sizeof(double) * m);
  f->mult = (double*)malloc(sizeof(double) * m);
  f->swap = (unsigned char*)malloc(m);
}

static void lu_free(lu_t* f) {
  free(f->u0);
  free(f->u1);
  free(f->u2);
  free(f->mult);
  free(f->swap);
}

/* Factor A = T_b - mu I.  Zero pivots are replaced by tiny (perturbation of
   the shift, as classical inverse iteration does). */
static void lu_factor(lu_t* f, const double* d, const double* es, double mu, double tiny) {
  int m = f->m;
  double w0 = d[0] - mu;            /* working row, column k   */
  double w1 = m > 1 ? es[0] : 0.0;  /* working row, column k+1 */
  for (int k = 0; k + 1 < m; ++k) {
    double c = es[k];                /* row k+1, column k   */
    double a1 = d[k + 1] - mu;       /* row k+1, column k+1 */
    double b1 = (k + 2 < m) ? es[k + 1] : 0.0; /* row k+1, column k+2 */
    if (fabs(w0) >= fabs(c)) {
      double mk = (w0 != 0.0) ? c / w0 : 0.0;
      if (w0 == 0.0) w0 = tiny;
      f->u0[k] = w0;
      f->u1[k] = w1;
      f->u2[k] = 0.0;
      f->mult[k] = mk;
      f->swap[k] = 0;
      w0 = a1 - mk * w1;
      w1 = b1;
    } else {
      double mk = w0 / c;
      f->u0[k] = c;
      f->u1[k] = a1;
      f->u2[k] = b1;
      f->mult[k] = mk;
      f->swap[k] = 1;
      double nw0 = w1 - mk * a1;
      double nw1 = -mk * b1;
      w0 = nw0;
      w1 = nw1;
    }
  }
  if (w0 == 0.0) w0 = tiny;
  f->u0[m - 1] = w0;
  f->u1[m - 1] = 0.0;
  f->u2[m - 1] = 0.0;
}

/* Solve in place: x <- A^{-1} x (with the row operations of the factor). */
static void lu_solve(const lu_t* f, double* x) {
  int m = f->m;
  for (int k = 0; k + 1 < m; ++k) {
    if (f->swap[k]) {
      double xk = x[k];
      x[k] = x[k + 1];
      x[k + 1] = xk - f->mult[k] * x[k + 1];
    } else {
      x[k + 1] -= f->mult[k] * x[k];
    }
  }
  /* rescale before an entry passes 2^400: the 2-norm squares the entries */
  const double big = 0x1p400;
  for (int k = m - 1; k >= 0; --k) {
    double v = x[k];
    if (k + 1 < m) v -= f->u1[k] * x[k + 1];
    if (k + 2 < m) v -= f->u2[k] * x[k + 2];
    v /= f->u0[k];
    x[k] = v;
    if (fabs(v) > big) { /* rescale to avoid overflow; direction unchanged */
      double s = 1.0 / fabs(v);
      for (int i = 0; i < m; ++i) x[i] *= s;
    }
  }
}

static double dot(int m, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int m, const double* a) { return sqrt(dot(m, a, a)); }

static uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Vectors of one cluster (consecutive eigenvalues mus[0..c) of one block):
   inverse iteration, each iterate re-orthogonalised (MGS, twice) against the
   cluster's earlier vectors.  Output columns vecs[j*m ...].  The block and
   the shifts are first scaled by the power of two that brings the block's
   norm tnorm into [1, 2): exact, leaves the vectors unchanged, and keeps the
   zero-pivot perturbation eps*||T_b|| and the iterates in the normal range
   for blocks of any magnitude. */
static void cluster_vectors(int m, const double* d_in, const double* es_in, int c, const double* mus,
                            double tnorm, uint64_t seed, double* vecs) {
  int kb = 0;
  if (tnorm > 0 && isfinite(tnorm)) {
    frexp(tnorm, &kb);
    kb = 1 - kb;
  }
  double* d = (double*)malloc(sizeof(double) * m);
  double* es = (double*)malloc(sizeof(double) * m);
  for (int i = 0; i < m; ++i) d[i] = ldexp(d_in[i], kb);
  for (int i = 0; i + 1 < m; ++i) es[i] = ldexp(es_in[i], kb);
  tnorm = ldexp(tnorm, kb);
  lu_t f;
  lu_alloc(&f, m);
  double* x = (double*)malloc(sizeof(double) * m);
  double tiny = ORACLE_EPS * (tnorm > 0 ? tnorm : 1.0);
  double prev_mu = -INFINITY;
  for (int j = 0; j < c; ++j) {
    double mu = ldexp(mus[j], kb);
    /* nearly equal shifts are pulled apart so each LU differs */
    double sep = 10.0 * ORACLE_EPS * fmax(fabs(mu), tiny);
    if (mu - prev_mu < sep) mu = prev_mu + sep;
    prev_mu = mu;
    lu_factor(&f, d, es, mu, tiny);
    uint64_t st = seed + 0x1000003ull * (uint64_t)j;
    for (int i = 0; i < m; ++i) x[i] = (double)(splitmix64(&st) >> 11) * 0x1p-53 * 2.0 - 1.0;
    double growth_target = 1.0 / (10.0 * m * ORACLE_EPS * (tnorm > 0 ? tnorm : 1.0));
    int extra = -1;
    for (int it = 0; it < 8; ++it) {
      double nx = nrm2(m, x);
      if (nx == 0.0) x[it % m] = 1.0, nx = 1.0;
      for (int i = 0; i < m; ++i) x[i] /= nx;
      lu_solve(&f, x);
      double grow = nrm2(m, x);
      for (int pass = 0; pass < 2; ++pass)
        for (int p = 0; p < j; ++p) {
          const double* v = vecs + (int64_t)p * m;
          double h = dot(m, v, x);
          for (int i = 0; i < m; ++i) x[i] -= h * v[i];
        }
      if (extra < 0 && grow >= growth_target) extra = 1; /* one more sweep */
      else if (extra > 0 && --extra == 0) break;
    }
    double nx = nrm2(m, x);
    double* out = vecs + (int64_t)j * m;
    for (int i = 0; i < m; ++i) out[i] = x[i] / nx;
  }
  free(x);
  free(d);
  free(es);
  lu_free(&f);
}

typedef struct {
  const double* d;
  const double* es;
  const int* starts;
  const eig_t* sel;       /* selected eigenvalues in output order */
  const int64_t* member;  /* output positions, grouped cluster by cluster */
  const int64_t* cl_first; /* cluster -> first entry of member[] */
  const int64_t* cl_count;
  const double* bnorm;    /* per block: max |eigenvalue| of the block */
  double* Z;
  int64_t ldz;
  int n;
} vec_ctx;

static void vec_task(void* vctx, int64_t cl) {
  vec_ctx* c = (vec_ctx*)vctx;
  const int64_t* pos = c->member + c->cl_first[cl];
  int cnt = (int)c->cl_count[cl];
  int b = c->sel[pos[0]].block;
  int s = c->starts[b], m = c->starts[b + 1] - s;
  double* mus = (double*)malloc(sizeof(double) * cnt);
  double* vecs = (double*)malloc(sizeof(double) * (int64_t)cnt * m);
  for (int j = 0; j < cnt; ++j) mus[j] = c->sel[pos[j]].value;
  cluster_vectors(m, c->d + s, c->es + s, cnt, mus, c->bnorm[b], 0x5EEDull + 7919ull * (uint64_t)pos[0], vecs);
  for (int j = 0; j < cnt; ++j) {
    double* col = c->Z + pos[j] * c->ldz;
    for (int i = 0; i < c->n; ++i) col[i] = 0.0;
    memcpy(col + s, vecs + (int64_t)j * m, sizeof(double) * m);
  }
  free(mus);
  free(vecs);
}

/*
 * oracle_eigh: eigenvalues il..iu (1-based, inclusive, over the whole split
 * T, ascending) into W[0..k), and if Z != NULL the eigenvectors as the
 * columns of Z (column-major, ldz >= n).  orfac <= 0 selects 1e-3.
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_eigh(int n, const double* d, const double* e, int il, int iu, double orfac, int nthreads,
                double* W, double* Z, int64_t ldz) {
  if (n < 0 || il < 1 || iu > n || il > iu + 1 || (Z && ldz < n)) return -1;
  if (n == 0 || iu < il) return 0;
  if (orfac <= 0) orfac = 1e-3;
  double* es = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  int* starts = (int*)malloc(sizeof(int) * (n + 1));
  int nb = oracle_split(n, d, e, es, starts);
  block_t* blocks = (block_t*)malloc(sizeof(block_t) * nb);
  for (int b = 0; b < nb; ++b) block_init(&blocks[b], starts[b + 1] - starts[b], d + starts[b], es + starts[b]);

  /* Which block eigenvalues to compute: with one block only il..iu (plus the
     two extreme ones for ||T||); with several, all of them, then merge. */
  int64_t nitems;
  int64_t *ib, *il_loc;
  if (nb == 1) {
    nitems = (int64_t)(iu - il + 1) + 2;
    ib = (int64_t*)malloc(sizeof(int64_t) * nitems);
    il_loc = (int64_t*)malloc(sizeof(int64_t) * nitems);
    for (int64_t t = 0; t < nitems - 2; ++t) ib[t] = 0, il_loc[t] = il + t;
    ib[nitems - 2] = 0, il_loc[nitems - 2] = 1;
    ib[nitems - 1] = 0, il_loc[nitems - 1] = n;
  } else {
    nitems = n;
    ib = (int64_t*)malloc(sizeof(int64_t) * nitems);
    il_loc = (int64_t*)malloc(sizeof(int64_t) * nitems);
    int64_t t = 0;
    for (int b = 0; b < nb; ++b)
      for (int k = 1; k <= blocks[b].m; ++k) ib[t] = b, il_loc[t] = k, ++t;
  }
  eig_t* all = (eig_t*)malloc(sizeof(eig_t) * nitems);
  bisect_ctx bc = {blocks, starts, ib, il_loc, all};
  parallel_for(nthreads, nitems, 4, bisect_task, &bc);

  int k = iu - il + 1;
  eig_t* sel;
  double tnorm;
  if (nb == 1) {
    sel = all; /* first k items are il..iu in order */
    tnorm = fmax(fabs(all[nitems - 2].value), fabs(all[nitems - 1].value));
  } else {
    qsort(all, nitems, sizeof(eig_t), eig_cmp);
    sel = all + (il - 1);
    tnorm = fmax(fabs(all[0].value), fabs(all[nitems - 1].value));
  }
  for (int j = 0; j < k; ++j) W[j] = sel[j].value;

  if (Z) {
    /* Inverse iteration works block by block, so its norm is the block's:
       ||T_b|| = max |eigenvalue of T_b| scales the reorthogonalisation
       threshold orfac*||T_b||, the zero-pivot perturbation and the growth
       test (as in the standard bisection + inverse iteration solvers). */
    double* bnorm = (double*)calloc(nb, sizeof(double));
    if (nb == 1) {
      bnorm[0] = tnorm;
    } else {
      for (int64_t t = 0; t < nitems; ++t)
        bnorm[all[t].block] = fmax(bnorm[all[t].block], fabs(all[t].value));
    }
    /* clusters: within each block, maximal runs of the block's selected
       eigenvalues, taken in the block's own order, whose consecutive gaps
       are at most orfac*||T_b||.  With several blocks a cluster's output
       positions need not be contiguous (eigenvalues of other blocks may lie
       between its members), so the members are listed by position. */
    member_t* ord = (member_t*)malloc(sizeof(member_t) * k);
    for (int j = 0; j < k; ++j) ord[j].block = sel[j].block, ord[j].local = sel[j].local, ord[j].pos = j;
    qsort(ord, k, sizeof(member_t), member_cmp);
    int64_t* member = (int64_t*)malloc(sizeof(int64_t) * k);
    int64_t* cl_first = (int64_t*)malloc(sizeof(int64_t) * k);
    int64_t* cl_count = (int64_t*)malloc(sizeof(int64_t) * k);
    int64_t ncl = 0;
    for (int t = 0; t < k; ++t) {
      member[t] = ord[t].pos;
      int join = 0;
      if (t > 0) {
        const eig_t* p = &sel[ord[t - 1].pos];
        const eig_t* q = &sel[ord[t].pos];
        join = p->block == q->block && p->local + 1 == q->local && q->value - p->value <= orfac * bnorm[q->block];
      }
      if (join) {
        cl_count[ncl - 1]++;
      } else {
        cl_first[ncl] = t;
        cl_count[ncl] = 1;
        ++ncl;
      }
    }
    vec_ctx vc = {d, es, starts, sel, member, cl_first, cl_count, bnorm, Z, ldz, n};
    parallel_for(nthreads, ncl, 1, vec_task, &vc);
    free(bnorm);
    free(ord);
    free(member);
    free(cl_first);
    free(cl_count);
  }

  free(all);
  free(ib);
  free(il_loc);
  for (int b = 0; b < nb; ++b) block_free(&blocks[b]);
  free(blocks);
  free(starts);
  free(es);
  return 0;
}

/* Single eigenvalue lambda_k (1-based) of the whole split T, by bisection on
   the Sturm count summed over all blocks. */
double oracle_kth_eigenvalue(int n, const double* d, const double* e, int k) {
  double* es = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  int* starts = (int*)malloc(sizeof(int) * (n + 1));
  int nb = oracle_split(n, d, e, es, starts);
  block_t* blocks = (block_t*)malloc(sizeof(block_t) * nb);
  double gl = INFINITY, gu = -INFINITY;
  for (int b = 0; b < nb; ++b) {
    block_init(&blocks[b], starts[b + 1] - starts[b], d + starts[b], es + starts[b]);
    if (blocks[b].gl < gl) gl = blocks[b].gl;
    if (blocks[b].gu > gu) gu = blocks[b].gu;
  }
  double lo = gl, hi = gu;
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= 2.0 * ORACLE_EPS * fmax(fabs(lo), fabs(hi))) break;
    int cnt = 0;
    for (int b = 0; b < nb; ++b)
      cnt += sturm_count_block(blocks[b].m, blocks[b].d, blocks[b].e2, mid, blocks[b].pivmin);
    if (cnt >= k)
      hi = mid;
    else
      lo = mid;
  }
  for (int b = 0; b < nb; ++b) block_free(&blocks[b]);
  free(blocks);
  free(starts);
  free(es);
  return 0.5 * (lo + hi);
}

/* Eigenvectors of the whole split T for c given (ascending, close) values,
   computed as one cluster (inverse iteration + MGS).  Columns of Z (n x c,
   ldz = n).  Used for sampled checks at sizes where the full solve is too
   slow. */
int oracle_cluster_vectors(int n, const double* d, const double* e, int c, const double* mus, double* Z) {
  if (n <= 0 || c <= 0) return -1;
  double* es = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  int* starts = (int*)malloc(sizeof(int) * (n + 1));
  oracle_split(n, d, e, es, starts);
  double tnorm = oracle_gershgorin_norm(n, d, e);
  cluster_vectors(n, d, es, c, mus, tnorm, 0xC1A5ull, Z);
  free(es);
  free(starts);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dense cyclic Jacobi (brute force for small n).  A = T (unsplit) is        */
/* rotated to diagonal form; V accumulates the rotations.  Eigenvalues are  */
/* returned ascending with the matching columns of V.                       */

int oracle_jacobi(int n, const double* d, const double* e, double* W, double* V) {
  if (n <= 0 || n > 512) return -1;
  double* A = (double*)calloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i) {
    A[i * n + i] = d[i];
    if (i + 1 < n) A[i * n + i + 1] = A[(i + 1) * n + i] = e[i];
  }
  for (int i = 0; i < n * n; ++i) V[i] = 0.0;
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2.0 * A[p * n + q] * A[p * n + q];
    if (sqrt(off) <= 1e-2 * ORACLE_EPS * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- J^T A J with J the rotation in the (p,q) plane */
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        A[p * n + q] = A[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) { /* V is column-major: V[col*n + row] */
          double vkp = V[p * n + k], vkq = V[q * n + k];
          V[p * n + k] = c * vkp - s * vkq;
          V[q * n + k] = s * vkp + c * vkq;
        }
      }
  }
  /* selection sort of the diagonal, ascending, moving columns of V along */
  for (int i = 0; i < n; ++i) W[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {
    int mi = i;
    for (int j = i + 1; j < n; ++j)
      if (W[j] < W[mi]) mi = j;
    if (mi != i) {
      double t = W[i];
      W[i] = W[mi];
      W[mi] = t;
      for (int k = 0; k < n; ++k) {
        double v = V[i * n + k];
        V[i * n + k] = V[mi * n + k];
        V[mi * n + k] = v;
      }
    }
  }
  free(A);
  return 0;
}
