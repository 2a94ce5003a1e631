// mrrr_static.cu -- mrrr_eigenvalues_static: eigenvalues il..iu of one
// tridiagonal with no device allocation and no caller workspace.
//
// Some callers cannot allocate device memory when they need eigenvalues: a
// process whose device memory is already reserved by another allocator (a
// deep-learning framework's caching allocator typically holds almost all of
// it, so a direct cudaMalloc fails), and latency-sensitive loops that cannot
// pay for cudaFree, which synchronises the whole device.  This entry point
// serves them: its scratch is one file-scope __device__ array that every GPU
// loading the library holds until the process exits.
//
// It is a variant of the root stage of the solver (mrrr_setup.cu: norm,
// power-of-two scaling, the root representation L D L^T = T - sigma I with
// the same shift ladder) followed by bisection of each wanted eigenvalue on
// that representation to full accuracy with the same Sturm count
// (negcount).  Two launches; the representation lives in the scratch array.
#include <cmath>
#include <mutex>

#include "mrrr_internal.cuh"

namespace {

using namespace mrrr;

constexpr int kStaticMaxN = MRRR_STATIC_MAX_N;
constexpr int kHeadDoubles = 32;  // header: 256 bytes, then the rows
constexpr double kPivmin = 0x1p-900;
constexpr int kMaxDevices = 64;

// Scratch: header (sigma, scale, lo0, hi0, pivmin, status) + one (D, LLD)
// row per matrix row.  Shared by every call on the device.
static __device__ __align__(256) double g_static_scratch[kHeadDoubles + 2 * kStaticMaxN];

struct StaticHead {
  double sigma;   // root shift (scaled coordinates)
  double scale;   // power of two with G(T) * scale in [1, 2)
  double lo0;     // bracket of the whole spectrum of L D L^T
  double hi0;
  double pivmin;
  int status;     // MRRR_OK, MRRR_ERR_NONFINITE or MRRR_ERR_NOCONV
  int pad_;
};
static_assert(sizeof(StaticHead) <= kHeadDoubles * sizeof(double), "header too large");

constexpr int kRootThreads = 256;

// One CTA: finiteness, G(T) and the Gershgorin interval by block reduction,
// then thread 0 builds the root representation row by row.  Every field of
// the header and every row 0..n-1 is written on each call, so nothing from
// an earlier call is read.
__global__ void __launch_bounds__(kRootThreads) k_static_root(int n, const double* __restrict__ d,
                                                              const double* __restrict__ e, int il, int iu,
                                                              double* scratch) {
  __shared__ double s_g[kRootThreads / 32], s_gl[kRootThreads / 32], s_gu[kRootThreads / 32];
  __shared__ int s_bad[kRootThreads / 32];
  double g = 0.0, gl = INFINITY, gu = -INFINITY;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = d[i];
    double r = 0.0;
    bad |= !isfinite(di);
    if (i > 0) r += fabs(e[i - 1]);
    if (i + 1 < n) {
      const double ei = e[i];
      bad |= !isfinite(ei);
      r += fabs(ei);
    }
    g = fmax(g, fabs(di) + r);
    gl = fmin(gl, di - r);
    gu = fmax(gu, di + r);
  }
  for (int o = 16; o; o >>= 1) {
    g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_g[warp] = g;
    s_gl[warp] = gl;
    s_gu[warp] = gu;
    s_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < kRootThreads / 32; ++w) {
    g = fmax(g, s_g[w]);
    gl = fmin(gl, s_gl[w]);
    gu = fmax(gu, s_gu[w]);
    bad |= s_bad[w] != 0;
  }
  StaticHead h{};
  h.pivmin = kPivmin;
  h.scale = 1.0;
  double2* rows = reinterpret_cast<double2*>(scratch + kHeadDoubles);
  if (bad) {
    h.status = MRRR_ERR_NONFINITE;
    *reinterpret_cast<StaticHead*>(scratch) = h;
    return;
  }
  if (g > 0.0) {
    int ex = 0;
    frexp(g, &ex);
    h.scale = ldexp(1.0, 1 - ex);
  }
  gl *= h.scale;
  gu *= h.scale;
  const double spdiam = gu - gl;
  if (n == 1 || !(spdiam > 0.0)) {  // n = 1 or a multiple of I: every eigenvalue is d_0
    h.sigma = d[0] * h.scale;
    h.lo0 = h.hi0 = 0.0;
    h.status = MRRR_OK;
    *reinterpret_cast<StaticHead*>(scratch) = h;
    return;
  }
  // shift at the Gershgorin end nearer the wanted range, moved outward until
  // every pivot has the sign of a definite factorization
  const bool left = (il + iu) <= (n + 1);
  bool ok = false;
  double sigma = left ? gl : gu;
  for (int t = 0; t < 12 && !ok; ++t) {
    double delta = (t == 0) ? 0.0 : spdiam * kEps * 4.0 * (double)(1LL << (2 * t));
    if (t == 11) delta = 0.05 * spdiam + kPivmin;
    sigma = left ? gl - delta : gu + delta;
    double D = d[0] * h.scale - sigma;
    ok = true;
    for (int i = 0; i < n - 1; ++i) {
      if (!(left ? D > kPivmin : D < -kPivmin) || !isfinite(D)) {
        ok = false;
        break;
      }
      const double ei = e[i] * h.scale;
      const double l = ei / D;
      const double LLD = l * (l * D);
      rows[i] = make_double2(D, LLD);
      D = d[i + 1] * h.scale - sigma - LLD;
    }
    if (ok && (!(left ? D > kPivmin : D < -kPivmin) || !isfinite(D))) ok = false;
    if (ok) rows[n - 1] = make_double2(D, 0.0);
  }
  h.sigma = sigma;
  // bracket of the shifted spectrum, widened against rounding
  const double pad = spdiam * 0x1p-20 + kPivmin;
  h.lo0 = (gl - sigma) - pad;
  h.hi0 = (gu - sigma) + pad;
  h.status = ok ? MRRR_OK : MRRR_ERR_NOCONV;
  *reinterpret_cast<StaticHead*>(scratch) = h;
}

// One thread per wanted eigenvalue j = il + t: bisection of [lo0, hi0] on the
// representation in the scratch rows to full accuracy (width at most 2 eps
// relative, or the two ends adjacent in floating point).  Device-side errors
// give NaN eigenvalues.
__global__ void k_static_bisect(int n, int il, int iu, double* __restrict__ W, const double* scratch) {
  const int k = iu - il + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const StaticHead h = *reinterpret_cast<const StaticHead*>(scratch);
  if (h.status != MRRR_OK) {
    W[t] = NAN;
    return;
  }
  if (!(h.hi0 > h.lo0)) {
    W[t] = h.sigma / h.scale;
    return;
  }
  const double2* rows = reinterpret_cast<const double2*>(scratch + kHeadDoubles);
  double lo = h.lo0, hi = h.hi0;
  bisect_interval(rows, n, il + t, h.pivmin, 2.0 * kEps, 0.0, 256, lo, hi);
  W[t] = (h.sigma + 0.5 * (lo + hi)) / h.scale;
}

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in and must never be
// passed to a kernel).  The cached address belongs to the device's primary
// context: it does not survive cudaDeviceReset (see the header).
mrrr_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MRRR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return MRRR_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return MRRR_OK;
}

}  // namespace

extern "C" mrrr_status mrrr_eigenvalues_static(int n, const double* d, const double* e, int il, int iu, double* W,
                                               mrrr_stream stream) {
  if (n < 0 || n > kStaticMaxN) return MRRR_ERR_ARG;
  if (n == 0) return MRRR_OK;
  if (!d || !W || (n > 1 && !e) || il < 1 || il > iu || iu > n) return MRRR_ERR_ARG;
  double* scratch = nullptr;
  const mrrr_status st = scratch_address(&scratch);
  if (st != MRRR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_static_root<<<1, kRootThreads, 0, s>>>(n, d, e, il, iu, scratch);
  if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
  const int k = iu - il + 1;
  k_static_bisect<<<(k + 127) / 128, 128, 0, s>>>(n, il, iu, W, scratch);
  if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
  return MRRR_OK;
}
