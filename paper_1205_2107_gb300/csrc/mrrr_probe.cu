// mrrr_probe.cu -- measurement support: the peak rates of this GPU's
// arithmetic units that the solver's roofline is quoted against.  The solve
// path is FP64 scalar work (Sturm counts, qd transforms) bound by the FP64
// FMA pipe; the backward pass's two n^3 contractions can run on the FP64
// pipe or on the FP64 tensor cores (mma.sync m8n8k4).  No vendor figure is
// assumed: each rate is timed here, on all SMs, with CUDA events.
//
// Kinds: 0 DFMA (flops, 2 per FMA), 1 DMMA m8n8k4 (flops, 512 per warp
// instruction), 2 FP64 division (1 per division), 3 FFMA (FP32 flops);
// and the two facts the interval engine's cost model rests on:
// 4 DFMA warp instructions per second with ONE active lane per warp (equal
// to kind 0 / 64 when a warp instruction costs the same whatever its active
// lanes), 5 cycles of one dependent FP64 FMA (one warp alone on an SM),
// 6 cycles of one dependent FP64 division plus an add (idem).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mrrr.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent accumulators per thread

// A sink the compiler cannot see through, so that the timed arithmetic is kept.
static __device__ double g_probe_sink[4];

__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(int iters, double seed) {
  double x[kChains];
  const double a = 1.0 + seed * 1e-9, b = 1e-7 * seed;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + c + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0.123456789) g_probe_sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(int iters, float seed) {
  float x[kChains];
  const float a = 1.0f + seed * 1e-6f, b = 1e-5f * seed;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + c + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0.123456789f) g_probe_sink[3] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ddiv(int iters, double seed) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.5 + seed + c;
  const double d = 1.0000001 + seed * 1e-12;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] / d;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0.123456789) g_probe_sink[2] = s;
}

// The DFMA chains of k_probe_dfma on lane 0 of every warp only.
__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma_lane0(int iters, double seed) {
  if ((threadIdx.x & 31) != 0) return;
  double x[kChains];
  const double a = 1.0 + seed * 1e-9, b = 1e-7 * seed;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + c + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0.123456789) g_probe_sink[0] = s;
}

// One warp, one dependent chain: SM clock cycles per step (FMA, or division
// plus add), from clock64() around the chain.
static __device__ long long g_probe_cycles;

__global__ void k_probe_chain(int iters, double seed, int div) {
  double x = 1.5 + seed;
  const double a = 1.0 + seed * 1e-9, b = 1e-7 * seed;
  const long long t0 = clock64();
  if (div) {
    for (int it = 0; it < iters; ++it) x = x / a + b;
  } else {
    for (int it = 0; it < iters; ++it) x = fma(x, a, b);
  }
  const long long t1 = clock64();
  if (x == 0.123456789) g_probe_sink[2] = x;
  if (threadIdx.x == 0) g_probe_cycles = t1 - t0;
}

// FP64 tensor-core MMA: D(8x8) = A(8x4) B(4x8) + C, one register each of A
// and B per lane, two of the accumulator; four independent accumulators.
__global__ void __launch_bounds__(kProbeThreads) k_probe_dmma(int iters, double seed) {
  const double a = 1.0 + seed * 1e-9, b = 1e-3 * seed + threadIdx.x * 1e-9;
  double acc[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = seed + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  if (s == 0.123456789) g_probe_sink[1] = s;
}

}  // namespace

extern "C" mrrr_status mrrr_probe_peak(int kind, double* rate) {
  if (!rate || kind < 0 || kind > 6) return MRRR_ERR_ARG;
  *rate = 0.0;
  if (kind == 5 || kind == 6) {  // latency: one warp, cycles per dependent step
    const int steps = 1 << 14;
    k_probe_chain<<<1, 32>>>(steps / 16, 0.5, kind == 6);  // warm-up
    k_probe_chain<<<1, 32>>>(steps, 0.5, kind == 6);
    long long cyc = 0;
    if (cudaMemcpyFromSymbol(&cyc, g_probe_cycles, sizeof(cyc)) != cudaSuccess) return MRRR_ERR_CUDA;
    *rate = (double)cyc / steps;
    return MRRR_OK;
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRRR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MRRR_ERR_CUDA;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return MRRR_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaStreamDestroy(s);
    return MRRR_ERR_CUDA;
  }
  const int blocks = nsm * 4;  // 32 warps per SM
  // iterations sized for roughly 30-50 ms per timed launch on a GB300-class part
  // (about 1.2 TFLOP/s FP64, 1.1 TFLOP/s DMMA, 70 G divisions/s, 38 TFLOP/s FP32)
  const int iters = kind == 2 ? 1 << 11 : kind == 3 ? 1 << 19 : kind == 1 ? 1 << 12 : 1 << 14;
  // (kind 4 runs the DFMA chains of kind 0, on one lane of each warp)
  auto launch = [&](int it) {
    if (kind == 0) k_probe_dfma<<<blocks, kProbeThreads, 0, s>>>(it, 0.5);
    if (kind == 1) k_probe_dmma<<<blocks, kProbeThreads, 0, s>>>(it, 0.5);
    if (kind == 2) k_probe_ddiv<<<blocks, kProbeThreads, 0, s>>>(it, 0.5);
    if (kind == 3) k_probe_ffma<<<blocks, kProbeThreads, 0, s>>>(it, 0.5f);
    if (kind == 4) k_probe_dfma_lane0<<<blocks, kProbeThreads, 0, s>>>(it, 0.5);
  };
  launch(iters / 16);  // warm-up
  float best = 0.f;
  mrrr_status st = MRRR_OK;
  for (int r = 0; r < 3 && st == MRRR_OK; ++r) {
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = MRRR_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == 0 || ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) st = MRRR_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st != MRRR_OK || best <= 0.f) return st == MRRR_OK ? MRRR_ERR_CUDA : st;
  const double threads = (double)blocks * kProbeThreads;
  double ops = 0.0;
  if (kind == 0 || kind == 3) ops = threads * kChains * (double)iters * 2.0;
  if (kind == 2) ops = threads * kChains * (double)iters;
  if (kind == 1) ops = threads / 32.0 * 4.0 * (double)iters * 512.0;
  if (kind == 4) ops = threads / 32.0 * kChains * (double)iters;  // warp instructions
  *rate = ops / (best * 1e-3);
  return MRRR_OK;
}
