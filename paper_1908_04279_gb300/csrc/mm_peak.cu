// Arithmetic roofs of the device, measured: the rate of fused multiply-adds
// that a kernel of independent dependency chains sustains, in float64, scalar
// float32 and packed two-value float32. These are the ceilings of the kernels
// that are bound by arithmetic issue rather than by memory: the float64
// substep (float64 pipe) and the local-step motor update (float32 pipe), whose
// data stay on chip for a whole call.
//
// Each thread runs kChains independent chains x <- x * b + c for `iters`
// iterations; b and c are kernel arguments (nothing folds at compile time),
// b < 1 keeps every chain bounded and away from subnormals. The chains' sum
// is stored only when it equals an impossible value, so the work is kept but
// nothing is written. The grid covers every SM with full blocks.
#include <cuda_runtime.h>

#include <cstdio>

#include "mm_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ double g_peak_sink;

__global__ void __launch_bounds__(kThreads) k_peak_f64(int iters, double b, double c) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = __fma_rn(x[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  if (s == -1.0) g_peak_sink = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32(int iters, float b, float c) {
  float x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = threadIdx.x * 1e-3f + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = __fmaf_rn(x[q], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  if (s == -1.0f) g_peak_sink = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32x2(int iters, float b, float c) {
  float2 x[kChains / 2];
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q)
    x[q] = make_float2(threadIdx.x * 1e-3f + 2 * q, threadIdx.x * 1e-3f + 2 * q + 1);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains / 2; ++q) x[q] = __ffma2_rn(x[q], b2, c2);
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q) s += x[q].x + x[q].y;
  if (s == -1.0f) g_peak_sink = s;
}

mm_status peak_fail(mm_status st, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "mm_alu_peak: %s: %s", what, cudaGetErrorString(e));
  mm::set_thread_error(buf);
  return st;
}

}  // namespace

extern "C" mm_status mm_alu_peak(int kind, double* fma_per_s, double* ms_per_launch,
                                 void* stream) {
  if (!fma_per_s || kind < 0 || kind > 2) {
    mm::set_thread_error("mm_alu_peak: kind must be 0, 1 or 2 and fma_per_s non-NULL");
    return MM_ERR_INVALID;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return peak_fail(MM_ERR_CUDA, "device query", e);
  const void* fn = kind == 0 ? (const void*)k_peak_f64
                             : (kind == 1 ? (const void*)k_peak_f32 : (const void*)k_peak_f32x2);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
  if (e != cudaSuccess || per_sm < 1) return peak_fail(MM_ERR_CUDA, "occupancy", e);
  const int blocks = sms * per_sm;
  // a launch of a few milliseconds at the expected rates (float64 is a small
  // fraction of the float32 rate on this part)
  const int iters = kind == 0 ? 2048 : 65536;
  cudaStream_t s = (cudaStream_t)stream;
  auto launch = [&]() {
    if (kind == 0)
      k_peak_f64<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7);
    else if (kind == 1)
      k_peak_f32<<<blocks, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f);
    else
      k_peak_f32x2<<<blocks, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return peak_fail(MM_ERR_CUDA, "event", e);
  }
  constexpr int kReps = 5;
  launch();  // warm-up (module load, clocks)
  cudaEventRecord(e0, s);
  for (int r = 0; r < kReps; ++r) launch();
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return peak_fail(MM_ERR_CUDA, "timed launches", e);
  const double per = (double)ms / kReps;
  const double fmas = (double)blocks * kThreads * kChains * (double)iters;
  *fma_per_s = fmas / (per * 1e-3);
  if (ms_per_launch) *ms_per_launch = per;
  return MM_OK;
}
