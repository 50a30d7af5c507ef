// Arithmetic peak probe: the FP32 and FP64 fused multiply-add rates this GPU sustains,
// measured with CUDA events.  The stencil kernels of the sweep are bound by instruction
// issue and FP32 arithmetic rather than by HBM, so their roofline fraction is stated
// against these measured rates as well as against the copy bandwidth.
//
// Every thread runs kChains independent multiply-add chains for `iters` rounds, so the
// pipes see kChains x (resident warps) independent instructions per dependency
// latency; the grid fills every SM at full occupancy.  The result is stored only when
// it equals an impossible sentinel (the stores are never taken but keep the chains live).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ns_adjoint.h"
#include "ns_common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_f32(int iters, float x, float y, float* out) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = x + 0.001f * (float)(threadIdx.x + i);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], x, y);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma_f32x2(int iters, float x, float y, float* out) {
  float2 a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(x + 0.001f * (float)(threadIdx.x + i), x - 0.002f * (float)i);
  const float2 xx = make_float2(x, x), yy = make_float2(y, y);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], xx, yy);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == -12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma_f64(int iters, double x, double y, float* out) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = x + 0.001 * (double)(threadIdx.x + i);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], x, y);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// flops of one thread's run: kChains chains x 16 multiply-adds (8 paired) x 2 flops
double flops_per_thread(int kind, int iters) { return (double)kChains * 16.0 * 2.0 * (double)iters; }

cudaError_t launch_kind(int kind, int blocks, int iters, float* out, cudaStream_t st) {
  ns::count_launch();
  if (kind == NS_PEAK_FP32)
    k_fma_f32<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, out);
  else if (kind == NS_PEAK_FP32X2)
    k_fma_f32x2<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, out);
  else
    k_fma_f64<<<blocks, kThreads, 0, st>>>(iters, 0.999, 1e-3, out);
  return cudaGetLastError();
}

}  // namespace

extern "C" int ns_measure_fma_peak(int kind, double* flops_per_s) {
  if (!flops_per_s || (kind != NS_PEAK_FP32 && kind != NS_PEAK_FP32X2 && kind != NS_PEAK_FP64))
    return NS_ERR_ARG;
  *flops_per_s = 0.0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NS_ERR_CUDA;
  const void* kern = kind == NS_PEAK_FP32 ? (const void*)k_fma_f32
                     : kind == NS_PEAK_FP32X2 ? (const void*)k_fma_f32x2
                                              : (const void*)k_fma_f64;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess)
    return NS_ERR_CUDA;
  const int blocks = std::max(1, per_sm) * sms;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = NS_ERR_CUDA;
  if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    // calibrate the round count to about 20 ms per launch, then keep the best of three
    int iters = 64;
    double best = 0.0;
    bool ok = true;
    for (int trial = 0; trial < 8 && ok; ++trial) {
      ok = cudaEventRecord(e0, st) == cudaSuccess && launch_kind(kind, blocks, iters, out, st) == cudaSuccess &&
           cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (!ok) break;
      if (ms < 10.f && trial < 5) {
        const double scale = ms > 0.01f ? 20.0 / ms : 64.0;
        iters = (int)std::min(1e8, iters * std::min(scale, 64.0));
        continue;
      }
      const double f = flops_per_thread(kind, iters) * blocks * kThreads / (ms * 1e-3);
      best = std::max(best, f);
    }
    if (ok && best > 0.0) {
      *flops_per_s = best;
      rc = NS_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}
