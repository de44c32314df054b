// alu_probe.cu -- fdtd_alu_probe: measured FMA throughput of this GPU, the
// denominator of the arithmetic roofline of the marches (the FP64 march is
// bound by the FP64 pipe, the double-float march by the FP32 pipe).
//
// Every thread runs kChains independent chains a = a * b + c (no chain can be
// shortened: each step needs the previous value), enough warps per SM to hide
// the pipe latency, for a fixed number of steps.  Time is taken with CUDA
// events around the timed launch on the caller's stream, after one untimed
// launch; flops = 2 per FMA (4 per packed f32x2 FMA).
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__device__ double g_sink_d;
__device__ float g_sink_f;

__global__ void __launch_bounds__(kProbeThreads) k_fma_f64(int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) g_sink_d = s;  // never true for these inputs; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_f32(int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) g_sink_f = s;
}

// packed pairs: one fma.rn.f32x2 does two FP32 FMAs
__device__ __forceinline__ unsigned long long pack2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
  return make_float2(x, y);
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_f32x2(int iters, float b, float c) {
  unsigned long long a[kChains];
  const unsigned long long bb = pack2(b, b), cc = pack2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = pack2(1e-3f * threadIdx.x + k, 2e-3f * threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    const float2 v = unpack2(a[k]);
    s += v.x + v.y;
  }
  if (s == -1.0f) g_sink_f = s;
}

}  // namespace

extern "C" fdtd_status fdtd_alu_probe(int32_t kind, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s || kind < 0 || kind > 2) return FDTD_ERR_INVALID_ARG;
  *flops_per_s = 0.0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FDTD_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = kind == 0 ? (const void*)k_fma_f64 : kind == 1 ? (const void*)k_fma_f32 : (const void*)k_fma_f32x2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kProbeThreads, 0) != cudaSuccess || per < 1)
    return FDTD_ERR_CUDA;
  const int grid = sms * per;
  // steps per thread: about 50 ms at the nominal rates (FP64 ~2 FMA/clk/SM, FP32 128/clk/SM)
  const int iters = kind == 0 ? 2000 : 80000;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return FDTD_ERR_CUDA;
  }
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    if (rep == 1) e = cudaEventRecord(e0, s);
    if (kind == 0) k_fma_f64<<<grid, kProbeThreads, 0, s>>>(iters, 1.0000001, 1e-9);
    else if (kind == 1) k_fma_f32<<<grid, kProbeThreads, 0, s>>>(iters, 1.0000001f, 1e-9f);
    else k_fma_f32x2<<<grid, kProbeThreads, 0, s>>>(iters, 1.0000001f, 1e-9f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(e1, s);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return FDTD_ERR_CUDA;
  const double fmas = (double)grid * kProbeThreads * iters * 4.0 * kChains * (kind == 2 ? 2.0 : 1.0);
  *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  return FDTD_OK;
}
