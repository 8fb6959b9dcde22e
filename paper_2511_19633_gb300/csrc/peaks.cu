// Arithmetic-pipe throughput of the current GPU, measured with the library's
// own dependent-chain microbenchmarks (the denominators of the shower's
// roofline: the shower is bound by scalar ALU work, not by HBM or tensor
// cores). Every thread runs eight independent chains of one instruction, so
// that enough instructions are in flight to fill the pipe; the grid holds
// 2048 threads per SM. The paper has no counterpart (it reports no roofline).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gaps_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256, kBlocksPerSm = 8;

// FP32 fused multiply-add: a = a * b + c (one FFMA per step)
__global__ void __launch_bounds__(kThreads) k_ffma(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 fused multiply-add (one DFMA per step)
__global__ void __launch_bounds__(kThreads) k_dfma(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// special-function unit: x = 2^(log2 x), one ex2 and one lg2 per step
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__global__ void __launch_bounds__(kThreads) k_mufu(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.5f + (float)(threadIdx.x + k) * 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = ex2(lg2(a[k]));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 32-bit integer multiply-add, low and high halves alternated (the
// operations of a Philox round): a = hi(a * m) ^ (a * m + c)
__global__ void __launch_bounds__(kThreads) k_imad(uint32_t* out, int iters, uint32_t m, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 2654435761u + (uint32_t)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __umulhi(a[k], m) ^ (a[k] * m + c);
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int gaps_alu_peak(int kind, int iters, double* ops_per_s, double* ms, void* stream) {
  if (!ops_per_s || kind < GAPS_PEAK_FFMA || kind > GAPS_PEAK_IMAD || iters < 1 || iters > (1 << 20))
    return -1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -6;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -5;
  const int blocks = n_sm * kBlocksPerSm;
  const size_t threads = (size_t)blocks * kThreads;
  void* buf = nullptr;
  if (cudaMalloc(&buf, threads * sizeof(double)) != cudaSuccess) return -5;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = 0;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = -5;
  // instructions per thread per launch, and lane operations per instruction
  double per_thread = 0.0;
  auto launch = [&]() {
    switch (kind) {
      case GAPS_PEAK_FFMA:
        k_ffma<<<blocks, kThreads, 0, st>>>((float*)buf, iters, 0.999f, 1e-3f);
        per_thread = (double)iters * 16 * kChains;
        break;
      case GAPS_PEAK_DFMA:
        k_dfma<<<blocks, kThreads, 0, st>>>((double*)buf, iters, 0.999, 1e-3);
        per_thread = (double)iters * 16 * kChains;
        break;
      case GAPS_PEAK_MUFU:
        k_mufu<<<blocks, kThreads, 0, st>>>((float*)buf, iters);
        per_thread = (double)iters * 8 * kChains * 2;
        break;
      default:
        k_imad<<<blocks, kThreads, 0, st>>>((uint32_t*)buf, iters, 0xD2511F53u, 0x9E3779B9u);
        per_thread = (double)iters * 8 * kChains;  // one product (both halves) per step
        break;
    }
  };
  // one warm-up launch, then the best of three timed ones
  float best = 0.0f;
  if (rc == 0) {
    launch();
    for (int r = 0; r < 3 && rc == 0; ++r) {
      if (cudaEventRecord(a, st) != cudaSuccess) rc = -5;
      launch();
      if (rc == 0 && cudaEventRecord(b, st) != cudaSuccess) rc = -5;
      if (rc == 0 && cudaEventSynchronize(b) != cudaSuccess) rc = -5;
      float t = 0.0f;
      if (rc == 0 && cudaEventElapsedTime(&t, a, b) != cudaSuccess) rc = -5;
      if (rc == 0 && (best == 0.0f || t < best)) best = t;
    }
    if (rc == 0 && cudaGetLastError() != cudaSuccess) rc = -5;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  if (rc != 0) return rc;
  *ops_per_s = per_thread * (double)threads / ((double)best * 1e-3);
  if (ms) *ms = best;
  return 0;
}
