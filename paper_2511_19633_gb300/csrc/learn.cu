// Device steps of the learned proposal's training pipeline that surround the
// shower's state collection, the teacher and the network's own training
// kernels: the canonical order of the logged states (a bitonic sort, so that
// training does not depend on the order in which the shower's atomic counter
// logged them), the floor of the targets, the network's initialisation, and
// the calibration of the margins per (class, eta bucket, bin) cell with the
// shower's BF16 inference numerics. The learned proposal itself is the
// build's own addition (the paper's overestimate is a fitted PDF-ratio bound,
// App. A.2); the host orchestration is gaps_train_learned_proposal.
#include <cmath>

#include "common.cuh"
#include "mlp_infer.cuh"

namespace gaps {
namespace {

// canonical order of a state {eta, s, dipole type, PDF index}: type, then PDF
// index, then eta, then s
__device__ __forceinline__ bool state_less(const float4& a, const float4& b) {
  if (a.z != b.z) return a.z < b.z;
  if (a.w != b.w) return a.w < b.w;
  if (a.x != b.x) return a.x < b.x;
  return a.y < b.y;
}

// one compare-exchange stage (j, k) of a bitonic sort of npow2 entries
__global__ void k_bitonic(float4* v, uint64_t npow2, uint64_t j, uint64_t k) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npow2; i += stride) {
    const uint64_t l = i ^ j;
    if (l <= i) continue;
    const bool up = (i & k) == 0;
    const float4 a = v[i], b = v[l];
    const bool swap = up ? state_less(b, a) : state_less(a, b);
    if (swap) {
      v[i] = b;
      v[l] = a;
    }
  }
}

__global__ void k_fill_inf(float4* v, uint64_t from, uint64_t to) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = from + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < to; i += stride)
    v[i] = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
}

__global__ void k_floor(float* t, uint64_t n, float lo) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) t[i] = fmaxf(t[i], lo);
}

// He initialisation: W1 ~ N(0, 2/4), W2 ~ N(0, 2/64), W3 ~ N(0, 1/64), biases
// 0.1 (hidden) and -1 (output); normal deviates by Box-Muller from Philox
// blocks (seed, parameter index)
__global__ void k_mlp_init(float* P, uint64_t seed) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kMlpParams) return;
  const int nW1 = kMlpH * kMlpIn, nb1 = kMlpH, nW2 = kMlpH * kMlpH, nb2 = kMlpH, nW3 = kMlpH;
  float sd = 0.0f, bias = 0.0f;
  if (q < nW1) sd = sqrtf(2.0f / kMlpIn);
  else if (q < nW1 + nb1) bias = 0.1f;
  else if (q < nW1 + nb1 + nW2) sd = sqrtf(2.0f / kMlpH);
  else if (q < nW1 + nb1 + nW2 + nb2) bias = 0.1f;
  else if (q < nW1 + nb1 + nW2 + nb2 + nW3) sd = sqrtf(1.0f / kMlpH);
  else bias = -1.0f;
  if (sd == 0.0f) {
    P[q] = bias;
    return;
  }
  uint32_t out[4];
  philox((uint32_t)q, 0x1417u, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32), out);
  const double u1 = u01(out[0], out[1]), u2 = u01(out[2], out[3]);
  P[q] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

// calibration cell of a row from its network inputs (the shower's own
// comparisons): (class, eta bucket, bin)
__device__ __forceinline__ int row_cell(const float* f) {
  const int cls = __float2int_rn((f[3] + 1.0f) * 21.5f);
  const int m = __float2int_rn((f[2] + 1.0f) * 4.0f - 0.5f);
  const int c = min(max(cls, 0), kIsrClasses - 1), mb = min(max(m, 0), kIsrBins - 1);
  return (c * kEtaBins + eta_bucket(f[0])) * kIsrBins + mb;
}

// order-preserving map of floats to signed integers (for atomicMax)
__device__ __forceinline__ int ordered(float x) {
  const int i = __float_as_int(x);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_cal_init(int* gap, unsigned* rows, int ncell) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ncell) {
    gap[q] = ordered(-INFINITY);
    rows[q] = 0;
  }
}

// per cell: the largest (target - network output) and the number of rows
__global__ void k_cal_accumulate(const float* feats, const float* targ, const float* out, uint64_t n, int* gap,
                                 unsigned* rows) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int c = row_cell(feats + 4 * r);
    atomicMax(&gap[c], ordered(targ[r] - out[r]));
    atomicAdd(&rows[c], 1u);
  }
}

// margin = largest gap + ln(1 + slack) where the cell has min_rows rows, else
// `unseen` (a height of one: the plain bound)
__global__ void k_cal_margins(const int* gap, const unsigned* rows, int ncell, unsigned min_rows, float log_slack,
                              float unseen, float* margins, unsigned* seen) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncell) return;
  const bool ok = rows[q] >= min_rows;
  margins[q] = ok ? unordered(gap[q]) + log_slack : unseen;
  if (ok) atomicAdd(seen, 1u);
}

// mean of the calibrated heights min(1, exp(out + margin)) and of the squared
// fit residual over one set (sums in FP64)
__global__ void k_cal_stats(const float* feats, const float* targ, const float* out, uint64_t n,
                            const float* margins, double* sums) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double h = 0.0, r2 = 0.0;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int c = row_cell(feats + 4 * r);
    h += fminf(expf(out[r] + margins[c]), 1.0f);
    const double d = (double)out[r] - (double)targ[r];
    r2 += d * d;
  }
  for (int off = 16; off > 0; off >>= 1) {
    h += __shfl_xor_sync(0xffffffffu, h, off);
    r2 += __shfl_xor_sync(0xffffffffu, r2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], h);
    atomicAdd(&sums[1], r2);
  }
}

unsigned grid_of(uint64_t n, int bs) {
  uint64_t b = (n + bs - 1) / bs;
  return (unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

// Sorts states[0 .. n) into the canonical order (ascending type, PDF index,
// eta, s). `states` must hold the next power of two of n entries (the tail is
// padding, overwritten).
cudaError_t sort_states(float4* states, uint64_t n, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  uint64_t np2 = 1;
  while (np2 < n) np2 <<= 1;
  // padding with +infinity, stored: every compare-exchange then has both ends
  k_fill_inf<<<grid_of(np2 - n, 256), 256, 0, st>>>(states, n, np2);
  for (uint64_t k = 2; k <= np2; k <<= 1)
    for (uint64_t j = k >> 1; j > 0; j >>= 1)
      k_bitonic<<<grid_of(np2, 256), 256, 0, st>>>(states, np2, j, k);
  return cudaGetLastError();
}

cudaError_t floor_values(float* t, uint64_t n, float lo, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_floor<<<grid_of(n, 256), 256, 0, st>>>(t, n, lo);
  return cudaGetLastError();
}

cudaError_t mlp_init(float* params, uint64_t seed, cudaStream_t st) {
  k_mlp_init<<<(kMlpParams + 127) / 128, 128, 0, st>>>(params, seed);
  return cudaGetLastError();
}

constexpr int kCalCells = kIsrClasses * kEtaBins * kIsrBins;

cudaError_t calibration_init(int* gap, unsigned* rows, cudaStream_t st) {
  k_cal_init<<<(kCalCells + 127) / 128, 128, 0, st>>>(gap, rows, kCalCells);
  return cudaGetLastError();
}

cudaError_t calibration_accumulate(const float* feats, const float* targ, const float* out, uint64_t n, int* gap,
                                   unsigned* rows, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_cal_accumulate<<<grid_of(n, 256), 256, 0, st>>>(feats, targ, out, n, gap, rows);
  return cudaGetLastError();
}

cudaError_t calibration_margins(const int* gap, const unsigned* rows, unsigned min_rows, float slack, float unseen,
                                float* margins, unsigned* seen, cudaStream_t st) {
  k_cal_margins<<<(kCalCells + 127) / 128, 128, 0, st>>>(gap, rows, kCalCells, min_rows, log1pf(slack), unseen,
                                                         margins, seen);
  return cudaGetLastError();
}

cudaError_t calibration_stats(const float* feats, const float* targ, const float* out, uint64_t n,
                              const float* margins, double* sums, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_cal_stats<<<grid_of(n, 256), 256, 0, st>>>(feats, targ, out, n, margins, sums);
  return cudaGetLastError();
}

}  // namespace gaps
