// Training of the learned-proposal network on the GPU with the library's own
// kernels: FP32 forward and backward passes of the 4 -> 64 -> 64 -> 1 ReLU
// network, the asymmetric squared (expectile) loss that biases the fit to
// lie above its targets, and Adam updates. Inference in the shower uses the
// BF16 tensor-core tile of mlp_infer.cuh; gaps_mlp_forward exposes both
// numerics for calibration and tests.
#include "common.cuh"
#include "mlp_infer.cuh"

namespace gaps {
namespace {

struct Layers {
  const float *W1, *b1, *W2, *b2, *W3;
  float b3;
};

__device__ __forceinline__ Layers layers_of(const float* P) {
  Layers L;
  L.W1 = P;
  L.b1 = L.W1 + kMlpH * kMlpIn;
  L.W2 = L.b1 + kMlpH;
  L.b2 = L.W2 + kMlpH * kMlpH;
  L.W3 = L.b2 + kMlpH;
  L.b3 = L.W3[kMlpH];
  return L;
}

__device__ float forward_one(const Layers& L, const float* x, float* h1, float* h2) {
  for (int i = 0; i < kMlpH; ++i) {
    float a = L.b1[i];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) a = fmaf(L.W1[i * kMlpIn + k], x[k], a);
    h1[i] = fmaxf(a, 0.0f);
  }
  for (int i = 0; i < kMlpH; ++i) {
    float a = L.b2[i];
    for (int k = 0; k < kMlpH; ++k) a = fmaf(L.W2[i * kMlpH + k], h1[k], a);
    h2[i] = fmaxf(a, 0.0f);
  }
  float y = L.b3;
  for (int k = 0; k < kMlpH; ++k) y = fmaf(L.W3[k], h2[k], y);
  return y;
}

// per-sample gradient accumulated into a block-shared buffer, then global
__global__ void k_loss_grad(const float* P, const float* X, const float* T, uint64_t n, float tau,
                            float* grad, float* loss) {
  extern __shared__ float sg[];  // kMlpParams + 1 (loss)
  for (int q = threadIdx.x; q <= kMlpParams; q += blockDim.x) sg[q] = 0.0f;
  __syncthreads();
  const Layers L = layers_of(P);
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    float h1[kMlpH], h2[kMlpH], d2[kMlpH];
    const float* x = X + 4 * s;
    float y = forward_one(L, x, h1, h2);
    float r = y - T[s];
    float w = r < 0.0f ? tau : 1.0f - tau;
    atomicAdd(&sg[kMlpParams], w * r * r / (float)n);
    float dy = 2.0f * w * r / (float)n;
    float* gW1 = sg;
    float* gb1 = gW1 + kMlpH * kMlpIn;
    float* gW2 = gb1 + kMlpH;
    float* gb2 = gW2 + kMlpH * kMlpH;
    float* gW3 = gb2 + kMlpH;
    atomicAdd(&gW3[kMlpH], dy);
    for (int k = 0; k < kMlpH; ++k) {
      atomicAdd(&gW3[k], dy * h2[k]);
      d2[k] = h2[k] > 0.0f ? dy * L.W3[k] : 0.0f;
    }
    for (int i = 0; i < kMlpH; ++i) {
      if (d2[i] == 0.0f) continue;
      atomicAdd(&gb2[i], d2[i]);
      for (int k = 0; k < kMlpH; ++k)
        if (h1[k] != 0.0f) atomicAdd(&gW2[i * kMlpH + k], d2[i] * h1[k]);
    }
    for (int k = 0; k < kMlpH; ++k) {
      if (h1[k] <= 0.0f) continue;
      float a = 0.0f;
      for (int i = 0; i < kMlpH; ++i) a = fmaf(L.W2[i * kMlpH + k], d2[i], a);
      atomicAdd(&gb1[k], a);
      for (int j = 0; j < kMlpIn; ++j) atomicAdd(&gW1[k * kMlpIn + j], a * x[j]);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kMlpParams; q += blockDim.x)
    if (sg[q] != 0.0f) atomicAdd(&grad[q], sg[q]);
  if (threadIdx.x == 0) atomicAdd(loss, sg[kMlpParams]);
}

__global__ void k_forward_f32(const float* P, const float* X, uint64_t n, float* out) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float h1[kMlpH], h2[kMlpH];
  out[s] = forward_one(layers_of(P), X + 4 * s, h1, h2);
}

// BF16 tensor-core forward, the numerics of the shower's inference
__global__ void k_forward_bf16(const float* P, const float* X, uint64_t n, float* out) {
  __shared__ MlpSmem S;
  __shared__ float feat[8][16][4];
  __shared__ float res[8][16];
  mlp_load_smem(S, P);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t tiles = (n + 15) / 16;
  for (uint64_t tile = (uint64_t)blockIdx.x * 8 + warp; tile < tiles; tile += (uint64_t)gridDim.x * 8) {
    for (int q = lane; q < 64; q += 32) {
      uint64_t row = tile * 16 + q / 4;
      feat[warp][q / 4][q % 4] = row < n ? X[4 * row + q % 4] : 0.0f;
    }
    __syncwarp();
    mlp_tile(S, feat[warp], res[warp]);
    if (lane < 16 && tile * 16 + lane < n) out[tile * 16 + lane] = res[warp][lane];
    __syncwarp();
  }
}

// The network's BF16 image in global memory for the shower's inference
__global__ void k_mlp_image(const float* P, MlpSmem* out) { mlp_load_smem(*out, P); }

// Minibatch Adam training, one block of 256 threads looping over minibatches
// of 256 rows drawn with replacement (Philox counter = step). Activations of
// the batch live in shared memory; the small GEMMs of the backward pass are
// spread over the threads.
constexpr int kB = 256;
struct TrainSmem {
  float x[kB][kMlpIn];
  float h1[kB][kMlpH];  // activations, then their gradients
  float h2[kB][kMlpH];
  float dy[kB];
  float p[kMlpParams];  // current parameters
  float g[kMlpParams];  // gradient of the batch
  float loss;
};

__global__ void __launch_bounds__(kB) k_train(float* P, float* m1, float* m2, const float* X, const float* T,
                                               uint64_t n, uint64_t steps, float lr, float tau, uint64_t seed,
                                               float* loss_hist, int hist_every) {
  extern __shared__ unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int q = tid; q < kMlpParams; q += kB) S.p[q] = P[q];
  __syncthreads();
  const float b1c = 0.9f, b2c = 0.999f, eps = 1e-8f;
  float b1t = 1.0f, b2t = 1.0f;
  for (uint64_t step = 0; step < steps; ++step) {
    // --- batch and forward pass: thread tid owns row tid
    uint32_t rnd[4];
    philox((uint32_t)step, (uint32_t)(step >> 32), (uint32_t)tid, 0x5eedu, (uint32_t)seed,
           (uint32_t)(seed >> 32), rnd);
    const uint64_t row = (((uint64_t)rnd[1] << 32) | rnd[0]) % n;
    for (int k = 0; k < kMlpIn; ++k) S.x[tid][k] = X[4 * row + k];
    const Layers L = layers_of(S.p);
    for (int i = 0; i < kMlpH; ++i) {
      float a = L.b1[i];
      for (int k = 0; k < kMlpIn; ++k) a = fmaf(L.W1[i * kMlpIn + k], S.x[tid][k], a);
      S.h1[tid][i] = fmaxf(a, 0.0f);
    }
    for (int i = 0; i < kMlpH; ++i) {
      float a = L.b2[i];
      for (int k = 0; k < kMlpH; ++k) a = fmaf(L.W2[i * kMlpH + k], S.h1[tid][k], a);
      S.h2[tid][i] = fmaxf(a, 0.0f);
    }
    float y = L.b3;
    for (int k = 0; k < kMlpH; ++k) y = fmaf(L.W3[k], S.h2[tid][k], y);
    const float r = y - T[row];
    const float w = r < 0.0f ? tau : 1.0f - tau;
    S.dy[tid] = 2.0f * w * r / (float)kB;
    if (tid == 0) S.loss = 0.0f;
    __syncthreads();
    atomicAdd(&S.loss, w * r * r / (float)kB);
    // --- output layer gradients
    float* gW1 = S.g;
    float* gb1 = gW1 + kMlpH * kMlpIn;
    float* gW2 = gb1 + kMlpH;
    float* gb2 = gW2 + kMlpH * kMlpH;
    float* gW3 = gb2 + kMlpH;
    if (tid < kMlpH) {
      float a = 0.0f;
      for (int b = 0; b < kB; ++b) a = fmaf(S.dy[b], S.h2[b][tid], a);
      gW3[tid] = a;
    } else if (tid == kMlpH) {
      float a = 0.0f;
      for (int b = 0; b < kB; ++b) a += S.dy[b];
      gW3[kMlpH] = a;
    }
    __syncthreads();
    // delta of layer 2 (in place of h2)
    for (int i = 0; i < kMlpH; ++i)
      S.h2[tid][i] = S.h2[tid][i] > 0.0f ? S.dy[tid] * L.W3[i] : 0.0f;
    __syncthreads();
    // layer-2 weight gradients: 4096 + 64 entries over 256 threads
    for (int q = tid; q < kMlpH * kMlpH + kMlpH; q += kB) {
      float a = 0.0f;
      if (q < kMlpH * kMlpH) {
        const int i = q / kMlpH, k = q % kMlpH;
        for (int b = 0; b < kB; ++b) a = fmaf(S.h2[b][i], S.h1[b][k], a);
        gW2[q] = a;
      } else {
        const int i = q - kMlpH * kMlpH;
        for (int b = 0; b < kB; ++b) a += S.h2[b][i];
        gb2[i] = a;
      }
    }
    __syncthreads();
    // delta of layer 1 (in place of h1)
    {
      float d1[kMlpH];
      for (int k = 0; k < kMlpH; ++k) {
        float a = 0.0f;
        if (S.h1[tid][k] > 0.0f)
          for (int i = 0; i < kMlpH; ++i) a = fmaf(L.W2[i * kMlpH + k], S.h2[tid][i], a);
        d1[k] = a;
      }
      __syncthreads();
      for (int k = 0; k < kMlpH; ++k) S.h1[tid][k] = d1[k];
    }
    __syncthreads();
    for (int q = tid; q < kMlpH * kMlpIn + kMlpH; q += kB) {
      float a = 0.0f;
      if (q < kMlpH * kMlpIn) {
        const int i = q / kMlpIn, k = q % kMlpIn;
        for (int b = 0; b < kB; ++b) a = fmaf(S.h1[b][i], S.x[b][k], a);
        gW1[q] = a;
      } else {
        const int i = q - kMlpH * kMlpIn;
        for (int b = 0; b < kB; ++b) a += S.h1[b][i];
        gb1[i] = a;
      }
    }
    __syncthreads();
    // --- Adam
    b1t *= b1c;
    b2t *= b2c;
    for (int q = tid; q < kMlpParams; q += kB) {
      const float gq = S.g[q];
      const float a = b1c * m1[q] + (1.0f - b1c) * gq;
      const float v = b2c * m2[q] + (1.0f - b2c) * gq * gq;
      m1[q] = a;
      m2[q] = v;
      S.p[q] -= lr * (a / (1.0f - b1t)) / (sqrtf(v / (1.0f - b2t)) + eps);
    }
    if (tid == 0 && loss_hist && hist_every > 0 && step % hist_every == 0) loss_hist[step / hist_every] = S.loss;
    __syncthreads();
  }
  for (int q = tid; q < kMlpParams; q += kB) P[q] = S.p[q];
}

}  // namespace

cudaError_t launch_mlp_image(const float* params, void* image, cudaStream_t stream) {
  k_mlp_image<<<1, 256, 0, stream>>>(params, reinterpret_cast<MlpSmem*>(image));
  return cudaGetLastError();
}
size_t mlp_image_bytes() { return kMlpSmemBytes; }

}  // namespace gaps

using namespace gaps;

extern "C" {

int gaps_mlp_loss_grad(const float* params, const float* features, const float* targets, uint64_t n, float tau,
                       float* grad, float* loss, void* stream) {
  if (!params || !features || !targets || !grad || !loss || n == 0 || !(tau > 0.0f && tau < 1.0f))
    return GAPS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), st) != cudaSuccess) return GAPS_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return GAPS_ERR_CUDA;
  const int bs = 128;
  k_loss_grad<<<(unsigned)((n + bs - 1) / bs), bs, (kMlpParams + 1) * sizeof(float), st>>>(
      params, features, targets, n, tau, grad, loss);
  return cudaGetLastError() == cudaSuccess ? GAPS_OK : GAPS_ERR_CUDA;
}

int gaps_mlp_forward(const float* params, const float* features, uint64_t n, int bf16, float* out,
                     void* stream) {
  if (!params || !features || !out) return GAPS_ERR_INVALID_ARG;
  if (n == 0) return GAPS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (bf16) {
    uint64_t tiles = (n + 15) / 16;
    unsigned blocks = (unsigned)((tiles + 7) / 8);
    if (blocks > 4096) blocks = 4096;
    k_forward_bf16<<<blocks, 256, 0, st>>>(params, features, n, out);
  } else {
    k_forward_f32<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(params, features, n, out);
  }
  return cudaGetLastError() == cudaSuccess ? GAPS_OK : GAPS_ERR_CUDA;
}

int gaps_mlp_train(float* params, float* adam_m, float* adam_v, const float* features, const float* targets,
                   uint64_t n, uint64_t steps, float lr, float tau, uint64_t seed, float* loss_history,
                   int history_every, void* stream) {
  if (!params || !adam_m || !adam_v || !features || !targets || n == 0) return GAPS_ERR_INVALID_ARG;
  if (!(lr > 0.0f) || !(tau > 0.0f && tau < 1.0f)) return GAPS_ERR_INVALID_ARG;
  const size_t smem = sizeof(TrainSmem);
  if (cudaFuncSetAttribute(k_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GAPS_ERR_CUDA;
  k_train<<<1, kB, smem, (cudaStream_t)stream>>>(params, adam_m, adam_v, features, targets, n, steps, lr, tau,
                                                 seed, loss_history, history_every);
  return cudaGetLastError() == cudaSuccess ? GAPS_OK : GAPS_ERR_CUDA;
}

}  // extern "C"
