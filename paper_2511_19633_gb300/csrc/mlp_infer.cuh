// Inference of the learned-proposal network (4 -> 64 -> 64 -> 1, ReLU) on
// tensor cores: BF16 weights and activations, FP32 accumulation, one warp per
// tile of 16 rows with mma.sync.m16n8k16. The accumulator fragments of a
// layer are repacked in registers as the A fragments of the next one.
//
// Parameter layout (FP32, 4545 values): W1 [64][4], b1 [64], W2 [64][64],
// b2 [64], W3 [64], b3.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace gaps {

constexpr int kMlpIn = 4, kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;
constexpr int kIsrClasses = 44, kIsrBins = 8, kEtaBins = 8;
// buckets of the first network input f0 = ln(eta)/7 + 1 for the calibration
// margins; the upper edges are eta = 1e-5, 1e-4, 1e-3, 1e-2, 0.1, 0.4, 0.7
__device__ __forceinline__ int eta_bucket(float f0) {
  const float edge[kEtaBins - 1] = {-0.6447f, -0.3158f, 0.0132f, 0.3421f, 0.6711f, 0.8691f, 0.9490f};
  int b = 0;
#pragma unroll
  for (int k = 0; k < kEtaBins - 1; ++k) b += f0 >= edge[k] ? 1 : 0;
  return b;
}

// shared-memory image, weights stored [n][k] so that the B fragment of
// m16n8k16 (k = 2t, 2t+1 and 2t+8, 2t+9 of column n = g) is two 32-bit loads.
// Rows are padded by 8 values: a row stride of 4 (mod 32) banks puts the 32
// lanes' loads of one fragment (8 rows g x 4 column pairs t) in 32 banks.
constexpr int kPad = 8;
struct MlpSmem {
  __nv_bfloat16 w1[kMlpH][16 + kPad];     // k padded from 4 to 16 with zeros
  __nv_bfloat16 w2[kMlpH][kMlpH + kPad];
  __nv_bfloat16 w3[8][kMlpH + kPad];      // output row 0; rows 1..7 zero
  float b1[kMlpH], b2[kMlpH], b3;
};
constexpr size_t kMlpSmemBytes = (sizeof(MlpSmem) + 15) / 16 * 16;

// cooperative fill of the image from FP32 parameters (all threads of a block)
__device__ inline void mlp_load_smem(MlpSmem& S, const float* P) {
  const float* W1 = P;
  const float* b1 = W1 + kMlpH * kMlpIn;
  const float* W2 = b1 + kMlpH;
  const float* b2 = W2 + kMlpH * kMlpH;
  const float* W3 = b2 + kMlpH;
  for (int q = threadIdx.x; q < kMlpH * 16; q += blockDim.x) {
    int n = q / 16, k = q % 16;
    S.w1[n][k] = __float2bfloat16_rn(k < kMlpIn ? W1[n * kMlpIn + k] : 0.0f);
  }
  for (int q = threadIdx.x; q < kMlpH * kMlpH; q += blockDim.x)
    S.w2[q / kMlpH][q % kMlpH] = __float2bfloat16_rn(W2[q]);
  for (int q = threadIdx.x; q < 8 * kMlpH; q += blockDim.x) {
    int n = q / kMlpH, k = q % kMlpH;
    S.w3[n][k] = __float2bfloat16_rn(n == 0 ? W3[k] : 0.0f);
  }
  for (int q = threadIdx.x; q < kMlpH; q += blockDim.x) { S.b1[q] = b1[q]; S.b2[q] = b2[q]; }
  if (threadIdx.x == 0) S.b3 = W3[kMlpH];
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One warp evaluates 16 rows: feat[r][0..3] -> out[r] (both in shared or
// global memory visible to the warp). All 32 lanes must call it. Layer 1 is
// kept as packed BF16 A fragments (16 registers); layers 2 and 3 are
// interleaved: the two layer-2 column tiles that form k-step j of layer 3 are
// computed, rectified, packed and consumed at once.
static __device__ __noinline__ void mlp_tile(const MlpSmem& S, const float (*feat)[4], float* out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  // layer 1: K = 16 (features 0..3, zero padding)
  a[0] = t < 2 ? pack_bf16(feat[g][2 * t], feat[g][2 * t + 1]) : 0u;
  a[1] = t < 2 ? pack_bf16(feat[g + 8][2 * t], feat[g + 8][2 * t + 1]) : 0u;
  a[2] = 0u;
  a[3] = 0u;
  uint32_t A1[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float h[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int nt = 2 * j + u, n = nt * 8 + g;
      h[u][0] = S.b1[nt * 8 + 2 * t];
      h[u][1] = S.b1[nt * 8 + 2 * t + 1];
      h[u][2] = h[u][0];
      h[u][3] = h[u][1];
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w1[n][2 * t]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w1[n][2 * t + 8]);
      mma16816(h[u], a, b0, b1);
    }
    A1[j][0] = pack_bf16(fmaxf(h[0][0], 0.0f), fmaxf(h[0][1], 0.0f));
    A1[j][1] = pack_bf16(fmaxf(h[0][2], 0.0f), fmaxf(h[0][3], 0.0f));
    A1[j][2] = pack_bf16(fmaxf(h[1][0], 0.0f), fmaxf(h[1][1], 0.0f));
    A1[j][3] = pack_bf16(fmaxf(h[1][2], 0.0f), fmaxf(h[1][3], 0.0f));
  }
  // layers 2 and 3: N = 8 for layer 3 (column 0 is the output), K = 64. The
  // k-step loop of layer 3 stays rolled: the tile runs inside the shower's
  // warp-cooperative rebuild, where instruction-cache footprint costs more
  // than the loop overhead.
  float o[4] = {S.b3, S.b3, S.b3, S.b3};
#pragma unroll 1
  for (int j3 = 0; j3 < 4; ++j3) {
    float h[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int nt = 2 * j3 + u, n = nt * 8 + g;
      h[u][0] = S.b2[nt * 8 + 2 * t];
      h[u][1] = S.b2[nt * 8 + 2 * t + 1];
      h[u][2] = h[u][0];
      h[u][3] = h[u][1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w2[n][16 * j + 2 * t]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w2[n][16 * j + 8 + 2 * t]);
        mma16816(h[u], A1[j], b0, b1);
      }
    }
    const uint32_t A3[4] = {pack_bf16(fmaxf(h[0][0], 0.0f), fmaxf(h[0][1], 0.0f)),
                            pack_bf16(fmaxf(h[0][2], 0.0f), fmaxf(h[0][3], 0.0f)),
                            pack_bf16(fmaxf(h[1][0], 0.0f), fmaxf(h[1][1], 0.0f)),
                            pack_bf16(fmaxf(h[1][2], 0.0f), fmaxf(h[1][3], 0.0f))};
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w3[g][16 * j3 + 2 * t]);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w3[g][16 * j3 + 8 + 2 * t]);
    mma16816(o, A3, b0, b1);
  }
  if (t == 0) {
    out[g] = o[0];
    out[g + 8] = o[2];
  }
  __syncwarp();
}

// NT 16-row tiles at once (rows feat[0 .. 16 NT) -> out): every weight
// fragment is loaded once and feeds the NT tiles' mma's, so their tensor-core
// work interleaves. For the dense pass; the same numerics as mlp_tile, row by
// row.
template <int NT>
__device__ __noinline__ void mlp_tiles(const MlpSmem& S, const float (*feat)[4], float* out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t X[NT][2];  // layer-1 inputs (K = 16: features 0..3, zero padding)
#pragma unroll
  for (int tt = 0; tt < NT; ++tt) {
    const float (*f)[4] = feat + 16 * tt;
    X[tt][0] = t < 2 ? pack_bf16(f[g][2 * t], f[g][2 * t + 1]) : 0u;
    X[tt][1] = t < 2 ? pack_bf16(f[g + 8][2 * t], f[g + 8][2 * t + 1]) : 0u;
  }
  uint32_t A1[NT][4][4];  // [tile][k-step of layer 2][fragment]
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int nt = 2 * j + u, n = nt * 8 + g;
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w1[n][2 * t]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w1[n][2 * t + 8]);
      const float c0 = S.b1[nt * 8 + 2 * t], c1 = S.b1[nt * 8 + 2 * t + 1];
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        const uint32_t a[4] = {X[tt][0], X[tt][1], 0u, 0u};
        float h[4] = {c0, c1, c0, c1};
        mma16816(h, a, b0, b1);
        A1[tt][j][2 * u] = pack_bf16(fmaxf(h[0], 0.0f), fmaxf(h[1], 0.0f));
        A1[tt][j][2 * u + 1] = pack_bf16(fmaxf(h[2], 0.0f), fmaxf(h[3], 0.0f));
      }
    }
  }
  // layers 2 and 3, k-step j3 of layer 3 = column tiles 2 j3, 2 j3 + 1 of layer 2
  float o[NT][4];
#pragma unroll
  for (int tt = 0; tt < NT; ++tt) o[tt][0] = o[tt][1] = o[tt][2] = o[tt][3] = S.b3;
#pragma unroll 1
  for (int j3 = 0; j3 < 4; ++j3) {
    float h[NT][2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int nt = 2 * j3 + u, n = nt * 8 + g;
      const float c0 = S.b2[nt * 8 + 2 * t], c1 = S.b2[nt * 8 + 2 * t + 1];
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        h[tt][u][0] = c0;
        h[tt][u][1] = c1;
        h[tt][u][2] = c0;
        h[tt][u][3] = c1;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w2[n][16 * j + 2 * t]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w2[n][16 * j + 8 + 2 * t]);
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) mma16816(h[tt][u], A1[tt][j], b0, b1);
      }
    }
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w3[g][16 * j3 + 2 * t]);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w3[g][16 * j3 + 8 + 2 * t]);
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      const uint32_t A3[4] = {pack_bf16(fmaxf(h[tt][0][0], 0.0f), fmaxf(h[tt][0][1], 0.0f)),
                              pack_bf16(fmaxf(h[tt][0][2], 0.0f), fmaxf(h[tt][0][3], 0.0f)),
                              pack_bf16(fmaxf(h[tt][1][0], 0.0f), fmaxf(h[tt][1][1], 0.0f)),
                              pack_bf16(fmaxf(h[tt][1][2], 0.0f), fmaxf(h[tt][1][3], 0.0f))};
      mma16816(o[tt], A3, b0, b1);
    }
  }
  if (t == 0) {
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      out[16 * tt + g] = o[tt][0];
      out[16 * tt + g + 8] = o[tt][2];
    }
  }
  __syncwarp();
}

}  // namespace gaps
