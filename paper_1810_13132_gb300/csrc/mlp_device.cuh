// mlp_device.cuh -- device pieces of the learned correction's MLP.
//
// The correction (not part of the paper) maps a host's feature vector to a
// log-space correction delta of the plain estimate:
//   x[80] -> GELU(W1 x + b1)[64] -> GELU(W2 h1 + b2)[64] -> w3 . h2 + b3,
// GELU in its tanh form.
// Feature definition (80 inputs): x[v] = #{registers with value v} / g for
// v = 0..63, x[64] = b/16, x[65] = ln(1 + n_plain)/16, x[66] = ln(1 + n_g)/16,
// x[67] = ln(1 + n_Z/Z), x[68] = V_Z/Z, x[69] = V/g, x[70..79] = 0.
// Registers never exceed 31, so histogram bins 32..63 are always zero: the
// kernels carry the 48 live inputs (bins 0..31, then x[64..79]) and skip the
// zero columns of W1 -- the same arithmetic as the full 80-input product.
//
// Arithmetic: BF16 inputs, weights and hidden activations fed to the tensor
// cores with mma.sync.m16n8k16 (FP32 accumulate); biases, GELU, the output
// layer and all gradients in FP32.  The matrices are 64 wide, so a warp-level
// m16n8k16 tile fits them exactly.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "packed_f32x2.cuh"

namespace vbk {

constexpr int kMlpIn = 80;       // inputs of the parameter layout
constexpr int kMlpLive = 48;     // live inputs carried by the kernels
constexpr int kMlpHid = 64;
// flat FP32 parameter vector: W1[64][80], b1[64], W2[64][64], b2[64], w3[64], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHid * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHid;
constexpr int kOffB2 = kOffW2 + kMlpHid * kMlpHid;
constexpr int kOffW3 = kOffB2 + kMlpHid;
constexpr int kOffB3 = kOffW3 + kMlpHid;
constexpr int kMlpParams = kOffB3 + 1;

// Column of W1 (80-input layout) holding live input k (0..47).
__host__ __device__ __forceinline__ int w1_col(int k) { return k < 32 ? k : k + 32; }

// BF16 weights in mma fragment order: for k-step kk and 8-column tile n, lane
// L's B fragment of W^T (two 32-bit words) is w1f[(kk * 8 + n) * 32 + L], so
// a warp reads a whole fragment with one conflict-free 8-byte load per lane.
//   layer 1: B[k][j] = W1[8n + j][w1_col(16kk + k)],  kk < 3
//   layer 2: B[k][j] = W2[8n + j][16kk + k],          kk < 4
constexpr int kW1Frags = (kMlpLive / 16) * 8 * 32;  // uint2 entries
constexpr int kW2Frags = (kMlpHid / 16) * 8 * 32;
struct MlpDevWeights {
  const uint2 *w1f;
  const uint2 *w2f;
  const float *b1, *b2, *w3, *b3;  // FP32 (global, or staged in shared memory)
};
// Padded row strides (elements) of the per-warp input and hidden tiles: 56 and
// 72 BF16 (28 and 36 words) put the 8 rows of a fragment in distinct banks.
constexpr int kXLd = 56;
constexpr int kHLd = 72;

// GELU in its tanh form, z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
// with the hardware tanh approximation (tanh.approx.f32).
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kGeluA = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float kGeluB = 0.044715f;

__device__ __forceinline__ float gelu_f(float z) {
  const float t = tanh_fast(kGeluA * z * (1.0f + kGeluB * z * z));
  return 0.5f * z * (1.0f + t);
}

// gelu_f of two values with packed FP32 arithmetic (z/2 + z/2 tanh(u)).
__device__ __forceinline__ float2 gelu_f2(float2 z) {
  const float2 in = f2_fma(f2_mul(z, z), make_float2(kGeluB, kGeluB), make_float2(1.0f, 1.0f));
  const float2 u = f2_mul(f2_mul(z, make_float2(kGeluA, kGeluA)), in);
  const float2 hz = f2_mul(z, make_float2(0.5f, 0.5f));
  return f2_fma(hz, make_float2(tanh_fast(u.x), tanh_fast(u.y)), hz);
}

__device__ __forceinline__ __nv_bfloat162 tanh_fast2(__nv_bfloat162 x) {
  uint32_t y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<uint32_t *>(&x)));
  return *reinterpret_cast<__nv_bfloat162 *>(&y);
}

// GELU (tanh form) of a BF16 pair in BF16 arithmetic.
__device__ __forceinline__ __nv_bfloat162 gelu_bf16x2(__nv_bfloat162 z) {
  const __nv_bfloat162 a = __float2bfloat162_rn(kGeluA), b = __float2bfloat162_rn(kGeluB);
  const __nv_bfloat162 one = __float2bfloat162_rn(1.0f), half = __float2bfloat162_rn(0.5f);
  const __nv_bfloat162 u = __hmul2(__hmul2(a, z), __hfma2(__hmul2(b, z), z, one));
  const __nv_bfloat162 t = tanh_fast2(u);
  return __hmul2(__hmul2(half, z), __hadd2(one, t));
}

__device__ __forceinline__ float gelu_grad_f(float z) {
  const float t = tanh_fast(kGeluA * z * (1.0f + kGeluB * z * z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluA * (1.0f + 3.0f * kGeluB * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A(16x16, row) * B(16x8, col) + D, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment loaders for m16n8k16.  With g = lane / 4 and c = 2 (lane % 4):
//   A regs: (g, c..c+1), (g+8, c..c+1), (g, c+8..c+9), (g+8, c+8..c+9)
//   B regs: (k = c..c+1, n = g), (k = c+8..c+9, n = g)
//   C regs: (g, c), (g, c+1), (g+8, c), (g+8, c+1)
// AT(r, k) and BT(k, n) return the BF16 element of the 16x16 / 16x8 tile.
template <class AT>
__device__ __forceinline__ void load_a(uint32_t (&a)[4], AT at) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = (lane & 3) * 2;
  a[0] = pack_bf16(at(g, c), at(g, c + 1));
  a[1] = pack_bf16(at(g + 8, c), at(g + 8, c + 1));
  a[2] = pack_bf16(at(g, c + 8), at(g, c + 9));
  a[3] = pack_bf16(at(g + 8, c + 8), at(g + 8, c + 9));
}

template <class BT>
__device__ __forceinline__ void load_b(uint32_t (&b)[2], BT bt) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = (lane & 3) * 2;
  b[0] = pack_bf16(bt(c, g), bt(c + 1, g));
  b[1] = pack_bf16(bt(c + 8, g), bt(c + 9, g));
}

// A fragment of a row-major BF16 tile (leading dimension ld elements) whose
// top-left corner is t: pairs of consecutive columns read as 32-bit words.
__device__ __forceinline__ void load_a_tile(uint32_t (&a)[4], const __nv_bfloat16 *t, int ld) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = (lane & 3) * 2;
  a[0] = *reinterpret_cast<const uint32_t *>(t + g * ld + c);
  a[1] = *reinterpret_cast<const uint32_t *>(t + (g + 8) * ld + c);
  a[2] = *reinterpret_cast<const uint32_t *>(t + g * ld + c + 8);
  a[3] = *reinterpret_cast<const uint32_t *>(t + (g + 8) * ld + c + 8);
}

// Forward of 32 rows by one warp, one 16-row tile at a time (32 FP32
// accumulators live instead of 64, for occupancy).  xs: the rows' live
// inputs, BF16 [32][kXLd] (first kMlpLive columns used); h1s: scratch BF16
// [16][kHLd] (one tile's hidden layer).  Returns delta of row (lane) in every
// lane.
__device__ __forceinline__ float mlp_forward_warp(const __nv_bfloat16 *xs,
                                                  __nv_bfloat16 *h1s,
                                                  const MlpDevWeights &w) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = (lane & 3) * 2;
  float part[2][2];  // [tile][row g / g+8]
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    float acc[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
    // layer 1: [16 x 48] x [48 x 64]
#pragma unroll
    for (int kk = 0; kk < kMlpLive / 16; ++kk) {
      uint32_t a[4];
      load_a_tile(a, xs + 16 * m * kXLd + 16 * kk, kXLd);
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const uint2 f = w.w1f[(kk * 8 + n) * 32 + lane];
        const uint32_t b[2] = {f.x, f.y};
        mma_bf16(acc[n], a, b);
      }
    }
    // bias + GELU -> h1 (BF16; its GELU runs on packed BF16 pairs)
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = g + 8 * h, j = 8 * n + c;
        const __nv_bfloat162 z = __floats2bfloat162_rn(acc[n][2 * h] + w.b1[j],
                                                       acc[n][2 * h + 1] + w.b1[j + 1]);
        *reinterpret_cast<__nv_bfloat162 *>(h1s + r * kHLd + j) = gelu_bf16x2(z);
      }
    __syncwarp();
    // layer 2: [16 x 64] x [64 x 64]
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
#pragma unroll
    for (int kk = 0; kk < kMlpHid / 16; ++kk) {
      uint32_t a[4];
      load_a_tile(a, h1s + 16 * kk, kHLd);
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const uint2 f = w.w2f[(kk * 8 + n) * 32 + lane];
        const uint32_t b[2] = {f.x, f.y};
        mma_bf16(acc[n], a, b);
      }
    }
    __syncwarp();  // h1s is rewritten by the next tile
    // output layer in FP32, two columns (j, j + 1) per packed instruction:
    // delta_r = sum_j GELU(z2[r][j]) w3[j] + b3
    float2 pp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // rows g, g + 8
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int j = 8 * n + c;
      const float2 b2 = *reinterpret_cast<const float2 *>(w.b2 + j);
      const float2 w3 = *reinterpret_cast<const float2 *>(w.w3 + j);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        pp[h] = f2_fma(gelu_f2(f2_add(make_float2(acc[n][2 * h], acc[n][2 * h + 1]), b2)), w3,
                       pp[h]);
    }
    part[m][0] = pp[0].x + pp[0].y;
    part[m][1] = pp[1].x + pp[1].y;
  }
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      part[m][h] += __shfl_xor_sync(0xffffffffu, part[m][h], 1);
      part[m][h] += __shfl_xor_sync(0xffffffffu, part[m][h], 2);
    }
  // row r lives in lanes 4*(r % 8) .. +3: tile r / 16, half (r / 8) % 2
  const int src = 4 * (lane & 7);
  const float d0 = __shfl_sync(0xffffffffu, part[0][0], src);
  const float d1 = __shfl_sync(0xffffffffu, part[0][1], src);
  const float d2 = __shfl_sync(0xffffffffu, part[1][0], src);
  const float d3 = __shfl_sync(0xffffffffu, part[1][1], src);
  const int slot = lane >> 3;
  const float delta = slot == 0 ? d0 : slot == 1 ? d1 : slot == 2 ? d2 : d3;
  __syncwarp();
  return delta + *w.b3;
}

}  // namespace vbk
