// mlp_device.cuh -- device pieces of the learned correction's MLP.
//
// The correction (not part of the paper) maps a host's feature vector to a
// log-space correction delta of the plain estimate:
//   x[80] -> GELU(W1 x + b1)[64] -> GELU(W2 h1 + b2)[64] -> w3 . h2 + b3.
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

// BF16 copies of the weights in the layouts the kernels read:
//   w1c[n][k] = W1[n][w1_col(k)]  (64 x 48),  w2[n][j] = W2[n][j]  (64 x 64)
struct MlpDevWeights {
  const __nv_bfloat16 *w1c;
  const __nv_bfloat16 *w2;
  const float *theta;  // FP32 master (biases and w3 are read from here)
};

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * __expf(-0.5f * z * z) * 0.39894228040143268f;
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

// Forward of 32 rows by one warp.  xs: the rows' live inputs, BF16
// [32][kMlpLive]; h1s: scratch BF16 [32][kMlpHid] (may alias nothing else).
// Returns delta of row (lane) in every lane.  z2 / h2 stay in registers.
__device__ __forceinline__ float mlp_forward_warp(const __nv_bfloat16 *xs,
                                                  __nv_bfloat16 *h1s,
                                                  const MlpDevWeights &w) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = (lane & 3) * 2;
  // layer 1: [32 x 48] x [48 x 64]
  float acc[2][8][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll
  for (int kk = 0; kk < kMlpLive / 16; ++kk) {
    uint32_t a[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
      load_a(a[m], [&](int r, int k) { return xs[(16 * m + r) * kMlpLive + 16 * kk + k]; });
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      uint32_t b[2];
      load_b(b, [&](int k, int j) { return w.w1c[(8 * n + j) * kMlpLive + 16 * kk + k]; });
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][n], a[m], b);
    }
  }
  // bias + GELU -> h1 (BF16) in shared memory
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 16 * m + g + (q >> 1) * 8, j = 8 * n + c + (q & 1);
        h1s[r * kMlpHid + j] = __float2bfloat16(gelu_f(acc[m][n][q] + w.theta[kOffB1 + j]));
      }
  __syncwarp();
  // layer 2: [32 x 64] x [64 x 64]
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll
  for (int kk = 0; kk < kMlpHid / 16; ++kk) {
    uint32_t a[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
      load_a(a[m], [&](int r, int k) { return h1s[(16 * m + r) * kMlpHid + 16 * kk + k]; });
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      uint32_t b[2];
      load_b(b, [&](int k, int j) { return w.w2[(8 * n + j) * kMlpHid + 16 * kk + k]; });
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][n], a[m], b);
    }
  }
  // output layer in FP32: delta_r = sum_j GELU(z2[r][j]) w3[j] + b3
  float part[4] = {0.f, 0.f, 0.f, 0.f};  // rows g, g+8, 16+g, 24+g
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 8 * n + c + (q & 1);
        part[2 * m + (q >> 1)] += gelu_f(acc[m][n][q] + w.theta[kOffB2 + j]) * w.theta[kOffW3 + j];
      }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    part[i] += __shfl_xor_sync(0xffffffffu, part[i], 1);
    part[i] += __shfl_xor_sync(0xffffffffu, part[i], 2);
  }
  // row r lives in lanes 4*(r % 8) .. +3, slot (r / 8)
  const int src = 4 * (lane & 7);
  const float d0 = __shfl_sync(0xffffffffu, part[0], src);
  const float d1 = __shfl_sync(0xffffffffu, part[1], src);
  const float d2 = __shfl_sync(0xffffffffu, part[2], src);
  const float d3 = __shfl_sync(0xffffffffu, part[3], src);
  const int slot = lane >> 3;
  const float delta = slot == 0 ? d0 : slot == 1 ? d1 : slot == 2 ? d2 : d3;
  __syncwarp();
  return delta + w.theta[kOffB3];
}

}  // namespace vbk
