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
// cores (FP32 accumulate); biases, GELU, the output layer and all gradients
// in FP32.  Inference runs on tcgen05 (128-row tiles, accumulators in tensor
// memory); training uses warp-level mma.sync.m16n8k16 tiles, whose 64-wide
// matrices fit a warp exactly.
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

// Inference weights: BF16 W1 (live columns) and W2, row-major [64][48] and
// [64][64] (row = hidden unit, so each is the K-major B operand of its
// layer), FP32 biases and output weights, and a device error word.
struct MlpDevWeights {
  const __nv_bfloat16 *w1c, *w2;
  const float *b1, *b2, *w3, *b3;
  unsigned int *err;
};

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

}  // namespace vbk
