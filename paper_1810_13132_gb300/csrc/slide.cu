// slide.cu -- slice boundary over the whole BDR pool (Sec. 3, Sec. 4.2).
//
//   gfast : Alg. 6 -- every DR slides (saturating +1), the DR of the highest
//           set bit of bsLBP1 is set to 0, bsLBP1 is cleared; then Alg. 2
//           reads the register (largest LBP1 whose DR is below k, else 0).
//   gsmall: Alg. 2 reads the register of the window that just closed, then
//           Alg. 8 slides every DR for the next slice.
// Fused into the same pass: the register array and the pool sums
// S_Z = sum_j 2^(32 - reg_j), V_Z = #{reg_j = 0} that the estimator needs
// for its noise term.  Exact 64-bit integer sums: the result does not depend
// on the reduction order.
//
// One thread per BDR, grid-stride; each DRV plane is a coalesced 4-byte
// stream.  The saturating increment is SWAR: a field is incremented unless
// all its w bits are set, so no carry ever crosses a field.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kSlideThreads = 256;

template <int W>
struct Fields {
  static constexpr uint32_t F = 32 / W;                       // fields per word
  static constexpr uint32_t FM = (1u << W) - 1u;              // one field
  static constexpr uint32_t PMAX = (31 + F - 1) / F;          // R <= 31
  static constexpr uint32_t lsb_mask() {
    uint32_t m = 0;
    for (uint32_t f = 0; f < F; ++f) m |= 1u << (f * W);
    return m;
  }
};

// Saturating +1 of every field of one word (fields past R hold DR_MAX and
// stay there).
template <int W>
__device__ __forceinline__ uint32_t sat_inc(uint32_t x) {
  constexpr uint32_t L = Fields<W>::lsb_mask();
  uint32_t all = x;
#pragma unroll
  for (int sft = 1; sft < W; ++sft) all &= x >> sft;
  return x + (L & ~all);
}

// Largest r in 1..R with DR[r] < k, else 0 (Alg. 2).
template <int W>
__device__ __forceinline__ uint32_t register_of(const uint32_t *words,
                                                uint32_t P, uint32_t R,
                                                uint32_t k) {
  constexpr uint32_t F = Fields<W>::F;
  uint32_t reg = 0;
#pragma unroll
  for (uint32_t p = 0; p < Fields<W>::PMAX; ++p) {
    if (p < P) {
#pragma unroll
      for (uint32_t f = 0; f < F; ++f) {
        const uint32_t r = p * F + f + 1;
        const uint32_t dr = (words[p] >> (f * W)) & Fields<W>::FM;
        if (r <= R && dr < k) reg = r;
      }
    }
  }
  return reg;
}

template <int W, bool GFAST>
__global__ void __launch_bounds__(kSlideThreads)
    slide_kernel(Dims d, DevState s) {
  constexpr uint32_t PMAX = Fields<W>::PMAX;
  constexpr uint32_t F = Fields<W>::F;
  unsigned long long S = 0, V = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d.Z;
       j += stride) {
    uint32_t w0[PMAX], w1[PMAX];
#pragma unroll
    for (uint32_t p = 0; p < PMAX; ++p)
      w0[p] = (p < d.P) ? __ldcs(s.drv + (uint64_t)p * d.Z + j) : 0u;
    uint32_t reg;
    if constexpr (GFAST) {
#pragma unroll
      for (uint32_t p = 0; p < PMAX; ++p) w1[p] = sat_inc<W>(w0[p]);
      const uint32_t bsv = __ldcs(s.bs + j);
      if (bsv) {
        const uint32_t r0 = 31u - (uint32_t)__clz(bsv);  // LBP1 - 1 of the top bit
        const uint32_t pw = r0 / F;
        const uint32_t clear = ~(Fields<W>::FM << ((r0 % F) * W));
#pragma unroll
        for (uint32_t p = 0; p < PMAX; ++p)
          if (p == pw) w1[p] &= clear;
        __stcs(s.bs + j, 0u);
      }
      reg = register_of<W>(w1, d.P, d.R, d.k);
    } else {
      reg = register_of<W>(w0, d.P, d.R, d.k);
#pragma unroll
      for (uint32_t p = 0; p < PMAX; ++p) w1[p] = sat_inc<W>(w0[p]);
    }
#pragma unroll
    for (uint32_t p = 0; p < PMAX; ++p)
      if (p < d.P && w1[p] != w0[p]) __stcs(s.drv + (uint64_t)p * d.Z + j, w1[p]);
    s.reg[j] = (uint8_t)reg;
    S += 1ull << (32u - reg);
    V += (reg == 0u);
  }
  // block reduction of the pool sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_down_sync(0xffffffffu, S, o);
    V += __shfl_down_sync(0xffffffffu, V, o);
  }
  __shared__ unsigned long long sS[kSlideThreads / 32], sV[kSlideThreads / 32];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { sS[warp] = S; sV[warp] = V; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t i = 1; i < blockDim.x / 32; ++i) { S += sS[i]; V += sV[i]; }
    atomicAdd(&s.sums[3], S);
    atomicAdd(&s.sums[4], V);
    __threadfence();
    // The last block to finish publishes the totals and resets the partials
    // for the next slide (the counter pattern keeps the slide one launch).
    const unsigned long long done = atomicAdd(&s.sums[2], 1ull);
    if (done == gridDim.x - 1) {
      __threadfence();
      s.sums[0] = atomicExch(&s.sums[3], 0ull);
      s.sums[1] = atomicExch(&s.sums[4], 0ull);
      s.sums[2] = 0ull;
    }
  }
}

template <int W>
cudaError_t launch_slide_t(const Dims &d, const DevState &s, bool gfast,
                           cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (gfast)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slide_kernel<W, true>, kSlideThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slide_kernel<W, false>, kSlideThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = (d.Z + kSlideThreads - 1) / kSlideThreads;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want;
  if (gfast)
    slide_kernel<W, true><<<(unsigned)grid, kSlideThreads, 0, st>>>(d, s);
  else
    slide_kernel<W, false><<<(unsigned)grid, kSlideThreads, 0, st>>>(d, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_slide(const Dims &d, const DevState &s, bool gfast,
                         cudaStream_t st) {
  switch (d.w) {
    case 1: return launch_slide_t<1>(d, s, gfast, st);
    case 2: return launch_slide_t<2>(d, s, gfast, st);
    case 3: return launch_slide_t<3>(d, s, gfast, st);
    case 4: return launch_slide_t<4>(d, s, gfast, st);
    case 5: return launch_slide_t<5>(d, s, gfast, st);
    case 6: return launch_slide_t<6>(d, s, gfast, st);
    case 7: return launch_slide_t<7>(d, s, gfast, st);
    case 8: return launch_slide_t<8>(d, s, gfast, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vbk
