// slide.cu -- slice boundary over the whole BDR pool (Sec. 3, Sec. 4.2).
//
//   gfast : Alg. 6 -- every DR slides (saturating +1), the DR of the highest
//           set bit of bsLBP1 is set to 0, bsLBP1 is cleared; then Alg. 2
//           reads the register (largest LBP1 whose DR is below k, else 0).
//   serial: Alg. 1 -- the same with nowLBP1 (the slice's largest LBP1)
//           instead of the highest bit of bsLBP1; nowLBP1 is cleared.
//   gsmall: Alg. 2 reads the register of the window that just closed, then
//           Alg. 8 slides every DR for the next slice.
// Fused into the same pass: the register array and the pool sums
// S_Z = sum_j 2^(32 - reg_j), V_Z = #{reg_j = 0} that the estimator needs
// for its noise term.  Exact 64-bit integer sums: the result does not depend
// on the reduction order.
//
// Streaming layout: each thread owns 4 consecutive BDRs and moves them with
// 16-byte accesses -- one uint4 per DRV plane, one uint4 of bsLBP1, one
// 4-byte store of the 4 registers -- so a warp moves 512 contiguous bytes
// per plane.  The field arithmetic is SWAR on whole words, both tests built
// on one carry-masked add (every field's low w-1 bits, top bits off, so no
// carry leaves a field):
//   saturating +1 : a field is incremented unless all its w bits are set;
//   active test   : DR >= k (inactive) exactly when DR + 2^w - k carries out
//                   of the field.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kSlideThreads = 256;

template <int W>
struct Fields {
  static constexpr uint32_t F = 32 / W;           // fields per word
  static constexpr uint32_t FM = (1u << W) - 1u;  // one field
  static constexpr uint32_t lsb() {      // the lowest bit of every field
    uint32_t m = 0;
    for (uint32_t f = 0; f < F; ++f) m |= 1u << (f * W);
    return m;
  }
  static constexpr uint32_t LSB = lsb();
};

// Saturating +1 of every field of one word.  A field is all ones exactly
// when adding 1 to its low W-1 bits carries into its top bit while that top
// bit is set: with the top bits masked off first, no carry leaves a field.
template <int W>
__device__ __forceinline__ uint32_t sat_inc(uint32_t x) {
  constexpr uint32_t L = Fields<W>::LSB, H = L << (W - 1);
  const uint32_t full = ((x & ~H) + L) & x & H;  // top bit of every all-ones field
  return x + (L ^ (full >> (W - 1)));
}

// The test DR < k (an active DR) on every field at once.  With c = 2^W - k,
// a field holds at least k exactly when x_f + c carries out of the field.
// The low W-1 bits of every field are added with the top bits masked off
// (no carry leaves a field), which gives the carry into each top bit; the
// carry out is then the majority of that carry, the field's top bit and
// c's top bit.  KTest holds c's low bits replicated into every field and
// the field tops if c's top bit is set (else 0).
struct KTest {
  uint32_t cl;  // (c mod 2^(W-1)) in every field
  uint32_t cm;  // every field's top bit if c >= 2^(W-1), else 0
};

// Top bit f*W + W - 1 set for every field f of x with value < k.
template <int W>
__device__ __forceinline__ uint32_t active_fields(uint32_t x, KTest kt) {
  constexpr uint32_t H = Fields<W>::LSB << (W - 1);
  const uint32_t t = (x & ~H) + kt.cl;
  const uint32_t carry = (x & t) | (kt.cm & (x | t));
  return H & ~carry;
}

// Alg. 2 on one BDR whose P words are w[0..P): the largest LBP1 r in 1..R
// with DR[r] < k, else 0.  Fields past R hold 2^w - 1 >= k: never active.
template <int W, int P>
__device__ __forceinline__ uint32_t register_of(const uint32_t (&w)[P], KTest kt) {
  uint32_t reg = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t a = active_fields<W>(w[p], kt);
    if (a) reg = (uint32_t)p * Fields<W>::F + (31u - (uint32_t)__clz(a)) / W + 1u;
  }
  return reg;
}

// gfast: zero the DR of the highest set bit of bsLBP1 (Alg. 6).
template <int W, int PMAX>
__device__ __forceinline__ void set_dr_of_top_bit(uint32_t (&w)[PMAX], uint32_t bsv) {
  if (bsv) {
    const uint32_t r0 = 31u - (uint32_t)__clz(bsv);  // LBP1 - 1
    const uint32_t pw = r0 / Fields<W>::F;
    const uint32_t clear = ~(Fields<W>::FM << ((r0 % Fields<W>::F) * W));
#pragma unroll
    for (int p = 0; p < PMAX; ++p)
      if ((uint32_t)p == pw) w[p] &= clear;
  }
}

// PCSA statistic of one BDR (gsmall: DR[r] active iff LBP1 r was seen in the
// window, a bitmap): the number of active DRs from LBP1 1 up to the first
// inactive one, i.e. the index of the bitmap's lowest unset position.
// Fields past R are never active, so the count stops at R.
template <int W, int P>
__device__ __forceinline__ uint32_t pcsa_of(const uint32_t (&w)[P], KTest kt) {
  uint32_t n = 0;
  bool run = true;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t inactive = ~active_fields<W>(w[p], kt) & (Fields<W>::LSB << (W - 1));
    if (run) {
      if (inactive) {
        n += (uint32_t)(__ffs(inactive) - 1) / W;
        run = false;
      } else {
        n += Fields<W>::F;
      }
    }
  }
  return n;
}

template <int W, int P, bool GFAST>
__device__ __forceinline__ uint32_t slide_one(uint32_t (&w)[P], uint32_t bsv,
                                              KTest kt, uint32_t *pcsa) {
  if constexpr (GFAST) {
#pragma unroll
    for (int p = 0; p < P; ++p) w[p] = sat_inc<W>(w[p]);
    set_dr_of_top_bit<W, P>(w, bsv);
    return register_of<W, P>(w, kt);
  } else {
    const uint32_t reg = register_of<W, P>(w, kt);
    *pcsa = pcsa_of<W, P>(w, kt);
#pragma unroll
    for (int p = 0; p < P; ++p) w[p] = sat_inc<W>(w[p]);
    return reg;
  }
}

__device__ __forceinline__ uint32_t comp(const uint4 &v, int c) {
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_comp(uint4 &v, int c, uint32_t x) {
  if (c == 0) v.x = x; else if (c == 1) v.y = x; else if (c == 2) v.z = x; else v.w = x;
}

// LAY: kLayoutGfast / kLayoutGsmall / kLayoutSerial
template <int W, int P, int LAY>
__global__ void __launch_bounds__(kSlideThreads)
    slide_kernel(Dims d, DevState s, KTest kt) {
  constexpr bool GFAST = LAY != kLayoutGsmall;  // fold a slice maximum (Alg. 1 / 6)
  unsigned long long S = 0, V = 0, L = 0, Pc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t quads = d.Z >> 2;
  for (uint64_t q = tid; q < quads; q += stride) {
    const uint64_t j = q << 2;
    uint4 v[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      v[p] = __ldcs(reinterpret_cast<const uint4 *>(s.drv + (uint64_t)p * d.Zs + j));
    uint4 bsq = make_uint4(0, 0, 0, 0);
    if constexpr (LAY == kLayoutGfast) bsq = __ldcs(reinterpret_cast<const uint4 *>(s.bs + j));
    if constexpr (LAY == kLayoutSerial) {
      // nowLBP1 of the 4 BDRs as the bit of that LBP1, so Alg. 1 and Alg. 6
      // share the fold
      const uint32_t nw = __ldcs(reinterpret_cast<const uint32_t *>(s.now + j));
      bsq = make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t nv = (nw >> (8 * c)) & 0xffu;
        set_comp(bsq, c, nv ? 1u << (nv - 1u) : 0u);
      }
    }
    uint32_t regs = 0, pcs = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t w[P];
#pragma unroll
      for (int p = 0; p < P; ++p) w[p] = comp(v[p], c);
      uint32_t pc = 0;
      const uint32_t reg = slide_one<W, P, GFAST>(w, comp(bsq, c), kt, &pc);
#pragma unroll
      for (int p = 0; p < P; ++p) set_comp(v[p], c, w[p]);
      regs |= reg << (8 * c);
      pcs |= pc << (8 * c);
      S += 1ull << (32u - reg);
      V += (reg == 0u);
      L += reg;
      Pc += pc;
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
      __stcs(reinterpret_cast<uint4 *>(s.drv + (uint64_t)p * d.Zs + j), v[p]);
    if constexpr (LAY == kLayoutGfast) {
      if (bsq.x | bsq.y | bsq.z | bsq.w)
        __stcs(reinterpret_cast<uint4 *>(s.bs + j), make_uint4(0, 0, 0, 0));
    }
    if constexpr (LAY == kLayoutSerial) {
      if (bsq.x | bsq.y | bsq.z | bsq.w) __stcs(reinterpret_cast<uint32_t *>(s.now + j), 0u);
    }
    __stcs(reinterpret_cast<uint32_t *>(s.reg + j), regs);
    if constexpr (LAY == kLayoutGsmall) __stcs(reinterpret_cast<uint32_t *>(s.pcsa + j), pcs);
  }
  // the last Z mod 4 BDRs, one thread each
  if (tid < (d.Z & 3u)) {
    const uint64_t j = (quads << 2) + tid;
    uint32_t w[P];
#pragma unroll
    for (int p = 0; p < P; ++p) w[p] = s.drv[(uint64_t)p * d.Zs + j];
    uint32_t bsv = 0u;
    if constexpr (LAY == kLayoutGfast) bsv = s.bs[j];
    if constexpr (LAY == kLayoutSerial) bsv = s.now[j] ? 1u << (s.now[j] - 1u) : 0u;
    uint32_t pc = 0;
    const uint32_t reg = slide_one<W, P, GFAST>(w, bsv, kt, &pc);
#pragma unroll
    for (int p = 0; p < P; ++p) s.drv[(uint64_t)p * d.Zs + j] = w[p];
    if (LAY == kLayoutGfast && bsv) s.bs[j] = 0u;
    if (LAY == kLayoutSerial && bsv) s.now[j] = 0u;
    s.reg[j] = (uint8_t)reg;
    if (LAY == kLayoutGsmall) s.pcsa[j] = (uint8_t)pc;
    S += 1ull << (32u - reg);
    V += (reg == 0u);
    L += reg;
    Pc += pc;
  }
  // block reduction of the pool sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_down_sync(0xffffffffu, S, o);
    V += __shfl_down_sync(0xffffffffu, V, o);
    L += __shfl_down_sync(0xffffffffu, L, o);
    Pc += __shfl_down_sync(0xffffffffu, Pc, o);
  }
  __shared__ unsigned long long sS[kSlideThreads / 32], sV[kSlideThreads / 32],
      sL[kSlideThreads / 32], sP[kSlideThreads / 32];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { sS[warp] = S; sV[warp] = V; sL[warp] = L; sP[warp] = Pc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t i = 1; i < blockDim.x / 32; ++i) {
      S += sS[i];
      V += sV[i];
      L += sL[i];
      Pc += sP[i];
    }
    atomicAdd(&s.sums[kSumSPart], S);
    atomicAdd(&s.sums[kSumVPart], V);
    atomicAdd(&s.sums[kSumLPart], L);
    atomicAdd(&s.sums[kSumPPart], Pc);
    __threadfence();
    // The last block to finish publishes the totals and resets the partials
    // for the next slide (the counter pattern keeps the slide one launch).
    const unsigned long long done = atomicAdd(&s.sums[kSumCounter], 1ull);
    if (done == gridDim.x - 1) {
      __threadfence();
      s.sums[kSumS] = atomicExch(&s.sums[kSumSPart], 0ull);
      s.sums[kSumV] = atomicExch(&s.sums[kSumVPart], 0ull);
      s.sums[kSumL] = atomicExch(&s.sums[kSumLPart], 0ull);
      s.sums[kSumP] = atomicExch(&s.sums[kSumPPart], 0ull);
      s.sums[kSumCounter] = 0ull;
    }
  }
}

template <int W, int P, int LAY>
cudaError_t launch_slide_l(const Dims &d, const DevState &s, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slide_kernel<W, P, LAY>, kSlideThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = ((d.Z >> 2) + kSlideThreads - 1) / kSlideThreads;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want ? want : 1;
  // k replicated into every even field (the subtrahend of the active test)
  // the DR < k test's constants for c = 2^W - k
  const uint32_t c = (1u << W) - d.k, H = Fields<W>::LSB << (W - 1);
  const KTest kt{(c & ((1u << (W - 1)) - 1u)) * Fields<W>::LSB, (c >> (W - 1)) & 1u ? H : 0u};
  slide_kernel<W, P, LAY><<<(unsigned)grid, kSlideThreads, 0, st>>>(d, s, kt);
  return cudaGetLastError();
}

template <int W, int P>
cudaError_t launch_slide_t(const Dims &d, const DevState &s, int layout, cudaStream_t st) {
  if (layout == kLayoutGfast) return launch_slide_l<W, P, kLayoutGfast>(d, s, st);
  if (layout == kLayoutSerial) return launch_slide_l<W, P, kLayoutSerial>(d, s, st);
  return launch_slide_l<W, P, kLayoutGsmall>(d, s, st);
}

// P = ceil(R / floor(32 / W)) DRV words per BDR, R = 32 - b_min in 16..31.
template <int W>
cudaError_t launch_slide_w(const Dims &d, const DevState &s, int layout, cudaStream_t st) {
  constexpr int F = 32 / W;
  constexpr int PLO = (16 + F - 1) / F, PHI = (31 + F - 1) / F;
  switch (d.P) {
#define VBK_SLIDE_P(PP) \
    case PP: if constexpr (PP >= PLO && PP <= PHI) return launch_slide_t<W, PP>(d, s, layout, st); break;
    VBK_SLIDE_P(1) VBK_SLIDE_P(2) VBK_SLIDE_P(3) VBK_SLIDE_P(4) VBK_SLIDE_P(5) VBK_SLIDE_P(6)
    VBK_SLIDE_P(7) VBK_SLIDE_P(8) VBK_SLIDE_P(9) VBK_SLIDE_P(10) VBK_SLIDE_P(11) VBK_SLIDE_P(12)
    VBK_SLIDE_P(13) VBK_SLIDE_P(14) VBK_SLIDE_P(15) VBK_SLIDE_P(16) VBK_SLIDE_P(31)
#undef VBK_SLIDE_P
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_slide(const Dims &d, const DevState &s, int layout, cudaStream_t st) {
  switch (d.w) {
    case 1: return launch_slide_w<1>(d, s, layout, st);
    case 2: return launch_slide_w<2>(d, s, layout, st);
    case 3: return launch_slide_w<3>(d, s, layout, st);
    case 4: return launch_slide_w<4>(d, s, layout, st);
    case 5: return launch_slide_w<5>(d, s, layout, st);
    case 6: return launch_slide_w<6>(d, s, layout, st);
    case 7: return launch_slide_w<7>(d, s, layout, st);
    case 8: return launch_slide_w<8>(d, s, layout, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vbk
