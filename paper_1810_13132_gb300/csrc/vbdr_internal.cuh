// vbdr_internal.cuh -- device-side definitions shared by the VBDR kernels.
//
// Data layout in HBM (per handle, Z physical BDRs):
//   drv   : P word planes of Z uint32 each, plane-major (drv[p * Z + j]).
//           Word p of BDR j packs the DRs of LBP1 values p*F+1 .. p*F+F,
//           F = floor(32 / w) fields of w bits, field f at bits [f*w, f*w+w).
//           Plane-major puts every BDR's first word (LBP1 1..F, which takes
//           1 - 2^-F of all updates because LBP1 is geometric) into one
//           contiguous 4*Z-byte plane, so the hot random updates of the
//           gsmall scan touch a quarter of the DRV footprint.
//   bs    : Z uint32, bsLBP1 of the gfast layout (bit r-1 <-> LBP1 r).
//   reg   : Z uint8, register of every BDR at the last slide (Alg. 2).
//   ktab  : 512 uint64, mix64(s1(i)) for virtual index i, s1(i) = H(i,2^32,A0)
//           (the first hash of Alg. 3, which depends only on i).
//   sums  : pool sums S_Z, V_Z and the block-completion counter of the slide.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vbk {

constexpr int kMaxLog2G = 16;
constexpr int kKtabSize = 512;  // virtual indices covered by the smem table

// SplitMix64 output mix (Steele, Lea & Flood 2014), used as the seeded hash
// H(x, N, A) of Sec. 4.1:  H(x,N,A) = (hi32(mix64(x ^ mix64(A))) * N) >> 32.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// hi32(mix64(x ^ K)) for a 32-bit x and a premixed seed K = mix64(A).
__device__ __forceinline__ uint32_t hash32(uint32_t x, uint64_t K) {
  return (uint32_t)(mix64((uint64_t)x ^ K) >> 32);
}

// Multiply-shift range reduction of a 32-bit hash onto [0, Z); Z = 2^32 is
// passed as zmul = 0 and means "the hash itself".
__device__ __forceinline__ uint32_t reduce32(uint32_t h, uint32_t zmul) {
  return zmul ? __umulhi(h, zmul) : h;
}

struct Dims {
  uint64_t Z;        // physical BDRs
  uint32_t zmul;     // Z as a 32-bit multiplier (0 when Z = 2^32)
  uint32_t k;        // window in slices
  uint32_t w;        // DR width in bits
  uint32_t F;        // DR fields per 32-bit word
  uint32_t P;        // DRV words (planes) per BDR
  uint32_t R;        // DRs per BDR = 32 - b_min
  uint32_t b;        // log2 g (group_rule 0)
  uint32_t b_min;    // smallest log2 g
  uint32_t group_rule;
  uint64_t A0, A1;   // seeds
  uint64_t K1;       // mix64(A1): premixed seed of the bip hash
};

struct DevState {
  uint32_t *drv;     // [P][Z]
  uint32_t *bs;      // [Z] (gfast only, else nullptr)
  uint8_t *reg;      // [Z]
  uint64_t *ktab;    // [kKtabSize]
  unsigned long long *sums;  // [0] S_Z, [1] V_Z, [2] slide block counter,
                             // [3] S partial, [4] V partial
};

// host b of aip (group_rule 1: four groups by the top two address bits)
__device__ __forceinline__ uint32_t host_b(const Dims &d, uint32_t aip) {
  return d.group_rule ? d.b_min + (aip >> 30) : d.b;
}

// ----- launchers (defined in the kernel translation units) -----
cudaError_t launch_init(const Dims &d, const DevState &s, cudaStream_t st);
cudaError_t launch_scan(const Dims &d, const DevState &s, bool gfast,
                        const uint32_t *pairs, uint64_t n, cudaStream_t st);
cudaError_t launch_slide(const Dims &d, const DevState &s, bool gfast,
                         cudaStream_t st);
cudaError_t launch_estimate(const Dims &d, const DevState &s,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st);

}  // namespace vbk
