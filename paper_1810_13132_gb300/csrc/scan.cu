// scan.cu -- per-slice IP-pair scan (Sec. 4.2): Alg. 7 (gfast), Alg. 9
// (gsmall) and Alg. 4's nowLBP1 maximum (serial layout, made safe for
// parallel threads by a byte-wise atomic max), with the per-pair steps of
// Alg. 4 and Alg. 3.
//
// Per pair:
//   bip' = H(bip, 2^32, A1); vidx = left b bits of bip'; x = bip' << b;
//   LBP1 = min(clz(x) + 1, 32 - b); pidx = H(aip, Z, H(vidx, 2^32, A0)).
// The update is idempotent and monotone during a scan -- gfast ORs bit
// LBP1-1 into bsLBP1[pidx] (Alg. 7), gsmall zeroes the DR of LBP1 in the DRV
// of pidx (Alg. 9), serial raises nowLBP1[pidx] to LBP1 (Alg. 4; Sec. 4.2's
// race, a lost larger value, cannot happen with an atomic max) -- so the
// state after the scan does not depend on thread order, and an update whose
// effect is already visible can be dropped.
//
// Design (each choice measured on GB300):
//   * streaming: 16-byte loads of two pairs (L1::no_allocate), UNROLL loads
//     in flight per thread, grid-stride over the slice;
//   * hashing: the 64-bit mix evaluated in 32-bit halves with the seed terms
//     precomputed (KEnt table in shared memory, 16 B per virtual index);
//   * update: the hot state (bsLBP1, or DRV word plane 0 for gsmall) is
//     L2-resident, and with Zipf traffic almost every update is already
//     applied (a heavy host's few BDRs saturate early in the slice).  So all
//     UNROLL*2 target words are first read (L1-cached loads: bits/fields only
//     move one way during a scan, so a stale copy can only cause a redundant
//     update, never a lost one), and only updates that would change the word
//     issue a red.or / red.and.  Two pairs of one thread that hit the same
//     word are merged first.  A warp-wide match.any de-duplication was
//     measured 3x slower than no de-duplication at all on this part (it runs
//     on the ADU pipe), so it is not used.
// The one random test load per pair is the limit: the L1TEX pipe serves
// about one such request per SM clock, 64M tests need about 0.2 ms, and the
// kernel takes 0.30 ms on a 64M-pair slice whatever the loads in flight per
// thread (2 to 8) or the register budget.  bucket.cu routes the updates to
// shared memory instead; it is exact too but slower on this part.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kScanThreads = 256;
constexpr int kUnroll = 4;

__device__ __forceinline__ uint4 ld_stream_v4(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t ld_ca(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_and(uint32_t *p, uint32_t v) {
  asm volatile("red.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Target word offset and update mask of one pair.
//   gfast : word = pidx (bsLBP1), mask = the bit to set
//   gsmall: word = plane * Zs + pidx (DRV), mask = the field bits to clear
//   serial: word = pidx (byte of nowLBP1), mask = LBP1 (the value to max in)
template <int W, bool MIXED>
__device__ __forceinline__ void pair_update(const Dims &d, const KEnt *kt, uint32_t aip,
                                            uint32_t bip, uint64_t &word, uint32_t &mask,
                                            unsigned int *chk) {
  const uint32_t b = MIXED ? d.b_min + (aip >> 30) : d.b;
  const uint32_t bipp = hash32(bip, d.K1);
  const uint32_t vidx = bipp >> (32 - b);
  const uint32_t x = bipp << b;
  const uint32_t r0 = min((uint32_t)__clz(x), 31u - b);  // LBP1 - 1
  const uint32_t pidx = reduce32(hash32(aip, kt[vidx]), d.zmul);
  if (!vbk_check(pidx < d.Z, chk, kChkPidx) || !vbk_check(r0 < d.R, chk, kChkRho)) {
    word = 0;
    mask = 0u;  // bounds-checked build: no update
    return;
  }
  if constexpr (W == 0) {
    word = pidx;
    mask = 1u << r0;
  } else if constexpr (W < 0) {
    word = pidx;
    mask = r0 + 1u;
  } else {
    constexpr uint32_t F = 32 / W;
    constexpr uint32_t FM = (1u << W) - 1u;
    word = (uint64_t)(r0 / F) * d.Zs + pidx;
    mask = FM << ((r0 % F) * W);
  }
}

// SMEM_KT: the seed table (g_max <= 512 entries) is staged in shared memory
// and read with shared-memory loads; otherwise it is read from global memory.
// Byte-wise max into nowLBP1 through a CAS on its 32-bit word.  A failed
// CAS means another thread raised that word (at most 4 * 31 times), so the
// loop ends; the iteration cap is a second guard.
__device__ __forceinline__ void byte_max(uint32_t *w, uint32_t sh, uint32_t v, uint32_t old) {
  for (int it = 0; it < 256 && ((old >> sh) & 0xffu) < v; ++it) {
    const uint32_t seen = atomicCAS(w, old, (old & ~(0xffu << sh)) | (v << sh));
    if (seen == old) break;
    old = seen;
  }
}

// W = 0: gfast; W = DR width: gsmall; W = -1: serial (nowLBP1 bytes)
template <int W, bool MIXED, bool SMEM_KT>
__global__ void __launch_bounds__(kScanThreads)
    scan_kernel(const uint4 *__restrict__ pairs2, uint64_t n_pairs, const uint64_t *n_dev,
                Dims d, DevState s) {
  // n_dev: the slice size read from device memory (a graph replayed for
  // slices of any size up to n_pairs); otherwise n_pairs is the size.
  if (n_dev) n_pairs = min(*n_dev, n_pairs);
  __shared__ KEnt kt_s[SMEM_KT ? kKtabSize : 1];
  const KEnt *kt;
  if constexpr (SMEM_KT) {
    const uint32_t gmax = 1u << (MIXED ? d.b_min + 3 : d.b);
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
    __syncthreads();
    kt = kt_s;
  } else {
    kt = s.ktab;
  }
  uint32_t *const state = (W == 0) ? s.bs : (W < 0 ? reinterpret_cast<uint32_t *>(s.now) : s.drv);

  const uint64_t units = n_pairs >> 1;  // whole 16-byte loads
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < units;
       base += stride * kUnroll) {
    uint4 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t idx = base + (uint64_t)u * stride;
      v[u] = idx < units ? ld_stream_v4(pairs2 + idx) : make_uint4(0, 0, 0, 0);
    }
    uint64_t word[2 * kUnroll];
    uint32_t mask[2 * kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool ok = base + (uint64_t)u * stride < units;
      pair_update<W, MIXED>(d, kt, v[u].x, v[u].y, word[2 * u], mask[2 * u], s.check);
      pair_update<W, MIXED>(d, kt, v[u].z, v[u].w, word[2 * u + 1], mask[2 * u + 1], s.check);
      if (!ok) mask[2 * u] = mask[2 * u + 1] = 0u;
      // adjacent pairs of one load on the same word: one update
      if (word[2 * u] == word[2 * u + 1]) {
        mask[2 * u] = W < 0 ? max(mask[2 * u], mask[2 * u + 1]) : (mask[2 * u] | mask[2 * u + 1]);
        mask[2 * u + 1] = 0u;
      }
    }
    uint32_t old[2 * kUnroll];
#pragma unroll
    for (int q = 0; q < 2 * kUnroll; ++q) {
      const uint64_t wi = W < 0 ? word[q] >> 2 : word[q];
      // serial: the update is a CAS that waits for its answer, so a stale L1
      // copy costs a round trip; read the current word from L2 instead
      old[q] = mask[q] ? (W < 0 ? __ldcg(state + wi) : ld_ca(state + wi))
                       : (W == 0 ? 0xffffffffu : 0u);
    }
#pragma unroll
    for (int q = 0; q < 2 * kUnroll; ++q) {
      if constexpr (W == 0) {
        if (~old[q] & mask[q]) red_or(state + word[q], mask[q]);
      } else if constexpr (W < 0) {
        const uint32_t sh = 8u * (uint32_t)(word[q] & 3u);
        if (((old[q] >> sh) & 0xffu) < mask[q]) byte_max(state + (word[q] >> 2), sh, mask[q], old[q]);
      } else {
        if (old[q] & mask[q]) red_and(state + word[q], ~mask[q]);
      }
    }
  }
  // An odd pair count leaves one pair outside the 16-byte loads.
  if ((n_pairs & 1u) && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(pairs2) + 2 * (n_pairs - 1);
    uint64_t word;
    uint32_t mask;
    pair_update<W, MIXED>(d, kt, p[0], p[1], word, mask, s.check);
    if constexpr (W == 0)
      red_or(state + word, mask);
    else if constexpr (W < 0)
      byte_max(state + (word >> 2), 8u * (uint32_t)(word & 3u), mask, state[word >> 2]);
    else
      red_and(state + word, ~mask);
  }
}

template <int W, bool MIXED>
cudaError_t launch_scan_t(const Dims &d, const DevState &s, const uint32_t *pairs, uint64_t n,
                          const uint64_t *n_dev, cudaStream_t st) {
  const bool smem_kt = (1u << (MIXED ? d.b_min + 3 : d.b)) <= (uint32_t)kKtabSize;
  auto kern = smem_kt ? scan_kernel<W, MIXED, true> : scan_kernel<W, MIXED, false>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t units = n >> 1;
  const uint64_t want = (units + kScanThreads - 1) / kScanThreads;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want ? want : 1;
  kern<<<(unsigned)grid, kScanThreads, 0, st>>>(reinterpret_cast<const uint4 *>(pairs), n, n_dev,
                                                d, s);
  return cudaGetLastError();
}

template <bool MIXED>
cudaError_t launch_scan_m(const Dims &d, const DevState &s, int layout, const uint32_t *pairs,
                          uint64_t n, const uint64_t *n_dev, cudaStream_t st) {
  if (layout == kLayoutGfast) return launch_scan_t<0, MIXED>(d, s, pairs, n, n_dev, st);
  if (layout == kLayoutSerial) return launch_scan_t<-1, MIXED>(d, s, pairs, n, n_dev, st);
  switch (d.w) {
    case 1: return launch_scan_t<1, MIXED>(d, s, pairs, n, n_dev, st);
    case 2: return launch_scan_t<2, MIXED>(d, s, pairs, n, n_dev, st);
    case 3: return launch_scan_t<3, MIXED>(d, s, pairs, n, n_dev, st);
    case 4: return launch_scan_t<4, MIXED>(d, s, pairs, n, n_dev, st);
    case 5: return launch_scan_t<5, MIXED>(d, s, pairs, n, n_dev, st);
    case 6: return launch_scan_t<6, MIXED>(d, s, pairs, n, n_dev, st);
    case 7: return launch_scan_t<7, MIXED>(d, s, pairs, n, n_dev, st);
    case 8: return launch_scan_t<8, MIXED>(d, s, pairs, n, n_dev, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_scan(const Dims &d, const DevState &s, int layout, const uint32_t *pairs,
                        uint64_t n, cudaStream_t st, const uint64_t *n_dev) {
  if (n == 0) return cudaSuccess;
  return d.group_rule ? launch_scan_m<true>(d, s, layout, pairs, n, n_dev, st)
                      : launch_scan_m<false>(d, s, layout, pairs, n, n_dev, st);
}

}  // namespace vbk
