// scan.cu -- per-slice IP-pair scan (Sec. 4.2): Alg. 7 (gfast) and Alg. 9
// (gsmall), with the per-pair steps of Alg. 4 and Alg. 3.
//
// One thread handles two pairs per 16-byte load (uint4 = {aip0, bip0, aip1,
// bip1}), UNROLL loads in flight per thread, grid-stride over the slice.
// Per pair:
//   bip' = H(bip, 2^32, A1); vidx = left b bits of bip'; x = bip' << b;
//   LBP1 = min(clz(x) + 1, 32 - b); pidx = H(aip, Z, H(vidx, 2^32, A0)).
// Updates are de-duplicated inside the warp before they reach L2:
//   gfast : lanes with equal pidx (match.any) OR their bits (redux.or) and
//           the lowest lane issues one red.or -- after a test of the word
//           (skipped when every bit is already set, which is the common case
//           for heavy hosts whose few BDRs saturate early in the slice).
//   gsmall: the same on (pidx, DRV word) with redux.and of the field-clear
//           masks; the hot plane 0 (LBP1 1..F) goes through the match, the
//           rare higher planes clear their field directly.
// Both updates are idempotent and commutative (OR of bits, AND-clear of
// fields), so the state after the scan does not depend on thread order.
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

struct PairHash {
  uint32_t pidx;
  uint32_t rho;
};

__device__ __forceinline__ PairHash hash_pair(const Dims &d,
                                              const uint64_t *kt,
                                              uint32_t aip, uint32_t bip) {
  const uint32_t b = host_b(d, aip);
  const uint32_t bipp = hash32(bip, d.K1);
  const uint32_t vidx = bipp >> (32 - b);
  const uint32_t x = bipp << b;
  const uint32_t rho = min((uint32_t)__clz(x) + 1u, 32u - b);
  PairHash ph;
  ph.pidx = reduce32(hash32(aip, kt[vidx]), d.zmul);
  ph.rho = rho;
  return ph;
}

// gfast update of one pair per lane; valid lanes carry bit != 0.
__device__ __forceinline__ void update_gfast(uint32_t *bs, uint32_t pidx,
                                             uint32_t bit, uint32_t lane) {
  const unsigned valid = __ballot_sync(0xffffffffu, bit != 0u);
  const unsigned peers = __match_any_sync(0xffffffffu, pidx);
  const uint32_t orbits = __reduce_or_sync(peers, bit);
  const unsigned mine = peers & valid;
  if (mine && lane == (uint32_t)(__ffs(mine) - 1)) {
    uint32_t *w = bs + pidx;
    const uint32_t old = __ldcg(w);
    if ((old & orbits) != orbits) atomicOr(w, orbits);
  }
}

// gsmall update: clear the w-bit DR of LBP1 rho at BDR pidx.
template <int W>
__device__ __forceinline__ void update_gsmall(uint32_t *drv, uint64_t Z,
                                              uint32_t pidx, uint32_t rho,
                                              bool valid, uint32_t lane) {
  constexpr uint32_t F = 32 / W;
  constexpr uint32_t FM = (W == 32) ? 0xffffffffu : ((1u << W) - 1u);
  const uint32_t r0 = rho - 1u;
  const uint32_t plane = r0 / F;
  const uint32_t clear = ~(FM << ((r0 % F) * W));
  const bool hot = valid && plane == 0;
  const unsigned hotmask = __ballot_sync(0xffffffffu, hot);
  const unsigned peers = __match_any_sync(0xffffffffu, hot ? pidx : 0xffffffffu);
  const uint32_t andmask = __reduce_and_sync(peers, hot ? clear : 0xffffffffu);
  const unsigned mine = peers & hotmask;
  if (hot && lane == (uint32_t)(__ffs(mine) - 1)) {
    uint32_t *w = drv + pidx;
    const uint32_t old = __ldcg(w);
    if (old & ~andmask) atomicAnd(w, andmask);
  }
  if (valid && plane != 0) {
    uint32_t *w = drv + (uint64_t)plane * Z + pidx;
    const uint32_t old = __ldcg(w);
    if (old & ~clear) atomicAnd(w, clear);
  }
}

template <int W>  // W = 0: gfast; W = DR width: gsmall
__global__ void __launch_bounds__(kScanThreads)
    scan_kernel(const uint4 *__restrict__ pairs2, uint64_t n_pairs, Dims d,
                DevState s) {
  __shared__ uint64_t kt_s[kKtabSize];
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  const bool kt_in_smem = gmax <= (uint32_t)kKtabSize;
  if (kt_in_smem)
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
  __syncthreads();
  const uint64_t *kt = kt_in_smem ? kt_s : s.ktab;

  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t units = n_pairs >> 1;  // whole uint4 loads
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // Warp-uniform loop: every lane of a warp runs the same iterations so the
  // warp collectives see all 32 lanes; out-of-range lanes are masked.
  const uint64_t warp_base0 =
      (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
  for (uint64_t base = warp_base0; base < units; base += stride * kUnroll) {
    uint4 v[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t idx = base + (uint64_t)u * stride + lane;
      ok[u] = idx < units;
      v[u] = ok[u] ? ld_stream_v4(pairs2 + idx) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const uint32_t aip = half ? v[u].z : v[u].x;
        const uint32_t bip = half ? v[u].w : v[u].y;
        const PairHash ph = hash_pair(d, kt, aip, bip);
        if constexpr (W == 0) {
          update_gfast(s.bs, ok[u] ? ph.pidx : 0u, ok[u] ? (1u << (ph.rho - 1u)) : 0u, lane);
        } else {
          update_gsmall<W>(s.drv, d.Z, ph.pidx, ph.rho, ok[u], lane);
        }
      }
    }
  }
  // An odd pair count leaves one pair outside the uint4 loads.
  if ((n_pairs & 1u) && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(pairs2) + 2 * (n_pairs - 1);
    const PairHash ph = hash_pair(d, kt, p[0], p[1]);
    if constexpr (W == 0) {
      atomicOr(s.bs + ph.pidx, 1u << (ph.rho - 1u));
    } else {
      constexpr uint32_t F = 32 / W;
      const uint32_t r0 = ph.rho - 1u;
      atomicAnd(s.drv + (uint64_t)(r0 / F) * d.Z + ph.pidx,
                ~(((1u << W) - 1u) << ((r0 % F) * W)));
    }
  }
}

template <int W>
cudaError_t launch_scan_t(const Dims &d, const DevState &s, const uint32_t *pairs,
                          uint64_t n, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel<W>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t units = n >> 1;
  const uint64_t want = (units + kScanThreads - 1) / kScanThreads;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want ? want : 1;
  scan_kernel<W><<<(unsigned)grid, kScanThreads, 0, st>>>(
      reinterpret_cast<const uint4 *>(pairs), n, d, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan(const Dims &d, const DevState &s, bool gfast,
                        const uint32_t *pairs, uint64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (gfast) return launch_scan_t<0>(d, s, pairs, n, st);
  switch (d.w) {
    case 1: return launch_scan_t<1>(d, s, pairs, n, st);
    case 2: return launch_scan_t<2>(d, s, pairs, n, st);
    case 3: return launch_scan_t<3>(d, s, pairs, n, st);
    case 4: return launch_scan_t<4>(d, s, pairs, n, st);
    case 5: return launch_scan_t<5>(d, s, pairs, n, st);
    case 6: return launch_scan_t<6>(d, s, pairs, n, st);
    case 7: return launch_scan_t<7>(d, s, pairs, n, st);
    case 8: return launch_scan_t<8>(d, s, pairs, n, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vbk
