// bucket.cu -- the per-slice pair scan of Sec. 4.2 (Alg. 7 for gfast, Alg. 9
// for gsmall) with the updates routed to the part of the BDR pool that owns
// them, so that the per-pair state work runs in shared memory.
//
// Why: the update of a pair touches one random 4-byte word of a 64 MiB
// (gfast) or 256 MiB (gsmall) state.  A kernel that tests or updates that word
// per pair issues one random L1TEX request per pair, and the L1TEX pipe
// serves about one such request per SM clock -- 64M pairs then need about
// 0.2 ms however the rest is arranged.  Here every pair costs shared-memory
// work only; the global state is touched once per BDR per pass, coalesced.
//
// The pool is cut into tiles of 2^16 consecutive BDRs.  A slice is processed
// in passes of at most kPassPairs pairs; each pass is two kernels:
//   A (route) : hash every pair (Alg. 4's vidx and LBP1, Alg. 3's pidx) and
//               emit the 4-byte record (pidx mod 2^16) << 5 | (LBP1 - 1)
//               into its tile's bucket.  A CTA takes 8192 pairs at a time,
//               counting-sorts their records by tile in shared memory,
//               reserves room in each tile's bucket with one global atomic per
//               tile, and copies the sorted runs out with coalesced stores.
//               A record that does not fit its bucket (an extremely skewed
//               slice) is applied at once with an atomic on the state.
//   B (apply) : one CTA per tile keeps one byte per BDR of the tile in shared
//               memory (LBP1 1..8, i.e. bits 0..7 of bsLBP1: all but 2^-8 of
//               the pairs), ORs in the bucket's records with shared atomics,
//               then writes every non-zero byte back with one global atomic
//               per BDR: OR into bsLBP1 (gfast) or AND of the DR fields to
//               zero into the DRV planes (gsmall).  Records of LBP1 above 8
//               are applied with a global atomic directly.
// Both updates are idempotent and commute, so the state after the scan is
// the one the per-pair algorithms give, whatever the order (bit for bit).
// The record buffer and the bucket fill counters belong to the handle; the
// apply kernel leaves every fill counter at zero for the next pass.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kRouteThreads = 512;
constexpr int kRouteUnroll = 8;                                   // uint4 loads per thread
constexpr uint32_t kBatchUnits = kRouteThreads * kRouteUnroll;   // 4096 uint4 = 8192 pairs
constexpr uint32_t kBatchPairs = 2 * kBatchUnits;
constexpr int kApplyThreads = 512;
constexpr uint32_t kLowBits = 8;  // LBP1 values kept in the apply kernel's bytes
constexpr size_t kApplySmem = kBucketTile;  // one byte per BDR of a tile

__device__ __forceinline__ uint4 ld_stream_v4(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_and(uint32_t *p, uint32_t v) {
  asm volatile("red.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// pidx and LBP1 - 1 of one pair (Alg. 4 and Alg. 3).
template <bool MIXED>
__device__ __forceinline__ void pair_hash(const Dims &d, const KEnt *kt, uint32_t aip,
                                          uint32_t bip, uint32_t &pidx, uint32_t &r0) {
  const uint32_t b = MIXED ? d.b_min + (aip >> 30) : d.b;
  const uint32_t bipp = hash32(bip, d.K1);
  const uint32_t vidx = bipp >> (32 - b);
  const uint32_t x = bipp << b;
  r0 = min((uint32_t)__clz(x), 31u - b);
  pidx = reduce32(hash32(aip, kt[vidx]), d.zmul);
}

// The update of one (pidx, LBP1 - 1) applied straight to the global state.
template <int W>
__device__ __forceinline__ void apply_direct(const Dims &d, const DevState &s, uint32_t pidx,
                                             uint32_t r0) {
  if constexpr (W == 0) {
    red_or(s.bs + pidx, 1u << r0);
  } else {
    constexpr uint32_t F = 32 / W, FM = (1u << W) - 1u;
    red_and(s.drv + (uint64_t)(r0 / F) * d.Zs + pidx, ~(FM << ((r0 % F) * W)));
  }
}

struct RouteSmem {
  KEnt kt[kKtabSize];
  uint32_t recs[kBatchPairs];  // tile << 21 | record, sorted by tile
  uint32_t cnt[kMaxBucketTiles];
  uint32_t off[kMaxBucketTiles];
  uint32_t base[kMaxBucketTiles];  // bucket position of the tile's first record this batch
  uint32_t total;
};

// Kernel A: units [u_begin, u_end) of the slice (uint4 = two pairs).
template <int W, bool MIXED>
__global__ void __launch_bounds__(kRouteThreads, 2)
    route_kernel(const uint4 *__restrict__ pairs2, uint64_t u_begin, uint64_t u_end,
                 const uint64_t *n_dev, Dims d, DevState s, BucketDev bk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  RouteSmem &S = *reinterpret_cast<RouteSmem *>(smraw);
  if (n_dev) {
    const uint64_t units = *n_dev >> 1;
    if (u_end > units) u_end = units;
  }
  const uint32_t tid = threadIdx.x;
  const uint32_t gmax = 1u << (MIXED ? d.b_min + 3 : d.b);
  for (uint32_t i = tid; i < gmax; i += kRouteThreads) S.kt[i] = s.ktab[i];
  const uint32_t NT = bk.ntiles;
  for (uint64_t b0 = u_begin + (uint64_t)blockIdx.x * kBatchUnits; b0 < u_end;
       b0 += (uint64_t)gridDim.x * kBatchUnits) {
    for (uint32_t t = tid; t < NT; t += kRouteThreads) S.cnt[t] = 0;
    __syncthreads();
    // hash the batch; each record takes the next slot of its tile
    uint32_t key[2 * kRouteUnroll], slot[2 * kRouteUnroll];
#pragma unroll
    for (int u = 0; u < kRouteUnroll; ++u) {
      const uint64_t idx = b0 + tid + (uint64_t)u * kRouteThreads;
      const bool ok = idx < u_end;
      const uint4 v = ok ? ld_stream_v4(pairs2 + idx) : make_uint4(0, 0, 0, 0);
      uint32_t p0, r0, p1, r1;
      pair_hash<MIXED>(d, S.kt, v.x, v.y, p0, r0);
      pair_hash<MIXED>(d, S.kt, v.z, v.w, p1, r1);
      const bool ok0 = ok && vbk_check(p0 < d.Z, s.check, kChkPidx) &&
                       vbk_check(r0 < d.R, s.check, kChkRho);
      const bool ok1 = ok && vbk_check(p1 < d.Z, s.check, kChkPidx) &&
                       vbk_check(r1 < d.R, s.check, kChkRho);
      key[2 * u] = ok0 ? ((p0 >> kBucketTileLog2) << 21) | ((p0 & (kBucketTile - 1)) << 5) | r0
                       : 0xffffffffu;
      key[2 * u + 1] = ok1 ? ((p1 >> kBucketTileLog2) << 21) | ((p1 & (kBucketTile - 1)) << 5) | r1
                           : 0xffffffffu;
    }
#pragma unroll
    for (int q = 0; q < 2 * kRouteUnroll; ++q)
      if (key[q] != 0xffffffffu) slot[q] = atomicAdd(&S.cnt[key[q] >> 21], 1u);
    __syncthreads();
    // each non-empty tile's room in its bucket (one global atomic per tile,
    // all issued at once), and the exclusive prefix of the counts (warp 0)
    for (uint32_t t = tid; t < NT; t += kRouteThreads) {
      const uint32_t c = S.cnt[t];
      S.base[t] = c ? atomicAdd(bk.fill + t, c) : 0u;
    }
    if (tid < 32) {
      uint32_t carry = 0;
      for (uint32_t t0 = 0; t0 < NT; t0 += 32) {
        const uint32_t t = t0 + tid;
        const uint32_t c = t < NT ? S.cnt[t] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (tid >= (uint32_t)o) x += y;
        }
        if (t < NT) S.off[t] = carry + x - c;
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
      if (tid == 0) S.total = carry;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2 * kRouteUnroll; ++q)
      if (key[q] != 0xffffffffu) S.recs[S.off[key[q] >> 21] + slot[q]] = key[q];
    // bucket position of sorted record i of tile t: base[t] + i - off[t]
    for (uint32_t t = tid; t < NT; t += kRouteThreads) S.base[t] -= S.off[t];
    __syncthreads();
    // copy-out: consecutive records of a tile go to consecutive bucket slots
    const uint32_t total = S.total;
    for (uint32_t i = tid; i < total; i += kRouteThreads) {
      const uint32_t kq = S.recs[i];
      const uint32_t t = kq >> 21;
      const uint32_t pos = S.base[t] + i;
      if (pos < bk.cap) {
        bk.recs[(uint64_t)t * bk.cap + pos] = kq & 0x1fffffu;
      } else {  // bucket full: apply this one at once
        const uint32_t pidx = (t << kBucketTileLog2) | ((kq >> 5) & (kBucketTile - 1));
        apply_direct<W>(d, s, pidx, kq & 31u);
      }
    }
    __syncthreads();
  }
}

// Kernel B: one CTA per tile.
template <int W>
__global__ void __launch_bounds__(kApplyThreads)
    apply_kernel(Dims d, DevState s, BucketDev bk) {
  extern __shared__ uint32_t bits[];  // kBucketTile / 4 words: one byte per BDR of the tile
  __shared__ uint32_t n_s;
  const uint32_t t = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) {
    const uint32_t f = bk.fill[t];
    n_s = f < bk.cap ? f : bk.cap;
  }
  __syncthreads();
  const uint32_t n = n_s;
  if (n == 0) return;  // fill is already 0
  for (uint32_t i = tid; i < kBucketTile / 4; i += kApplyThreads) bits[i] = 0u;
  __syncthreads();
  const uint64_t tile0 = (uint64_t)t << kBucketTileLog2;
  const uint32_t *rec = bk.recs + (uint64_t)t * bk.cap;
  for (uint32_t i = tid; i < n; i += kApplyThreads) {
    const uint32_t r = rec[i];
    const uint32_t off = r >> 5, r0 = r & 31u;
    if (r0 < kLowBits)
      atomicOr(&bits[off >> 2], 1u << (8u * (off & 3u) + r0));
    else
      apply_direct<W>(d, s, (uint32_t)(tile0 + off), r0);
  }
  __syncthreads();
  if (tid == 0) bk.fill[t] = 0u;  // the bucket is consumed
  const uint64_t left = d.Z - tile0;
  const uint32_t nb = left < kBucketTile ? (uint32_t)left : kBucketTile;
  for (uint32_t j = tid; j < nb; j += kApplyThreads) {
    const uint32_t v = (bits[j >> 2] >> (8u * (j & 3u))) & 0xffu;
    if (!v) continue;
    const uint64_t pidx = tile0 + j;
    if constexpr (W == 0) {
      red_or(s.bs + pidx, v);
    } else {
      // LBP1 - 1 = 0..7 spans the DR fields of the first one or two planes
      constexpr uint32_t F = 32 / W, FM = (1u << W) - 1u;
      uint32_t m = 0;
#pragma unroll
      for (uint32_t r = 0; r < kLowBits; ++r) {
        if (r == F) {  // the first plane is complete
          if (m) red_and(s.drv + pidx, ~m);
          m = 0;
        }
        if ((v >> r) & 1u) m |= FM << ((r % F) * W);
      }
      if (m) red_and(s.drv + (uint64_t)((kLowBits - 1) / F) * d.Zs + pidx, ~m);
    }
  }
}

// The odd last pair of a slice (outside the 16-byte loads).
template <int W, bool MIXED>
__global__ void tail_pair_kernel(const uint32_t *pairs, uint64_t n, const uint64_t *n_dev, Dims d,
                                 DevState s) {
  if (n_dev) n = min(*n_dev, n);
  if (!(n & 1u)) return;
  uint32_t pidx, r0;
  pair_hash<MIXED>(d, s.ktab, pairs[2 * (n - 1)], pairs[2 * (n - 1) + 1], pidx, r0);
  if (vbk_check(pidx < d.Z, s.check, kChkPidx)) apply_direct<W>(d, s, pidx, r0);
}

template <int W, bool MIXED>
cudaError_t launch_t(const Dims &d, const DevState &s, const BucketDev &bk, const uint32_t *pairs,
                     uint64_t n, const uint64_t *n_dev, cudaStream_t st) {
  auto route = route_kernel<W, MIXED>;
  const size_t smem = sizeof(RouteSmem);
  cudaError_t e = cudaFuncSetAttribute(route, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kApplySmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, route, kRouteThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t units = n >> 1;
  const uint64_t pass_units = bk.pass_pairs >> 1;
  for (uint64_t u0 = 0; u0 < units; u0 += pass_units) {
    const uint64_t u1 = units - u0 < pass_units ? units : u0 + pass_units;
    const uint64_t batches = (u1 - u0 + kBatchUnits - 1) / kBatchUnits;
    uint64_t grid = (uint64_t)sms * per_sm;
    if (batches < grid) grid = batches;
    route<<<(unsigned)grid, kRouteThreads, smem, st>>>(reinterpret_cast<const uint4 *>(pairs), u0,
                                                       u1, n_dev, d, s, bk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    apply_kernel<W><<<bk.ntiles, kApplyThreads, kApplySmem, st>>>(d, s, bk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n & 1u) {
    tail_pair_kernel<W, MIXED><<<1, 1, 0, st>>>(pairs, n, n_dev, d, s);
    e = cudaGetLastError();
  }
  return e;
}

template <bool MIXED>
cudaError_t launch_m(const Dims &d, const DevState &s, const BucketDev &bk, int layout,
                     const uint32_t *pairs, uint64_t n, const uint64_t *n_dev, cudaStream_t st) {
  if (layout == kLayoutGfast) return launch_t<0, MIXED>(d, s, bk, pairs, n, n_dev, st);
  switch (d.w) {
    case 1: return launch_t<1, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 2: return launch_t<2, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 3: return launch_t<3, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 4: return launch_t<4, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 5: return launch_t<5, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 6: return launch_t<6, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 7: return launch_t<7, MIXED>(d, s, bk, pairs, n, n_dev, st);
    case 8: return launch_t<8, MIXED>(d, s, bk, pairs, n, n_dev, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool bucket_scan_applies(const Dims &d, int layout) {
  if (layout != kLayoutGfast && layout != kLayoutGsmall) return false;
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  return gmax <= (uint32_t)kKtabSize &&
         (d.Z + kBucketTile - 1) / kBucketTile <= (uint64_t)kMaxBucketTiles;
}

cudaError_t launch_scan_bucketed(const Dims &d, const DevState &s, const BucketDev &bk, int layout,
                                 const uint32_t *pairs, uint64_t n, cudaStream_t st,
                                 const uint64_t *n_dev) {
  if (n == 0) return cudaSuccess;
  return d.group_rule ? launch_m<true>(d, s, bk, layout, pairs, n, n_dev, st)
                      : launch_m<false>(d, s, bk, layout, pairs, n, n_dev, st);
}

}  // namespace vbk
