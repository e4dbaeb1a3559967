// bucket.cu -- the per-slice pair scan of Sec. 4.2 (Alg. 7 for gfast, Alg. 9
// for gsmall) with the updates routed to the part of the BDR pool that owns
// them, so that the per-pair state work runs in shared memory.
//
// Why: the update of a pair touches one random 4-byte word of a 64 MiB
// (gfast) or 256 MiB (gsmall) state.  A kernel that tests or updates that word
// per pair issues one random L1TEX request per pair, and the L1TEX pipe
// serves about one such request per SM clock -- 64M pairs then need about
// 0.2 ms however the rest is arranged.  Here every pair costs shared-memory
// work only, and the global state is read and written once per scan call,
// with coalesced 16-byte accesses.
//
// The pool is cut into tiles of 2^16 consecutive BDRs.  A slice is processed
// in passes of at most pass_pairs pairs; each pass is two kernels:
//   route : a fixed grid of ncta CTAs hashes the pairs (Alg. 4's vidx and
//           LBP1, Alg. 3's pidx).  A CTA takes 8192 pairs at a time,
//           counting-sorts their records (pidx mod 2^16) << 3 | (LBP1 - 1) by
//           tile in shared memory and appends each tile's run to the CTA's
//           own region of that tile's bucket (cap records), so no two CTAs
//           write the same place and no global atomic is needed.  A pair of
//           LBP1 above 8 (a 2^-8 share), or a record that finds its region
//           full, is applied at once with an atomic on the state.
//   apply : one CTA per tile keeps one byte per BDR of the tile in shared
//           memory -- bit r is LBP1 r + 1 seen in this scan call -- and ORs in
//           the tile's records of every route CTA with shared atomics.
//           Between passes the bytes live in a global array (lb); the last
//           pass folds them into the state: OR into bsLBP1 (gfast) or zero
//           the DR fields (gsmall), with plain read-modify-write of whole
//           16-byte groups (no other kernel writes the state meanwhile).
// Both updates are idempotent and commute, so the state after the scan is
// the one the per-pair algorithms give, whatever the order (bit for bit).
#include <algorithm>

#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kRouteThreads = 512;
constexpr int kRouteUnroll = 8;                                   // uint4 loads per thread
constexpr uint32_t kBatchUnits = kRouteThreads * kRouteUnroll;   // 4096 uint4 = 8192 pairs
constexpr uint32_t kBatchPairs = 2 * kBatchUnits;
constexpr int kRouteCtasPerSm = 2;
constexpr int kApplyThreads = 512;
constexpr uint32_t kLowBits = 8;            // LBP1 1..8 go through the buckets
constexpr size_t kApplySmem = kBucketTile;  // one byte per BDR of a tile
constexpr uint32_t kKeyTileShift = 19;      // smem key: tile << 19 | off16 << 3 | r0
constexpr uint32_t kNoKey = 0xffffffffu;

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

// Exclusive prefix over the n <= 2048 values v[0..n) of shared memory, in
// place, by the whole block (512 threads, each summing up to 4 neighbours);
// returns the total.  wsum: 17 words of scratch.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t *v, uint32_t n, uint32_t *wsum) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t per = (n + kRouteThreads - 1) / kRouteThreads;  // <= 4
  const uint32_t i0 = tid * per;
  uint32_t loc[4] = {0, 0, 0, 0}, sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < 4; ++k)
    if (k < per && i0 + k < n) {
      loc[k] = v[i0 + k];
      sum += loc[k];
    }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kRouteThreads / 32 ? wsum[lane] : 0u;
    uint32_t z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= (uint32_t)o) z += y;
    }
    if (lane < kRouteThreads / 32) wsum[lane] = z - w;
    if (lane == kRouteThreads / 32 - 1) wsum[16] = z;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + x - sum;
#pragma unroll
  for (uint32_t k = 0; k < 4; ++k)
    if (k < per && i0 + k < n) {
      v[i0 + k] = run;
      run += loc[k];
    }
  return wsum[16];
}

// Route, one pass: units [u_begin, u_end) of the slice (uint4 = two pairs).
// Dynamic shared memory: kt[kKtabSize] KEnt, keys[kBatchPairs], then four
// arrays of ntiles words (counts / offsets, region fill, base, counts) and
// 17 words of scratch.
template <int W, bool MIXED>
__global__ void __launch_bounds__(kRouteThreads, kRouteCtasPerSm)
    route_kernel(const uint4 *__restrict__ pairs2, uint64_t u_begin, uint64_t u_end,
                 const uint64_t *n_dev, Dims d, DevState s, BucketDev bk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  KEnt *kt = reinterpret_cast<KEnt *>(smraw);
  uint32_t *keys = reinterpret_cast<uint32_t *>(kt + kKtabSize);
  const uint32_t NT = bk.ntiles;
  uint32_t *cnt = keys + kBatchPairs;  // counts, then exclusive offsets
  uint32_t *rfill = cnt + NT;          // records in this CTA's region of each tile
  uint32_t *base = rfill + NT;         // region position of sorted record 0, per tile
  uint32_t *cnt2 = base + NT;          // the batch's counts
  uint32_t *scratch = cnt2 + NT;       // 17 words
  if (n_dev) {
    const uint64_t units = *n_dev >> 1;
    if (u_end > units) u_end = units;
  }
  const uint32_t tid = threadIdx.x;
  const uint32_t gmax = 1u << (MIXED ? d.b_min + 3 : d.b);
  for (uint32_t i = tid; i < gmax; i += kRouteThreads) kt[i] = s.ktab[i];
  for (uint32_t t = tid; t < NT; t += kRouteThreads) rfill[t] = 0;
  uint32_t *region = bk.recs + (uint64_t)blockIdx.x * NT * bk.cap;
  for (uint64_t b0 = u_begin + (uint64_t)blockIdx.x * kBatchUnits; b0 < u_end;
       b0 += (uint64_t)gridDim.x * kBatchUnits) {
    for (uint32_t t = tid; t < NT; t += kRouteThreads) cnt[t] = 0;
    __syncthreads();
    uint32_t key[2 * kRouteUnroll], slot[2 * kRouteUnroll];
#pragma unroll
    for (int u = 0; u < kRouteUnroll; ++u) {
      const uint64_t idx = b0 + tid + (uint64_t)u * kRouteThreads;
      const bool ok = idx < u_end;
      const uint4 v = ok ? ld_stream_v4(pairs2 + idx) : make_uint4(0, 0, 0, 0);
      uint32_t p[2], r[2];
      pair_hash<MIXED>(d, kt, v.x, v.y, p[0], r[0]);
      pair_hash<MIXED>(d, kt, v.z, v.w, p[1], r[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t k = kNoKey;
        if (ok && vbk_check(p[h] < d.Z, s.check, kChkPidx) &&
            vbk_check(r[h] < d.R, s.check, kChkRho)) {
          if (r[h] < kLowBits)
            k = ((p[h] >> kBucketTileLog2) << kKeyTileShift) |
                ((p[h] & (kBucketTile - 1)) << 3) | r[h];
          else
            apply_direct<W>(d, s, p[h], r[h]);  // LBP1 above 8: rare
        }
        key[2 * u + h] = k;
      }
    }
#pragma unroll
    for (int q = 0; q < 2 * kRouteUnroll; ++q)
      if (key[q] != kNoKey) slot[q] = atomicAdd(&cnt[key[q] >> kKeyTileShift], 1u);
    __syncthreads();
    for (uint32_t t = tid; t < NT; t += kRouteThreads) cnt2[t] = cnt[t];
    const uint32_t total = block_exclusive_scan(cnt, NT, scratch);  // cnt: offsets now
    __syncthreads();
    for (uint32_t t = tid; t < NT; t += kRouteThreads) {
      base[t] = rfill[t] - cnt[t];
      rfill[t] += cnt2[t];
    }
#pragma unroll
    for (int q = 0; q < 2 * kRouteUnroll; ++q)
      if (key[q] != kNoKey) keys[cnt[key[q] >> kKeyTileShift] + slot[q]] = key[q];
    __syncthreads();
    // copy-out: the consecutive records of a tile go to consecutive places of
    // this CTA's region of the tile
    for (uint32_t i = tid; i < total; i += kRouteThreads) {
      const uint32_t kq = keys[i];
      const uint32_t t = kq >> kKeyTileShift;
      const uint32_t pos = base[t] + i;
      const uint32_t rec = kq & ((1u << kKeyTileShift) - 1u);
      if (pos < bk.cap)
        region[(uint64_t)t * bk.cap + pos] = rec;
      else  // region full: apply this one at once
        apply_direct<W>(d, s, (t << kBucketTileLog2) | (rec >> 3), rec & 7u);
    }
    __syncthreads();
  }
  // every CTA of the grid publishes its region fills (0 if it had no batch)
  for (uint32_t t = tid; t < NT; t += kRouteThreads)
    bk.fill[(uint64_t)blockIdx.x * NT + t] = rfill[t];
}

// Apply, one pass: one CTA per tile.  first: the tile's bytes start at 0
// (else they are loaded from lb); last: fold them into the state (else store
// them to lb).
template <int W>
__global__ void __launch_bounds__(kApplyThreads)
    apply_kernel(Dims d, DevState s, BucketDev bk, int first, int last) {
  extern __shared__ __align__(16) uint32_t bits[];  // kBucketTile bytes
  __shared__ uint32_t any_s;
  const uint32_t t = blockIdx.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t NT = bk.ntiles;
  if (tid == 0) any_s = 0;
  __syncthreads();
  uint32_t mine = 0;
  for (uint32_t c = tid; c < bk.ncta; c += kApplyThreads) mine |= bk.fill[(uint64_t)c * NT + t];
  if (mine) any_s = 1;
  __syncthreads();
  if (!any_s && !first && !last) return;  // no record: the tile's bytes are unchanged
  uint4 *bits4 = reinterpret_cast<uint4 *>(bits);
  uint4 *lb4 = reinterpret_cast<uint4 *>(bk.lb + ((uint64_t)t << kBucketTileLog2));
  constexpr uint32_t kWords4 = kBucketTile / 16;
  for (uint32_t i = tid; i < kWords4; i += kApplyThreads)
    bits4[i] = first ? make_uint4(0, 0, 0, 0) : lb4[i];
  __syncthreads();
  if (any_s) {
    for (uint32_t c = warp; c < bk.ncta; c += kApplyThreads / 32) {
      const uint32_t f = bk.fill[(uint64_t)c * NT + t];
      const uint32_t n = f < bk.cap ? f : bk.cap;
      const uint32_t *rec = bk.recs + ((uint64_t)c * NT + t) * bk.cap;
      for (uint32_t i = lane; i < n; i += 32) {
        const uint32_t r = rec[i];
        const uint32_t off = r >> 3;
        atomicOr(&bits[off >> 2], 1u << (8u * (off & 3u) + (r & 7u)));
      }
    }
  }
  __syncthreads();
  if (!last) {
    for (uint32_t i = tid; i < kWords4; i += kApplyThreads) lb4[i] = bits4[i];
    return;
  }
  // fold into the state: groups of 4 BDRs (one 16-byte access per plane)
  const uint64_t tile0 = (uint64_t)t << kBucketTileLog2;
  const uint64_t left = d.Z - tile0;
  const uint32_t nb = left < kBucketTile ? (uint32_t)left : kBucketTile;
  for (uint32_t q = tid; q < (nb + 3) / 4; q += kApplyThreads) {
    const uint32_t v = bits[q];
    if (!v) continue;
    const uint64_t j0 = tile0 + 4ull * q;
    if constexpr (W == 0) {
      if (j0 + 4 <= d.Z) {
        uint4 *p = reinterpret_cast<uint4 *>(s.bs + j0);
        uint4 b = *p;
        b.x |= v & 0xffu;
        b.y |= (v >> 8) & 0xffu;
        b.z |= (v >> 16) & 0xffu;
        b.w |= v >> 24;
        *p = b;
      } else {  // the pool's last, partial group
        for (uint32_t k = 0; k < 4 && j0 + k < d.Z; ++k) s.bs[j0 + k] |= (v >> (8 * k)) & 0xffu;
      }
    } else {
      // LBP1 - 1 = 0..7: fields of plane 0 (r < F) and, if F < 8, plane 1
      constexpr uint32_t F = 32 / W, FM = (1u << W) - 1u;
      constexpr uint32_t kPlanes = F < kLowBits ? 2 : 1;
#pragma unroll
      for (uint32_t pl = 0; pl < kPlanes; ++pl) {
        uint32_t m[4];
        bool touch = false;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
          const uint32_t byte = (v >> (8 * k)) & 0xffu;
          uint32_t mk = 0;
#pragma unroll
          for (uint32_t r = pl * F; r < kLowBits && r < (pl + 1) * F; ++r)
            if ((byte >> r) & 1u) mk |= FM << ((r - pl * F) * W);
          m[k] = mk;
          touch |= mk != 0;
        }
        if (!touch) continue;
        uint4 *p = reinterpret_cast<uint4 *>(s.drv + (uint64_t)pl * d.Zs + j0);
        uint4 w4 = *p;  // planes are Zs words long, Zs a multiple of 4
        w4.x &= ~m[0];
        w4.y &= ~m[1];
        w4.z &= ~m[2];
        w4.w &= ~m[3];
        *p = w4;
      }
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

size_t route_smem(uint32_t ntiles) {
  return kKtabSize * sizeof(KEnt) + kBatchPairs * sizeof(uint32_t) +
         (4 * (size_t)ntiles + 17) * sizeof(uint32_t);
}

template <int W, bool MIXED>
cudaError_t launch_t(const Dims &d, const DevState &s, const BucketDev &bk, const uint32_t *pairs,
                     uint64_t n, const uint64_t *n_dev, cudaStream_t st) {
  auto route = route_kernel<W, MIXED>;
  const size_t smem = route_smem(bk.ntiles);
  cudaError_t e = cudaFuncSetAttribute(route, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kApplySmem);
  if (e != cudaSuccess) return e;
  const uint64_t units = n >> 1;
  const uint64_t pass_units = bk.pass_pairs >> 1;
  const uint64_t passes = units ? (units + pass_units - 1) / pass_units : 0;
  for (uint64_t p = 0; p < passes; ++p) {
    const uint64_t u0 = p * pass_units;
    const uint64_t u1 = std::min(units, u0 + pass_units);
    route<<<bk.ncta, kRouteThreads, smem, st>>>(reinterpret_cast<const uint4 *>(pairs), u0, u1,
                                                n_dev, d, s, bk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    apply_kernel<W><<<bk.ntiles, kApplyThreads, kApplySmem, st>>>(d, s, bk, p == 0,
                                                                  p + 1 == passes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // the odd last pair: the parity of a device-side count is only known on
  // the device, so with n_dev the kernel always runs and decides there
  if ((n & 1u) || n_dev) {
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

// Sizes of the bucketed scan's buffers: a route grid of ncta CTAs, ntiles
// tiles, each CTA's region of a tile holding cap records.  The record buffer
// aims at 2^24 words (64 MiB, so that one pass's records stay in L2), at
// least 2^20 for small pools, and a region is at least 128 records; a pass
// routes as many pairs as fill a region to 80% of (cap - 64) on average,
// which leaves room for the spread of a CTA's share of a tile.
void bucket_layout(uint64_t Z, int sms, BucketDev *bk) {
  const uint64_t nt = (Z + kBucketTile - 1) / kBucketTile;
  const uint64_t ncta = (uint64_t)std::max(sms, 1) * kRouteCtasPerSm;
  const uint64_t budget = std::min<uint64_t>(std::max<uint64_t>(nt * kBucketTile, 1ull << 20),
                                             1ull << 24);
  const uint64_t cap = std::max<uint64_t>(128, budget / (ncta * nt));
  const uint64_t mean = (cap - 64) * 4 / 5;
  bk->ntiles = (uint32_t)nt;
  bk->ncta = (uint32_t)ncta;
  bk->cap = (uint32_t)cap;
  bk->pass_pairs = std::max<uint64_t>((mean * ncta * nt) & ~((uint64_t)kBatchPairs - 1),
                                      kBatchPairs);
}

uint64_t bucket_bytes(const BucketDev &bk) {
  return 4ull * bk.ncta * bk.ntiles * bk.cap + 4ull * bk.ncta * bk.ntiles +
         ((uint64_t)bk.ntiles << kBucketTileLog2);
}

cudaError_t launch_scan_bucketed(const Dims &d, const DevState &s, const BucketDev &bk, int layout,
                                 const uint32_t *pairs, uint64_t n, cudaStream_t st,
                                 const uint64_t *n_dev) {
  if (n == 0) return cudaSuccess;
  return d.group_rule ? launch_m<true>(d, s, bk, layout, pairs, n, n_dev, st)
                      : launch_m<false>(d, s, bk, layout, pairs, n, n_dev, st);
}

}  // namespace vbk
