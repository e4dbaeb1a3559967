// shard.cu -- the steps a VBDR pool spread over several GPUs needs beyond the
// single-GPU path (the paper's data parallelism of Sec. 4.2: pairs are
// independent, and every update is an OR of a bsLBP1 bit or the zeroing of
// a DR, both commutative and idempotent).
//
//   Pair-sharded replicas: each rank scans its share of a slice into a full
//   replica; before the slide the replicas' slice states are merged -- OR
//   of bsLBP1 (gfast), field-wise minimum of the DRs (gsmall), maximum of
//   nowLBP1 (serial) -- and every rank slides the same merged state.
//
//   Pool-partitioned: rank r owns the physical BDRs [r Zr, (r + 1) Zr),
//   Zr = ceil(Z / ranks).  Each rank hashes its share of the pairs into
//   4-byte records pidx << 5 | (LBP1 - 1) grouped by owner, the ranks
//   exchange them (all-to-all), each applies the records it received to its
//   own range and slides; the other ranges of its pool stay empty, so their
//   registers are 0 and a byte-wise maximum over the ranks' register arrays
//   gives the whole pool's registers, installed with vbdr_set_registers.
//
// The exchange itself is the caller's (NCCL, or any transport): these calls
// only read and write device buffers.
#include <algorithm>

#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kRouteThreads = 256;
constexpr int kRoutePairs = 8;  // pairs per thread per batch
constexpr uint32_t kBatch = kRouteThreads * kRoutePairs;
constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_and(uint32_t *p, uint32_t v) {
  asm volatile("red.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void byte_max(uint32_t *w, uint32_t sh, uint32_t v) {
  uint32_t old = *w;
  for (int it = 0; it < 256 && ((old >> sh) & 0xffu) < v; ++it) {
    const uint32_t seen = atomicCAS(w, old, (old & ~(0xffu << sh)) | (v << sh));
    if (seen == old) break;
    old = seen;
  }
}

// Records of n pairs grouped by owner rank: a block counting-sorts a batch
// of records by owner in shared memory, reserves room in every owner's
// group with one global atomic, and copies its runs out.  A record whose
// group is full is counted but not written (the caller sees fill > cap).
__global__ void __launch_bounds__(kRouteThreads)
    route_records_kernel(const uint32_t *__restrict__ pairs, uint64_t n, Dims d, DevState s,
                         uint32_t ranks, uint64_t zr, uint32_t *__restrict__ recs, uint64_t cap,
                         unsigned long long *__restrict__ fill) {
  __shared__ KEnt kt[kKtabSize];
  __shared__ uint32_t rec_s[kBatch];
  __shared__ uint16_t own_s[kBatch];
  __shared__ uint32_t cnt[kMaxRanks], off[kMaxRanks];
  __shared__ unsigned long long base[kMaxRanks];
  __shared__ uint32_t total;
  const uint32_t tid = threadIdx.x;
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  for (uint32_t i = tid; i < gmax; i += kRouteThreads) kt[i] = s.ktab[i];
  for (uint64_t b0 = (uint64_t)blockIdx.x * kBatch; b0 < n; b0 += (uint64_t)gridDim.x * kBatch) {
    for (uint32_t r = tid; r < ranks; r += kRouteThreads) cnt[r] = 0;
    __syncthreads();
    uint32_t key[kRoutePairs], own[kRoutePairs], slot[kRoutePairs];
#pragma unroll
    for (int u = 0; u < kRoutePairs; ++u) {
      const uint64_t i = b0 + tid + (uint64_t)u * kRouteThreads;
      key[u] = kNone;
      own[u] = 0;
      if (i < n) {
        const uint32_t aip = pairs[2 * i], bip = pairs[2 * i + 1];
        const uint32_t b = host_b(d, aip);
        const uint32_t bipp = hash32(bip, d.K1);
        const uint32_t vidx = bipp >> (32 - b);
        const uint32_t r0 = min((uint32_t)__clz(bipp << b), 31u - b);
        const uint32_t pidx = reduce32(hash32(aip, kt[vidx]), d.zmul);
        if (vbk_check(pidx < d.Z, s.check, kChkPidx) && vbk_check(r0 < d.R, s.check, kChkRho)) {
          key[u] = (pidx << 5) | r0;
          own[u] = (uint32_t)(pidx / zr);
        }
      }
      slot[u] = key[u] != kNone ? atomicAdd(&cnt[own[u]], 1u) : 0u;
    }
    __syncthreads();
    for (uint32_t r = tid; r < ranks; r += kRouteThreads)
      base[r] = cnt[r] ? atomicAdd(fill + r, (unsigned long long)cnt[r]) : 0ull;
    if (tid == 0) {
      uint32_t run = 0;
      for (uint32_t r = 0; r < ranks; ++r) {
        off[r] = run;
        run += cnt[r];
      }
      total = run;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kRoutePairs; ++u)
      if (key[u] != kNone) {
        rec_s[off[own[u]] + slot[u]] = key[u];
        own_s[off[own[u]] + slot[u]] = (uint16_t)own[u];
      }
    __syncthreads();
    for (uint32_t i = tid; i < total; i += kRouteThreads) {
      const uint32_t r = own_s[i];
      const unsigned long long pos = base[r] + (i - off[r]);
      if (pos < cap) recs[(uint64_t)r * cap + pos] = rec_s[i];
    }
    __syncthreads();
  }
}

// Records pidx << 5 | (LBP1 - 1) applied to the state: Alg. 7 (gfast),
// Alg. 9 (gsmall) or Alg. 4's maximum (serial), test first.
template <int W>
__global__ void __launch_bounds__(256)
    apply_records_kernel(const uint32_t *__restrict__ recs, uint64_t n, Dims d, DevState s) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t rec = recs[i];
    const uint32_t pidx = rec >> 5, r0 = rec & 31u;
    if (!vbk_check(pidx < d.Z, s.check, kChkPidx) || !vbk_check(r0 < d.R, s.check, kChkRho))
      continue;
    if constexpr (W == 0) {
      const uint32_t m = 1u << r0;
      if (!(__ldcg(s.bs + pidx) & m)) red_or(s.bs + pidx, m);
    } else if constexpr (W < 0) {
      uint32_t *w = reinterpret_cast<uint32_t *>(s.now) + (pidx >> 2);
      byte_max(w, 8u * (pidx & 3u), r0 + 1u);
    } else {
      constexpr uint32_t F = 32 / W, FM = (1u << W) - 1u;
      uint32_t *w = s.drv + (uint64_t)(r0 / F) * d.Zs + pidx;
      const uint32_t m = FM << ((r0 % F) * W);
      if (__ldcg(w) & m) red_and(w, ~m);
    }
  }
}

// Field-wise minimum of two DRV words of w-bit fields.
template <int W>
__device__ __forceinline__ uint32_t field_min(uint32_t a, uint32_t b) {
  constexpr uint32_t F = 32 / W, FM = (1u << W) - 1u;
  uint32_t out = 0;
#pragma unroll
  for (uint32_t f = 0; f < F; ++f) {
    const uint32_t x = (a >> (f * W)) & FM, y = (b >> (f * W)) & FM;
    out |= (x < y ? x : y) << (f * W);
  }
  return out | (a & ~((F * W >= 32) ? 0xffffffffu : ((1u << (F * W)) - 1u)));
}

// Merge another replica's slice state into this one.
template <int W>
__global__ void __launch_bounds__(256)
    merge_kernel(const uint32_t *__restrict__ other, uint64_t words, Dims d, DevState s) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
    const uint32_t o = other[i];
    if constexpr (W == 0) {
      s.bs[i] |= o;
    } else if constexpr (W < 0) {
      uint32_t *w = reinterpret_cast<uint32_t *>(s.now) + i;
      const uint32_t a = *w;
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t x = (a >> (8 * q)) & 0xffu, y = (o >> (8 * q)) & 0xffu;
        m |= (x > y ? x : y) << (8 * q);
      }
      *w = m;
    } else {
      s.drv[i] = field_min<W>(s.drv[i], o);
    }
  }
}

template <int W>
cudaError_t launch_apply_w(const Dims &d, const DevState &s, const uint32_t *recs, uint64_t n,
                           cudaStream_t st) {
  const uint64_t grid = std::min<uint64_t>((n + 255) / 256, 152ull * 8);
  apply_records_kernel<W><<<(unsigned)grid, 256, 0, st>>>(recs, n, d, s);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_merge_w(const Dims &d, const DevState &s, const uint32_t *other, uint64_t words,
                           cudaStream_t st) {
  const uint64_t grid = std::min<uint64_t>((words + 255) / 256, 152ull * 8);
  merge_kernel<W><<<(unsigned)grid, 256, 0, st>>>(other, words, d, s);
  return cudaGetLastError();
}

template <template <int> class Fn, typename... A>
cudaError_t by_layout(int layout, uint32_t w, A... a) {
  if (layout == kLayoutGfast) return Fn<0>::run(a...);
  if (layout == kLayoutSerial) return Fn<-1>::run(a...);
  switch (w) {
    case 1: return Fn<1>::run(a...);
    case 2: return Fn<2>::run(a...);
    case 3: return Fn<3>::run(a...);
    case 4: return Fn<4>::run(a...);
    case 5: return Fn<5>::run(a...);
    case 6: return Fn<6>::run(a...);
    case 7: return Fn<7>::run(a...);
    case 8: return Fn<8>::run(a...);
    default: return cudaErrorInvalidValue;
  }
}

template <int W>
struct ApplyFn {
  static cudaError_t run(const Dims &d, const DevState &s, const uint32_t *r, uint64_t n,
                         cudaStream_t st) {
    return launch_apply_w<W>(d, s, r, n, st);
  }
};
template <int W>
struct MergeFn {
  static cudaError_t run(const Dims &d, const DevState &s, const uint32_t *o, uint64_t words,
                         cudaStream_t st) {
    return launch_merge_w<W>(d, s, o, words, st);
  }
};

}  // namespace

cudaError_t launch_route_records(const Dims &d, const DevState &s, const uint32_t *pairs, uint64_t n,
                                 uint32_t ranks, uint32_t *recs, uint64_t cap,
                                 unsigned long long *fill, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(fill, 0, ranks * sizeof(unsigned long long), st);
  if (e != cudaSuccess || n == 0) return e;
  const uint64_t zr = (d.Z + ranks - 1) / ranks;
  const uint64_t grid = std::min<uint64_t>((n + kBatch - 1) / kBatch, 152ull * 4);
  route_records_kernel<<<(unsigned)grid, kRouteThreads, 0, st>>>(pairs, n, d, s, ranks, zr, recs,
                                                                  cap, fill);
  return cudaGetLastError();
}

cudaError_t launch_apply_records(const Dims &d, const DevState &s, int layout, const uint32_t *recs,
                                 uint64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return by_layout<ApplyFn>(layout, d.w, d, s, recs, n, st);
}

cudaError_t launch_merge_slice_state(const Dims &d, const DevState &s, int layout,
                                     const uint32_t *other, uint64_t words, cudaStream_t st) {
  if (words == 0) return cudaSuccess;
  return by_layout<MergeFn>(layout, d.w, d, s, other, words, st);
}

}  // namespace vbk
