// plan.cu -- planned estimate for a fixed host list (Sec. 4.1 Alg. 5 with
// Alg. 3, evaluated register-chunk by register-chunk).
//
// The plain estimate (estimate.cu) gathers every virtual register of every
// host from the byte array reg[Z]: H g random one-byte reads, bound by the
// L2 random-sector rate.  The map from (host, virtual index i) to physical
// BDR (Alg. 3) depends only on the host address, i and the handle's
// configuration, so for a host list that is estimated again after every
// slide it can be computed once.  A plan stores it sorted by register chunk
// (2^15 BDRs, 32 KiB of reg):
//
//   hosts are cut into blocks of HB (<= 7000); for block blk and chunk c the
//   group (blk, c) lists, for every virtual register of the block's hosts
//   that Alg. 3 sends into chunk c, (local host << 15) | (pidx mod 2^15);
//   groups are padded to whole uint4s with entries of a spare host slot.
//
// The planned estimate runs one CTA per block: a producer warp streams reg
// chunk by chunk, together with the chunk's group of entries, into a 3-slot
// shared-memory ring with TMA bulk copies (cp.async.bulk, completion on an
// mbarrier); 31 consumer warps walk the staged group, read each register
// from shared memory and add its term to the host's exact sums with one
// shared atomic:
//   M = 0      -> V   += 1                 (contributes 2^32 to S)
//   M in 1..16 -> Shi += 2^(16 - M)        (2^(32-M) = Shi unit 2^16)
//   M > 16     -> Slo += 2^(32 - M)
// so S = V 2^32 + Shi 2^16 + Slo exactly (each field < 2^32 for g <= 2^16).
// The sums are the same integers as the gather kernel's; the finish is the
// same function (host_estimate), so both estimates agree bit for bit.
//
// Every wait on an mbarrier is bounded (0.2 s of %globaltimer); a wait that
// expires sets the plan's error word, the producer first waits (bounded) for
// its copies in flight, and the block's outputs are written as NaN.
#include "vbdr_internal.cuh"
#include "async_sm100.cuh"
#include "packed_f32x2.cuh"

namespace vbk {
namespace {

constexpr uint32_t kEntCap = 4096;  // entries of a group staged in shared memory
constexpr int kConsumerWarps = 31;
constexpr int kPlanThreads = (kConsumerWarps + 1) * 32;
constexpr int kBuildThreads = 1024;
constexpr uint32_t kChunkBytes = (uint32_t)kPlanChunk;

// Every mbarrier wait gives up after this long (a wait that long is a failure).
constexpr uint64_t kPlanWaitNs = 200000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  return mbar_wait_bounded(b, parity, kPlanWaitNs);
}

__device__ __forceinline__ uint4 ld_stream(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Block blk's hosts: [blk HB, min((blk + 1) HB, n)).
__device__ __forceinline__ uint32_t block_hosts(const PlanDev &p, uint32_t blk) {
  const uint64_t h0 = (uint64_t)blk * p.HB;
  const uint64_t left = p.n - h0;
  return left < p.HB ? (uint32_t)left : p.HB;
}

// Building, pass 1: per block, the number of virtual registers that Alg. 3
// sends into each chunk (shared counters, then one store per chunk).
__global__ void __launch_bounds__(kBuildThreads)
    plan_count_kernel(Dims d, DevState s, PlanDev p) {
  extern __shared__ uint32_t cnt[];
  const uint32_t blk = blockIdx.x;
  for (uint32_t c = threadIdx.x; c < p.nchunks; c += blockDim.x) cnt[c] = 0;
  __syncthreads();
  const uint32_t nh = block_hosts(p, blk);
  const uint32_t *aips = p.aips + (uint64_t)blk * p.HB;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (uint32_t h = warp; h < nh; h += warps) {
    const uint32_t aip = aips[h];
    const uint32_t g = 1u << host_b(d, aip);
    for (uint32_t i = lane; i < g; i += 32) {
      const uint32_t pidx = reduce32(hash32(aip, s.ktab[i]), d.zmul);
      if (!vbk_check(pidx < d.Z, s.check, kChkPidx)) continue;
      atomicAdd(&cnt[pidx >> kPlanChunkLog2], 1u);
    }
  }
  __syncthreads();
  for (uint32_t c = threadIdx.x; c < p.nchunks; c += blockDim.x)
    p.counts[(uint64_t)blk * p.nchunks + c] = cnt[c];
}

// Building, pass 2: every virtual register takes the next free slot of its
// group (the slot order within a group is immaterial: the sums are exact).
__global__ void __launch_bounds__(kBuildThreads)
    plan_fill_kernel(Dims d, DevState s, PlanDev p) {
  extern __shared__ uint32_t cur[];
  const uint32_t blk = blockIdx.x;
  for (uint32_t c = threadIdx.x; c < p.nchunks; c += blockDim.x) cur[c] = 0;
  __syncthreads();
  const uint32_t nh = block_hosts(p, blk);
  const uint32_t *aips = p.aips + (uint64_t)blk * p.HB;
  const unsigned long long *goff = p.goff + (uint64_t)blk * p.nchunks;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (uint32_t h = warp; h < nh; h += warps) {
    const uint32_t aip = aips[h];
    const uint32_t g = 1u << host_b(d, aip);
    for (uint32_t i = lane; i < g; i += 32) {
      const uint32_t pidx = reduce32(hash32(aip, s.ktab[i]), d.zmul);
      if (!vbk_check(pidx < d.Z, s.check, kChkPidx)) continue;
      const uint32_t c = pidx >> kPlanChunkLog2;
      const uint32_t slot = atomicAdd(&cur[c], 1u);
      p.entries[goff[c] + slot] = (h << kPlanChunkLog2) | (pidx & (kChunkBytes - 1));
    }
  }
  __syncthreads();
  // the group's padding: entries of the spare host slot kPlanMaxHB
  for (uint32_t c = threadIdx.x; c < p.nchunks; c += blockDim.x)
    for (unsigned long long q = goff[c] + cur[c]; q < goff[c + 1]; ++q) p.entries[q] = kPlanPad;
}

// Building, pass 3: the order of a group's staged entries (the first
// kEntCap) is chosen so that the 32 entries one warp instruction takes --
// lane L holds the uint4 at position 32 r + L, so for component j the
// entries at 128 r + 4 L + j -- meet 32 different shared-memory banks
// wherever the group allows it: entry positions with (pos >> 2) mod 32 = b
// are given to entries of bank b, in order; the entries left over fill the
// remaining positions.  The bank is the register byte's (plain plans: the
// chunk reads) or the host's (learned plans: the histogram atomics, see
// take_bin).  The sums are order independent, so the results do not change.
constexpr uint32_t kSortThreads = 1024;
// The bank an entry's position asks for: its register byte's bank (plain
// plans: the reads of the chunk then take distinct banks), or its host's
// index mod 32 (learned plans: the histogram atomics' bank follows the host)
__device__ __forceinline__ uint32_t sort_bank(uint32_t e, int by_host) {
  return by_host ? (e >> kPlanChunkLog2) & 31u : ((e & (kChunkBytes - 1)) >> 2) & 31u;
}
constexpr size_t kSortSmem = kEntCap * (3 * sizeof(uint32_t) + sizeof(uint16_t));
__global__ void __launch_bounds__(kSortThreads)
    plan_sort_kernel(PlanDev p, int by_host) {
  extern __shared__ uint32_t sort_smem[];  // kSortSmem bytes
  uint32_t *in = sort_smem, *out = sort_smem + kEntCap, *hole = sort_smem + 2 * kEntCap;
  uint16_t *rank = reinterpret_cast<uint16_t *>(sort_smem + 3 * kEntCap);
  __shared__ uint32_t cnt[32], cap[32], warp_holes[32], n_left;
  const uint32_t blk = blockIdx.x, tid = threadIdx.x;
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const unsigned long long *goff = p.goff + (uint64_t)blk * p.nchunks;
  for (uint32_t c = 0; c < p.nchunks; ++c) {
    const unsigned long long q0 = goff[c], len = goff[c + 1] - q0;
    const uint32_t P = len < kEntCap ? (uint32_t)len : kEntCap;  // a multiple of 4
    if (P == 0) continue;
    if (tid < 32) cnt[tid] = 0;
    if (tid == 0) n_left = 0;
    __syncthreads();
    for (uint32_t i = tid; i < P; i += kSortThreads) {
      const uint32_t e = p.entries[q0 + i];
      in[i] = e;
      rank[i] = (uint16_t)atomicAdd(&cnt[sort_bank(e, by_host)], 1u);
    }
    // positions of bank b: 128 r + 4 b + j < P
    if (tid < 32) {
      const uint32_t full = P / 128, rest = P % 128;
      const uint32_t lo = 4 * tid;
      cap[tid] = 4 * full + (rest > lo ? min(rest - lo, 4u) : 0u);
    }
    for (uint32_t i = tid; i < P; i += kSortThreads) out[i] = 0xffffffffu;
    __syncthreads();
    for (uint32_t i = tid; i < P; i += kSortThreads) {
      const uint32_t e = in[i], b = sort_bank(e, by_host), k = rank[i];
      if (k < cap[b]) out[128 * (k >> 2) + 4 * b + (k & 3)] = e;
    }
    __syncthreads();
    // the free positions, in increasing order (block-wide count of each
    // thread's run of 4 positions)
    uint32_t mine = 0;
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t pos = 4 * tid + j;
      mine += pos < P && out[pos] == 0xffffffffu;
    }
    uint32_t x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) warp_holes[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = warp_holes[lane], v = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += y;
      }
      warp_holes[lane] = v - w;  // exclusive prefix over warps
    }
    __syncthreads();
    uint32_t h = warp_holes[warp] + x - mine;
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t pos = 4 * tid + j;
      if (pos < P && out[pos] == 0xffffffffu) hole[h++] = pos;
    }
    __syncthreads();
    for (uint32_t i = tid; i < P; i += kSortThreads) {
      const uint32_t e = in[i], b = sort_bank(e, by_host);
      if (rank[i] >= cap[b]) out[hole[atomicAdd(&n_left, 1u)]] = e;
    }
    __syncthreads();
    for (uint32_t i = tid; i < P; i += kSortThreads) p.entries[q0 + i] = out[i];
    __syncthreads();
  }
}

// ----- the ring of the planned kernels -----
// A 3-slot shared-memory ring; slot k holds one step: a 32 KiB register chunk
// (from L2, the register array is small) and the chunk's group of entries
// (its first ECAP entries, from DRAM), both TMA bulk copies completing on the
// slot's full barrier.  Beside them the producer leaves the group's size (in
// uint4s) and offset, so the consumers need no global load per step.  Block
// blk visits the chunks in the rotated order c0, c0 + 1, ... (mod nchunks)
// from c0 = blk nchunks / NB: at any moment the blocks read different
// chunks, where a common order makes all SMs read one chunk at once and
// concentrates the register stream on a few L2 slices.
constexpr uint32_t kRingSlots = 3;
template <uint32_t ECAP>
struct PlanRing {
  unsigned char reg[kRingSlots][kChunkBytes];
  uint4 ents[kRingSlots][ECAP / 4];
  unsigned long long lo[kRingSlots];
  uint32_t nq[kRingSlots];
  uint64_t full[kRingSlots], empty[kRingSlots];
};

__device__ __forceinline__ uint32_t first_chunk(uint32_t blk, uint32_t nblk, uint32_t nch) {
  return (uint32_t)(((uint64_t)blk * nch) / nblk);
}

template <uint32_t ECAP>
__device__ void ring_init(PlanRing<ECAP> &r) {
  for (uint32_t i = 0; i < kRingSlots; ++i) {
    mbar_init(&r.full[i], 1);
    mbar_init(&r.empty[i], kConsumerWarps);
  }
}

// The producer warp: step ch into slot ch mod 3 once the consumers released
// the slot's previous step; lane 0 issues the copies.  The group offsets of
// the chunks are read 32 steps at a time, one per lane, a batch ahead of
// use, and handed to lane 0 by shuffles: a load per step would put an L2
// round trip into the issue of every 16th step.  false if a wait expired;
// every copy issued has landed (or its wait expired) when it returns.
template <uint32_t ECAP>
__device__ bool ring_produce(PlanRing<ECAP> &r, const DevState &s, const PlanDev &p,
                             const unsigned long long *goff, uint32_t c0, uint32_t nch) {
  const uint32_t lane = threadIdx.x & 31u;
  // offsets (lo, hi) of the chunk of step base + lane
  auto fetch = [&](uint32_t base, unsigned long long &lo, unsigned long long &hi) {
    lo = hi = 0;
    if (base + lane < nch) {
      const uint32_t c = (uint32_t)(((uint64_t)c0 + base + lane) % nch);
      lo = goff[c];
      hi = goff[c + 1];
    }
  };
  unsigned long long cur_lo, cur_hi, nxt_lo, nxt_hi;
  fetch(0, cur_lo, cur_hi);
  fetch(32, nxt_lo, nxt_hi);
  bool ok = true;
  uint32_t issued = 0, cc = c0, slot = 0, par = 0;
  for (uint32_t ch = 0; ch < nch; ++ch) {
    if (ch && (ch & 31u) == 0) {
      cur_lo = nxt_lo;
      cur_hi = nxt_hi;
      fetch(ch + 32, nxt_lo, nxt_hi);
    }
    const unsigned long long lo = __shfl_sync(0xffffffffu, cur_lo, ch & 31u);
    const unsigned long long hi = __shfl_sync(0xffffffffu, cur_hi, ch & 31u);
    if (ch >= kRingSlots) {
      const bool done = mbar_wait(&r.empty[slot], par ^ 1u);
      if (!__all_sync(0xffffffffu, done)) {
        ok = false;
        break;
      }
    }
    if (lane == 0) {
      const unsigned long long ne = hi - lo;
      const uint32_t bytes = 4u * (uint32_t)(ne < ECAP ? ne : ECAP);
      // published to the consumers by the arrive below (release) and their
      // wait on the barrier (acquire)
      r.lo[slot] = lo;
      r.nq[slot] = (uint32_t)(ne >> 2);
      mbar_expect_tx(&r.full[slot], kChunkBytes + bytes);
      bulk_load_g2s(r.reg[slot], s.reg + (uint64_t)cc * kChunkBytes, kChunkBytes, &r.full[slot]);
      if (bytes) bulk_load_g2s(r.ents[slot], p.entries + lo, bytes, &r.full[slot]);
    }
    __syncwarp();
    issued = ch + 1;
    if (++cc == nch) cc = 0;
    if (++slot == kRingSlots) {
      slot = 0;
      par ^= 1u;
    }
  }
  // the last phase of every slot used: each issued copy lands before the
  // block may finish
  for (uint32_t ch = issued > kRingSlots ? issued - kRingSlots : 0u; ch < issued; ++ch)
    if (!mbar_wait(&r.full[ch % kRingSlots], (ch / kRingSlots) & 1u)) ok = false;
  return __all_sync(0xffffffffu, ok);
}

// The consumers (warps 0 .. kConsumerWarps - 1): for every step, take(ring,
// e) on each entry of the step's group (ring: the step's register chunk).
// Thread t starts at uint4 (t + 160 step) mod T of a group: the threads left
// without work by a group smaller than T move by five warps from step to
// step, so no warp idles more than the others.  A group larger than ECAP is
// finished from global memory.  false if a wait expired.
template <uint32_t ECAP, class Take>
__device__ bool ring_consume(PlanRing<ECAP> &r, const PlanDev &p, uint32_t nch, Take &&take) {
  const uint32_t T = kConsumerWarps * 32, lane = threadIdx.x & 31u;
  uint32_t lead = threadIdx.x, slot = 0, par = 0;
  for (uint32_t ch = 0; ch < nch; ++ch) {
    if (!mbar_wait(&r.full[slot], par)) return false;
    const unsigned char *ring = r.reg[slot];
    const uint4 *ents = r.ents[slot];
    const uint32_t nq = r.nq[slot], nq_s = min(nq, ECAP / 4);
    for (uint32_t q = lead; q < nq_s; q += T) {
      const uint4 e = ents[q];
      take(ring, e.x);
      take(ring, e.y);
      take(ring, e.z);
      take(ring, e.w);
    }
    if (nq > ECAP / 4) {
      const uint4 *grp = reinterpret_cast<const uint4 *>(p.entries) + (r.lo[slot] >> 2);
      for (uint32_t q = ECAP / 4 + lead; q < nq; q += T) {
        const uint4 e = ld_stream(grp + q);
        take(ring, e.x);
        take(ring, e.y);
        take(ring, e.z);
        take(ring, e.w);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.empty[slot]);
    lead += 160u;
    if (lead >= T) lead -= T;
    if (++slot == kRingSlots) {
      slot = 0;
      par ^= 1u;
    }
  }
  return true;
}

// ----- the planned estimate -----
// Per host three 32-bit words, one shared atomic per plan entry:
//   M = 0      -> V   += 1                 (contributes 2^32 to S)
//   M in 1..16 -> Shi += 2^(16 - M)        (2^(32-M) = Shi unit 2^16)
//   M > 16     -> Slo += 2^(32 - M)
// so S = V 2^32 + Shi 2^16 + Slo exactly (each field < 2^32 for g <= 2^16).
// The kernel with the compact learned correction also needs the counts of
// the register values 0..3, and packs them into the same three words:
//   M = 0, 1, 2  -> P += 2^(10 M)        (#{M = 0} = V, #{M = 1}, #{M = 2}
//                                         in three 10-bit fields)
//   M = 3        -> H += 2^22            (#{M = 3} in H's bits 22..31)
//   M in 4..16   -> H += 2^(16 - M)
//   M > 16       -> L += 2^(32 - M)
// For g <= 512 every count is at most 512 < 2^10 and the low part of H at
// most 512 2^12 = 2^21 < 2^22, so no field overflows into the next and
//   S = V 2^32 + n1 2^31 + n2 2^30 + n3 2^29 + (H mod 2^22) 2^16 + L.
constexpr uint32_t kAccRow = kPlanMaxHB + 1;  // + the spare slot of padding entries
struct PlanSmem {
  PlanRing<kEntCap> r;
  uint32_t acc[3][kAccRow];  // V, Shi, Slo (packed: P, H, L)
  double nZZ;
  int bad;
};
static_assert(sizeof(PlanSmem) <= 227 * 1024, "shared memory of one CTA");

// One entry: register M of the chunk in the ring, added to its host's words.
// which = (M + 15) >> 4 picks V (M = 0), Shi (1..16) or Slo (17..32), and
// 1 << ((16 - M) & 15) is 1, 2^(16-M) or 2^(32-M) respectively.  The word
// index is at most 2, the shift below 32 and the host slot at most
// kPlanMaxHB, so every access stays inside the accumulators whatever the
// entry or register value.
template <bool PACKED>
__device__ __forceinline__ void take(const unsigned char *ring, uint32_t *acc, uint32_t e,
                                     unsigned int *chk) {
  const uint32_t M = ring[e & (kChunkBytes - 1)];
  if (!vbk_check(M <= 32u && (e >> kPlanChunkLog2) <= kPlanMaxHB, chk, kChkPlan)) return;
  const uint32_t lh = min(e >> kPlanChunkLog2, kPlanMaxHB);
  if constexpr (PACKED) {
    const bool low = M <= 2u;
    const uint32_t which = low ? 0u : min((M + 15u) >> 4, 2u);
    const uint32_t sh = low ? 10u * M : (M == 3u ? 22u : (16u - M) & 15u);
    atomicAdd(acc + which * kAccRow + lh, 1u << sh);
  } else {
    const uint32_t which = min((M + 15u) >> 4, 2u);
    atomicAdd(acc + which * kAccRow + lh, 1u << ((16u - M) & 15u));
  }
}

// The compact learned correction (not in the paper): ten inputs -- the
// counts of register values 0..3 over g, log2 g / 16, ln(1 + n_plain) / 16,
// ln(1 + n_g) / 16, ln(1 + n_Z / Z), V_Z / Z, V / g -- through two layers of
// 16 tanh-form GELUs to delta; the estimate becomes
// max(0, exp(ln(1 + n_plain) + delta) - 1) unless n_plain > nmax.  FP32 with
// the fast exponential, logarithm and division (each within a few ulp; the
// network is a correction of order one, so absolute errors of 1e-6 are
// immaterial).  Parameters: W1 [16][10], b1 [16], W2 [16][16], b2 [16],
// w3 [16], b3.
constexpr int kCIn = 10, kCHid = 16;
constexpr int kCParams = kCHid * kCIn + kCHid + kCHid * kCHid + kCHid + kCHid + 1;
static_assert(kCParams == kCompactParams, "parameter count of the compact network");
// Offsets of the parameters in CompactParams::w (the API's layout).
constexpr int kCW1 = 0, kCB1 = kCW1 + kCHid * kCIn, kCW2 = kCB1 + kCHid,
              kCB2 = kCW2 + kCHid * kCHid, kCW3 = kCB2 + kCHid, kCB3 = kCW3 + kCHid;

// The network runs on pairs of units with Blackwell's packed FP32 arithmetic
// (fma.rn.f32x2 / mul.rn.f32x2: two IEEE single-precision operations per
// instruction, each rounded as its scalar form).  The launcher reorders the
// weights into unit pairs -- W1 pair (i, p) = (W1[2p][i], W1[2p+1][i]), and
// so on for b1, W2, b2, w3 -- and passes them by value: every launch carries
// its own copy in the kernel's parameter space, where the unrolled network
// reads each pair as an operand (no shared-memory load per weight).
struct CompactPairs {
  float2 w1[kCIn][kCHid / 2];
  float2 b1[kCHid / 2];
  float2 w2[kCHid][kCHid / 2];
  float2 b2[kCHid / 2];
  float2 w3[kCHid / 2];
  float b3;
};

__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// GELU in its tanh form on two units: z/2 (1 + tanh(u)), u = sqrt(2/pi)
// (z + 0.044715 z^3), written as z / (1 + 2^(z (c1 + c2 z^2))) with
// c1 = -2 sqrt(2/pi) log2(e), c2 = 0.044715 c1: one fast exponential and one
// fast reciprocal per unit.
__device__ __forceinline__ float2 gelu2(float2 z) {
  constexpr float c1 = -2.0f * 0.7978845608028654f * 1.4426950408889634f;
  constexpr float c2 = 0.044715f * c1;
  const float2 t = f2_mul(z, f2_fma(f2_mul(z, z), make_float2(c2, c2), make_float2(c1, c1)));
  const float2 r = make_float2(rcp_fast(1.0f + ex2_fast(t.x)), rcp_fast(1.0f + ex2_fast(t.y)));
  return f2_mul(z, r);
}

__device__ __forceinline__ float compact_delta(const CompactPairs &P, const float (&x)[kCIn]) {
  constexpr int NP = kCHid / 2;
  float2 h1[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) h1[p] = P.b1[p];
#pragma unroll
  for (int i = 0; i < kCIn; ++i) {
    const float2 xi = make_float2(x[i], x[i]);
#pragma unroll
    for (int p = 0; p < NP; ++p) h1[p] = f2_fma(P.w1[i][p], xi, h1[p]);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) h1[p] = gelu2(h1[p]);
  float2 h2[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) h2[p] = P.b2[p];
#pragma unroll
  for (int i = 0; i < kCHid; ++i) {
    const float hi = (i & 1) ? h1[i >> 1].y : h1[i >> 1].x;
    const float2 hb = make_float2(hi, hi);
#pragma unroll
    for (int p = 0; p < NP; ++p) h2[p] = f2_fma(P.w2[i][p], hb, h2[p]);
  }
  float2 acc0 = make_float2(0.0f, 0.0f), acc1 = acc0;
#pragma unroll
  for (int p = 0; p < NP; p += 2) {
    acc0 = f2_fma(P.w3[p], gelu2(h2[p]), acc0);
    acc1 = f2_fma(P.w3[p + 1], gelu2(h2[p + 1]), acc1);
  }
  return P.b3 + ((acc0.x + acc0.y) + (acc1.x + acc1.y));
}

// CORR: also the compact correction's inputs.  Instead of the estimate the
// kernel then writes one record per host for compact_correct_kernel:
// {P (V, n1, n2), n3 | b << 10 | (n_plain > nmax) << 31, n_g, n_plain}, the
// last two as FP32 (n_plain NaN for a block whose wait expired), and after
// them record n = {ln(1 + n_Z / Z), V_Z / Z} (FP32).  The network
// runs in a kernel of its own: here one CTA per SM, capped at 64 registers a
// thread, would evaluate about 6600 hosts' networks with 32 warps.
template <bool CORR>
__global__ void __launch_bounds__(kPlanThreads, 1)
    planned_estimate_kernel(Dims d, DevState s, EstConst c, PlanDev p, float nmax,
                            float *__restrict__ out, uint4 *__restrict__ rec) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PlanSmem &S = *reinterpret_cast<PlanSmem *>(smem_raw);
  const uint32_t blk = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nh = block_hosts(p, blk);
  for (uint32_t i = threadIdx.x; i < 3 * kAccRow; i += blockDim.x) (&S.acc[0][0])[i] = 0;
  if (threadIdx.x == 0) {
    ring_init(S.r);
    S.nZZ = pool_noise(d, s, c);
    S.bad = 0;
  }
  __syncthreads();
  const uint32_t nch = p.nchunks, c0 = first_chunk(blk, p.NB, nch);
  const unsigned long long *goff = p.goff + (uint64_t)blk * nch;
  if (warp == kConsumerWarps) {
    if (!ring_produce(S.r, s, p, goff, c0, nch) && lane == 0) S.bad = 1;
  } else {
    uint32_t *acc = &S.acc[0][0];
    unsigned int *chk = s.check;
    if (!ring_consume(S.r, p, nch,
                      [&](const unsigned char *ring, uint32_t e) { take<CORR>(ring, acc, e, chk); }))
      S.bad = 1;
  }
  __syncthreads();
  const bool bad = S.bad != 0;
  if (bad && threadIdx.x == 0) atomicOr(p.err, 1u);
  const double nZZ = S.nZZ;
  const uint64_t h0 = (uint64_t)blk * p.HB;
  for (uint32_t lh = threadIdx.x; lh < nh; lh += blockDim.x) {
    const uint32_t P = S.acc[0][lh], H = S.acc[1][lh];
    const uint32_t b = host_b(d, p.aips[h0 + lh]);
    if constexpr (CORR) {
      const uint32_t V = P & 1023u, n1 = (P >> 10) & 1023u, n2 = P >> 20, n3 = H >> 22;
      const unsigned long long Sum =
          ((unsigned long long)V << 32) + ((unsigned long long)n1 << 31) +
          ((unsigned long long)n2 << 30) + ((unsigned long long)n3 << 29) +
          ((unsigned long long)(H & 0x3fffffu) << 16) + S.acc[2][lh];
      double n_g = 0.0;
      const double est = host_estimate(Sum, V, b, c, s.lnv, nZZ, &n_g);
      const uint32_t keep = est > (double)nmax ? 1u : 0u;
      const float r = bad ? __int_as_float(0x7fc00000) : (float)est;
      rec[h0 + lh] = make_uint4(P, n3 | (b << 10) | (keep << 31), __float_as_uint((float)n_g),
                                __float_as_uint(r));
      // record n: the pool's two inputs, the same for every host
      if (blk == 0 && lh == 0)
        rec[p.n] = make_uint4(__float_as_uint(__logf(1.0f + (float)nZZ)),
                              __float_as_uint((float)((double)s.sums[1] / (double)d.Z)), 0u, 0u);
    } else {
      const unsigned long long Sum =
          ((unsigned long long)P << 32) + ((unsigned long long)H << 16) + S.acc[2][lh];
      const double est = host_estimate(Sum, P, b, c, s.lnv, nZZ, nullptr);
      out[h0 + lh] = bad ? __int_as_float(0x7fc00000) : (float)est;
    }
  }
}

// The compact correction of n hosts from their records (one thread a host):
// the ten inputs, the network, and max(0, exp(ln(1 + n_plain) + delta) - 1)
// into out; hosts above nmax (and NaN estimates) keep n_plain.
constexpr int kCorrThreads = 256;
__global__ void __launch_bounds__(kCorrThreads)
    compact_correct_kernel(const uint4 *__restrict__ rec, uint64_t n,
                           const __grid_constant__ CompactPairs net,
                           float *__restrict__ out) {
  const uint4 pool = rec[n];  // the pool's two inputs
  const float x_noise = __uint_as_float(pool.x), x_vz = __uint_as_float(pool.y);
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 q = rec[h];
    const float r = __uint_as_float(q.w);
    float o = r;
    if (!(q.y >> 31) && r == r) {
      const uint32_t V = q.x & 1023u, n1 = (q.x >> 10) & 1023u, n2 = q.x >> 20;
      const uint32_t n3 = q.y & 1023u, b = (q.y >> 10) & 31u;
      const float inv_g = __uint_as_float((127u - b) << 23);  // 2^-b, exact
      const float l1p = __logf(1.0f + r);
      const float x[kCIn] = {(float)V * inv_g, (float)n1 * inv_g, (float)n2 * inv_g,
                             (float)n3 * inv_g, (float)b * 0.0625f, l1p * 0.0625f,
                             __logf(1.0f + __uint_as_float(q.z)) * 0.0625f, x_noise, x_vz,
                             (float)V * inv_g};
      o = fmaxf(__expf(l1p + compact_delta(net, x)) - 1.0f, 0.0f);
    }
    out[h] = o;
  }
}

// ----- the learned correction's features from a plan -----
// A plan built for the learned correction has at most kLearnMaxHB hosts per
// block (two waves of one CTA per SM for 1M hosts), so that every host of a
// block can keep a 32-bin histogram of its register values in shared memory:
// 32 one-byte bins per host (8 words, the word of value M at (M / 4) xor
// (host / 4 mod 8)), one shared atomic per plan entry.  A byte bin
// can only reach 256 when all of a host's g >= 256 registers hold one value;
// the bins then no longer sum to g, and that host is recounted exactly from
// the registers (Alg. 3 again, rare).  From the exact counts the block
// derives what the gather kernel computes -- S, V, the plain estimate, the
// feature row -- with the same operations, so both paths give the same bits.
// a learned plan's groups average HB g / chunks (1650 entries for 1M hosts of
// g = 256 over 2^24 registers); the first kLearnEntCap are staged, any rest is
// read from global memory
constexpr uint32_t kLearnEntCap = 2048;
struct LearnSmem {
  PlanRing<kLearnEntCap> r;
  uint32_t bins[kLearnMaxHB + 1][8];  // + the spare slot of padding entries
  double nZZ;
  int bad;
};
static_assert(sizeof(LearnSmem) <= 227 * 1024, "shared memory of one CTA");

__device__ __forceinline__ void take_bin(const unsigned char *ring, uint32_t *bins, uint32_t e,
                                         unsigned int *chk) {
  const uint32_t M = ring[e & (kChunkBytes - 1)];
  if (!vbk_check(M < 32u, chk, kChkPlan)) return;
  // M mod 32 and the host slot at most kLearnMaxHB keep every access inside
  // the bins whatever the entry or register value
  const uint32_t lh = min(e >> kPlanChunkLog2, kLearnMaxHB), m = M & 31u;
  // word (M / 4) of the host's 8, swizzled by host bits 2..4: the values of
  // one warp's entries cluster, so without it their atomics fall in the
  // banks 8 lh + const; with it the bank is 8 (lh mod 4) + (M / 4 xor
  // (lh / 4 mod 8)), all 32 banks for 32 consecutive hosts
  atomicAdd(bins + lh * 8 + ((m >> 2) ^ ((lh >> 2) & 7u)), 1u << (8u * (m & 3u)));
}

// Exact histogram of one host's g virtual registers (Alg. 3, gathered).
__device__ __noinline__ void recount_host(const Dims &d, const DevState &s, uint32_t aip,
                                          uint32_t g, uint16_t *rc) {
  for (int m = 0; m < 32; ++m) rc[m] = 0;
  for (uint32_t i = 0; i < g; ++i) {
    const uint32_t pidx = reduce32(hash32(aip, s.ktab[i]), d.zmul);
    if (!vbk_check(pidx < d.Z, s.check, kChkPidx)) continue;
    const uint32_t M = s.reg[pidx];
    if (vbk_check(M < 32u, s.check, kChkReg)) rc[M & 31u]++;
  }
}

__global__ void __launch_bounds__(kPlanThreads, 1)
    planned_features_kernel(Dims d, DevState s, EstConst c, PlanDev p, float *__restrict__ out,
                            __nv_bfloat16 *__restrict__ feat) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  LearnSmem &S = *reinterpret_cast<LearnSmem *>(smem_raw);
  const uint32_t blk = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nh = block_hosts(p, blk);
  for (uint32_t i = threadIdx.x; i < (kLearnMaxHB + 1) * 8; i += blockDim.x) (&S.bins[0][0])[i] = 0;
  if (threadIdx.x == 0) {
    ring_init(S.r);
    S.nZZ = pool_noise(d, s, c);
    S.bad = 0;
  }
  __syncthreads();
  const uint32_t nch = p.nchunks, c0 = first_chunk(blk, p.NB, nch);
  const unsigned long long *goff = p.goff + (uint64_t)blk * nch;
  if (warp == kConsumerWarps) {
    if (!ring_produce(S.r, s, p, goff, c0, nch) && lane == 0) S.bad = 1;
  } else {
    uint32_t *bins = &S.bins[0][0];
    unsigned int *chk = s.check;
    if (!ring_consume(S.r, p, nch, [&](const unsigned char *ring, uint32_t e) {
          take_bin(ring, bins, e, chk);
        }))
      S.bad = 1;
  }
  __syncthreads();
  const bool bad = S.bad != 0;
  if (bad && threadIdx.x == 0) atomicOr(p.err, 1u);
  const double nZZ = S.nZZ;
  const uint64_t h0 = (uint64_t)blk * p.HB;
  for (uint32_t lh = threadIdx.x; lh < nh; lh += blockDim.x) {
    const uint32_t aip = p.aips[h0 + lh];
    const uint32_t b = host_b(d, aip), g = 1u << b;
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t v = S.bins[lh][w];
      total += (v & 0xffu) + ((v >> 8) & 0xffu) + ((v >> 16) & 0xffu) + (v >> 24);
    }
    // a bin overflowed (the bins no longer sum to g): recount this host from
    // the registers into 16-bit counts
    const bool slow = total != g;
    uint16_t rc[32];
    if (slow) recount_host(d, s, aip, g, rc);
    auto count = [&](int m) -> uint32_t {
      return slow ? (uint32_t)rc[m]
                  : (S.bins[lh][(uint32_t)(m >> 2) ^ ((lh >> 2) & 7u)] >> (8 * (m & 3))) & 0xffu;
    };
    unsigned long long Sum = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) Sum += (unsigned long long)count(m) << (32 - m);
    const uint32_t V = count(0);
    double n_g = 0.0;
    const double est = host_estimate(Sum, V, b, c, s.lnv, nZZ, &n_g);
    const uint64_t row = h0 + lh;
    out[row] = bad ? __int_as_float(0x7fc00000) : (float)est;
    // the feature row: bins / g, then the noise statistics (as the gather
    // kernel writes them), 16 bytes at a time
    const float inv_g = 1.0f / (float)g;
    uint4 *dst = reinterpret_cast<uint4 *>(feat + row * kMlpLive);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __align__(16) __nv_bfloat16 x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = __float2bfloat16((float)count(8 * q + k) * inv_g);
      dst[q] = *reinterpret_cast<const uint4 *>(x);
    }
    __align__(16) __nv_bfloat16 x[16];
    x[0] = __float2bfloat16((float)b * 0.0625f);
    x[1] = __float2bfloat16(log1pf((float)est) * 0.0625f);
    x[2] = __float2bfloat16(log1pf((float)n_g) * 0.0625f);
    x[3] = __float2bfloat16(log1pf((float)nZZ));
    x[4] = __float2bfloat16((float)((double)s.sums[1] / (double)d.Z));
    x[5] = __float2bfloat16((float)V / (float)g);
#pragma unroll
    for (int q = 6; q < 16; ++q) x[q] = __float2bfloat16(0.f);
    dst[4] = reinterpret_cast<const uint4 *>(x)[0];
    dst[5] = reinterpret_cast<const uint4 *>(x)[1];
  }
}

}  // namespace

cudaError_t launch_planned_features(const Dims &d, const DevState &s, const EstConst &c,
                                    const PlanDev &p, float *out, __nv_bfloat16 *feat,
                                    cudaStream_t st) {
  if (p.NB == 0) return cudaSuccess;
  const int smem = (int)sizeof(LearnSmem);
  cudaError_t e = cudaFuncSetAttribute(planned_features_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  planned_features_kernel<<<p.NB, kPlanThreads, smem, st>>>(d, s, c, p, out, feat);
  return cudaGetLastError();
}

cudaError_t launch_plan_count(const Dims &d, const DevState &s, const PlanDev &p, cudaStream_t st) {
  if (p.NB == 0) return cudaSuccess;
  plan_count_kernel<<<p.NB, kBuildThreads, p.nchunks * sizeof(uint32_t), st>>>(d, s, p);
  return cudaGetLastError();
}

cudaError_t launch_plan_fill(const Dims &d, const DevState &s, const PlanDev &p, cudaStream_t st) {
  if (p.NB == 0) return cudaSuccess;
  plan_fill_kernel<<<p.NB, kBuildThreads, p.nchunks * sizeof(uint32_t), st>>>(d, s, p);
  return cudaGetLastError();
}

cudaError_t launch_plan_sort(const PlanDev &p, bool by_host, cudaStream_t st) {
  if (p.NB == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(plan_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSortSmem);
  if (e != cudaSuccess) return e;
  plan_sort_kernel<<<p.NB, kSortThreads, kSortSmem, st>>>(p, by_host ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_planned_estimate(const Dims &d, const DevState &s, const EstConst &c,
                                   const PlanDev &p, const CompactParams *net,
                                   uint4 *compact_rec, float *out, cudaStream_t st) {
  if (p.NB == 0) return cudaSuccess;
  const int smem = (int)sizeof(PlanSmem);
  auto k = net ? planned_estimate_kernel<true> : planned_estimate_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k<<<p.NB, kPlanThreads, smem, st>>>(d, s, c, p, net ? net->nmax : 0.0f, out, compact_rec);
  e = cudaGetLastError();
  if (e != cudaSuccess || !net) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (p.n + kCorrThreads - 1) / kCorrThreads;
  const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
  CompactPairs pr;
  const float *w = net->w;
  for (int i = 0; i < kCIn; ++i)
    for (int q = 0; q < kCHid / 2; ++q)
      pr.w1[i][q] = make_float2(w[kCW1 + (2 * q) * kCIn + i], w[kCW1 + (2 * q + 1) * kCIn + i]);
  for (int i = 0; i < kCHid; ++i)
    for (int q = 0; q < kCHid / 2; ++q)
      pr.w2[i][q] = make_float2(w[kCW2 + (2 * q) * kCHid + i], w[kCW2 + (2 * q + 1) * kCHid + i]);
  for (int q = 0; q < kCHid / 2; ++q) {
    pr.b1[q] = make_float2(w[kCB1 + 2 * q], w[kCB1 + 2 * q + 1]);
    pr.b2[q] = make_float2(w[kCB2 + 2 * q], w[kCB2 + 2 * q + 1]);
    pr.w3[q] = make_float2(w[kCW3 + 2 * q], w[kCW3 + 2 * q + 1]);
  }
  pr.b3 = w[kCB3];
  compact_correct_kernel<<<(unsigned)(want < cap ? want : cap), kCorrThreads, 0, st>>>(
      compact_rec, p.n, pr, out);
  return cudaGetLastError();
}

}  // namespace vbk
