// vbdr_internal.cuh -- device-side definitions shared by the VBDR kernels.
//
// Data layout in HBM (per handle, Z physical BDRs):
//   drv   : P word planes of Z uint32 each, plane-major (drv[p * Zs + j],
//           Zs = Z rounded up to a multiple of 4 so every plane is 16 B
//           aligned for vector access).
//           Word p of BDR j packs the DRs of LBP1 values p*F+1 .. p*F+F,
//           F = floor(32 / w) fields of w bits, field f at bits [f*w, f*w+w).
//           Plane-major puts every BDR's first word (LBP1 1..F, which takes
//           1 - 2^-F of all updates because LBP1 is geometric) into one
//           contiguous 4*Z-byte plane, so the hot random updates of the
//           gsmall scan touch a quarter of the DRV footprint.
//   bs    : Z uint32, bsLBP1 of the gfast layout (bit r-1 <-> LBP1 r).
//   now   : Zs uint8, nowLBP1 of the serial layout (the slice's largest LBP1).
//   reg   : Z uint8, register of every BDR at the last slide (Alg. 2).
//   ktab  : max(g_max, 512) KEnt, the premixed seed mix64(s1(i)) of virtual
//           index i, s1(i) = H(i,2^32,A0) (the first hash of Alg. 3, which
//           depends only on i), split as KEnt.
//   sums  : pool sums S_Z, V_Z and the block-completion counter of the slide.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlp_device.cuh"

struct vbdr_mlp;

namespace vbk {

constexpr int kMaxLog2G = 16;
constexpr int kLayoutGfast = 0, kLayoutGsmall = 1, kLayoutSerial = 2;  // vbdr_layout
constexpr int kKtabSize = 512;  // virtual indices covered by the smem table
constexpr int kLnTab = 513;     // ln(v) tabulated for v = 0..512 (entry 0 unused)

// SplitMix64 output mix (Steele, Lea & Flood 2014), used as the seeded hash
// H(x, N, A) of Sec. 4.1:  H(x,N,A) = (hi32(mix64(x ^ mix64(A))) * N) >> 32.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// A premixed seed K = mix64(A) split for evaluating hi32(mix64(x ^ K)) of a
// 32-bit x in 32-bit halves: the high half of x ^ K is K's, so the terms of
// the first xor-shift and first multiply that depend on it alone are
// precomputed (hi1 = Khi ^ (Khi >> 30), t1 = hi1 * C1lo).
struct KEnt {
  uint32_t lo, hi, hi1, t1;
};

constexpr uint64_t kMixC1 = 0xbf58476d1ce4e5b9ULL, kMixC2 = 0x94d049bb133111ebULL;

__host__ __device__ __forceinline__ KEnt make_kent(uint64_t K) {
  KEnt e;
  e.lo = (uint32_t)K;
  e.hi = (uint32_t)(K >> 32);
  e.hi1 = e.hi ^ (e.hi >> 30);
  e.t1 = e.hi1 * (uint32_t)kMixC1;
  return e;
}

// hi32(mix64(x ^ K)) -- the same value as mix64 above, in 32-bit pieces:
//   z ^= z >> 30 ; z *= C1 ; z ^= z >> 27 ; z *= C2 ; z ^= z >> 31
// of which only the high word of the last two steps is needed.
__device__ __forceinline__ uint32_t hash32(uint32_t x, const KEnt &k) {
  constexpr uint32_t C1lo = (uint32_t)kMixC1, C1hi = (uint32_t)(kMixC1 >> 32);
  constexpr uint32_t C2lo = (uint32_t)kMixC2, C2hi = (uint32_t)(kMixC2 >> 32);
  const uint32_t lo0 = x ^ k.lo;
  const uint32_t lo1 = lo0 ^ __funnelshift_r(lo0, k.hi, 30);
  const uint64_t p = (uint64_t)lo1 * C1lo;
  const uint32_t lo2 = (uint32_t)p;
  const uint32_t hi2 = (uint32_t)(p >> 32) + lo1 * C1hi + k.t1;
  const uint32_t lo3 = lo2 ^ __funnelshift_r(lo2, hi2, 27);
  const uint32_t hi3 = hi2 ^ (hi2 >> 27);
  const uint32_t hi4 = __umulhi(lo3, C2lo) + lo3 * C2hi + hi3 * C2lo;
  return hi4 ^ (hi4 >> 31);
}

// Multiply-shift range reduction of a 32-bit hash onto [0, Z); Z = 2^32 is
// passed as zmul = 0 and means "the hash itself".
__device__ __forceinline__ uint32_t reduce32(uint32_t h, uint32_t zmul) {
  return zmul ? __umulhi(h, zmul) : h;
}

struct Dims {
  uint64_t Z;        // physical BDRs
  uint64_t Zs;       // DRV plane stride in words: Z rounded up to 4 (16 B)
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
  KEnt K1;           // mix64(A1): premixed seed of the bip hash
};

// Per-handle FP64 constants of the estimator, indexed by b = log2 g (each
// computed on the host with the same IEEE operations, in the same order, as
// the plain formula): amm[b] = alpha_g * g * g, kz[b] = Z * g / (Z - g),
// lng[b] = ln g; amm_Z = alpha_Z * Z * Z for the pool.
// LogLog and PCSA (the BDR pool serves both, Sec. 4.1): ll[b] = alpha^LL_g g
// with alpha^LL_m = (Gamma(-1/m) (1 - 2^(1/m)) / ln 2)^(-m) (Durand &
// Flajolet 2003), pc[b] = g / 0.77351 (Flajolet & Martin 1985); ll_Z, pc_Z
// the same for the pool.
struct EstConst {
  double amm[kMaxLog2G + 1];
  double kz[kMaxLog2G + 1];
  double lng[kMaxLog2G + 1];
  double amm_Z;
  double ll[kMaxLog2G + 1];
  double pc[kMaxLog2G + 1];
  double ll_Z, pc_Z;
  double inv_g[kMaxLog2G + 1];  // 2^-b exactly
};

// 2^-32: S 2^-32 is the harmonic sum of 2^-M (a multiplication by a power of
// two is exact, the same value as ldexp without its range handling).
constexpr double kTwoM32 = 0x1p-32;

struct DevState {
  uint32_t *drv;     // [P][Zs]
  uint32_t *bs;      // [Z] (gfast only, else nullptr)
  uint8_t *now;      // [Zs] nowLBP1 (serial only, else nullptr)
  uint8_t *reg;      // [Z]
  uint8_t *pcsa;     // [Zs] gsmall only: PCSA statistic of the closed window
  KEnt *ktab;        // [max(g_max, kKtabSize)]
  double *lnv;       // [kLnTab] ln(v)
  unsigned long long *sums;  // [kSums]: pool sums of the last slide and the
                             // partials of their reduction (kSum* below)
  unsigned int *check;       // bounds-checked build: violations seen (kChk*)
};

// Bounds-checked build (-DVBDR_CHECK): kernels test their indices and
// register values, skip an access that would leave its buffer and record
// the violation in DevState::check.  In the normal build vbk_check is the
// constant true and the tests vanish.
#ifdef VBDR_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
enum : unsigned int { kChkPidx = 1u, kChkRho = 2u, kChkReg = 4u, kChkPlan = 8u };
__device__ __forceinline__ bool vbk_check(bool ok, unsigned int *flags, unsigned int bit) {
  if constexpr (kChecked) {
    if (!ok && flags) atomicOr(flags, bit);
    return ok;
  } else {
    return true;
  }
}

// Slots of DevState::sums.  Totals: S_Z = sum 2^(32 - reg), V_Z = #{reg = 0},
// L_Z = sum reg (LogLog), P_Z = sum pcsa (PCSA); each has a partial that the
// reducing launch accumulates and its last block moves into the total.
enum : int {
  kSumS = 0, kSumV = 1, kSumCounter = 2, kSumSPart = 3, kSumVPart = 4,
  kSumL = 5, kSumLPart = 6, kSumP = 7, kSumPPart = 8, kSums = 16
};

// host b of aip (group_rule 1: four groups by the top two address bits)
__device__ __forceinline__ uint32_t host_b(const Dims &d, uint32_t aip) {
  return d.group_rule ? d.b_min + (aip >> 30) : d.b;
}

// Pool noise term n_Z / Z of the estimator (Sec. 4.1) from the pool sums of
// the last slide: HLL of the Z registers, small-range linear counting.
__device__ __forceinline__ double pool_noise(const Dims &d, const DevState &s, const EstConst &c) {
  const double Z = (double)d.Z;
  const unsigned long long S_Z = s.sums[0], V_Z = s.sums[1];
  double E = c.amm_Z / ((double)S_Z * kTwoM32);
  if (E <= 2.5 * Z && V_Z > 0) E = Z * log(Z / (double)V_Z);
  return E / Z;
}

// Estimate of one host (log2 g = b) from the exact sums of its g virtual
// registers, S = sum_i 2^(32 - M_i) and V = #{M_i = 0}:
//   n_g = alpha_g g^2 / (S 2^-32), or g ln(g / V) when at most 2.5 g and
//   V > 0;  n = max(0, Z g / (Z - g) * (n_g / g - nZZ)).
// lnv: ln v for v < kLnTab.  Every kernel that estimates calls this, so
// their results agree bit for bit.
// The quotient alpha_g g^2 / x (x = S 2^-32) is the costly FP64 operation
// here (GB300's FP64 rate is low).  Where the sign of alpha_g g^2 - 2.5 g x,
// computed with one rounding by fma, is <= 0, the exact quotient is at most
// 2.5 g and so is its rounded value: linear counting is chosen without it.
// Otherwise the quotient is computed and compared as written, so the
// decision is always the one the rounded quotient makes.
__device__ __forceinline__ double host_estimate(unsigned long long S, uint32_t V, uint32_t b,
                                                const EstConst &c, const double *lnv, double nZZ,
                                                double *n_g_out) {
  const double g = (double)(1u << b), t = 2.5 * g, x = (double)S * kTwoM32;
  double n_g;
  bool lc = V > 0 && __fma_rn(-t, x, c.amm[b]) <= 0.0;
  if (!lc) {
    n_g = c.amm[b] / x;
    lc = n_g <= t && V > 0;
  }
  if (lc) n_g = g * (V < (uint32_t)kLnTab ? c.lng[b] - lnv[V] : log(g / (double)V));
  double est = c.kz[b] * (n_g * c.inv_g[b] - nZZ);
  if (!(est > 0.0)) est = 0.0;
  if (n_g_out) *n_g_out = n_g;
  return est;
}

// ----- launchers (defined in the kernel translation units) -----
cudaError_t launch_init(const Dims &d, const DevState &s, cudaStream_t st);
cudaError_t launch_scan(const Dims &d, const DevState &s, int layout,
                        const uint32_t *pairs, uint64_t n, cudaStream_t st,
                        const uint64_t *n_dev = nullptr);
cudaError_t launch_slide(const Dims &d, const DevState &s, int layout,
                         cudaStream_t st);
// Launch shape of the estimate kernel: lanes cooperating on one host and
// threads per block.  kEstCandidates is the autotuner's search space; the
// first entry is the default.
struct EstLaunch {
  int lanes;
  int threads;
};
constexpr int kNumEstCandidates = 9;
extern const EstLaunch kEstCandidates[kNumEstCandidates];

cudaError_t launch_estimate(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st, EstLaunch cfg);
cudaError_t launch_features(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, __nv_bfloat16 *feat, float *plain,
                            cudaStream_t st, EstLaunch cfg);
MlpDevWeights mlp_weights(const vbdr_mlp *m);
cudaError_t launch_mlp_correct(const vbdr_mlp *m, const __nv_bfloat16 *X, uint64_t n, float *est,
                               cudaStream_t st);
float mlp_nmax(const vbdr_mlp *m);
cudaError_t launch_load_virtual(const Dims &d, const DevState &s, const uint32_t *aips,
                                const uint64_t *offsets, uint64_t n, const uint8_t *vregs,
                                cudaStream_t st);
cudaError_t launch_pool_sums(const uint8_t *reg, const uint8_t *pcsa, uint64_t Z,
                             unsigned long long *sums, cudaStream_t st);
cudaError_t launch_estimate_alt(const Dims &d, const DevState &s, const EstConst &c,
                                const uint32_t *aips, uint64_t n, float *out, int which,
                                cudaStream_t st, EstLaunch cfg);

// ----- bucketed scan (bucket.cu) -----
// Pool tiles of 2^16 BDRs.  Each pass, route CTA c appends the records
// (pidx mod 2^16) << 3 | (LBP1 - 1) of tile t to its own region
// recs[(c ntiles + t) cap ...] and publishes the count in fill[c ntiles + t];
// one apply CTA per tile then ORs them into the tile's bytes (lb between
// passes: one byte per BDR, bit r = LBP1 r + 1 seen).
constexpr uint32_t kBucketTileLog2 = 16;
constexpr uint32_t kBucketTile = 1u << kBucketTileLog2;
constexpr uint32_t kMaxBucketTiles = 2048;  // Z <= 2^27
struct BucketDev {
  uint32_t *recs;       // [ncta][ntiles][cap]
  uint32_t *fill;       // [ncta][ntiles]
  uint8_t *lb;          // [ntiles * 2^16]
  uint32_t ntiles;
  uint32_t ncta;        // route grid
  uint32_t cap;         // records per CTA region of a tile
  uint64_t pass_pairs;  // pairs routed per pass (a multiple of the route batch)
};
bool bucket_scan_applies(const Dims &d, int layout);
void bucket_layout(uint64_t Z, int sms, BucketDev *bk);
uint64_t bucket_bytes(const BucketDev &bk);
cudaError_t launch_scan_bucketed(const Dims &d, const DevState &s, const BucketDev &bk, int layout,
                                 const uint32_t *pairs, uint64_t n, cudaStream_t st,
                                 const uint64_t *n_dev = nullptr);

// ----- several GPUs (shard.cu) -----
constexpr uint32_t kMaxRanks = 256;
cudaError_t launch_route_records(const Dims &d, const DevState &s, const uint32_t *pairs, uint64_t n,
                                 uint32_t ranks, uint32_t *recs, uint64_t cap,
                                 unsigned long long *fill, cudaStream_t st);
cudaError_t launch_apply_records(const Dims &d, const DevState &s, int layout, const uint32_t *recs,
                                 uint64_t n, cudaStream_t st);
cudaError_t launch_merge_slice_state(const Dims &d, const DevState &s, int layout,
                                     const uint32_t *other, uint64_t words, cudaStream_t st);

// ----- estimate plans (plan.cu) -----
// Register chunk of the planned estimate: 2^15 BDRs (32 KiB of reg); the
// register array is allocated in whole chunks.
constexpr int kPlanChunkLog2 = 15;
constexpr uint64_t kPlanChunk = 1ull << kPlanChunkLog2;
constexpr uint32_t kPlanMaxHB = 7000;       // hosts per block (shared accumulators)
constexpr uint32_t kLearnMaxHB = 3300;      // hosts per block of a learned-correction plan
constexpr uint32_t kPlanMaxChunks = 8192;   // Z <= 2^28
constexpr uint32_t kPlanPad = kPlanMaxHB << kPlanChunkLog2;  // padding: spare host slot
// Device view of a plan: hosts [blk HB, (blk + 1) HB) form block blk; the
// entries of group (blk, c) -- one per virtual register of the block's hosts
// that Alg. 3 maps into chunk c, (local host << 15) | (pidx mod 2^15) --
// occupy [goff[blk nchunks + c], goff[blk nchunks + c + 1]), padded with
// kPlanPad to a multiple of 4.
struct PlanDev {
  const uint32_t *aips;     // [n]
  uint32_t *entries;        // [goff[NB nchunks]]
  unsigned long long *goff; // [NB nchunks + 1]
  uint32_t *counts;         // [NB nchunks] (building)
  uint32_t *err;            // bounded-wait failures
  uint64_t n;
  uint32_t HB, NB, nchunks;
};
cudaError_t launch_plan_count(const Dims &d, const DevState &s, const PlanDev &p, cudaStream_t st);
cudaError_t launch_plan_fill(const Dims &d, const DevState &s, const PlanDev &p, cudaStream_t st);
cudaError_t launch_plan_sort(const PlanDev &p, bool by_host, cudaStream_t st);
// The compact learned correction's FP32 parameters (W1 [16][10], b1, W2
// [16][16], b2, w3, b3) and nmax.
constexpr int kCompactParams = 465;  // 16 x 10 + 16 + 16 x 16 + 16 + 16 + 1
struct CompactParams {
  float w[kCompactParams];
  float nmax;
};
// net: NULL for the plain estimate, else the compact learned correction
// (every g <= 512), with compact_rec a device buffer of p.n + 1 records (16
// bytes each) between the planned kernel and the correction kernel
cudaError_t launch_planned_estimate(const Dims &d, const DevState &s, const EstConst &c,
                                   const PlanDev &p, const CompactParams *net,
                                   uint4 *compact_rec, float *out, cudaStream_t st);
cudaError_t launch_planned_features(const Dims &d, const DevState &s, const EstConst &c,
                                    const PlanDev &p, float *out, __nv_bfloat16 *feat,
                                    cudaStream_t st);

}  // namespace vbk
