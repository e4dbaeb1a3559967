// estimate.cu -- per-host cardinality estimation (Sec. 4.1 Alg. 5 with
// Alg. 3, and the estimator of the virtual register sharing HyperLogLog that
// Sec. 4.1 cites; Sec. 4.2: registers are read-only here, so any number of
// hosts are estimated in parallel).
//
// Work split: one persistent wave of blocks; a warp owns a batch of 32 hosts.
//   gather : groups of T lanes (T = 8, 16 or 32, chosen per workload by the
//            autotuner of api.cu) take the batch's hosts in turn; the T lanes
//            of a group visit the host's g virtual indices (i = sub + T u),
//            map each to its physical BDR pidx = H(aip, Z, s1(i)) and gather
//            the byte register reg[pidx] (8 gathers in flight per lane); the
//            group sums S = sum_i 2^(32 - M_i) exactly in 64-bit integers and
//            counts V = #{M_i = 0}.  Hosts of mixed g (64..512) share a
//            launch; small T keeps lanes busy on small g.
//   finish : every lane evaluates its own host's estimate in FP64, so the
//            (slow) FP64 pipe runs with all 32 lanes busy:
//              n_g = HLL(g, S, V), n_Z = HLL(Z, S_Z, V_Z) (once per block),
//              n   = max(0, Z g / (Z - g) * (n_g / g - n_Z / Z)),
//            HLL(m, S, V) = alpha_m m^2 / (S 2^-32), replaced by m ln(m / V)
//            when at most 2.5 m and V > 0 (small-range linear counting).
//            The constants alpha_g g^2, Z g / (Z - g) and ln v (v <= 512)
//            are tabulated once per handle in FP64; the raw estimate and the
//            linear-counting decision are computed with the same IEEE
//            operations as the plain formula, so the decision is exact.
//            The result is rounded to FP32.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kMaxEstWarps = 16;  // blocks of up to 512 threads
constexpr int kGatherUnroll = 8;
// What the kernel produces per host: the estimate, or also the learned
// correction's feature row.
// kLogLog / kPcsa: the same walk over the host's virtual BDRs summing the
// register (Alg. 5's getSumLBP1, the LogLog statistic) or the PCSA statistic
// of each BDR, finished with that estimator and the same noise removal.
enum EstMode { kPlain = 0, kFeatures = 1, kLogLog = 2, kPcsa = 3 };

// A warp owns a batch of 32 hosts and splits its lanes into 32/T groups of
// T lanes; in T steps each group gathers one host of the batch.  The host
// results land in shared memory so that lane q finishes host q.
// kFeatures also counts each host's register values: every lane keeps a
// private 32-bin byte histogram (a shared-memory row of 36 bytes, so the 32
// lanes' rows fall in distinct banks; one shared atomic add per value), the
// group then adds its rows with packed 16-bit SIMD sums (each lane reads 8
// words), writes bin / g of the feature row, and derives S and V from the
// bins instead of accumulating them per value.  The finishing lane writes the
// noise statistics of the row.
template <bool SMEM_KT, int T, int MODE>  // seed table in shared memory (g_max <= 512)
__global__ void __launch_bounds__(kMaxEstWarps * 32)
    estimate_kernel(const uint32_t *__restrict__ aips, uint64_t n,
                    float *__restrict__ out, Dims d, DevState s, EstConst c,
                    __nv_bfloat16 *__restrict__ feat_out) {
  static_assert(T == 8 || T == 16 || T == 32, "lanes per host");
  constexpr uint32_t G = 32 / T;  // hosts gathered at once per warp
  constexpr int WARPS = kMaxEstWarps;
  constexpr bool HIST = MODE == kFeatures;
  constexpr bool SUM = MODE == kLogLog || MODE == kPcsa;  // plain sum of the values
  const uint8_t *vals = MODE == kPcsa ? s.pcsa : s.reg;
  __shared__ KEnt kt_s[SMEM_KT ? kKtabSize : 1];
  __shared__ double lnv_s[kLnTab];
  __shared__ double nZZ_s;
  __shared__ unsigned long long resS[WARPS][32];
  __shared__ uint32_t resV[WARPS][32];
  __shared__ uint32_t hrow[HIST ? WARPS : 1][32][9];  // private histograms
  if constexpr (SMEM_KT) {
    const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
  }
  for (uint32_t i = threadIdx.x; i < (uint32_t)kLnTab; i += blockDim.x) lnv_s[i] = s.lnv[i];
  if (threadIdx.x == 0) {
    // pool estimate per register, n_Z / Z
    if constexpr (MODE == kLogLog)
      nZZ_s = c.ll_Z * exp2((double)s.sums[kSumL] / (double)d.Z) / (double)d.Z;
    else if constexpr (MODE == kPcsa)
      nZZ_s = c.pc_Z * exp2((double)s.sums[kSumP] / (double)d.Z) / (double)d.Z;
    else
      nZZ_s = pool_noise(d, s, c);
  }
  __syncthreads();
  const KEnt *kt = SMEM_KT ? kt_s : s.ktab;
  const double nZZ = nZZ_s;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wib = threadIdx.x >> 5;
  const uint32_t grp = lane / T, sub = lane % T;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;

  for (uint64_t hb = warp * 32; hb < n; hb += warps * 32) {
    const uint64_t h_l = hb + lane;
    const uint32_t aip_l = h_l < n ? __ldg(aips + h_l) : 0u;
    const uint32_t nb = (n - hb) < 32 ? (uint32_t)(n - hb) : 32u;
#pragma unroll 1
    for (uint32_t t = 0; t < T; ++t) {
      const uint32_t j = grp + G * t;  // batch slot this group gathers now
      const uint32_t aip = __shfl_sync(0xffffffffu, aip_l, j & 31u);
      const bool valid = j < nb;
      const uint32_t g = valid ? 1u << host_b(d, aip) : 0u;
      unsigned long long S = 0;
      uint32_t V = 0;
      if constexpr (HIST) {
#pragma unroll
        for (int q = 0; q < 8; ++q) hrow[wib][lane][q] = 0u;
      }
      for (uint32_t base = 0; base < g; base += T * kGatherUnroll) {
        uint32_t M[kGatherUnroll];
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) {
          const uint32_t i = base + T * u + sub;
          M[u] = 0xffu;
          if (i < g) {
            const uint32_t pidx = reduce32(hash32(aip, kt[i]), d.zmul);
            if (vbk_check(pidx < d.Z, s.check, kChkPidx)) {
              M[u] = __ldg(vals + pidx);
              // the checked build skips and records a value above 32; the
              // plain estimate of the normal build reads it as 32 (registers
              // a caller supplies; the handle's own never exceed 32)
              if (!vbk_check(M[u] <= 32u, s.check, kChkReg)) M[u] = 0xffu;
              else if constexpr (MODE == kPlain) M[u] = min(M[u], 32u);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) {
          if (M[u] != 0xffu) {
            if constexpr (HIST) {
              atomicAdd(&hrow[wib][lane][M[u] >> 2], 1u << (8u * (M[u] & 3u)));
            } else if constexpr (SUM) {
              S += M[u];
            } else {
              S += 1ull << (32u - M[u]);
              V += (M[u] == 0u);
            }
          }
        }
      }
      if constexpr (HIST) {
        // bins 4w..4w+3 (w = sub % 8) summed over the group's rows: 16-bit
        // fields, bins 4w and 4w+2 in lo, 4w+1 and 4w+3 in hi
        __syncwarp();
        const uint32_t word = sub & 7u;
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (uint32_t r = sub >> 3; r < (uint32_t)T; r += T / 8) {
          const uint32_t v = hrow[wib][grp * T + r][word];
          lo += v & 0x00ff00ffu;
          hi += (v >> 8) & 0x00ff00ffu;
        }
#pragma unroll
        for (int o = 8; o < T; o <<= 1) {
          lo += __shfl_xor_sync(0xffffffffu, lo, o, T);
          hi += __shfl_xor_sync(0xffffffffu, hi, o, T);
        }
        const uint32_t c0 = lo & 0xffffu, c1 = hi & 0xffffu, c2 = lo >> 16, c3 = hi >> 16;
        const uint32_t b0 = 4u * word;
        if (valid && sub < 8) {
          const float inv_g = 1.0f / (float)g;
          __align__(8) __nv_bfloat16 f[4] = {
              __float2bfloat16((float)c0 * inv_g), __float2bfloat16((float)c1 * inv_g),
              __float2bfloat16((float)c2 * inv_g), __float2bfloat16((float)c3 * inv_g)};
          *reinterpret_cast<uint2 *>(feat_out + (hb + j) * kMlpLive + b0) =
              *reinterpret_cast<const uint2 *>(f);
        }
        // S and V from the bins: bin b contributes count * 2^(32 - b); the
        // 8 lanes sub % 8 = 0..7 of any row subset cover all 32 bins once
        S = ((unsigned long long)c0 << (32u - b0)) + ((unsigned long long)c1 << (31u - b0)) +
            ((unsigned long long)c2 << (30u - b0)) + ((unsigned long long)c3 << (29u - b0));
        S = b0 + 3u <= 32u ? S : 0ull;
        V = word == 0 ? c0 : 0u;
        __syncwarp();
      }
      // HIST: every row subset already holds the bin totals -> sum 8 lanes
#pragma unroll
      for (int o = (HIST ? 4 : T / 2); o > 0; o >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, o, T);
        V += __shfl_xor_sync(0xffffffffu, V, o, T);
      }
      if (sub == 0 && valid) {
        resS[wib][j] = S;
        resV[wib][j] = V;
      }
    }
    __syncwarp();
    if (h_l < n) {
      const unsigned long long myS = resS[wib][lane];
      const uint32_t myV = resV[wib][lane];
      const uint32_t b = host_b(d, aip_l);
      double n_g = 0.0, est;
      if constexpr (SUM) {
        // n_g = const_g 2^(sum / g); n = Z g / (Z - g) (n_g / g - n_Z / Z)
        const double base = MODE == kLogLog ? c.ll[b] : c.pc[b];
        n_g = base * exp2((double)myS * c.inv_g[b]);
        est = c.kz[b] * (n_g * c.inv_g[b] - nZZ);
        if (!(est > 0.0)) est = 0.0;
      } else {
        est = host_estimate(myS, myV, b, c, lnv_s, nZZ, &n_g);
      }
      if constexpr (MODE != kFeatures) {
        out[h_l] = (float)est;
      } else {
        __align__(16) __nv_bfloat16 x[16];
        x[0] = __float2bfloat16((float)b * 0.0625f);
        x[1] = __float2bfloat16(log1pf((float)est) * 0.0625f);
        x[2] = __float2bfloat16(log1pf((float)n_g) * 0.0625f);
        x[3] = __float2bfloat16(log1pf((float)nZZ));
        x[4] = __float2bfloat16((float)((double)s.sums[1] / (double)d.Z));
        x[5] = __float2bfloat16((float)myV / (float)(1u << b));
#pragma unroll
        for (int q = 6; q < 16; ++q) x[q] = __float2bfloat16(0.f);
        uint4 *dst = reinterpret_cast<uint4 *>(feat_out + h_l * kMlpLive + 32);
        dst[0] = *reinterpret_cast<const uint4 *>(&x[0]);
        dst[1] = *reinterpret_cast<const uint4 *>(&x[8]);
        out[h_l] = (float)est;
      }
    }
    __syncwarp();
  }
}

template <bool SMEM_KT, int MODE>
void *estimate_kernel_ptr(int T) {
  switch (T) {
    case 8: return (void *)estimate_kernel<SMEM_KT, 8, MODE>;
    case 16: return (void *)estimate_kernel<SMEM_KT, 16, MODE>;
    default: return (void *)estimate_kernel<SMEM_KT, 32, MODE>;
  }
}

template <int MODE>
cudaError_t launch_mode(const Dims &d, const DevState &s, const EstConst &c, const uint32_t *aips,
                        uint64_t n, float *out, cudaStream_t st, EstLaunch cfg,
                        __nv_bfloat16 *feat) {
  if (n == 0) return cudaSuccess;
  const int threads = cfg.threads;
  if (threads < 32 || threads > kMaxEstWarps * 32 || threads % 32) return cudaErrorInvalidValue;
  const bool smem_kt = (1u << (d.group_rule ? d.b_min + 3 : d.b)) <= (uint32_t)kKtabSize;
  void *kern = smem_kt ? estimate_kernel_ptr<true, MODE>(cfg.lanes)
                       : estimate_kernel_ptr<false, MODE>(cfg.lanes);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t hosts_per_block = (uint64_t)(threads / 32) * 32;
  const uint64_t want = (n + hosts_per_block - 1) / hosts_per_block;
  uint64_t grid = (uint64_t)sms * per_sm;  // persistent: one wave, grid-stride
  if (want < grid) grid = want;
  void *args[] = {(void *)&aips, (void *)&n, (void *)&out, (void *)&d,
                  (void *)&s,    (void *)&c, (void *)&feat};
  return cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(threads), args, 0, st);
}

}  // namespace

const EstLaunch kEstCandidates[kNumEstCandidates] = {
    {32, 256}, {16, 256}, {8, 256}, {32, 128}, {16, 128},
    {8, 128},  {32, 512}, {16, 512}, {8, 512}};

cudaError_t launch_estimate(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st, EstLaunch cfg) {
  return launch_mode<kPlain>(d, s, c, aips, n, out, st, cfg, nullptr);
}

cudaError_t launch_estimate_alt(const Dims &d, const DevState &s, const EstConst &c,
                                const uint32_t *aips, uint64_t n, float *out, int which,
                                cudaStream_t st, EstLaunch cfg) {
  if (which == 1) return launch_mode<kLogLog>(d, s, c, aips, n, out, st, cfg, nullptr);
  if (which == 2) return launch_mode<kPcsa>(d, s, c, aips, n, out, st, cfg, nullptr);
  return cudaErrorInvalidValue;
}

cudaError_t launch_features(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, __nv_bfloat16 *feat, float *plain,
                            cudaStream_t st, EstLaunch cfg) {
  return launch_mode<kFeatures>(d, s, c, aips, n, plain, st, cfg, feat);
}

}  // namespace vbk
