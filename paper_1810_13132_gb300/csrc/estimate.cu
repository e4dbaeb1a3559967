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
#include "mlp_device.cuh"
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kMaxEstWarps = 16;  // blocks of up to 512 threads
constexpr int kGatherUnroll = 8;
constexpr int kLearnedWarps = 4;  // block shape of the feature / learned modes

// What the kernel produces per host.
enum EstMode { kPlain = 0, kFeatures = 1, kLearned = 2 };

// A warp owns a batch of 32 hosts and splits its lanes into 32/T groups of
// T lanes; in T steps each group gathers one host of the batch.  The host
// results land in shared memory so that lane q finishes host q.
// kFeatures / kLearned also count each host's register values: every lane
// keeps a private 32-bin byte histogram (a shared-memory row of 36 bytes, so
// the 32 lanes' rows fall in distinct banks), the group adds its rows per bin
// and writes bin / g into the batch's BF16 feature tile; the finishing lane
// adds the noise statistics.  kLearned then runs the MLP on the tile
// (mma.sync, 32 hosts per warp) and corrects the estimate.
template <bool SMEM_KT, int T, int MODE>  // seed table in shared memory (g_max <= 512)
__global__ void __launch_bounds__(MODE == kPlain ? kMaxEstWarps * 32 : kLearnedWarps * 32)
    estimate_kernel(const uint32_t *__restrict__ aips, uint64_t n,
                    float *__restrict__ out, Dims d, DevState s, EstConst c,
                    MlpDevWeights mw, float nmax, __nv_bfloat16 *__restrict__ feat_out) {
  static_assert(T == 8 || T == 16 || T == 32, "lanes per host");
  constexpr uint32_t G = 32 / T;  // hosts gathered at once per warp
  constexpr int WARPS = MODE == kPlain ? kMaxEstWarps : kLearnedWarps;
  constexpr bool HIST = MODE != kPlain;
  __shared__ KEnt kt_s[SMEM_KT ? kKtabSize : 1];
  __shared__ double lnv_s[kLnTab];
  __shared__ double nZZ_s;
  __shared__ unsigned long long resS[WARPS][32];
  __shared__ uint32_t resV[WARPS][32];
  __shared__ uint32_t hrow[HIST ? WARPS : 1][32][9];                    // private histograms
  __shared__ __align__(16) __nv_bfloat16 ftile[HIST ? WARPS : 1][32][kMlpLive];
  __shared__ __align__(16) __nv_bfloat16 h1tile[MODE == kLearned ? WARPS : 1][32][kMlpHid];
  if constexpr (SMEM_KT) {
    const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
  }
  for (uint32_t i = threadIdx.x; i < (uint32_t)kLnTab; i += blockDim.x) lnv_s[i] = s.lnv[i];
  if (threadIdx.x == 0) {
    // pool noise term n_Z / Z from the sums of the last slide
    const double Z = (double)d.Z;
    const unsigned long long S_Z = s.sums[0], V_Z = s.sums[1];
    double E = c.amm_Z / ldexp((double)S_Z, -32);
    if (E <= 2.5 * Z && V_Z > 0) E = Z * log(Z / (double)V_Z);
    nZZ_s = E / Z;
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
        for (int q = 0; q < 9; ++q) hrow[wib][lane][q] = 0u;
      }
      for (uint32_t base = 0; base < g; base += T * kGatherUnroll) {
        uint32_t M[kGatherUnroll];
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) {
          const uint32_t i = base + T * u + sub;
          M[u] = 0xffu;
          if (i < g) {
            const uint32_t pidx = reduce32(hash32(aip, kt[i]), d.zmul);
            M[u] = __ldg(s.reg + pidx);
          }
        }
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) {
          if (M[u] != 0xffu) {
            S += 1ull << (32u - M[u]);
            V += (M[u] == 0u);
            if constexpr (HIST) atomicAdd(&hrow[wib][lane][M[u] >> 2], 1u << (8u * (M[u] & 3u)));
          }
        }
      }
      if constexpr (HIST) {
        __syncwarp();
        if (valid) {
          const float inv_g = 1.0f / (float)g;
#pragma unroll
          for (uint32_t bb = 0; bb < 32 / T; ++bb) {
            const uint32_t bin = sub + T * bb;
            uint32_t cnt = 0;
            for (uint32_t r = 0; r < T; ++r)
              cnt += (hrow[wib][grp * T + r][bin >> 2] >> (8u * (bin & 3u))) & 0xffu;
            ftile[wib][j][bin] = __float2bfloat16((float)cnt * inv_g);
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) {
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
      const double g = (double)(1u << b);
      double n_g = c.amm[b] / ldexp((double)myS, -32);
      if (n_g <= 2.5 * g && myV > 0)
        n_g = g * (myV < (uint32_t)kLnTab ? c.lng[b] - lnv_s[myV] : log(g / (double)myV));
      double est = c.kz[b] * (ldexp(n_g, -(int)b) - nZZ);
      if (!(est > 0.0)) est = 0.0;
      if constexpr (MODE == kPlain) {
        out[h_l] = (float)est;
      } else {
        __nv_bfloat16 *x = &ftile[wib][lane][32];
        x[0] = __float2bfloat16((float)b * 0.0625f);
        x[1] = __float2bfloat16(log1pf((float)est) * 0.0625f);
        x[2] = __float2bfloat16(log1pf((float)n_g) * 0.0625f);
        x[3] = __float2bfloat16(log1pf((float)nZZ));
        x[4] = __float2bfloat16((float)((double)s.sums[1] / (double)d.Z));
        x[5] = __float2bfloat16((float)myV / (float)(1u << b));
#pragma unroll
        for (int q = 6; q < 16; ++q) x[q] = __float2bfloat16(0.f);
        resS[wib][lane] = __double_as_longlong(est);
      }
    }
    if constexpr (MODE == kFeatures) {
      __syncwarp();
      for (uint32_t i = lane; i < 32 * kMlpLive; i += 32) {
        const uint64_t r = hb + i / kMlpLive;
        if (r < n) feat_out[r * kMlpLive + i % kMlpLive] = ftile[wib][i / kMlpLive][i % kMlpLive];
      }
      if (h_l < n) out[h_l] = (float)__longlong_as_double(resS[wib][lane]);
    } else if constexpr (MODE == kLearned) {
      __syncwarp();
      if (h_l >= n) {  // rows past the end: defined inputs for the tensor cores
        for (int q = 0; q < kMlpLive; ++q) ftile[wib][lane][q] = __float2bfloat16(0.f);
      }
      __syncwarp();
      const float delta = mlp_forward_warp(&ftile[wib][0][0], &h1tile[wib][0][0], mw);
      if (h_l < n) {
        const float plain = (float)__longlong_as_double(resS[wib][lane]);
        float corr = expm1f(log1pf(plain) + delta);
        if (!(corr > 0.f)) corr = 0.f;
        out[h_l] = plain > nmax ? plain : corr;
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
                        uint64_t n, float *out, cudaStream_t st, EstLaunch cfg, MlpDevWeights mw,
                        float nmax, __nv_bfloat16 *feat) {
  if (n == 0) return cudaSuccess;
  const int threads = MODE == kPlain ? cfg.threads : kLearnedWarps * 32;
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
  void *args[] = {(void *)&aips, (void *)&n, (void *)&out, (void *)&d, (void *)&s,
                  (void *)&c,    (void *)&mw, (void *)&nmax, (void *)&feat};
  return cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(threads), args, 0, st);
}

}  // namespace

const EstLaunch kEstCandidates[kNumEstCandidates] = {
    {32, 256}, {16, 256}, {8, 256}, {32, 128}, {16, 128},
    {8, 128},  {32, 512}, {16, 512}, {8, 512}};

cudaError_t launch_estimate(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st, EstLaunch cfg) {
  return launch_mode<kPlain>(d, s, c, aips, n, out, st, cfg, MlpDevWeights{}, 0.f, nullptr);
}

cudaError_t launch_features(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, __nv_bfloat16 *feat, float *plain,
                            cudaStream_t st, EstLaunch cfg) {
  return launch_mode<kFeatures>(d, s, c, aips, n, plain, st, cfg, MlpDevWeights{}, 0.f, feat);
}

cudaError_t launch_estimate_learned(const Dims &d, const DevState &s, const EstConst &c,
                                    const uint32_t *aips, uint64_t n, float *out, cudaStream_t st,
                                    EstLaunch cfg, MlpDevWeights mw, float nmax) {
  return launch_mode<kLearned>(d, s, c, aips, n, out, st, cfg, mw, nmax, nullptr);
}

}  // namespace vbk
