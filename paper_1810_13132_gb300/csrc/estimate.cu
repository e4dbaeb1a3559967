// estimate.cu -- per-host cardinality estimation (Sec. 4.1 Alg. 5 with
// Alg. 3, and the estimator of the virtual register sharing HyperLogLog that
// Sec. 4.1 cites; Sec. 4.2: registers are read-only here, so any number of
// hosts are estimated in parallel).
//
// Work split: a warp owns a batch of 32 hosts.
//   gather : for each host of the batch in turn, the 32 lanes visit its g
//            virtual indices (i = lane + 32u), map each to its physical BDR
//            pidx = H(aip, Z, s1(i)) and gather the byte register reg[pidx]
//            (8 gathers in flight per lane); the warp sums
//            S = sum_i 2^(32 - M_i) exactly in 64-bit integers and counts
//            V = #{M_i = 0}; lane q keeps host q's (S, V).
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

constexpr int kEstThreads = 256;
constexpr int kGatherUnroll = 8;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kEstThreads)
    estimate_kernel(const uint32_t *__restrict__ aips, uint64_t n,
                    float *__restrict__ out, Dims d, DevState s, EstConst c) {
  __shared__ KEnt kt_s[kKtabSize];
  __shared__ double lnv_s[kLnTab];
  __shared__ double nZZ_s;
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  const bool kt_in_smem = gmax <= (uint32_t)kKtabSize;
  if (kt_in_smem)
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
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
  const KEnt *kt = kt_in_smem ? kt_s : s.ktab;
  const double nZZ = nZZ_s;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  for (uint64_t hb = warp * 32; hb < n; hb += warps * 32) {
    const uint64_t h_l = hb + lane;
    const uint32_t aip_l = h_l < n ? __ldg(aips + h_l) : 0u;
    const uint32_t nb = (n - hb) < 32 ? (uint32_t)(n - hb) : 32u;
    unsigned long long myS = 0;
    uint32_t myV = 0;
    for (uint32_t q = 0; q < nb; ++q) {
      const uint32_t aip = __shfl_sync(0xffffffffu, aip_l, q);
      const uint32_t g = 1u << host_b(d, aip);
      unsigned long long S = 0;
      uint32_t V = 0;
      for (uint32_t base = 0; base < g; base += 32 * kGatherUnroll) {
        uint32_t M[kGatherUnroll];
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) {
          const uint32_t i = base + 32u * u + lane;
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
          }
        }
      }
      S = warp_sum_u64(S);
      V = __reduce_add_sync(0xffffffffu, V);
      if (lane == q) {
        myS = S;
        myV = V;
      }
    }
    if (h_l < n) {
      const uint32_t b = host_b(d, aip_l);
      const double g = (double)(1u << b);
      double n_g = c.amm[b] / ldexp((double)myS, -32);
      if (n_g <= 2.5 * g && myV > 0)
        n_g = g * (myV < (uint32_t)kLnTab ? c.lng[b] - lnv_s[myV] : log(g / (double)myV));
      double est = c.kz[b] * (ldexp(n_g, -(int)b) - nZZ);
      if (!(est > 0.0)) est = 0.0;
      out[h_l] = (float)est;
    }
  }
}

}  // namespace

cudaError_t launch_estimate(const Dims &d, const DevState &s, const EstConst &c,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, estimate_kernel, kEstThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t hosts_per_block = (kEstThreads / 32) * 32;
  const uint64_t want = (n + hosts_per_block - 1) / hosts_per_block;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want;
  estimate_kernel<<<(unsigned)grid, kEstThreads, 0, st>>>(aips, n, out, d, s, c);
  return cudaGetLastError();
}

}  // namespace vbk
