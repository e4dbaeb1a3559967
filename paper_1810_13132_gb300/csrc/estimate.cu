// estimate.cu -- per-host cardinality estimation (Sec. 4.1 Alg. 5 with
// Alg. 3, and the estimator of the virtual register sharing HyperLogLog that
// Sec. 4.1 cites; Sec. 4.2: registers are read-only here, so any number of
// hosts are estimated in parallel).
//
// A group of T lanes (T = 32 by default) owns one host: lane l visits the
// virtual indices i = l, l+T, ... < g, maps each to its physical BDR
// pidx = H(aip, Z, s1(i)) and gathers the byte register reg[pidx] (the
// 1-byte-per-BDR register array is L2-resident).  Per host the lanes sum
// S = sum_i 2^(32 - M_i) exactly in 64-bit integers and count V = #{M_i = 0},
// then the group leader evaluates, in FP64,
//   n_g = HLL(g, S, V), n_Z = HLL(Z, S_Z, V_Z),
//   n   = max(0, Z g / (Z - g) * (n_g / g - n_Z / Z)),
// HLL(m, S, V) = alpha_m m^2 / (S 2^-32), replaced by m ln(m / V) when it is
// at most 2.5 m and V > 0 (small-range linear counting), and writes n as
// FP32.
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kEstThreads = 256;

__device__ __forceinline__ double hll_alpha(double m) {
  if (m == 16.0) return 0.673;
  if (m == 32.0) return 0.697;
  if (m == 64.0) return 0.709;
  return 0.7213 / (1.0 + 1.079 / m);
}

__device__ __forceinline__ double hll(double m, unsigned long long S,
                                      unsigned long long V) {
  const double harmonic = ldexp((double)S, -32);
  double E = hll_alpha(m) * m * m / harmonic;
  if (E <= 2.5 * m && V > 0) E = m * log(m / (double)V);
  return E;
}

template <int T>  // lanes per host: 8, 16 or 32
__global__ void __launch_bounds__(kEstThreads)
    estimate_kernel(const uint32_t *__restrict__ aips, uint64_t n,
                    float *__restrict__ out, Dims d, DevState s) {
  __shared__ uint64_t kt_s[kKtabSize];
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  const bool kt_in_smem = gmax <= (uint32_t)kKtabSize;
  if (kt_in_smem)
    for (uint32_t i = threadIdx.x; i < gmax; i += blockDim.x) kt_s[i] = s.ktab[i];
  __syncthreads();
  const uint64_t *kt = kt_in_smem ? kt_s : s.ktab;

  const double Z = (double)d.Z;
  const unsigned long long S_Z = s.sums[0], V_Z = s.sums[1];
  const uint32_t sub = threadIdx.x % T;
  const uint64_t groups = (uint64_t)gridDim.x * (blockDim.x / T);
  const uint64_t g0 = (uint64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T;
  // group-uniform trip count so that the shuffles see every lane
  for (uint64_t hb = g0 - (g0 % (32 / T)); hb < n; hb += groups) {
    const uint64_t h = hb + (g0 % (32 / T));
    const bool valid = h < n;
    const uint32_t aip = valid ? __ldg(aips + h) : 0u;
    const uint32_t b = host_b(d, aip);
    const uint32_t g = 1u << b;
    unsigned long long S = 0, V = 0;
    if (valid) {
      for (uint32_t i = sub; i < g; i += T) {
        const uint32_t pidx = reduce32(hash32(aip, kt[i]), d.zmul);
        const uint32_t M = __ldg(s.reg + pidx);
        S += 1ull << (32u - M);
        V += (M == 0u);
      }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
      S += __shfl_down_sync(0xffffffffu, S, o, T);
      V += __shfl_down_sync(0xffffffffu, V, o, T);
    }
    if (valid && sub == 0) {
      const double gd = (double)g;
      const double n_g = hll(gd, S, V);
      const double n_Z = hll(Z, S_Z, V_Z);
      double est = (Z * gd / (Z - gd)) * (n_g / gd - n_Z / Z);
      if (!(est > 0.0)) est = 0.0;
      out[h] = (float)est;
    }
  }
}

}  // namespace

cudaError_t launch_estimate(const Dims &d, const DevState &s,
                            const uint32_t *aips, uint64_t n, float *out,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, estimate_kernel<32>, kEstThreads, 0);
  if (per_sm < 1) per_sm = 1;
  constexpr int T = 32;
  const uint64_t per_block = kEstThreads / T;
  const uint64_t want = (n + per_block - 1) / per_block;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (want < grid) grid = want;
  estimate_kernel<T><<<(unsigned)grid, kEstThreads, 0, st>>>(aips, n, out, d, s);
  return cudaGetLastError();
}

}  // namespace vbk
