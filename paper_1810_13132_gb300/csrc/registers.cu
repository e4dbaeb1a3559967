// registers.cu -- register-level state loading and pool sums.
//
// launch_load_virtual: the register array becomes, for every physical BDR,
// the largest value among the virtual registers that Alg. 3 maps onto it
// (host aip's virtual index i -> BDR H(aip, Z, s1(i))); BDRs that no virtual
// register maps to hold 0.  This is how a workload too large to scan (4M
// hosts with cardinalities up to 1e7) is put under the estimator.
// launch_pool_sums: S_Z = sum_j 2^(32 - reg_j), V_Z = #{reg_j = 0}, L_Z =
// sum_j reg_j and P_Z = sum_j pcsa_j (0 without a PCSA array).
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr int kThreads = 256;

// max into one byte of the register array through a CAS on its 32-bit word.
// Each failed CAS means another thread raised that word, which happens at
// most 4 * 255 times, so the loop ends; the cap is a second guard.
__device__ __forceinline__ void byte_max(uint8_t *reg, uint32_t j, uint32_t v) {
  uint32_t *word = reinterpret_cast<uint32_t *>(reg + (j & ~3u));
  const uint32_t sh = (j & 3u) * 8u;
  uint32_t old = *reinterpret_cast<volatile uint32_t *>(word);
  for (int it = 0; it < 4096 && ((old >> sh) & 0xffu) < v; ++it) {
    const uint32_t want = (old & ~(0xffu << sh)) | (v << sh);
    const uint32_t seen = atomicCAS(word, old, want);
    if (seen == old) break;
    old = seen;
  }
}

// One warp per host; lanes over the host's virtual indices.
__global__ void __launch_bounds__(kThreads)
    load_virtual_kernel(const uint32_t *__restrict__ aips, const uint64_t *__restrict__ offsets,
                        uint64_t n, const uint8_t *__restrict__ vregs, Dims d, DevState s) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t h = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); h < n;
       h += warps) {
    const uint32_t aip = aips[h];
    const uint32_t g = 1u << host_b(d, aip);
    const uint8_t *v = vregs + offsets[h];
    for (uint32_t i = lane; i < g; i += 32) {
      const uint32_t val = v[i];
      const uint32_t pidx = reduce32(hash32(aip, s.ktab[i]), d.zmul);
      if (val && vbk_check(pidx < d.Z, s.check, kChkPidx) && vbk_check(val <= d.R, s.check, kChkReg))
        byte_max(s.reg, pidx, val);
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    pool_sums_kernel(const uint8_t *__restrict__ reg, const uint8_t *__restrict__ pcsa, uint64_t Z,
                     unsigned long long *sums) {
  unsigned long long S = 0, V = 0, L = 0, Pc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < Z; j += stride) {
    const uint32_t M = reg[j];
    S += 1ull << (32u - M);
    V += (M == 0u);
    L += M;
    if (pcsa) Pc += pcsa[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_down_sync(0xffffffffu, S, o);
    V += __shfl_down_sync(0xffffffffu, V, o);
    L += __shfl_down_sync(0xffffffffu, L, o);
    Pc += __shfl_down_sync(0xffffffffu, Pc, o);
  }
  __shared__ unsigned long long sS[kThreads / 32], sV[kThreads / 32], sL[kThreads / 32],
      sP[kThreads / 32];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { sS[warp] = S; sV[warp] = V; sL[warp] = L; sP[warp] = Pc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t i = 1; i < blockDim.x / 32; ++i) {
      S += sS[i];
      V += sV[i];
      L += sL[i];
      Pc += sP[i];
    }
    atomicAdd(&sums[kSumSPart], S);
    atomicAdd(&sums[kSumVPart], V);
    atomicAdd(&sums[kSumLPart], L);
    atomicAdd(&sums[kSumPPart], Pc);
    __threadfence();
    if (atomicAdd(&sums[kSumCounter], 1ull) == gridDim.x - 1) {
      __threadfence();
      sums[kSumS] = atomicExch(&sums[kSumSPart], 0ull);
      sums[kSumV] = atomicExch(&sums[kSumVPart], 0ull);
      sums[kSumL] = atomicExch(&sums[kSumLPart], 0ull);
      sums[kSumP] = atomicExch(&sums[kSumPPart], 0ull);
      sums[kSumCounter] = 0ull;
    }
  }
}

int grid_for(uint64_t units, int per_sm_cap) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t grid = (units + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)sms * per_sm_cap;
  if (grid > cap) grid = cap;
  return grid ? (int)grid : 1;
}

}  // namespace

cudaError_t launch_load_virtual(const Dims &d, const DevState &s, const uint32_t *aips,
                                const uint64_t *offsets, uint64_t n, const uint8_t *vregs,
                                cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s.reg, 0, d.Z, st);
  if (e != cudaSuccess || n == 0) return e;
  load_virtual_kernel<<<grid_for(n * 32, 8), kThreads, 0, st>>>(aips, offsets, n, vregs, d, s);
  return cudaGetLastError();
}

cudaError_t launch_pool_sums(const uint8_t *reg, const uint8_t *pcsa, uint64_t Z,
                             unsigned long long *sums, cudaStream_t st) {
  pool_sums_kernel<<<grid_for(Z, 8), kThreads, 0, st>>>(reg, pcsa, Z, sums);
  return cudaGetLastError();
}

}  // namespace vbk
