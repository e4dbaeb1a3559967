// noalloc.cu -- vbdr_estimate_registers_noalloc: host estimates from a
// register array the caller already holds, without allocating anything.
//
// Its working memory is one file-scope __device__ array (kScratchBytes,
// below) that every GPU which loads this library keeps until the process
// exits.  Host code cannot use the array's name as a device address (on the
// host it names a stand-in object), so the first call on each device, with
// that device current, resolves the device address once with
// cudaGetSymbolAddress and caches it; every later call on that device reuses
// it.  That first call should therefore come before any stream capture.
//
// All calls share the array and it keeps the contents of the last call, so
// each call first rebuilds what it reads (seed table, ln table) and clears
// the accumulators that must start at zero.  Calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array and
// must be serialised by the caller.  The cached address belongs to the CUDA
// context it was resolved in; after cudaDeviceReset it is stale (documented
// in the header: no call after a device reset in the same process).
#include <cmath>
#include <mutex>

#include "../../include/vbdr.h"
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

constexpr uint32_t kNoallocMaxLog2G = 9;  // g <= 512: the seed table's capacity

// Layout of the scratch array.
struct NoallocScratch {
  KEnt ktab[kKtabSize];            // 8 KiB: seed table of the virtual indices
  double lnv[kLnTab];              // 4104 B: ln(v), v = 0..512
  unsigned long long sums[8];      // pool sums, reduction partials, block counter
};
constexpr size_t kScratchBytes = sizeof(NoallocScratch);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device address of g_noalloc_scratch, resolved once per device.
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(NoallocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<NoallocScratch *>(g_scratch_addr[dev]);
  return cudaSuccess;
}

// Rebuild the tables for this call's seed and clear the accumulators.
__global__ void noalloc_prepare_kernel(NoallocScratch *sc, uint64_t A0, uint32_t g) {
  const uint64_t K0 = mix64(A0);
  for (uint32_t i = threadIdx.x; i < g; i += blockDim.x)
    sc->ktab[i] = make_kent(mix64(mix64((uint64_t)i ^ K0) >> 32));
  for (uint32_t v = threadIdx.x; v < (uint32_t)kLnTab; v += blockDim.x)
    sc->lnv[v] = v ? log((double)v) : 0.0;
  if (threadIdx.x < 8) sc->sums[threadIdx.x] = 0ull;
}

// Pool sums S_Z = sum_j 2^(32 - reg_j), V_Z = #{reg_j = 0} over the caller's
// registers (values above 32 read as 32, as in the estimate's gather); the
// last block publishes them into sums[0], sums[1].
__global__ void __launch_bounds__(256)
    noalloc_pool_sums_kernel(const uint8_t *__restrict__ reg, uint64_t Z, NoallocScratch *sc) {
  unsigned long long S = 0, V = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < Z; j += stride) {
    const uint32_t M = min((uint32_t)reg[j], 32u);  // a caller's value above 32 reads as 32
    S += 1ull << (32u - M);
    V += (M == 0u);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_down_sync(0xffffffffu, S, o);
    V += __shfl_down_sync(0xffffffffu, V, o);
  }
  __shared__ unsigned long long sS[8], sV[8];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { sS[warp] = S; sV[warp] = V; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t i = 1; i < blockDim.x / 32; ++i) { S += sS[i]; V += sV[i]; }
    atomicAdd(&sc->sums[3], S);
    atomicAdd(&sc->sums[4], V);
    __threadfence();
    if (atomicAdd(&sc->sums[2], 1ull) == gridDim.x - 1) {
      __threadfence();
      sc->sums[0] = atomicExch(&sc->sums[3], 0ull);
      sc->sums[1] = atomicExch(&sc->sums[4], 0ull);
      sc->sums[2] = 0ull;
    }
  }
}

double hll_alpha_host(double m) {
  if (m == 16.0) return 0.673;
  if (m == 32.0) return 0.697;
  if (m == 64.0) return 0.709;
  return 0.7213 / (1.0 + 1.079 / m);
}

}  // namespace
}  // namespace vbk

extern "C" int vbdr_estimate_registers_noalloc(const uint8_t *d_reg, uint64_t num_bdr,
                                               uint32_t log2_g, uint64_t seed,
                                               const uint32_t *d_aips, uint64_t n_hosts,
                                               float *d_out, void *stream) {
  using namespace vbk;
  if (log2_g < 1) return VBDR_EINVAL;
  if (log2_g > kNoallocMaxLog2G) return VBDR_ERANGE;
  // the exact pool sum sum_j 2^(32 - reg_j) <= Z 2^32 must fit 64 bits
  if (num_bdr == 0 || num_bdr >= (1ull << 32) || num_bdr <= (1ull << log2_g)) return VBDR_EINVAL;
  if (!d_reg) return VBDR_EINVAL;
  if (n_hosts == 0) return VBDR_OK;
  if (!d_aips || !d_out || ((uintptr_t)d_aips & 3u) || ((uintptr_t)d_out & 3u))
    return VBDR_EINVAL;
  NoallocScratch *sc = nullptr;
  if (scratch_for_current_device(&sc) != cudaSuccess) return VBDR_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;

  Dims d = {};
  d.Z = num_bdr;
  d.Zs = (num_bdr + 3) & ~3ull;
  d.zmul = (uint32_t)num_bdr;
  d.b = log2_g;
  d.b_min = log2_g;
  d.group_rule = 0;
  d.A0 = seed;
  // the estimate reads only the registers, the seed table, ln table and sums
  DevState s = {};
  s.reg = const_cast<uint8_t *>(d_reg);
  s.ktab = sc->ktab;
  s.lnv = sc->lnv;
  s.sums = sc->sums;
  EstConst c = {};  // the plain estimate reads amm, kz, lng, inv_g and amm_Z
  const double Z = (double)num_bdr;
  for (int b = 0; b <= kMaxLog2G; ++b) {
    const double g = (double)(1u << b);
    c.amm[b] = hll_alpha_host(g) * g * g;
    c.kz[b] = Z * g / (Z - g);
    c.lng[b] = std::log(g);
    c.inv_g[b] = std::ldexp(1.0, -b);
  }
  c.amm_Z = hll_alpha_host(Z) * Z * Z;

  noalloc_prepare_kernel<<<1, 256, 0, st>>>(sc, seed, 1u << log2_g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return VBDR_ECUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t grid = (num_bdr + 255) / 256;
  if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
  noalloc_pool_sums_kernel<<<(unsigned)grid, 256, 0, st>>>(d_reg, num_bdr, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return VBDR_ECUDA;
  e = launch_estimate(d, s, c, d_aips, n_hosts, d_out, st, kEstCandidates[0]);
  return e == cudaSuccess ? VBDR_OK : VBDR_ECUDA;
}
