// api.cu -- the C ABI of include/vbdr.h: argument checks, device state
// ownership, host-buffer staging, and the state-initialisation kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vbdr.h"
#include "vbdr_internal.cuh"

using vbk::DevState;

namespace {
// NVTX range over an entry point (tracing tools show the library's calls on
// the timeline beside its kernels; without a tool attached it costs a
// branch).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
using vbk::Dims;
using vbk::EstConst;

struct vbdr {
  Dims d;
  DevState s;
  vbk::EstConst est;
  vbk::EstLaunch est_cfg;  // estimate launch shape (autotuned or set)
  int layout;
  int device;
  int sticky;          // first CUDA error seen (VBDR_ECUDA once set)
  bool slid;           // at least one slide done
  // host-buffer staging (allocated on first use)
  cudaStream_t copy_stream;
  cudaEvent_t ev_copied[2], ev_free[2];
  uint32_t *stage[2];
  uint64_t stage_pairs;  // capacity of one staging buffer, in pairs
  uint32_t *d_aips;
  float *d_out;
  uint64_t est_cap;
  uint16_t *d_feat;     // feature rows of the learned estimate [feat_cap][48]
  uint64_t feat_cap;
  uint4 *d_crec;        // records of the compact correction [crec_cap]
  uint64_t crec_cap;
  vbk::BucketDev bk;    // buffers of the bucketed scan (allocated when it is selected)
  int scan_mode;        // VBDR_SCAN_DIRECT (default) or VBDR_SCAN_BUCKETED
};

// A host list's estimate plan (plan.cu): device arrays plus the handle
// configuration it was built for.
struct vbdr_plan {
  int device;
  uint64_t Z;
  uint32_t b, b_min, group_rule;
  uint64_t A0;
  vbk::PlanDev dev;
  uint32_t *aips;  // owned copy of the host list
  uint64_t n_entries;
  uint64_t bytes;  // device bytes held
};

namespace {

// InitDR on every DR (Sec. 3): every field = 2^w - 1; bsLBP1 = 0; registers 0;
// the virtual-index seed table; the pool-sum accumulators.
__global__ void init_kernel(Dims d, DevState s, uint32_t word_init, uint32_t ktab_n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t j = tid; j < d.Zs; j += stride) {
    for (uint32_t p = 0; p < d.P; ++p) s.drv[(uint64_t)p * d.Zs + j] = word_init;
    if (j < d.Z) {
      if (s.bs) s.bs[j] = 0u;
      s.reg[j] = 0u;
    }
  }
  // Alg. 3's first hash depends on the virtual index only:
  // s1(i) = H(i, 2^32, A0), stored premixed as mix64(s1(i)).
  const uint64_t K0 = vbk::mix64(d.A0);
  for (uint64_t i = tid; i < ktab_n; i += stride) {
    const uint64_t s1 = vbk::mix64(i ^ K0) >> 32;
    s.ktab[i] = vbk::make_kent(vbk::mix64(s1));
  }
  if (tid < vbk::kSums) s.sums[tid] = 0ull;
  if (tid == 0) *s.check = 0u;
  if (s.pcsa)
    for (uint64_t j = tid; j < d.Zs; j += stride) s.pcsa[j] = 0u;
}

// HyperLogLog bias constant alpha_m (Flajolet et al. 2007).
double hll_alpha(double m) {
  if (m == 16.0) return 0.673;
  if (m == 32.0) return 0.697;
  if (m == 64.0) return 0.709;
  return 0.7213 / (1.0 + 1.079 / m);
}

// LogLog bias constant (Durand & Flajolet 2003):
//   alpha_m = (Gamma(-1/m) (1 - 2^(1/m)) / ln 2)^(-m),
// with 1 - 2^(1/m) taken as -expm1(ln 2 / m) so that large m keep their
// digits.  PCSA's correction factor phi (Flajolet & Martin 1985).
double loglog_alpha(double m) {
  const double base = std::tgamma(-1.0 / m) * -std::expm1(std::log(2.0) / m) / std::log(2.0);
  return std::pow(base, -m);
}
constexpr double kPcsaPhi = 0.77351;

void fill_est_const(const Dims &d, EstConst *c) {
  const double Z = (double)d.Z;
  for (int b = 0; b <= vbk::kMaxLog2G; ++b) {
    const double g = (double)(1u << b);
    c->amm[b] = hll_alpha(g) * g * g;
    c->kz[b] = Z * g / (Z - g);
    c->lng[b] = std::log(g);
  }
  c->amm_Z = hll_alpha(Z) * Z * Z;
  for (int b = 0; b <= vbk::kMaxLog2G; ++b) {
    const double g = (double)(1u << b);
    c->ll[b] = b ? loglog_alpha(g) * g : 0.0;
    c->pc[b] = g / kPcsaPhi;
    c->inv_g[b] = std::ldexp(1.0, -b);
  }
  c->ll_Z = loglog_alpha(Z) * Z;
  c->pc_Z = Z / kPcsaPhi;
}

// VBDR_VERBOSE=1 names on stderr the CUDA error behind a VBDR_ECUDA.
void report_cuda(cudaError_t e) {
  static const bool verbose = [] {
    const char *v = std::getenv("VBDR_VERBOSE");
    return v && v[0] == '1';
  }();
  if (verbose) std::fprintf(stderr, "vbdr: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
}

int fail_cuda(vbdr *h, cudaError_t e) {
  if (e != cudaSuccess) {
    report_cuda(e);
    h->sticky = VBDR_ECUDA;
    return VBDR_ECUDA;
  }
  return VBDR_OK;
}

// Largest log2 g of any host of the handle.
uint32_t max_log2_g(const Dims &d) { return d.group_rule ? d.b_min + 3 : d.b; }

// The feature histogram counts a host's register values in 8-bit fields per
// lane and 16-bit fields per host: g <= 512 keeps every count in range.
constexpr uint32_t kMaxFeatureLog2G = 9;

uint32_t ktab_entries(const Dims &d) {
  const uint32_t gmax = 1u << (d.group_rule ? d.b_min + 3 : d.b);
  return gmax > (uint32_t)vbk::kKtabSize ? gmax : (uint32_t)vbk::kKtabSize;
}

void free_state(vbdr *h) {
  cudaFree(h->s.drv);
  cudaFree(h->s.bs);
  cudaFree(h->s.now);
  cudaFree(h->s.reg);
  cudaFree(h->s.pcsa);
  cudaFree(h->s.ktab);
  cudaFree(h->s.lnv);
  cudaFree(h->s.sums);
  cudaFree(h->s.check);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->stage[i]);
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  cudaFree(h->d_aips);
  cudaFree(h->d_out);
  cudaFree(h->d_feat);
  cudaFree(h->d_crec);
  cudaFree(h->bk.recs);
  cudaFree(h->bk.fill);
  cudaFree(h->bk.lb);
}

// Slices of at least this many pairs take the bucketed scan (bucket.cu); its
// apply pass costs a fixed amount per non-empty pool tile, which smaller
// slices do not repay.
constexpr uint64_t kBucketMinPairs = 1ull << 18;

// The scan of n pairs (n_dev: device-side count up to n, for graphs).
cudaError_t scan_any(vbdr *h, const uint32_t *pairs, uint64_t n, cudaStream_t st,
                     const uint64_t *n_dev = nullptr) {
  if (h->scan_mode == VBDR_SCAN_BUCKETED && h->bk.recs && n >= kBucketMinPairs)
    return vbk::launch_scan_bucketed(h->d, h->s, h->bk, h->layout, pairs, n, st, n_dev);
  return vbk::launch_scan(h->d, h->s, h->layout, pairs, n, st, n_dev);
}

}  // namespace

extern "C" {

const char *vbdr_strerror(int status) {
  switch (status) {
    case VBDR_OK: return "ok";
    case VBDR_EINVAL: return "invalid argument";
    case VBDR_ENOMEM: return "out of memory";
    case VBDR_ECUDA: return "CUDA error (handle unusable)";
    case VBDR_ERANGE: return "size exceeds capacity";
    case VBDR_EORDER: return "call out of order (no slide yet)";
    case VBDR_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
  }
}

int vbdr_create(const vbdr_config *cfg, vbdr_t *out) {
  if (!out) return VBDR_EINVAL;
  *out = nullptr;
  if (!cfg || cfg->reserved != 0) return VBDR_EINVAL;
  if (cfg->k < 1 || cfg->k > 255) return VBDR_EINVAL;
  if (cfg->layout != VBDR_GFAST && cfg->layout != VBDR_GSMALL && cfg->layout != VBDR_SERIAL)
    return VBDR_EINVAL;
  if (cfg->group_rule > 1) return VBDR_EINVAL;
  const uint32_t b_min = cfg->log2_g_min ? cfg->log2_g_min : cfg->log2_g;
  if (b_min < 1 || b_min > (uint32_t)vbk::kMaxLog2G) return VBDR_EINVAL;
  if (cfg->group_rule == 0 &&
      (cfg->log2_g < b_min || cfg->log2_g > (uint32_t)vbk::kMaxLog2G))
    return VBDR_EINVAL;
  if (cfg->group_rule == 1 && b_min + 3 > 9) return VBDR_EINVAL;
  const uint32_t b_max = cfg->group_rule ? b_min + 3 : cfg->log2_g;
  // the exact pool sum sum_j 2^(32 - reg_j) <= Z 2^32 must fit 64 bits
  if (cfg->num_bdr == 0 || cfg->num_bdr >= (1ull << 32) ||
      cfg->num_bdr <= (1ull << b_max))
    return VBDR_EINVAL;

  vbdr *h = new (std::nothrow) vbdr();
  if (!h) return VBDR_ENOMEM;
  std::memset(h, 0, sizeof(*h));
  Dims &d = h->d;
  d.Z = cfg->num_bdr;
  d.Zs = (d.Z + 3) & ~3ull;
  d.zmul = (uint32_t)d.Z;
  d.k = cfg->k;
  d.w = 0;
  while ((1u << d.w) < cfg->k + 1) ++d.w;
  d.F = 32 / d.w;
  d.R = 32 - b_min;
  d.P = (d.R + d.F - 1) / d.F;
  d.b = cfg->group_rule ? b_min : cfg->log2_g;
  d.b_min = b_min;
  d.group_rule = cfg->group_rule;
  d.A0 = cfg->seed;
  d.A1 = vbk::mix64(cfg->seed + 0x9e3779b97f4a7c15ULL);
  d.K1 = vbk::make_kent(vbk::mix64(d.A1));
  h->layout = (int)cfg->layout;
  cudaGetDevice(&h->device);

  uint32_t word_init = 0;
  for (uint32_t f = 0; f < d.F; ++f) word_init |= ((1u << d.w) - 1u) << (f * d.w);

  const uint32_t kn = ktab_entries(d);
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&h->s.drv, (size_t)d.P * d.Zs * sizeof(uint32_t));
  if (e == cudaSuccess && h->layout == VBDR_GFAST)
    e = cudaMalloc(&h->s.bs, (size_t)d.Z * sizeof(uint32_t));
  if (e == cudaSuccess && h->layout == VBDR_SERIAL) {
    e = cudaMalloc(&h->s.now, (size_t)d.Zs);
    if (e == cudaSuccess) e = cudaMemset(h->s.now, 0, (size_t)d.Zs);
  }
  // registers: whole 32-bit words, and whole plan chunks (the planned
  // estimate copies reg chunk by chunk)
  const uint64_t reg_bytes =
      std::max<uint64_t>(d.Zs, (d.Z + vbk::kPlanChunk - 1) / vbk::kPlanChunk * vbk::kPlanChunk);
  if (e == cudaSuccess) e = cudaMalloc(&h->s.reg, (size_t)reg_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->s.reg, 0, (size_t)reg_bytes);
  if (e == cudaSuccess && h->layout == VBDR_GSMALL) e = cudaMalloc(&h->s.pcsa, (size_t)d.Zs);
  if (e == cudaSuccess) e = cudaMalloc(&h->s.ktab, (size_t)kn * sizeof(vbk::KEnt));
  if (e == cudaSuccess) e = cudaMalloc(&h->s.lnv, vbk::kLnTab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->s.sums, vbk::kSums * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->s.check, sizeof(unsigned int));
  if (e == cudaSuccess) {
    double lnv[vbk::kLnTab];
    lnv[0] = 0.0;
    for (int v = 1; v < vbk::kLnTab; ++v) lnv[v] = std::log((double)v);
    e = cudaMemcpy(h->s.lnv, lnv, sizeof(lnv), cudaMemcpyHostToDevice);
  }
  fill_est_const(d, &h->est);
  h->est_cfg = vbk::kEstCandidates[0];
  if (e != cudaSuccess) {
    cudaGetLastError();
    report_cuda(e);
    free_state(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? VBDR_ENOMEM : VBDR_ECUDA;
  }
  init_kernel<<<1024, 256>>>(d, h->s, word_init, kn);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    report_cuda(e);
    free_state(h);
    delete h;
    return VBDR_ECUDA;
  }
  *out = h;
  return VBDR_OK;
}

int vbdr_destroy(vbdr_t h) {
  if (!h) return VBDR_OK;
  cudaDeviceSynchronize();
  free_state(h);
  delete h;
  return VBDR_OK;
}

int vbdr_set_scan_mode(vbdr_t h, int mode) {
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (mode == VBDR_SCAN_DIRECT) {
    h->scan_mode = mode;
    return VBDR_OK;
  }
  if (mode != VBDR_SCAN_BUCKETED) return VBDR_EINVAL;
  if (!vbk::bucket_scan_applies(h->d, h->layout)) return VBDR_EINVAL;
  if (!h->bk.recs) {  // the buffers, once per handle
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(h, e);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    vbk::BucketDev bk = {};
    vbk::bucket_layout(h->d.Z, sms, &bk);
    const size_t regions = (size_t)bk.ncta * bk.ntiles;
    e = cudaMalloc(&bk.recs, regions * bk.cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&bk.fill, regions * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&bk.lb, (size_t)bk.ntiles << vbk::kBucketTileLog2);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(bk.recs);
      cudaFree(bk.fill);
      cudaFree(bk.lb);
      return e == cudaErrorMemoryAllocation ? VBDR_ENOMEM : fail_cuda(h, e);
    }
    h->bk = bk;
  }
  h->scan_mode = mode;
  return VBDR_OK;
}

int vbdr_get_dims(vbdr_t h, uint32_t *R, uint32_t *w, uint32_t *words) {
  if (!h) return VBDR_EINVAL;
  if (R) *R = h->d.R;
  if (w) *w = h->d.w;
  if (words) *words = h->d.P;
  return VBDR_OK;
}

int vbdr_scan_slice(vbdr_t h, const uint32_t *d_pairs, uint64_t n, void *stream) {
  NvtxRange nvtx("vbdr_scan_slice");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (n == 0) return VBDR_OK;
  if (!d_pairs || ((uintptr_t)d_pairs & 15u)) return VBDR_EINVAL;
  return fail_cuda(h, scan_any(h, d_pairs, n, (cudaStream_t)stream));
}

int vbdr_scan_slice_devn(vbdr_t h, const uint32_t *d_pairs, const uint64_t *d_n,
                         uint64_t max_n, void *stream) {
  NvtxRange nvtx("vbdr_scan_slice_devn");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (max_n == 0) return VBDR_OK;
  if (!d_pairs || !d_n || ((uintptr_t)d_pairs & 15u) || ((uintptr_t)d_n & 7u)) return VBDR_EINVAL;
  return fail_cuda(h, scan_any(h, d_pairs, max_n, (cudaStream_t)stream, d_n));
}

int vbdr_scan_slice_host(vbdr_t h, const uint32_t *h_pairs, uint64_t n, void *stream) {
  NvtxRange nvtx("vbdr_scan_slice_host");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (n == 0) return VBDR_OK;
  if (!h_pairs) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (!h->stage[0]) {
    const uint64_t cap = 8ull << 20;  // 8M pairs (64 MiB) per staging buffer
    for (int i = 0; i < 2; ++i) {
      e = cudaMalloc(&h->stage[i], cap * 8);
      if (e != cudaSuccess) { cudaGetLastError(); return VBDR_ENOMEM; }
      if (cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_free[i], cudaEventDisableTiming) != cudaSuccess)
        return fail_cuda(h, cudaErrorUnknown);
    }
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail_cuda(h, cudaErrorUnknown);
    h->stage_pairs = cap;
    // both buffers start free
    for (int i = 0; i < 2; ++i) {
      e = cudaEventRecord(h->ev_free[i], h->copy_stream);
      if (e != cudaSuccess) return fail_cuda(h, e);
    }
  }
  // The copies wait only for their staging buffer (ev_free), not for earlier
  // work on the caller's stream: a slice's pairs cross to the device while
  // the previous slice's slide and estimate still run.  The scans themselves
  // are ordered on the stream.
  uint64_t done = 0;
  int buf = 0;
  while (done < n) {
    uint64_t cnt = n - done;
    if (cnt > h->stage_pairs) cnt = h->stage_pairs;
    e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[buf], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->stage[buf], h_pairs + 2 * done, cnt * 8,
                          cudaMemcpyHostToDevice, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[buf], h->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_copied[buf], 0);
    if (e != cudaSuccess) return fail_cuda(h, e);
    e = scan_any(h, h->stage[buf], cnt, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_free[buf], st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    done += cnt;
    buf ^= 1;
  }
  return VBDR_OK;
}

int vbdr_slide(vbdr_t h, void *stream) {
  NvtxRange nvtx("vbdr_slide");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  int rc = fail_cuda(h, vbk::launch_slide(h->d, h->s, h->layout,
                                           (cudaStream_t)stream));
  if (rc == VBDR_OK) h->slid = true;
  return rc;
}

int vbdr_estimate(vbdr_t h, const uint32_t *d_aips, uint64_t n, float *d_out,
                  void *stream) {
  NvtxRange nvtx("vbdr_estimate");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n == 0) return VBDR_OK;
  if (!d_aips || !d_out || ((uintptr_t)d_aips & 3u) || ((uintptr_t)d_out & 3u))
    return VBDR_EINVAL;
  return fail_cuda(h, vbk::launch_estimate(h->d, h->s, h->est, d_aips, n, d_out,
                                            (cudaStream_t)stream, h->est_cfg));
}

int vbdr_estimate_alt(vbdr_t h, const uint32_t *d_aips, uint64_t n, float *d_out,
                      int estimator, void *stream) {
  NvtxRange nvtx("vbdr_estimate_alt");
  if (!h) return VBDR_EINVAL;
  if (estimator == VBDR_EST_HLL) return vbdr_estimate(h, d_aips, n, d_out, stream);
  if (estimator != VBDR_EST_LOGLOG && estimator != VBDR_EST_PCSA) return VBDR_EINVAL;
  if (estimator == VBDR_EST_PCSA && h->layout != VBDR_GSMALL) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n == 0) return VBDR_OK;
  if (!d_aips || !d_out || ((uintptr_t)d_aips & 3u) || ((uintptr_t)d_out & 3u))
    return VBDR_EINVAL;
  return fail_cuda(h, vbk::launch_estimate_alt(h->d, h->s, h->est, d_aips, n, d_out, estimator,
                                                (cudaStream_t)stream, h->est_cfg));
}

int vbdr_estimate_host(vbdr_t h, const uint32_t *h_aips, uint64_t n, float *h_out,
                       void *stream) {
  NvtxRange nvtx("vbdr_estimate_host");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n == 0) return VBDR_OK;
  if (!h_aips || !h_out) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (n > h->est_cap) {
    // wait until earlier estimates that use the old buffers are done
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    cudaFree(h->d_aips);
    cudaFree(h->d_out);
    h->d_aips = nullptr;
    h->d_out = nullptr;
    h->est_cap = 0;
    if (cudaMalloc(&h->d_aips, n * 4) != cudaSuccess ||
        cudaMalloc(&h->d_out, n * 4) != cudaSuccess) {
      cudaGetLastError();
      return VBDR_ENOMEM;
    }
    h->est_cap = n;
  }
  e = cudaMemcpyAsync(h->d_aips, h_aips, n * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = vbk::launch_estimate(h->d, h->s, h->est, h->d_aips, n, h->d_out, st, h->est_cfg);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, h->d_out, n * 4, cudaMemcpyDeviceToHost, st);
  return fail_cuda(h, e);
}

int vbdr_features(vbdr_t h, const uint32_t *d_aips, uint64_t n, uint16_t *d_X, float *d_plain,
                  void *stream) {
  NvtxRange nvtx("vbdr_features");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n == 0) return VBDR_OK;
  // feature rows are written with 8- and 16-byte stores
  if (!d_aips || !d_X || ((uintptr_t)d_aips & 3u) || ((uintptr_t)d_X & 15u)) return VBDR_EINVAL;
  if (d_plain && ((uintptr_t)d_plain & 3u)) return VBDR_EINVAL;
  if (max_log2_g(h->d) > kMaxFeatureLog2G) return VBDR_ERANGE;
  float *plain = d_plain;
  cudaStream_t st = (cudaStream_t)stream;
  if (!plain) {  // the kernel always writes the plain estimates: use the staging buffer
    if (n > h->est_cap) return VBDR_ERANGE;
    plain = h->d_out;
  }
  return fail_cuda(h, vbk::launch_features(h->d, h->s, h->est, d_aips, n,
                                           reinterpret_cast<__nv_bfloat16 *>(d_X), plain, st,
                                           h->est_cfg));
}

int vbdr_estimate_learned(vbdr_t h, vbdr_mlp_t m, const uint32_t *d_aips, uint64_t n,
                          float *d_out, void *stream) {
  NvtxRange nvtx("vbdr_estimate_learned");
  if (!h || !m) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n == 0) return VBDR_OK;
  if (!d_aips || !d_out || ((uintptr_t)d_aips & 3u) || ((uintptr_t)d_out & 3u))
    return VBDR_EINVAL;
  if (max_log2_g(h->d) > kMaxFeatureLog2G) return VBDR_ERANGE;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > h->feat_cap) {
    // feature rows live in a buffer owned by the handle, grown here (never
    // inside a graph capture: the service sizes it before capturing)
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    cudaFree(h->d_feat);
    h->d_feat = nullptr;
    h->feat_cap = 0;
    if (cudaMalloc(&h->d_feat, n * vbk::kMlpLive * sizeof(uint16_t)) != cudaSuccess) {
      cudaGetLastError();
      return VBDR_ENOMEM;
    }
    h->feat_cap = n;
  }
  // gather + histogram (plain launch shape) -> feature rows and plain
  // estimates; then the MLP on the tensor cores corrects them in place
  cudaError_t e = vbk::launch_features(h->d, h->s, h->est, d_aips, n,
                                       reinterpret_cast<__nv_bfloat16 *>(h->d_feat), d_out, st,
                                       h->est_cfg);
  if (e == cudaSuccess)
    e = vbk::launch_mlp_correct(m, reinterpret_cast<const __nv_bfloat16 *>(h->d_feat), n, d_out, st);
  return fail_cuda(h, e);
}

int vbdr_load_virtual_registers(vbdr_t h, const uint32_t *d_aips, const uint64_t *d_offsets,
                                uint64_t n_hosts, const uint8_t *d_vregs, void *stream) {
  NvtxRange nvtx("vbdr_load_virtual_registers");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (n_hosts && (!d_aips || !d_offsets || !d_vregs)) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = vbk::launch_load_virtual(h->d, h->s, d_aips, d_offsets, n_hosts, d_vregs, st);
  // no PCSA statistics at register level: they read as 0
  if (e == cudaSuccess && h->s.pcsa) e = cudaMemsetAsync(h->s.pcsa, 0, h->d.Zs, st);
  if (e == cudaSuccess) e = vbk::launch_pool_sums(h->s.reg, h->s.pcsa, h->d.Z, h->s.sums, st);
  int rc = fail_cuda(h, e);
  if (rc == VBDR_OK) h->slid = true;
  return rc;
}

int vbdr_set_estimate_launch(vbdr_t h, uint32_t lanes, uint32_t threads) {
  if (!h) return VBDR_EINVAL;
  if ((lanes != 8 && lanes != 16 && lanes != 32) || threads < 32 || threads > 512 ||
      threads % 32)
    return VBDR_EINVAL;
  h->est_cfg = vbk::EstLaunch{(int)lanes, (int)threads};
  return VBDR_OK;
}

int vbdr_autotune_estimate(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts, float *d_out,
                           uint32_t *lanes, uint32_t *threads, void *stream) {
  NvtxRange nvtx("vbdr_autotune_estimate");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->slid) return VBDR_EORDER;
  if (n_hosts == 0 || !d_aips || !d_out) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail_cuda(h, cudaErrorUnknown);
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail_cuda(h, cudaErrorUnknown);
  }
  float best = 1e30f;
  vbk::EstLaunch best_cfg = vbk::kEstCandidates[0];
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < vbk::kNumEstCandidates && e == cudaSuccess; ++c) {
    const vbk::EstLaunch cfg = vbk::kEstCandidates[c];
    // one untimed launch, then the mean of two timed launches
    e = vbk::launch_estimate(h->d, h->s, h->est, d_aips, n_hosts, d_out, st, cfg);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r)
      e = vbk::launch_estimate(h->d, h->s, h->est, d_aips, n_hosts, d_out, st, cfg);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_cfg = cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail_cuda(h, e);
  h->est_cfg = best_cfg;
  if (lanes) *lanes = (uint32_t)best_cfg.lanes;
  if (threads) *threads = (uint32_t)best_cfg.threads;
  return VBDR_OK;
}

namespace {
// Checkpoint layout: header, then the raw device buffers in a fixed order.
struct CkptHeader {
  char magic[8];  // "VBDRCKP2"
  uint32_t k, log2_g, log2_g_min, group_rule, layout, slid;
  uint64_t num_bdr, seed, drv_bytes, slice_bytes, reg_bytes, pcsa_bytes;
};

void ckpt_sizes(const vbdr *h, uint64_t *drv, uint64_t *slice, uint64_t *reg, uint64_t *pcsa) {
  *drv = (uint64_t)h->d.P * h->d.Zs * 4;
  *slice = h->s.bs ? h->d.Z * 4 : (h->s.now ? h->d.Zs : 0);
  *reg = h->d.Zs;
  *pcsa = h->s.pcsa ? h->d.Zs : 0;
}
constexpr uint64_t kCkptSums = vbk::kSums * sizeof(unsigned long long);

void fill_header(const vbdr *h, CkptHeader *hd) {
  std::memset(hd, 0, sizeof(*hd));
  std::memcpy(hd->magic, "VBDRCKP2", 8);
  hd->k = h->d.k;
  hd->log2_g = h->d.b;
  hd->log2_g_min = h->d.b_min;
  hd->group_rule = h->d.group_rule;
  hd->layout = (uint32_t)h->layout;
  hd->slid = h->slid ? 1u : 0u;
  hd->num_bdr = h->d.Z;
  hd->seed = h->d.A0;
  ckpt_sizes(h, &hd->drv_bytes, &hd->slice_bytes, &hd->reg_bytes, &hd->pcsa_bytes);
}
}  // namespace

int vbdr_state_bytes(vbdr_t h, uint64_t *bytes) {
  if (!h || !bytes) return VBDR_EINVAL;
  uint64_t a, b, c, q;
  ckpt_sizes(h, &a, &b, &c, &q);
  *bytes = sizeof(CkptHeader) + a + b + c + q + kCkptSums;
  return VBDR_OK;
}

int vbdr_save(vbdr_t h, void *h_buf, uint64_t cap, void *stream) {
  NvtxRange nvtx("vbdr_save");
  if (!h || !h_buf) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  uint64_t need = 0;
  vbdr_state_bytes(h, &need);
  if (cap < need) return VBDR_ERANGE;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(h, e);
  CkptHeader hd;
  fill_header(h, &hd);
  uint8_t *p = static_cast<uint8_t *>(h_buf);
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  e = cudaMemcpy(p, h->s.drv, hd.drv_bytes, cudaMemcpyDeviceToHost);
  p += hd.drv_bytes;
  if (e == cudaSuccess && hd.slice_bytes)
    e = cudaMemcpy(p, h->s.bs ? (void *)h->s.bs : (void *)h->s.now, hd.slice_bytes,
                   cudaMemcpyDeviceToHost);
  p += hd.slice_bytes;
  if (e == cudaSuccess) e = cudaMemcpy(p, h->s.reg, hd.reg_bytes, cudaMemcpyDeviceToHost);
  p += hd.reg_bytes;
  if (e == cudaSuccess && hd.pcsa_bytes)
    e = cudaMemcpy(p, h->s.pcsa, hd.pcsa_bytes, cudaMemcpyDeviceToHost);
  p += hd.pcsa_bytes;
  if (e == cudaSuccess) e = cudaMemcpy(p, h->s.sums, kCkptSums, cudaMemcpyDeviceToHost);
  return fail_cuda(h, e);
}

int vbdr_load(vbdr_t h, const void *h_buf, uint64_t len, void *stream) {
  NvtxRange nvtx("vbdr_load");
  if (!h || !h_buf) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  uint64_t need = 0;
  vbdr_state_bytes(h, &need);
  if (len < need) return VBDR_EINVAL;
  CkptHeader mine, hd;
  fill_header(h, &mine);
  std::memcpy(&hd, h_buf, sizeof(hd));
  mine.slid = hd.slid;  // the one field that may differ
  if (std::memcmp(&mine, &hd, sizeof(hd)) != 0) return VBDR_EINVAL;  // other configuration
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  const uint8_t *p = static_cast<const uint8_t *>(h_buf) + sizeof(hd);
  if (e == cudaSuccess) e = cudaMemcpy(h->s.drv, p, hd.drv_bytes, cudaMemcpyHostToDevice);
  p += hd.drv_bytes;
  if (e == cudaSuccess && hd.slice_bytes)
    e = cudaMemcpy(h->s.bs ? (void *)h->s.bs : (void *)h->s.now, p, hd.slice_bytes,
                   cudaMemcpyHostToDevice);
  p += hd.slice_bytes;
  if (e == cudaSuccess) e = cudaMemcpy(h->s.reg, p, hd.reg_bytes, cudaMemcpyHostToDevice);
  p += hd.reg_bytes;
  if (e == cudaSuccess && hd.pcsa_bytes)
    e = cudaMemcpy(h->s.pcsa, p, hd.pcsa_bytes, cudaMemcpyHostToDevice);
  p += hd.pcsa_bytes;
  if (e == cudaSuccess) e = cudaMemcpy(h->s.sums, p, kCkptSums, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) h->slid = hd.slid != 0;
  return fail_cuda(h, e);
}

int vbdr_copy_state(vbdr_t h, uint8_t *h_dr, uint32_t *h_bs, uint8_t *h_reg,
                    void *stream) {
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  cudaStream_t st = (cudaStream_t)stream;
  const Dims &d = h->d;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(h, e);
  if (h_dr) {
    std::vector<uint32_t> words;
    try {
      words.resize((size_t)d.P * d.Zs);
    } catch (...) {
      return VBDR_ENOMEM;
    }
    e = cudaMemcpy(words.data(), h->s.drv, words.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const uint32_t fm = (1u << d.w) - 1u;
    for (uint64_t j = 0; j < d.Z; ++j)
      for (uint32_t r = 1; r <= d.R; ++r) {
        const uint32_t p = (r - 1) / d.F, f = (r - 1) % d.F;
        h_dr[j * d.R + (r - 1)] = (uint8_t)((words[(size_t)p * d.Zs + j] >> (f * d.w)) & fm);
      }
  }
  if (h_bs) {
    if (h->s.bs) {
      e = cudaMemcpy(h_bs, h->s.bs, d.Z * 4, cudaMemcpyDeviceToHost);
    } else if (h->s.now) {  // serial: nowLBP1 values
      std::vector<uint8_t> now(d.Z);
      e = cudaMemcpy(now.data(), h->s.now, d.Z, cudaMemcpyDeviceToHost);
      for (uint64_t j = 0; j < d.Z; ++j) h_bs[j] = now[j];
    } else {
      std::memset(h_bs, 0, d.Z * 4);
    }
    if (e != cudaSuccess) return fail_cuda(h, e);
  }
  if (h_reg) {
    e = cudaMemcpy(h_reg, h->s.reg, d.Z, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(h, e);
  }
  return VBDR_OK;
}

int vbdr_copy_pool_sums(vbdr_t h, uint64_t *S_Z, uint64_t *V_Z, void *stream) {
  if (!h || !S_Z || !V_Z) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  unsigned long long v[2];
  cudaError_t e = cudaMemcpyAsync(v, h->s.sums, sizeof(v), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(h, e);
  *S_Z = v[0];
  *V_Z = v[1];
  return VBDR_OK;
}

int vbdr_check_flags(vbdr_t h, uint32_t *flags, int *checked_build) {
  if (!h || !flags) return VBDR_EINVAL;
  if (checked_build) *checked_build = vbk::kChecked ? 1 : 0;
  if (h->sticky) return h->sticky;
  unsigned int v = 0;
  cudaError_t e = cudaMemcpy(&v, h->s.check, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda(h, e);
  *flags = v;
  return VBDR_OK;
}

int vbdr_copy_pool_sums_alt(vbdr_t h, uint64_t *L_Z, uint64_t *P_Z, void *stream) {
  if (!h || !L_Z || !P_Z) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  unsigned long long v[vbk::kSums];
  cudaError_t e = cudaMemcpyAsync(v, h->s.sums, sizeof(v), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(h, e);
  *L_Z = v[vbk::kSumL];
  *P_Z = v[vbk::kSumP];
  return VBDR_OK;
}

int vbdr_copy_pcsa(vbdr_t h, uint8_t *h_pcsa, void *stream) {
  if (!h || !h_pcsa) return VBDR_EINVAL;
  if (h->layout != VBDR_GSMALL) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  cudaError_t e = cudaMemcpyAsync(h_pcsa, h->s.pcsa, h->d.Z, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return fail_cuda(h, e);
}

/* ------------------------------------------------------- several GPUs */

namespace {
// The slice state the replicas merge: bsLBP1 (gfast), the DRV (gsmall; the
// scan zeroes DRs in place), nowLBP1 as words (serial).
void slice_state_of(const vbdr *h, uint32_t **ptr, uint64_t *words) {
  if (h->layout == VBDR_GFAST) {
    *ptr = h->s.bs;
    *words = h->d.Z;
  } else if (h->layout == VBDR_GSMALL) {
    *ptr = h->s.drv;
    *words = (uint64_t)h->d.P * h->d.Zs;
  } else {
    *ptr = reinterpret_cast<uint32_t *>(h->s.now);
    *words = h->d.Zs / 4;
  }
}
}  // namespace

int vbdr_state_pointers(vbdr_t h, uint32_t **d_slice_state, uint64_t *slice_words,
                        uint8_t **d_reg, uint8_t **d_pcsa) {
  if (!h) return VBDR_EINVAL;
  uint32_t *p = nullptr;
  uint64_t w = 0;
  slice_state_of(h, &p, &w);
  if (d_slice_state) *d_slice_state = p;
  if (slice_words) *slice_words = w;
  if (d_reg) *d_reg = h->s.reg;
  if (d_pcsa) *d_pcsa = h->s.pcsa;
  return VBDR_OK;
}

int vbdr_route_records(vbdr_t h, const uint32_t *d_pairs, uint64_t n, uint32_t n_ranks,
                       uint32_t *d_recs, uint64_t cap, uint64_t *d_fill, void *stream) {
  NvtxRange nvtx("vbdr_route_records");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (n_ranks < 1 || n_ranks > vbk::kMaxRanks || h->d.Z > (1ull << 27)) return VBDR_EINVAL;
  if (!d_fill || ((uintptr_t)d_fill & 7u)) return VBDR_EINVAL;
  if (n && (!d_pairs || !d_recs || ((uintptr_t)d_pairs & 3u) || ((uintptr_t)d_recs & 3u)))
    return VBDR_EINVAL;
  if ((h->d.group_rule ? 1u << (h->d.b_min + 3) : 1u << h->d.b) > (uint32_t)vbk::kKtabSize)
    return VBDR_ERANGE;
  return fail_cuda(h, vbk::launch_route_records(h->d, h->s, d_pairs, n, n_ranks, d_recs, cap,
                                                reinterpret_cast<unsigned long long *>(d_fill),
                                                (cudaStream_t)stream));
}

int vbdr_apply_records(vbdr_t h, const uint32_t *d_recs, uint64_t n, void *stream) {
  NvtxRange nvtx("vbdr_apply_records");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (n == 0) return VBDR_OK;
  if (!d_recs || ((uintptr_t)d_recs & 3u) || h->d.Z > (1ull << 27)) return VBDR_EINVAL;
  return fail_cuda(h, vbk::launch_apply_records(h->d, h->s, h->layout, d_recs, n,
                                                (cudaStream_t)stream));
}

int vbdr_merge_slice_state(vbdr_t h, const uint32_t *d_other, void *stream) {
  NvtxRange nvtx("vbdr_merge_slice_state");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!d_other || ((uintptr_t)d_other & 3u)) return VBDR_EINVAL;
  uint32_t *p = nullptr;
  uint64_t w = 0;
  slice_state_of(h, &p, &w);
  return fail_cuda(h, vbk::launch_merge_slice_state(h->d, h->s, h->layout, d_other, w,
                                                    (cudaStream_t)stream));
}

int vbdr_set_registers(vbdr_t h, const uint8_t *d_reg, const uint8_t *d_pcsa, void *stream) {
  NvtxRange nvtx("vbdr_set_registers");
  if (!h) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!d_reg || (d_pcsa && !h->s.pcsa)) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h->s.reg, d_reg, h->d.Z, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && d_pcsa)
    e = cudaMemcpyAsync(h->s.pcsa, d_pcsa, h->d.Z, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = vbk::launch_pool_sums(h->s.reg, h->s.pcsa, h->d.Z, h->s.sums, st);
  int rc = fail_cuda(h, e);
  if (rc == VBDR_OK) h->slid = true;
  return rc;
}

/* ---------------------------------------------------------------- plans */

}  // extern "C"

namespace {
int plan_create(vbdr_t h, const uint32_t *d_aips, uint64_t n, uint32_t max_hb, vbdr_plan_t *out,
                void *stream);
}  // namespace

extern "C" {

int vbdr_plan_create(vbdr_t h, const uint32_t *d_aips, uint64_t n, vbdr_plan_t *out,
                     void *stream) {
  NvtxRange nvtx("vbdr_plan_create");
  return plan_create(h, d_aips, n, vbk::kPlanMaxHB, out, stream);
}

int vbdr_plan_create_learned(vbdr_t h, const uint32_t *d_aips, uint64_t n, vbdr_plan_t *out,
                             void *stream) {
  NvtxRange nvtx("vbdr_plan_create_learned");
  return plan_create(h, d_aips, n, vbk::kLearnMaxHB, out, stream);
}

}  // extern "C"

namespace {
int plan_create(vbdr_t h, const uint32_t *d_aips, uint64_t n, uint32_t max_hb, vbdr_plan_t *out,
                void *stream) {
  if (!h || !out) return VBDR_EINVAL;
  *out = nullptr;
  if (h->sticky) return h->sticky;
  if (n > 0 && (!d_aips || ((uintptr_t)d_aips & 3u))) return VBDR_EINVAL;
  const Dims &d = h->d;
  const uint64_t nchunks = (d.Z + vbk::kPlanChunk - 1) / vbk::kPlanChunk;
  if (nchunks > vbk::kPlanMaxChunks) return VBDR_ERANGE;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (sms < 1) sms = 1;
  // blocks of at most max_hb hosts, a whole number of waves of one block per SM
  const uint64_t per_wave = (uint64_t)sms * max_hb;
  const uint64_t waves = n ? (n + per_wave - 1) / per_wave : 0;
  const uint64_t HB = n ? (n + (uint64_t)sms * waves - 1) / ((uint64_t)sms * waves) : 1;
  const uint64_t NB = (n + HB - 1) / HB;

  vbdr_plan *p = new (std::nothrow) vbdr_plan;
  if (!p) return VBDR_ENOMEM;
  std::memset(p, 0, sizeof(*p));
  p->device = h->device;
  p->Z = d.Z;
  p->b = d.b;
  p->b_min = d.b_min;
  p->group_rule = d.group_rule;
  p->A0 = d.A0;
  vbk::PlanDev &pd = p->dev;
  pd.n = n;
  pd.HB = (uint32_t)HB;
  pd.NB = (uint32_t)NB;
  pd.nchunks = (uint32_t)nchunks;
  const uint64_t ngroups = NB * nchunks;
  std::vector<uint32_t> counts(ngroups);
  std::vector<unsigned long long> goff(ngroups + 1);
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    cudaGetLastError();
    cudaFree(p->aips);
    cudaFree(pd.entries);
    cudaFree(pd.goff);
    cudaFree(pd.counts);
    cudaFree(pd.err);
    delete p;
    return err == cudaErrorMemoryAllocation ? VBDR_ENOMEM : fail_cuda(h, err);
  };
  e = cudaMalloc(&p->aips, std::max<uint64_t>(n, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&pd.goff, (ngroups + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&pd.counts, std::max<uint64_t>(ngroups, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&pd.err, 4);
  if (e != cudaSuccess) return fail(e);
  pd.aips = p->aips;
  if (n) e = cudaMemcpyAsync(p->aips, d_aips, n * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pd.err, 0, 4, st);
  if (e == cudaSuccess) e = vbk::launch_plan_count(d, h->s, pd, st);
  if (e == cudaSuccess && ngroups)
    e = cudaMemcpyAsync(counts.data(), pd.counts, ngroups * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  // group offsets, each group padded to whole uint4s of entries
  unsigned long long run = 0;
  for (uint64_t i = 0; i < ngroups; ++i) {
    goff[i] = run;
    run += (counts[i] + 3ull) & ~3ull;
  }
  goff[ngroups] = run;
  p->n_entries = run;
  e = cudaMalloc(&pd.entries, std::max<unsigned long long>(run, 4) * 4);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pd.goff, goff.data(), (ngroups + 1) * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = vbk::launch_plan_fill(d, h->s, pd, st);
  if (e == cudaSuccess) e = vbk::launch_plan_sort(pd, max_hb <= vbk::kLearnMaxHB, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  cudaFree(pd.counts);
  pd.counts = nullptr;
  p->bytes = std::max<uint64_t>(n, 1) * 4 + (ngroups + 1) * 8 + std::max<unsigned long long>(run, 4) * 4 + 4;
  *out = p;
  return VBDR_OK;
}
}  // namespace

extern "C" {

int vbdr_plan_destroy(vbdr_plan_t p) {
  if (!p) return VBDR_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  cudaFree(p->aips);
  cudaFree(p->dev.entries);
  cudaFree(p->dev.goff);
  cudaFree(p->dev.counts);
  cudaFree(p->dev.err);
  if (cur != p->device) cudaSetDevice(cur);
  delete p;
  return VBDR_OK;
}

int vbdr_plan_info(vbdr_plan_t p, uint64_t *n_hosts, uint64_t *n_entries, uint64_t *device_bytes) {
  if (!p) return VBDR_EINVAL;
  if (n_hosts) *n_hosts = p->dev.n;
  if (n_entries) *n_entries = p->n_entries;
  if (device_bytes) *device_bytes = p->bytes;
  return VBDR_OK;
}

int vbdr_plan_status(vbdr_plan_t p) {
  if (!p) return VBDR_EINVAL;
  uint32_t err = 0;
  if (cudaMemcpy(&err, p->dev.err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return VBDR_ECUDA;
  }
  return err ? VBDR_ETIMEOUT : VBDR_OK;
}

namespace {
bool plan_matches(const vbdr *h, const vbdr_plan *p) {
  return p->device == h->device && p->Z == h->d.Z && p->b == h->d.b && p->b_min == h->d.b_min &&
         p->group_rule == h->d.group_rule && p->A0 == h->d.A0;
}
}  // namespace

int vbdr_estimate_planned(vbdr_t h, vbdr_plan_t p, float *d_out, void *stream) {
  NvtxRange nvtx("vbdr_estimate_planned");
  if (!h || !p) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!plan_matches(h, p)) return VBDR_EINVAL;
  if (!h->slid) return VBDR_EORDER;
  if (p->dev.n == 0) return VBDR_OK;
  if (!d_out || ((uintptr_t)d_out & 3u)) return VBDR_EINVAL;
  return fail_cuda(h, vbk::launch_planned_estimate(h->d, h->s, h->est, p->dev, nullptr, nullptr,
                                                   d_out, (cudaStream_t)stream));
}

int vbdr_estimate_planned_compact(vbdr_t h, vbdr_plan_t p, const float *h_theta, float nmax,
                                  float *d_out, void *stream) {
  NvtxRange nvtx("vbdr_estimate_planned_compact");
  if (!h || !p || !h_theta) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!plan_matches(h, p)) return VBDR_EINVAL;
  if (!h->slid) return VBDR_EORDER;
  if (max_log2_g(h->d) > kMaxFeatureLog2G) return VBDR_ERANGE;
  const uint64_t n = p->dev.n;
  if (n == 0) return VBDR_OK;
  if (!d_out || ((uintptr_t)d_out & 3u)) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (n + 1 > h->crec_cap) {  // the records' buffer, grown outside any capture
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    cudaFree(h->d_crec);
    h->d_crec = nullptr;
    h->crec_cap = 0;
    if (cudaMalloc(&h->d_crec, (n + 1) * sizeof(uint4)) != cudaSuccess) {
      cudaGetLastError();
      return VBDR_ENOMEM;
    }
    h->crec_cap = n + 1;
  }
  vbk::CompactParams net;
  std::memcpy(net.w, h_theta, sizeof(net.w));
  net.nmax = nmax;
  return fail_cuda(h, vbk::launch_planned_estimate(h->d, h->s, h->est, p->dev, &net, h->d_crec,
                                                   d_out, st));
}

int vbdr_estimate_learned_planned(vbdr_t h, vbdr_mlp_t m, vbdr_plan_t p, float *d_out,
                                  void *stream) {
  NvtxRange nvtx("vbdr_estimate_learned_planned");
  if (!h || !p || !m) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!plan_matches(h, p) || p->dev.HB > vbk::kLearnMaxHB) return VBDR_EINVAL;
  if (!h->slid) return VBDR_EORDER;
  const uint64_t n = p->dev.n;
  if (n == 0) return VBDR_OK;
  if (!d_out || ((uintptr_t)d_out & 3u)) return VBDR_EINVAL;
  if (max_log2_g(h->d) > kMaxFeatureLog2G) return VBDR_ERANGE;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > h->feat_cap) {  // the feature rows' buffer, grown outside any capture
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    cudaFree(h->d_feat);
    h->d_feat = nullptr;
    h->feat_cap = 0;
    if (cudaMalloc(&h->d_feat, n * vbk::kMlpLive * sizeof(uint16_t)) != cudaSuccess) {
      cudaGetLastError();
      return VBDR_ENOMEM;
    }
    h->feat_cap = n;
  }
  __nv_bfloat16 *X = reinterpret_cast<__nv_bfloat16 *>(h->d_feat);
  cudaError_t e = vbk::launch_planned_features(h->d, h->s, h->est, p->dev, d_out, X, st);
  if (e == cudaSuccess) e = vbk::launch_mlp_correct(m, X, n, d_out, st);
  return fail_cuda(h, e);
}

int vbdr_estimate_planned_host(vbdr_t h, vbdr_plan_t p, float *h_out, void *stream) {
  NvtxRange nvtx("vbdr_estimate_planned_host");
  if (!h || !p) return VBDR_EINVAL;
  if (h->sticky) return h->sticky;
  if (!plan_matches(h, p)) return VBDR_EINVAL;
  if (!h->slid) return VBDR_EORDER;
  const uint64_t n = p->dev.n;
  if (n == 0) return VBDR_OK;
  if (!h_out) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (n > h->est_cap) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(h, e);
    cudaFree(h->d_aips);
    cudaFree(h->d_out);
    h->d_aips = nullptr;
    h->d_out = nullptr;
    h->est_cap = 0;
    if (cudaMalloc(&h->d_aips, n * 4) != cudaSuccess ||
        cudaMalloc(&h->d_out, n * 4) != cudaSuccess) {
      cudaGetLastError();
      return VBDR_ENOMEM;
    }
    h->est_cap = n;
  }
  e = vbk::launch_planned_estimate(h->d, h->s, h->est, p->dev, nullptr, nullptr, h->d_out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, h->d_out, n * 4, cudaMemcpyDeviceToHost, st);
  return fail_cuda(h, e);
}

}  // extern "C"
