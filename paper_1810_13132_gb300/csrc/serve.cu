// serve.cu -- streaming service: many VBDR instances ("tenants") served at
// once on one GPU, each slice replayed as a CUDA graph.
//
// A tenant is one monitored link: its own BDR pool (device resident for its
// whole life), host list, copy and compute streams and two captured graphs
// (one per staging buffer).  A graph holds the whole per-slice path:
//   scan (pair count read from device memory, so one graph serves any slice
//   size) -> slide -> estimate (plain, or with the learned correction fused)
//   -> copy of the estimates to pinned host memory.
// Slices of one tenant are served in order; two may be in flight (the next
// slice's host-to-device copy runs on the copy stream while the previous
// slice's graph runs).  Tenants are independent and their streams overlap on
// the device.
//
// Admission: every tenant's device footprint is known when it asks to open;
// the server keeps the sum under its memory budget and a tenant that does not
// fit waits (bounded) until others close and free their slots -- new streams
// join while admitted ones keep running, continuous-batching style.
// Waiting is host-side only (condition variable, event polling with a
// deadline); no kernel here waits on anything.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/vbdr.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  uint32_t *d_pairs = nullptr;
  uint64_t *d_n = nullptr;
  uint64_t *h_n = nullptr;   // pinned, source of the device pair count
  float *d_out = nullptr;
  float *h_out = nullptr;    // pinned estimates
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t copied = nullptr, start = nullptr, end = nullptr;
  uint64_t ticket = 0;       // ticket in flight (0: free)
  Clock::time_point submitted;
};

struct Tenant {
  bool used = false;
  vbdr_t h = nullptr;
  uint64_t bytes = 0;
  uint64_t max_pairs = 0;
  uint64_t n_hosts = 0;
  uint32_t *d_aips = nullptr;
  cudaStream_t copy = nullptr, compute = nullptr;
  Slot slot[2];
  uint64_t next_ticket = 1;
};

}  // namespace

struct vbdr_server {
  vbdr_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  // Serialises tenant set-up (state creation, eager launches, graph capture)
  // and tear-down across threads: device-wide calls such as
  // cudaDeviceSynchronize or cudaFree must not run while another thread
  // captures a graph.
  std::mutex setup_mu;
  uint64_t in_use = 0;
  std::vector<Tenant> tenants;
};

namespace {

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return VBDR_OK;
  const char *v = std::getenv("VBDR_VERBOSE");  // name the failing CUDA error
  if (v && v[0] == '1') std::fprintf(stderr, "vbdr server: CUDA error %d (%s)\n", (int)e,
                                     cudaGetErrorString(e));
  return VBDR_ECUDA;
}

void free_tenant(Tenant &t) {
  if (t.compute) cudaStreamSynchronize(t.compute);
  if (t.copy) cudaStreamSynchronize(t.copy);
  for (Slot &s : t.slot) {
    if (s.exec) cudaGraphExecDestroy(s.exec);
    cudaFree(s.d_pairs);
    cudaFree(s.d_n);
    cudaFree(s.d_out);
    cudaFreeHost(s.h_n);
    cudaFreeHost(s.h_out);
    if (s.copied) cudaEventDestroy(s.copied);
    if (s.start) cudaEventDestroy(s.start);
    if (s.end) cudaEventDestroy(s.end);
    s = Slot();
  }
  cudaFree(t.d_aips);
  if (t.copy) cudaStreamDestroy(t.copy);
  if (t.compute) cudaStreamDestroy(t.compute);
  vbdr_destroy(t.h);
  t = Tenant();
}

// Capture one slot's per-slice graph on the tenant's compute stream.
int capture_slot(Tenant &t, Slot &s, vbdr_mlp_t mlp) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(t.compute, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_rc(e);
  int rc = vbdr_scan_slice_devn(t.h, s.d_pairs, s.d_n, t.max_pairs, t.compute);
  if (rc == VBDR_OK) rc = vbdr_slide(t.h, t.compute);
  if (rc == VBDR_OK)
    rc = mlp ? vbdr_estimate_learned(t.h, mlp, t.d_aips, t.n_hosts, s.d_out, t.compute)
             : vbdr_estimate(t.h, t.d_aips, t.n_hosts, s.d_out, t.compute);
  if (rc == VBDR_OK)
    rc = cuda_rc(cudaMemcpyAsync(s.h_out, s.d_out, t.n_hosts * sizeof(float),
                                 cudaMemcpyDeviceToHost, t.compute));
  e = cudaStreamEndCapture(t.compute, &g);
  if (rc != VBDR_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != VBDR_OK ? rc : cuda_rc(e);
  }
  e = cudaGraphInstantiate(&s.exec, g, 0);
  cudaGraphDestroy(g);
  return cuda_rc(e);
}

}  // namespace

extern "C" {

uint64_t vbdr_server_tenant_bytes(const vbdr_config *cfg, uint64_t max_pairs, uint64_t n_hosts) {
  if (!cfg || cfg->k == 0) return 0;
  uint32_t w = 0;
  while ((1u << w) < cfg->k + 1) ++w;
  const uint32_t b_min = cfg->log2_g_min ? cfg->log2_g_min : cfg->log2_g;
  const uint32_t R = 32 - b_min, F = 32 / w, P = (R + F - 1) / F;
  const uint64_t Zs = (cfg->num_bdr + 3) & ~3ull;
  const uint64_t chunk = 1ull << 15;  // registers are allocated in whole 32 KiB chunks
  const uint64_t reg = std::max<uint64_t>(Zs, (cfg->num_bdr + chunk - 1) / chunk * chunk);
  uint64_t bytes = Zs * 4ull * P + reg + (cfg->layout == VBDR_GFAST ? 4 * cfg->num_bdr : 0) +
                   (cfg->layout == VBDR_SERIAL ? Zs : 0) +
                   (cfg->layout == VBDR_GSMALL ? Zs : 0);  // PCSA statistics
  bytes += 64ull << 10;                                // tables, sums
  bytes += 2 * (max_pairs * 8 + 8 + n_hosts * 4);      // staging slots
  bytes += n_hosts * 4;                                // host list
  return bytes;
}

int vbdr_server_create(const vbdr_server_config *cfg, vbdr_server_t *out) {
  if (!out) return VBDR_EINVAL;
  *out = nullptr;
  if (!cfg || cfg->max_tenants == 0 || cfg->max_tenants > 1024 || cfg->reserved) return VBDR_EINVAL;
  vbdr_server *s = new (std::nothrow) vbdr_server();
  if (!s) return VBDR_ENOMEM;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->tenants.resize(cfg->max_tenants);
  *out = s;
  return VBDR_OK;
}

int vbdr_server_destroy(vbdr_server_t s) {
  if (!s) return VBDR_OK;
  for (Tenant &t : s->tenants)
    if (t.used) free_tenant(t);
  delete s;
  return VBDR_OK;
}

int vbdr_server_open(vbdr_server_t s, const vbdr_config *cfg, uint64_t max_pairs,
                     const uint32_t *h_aips, uint64_t n_hosts, vbdr_mlp_t mlp,
                     uint32_t timeout_ms, uint32_t *tenant) {
  if (!s || !cfg || !tenant || max_pairs == 0 || n_hosts == 0 || !h_aips) return VBDR_EINVAL;
  const uint64_t need = vbdr_server_tenant_bytes(cfg, max_pairs, n_hosts);
  if (need == 0 || need > s->cfg.device_budget_bytes) return VBDR_ERANGE;
  uint32_t id = 0;
  {
    // admission: wait for a free slot and room in the budget
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
      bool slot = false;
      for (id = 0; id < s->tenants.size(); ++id)
        if (!s->tenants[id].used) { slot = true; break; }
      if (slot && s->in_use + need <= s->cfg.device_budget_bytes) break;
      if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout) return VBDR_ETIMEOUT;
    }
    s->tenants[id].used = true;  // reserve
    s->tenants[id].bytes = need;
    s->in_use += need;
  }
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> setup(s->setup_mu);
  Tenant &t = s->tenants[id];
  t.max_pairs = max_pairs;
  t.n_hosts = n_hosts;
  int rc = vbdr_create(cfg, &t.h);
  cudaError_t e = cudaSuccess;
  if (rc == VBDR_OK) e = cudaStreamCreateWithFlags(&t.copy, cudaStreamNonBlocking);
  if (rc == VBDR_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&t.compute, cudaStreamNonBlocking);
  if (rc == VBDR_OK && e == cudaSuccess) e = cudaMalloc(&t.d_aips, n_hosts * 4);
  if (rc == VBDR_OK && e == cudaSuccess)
    e = cudaMemcpy(t.d_aips, h_aips, n_hosts * 4, cudaMemcpyHostToDevice);
  for (Slot &sl : t.slot) {
    if (rc != VBDR_OK || e != cudaSuccess) break;
    e = cudaMalloc(&sl.d_pairs, max_pairs * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_n, 8);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, n_hosts * 4);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_n, 8, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_out, n_hosts * 4, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.start);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.end);
    if (e == cudaSuccess) e = cudaMemset(sl.d_n, 0, 8);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = e == cudaErrorMemoryAllocation ? VBDR_ENOMEM : cuda_rc(e);
  }
  // The estimate call refuses to run before a first slide, so close one empty
  // slice eagerly before capturing: on the fresh state (every DR saturated,
  // no bit set) a slide changes nothing, and inside the graphs every estimate
  // follows that graph's own slide.
  if (rc == VBDR_OK) rc = vbdr_slide(t.h, t.compute);
  // one eager estimate sizes the handle's buffers outside the capture
  if (rc == VBDR_OK)
    rc = mlp ? vbdr_estimate_learned(t.h, mlp, t.d_aips, t.n_hosts, t.slot[0].d_out, t.compute)
             : vbdr_estimate(t.h, t.d_aips, t.n_hosts, t.slot[0].d_out, t.compute);
  if (rc == VBDR_OK) rc = cuda_rc(cudaStreamSynchronize(t.compute));
  if (rc == VBDR_OK) rc = capture_slot(t, t.slot[0], mlp);
  if (rc == VBDR_OK) rc = capture_slot(t, t.slot[1], mlp);
  if (rc != VBDR_OK) {
    free_tenant(t);
    setup.unlock();
    std::lock_guard<std::mutex> lock(s->mu);
    s->in_use -= need;
    s->cv.notify_all();
    return rc;
  }
  *tenant = id;
  return VBDR_OK;
}

int vbdr_server_close(vbdr_server_t s, uint32_t tenant) {
  if (!s || tenant >= s->tenants.size() || !s->tenants[tenant].used) return VBDR_EINVAL;
  Tenant &t = s->tenants[tenant];
  const uint64_t bytes = t.bytes;
  {
    std::lock_guard<std::mutex> setup(s->setup_mu);
    free_tenant(t);
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->in_use -= bytes;
  s->cv.notify_all();
  return VBDR_OK;
}

int vbdr_server_submit(vbdr_server_t s, uint32_t tenant, const uint32_t *h_pairs, uint64_t n,
                       uint64_t *ticket) {
  if (!s || tenant >= s->tenants.size() || !s->tenants[tenant].used || !ticket) return VBDR_EINVAL;
  Tenant &t = s->tenants[tenant];
  if (n > t.max_pairs) return VBDR_ERANGE;
  if (n && !h_pairs) return VBDR_EINVAL;
  const uint64_t tk = t.next_ticket;
  Slot &sl = t.slot[tk & 1];
  if (sl.ticket) return VBDR_EORDER;  // two slices already in flight: wait one first
  sl.submitted = Clock::now();
  *sl.h_n = n;
  // copy stream: after the slot's previous graph finished with its buffers
  cudaError_t e = cudaStreamWaitEvent(t.copy, sl.end, 0);
  if (e == cudaSuccess && n)
    e = cudaMemcpyAsync(sl.d_pairs, h_pairs, n * 8, cudaMemcpyHostToDevice, t.copy);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_n, sl.h_n, 8, cudaMemcpyHostToDevice, t.copy);
  if (e == cudaSuccess) e = cudaEventRecord(sl.copied, t.copy);
  // compute stream: slices in order, each after its copy
  if (e == cudaSuccess) e = cudaStreamWaitEvent(t.compute, sl.copied, 0);
  if (e == cudaSuccess) e = cudaEventRecord(sl.start, t.compute);
  if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, t.compute);
  if (e == cudaSuccess) e = cudaEventRecord(sl.end, t.compute);
  if (e != cudaSuccess) return VBDR_ECUDA;
  sl.ticket = tk;
  t.next_ticket++;
  *ticket = tk;
  return VBDR_OK;
}

int vbdr_server_wait(vbdr_server_t s, uint32_t tenant, uint64_t ticket, float *h_out,
                     uint32_t timeout_ms, float *device_ms, float *e2e_ms) {
  if (!s || tenant >= s->tenants.size() || !s->tenants[tenant].used) return VBDR_EINVAL;
  Tenant &t = s->tenants[tenant];
  Slot &sl = t.slot[ticket & 1];
  if (sl.ticket != ticket || ticket == 0) return VBDR_EINVAL;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    const cudaError_t q = cudaEventQuery(sl.end);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return VBDR_ECUDA;
    if (Clock::now() >= deadline) return VBDR_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  const auto done = Clock::now();
  if (h_out) std::memcpy(h_out, sl.h_out, t.n_hosts * sizeof(float));
  float ms = 0.f;
  if (device_ms) {
    cudaEventElapsedTime(&ms, sl.start, sl.end);
    *device_ms = ms;
  }
  if (e2e_ms)
    *e2e_ms = std::chrono::duration<float, std::milli>(done - sl.submitted).count();
  sl.ticket = 0;
  return VBDR_OK;
}

int vbdr_server_in_use(vbdr_server_t s, uint64_t *bytes, uint32_t *tenants) {
  if (!s) return VBDR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (bytes) *bytes = s->in_use;
  if (tenants) {
    uint32_t c = 0;
    for (const Tenant &t : s->tenants) c += t.used;
    *tenants = c;
  }
  return VBDR_OK;
}

int vbdr_server_tenant_handle(vbdr_server_t s, uint32_t tenant, vbdr_t *out) {
  if (!out) return VBDR_EINVAL;
  *out = nullptr;
  if (!s || tenant >= s->tenants.size() || !s->tenants[tenant].used) return VBDR_EINVAL;
  *out = s->tenants[tenant].h;
  return VBDR_OK;
}

}  // extern "C"
