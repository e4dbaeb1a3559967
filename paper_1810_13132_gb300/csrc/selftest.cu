// selftest.cu -- failure detection of the device-side waits.
//
// The planned estimate waits on mbarriers (the TMA copies of its ring and
// the consumers' releases) with a bounded wait: a wait that outlasts its
// limit returns false, the kernel records the failure in an error word and
// finishes.  This entry point exercises that path on the GPU without a
// fault: one warp waits on an mbarrier that nothing ever arrives on.
#include "../../include/vbdr.h"
#include "async_sm100.cuh"
#include "vbdr_internal.cuh"

namespace vbk {
namespace {

__global__ void bounded_wait_probe_kernel(uint64_t limit_ns, unsigned int *timed_out) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  __syncthreads();
  if (!mbar_wait_bounded(&mbar, 0, limit_ns)) atomicAdd(timed_out, 1u);
}

}  // namespace
}  // namespace vbk

extern "C" {

int vbdr_selftest_bounded_wait(uint32_t limit_us, void *stream) {
  if (limit_us == 0 || limit_us > 10000000u) return VBDR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int *d_count = nullptr, h_count = 0;
  cudaError_t e = cudaMalloc(&d_count, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    vbk::bounded_wait_probe_kernel<<<1, 32, 0, st>>>((uint64_t)limit_us * 1000ull, d_count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_count, d_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VBDR_ECUDA;
  }
  return h_count == 32u ? VBDR_ETIMEOUT : VBDR_OK;
}

}  // extern "C"
