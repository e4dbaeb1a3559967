// mlp.cu -- training and standalone inference of the learned correction's
// MLP (see mlp_device.cuh for the network and the feature definition).
//
// Training step = one launch of train_tile_kernel over the batch (a block
// takes a tile of 128 samples: forward on the tensor cores, loss gradient,
// backward -- dH1 = dZ2 W2 and the weight gradients dW2 = dZ2^T H1,
// dW1 = dZ1^T X as mma.sync GEMMs over the tile's samples -- and atomically
// adds its FP32 partial gradients) followed by adamw_kernel, which updates
// the FP32 master parameters, refreshes the BF16 weight copies and clears
// the gradient buffer.  The whole loop over epochs and batches runs here in
// the library; the caller passes the training set once.
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/vbdr.h"
#include "mlp_device.cuh"
#include "vbdr_internal.cuh"

struct vbdr_mlp {
  float *theta;          // FP32 master parameters [kMlpParams]
  float *grad;           // FP32 gradient accumulator [kMlpParams]
  float *adam_m, *adam_v;
  __nv_bfloat16 *w1c;    // [64][48]
  __nv_bfloat16 *w2;     // [64][64]
  uint2 *w1f, *w2f;      // BF16 weights in mma fragment order (inference)
  float *loss;           // [2]: sum of squared errors, samples
  float nmax;            // plain estimates above this fall back uncorrected
  uint64_t step;
  int sticky;
};

namespace vbk {
namespace {

constexpr int kTile = 128;          // samples per block
constexpr int kTrainThreads = 128;  // 4 warps, 32 samples each

struct TrainSmem {
  __nv_bfloat16 x[kTile][kMlpLive];
  float z1[kTile][kMlpHid];
  __nv_bfloat16 h1[kTile][kMlpHid];
  float z2[kTile][kMlpHid];
  __nv_bfloat16 dz2[kTile][kMlpHid];
  __nv_bfloat16 dz1[kTile][kMlpHid];
  __nv_bfloat16 w1c[kMlpHid][kMlpLive];
  __nv_bfloat16 w2[kMlpHid][kMlpHid];
  float g[kTile];
};

// One tile of the batch: forward, backward, partial gradients.
__global__ void __launch_bounds__(kTrainThreads)
    train_tile_kernel(const __nv_bfloat16 *__restrict__ X, const float *__restrict__ y,
                      uint64_t n, const float *__restrict__ theta,
                      const __nv_bfloat16 *__restrict__ w1c, const __nv_bfloat16 *__restrict__ w2,
                      float *grad, float *loss, float inv_batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, c = (lane & 3) * 2;
  const uint64_t row0 = (uint64_t)blockIdx.x * kTile;
  for (int i = tid; i < kTile * kMlpLive; i += blockDim.x) {
    const int r = i / kMlpLive, k = i % kMlpLive;
    S.x[r][k] = row0 + r < n ? X[(row0 + r) * kMlpLive + k] : __float2bfloat16(0.f);
  }
  for (int i = tid; i < kMlpHid * kMlpLive; i += blockDim.x) S.w1c[i / kMlpLive][i % kMlpLive] = w1c[i];
  for (int i = tid; i < kMlpHid * kMlpHid; i += blockDim.x) S.w2[i / kMlpHid][i % kMlpHid] = w2[i];
  __syncthreads();

  const int rb = 32 * warp;  // this warp's rows
  float acc[2][8][4];
  auto zero = [&]() {
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][j][q] = 0.f;
  };
  // ---- layer 1
  zero();
#pragma unroll
  for (int kk = 0; kk < kMlpLive / 16; ++kk) {
    uint32_t a[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
      load_a(a[m], [&](int r, int k) { return S.x[rb + 16 * m + r][16 * kk + k]; });
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t b[2];
      load_b(b, [&](int k, int col) { return S.w1c[8 * j + col][16 * kk + k]; });
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][j], a[m], b);
    }
  }
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + 16 * m + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        const float z = acc[m][j][q] + theta[kOffB1 + col];
        S.z1[r][col] = z;
        S.h1[r][col] = __float2bfloat16(gelu_f(z));
      }
  __syncwarp();
  // ---- layer 2
  zero();
#pragma unroll
  for (int kk = 0; kk < kMlpHid / 16; ++kk) {
    uint32_t a[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
      load_a(a[m], [&](int r, int k) { return S.h1[rb + 16 * m + r][16 * kk + k]; });
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t b[2];
      load_b(b, [&](int k, int col) { return S.w2[8 * j + col][16 * kk + k]; });
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][j], a[m], b);
    }
  }
  float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + 16 * m + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        const float z = acc[m][j][q] + theta[kOffB2 + col];
        S.z2[r][col] = z;
        part[2 * m + (q >> 1)] += gelu_f(z) * theta[kOffW3 + col];
      }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    part[i] += __shfl_xor_sync(0xffffffffu, part[i], 1);
    part[i] += __shfl_xor_sync(0xffffffffu, part[i], 2);
  }
  if ((lane & 3) == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + 16 * (i >> 1) + gq + 8 * (i & 1);
      const float d = part[i] + theta[kOffB3];
      const bool ok = row0 + r < n;
      const float e = ok ? d - y[row0 + r] : 0.f;
      S.g[r] = 2.f * e * inv_batch;  // d loss / d delta_r
      if (ok) atomicAdd(&loss[0], e * e);
    }
  }
  __syncwarp();
  // ---- output layer gradients and dZ2 (this warp's rows)
  float gw3[8][2] = {}, gb2[8][2] = {};
  float gb3 = 0.f;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + 16 * m + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        const float z = S.z2[r][col], gr = S.g[r];
        gw3[j][q & 1] += gr * gelu_f(z);
        const float dz = gr * theta[kOffW3 + col] * gelu_grad_f(z);
        gb2[j][q & 1] += dz;
        S.dz2[r][col] = __float2bfloat16(dz);
      }
  // reduce over the 8 row groups (lanes with equal lane % 4)
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        gw3[j][h] += __shfl_xor_sync(0xffffffffu, gw3[j][h], o);
        gb2[j][h] += __shfl_xor_sync(0xffffffffu, gb2[j][h], o);
      }
  if (lane < 4) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        atomicAdd(&grad[kOffW3 + 8 * j + c + h], gw3[j][h]);
        atomicAdd(&grad[kOffB2 + 8 * j + c + h], gb2[j][h]);
      }
  }
  gb3 = S.g[rb + lane];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
  if (lane == 0) atomicAdd(&grad[kOffB3], gb3);
  __syncthreads();

  // ---- dW2 = dZ2^T H1: warp computes rows 16*warp .. +15 of dW2, K = tile
  {
    float cw[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) cw[j][q] = 0.f;
    const int mb = 16 * warp;
#pragma unroll 2
    for (int kk = 0; kk < kTile / 16; ++kk) {
      uint32_t a[4];
      load_a(a, [&](int r, int k) { return S.dz2[16 * kk + k][mb + r]; });
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        load_b(b, [&](int k, int col) { return S.h1[16 * kk + k][8 * j + col]; });
        mma_bf16(cw[j], a, b);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = mb + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        atomicAdd(&grad[kOffW2 + r * kMlpHid + col], cw[j][q]);
      }
  }
  // ---- dH1 = dZ2 W2 (this warp's rows), dZ1 = dH1 * GELU'(Z1)
  zero();
#pragma unroll
  for (int kk = 0; kk < kMlpHid / 16; ++kk) {
    uint32_t a[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
      load_a(a[m], [&](int r, int k) { return S.dz2[rb + 16 * m + r][16 * kk + k]; });
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t b[2];
      load_b(b, [&](int k, int col) { return S.w2[16 * kk + k][8 * j + col]; });
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][j], a[m], b);
    }
  }
  float gb1[8][2] = {};
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + 16 * m + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        const float dz = acc[m][j][q] * gelu_grad_f(S.z1[r][col]);
        gb1[j][q & 1] += dz;
        S.dz1[r][col] = __float2bfloat16(dz);
      }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) gb1[j][h] += __shfl_xor_sync(0xffffffffu, gb1[j][h], o);
  if (lane < 4) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) atomicAdd(&grad[kOffB1 + 8 * j + c + h], gb1[j][h]);
  }
  __syncthreads();
  // ---- dW1 = dZ1^T X: warp computes rows 16*warp .. +15, the 48 live columns
  {
    float cw[6][4];
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) cw[j][q] = 0.f;
    const int mb = 16 * warp;
#pragma unroll 2
    for (int kk = 0; kk < kTile / 16; ++kk) {
      uint32_t a[4];
      load_a(a, [&](int r, int k) { return S.dz1[16 * kk + k][mb + r]; });
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        uint32_t b[2];
        load_b(b, [&](int k, int col) { return S.x[16 * kk + k][8 * j + col]; });
        mma_bf16(cw[j], a, b);
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = mb + gq + (q >> 1) * 8, col = 8 * j + c + (q & 1);
        atomicAdd(&grad[kOffW1 + r * kMlpIn + w1_col(col)], cw[j][q]);
      }
  }
  if (tid == 0) atomicAdd(&loss[1], (float)(n - row0 < (uint64_t)kTile ? n - row0 : kTile));
}

// AdamW on the FP32 master (decoupled weight decay on W1, W2, w3), then
// the BF16 copies, then the gradient is cleared for the next step.
__global__ void adamw_kernel(float *theta, float *grad, float *m, float *v,
                             __nv_bfloat16 *w1c, __nv_bfloat16 *w2, float lr, float wd,
                             float b1, float b2, float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const bool is_weight = i < kOffB1 || (i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3);
    float t = theta[i];
    if (is_weight) t -= lr * wd * t;
    t -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    theta[i] = t;
    grad[i] = 0.f;
  }
}

__device__ __forceinline__ uint32_t pack_rn(float lo, float hi) {
  return pack_bf16(__float2bfloat16(lo), __float2bfloat16(hi));
}

// BF16 copies of W1 (live columns) and W2 from the master, row-major for the
// training kernel and in mma fragment order for inference.
__global__ void refresh_bf16_kernel(const float *theta, __nv_bfloat16 *w1c, __nv_bfloat16 *w2,
                                    uint2 *w1f, uint2 *w2f) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int i = tid; i < kMlpHid * kMlpLive; i += nth)
    w1c[i] = __float2bfloat16(theta[kOffW1 + (i / kMlpLive) * kMlpIn + w1_col(i % kMlpLive)]);
  for (int i = tid; i < kMlpHid * kMlpHid; i += nth) w2[i] = __float2bfloat16(theta[kOffW2 + i]);
  // fragment entry e = (kk * 8 + n) * 32 + lane: B[k][j] = W[8n + j][16kk + k]
  for (int e = tid; e < kW1Frags + kW2Frags; e += nth) {
    const bool l1 = e < kW1Frags;
    const int f = l1 ? e : e - kW1Frags;
    const int lane = f & 31, n = (f >> 5) & 7, kk = f >> 8;
    const int row = 8 * n + (lane >> 2), k0 = 16 * kk + 2 * (lane & 3);
    auto W = [&](int k) {
      return l1 ? theta[kOffW1 + row * kMlpIn + w1_col(k)] : theta[kOffW2 + row * kMlpHid + k];
    };
    const uint2 v = make_uint2(pack_rn(W(k0), W(k0 + 1)), pack_rn(W(k0 + 8), W(k0 + 9)));
    if (l1) w1f[f] = v; else w2f[f] = v;
  }
}

// 16-byte asynchronous copy global -> shared (zero-filled when src_bytes = 0).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Start copying rows [r0, r0 + 32) of X into a padded tile (rows past n: 0).
__device__ __forceinline__ void prefetch_rows(const __nv_bfloat16 *X, uint64_t n, uint64_t r0,
                                              __nv_bfloat16 *xs) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < 32 * (kMlpLive / 8); i += 32) {
    const int r = i / (kMlpLive / 8), q = i % (kMlpLive / 8);
    const bool ok = r0 + r < n;
    cp_async16(xs + r * kXLd + 8 * q, ok ? (const void *)(X + (r0 + r) * kMlpLive + 8 * q)
                                          : (const void *)X, ok ? 16u : 0u);
  }
  cp_async_commit();
}

template <int WARPS>
__device__ __forceinline__ MlpDevWeights stage_weights(const MlpDevWeights &w, uint2 *w1s,
                                                       uint2 *w2s, float *bs) {
  for (int i = threadIdx.x; i < kW1Frags; i += WARPS * 32) w1s[i] = w.w1f[i];
  for (int i = threadIdx.x; i < kW2Frags; i += WARPS * 32) w2s[i] = w.w2f[i];
  for (int i = threadIdx.x; i < kMlpHid; i += WARPS * 32) {
    bs[i] = w.b1[i];
    bs[kMlpHid + i] = w.b2[i];
    bs[2 * kMlpHid + i] = w.w3[i];
  }
  if (threadIdx.x == 0) bs[3 * kMlpHid] = *w.b3;
  __syncthreads();
  return MlpDevWeights{w1s, w2s, bs, bs + kMlpHid, bs + 2 * kMlpHid, bs + 3 * kMlpHid};
}

constexpr int kFwdWarps = 8;

// Shared memory of the forward / correction kernels (dynamic, > 48 KB).
struct FwdSmem {
  uint2 w1s[kW1Frags];
  uint2 w2s[kW2Frags];
  float bs[3 * kMlpHid + 4];
  __nv_bfloat16 xs[kFwdWarps][2][32 * kXLd];  // double-buffered input rows
  __nv_bfloat16 h1s[kFwdWarps][16 * kHLd];     // one tile's hidden layer
};

// One warp per 32 rows (grid-stride); the next task's rows are copied in
// while the current ones run through the network.  CORRECT: est (the plain
// estimates) is replaced by the corrected estimate unless above nmax;
// otherwise delta is written to est.
template <bool CORRECT>
__global__ void __launch_bounds__(kFwdWarps * 32)
    mlp_rows_kernel(const __nv_bfloat16 *__restrict__ X, uint64_t n, MlpDevWeights w, float nmax,
                    float *__restrict__ est) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem &S = *reinterpret_cast<FwdSmem *>(smem_raw);
  const MlpDevWeights ws = stage_weights<kFwdWarps>(w, S.w1s, S.w2s, S.bs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t step = (uint64_t)gridDim.x * kFwdWarps * 32;
  uint64_t r0 = ((uint64_t)blockIdx.x * kFwdWarps + warp) * 32;
  int buf = 0;
  if (r0 < n) prefetch_rows(X, n, r0, S.xs[warp][0]);
  for (; r0 < n; r0 += step, buf ^= 1) {
    if (r0 + step < n) {
      prefetch_rows(X, n, r0 + step, S.xs[warp][buf ^ 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const float d = mlp_forward_warp(S.xs[warp][buf], S.h1s[warp], ws);
    if (r0 + lane < n) {
      if constexpr (CORRECT) {
        const float plain = est[r0 + lane];
        float corr = expm1f(log1pf(plain) + d);
        if (!(corr > 0.f)) corr = 0.f;
        est[r0 + lane] = plain > nmax ? plain : corr;
      } else {
        est[r0 + lane] = d;
      }
    }
    __syncwarp();  // the buffer is refilled two tasks later
  }
}

template <bool CORRECT>
cudaError_t launch_mlp_rows(const __nv_bfloat16 *X, uint64_t n, MlpDevWeights w, float nmax,
                            float *est, cudaStream_t st) {
  const int smem = (int)sizeof(FwdSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_rows_kernel<CORRECT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_rows_kernel<CORRECT>, kFwdWarps * 32, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t tasks = (n + 31) / 32;
  uint64_t grid = (tasks + kFwdWarps - 1) / kFwdWarps;
  if (grid > (uint64_t)sms * per_sm) grid = (uint64_t)sms * per_sm;  // persistent wave
  mlp_rows_kernel<CORRECT><<<(unsigned)grid, kFwdWarps * 32, smem, st>>>(X, n, w, nmax, est);
  return cudaGetLastError();
}

// splitmix64 stream for the initial weights (uniform(-a, a) per layer)
uint64_t init_rng(uint64_t *state) {
  *state += 0x9e3779b97f4a7c15ULL;
  return mix64(*state);
}

}  // namespace
}  // namespace vbk

using namespace vbk;

namespace {
int mlp_fail(vbdr_mlp *m, cudaError_t e) {
  if (e != cudaSuccess) {
    m->sticky = VBDR_ECUDA;
    return VBDR_ECUDA;
  }
  return VBDR_OK;
}
}  // namespace

extern "C" {

int vbdr_mlp_num_params(void) { return kMlpParams; }

int vbdr_mlp_create(uint64_t seed, vbdr_mlp_t *out) {
  if (!out) return VBDR_EINVAL;
  *out = nullptr;
  vbdr_mlp *m = new (std::nothrow) vbdr_mlp();
  if (!m) return VBDR_ENOMEM;
  std::memset(m, 0, sizeof(*m));
  cudaError_t e = cudaMalloc(&m->theta, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->w1c, kMlpHid * kMlpLive * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->w2, kMlpHid * kMlpHid * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->w1f, kW1Frags * sizeof(uint2));
  if (e == cudaSuccess) e = cudaMalloc(&m->w2f, kW2Frags * sizeof(uint2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    vbdr_mlp_destroy(m);
    return VBDR_ENOMEM;
  }
  // He-style uniform init from a seeded splitmix64 stream; biases zero
  float *h = new (std::nothrow) float[kMlpParams];
  if (!h) {
    vbdr_mlp_destroy(m);
    return VBDR_ENOMEM;
  }
  uint64_t st = seed;
  auto uni = [&](float a) {
    const uint64_t r = vbk::init_rng(&st);
    return (float)((double)(r >> 11) * 0x1.0p-53 * 2.0 - 1.0) * a;
  };
  for (int i = 0; i < kMlpParams; ++i) h[i] = 0.f;
  for (int i = 0; i < kMlpHid * kMlpIn; ++i) h[kOffW1 + i] = uni(std::sqrt(6.f / kMlpLive));
  for (int i = 0; i < kMlpHid * kMlpHid; ++i) h[kOffW2 + i] = uni(std::sqrt(6.f / kMlpHid));
  for (int i = 0; i < kMlpHid; ++i) h[kOffW3 + i] = uni(std::sqrt(3.f / kMlpHid)) * 0.1f;
  m->nmax = 3.0e38f;
  const int rc = vbdr_mlp_set_params(m, h, m->nmax);
  delete[] h;
  if (rc != VBDR_OK) {
    vbdr_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return VBDR_OK;
}

int vbdr_mlp_destroy(vbdr_mlp_t m) {
  if (!m) return VBDR_OK;
  cudaDeviceSynchronize();
  cudaFree(m->theta);
  cudaFree(m->grad);
  cudaFree(m->adam_m);
  cudaFree(m->adam_v);
  cudaFree(m->w1c);
  cudaFree(m->w2);
  cudaFree(m->loss);
  cudaFree(m->w1f);
  cudaFree(m->w2f);
  delete m;
  return VBDR_OK;
}

int vbdr_mlp_set_params(vbdr_mlp_t m, const float *h_params, float nmax) {
  if (!m || !h_params) return VBDR_EINVAL;
  if (m->sticky) return m->sticky;
  cudaError_t e = cudaMemcpy(m->theta, h_params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->grad, 0, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, kMlpParams * sizeof(float));
  if (e == cudaSuccess) {
    refresh_bf16_kernel<<<64, 256>>>(m->theta, m->w1c, m->w2, m->w1f, m->w2f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  m->nmax = nmax;
  m->step = 0;
  return mlp_fail(m, e);
}

int vbdr_mlp_get_params(vbdr_mlp_t m, float *h_params, float *nmax) {
  if (!m || !h_params) return VBDR_EINVAL;
  if (m->sticky) return m->sticky;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(h_params, m->theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
  if (nmax) *nmax = m->nmax;
  return mlp_fail(m, e);
}

int vbdr_mlp_gradient(vbdr_mlp_t m, const uint16_t *d_X, const float *d_y, uint64_t n,
                      float *h_grad, float *h_loss, void *stream) {
  if (!m || !d_X || !d_y || !h_grad || n == 0) return VBDR_EINVAL;
  if (m->sticky) return m->sticky;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, kMlpParams * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, 2 * sizeof(float), st);
  if (e == cudaSuccess) {
    train_tile_kernel<<<(unsigned)((n + kTile - 1) / kTile), kTrainThreads, smem, st>>>(
        reinterpret_cast<const __nv_bfloat16 *>(d_X), d_y, n, m->theta, m->w1c, m->w2, m->grad,
        m->loss, 1.0f / (float)n);
    e = cudaGetLastError();
  }
  float lsum[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_grad, m->grad, kMlpParams * sizeof(float),
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lsum, m->loss, sizeof(lsum), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, kMlpParams * sizeof(float), st);
  if (h_loss) *h_loss = lsum[1] > 0 ? lsum[0] / lsum[1] : 0.f;
  return mlp_fail(m, e);
}

int vbdr_mlp_train(vbdr_mlp_t m, const uint16_t *d_X, const float *d_y, uint64_t n,
                   uint32_t epochs, uint32_t batch, float lr, float weight_decay,
                   uint64_t shuffle_seed, float *h_epoch_loss, void *stream) {
  if (!m || !d_X || !d_y || n == 0 || batch == 0 || epochs == 0) return VBDR_EINVAL;
  if (m->sticky) return m->sticky;
  (void)shuffle_seed;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return mlp_fail(m, e);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const uint64_t nb = (n + batch - 1) / batch;
  for (uint32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    e = cudaMemsetAsync(m->loss, 0, 2 * sizeof(float), st);
    // batches are contiguous slices; the caller shuffles the set once
    for (uint64_t bi = 0; bi < nb && e == cudaSuccess; ++bi) {
      const uint64_t r0 = bi * batch;
      const uint64_t cnt = (n - r0) < batch ? (n - r0) : batch;
      train_tile_kernel<<<(unsigned)((cnt + kTile - 1) / kTile), kTrainThreads, smem, st>>>(
          reinterpret_cast<const __nv_bfloat16 *>(d_X) + r0 * kMlpLive, d_y + r0, cnt, m->theta,
          m->w1c, m->w2, m->grad, m->loss, 1.0f / (float)cnt);
      e = cudaGetLastError();
      if (e != cudaSuccess) break;
      ++m->step;
      const float bc1 = 1.f - std::pow(b1, (float)m->step);
      const float bc2 = 1.f - std::pow(b2, (float)m->step);
      adamw_kernel<<<37, 256, 0, st>>>(m->theta, m->grad, m->adam_m, m->adam_v, m->w1c, m->w2, lr,
                                       weight_decay, b1, b2, eps, bc1, bc2);
      e = cudaGetLastError();
      if (e == cudaSuccess) {
        refresh_bf16_kernel<<<16, 256, 0, st>>>(m->theta, m->w1c, m->w2, m->w1f, m->w2f);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess && h_epoch_loss) {
      float lsum[2];
      e = cudaMemcpyAsync(lsum, m->loss, sizeof(lsum), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      h_epoch_loss[ep] = lsum[1] > 0 ? lsum[0] / lsum[1] : 0.f;
    }
  }
  return mlp_fail(m, e);
}

int vbdr_mlp_forward(vbdr_mlp_t m, const uint16_t *d_X, uint64_t n, float *d_delta, void *stream) {
  if (!m) return VBDR_EINVAL;
  if (m->sticky) return m->sticky;
  if (n == 0) return VBDR_OK;
  if (!d_X || !d_delta || ((uintptr_t)d_X & 15)) return VBDR_EINVAL;
  return mlp_fail(m, launch_mlp_rows<false>(reinterpret_cast<const __nv_bfloat16 *>(d_X), n,
                                            mlp_weights(m), 0.f, d_delta, (cudaStream_t)stream));
}

}  // extern "C"

namespace vbk {
cudaError_t launch_mlp_correct(const vbdr_mlp *m, const __nv_bfloat16 *X, uint64_t n, float *est,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return launch_mlp_rows<true>(X, n, mlp_weights(m), m->nmax, est, st);
}

MlpDevWeights mlp_weights(const vbdr_mlp *m) {
  return MlpDevWeights{m->w1f, m->w2f, m->theta + kOffB1, m->theta + kOffB2, m->theta + kOffW3,
                       m->theta + kOffB3};
}
float mlp_nmax(const vbdr_mlp *m) { return m->nmax; }
}  // namespace vbk
