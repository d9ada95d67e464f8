// bs_internal.cuh -- shared internals of libbs (not part of the C ABI).
//
// Compiled with --fmad=false: a*b+c is never contracted.  Every fused
// multiply-add in the library is an explicit fma()/fmaf(), so results are
// reproducible and match the definitions bit for bit where they promise to.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "bs.h"
#include "bs_check.cuh"

namespace bs {

// ------------------------------------------------------------ errors

int fail(int status, const char *fmt, ...);  // records detail, returns status
void clear_error();

#define BS_CUDA_TRY(call)                                                     \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return ::bs::fail(BS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,          \
                        cudaGetErrorString(e_), __FILE__, __LINE__);          \
  } while (0)

#define BS_LAUNCH_CHECK()                                                     \
  do {                                                                        \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess)                                                    \
      return ::bs::fail(BS_ERR_CUDA, "kernel launch failed: %s (%s:%d)",      \
                        cudaGetErrorString(e_), __FILE__, __LINE__);          \
  } while (0)

#define BS_ARG(cond, ...)                                                     \
  do {                                                                        \
    if (!(cond)) return ::bs::fail(BS_ERR_ARG, __VA_ARGS__);                  \
  } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------ device

struct DeviceInfo {
  int device = -1;
  int sms = 0;               // streaming multiprocessors
  int max_threads_sm = 0;    // resident threads per SM
};
// Properties of the current device (cached per device).
int device_info(DeviceInfo *out);

// ------------------------------------------------------------ launch shapes

constexpr int kStreamBlock = 256;   // threads per block, streaming kernels
constexpr int kReduceBlock = 256;   // threads per block, reductions
constexpr int kMaxPartials = 4096;  // per-block partials a workspace holds

// Grid for a grid-stride streaming kernel over `work` items of which each
// thread handles `per_thread` per sweep: a multiple of the SM count, never
// more blocks than there is work.
int stream_grid(int64_t work, int per_thread, int block, int blocks_per_sm);

// Resident blocks per SM of `kernel` at `block` threads on the current
// device (queried once per kernel and device, then cached).
int occupancy_blocks(const void *kernel, int block);

// As occupancy_blocks for launches with `smem` bytes of dynamic shared
// memory; first raises the kernel's dynamic shared-memory limit to `smem`
// (once per kernel and device).  A kernel template instantiated in several
// translation units has one host entry per unit, each registered on its own,
// so the limit is kept per entry address.  Returns 0 when the device refuses
// the limit or fits no block.
int occupancy_blocks_smem(const void *kernel, int block, int smem);

}  // namespace bs

// Workspace for single-launch reductions.
struct bs_workspace {
  int device;
  double *partials;        // [kMaxPartials]
  unsigned int *counter;   // arrival counter, 0 between launches
};

// ------------------------------------------------------------ device helpers

namespace bs {

// Sum over a block of BLOCK threads in a fixed order (shuffle tree within
// warps, then warp 0 over the warp sums).  Result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
  static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block");
  __shared__ double s_warp[BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  v = 0.0;
  if (warp == 0) {
    v = lane < BLOCK / 32 ? s_warp[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();  // s_warp may be reused by the caller
  return v;
}

// Last-block-done combine.  Every block calls it with its partial (valid in
// thread 0).  Returns true in all threads of the last block to arrive; in
// that block *total receives the sum of all partials, taken in block-index
// order independent of arrival order (valid in thread 0).  The arrival
// counter is reset to zero for the next launch.
template <int BLOCK>
__device__ __forceinline__ bool grid_combine(double partial, double *partials,
                                             unsigned int *counter,
                                             double *total) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = partial;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double v = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += BLOCK)
    v = v + __ldcg(partials + b);
  v = block_sum<BLOCK>(v);
  if (threadIdx.x == 0) {
    *total = v;
    *counter = 0u;
  }
  return true;
}

// Two-value form of grid_combine: partials holds 2*gridDim.x doubles.
template <int BLOCK>
__device__ __forceinline__ bool grid_combine2(double p0, double p1, double *partials,
                                              unsigned int *counter, double *t0,
                                              double *t1) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = p0;
    partials[2 * blockIdx.x + 1] = p1;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double v0 = 0.0, v1 = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    v0 = v0 + __ldcg(partials + 2 * b);
    v1 = v1 + __ldcg(partials + 2 * b + 1);
  }
  v0 = block_sum<BLOCK>(v0);
  v1 = block_sum<BLOCK>(v1);
  if (threadIdx.x == 0) {
    *t0 = v0;
    *t1 = v1;
    *counter = 0u;
  }
  return true;
}

// Streaming loads/stores that do not linger in the caches.
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(double2 *p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float4 *p, float4 v) { __stcs(p, v); }

}  // namespace bs
