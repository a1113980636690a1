// Shared device/host helpers of the CASPT2 library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/caspt2.h"

#define CASPT2_CUDA_TRY(expr)                                  \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return CASPT2_ECUDA;                \
  } while (0)

namespace caspt2 {

constexpr int kMaxStates = 16;   // n <= 16 reference states

// Number of kernels this thread has launched through the library (read by the
// C ABI around a solve to report launches per solve).
inline long& launch_counter() {
  static thread_local long count = 0;
  return count;
}

// Block-wide FP64 sum in a fixed order (warp shuffle tree, then warp 0 over the
// per-warp partials).  Every thread must call it; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* smem32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) smem32[warp] = v;
  __syncthreads();
  v = (threadIdx.x < nwarp) ? smem32[threadIdx.x] : 0.0;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// 1/d for the energy denominators: Newton's iteration x <- x + x (1 - d x) from the
// hardware's approximate double reciprocal (rcp.approx.ftz.f64, about 20 correct bits);
// two steps take the seed past double precision (error within an ulp or so).  d must be
// a normal number.
__device__ __forceinline__ double recip(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  return fma(x, e, x);
}

__device__ __forceinline__ double block_min(double v, double* smem32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) smem32[warp] = v;
  __syncthreads();
  v = (threadIdx.x < nwarp) ? smem32[threadIdx.x] : 1e300;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  return v;
}

}  // namespace caspt2
