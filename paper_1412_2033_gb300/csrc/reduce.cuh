// Deterministic block reductions (fixed shuffle tree, fixed block order).
#pragma once

#include <cuda_runtime.h>

namespace ghb {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one double per thread; the result is valid in thread 0.  `scratch`
// holds 32 doubles of shared memory.  Contains barriers: call from all threads.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (lane < nw) ? scratch[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

}  // namespace ghb
