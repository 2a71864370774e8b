// Block and grid reductions used by the CG kernels.
#pragma once
#include <cuda_runtime.h>

namespace gsw {

// ------------------------------------------------------------------------------
// Reductions: warp shuffle, block tree, and a deterministic last-block finish.
// ------------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) v = warp_sum(v);
  return v;
}

// Each block contributes NQ partial sums; the last block to arrive sums all
// partials in block order (so the result does not depend on scheduling) and
// returns true in every thread of that block, with the totals in out[] of
// thread 0.
template <int NQ>
__device__ __forceinline__ bool last_block_reduce(const double (&vals)[NQ], double* partials,
                                  unsigned int* counter, double (&out)[NQ]) {
  __shared__ double sh[32];
  __shared__ int am_last;
  const unsigned int G = gridDim.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = block_sum(vals[q], sh);
    if (threadIdx.x == 0) partials[q * G + blockIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    am_last = (prev == G - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double acc = 0.0;
    for (unsigned int i = threadIdx.x; i < G; i += blockDim.x)
      acc += ((volatile double*)partials)[q * G + i];
    out[q] = block_sum(acc, sh);
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

}  // namespace gsw
