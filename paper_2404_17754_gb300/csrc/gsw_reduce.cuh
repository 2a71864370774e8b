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
  // Eight independent L2 loads in flight per thread (a single dependent chain
  // of ~G / blockDim.x loads would leave the GPU idle for tens of
  // microseconds at the end of a large grid); the fixed accumulator pattern
  // keeps the order of summation independent of scheduling.
  const unsigned int B = blockDim.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double* pq = partials + (size_t)q * G;
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.0;
    unsigned int i = threadIdx.x;
    for (; i + 7 * B < G; i += 8 * B) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldcg(pq + i + j * B);
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] += v[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i + j * B < G) a[j] += __ldcg(pq + i + j * B);
    const double acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    out[q] = block_sum(acc, sh);
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ------------------------------------------------------------------------------
// FP32 versions for the reduced-precision kernels: the FP64 pipe of this GPU
// retires a warp-wide double add in tens of cycles, so the inner solve keeps
// its partial sums, partials and final sums in FP32.
// ------------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float block_sum_f(float v, float* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_f(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.f;
  if (warp == 0) v = warp_sum_f(v);
  return v;
}

// As last_block_reduce, in FP32 (partials: NQ * gridDim.x floats).
template <int NQ>
__device__ __forceinline__ bool last_block_reduce_f(const float (&vals)[NQ], float* partials,
                                                    unsigned int* counter, float (&out)[NQ]) {
  __shared__ float shf[32];
  __shared__ int am_last_f;
  const unsigned int G = gridDim.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float s = block_sum_f(vals[q], shf);
    if (threadIdx.x == 0) partials[q * G + blockIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    am_last_f = (prev == G - 1);
  }
  __syncthreads();
  if (!am_last_f) return false;
  __threadfence();
  const unsigned int B = blockDim.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float* pq = partials + (size_t)q * G;
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.f;
    unsigned int i = threadIdx.x;
    for (; i + 7 * B < G; i += 8 * B) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldcg(pq + i + j * B);
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] += v[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i + j * B < G) a[j] += __ldcg(pq + i + j * B);
    const float acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    out[q] = block_sum_f(acc, shf);
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

}  // namespace gsw
