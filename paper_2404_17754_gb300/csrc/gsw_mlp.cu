// Learned initial guess for the per-step CG solve: a per-node MLP that maps
// the last four displacement increments (scaled by the RMS of the latest one)
// and the node's layer properties to a correction of the Newmark predictor.
//
//   x (16)  = [du_{s-1}, du_{s-2}, du_{s-3}, du_{s-4}] / sigma ++ [Vs/1000, Vp/3000, rho/2000, h/0.05]
//   h1 = relu(x W1 + b1) (64), h2 = relu(h1 W2 + b2) (64), o = h2 W3 + b3 (3)
//   du0 = dt v + dt^2/2 a + sigma * o
//
// Inference runs on the tensor cores: BF16 operands, FP32 accumulation, with
// mma.m16n8k16; the accumulator fragment of one layer is exactly the operand
// fragment of the next (after bias, ReLU and BF16 rounding), so a warp carries
// 16 nodes through all three layers in registers.  Training (on the solutions
// of the first steps) runs in FP32: a fused forward/backward kernel per batch
// chunk with the weight gradients reduced in shared memory, then Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsw_internal.cuh"
#include "gsw_reduce.cuh"

namespace gsw {

// parameter offsets in the packed vector (row-major W[in][out])
constexpr int kW1 = 0, kB1 = 1024, kW2 = 1088, kB2 = 5184, kW3 = 5248, kB3 = 5440;
static_assert(kB3 + 3 == kMlpParams, "parameter count");
// packed BF16 operand fragments: layer 1 (8 n-tiles), layer 2 (4 k-tiles x 8 n-tiles),
// layer 3 (4 k-tiles, N padded 3 -> 8); 2 registers per lane per fragment
constexpr int kF1 = 0, kF2 = kF1 + 8 * 32 * 2, kF3 = kF2 + 32 * 32 * 2, kFrag = kF3 + 4 * 32 * 2;
constexpr int kBias = kFrag;  // FP32 biases (64 + 64 + 8) follow the fragments
constexpr int kPacked = kBias + 136;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Operand fragment of B (K x N, "col") for lane (g = lane/4, t = lane%4):
// reg0 = (B[2t][g], B[2t+1][g]), reg1 = (B[2t+8][g], B[2t+9][g]).
__global__ void mlp_pack_kernel(const float* __restrict__ theta, uint32_t* packed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  // layer 1: K = 16, N = 64
  if (tid < 8 * 32) {
    const int nt = tid / 32, lane = tid % 32, g = lane / 4, t = lane % 4;
    const int n = 8 * nt + g;
    auto W = [&](int k) { return theta[kW1 + k * 64 + n]; };
    packed[kF1 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
    packed[kF1 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
  }
  // layer 2: K = 64 (4 k-tiles), N = 64
  if (tid < 32 * 32) {
    const int kt = tid / 256, nt = (tid / 32) % 8, lane = tid % 32, g = lane / 4, t = lane % 4;
    const int n = 8 * nt + g, k0 = 16 * kt;
    auto W = [&](int k) { return theta[kW2 + (k0 + k) * 64 + n]; };
    packed[kF2 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
    packed[kF2 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
  }
  // layer 3: K = 64, N = 3 padded to 8
  if (tid < 4 * 32) {
    const int kt = tid / 32, lane = tid % 32, g = lane / 4, t = lane % 4;
    const int k0 = 16 * kt;
    auto W = [&](int k) { return g < 3 ? theta[kW3 + (k0 + k) * 3 + g] : 0.f; };
    packed[kF3 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
    packed[kF3 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
  }
  if (tid < 136) {
    float b = 0.f;
    if (tid < 64)
      b = theta[kB1 + tid];
    else if (tid < 128)
      b = theta[kB2 + tid - 64];
    else if (tid < 131)
      b = theta[kB3 + tid - 128];
    reinterpret_cast<float*>(packed)[kBias + tid] = b;
  }
}

// Per-node layer features (Vs/1000, Vp/3000, rho/2000, h/0.05) of the lowest
// material index among the elements touching the node.
__global__ void node_material_kernel(ModelView m, int32_t* node_mat) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const int mt = m.emat[e];
  for (int k = 0; k < 10; ++k) atomicMin(node_mat + m.conn[k * m.E + e], mt);
}
__global__ void node_features_kernel(int64_t N, const int32_t* node_mat, const MatCoef* mat, int n_mat,
                                     float* nodef) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int mt = node_mat[n];
  const MatCoef c = mat[(mt >= 0 && mt < n_mat) ? mt : 0];  // a node in no element takes layer 0
  nodef[4 * n] = (float)(c.Vs / 1000.0);
  nodef[4 * n + 1] = (float)(c.Vp / 3000.0);
  nodef[4 * n + 2] = (float)(c.rho / 2000.0);
  nodef[4 * n + 3] = (float)(c.h / 0.05);
}

// sigma = RMS over all DOF of the latest increment (history slot `head`).
__global__ void mlp_sigma_kernel(int64_t N, const float* __restrict__ hist, int head, double* partials,
                                 MlpScalars* ms) {
  const float* h = hist + (int64_t)head * 3 * N;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)h[i] * h[i];
  double vals[1] = {s}, out[1];
  if (last_block_reduce<1>(vals, partials, &ms->counter, out) && threadIdx.x == 0) {
    const double sg = sqrt(out[0] / (3.0 * N));
    ms->sigma = sg > 0.0 ? sg : 1.0;
  }
}

// RMS of du - base (the correction the network should have made to the
// extrapolated guess of the step just converged): the output scale of the
// correction to an extrapolated base, far smaller than the increment itself.
__global__ void mlp_sigma_e_kernel(int64_t N, const double* __restrict__ du, const double* __restrict__ base,
                                   double* partials, MlpScalars* ms) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    const double e = du[i] - base[i];
    s = fma(e, e, s);
  }
  double vals[1] = {s}, out[1];
  if (last_block_reduce<1>(vals, partials, &ms->counter, out) && threadIdx.x == 0) {
    const double sg = sqrt(out[0] / (3.0 * N));
    ms->sigma_e = sg > 0.0 ? sg : ms->sigma;
  }
}
void launch_mlp_sigma_e(int64_t N, const double* du, const double* base, double* partials, MlpScalars* ms,
                        cudaStream_t s) {
  mlp_sigma_e_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(N, du, base, partials, ms);
}

__device__ __forceinline__ float node_feature(const float* __restrict__ hist, const float* __restrict__ nodef,
                                              int64_t N, int head, int64_t n, int f, float inv_sigma) {
  if (f < 12) {
    const int k = f / 3, c = f % 3;
    const int slot = (head - k + 4) & 3;
    return hist[((int64_t)slot * N + n) * 3 + c] * inv_sigma;
  }
  return nodef[4 * n + (f - 12)];
}

// Tensor-core inference over all nodes: x <- dt v + dt^2/2 a + sigma * MLP(features).
__global__ void __launch_bounds__(128) mlp_infer_kernel(int64_t N, const float* __restrict__ hist, int head,
                                                        const float* __restrict__ nodef,
                                                        const double* __restrict__ v, const double* __restrict__ a,
                                                        double dt, const uint32_t* __restrict__ packed,
                                                        const MlpScalars* ms, double* __restrict__ x,
                                                        const float* __restrict__ xin, float* __restrict__ yout,
                                                        const double* __restrict__ x_base) {
  __shared__ uint32_t wf[kFrag];
  __shared__ float bias[136];
  __shared__ __nv_bfloat16 feat[4][16][16];
  for (int i = threadIdx.x; i < kFrag; i += blockDim.x) wf[i] = packed[i];
  for (int i = threadIdx.x; i < 136; i += blockDim.x) bias[i] = reinterpret_cast<const float*>(packed)[kBias + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const double sigma = ms ? ms->sigma : 1.0;
  const double sigma_e = ms ? ms->sigma_e : 1.0;
  const float inv_sigma = (float)(1.0 / sigma);
  const int64_t n_tiles = (N + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < n_tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t base = tile * 16;
    // features of the tile's 16 nodes: lanes 0..15 one node each (xin: explicit features)
    if (lane < 16) {
      const int64_t n = base + lane;
      for (int f = 0; f < 16; ++f) {
        float val = 0.f;
        if (n < N) val = xin ? xin[n * 16 + f] : node_feature(hist, nodef, N, head, n, f, inv_sigma);
        feat[warp][lane][f] = __float2bfloat16_rn(val);
      }
    }
    __syncwarp();
    uint32_t A[4];
    {
      const __nv_bfloat16* r0 = &feat[warp][g][0];
      const __nv_bfloat16* r1 = &feat[warp][g + 8][0];
      A[0] = *reinterpret_cast<const uint32_t*>(r0 + 2 * t);
      A[1] = *reinterpret_cast<const uint32_t*>(r1 + 2 * t);
      A[2] = *reinterpret_cast<const uint32_t*>(r0 + 2 * t + 8);
      A[3] = *reinterpret_cast<const uint32_t*>(r1 + 2 * t + 8);
    }
    __syncwarp();
    // layer 1
    float C1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
      C1[nt][0] = b0;
      C1[nt][1] = b1;
      C1[nt][2] = b0;
      C1[nt][3] = b1;
      mma_bf16(C1[nt], A, wf[kF1 + 2 * (nt * 32 + lane)], wf[kF1 + 2 * (nt * 32 + lane) + 1]);
    }
    uint32_t A2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A2[kt][0] = pack_bf16(fmaxf(C1[2 * kt][0], 0.f), fmaxf(C1[2 * kt][1], 0.f));
      A2[kt][1] = pack_bf16(fmaxf(C1[2 * kt][2], 0.f), fmaxf(C1[2 * kt][3], 0.f));
      A2[kt][2] = pack_bf16(fmaxf(C1[2 * kt + 1][0], 0.f), fmaxf(C1[2 * kt + 1][1], 0.f));
      A2[kt][3] = pack_bf16(fmaxf(C1[2 * kt + 1][2], 0.f), fmaxf(C1[2 * kt + 1][3], 0.f));
    }
    // layer 2
    float C2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = bias[64 + 8 * nt + 2 * t], b1 = bias[64 + 8 * nt + 2 * t + 1];
      C2[nt][0] = b0;
      C2[nt][1] = b1;
      C2[nt][2] = b0;
      C2[nt][3] = b1;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const int fi = kF2 + 2 * ((kt * 8 + nt) * 32 + lane);
        mma_bf16(C2[nt], A2[kt], wf[fi], wf[fi + 1]);
      }
    }
    uint32_t A3[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A3[kt][0] = pack_bf16(fmaxf(C2[2 * kt][0], 0.f), fmaxf(C2[2 * kt][1], 0.f));
      A3[kt][1] = pack_bf16(fmaxf(C2[2 * kt][2], 0.f), fmaxf(C2[2 * kt][3], 0.f));
      A3[kt][2] = pack_bf16(fmaxf(C2[2 * kt + 1][0], 0.f), fmaxf(C2[2 * kt + 1][1], 0.f));
      A3[kt][3] = pack_bf16(fmaxf(C2[2 * kt + 1][2], 0.f), fmaxf(C2[2 * kt + 1][3], 0.f));
    }
    // layer 3 (columns 0..2 are the output)
    float C3[4];
    {
      const float b0 = bias[128 + 2 * t], b1 = bias[128 + 2 * t + 1];
      C3[0] = b0;
      C3[1] = b1;
      C3[2] = b0;
      C3[3] = b1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma_bf16(C3, A3[kt], wf[kF3 + 2 * (kt * 32 + lane)], wf[kF3 + 2 * (kt * 32 + lane) + 1]);
    // lane (g, t) holds rows g, g+8 and columns 2t, 2t+1
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t n = base + g + 8 * half;
      if (n >= N) continue;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int c = 2 * t + cc;
        if (c >= 3) continue;
        const float o = C3[2 * half + cc];
        if (yout) {
          yout[n * 3 + c] = o;
        } else {
          const int64_t k = 3 * n + c;
          // the network corrects a base guess: the extrapolated one when given,
          // else the Newmark predictor
          const double b0 = x_base ? x_base[k] : fma(dt, v[k], 0.5 * dt * dt * a[k]);
          x[k] = b0 + (x_base ? sigma_e : sigma) * (double)o;
        }
      }
    }
  }
}

// Diagnostics: the features and the base guess that the next step's inference
// would use, for the listed nodes only (X [n][16], base [n][3]).
__global__ void mlp_inputs_kernel(int n, const int32_t* __restrict__ nodes, int64_t N, const float* __restrict__ hist,
                                  int head, const float* __restrict__ nodef, const MlpScalars* ms,
                                  const double* __restrict__ v, const double* __restrict__ a, double dt,
                                  const double* __restrict__ x_base, float* X, double* base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t nd = nodes[i];
  const float inv_sigma = (float)(1.0 / ms->sigma);
  for (int f = 0; f < 16; ++f) X[(int64_t)i * 16 + f] = node_feature(hist, nodef, N, head, nd, f, inv_sigma);
  for (int c = 0; c < 3; ++c) {
    const int64_t k = 3 * nd + c;
    base[(int64_t)i * 3 + c] = x_base ? x_base[k] : fma(dt, v[k], 0.5 * dt * dt * a[k]);
  }
}

// Training samples: node = hash(seed, step, iter, i) mod N; features as in
// inference (FP32), target = (du_s - base guess) / sigma (base: the extrapolated
// guess when given, else the Newmark predictor).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__global__ void mlp_sample_kernel(int64_t N, int B, uint32_t seed, int step, int iter,
                                  const float* __restrict__ hist, int head, const float* __restrict__ nodef,
                                  const double* __restrict__ du, const double* __restrict__ v,
                                  const double* __restrict__ a, double dt, const MlpScalars* ms, float* X,
                                  float* Y, const double* __restrict__ x_base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const uint32_t h = mix32(seed ^ mix32((uint32_t)step * 0x9E3779B9U ^ mix32((uint32_t)iter * 0x85EBCA6BU ^ (uint32_t)i)));
  const int64_t n = (int64_t)(h % (uint32_t)N);
  const double sigma = ms->sigma;
  const double out_scale = x_base ? ms->sigma_e : sigma;
  const float inv_sigma = (float)(1.0 / sigma);
  for (int f = 0; f < 16; ++f) X[(int64_t)i * 16 + f] = node_feature(hist, nodef, N, head, n, f, inv_sigma);
  for (int c = 0; c < 3; ++c) {
    const int64_t k = 3 * n + c;
    const double b0 = x_base ? x_base[k] : fma(dt, v[k], 0.5 * dt * dt * a[k]);
    Y[(int64_t)i * 3 + c] = (float)((du[k] - b0) / out_scale);
  }
}

// Forward + backward of a chunk of kMlpChunk samples (one per thread) in FP32,
// weight gradients reduced over the chunk in shared memory and added to grad.
constexpr int kMlpChunk = 64;
__global__ void __launch_bounds__(kMlpChunk) mlp_fwdbwd_kernel(int B, const float* __restrict__ X,
                                                               const float* __restrict__ Y,
                                                               const float* __restrict__ theta, float* grad,
                                                               double* loss) {
  extern __shared__ float sm[];
  float* W = sm;                              // kMlpParams
  float* xs = W + kMlpParams;                 // [chunk][16]
  float* z1 = xs + kMlpChunk * 16;            // [chunk][64] pre-activation, later delta1
  float* z2 = z1 + kMlpChunk * 64;            // [chunk][64] pre-activation, later delta2
  float* h1 = z2 + kMlpChunk * 64;            // [chunk][64]
  float* h2 = h1 + kMlpChunk * 64;            // [chunk][64]
  float* d3 = h2 + kMlpChunk * 64;            // [chunk][3]
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) W[i] = theta[i];
  const int s = threadIdx.x;
  const int64_t gi = (int64_t)blockIdx.x * kMlpChunk + s;
  const bool ok = gi < B;
  for (int f = 0; f < 16; ++f) xs[s * 16 + f] = ok ? X[gi * 16 + f] : 0.f;
  __syncthreads();
  // forward
  for (int j = 0; j < 64; ++j) {
    float acc = W[kB1 + j];
    for (int f = 0; f < 16; ++f) acc = fmaf(xs[s * 16 + f], W[kW1 + f * 64 + j], acc);
    z1[s * 64 + j] = acc;
    h1[s * 64 + j] = fmaxf(acc, 0.f);
  }
  for (int j = 0; j < 64; ++j) {
    float acc = W[kB2 + j];
    for (int k = 0; k < 64; ++k) acc = fmaf(h1[s * 64 + k], W[kW2 + k * 64 + j], acc);
    z2[s * 64 + j] = acc;
    h2[s * 64 + j] = fmaxf(acc, 0.f);
  }
  float sq = 0.f;
  for (int c = 0; c < 3; ++c) {
    float acc = W[kB3 + c];
    for (int k = 0; k < 64; ++k) acc = fmaf(h2[s * 64 + k], W[kW3 + k * 3 + c], acc);
    const float diff = ok ? acc - Y[gi * 3 + c] : 0.f;
    sq = fmaf(diff, diff, sq);
    d3[s * 3 + c] = 2.f * diff / (float)B;
  }
  // backward: delta2 (in z2), delta1 (in z1)
  for (int k = 0; k < 64; ++k) {
    float acc = 0.f;
    for (int c = 0; c < 3; ++c) acc = fmaf(d3[s * 3 + c], W[kW3 + k * 3 + c], acc);
    z2[s * 64 + k] = z2[s * 64 + k] > 0.f ? acc : 0.f;
  }
  for (int k = 0; k < 64; ++k) {
    float acc = 0.f;
    for (int j = 0; j < 64; ++j) acc = fmaf(z2[s * 64 + j], W[kW2 + k * 64 + j], acc);
    z1[s * 64 + k] = z1[s * 64 + k] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // weight gradients over the chunk: each thread owns parameters p = tid + k * chunk
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) {
    float acc = 0.f;
    if (p < kB1) {
      const int f = p / 64, j = p % 64;
      for (int q = 0; q < kMlpChunk; ++q) acc = fmaf(xs[q * 16 + f], z1[q * 64 + j], acc);
    } else if (p < kW2) {
      const int j = p - kB1;
      for (int q = 0; q < kMlpChunk; ++q) acc += z1[q * 64 + j];
    } else if (p < kB2) {
      const int k = (p - kW2) / 64, j = (p - kW2) % 64;
      for (int q = 0; q < kMlpChunk; ++q) acc = fmaf(h1[q * 64 + k], z2[q * 64 + j], acc);
    } else if (p < kW3) {
      const int j = p - kB2;
      for (int q = 0; q < kMlpChunk; ++q) acc += z2[q * 64 + j];
    } else if (p < kB3) {
      const int k = (p - kW3) / 3, c = (p - kW3) % 3;
      for (int q = 0; q < kMlpChunk; ++q) acc = fmaf(h2[q * 64 + k], d3[q * 3 + c], acc);
    } else {
      const int c = p - kB3;
      for (int q = 0; q < kMlpChunk; ++q) acc += d3[q * 3 + c];
    }
    atomicAdd(grad + p, acc);
  }
  // loss (mean square over the batch)
  __shared__ double shl[32];
  double l = block_sum((double)sq, shl);
  if (threadIdx.x == 0) atomicAdd(loss, l / (double)B);
}

__global__ void mlp_adam_kernel(float* theta, float* grad, float* m, float* v, int t, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
  theta[i] -= lr * mh / (sqrtf(vh) + eps);
  grad[i] = 0.f;
}

__global__ void hist_push_kernel(int64_t N, const double* __restrict__ du, float* hist, int slot,
                                 const CgScalars* cg, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  const bool zero = cg->zero_rhs != 0;
  float* h = hist + (int64_t)slot * 3 * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x)
    h[i] = zero ? 0.f : (float)du[i];
}

// ------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------

void launch_mlp_pack(const float* theta, uint32_t* packed, cudaStream_t s) {
  mlp_pack_kernel<<<(32 * 32 + 127) / 128, 128, 0, s>>>(theta, packed);
}
void launch_node_features(const ModelView& m, int n_mat, int32_t* node_mat, float* nodef, cudaStream_t s) {
  cudaMemsetAsync(node_mat, 0x7f, sizeof(int32_t) * m.N, s);
  node_material_kernel<<<(unsigned)((m.E + 255) / 256), 256, 0, s>>>(m, node_mat);
  node_features_kernel<<<(unsigned)((m.N + 255) / 256), 256, 0, s>>>(m.N, node_mat, m.mat, n_mat, nodef);
}
void launch_mlp_sigma(int64_t N, const float* hist, int head, double* partials, MlpScalars* ms, cudaStream_t s) {
  mlp_sigma_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(N, hist, head, partials, ms);
}
void launch_mlp_infer(int64_t N, const float* hist, int head, const float* nodef, const double* v, const double* a,
                      double dt, const uint32_t* packed, const MlpScalars* ms, double* x, const float* xin,
                      float* yout, cudaStream_t s, const double* x_base) {
  const int64_t tiles = (N + 15) / 16;
  int64_t blocks = (tiles + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  mlp_infer_kernel<<<(unsigned)blocks, 128, 0, s>>>(N, hist, head, nodef, v, a, dt, packed, ms, x, xin, yout, x_base);
}
void launch_mlp_sample(int64_t N, int B, uint32_t seed, int step, int iter, const float* hist, int head,
                       const float* nodef, const double* du, const double* v, const double* a, double dt,
                       const MlpScalars* ms, float* X, float* Y, cudaStream_t s, const double* x_base) {
  mlp_sample_kernel<<<(B + 255) / 256, 256, 0, s>>>(N, B, seed, step, iter, hist, head, nodef, du, v, a, dt, ms, X, Y,
                                                    x_base);
}
size_t mlp_fwdbwd_smem() { return sizeof(float) * (kMlpParams + kMlpChunk * (16 + 4 * 64 + 3)); }
int launch_mlp_fwdbwd(int B, const float* X, const float* Y, const float* theta, float* grad, double* loss,
                      cudaStream_t s) {
  static bool attr = false;
  const size_t smem = mlp_fwdbwd_smem();
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_fwdbwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 1;
    attr = true;
  }
  mlp_fwdbwd_kernel<<<(B + kMlpChunk - 1) / kMlpChunk, kMlpChunk, smem, s>>>(B, X, Y, theta, grad, loss);
  return 0;
}
void launch_mlp_adam(float* theta, float* grad, float* m, float* v, int t, float lr, cudaStream_t s) {
  mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, grad, m, v, t, lr);
}
void launch_hist_push(int64_t N, const double* du, float* hist, int slot, const CgScalars* cg, cudaStream_t s,
                      const StepState* ss) {
  hist_push_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(N, du, hist, slot, cg, ss);
}
void launch_mlp_inputs(int n, const int32_t* nodes, int64_t N, const float* hist, int head, const float* nodef,
                       const MlpScalars* ms, const double* v, const double* a, double dt, const double* x_base, float* X,
                       double* base, cudaStream_t s) {
  mlp_inputs_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, nodes, N, hist, head, nodef, ms, v, a, dt, x_base, X, base);
}
int mlp_packed_words() { return kPacked; }

}  // namespace gsw
