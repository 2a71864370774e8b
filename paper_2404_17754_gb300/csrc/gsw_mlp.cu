// Learned initial guess for the per-step CG solve: a per-node MLP that maps
// the backward differences of the last four displacement increments (each
// scaled by its RMS) and the node's layer properties to a correction of the
// step's base guess (the Newmark predictor, or the polynomial extrapolation).
//
//   x (16)  = [D_0 / s_0, D_1 / s_1, D_2 / s_2, D_3 / s_3] ++ [Vs/1000, Vp/3000, rho/2000, h/0.05],
//             D_k = sum_j (-1)^j C(k, j) du_{s-1-j}, s_k = RMS(D_k)
//   h1 = relu(x W1 + b1) (64), h2 = relu(h1 W2 + b2) (64), o = h2 W3 + b3 (3)
//   du0 = base + sigma_e * o, sigma_e = RMS of the previous step's correction
//
// Inference runs on the tensor cores: BF16 operands, FP32 accumulation, with
// mma.m16n8k16; the accumulator fragment of one layer is exactly the operand
// fragment of the next (after bias, ReLU and BF16 rounding), so a warp carries
// 16 nodes through all three layers in registers.  Training (on the solutions
// of the first steps) runs on the tensor cores too: forward, back-propagated
// errors and weight gradients as BF16 products with FP32 accumulation, then
// Adam on FP32 master weights.
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
// The forward weights as BF16 B fragments (layer 1: 8 n-tiles; layer 2: 4
// k-tiles x 8 n-tiles; layer 3: 4 k-tiles, N padded 3 -> 8) and the FP32
// biases (64 + 64 + 8), written by threads tid0, tid0 + stride, ...
__device__ void build_fwd_frags(const float* __restrict__ theta, uint32_t* frag, float* bias, int tid0, int stride) {
  for (int tid = tid0; tid < 32 * 32; tid += stride) {
    const int lane = tid % 32, g = lane / 4, t = lane % 4;
    if (tid < 8 * 32) {  // layer 1: K = 16, N = 64
      const int n = 8 * (tid / 32) + g;
      auto W = [&](int k) { return theta[kW1 + k * 64 + n]; };
      frag[kF1 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
      frag[kF1 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
    }
    {  // layer 2: K = 64 (4 k-tiles), N = 64
      const int kt = tid / 256, nt = (tid / 32) % 8;
      const int n = 8 * nt + g, k0 = 16 * kt;
      auto W = [&](int k) { return theta[kW2 + (k0 + k) * 64 + n]; };
      frag[kF2 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
      frag[kF2 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
    }
    if (tid < 4 * 32) {  // layer 3: K = 64, N = 3 padded to 8
      const int k0 = 16 * (tid / 32);
      auto W = [&](int k) { return g < 3 ? theta[kW3 + (k0 + k) * 3 + g] : 0.f; };
      frag[kF3 + 2 * tid] = pack_bf16(W(2 * t), W(2 * t + 1));
      frag[kF3 + 2 * tid + 1] = pack_bf16(W(2 * t + 8), W(2 * t + 9));
    }
    if (tid < 136) {
      float b = 0.f;
      if (tid < 64)
        b = theta[kB1 + tid];
      else if (tid < 128)
        b = theta[kB2 + tid - 64];
      else if (tid < 131)
        b = theta[kB3 + tid - 128];
      bias[tid] = b;
    }
  }
}

__global__ void mlp_pack_kernel(const float* __restrict__ theta, uint32_t* packed) {
  build_fwd_frags(theta, packed, reinterpret_cast<float*>(packed) + kBias, blockIdx.x * blockDim.x + threadIdx.x,
                  gridDim.x * blockDim.x);
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

// sigma_k = RMS over all DOF of the backward difference D_k (1 if zero).
__global__ void mlp_sigma_kernel(int64_t N, const double* __restrict__ hist, double* partials, MlpScalars* ms) {
  double sq[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t n3 = 3 * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) sq[k] = fma(hist[k * n3 + i], hist[k * n3 + i], sq[k]);
  double out[4];
  if (last_block_reduce<4>(sq, partials, &ms->counter, out) && threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double sg = sqrt(out[k] / (double)n3);
      ms->sigma[k] = sg > 0.0 ? sg : 1.0;
    }
  }
}

// RMS of du - base (the correction the network should have made to the base
// guess of the step just converged): the output scale of the next step's
// correction, far smaller than the increment itself.
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
    ms->sigma_e = sg > 0.0 ? sg : ms->sigma[0];
  }
}
void launch_mlp_sigma_e(int64_t N, const double* du, const double* base, double* partials, MlpScalars* ms,
                        cudaStream_t s) {
  mlp_sigma_e_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(N, du, base, partials, ms);
}

__device__ __forceinline__ float node_feature(const double* __restrict__ hist, const float* __restrict__ nodef,
                                              int64_t N, int64_t n, int f, const float (&inv_sigma)[4]) {
  if (f < 12) {
    const int k = f / 3, c = f % 3;
    return (float)hist[((int64_t)k * N + n) * 3 + c] * inv_sigma[k];
  }
  return nodef[4 * n + (f - 12)];
}

// Tensor-core inference over all nodes: x <- base + sigma_e * MLP(features).
__global__ void __launch_bounds__(128) mlp_infer_kernel(int64_t N, const double* __restrict__ hist,
                                                        const float* __restrict__ nodef,
                                                        const uint32_t* __restrict__ packed,
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
  const double sigma_e = ms ? ms->sigma_e : 1.0;
  float inv_sigma[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_sigma[k] = ms ? (float)(1.0 / ms->sigma[k]) : 1.f;
  const int64_t n_tiles = (N + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < n_tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t base = tile * 16;
    // features of the tile's 16 nodes: lanes 0..15 one node each (xin: explicit features)
    if (lane < 16) {
      const int64_t n = base + lane;
      for (int f = 0; f < 16; ++f) {
        float val = 0.f;
        if (n < N) val = xin ? xin[n * 16 + f] : node_feature(hist, nodef, N, n, f, inv_sigma);
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
          // the network corrects the step's base guess (predictor or extrapolation)
          const int64_t k = 3 * n + c;
          x[k] = x_base[k] + sigma_e * (double)o;
        }
      }
    }
  }
}

// Diagnostics: the features and the base guess that the next step's inference
// would use, for the listed nodes only (X [n][16], base_out [n][3]).
__global__ void mlp_inputs_kernel(int n, const int32_t* __restrict__ nodes, int64_t N, const double* __restrict__ hist,
                                  const float* __restrict__ nodef, const MlpScalars* ms,
                                  const double* __restrict__ base, float* X, double* base_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t nd = nodes[i];
  float inv_sigma[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_sigma[k] = (float)(1.0 / ms->sigma[k]);
  for (int f = 0; f < 16; ++f) X[(int64_t)i * 16 + f] = node_feature(hist, nodef, N, nd, f, inv_sigma);
  for (int c = 0; c < 3; ++c) base_out[(int64_t)i * 3 + c] = base[3 * nd + c];
}

// The Newmark predictor dt v + dt^2/2 a (the base guess at guess order 0).
__global__ void predictor_kernel(int64_t n3, const double* __restrict__ v, const double* __restrict__ a, double dt,
                                 double* __restrict__ x) {
  const double h = 0.5 * dt * dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(dt, v[i], h * a[i]);
}

// Training samples: node = hash(seed, step, iter, i) mod N; features as in
// inference (FP32), target = (du_s - base_s) / sigma_e (sigma_e: the RMS of
// this step's correction du_s - base_s).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__global__ void mlp_sample_kernel(int64_t N, int B, uint32_t seed, int step, int iter,
                                  const double* __restrict__ hist, const float* __restrict__ nodef,
                                  const double* __restrict__ du, const double* __restrict__ base,
                                  const MlpScalars* ms, float* X, float* Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const uint32_t h = mix32(seed ^ mix32((uint32_t)step * 0x9E3779B9U ^ mix32((uint32_t)iter * 0x85EBCA6BU ^ (uint32_t)i)));
  const int64_t n = (int64_t)(h % (uint32_t)N);
  float inv_sigma[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_sigma[k] = (float)(1.0 / ms->sigma[k]);
  const double inv_e = 1.0 / ms->sigma_e;
  for (int f = 0; f < 16; ++f) X[(int64_t)i * 16 + f] = node_feature(hist, nodef, N, n, f, inv_sigma);
  for (int c = 0; c < 3; ++c) {
    const int64_t k = 3 * n + c;
    Y[(int64_t)i * 3 + c] = (float)((du[k] - base[k]) * inv_e);
  }
}

// Training on the tensor cores: forward and backward of the mean squared
// error over the batch with BF16 operands and FP32 accumulation
// (mma.m16n8k16), gradients added to grad (FP32), loss to *loss.  A CTA of
// four warps takes chunks of 64 samples (16 per warp):
//   forward   the inference chain (the C fragment of one layer, after bias,
//             ReLU and BF16 rounding, is the A fragment of the next);
//   backward  d3 = 2 (o - y) / B; dz2 = (d3 W3^T) * [z2 > 0];
//             dz1 = (dz2 W2^T) * [z1 > 0] (each rounded to BF16 before its
//             product, the ReLU masks taken from the forward fragments);
//   gradients dW1 = X^T dz1, dW2 = h1^T dz2, dW3 = h2^T d3: products over the
//             chunk's 64 samples (K), from the activations and errors staged
//             in shared memory, accumulated in registers over the CTA's
//             chunks; bias gradients are FP32 column sums.
constexpr int kTcChunk = 64;
constexpr int kTcThreads = 128;
// dynamic shared memory layout (32-bit words)
constexpr int kSmWf = 0;                          // forward fragments [kFrag]
constexpr int kSmBias = kSmWf + kFrag;            // FP32 biases [136]
constexpr int kSmW3t = kSmBias + 136;             // W3^T B fragments [8 n-tiles][32][2]
constexpr int kSmW2t = kSmW3t + 8 * 32 * 2;       // W2^T B fragments [4 k-tiles][8 n-tiles][32][2]
constexpr int kSmX = kSmW2t + 32 * 32 * 2;        // X [64][16] bf16
constexpr int kSmH1 = kSmX + kTcChunk * 16 / 2;   // h1 [64][64] bf16
constexpr int kSmH2 = kSmH1 + kTcChunk * 64 / 2;  // h2 [64][64] bf16
constexpr int kSmZ1 = kSmH2 + kTcChunk * 64 / 2;  // dz1 [64][64] bf16
constexpr int kSmZ2 = kSmZ1 + kTcChunk * 64 / 2;  // dz2 [64][64] bf16
constexpr int kSmD3 = kSmZ2 + kTcChunk * 64 / 2;  // d3 [64][8] bf16
constexpr int kSmDb = kSmD3 + kTcChunk * 8 / 2;   // bias gradients db1 [64], db2 [64], db3 [8] (FP32)
constexpr int kSmLoss = kSmDb + 136;              // loss partial (FP32)
constexpr int kSmWords = kSmLoss + 4;

__device__ __forceinline__ uint32_t pack_raw(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// A fragment of act^T (m = unit, k = sample) from act [sample][S] (bf16).
template <int S>
__device__ __forceinline__ void frag_at(const uint16_t* act, int m0, int k0, int g, int t, uint32_t (&a)[4]) {
  const uint16_t* c0 = act + m0 + g;
  a[0] = pack_raw(c0[(k0 + 2 * t) * S], c0[(k0 + 2 * t + 1) * S]);
  a[1] = pack_raw(c0[(k0 + 2 * t) * S + 8], c0[(k0 + 2 * t + 1) * S + 8]);
  a[2] = pack_raw(c0[(k0 + 2 * t + 8) * S], c0[(k0 + 2 * t + 9) * S]);
  a[3] = pack_raw(c0[(k0 + 2 * t + 8) * S + 8], c0[(k0 + 2 * t + 9) * S + 8]);
}
// B fragment of err (k = sample, n = unit) from err [sample][S] (bf16).
template <int S>
__device__ __forceinline__ void frag_b(const uint16_t* err, int k0, int n0, int g, int t, uint32_t& b0, uint32_t& b1) {
  const uint16_t* c0 = err + n0 + g;
  b0 = pack_raw(c0[(k0 + 2 * t) * S], c0[(k0 + 2 * t + 1) * S]);
  b1 = pack_raw(c0[(k0 + 2 * t + 8) * S], c0[(k0 + 2 * t + 9) * S]);
}
// Column sums over the warp's 16 rows of a C fragment pair (rows g, g + 8),
// added to acc[col] in shared memory by lanes 0..3.
__device__ __forceinline__ void colsum_add(float v0, float v1, float* acc, int col, int lane) {
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane < 4) {
    atomicAdd(acc + col, v0);
    atomicAdd(acc + col + 1, v1);
  }
}

__global__ void __launch_bounds__(kTcThreads) mlp_train_tc_kernel(int B, const float* __restrict__ X,
                                                                   const float* __restrict__ Y,
                                                                   const float* __restrict__ theta, float* grad,
                                                                   double* loss) {
  extern __shared__ uint32_t smw[];
  uint32_t* wf = smw + kSmWf;
  float* bias = reinterpret_cast<float*>(smw + kSmBias);
  uint32_t* w3t = smw + kSmW3t;
  uint32_t* w2t = smw + kSmW2t;
  uint16_t* xs = reinterpret_cast<uint16_t*>(smw + kSmX);
  uint16_t* h1s = reinterpret_cast<uint16_t*>(smw + kSmH1);
  uint16_t* h2s = reinterpret_cast<uint16_t*>(smw + kSmH2);
  uint16_t* z1s = reinterpret_cast<uint16_t*>(smw + kSmZ1);
  uint16_t* z2s = reinterpret_cast<uint16_t*>(smw + kSmZ2);
  uint16_t* d3s = reinterpret_cast<uint16_t*>(smw + kSmD3);
  float* db = reinterpret_cast<float*>(smw + kSmDb);
  float* lsum = reinterpret_cast<float*>(smw + kSmLoss);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  build_fwd_frags(theta, wf, bias, tid, kTcThreads);
  // backward operands: W3^T (k = output padded to 16, n = hidden) and W2^T (k = j, n = i)
  for (int q = tid; q < 8 * 32; q += kTcThreads) {
    const int nt = q / 32, l = q % 32, gg = l / 4, tt = l % 4, n = 8 * nt + gg;
    auto W3 = [&](int c) { return c < 3 ? theta[kW3 + n * 3 + c] : 0.f; };
    w3t[2 * q] = pack_bf16(W3(2 * tt), W3(2 * tt + 1));
    w3t[2 * q + 1] = 0u;
  }
  for (int q = tid; q < 32 * 32; q += kTcThreads) {
    const int kt = q / 256, nt = (q / 32) % 8, l = q % 32, gg = l / 4, tt = l % 4;
    const int n = 8 * nt + gg, k0 = 16 * kt;
    auto W2 = [&](int k) { return theta[kW2 + n * 64 + k0 + k]; };
    w2t[2 * q] = pack_bf16(W2(2 * tt), W2(2 * tt + 1));
    w2t[2 * q + 1] = pack_bf16(W2(2 * tt + 8), W2(2 * tt + 9));
  }
  for (int q = tid; q < 140; q += kTcThreads) (q < 136 ? db[q] : lsum[q - 136]) = 0.f;
  float acc2[8][4], acc1[2][4], acc3[4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc2[i][q] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) acc1[0][q] = acc1[1][q] = acc3[q] = 0.f;
  float lpart = 0.f;
  const float inv2B = 2.f / (float)B;
  __syncthreads();
  const int n_chunks = (B + kTcChunk - 1) / kTcChunk;
  for (int ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int base = ch * kTcChunk + 16 * warp;  // first sample of this warp
    const int r0 = 16 * warp;                    // its first row in the staging arrays
    if (lane < 16) {
      const int64_t gi = base + lane;
#pragma unroll
      for (int f = 0; f < 16; f += 2) {
        const float a = gi < B ? X[gi * 16 + f] : 0.f, b = gi < B ? X[gi * 16 + f + 1] : 0.f;
        *reinterpret_cast<uint32_t*>(xs + (r0 + lane) * 16 + f) = pack_bf16(a, b);
      }
    }
    __syncwarp();
    uint32_t A[4];
    {
      const uint16_t* x0 = xs + (r0 + g) * 16;
      const uint16_t* x1 = xs + (r0 + g + 8) * 16;
      A[0] = *reinterpret_cast<const uint32_t*>(x0 + 2 * t);
      A[1] = *reinterpret_cast<const uint32_t*>(x1 + 2 * t);
      A[2] = *reinterpret_cast<const uint32_t*>(x0 + 2 * t + 8);
      A[3] = *reinterpret_cast<const uint32_t*>(x1 + 2 * t + 8);
    }
    // ---- forward ----
    uint32_t mask1 = 0u, mask2 = 0u;
    uint32_t A2[4][4];
    {
      float C1[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
        C1[nt][0] = b0;
        C1[nt][1] = b1;
        C1[nt][2] = b0;
        C1[nt][3] = b1;
        mma_bf16(C1[nt], A, wf[kF1 + 2 * (nt * 32 + lane)], wf[kF1 + 2 * (nt * 32 + lane) + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) mask1 |= (C1[nt][q] > 0.f ? 1u : 0u) << (4 * nt + q);
        const uint32_t lo = pack_bf16(fmaxf(C1[nt][0], 0.f), fmaxf(C1[nt][1], 0.f));
        const uint32_t hi = pack_bf16(fmaxf(C1[nt][2], 0.f), fmaxf(C1[nt][3], 0.f));
        *reinterpret_cast<uint32_t*>(h1s + (r0 + g) * 64 + 8 * nt + 2 * t) = lo;
        *reinterpret_cast<uint32_t*>(h1s + (r0 + g + 8) * 64 + 8 * nt + 2 * t) = hi;
        A2[nt >> 1][(nt & 1) * 2] = lo;
        A2[nt >> 1][(nt & 1) * 2 + 1] = hi;
      }
    }
    uint32_t A3[4][4];
    {
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
#pragma unroll
        for (int q = 0; q < 4; ++q) mask2 |= (C2[nt][q] > 0.f ? 1u : 0u) << (4 * nt + q);
        const uint32_t lo = pack_bf16(fmaxf(C2[nt][0], 0.f), fmaxf(C2[nt][1], 0.f));
        const uint32_t hi = pack_bf16(fmaxf(C2[nt][2], 0.f), fmaxf(C2[nt][3], 0.f));
        *reinterpret_cast<uint32_t*>(h2s + (r0 + g) * 64 + 8 * nt + 2 * t) = lo;
        *reinterpret_cast<uint32_t*>(h2s + (r0 + g + 8) * 64 + 8 * nt + 2 * t) = hi;
        A3[nt >> 1][(nt & 1) * 2] = lo;
        A3[nt >> 1][(nt & 1) * 2 + 1] = hi;
      }
    }
    float C3[4];
    {
      const float b0 = bias[128 + 2 * t], b1 = bias[128 + 2 * t + 1];
      C3[0] = b0;
      C3[1] = b1;
      C3[2] = b0;
      C3[3] = b1;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
        mma_bf16(C3, A3[kt], wf[kF3 + 2 * (kt * 32 + lane)], wf[kF3 + 2 * (kt * 32 + lane) + 1]);
    }
    // ---- output error d3 = 2 (o - y) / B (rows g, g + 8; columns 2t, 2t + 1) ----
    float d3[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + 8 * (q >> 1), col = 2 * t + (q & 1);
      const int64_t gi = base + row;
      float e = 0.f;
      if (col < 3 && gi < B) {
        const float diff = C3[q] - Y[gi * 3 + col];
        lpart = fmaf(diff, diff, lpart);
        e = diff * inv2B;
      }
      d3[q] = e;
    }
    {
      const uint32_t lo = pack_bf16(d3[0], d3[1]), hi = pack_bf16(d3[2], d3[3]);
      *reinterpret_cast<uint32_t*>(d3s + (r0 + g) * 8 + 2 * t) = lo;
      *reinterpret_cast<uint32_t*>(d3s + (r0 + g + 8) * 8 + 2 * t) = hi;
      colsum_add(d3[0] + d3[2], d3[1] + d3[3], db + 128, 2 * t, lane);
      // ---- dz2 = (d3 W3^T) * [z2 > 0] ----
      const uint32_t Ad[4] = {lo, hi, 0u, 0u};
      uint32_t A4[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float C[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(C, Ad, w3t[2 * (nt * 32 + lane)], 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) C[q] = ((mask2 >> (4 * nt + q)) & 1u) ? C[q] : 0.f;
        colsum_add(C[0] + C[2], C[1] + C[3], db + 64, 8 * nt + 2 * t, lane);
        const uint32_t zlo = pack_bf16(C[0], C[1]), zhi = pack_bf16(C[2], C[3]);
        *reinterpret_cast<uint32_t*>(z2s + (r0 + g) * 64 + 8 * nt + 2 * t) = zlo;
        *reinterpret_cast<uint32_t*>(z2s + (r0 + g + 8) * 64 + 8 * nt + 2 * t) = zhi;
        A4[nt >> 1][(nt & 1) * 2] = zlo;
        A4[nt >> 1][(nt & 1) * 2 + 1] = zhi;
      }
      // ---- dz1 = (dz2 W2^T) * [z1 > 0] ----
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float C[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
          const int fi = 2 * ((kt * 8 + nt) * 32 + lane);
          mma_bf16(C, A4[kt], w2t[fi], w2t[fi + 1]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) C[q] = ((mask1 >> (4 * nt + q)) & 1u) ? C[q] : 0.f;
        colsum_add(C[0] + C[2], C[1] + C[3], db, 8 * nt + 2 * t, lane);
        *reinterpret_cast<uint32_t*>(z1s + (r0 + g) * 64 + 8 * nt + 2 * t) = pack_bf16(C[0], C[1]);
        *reinterpret_cast<uint32_t*>(z1s + (r0 + g + 8) * 64 + 8 * nt + 2 * t) = pack_bf16(C[2], C[3]);
      }
    }
    __syncthreads();
    // ---- weight gradients over the chunk's 64 samples ----
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const int k0 = 16 * kt;
      uint32_t a[4], b0, b1;
      frag_at<64>(h1s, 16 * warp, k0, g, t, a);  // dW2 rows 16w.. (hidden in)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        frag_b<64>(z2s, k0, 8 * nt, g, t, b0, b1);
        mma_bf16(acc2[nt], a, b0, b1);
      }
      frag_at<16>(xs, 0, k0, g, t, a);  // dW1 (16 features), columns 16w..16w+15
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        frag_b<64>(z1s, k0, 8 * (2 * warp + q), g, t, b0, b1);
        mma_bf16(acc1[q], a, b0, b1);
      }
      frag_at<64>(h2s, 16 * warp, k0, g, t, a);  // dW3 rows 16w.. (hidden)
      frag_b<8>(d3s, k0, 0, g, t, b0, b1);
      mma_bf16(acc3, a, b0, b1);
    }
    __syncthreads();
  }
  // ---- add the CTA's gradients and loss ----
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = g + 8 * (q >> 1), cc = 2 * t + (q & 1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) atomicAdd(grad + kW2 + (16 * warp + rr) * 64 + 8 * nt + cc, acc2[nt][q]);
#pragma unroll
    for (int h = 0; h < 2; ++h) atomicAdd(grad + kW1 + rr * 64 + 8 * (2 * warp + h) + cc, acc1[h][q]);
    if (cc < 3) atomicAdd(grad + kW3 + (16 * warp + rr) * 3 + cc, acc3[q]);
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) lpart += __shfl_xor_sync(0xffffffffu, lpart, o);
  if (lane == 0) atomicAdd(lsum, lpart);
  __syncthreads();
  for (int q = tid; q < 131; q += kTcThreads) {
    const int p = q < 64 ? kB1 + q : (q < 128 ? kB2 + q - 64 : kB3 + q - 128);
    atomicAdd(grad + p, db[q]);
  }
  if (tid == 0) atomicAdd(loss, (double)lsum[0] / (double)B);
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

// Push a converged increment into the difference history: D_0' = du and
// D_k' = D_{k-1}' - D_{k-1} (the backward differences of the last four
// increments; before four pushes the missing increments count as zero).
__global__ void hist_push_kernel(int64_t N, const double* __restrict__ du, double* hist, const CgScalars* cg,
                                 const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  const bool zero = cg->zero_rhs != 0;
  const int64_t n3 = 3 * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double d0 = zero ? 0.0 : du[i];
    const double o0 = hist[i], o1 = hist[n3 + i], o2 = hist[2 * n3 + i];
    const double d1 = d0 - o0, d2 = d1 - o1, d3 = d2 - o2;
    hist[i] = d0;
    hist[n3 + i] = d1;
    hist[2 * n3 + i] = d2;
    hist[3 * n3 + i] = d3;
  }
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
void launch_mlp_sigma(int64_t N, const double* hist, double* partials, MlpScalars* ms, cudaStream_t s) {
  // four sums per CTA: the partials buffer holds 4 x (kMaxNodeBlocks / 2)
  int g = node_blocks(3 * N);
  if (g > kMaxNodeBlocks / 2) g = kMaxNodeBlocks / 2;
  mlp_sigma_kernel<<<g, kNodeThreads, 0, s>>>(N, hist, partials, ms);
}
void launch_mlp_infer(int64_t N, const double* hist, const float* nodef, const uint32_t* packed, const MlpScalars* ms,
                      double* x, const float* xin, float* yout, cudaStream_t s, const double* x_base) {
  const int64_t tiles = (N + 15) / 16;
  int64_t blocks = (tiles + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  mlp_infer_kernel<<<(unsigned)blocks, 128, 0, s>>>(N, hist, nodef, packed, ms, x, xin, yout, x_base);
}
void launch_mlp_sample(int64_t N, int B, uint32_t seed, int step, int iter, const double* hist, const float* nodef,
                       const double* du, const double* base, const MlpScalars* ms, float* X, float* Y,
                       cudaStream_t s) {
  mlp_sample_kernel<<<(B + 255) / 256, 256, 0, s>>>(N, B, seed, step, iter, hist, nodef, du, base, ms, X, Y);
}
int launch_mlp_fwdbwd(int B, const float* X, const float* Y, const float* theta, float* grad, double* loss,
                      cudaStream_t s) {
  static bool attr = false;
  const int smem = kSmWords * 4;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return 1;
    attr = true;
  }
  const int chunks = (B + kTcChunk - 1) / kTcChunk;
  const int grid = chunks < 152 * 2 ? chunks : 152 * 2;
  mlp_train_tc_kernel<<<grid, kTcThreads, smem, s>>>(B, X, Y, theta, grad, loss);
  return 0;
}
void launch_mlp_adam(float* theta, float* grad, float* m, float* v, int t, float lr, cudaStream_t s) {
  mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, grad, m, v, t, lr);
}
void launch_hist_push(int64_t N, const double* du, double* hist, const CgScalars* cg, cudaStream_t s,
                      const StepState* ss) {
  hist_push_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(N, du, hist, cg, ss);
}
void launch_predictor(int64_t N, const double* v, const double* a, double dt, double* x, cudaStream_t s) {
  predictor_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, v, a, dt, x);
}
void launch_mlp_inputs(int n, const int32_t* nodes, int64_t N, const double* hist, const float* nodef,
                       const MlpScalars* ms, const double* base, float* X, double* base_out, cudaStream_t s) {
  mlp_inputs_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, nodes, N, hist, nodef, ms, base, X, base_out);
}
int mlp_packed_words() { return kPacked; }

}  // namespace gsw
