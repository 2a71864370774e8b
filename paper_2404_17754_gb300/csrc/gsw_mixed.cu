// Mixed-precision solve: flexible CG in FP64 with a reduced-precision inner
// PCG as the variable preconditioner (Section 3, computational-cost
// paragraph: conjugate gradients with variable preconditioning).
//
// Outer iteration (FP64 residual, dot products and update):
//   r = b - A x0;  z = P(r);  p = z
//   repeat: q = A p; alpha = r.z / p.q; x += alpha p; r -= alpha q
//           z' = P(r); beta = z'.(r' - r) / (r.z) = -alpha z'.q / (r.z); p = z' + beta p
// (Polak-Ribiere beta keeps CG's short recurrence valid when P varies.)
//
// Inner solve P(r): a fixed number of block-Jacobi PCG iterations on A in
// FP32 arithmetic, with the search direction stored in FP32 or FP16 and the
// barycentric gradients in FP32 or FP16 (volumes FP32).  The right-hand side
// is the outer residual scaled so that the preconditioned residual D^-1 s,
// which seeds the stored search direction, has entries of order one (FP16
// keeps 3 significant digits between 6e-5 and 6.5e4).  The element-by-element product assembles each block of
// elements in shared memory over the block's unique nodes (local numbering
// built on the GPU at setup) and writes every node once per block: a plain
// store for nodes no other block touches, an atomic add otherwise.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsw_dword.cuh"
#include "gsw_ebe.cuh"
#include "gsw_internal.cuh"
#include "gsw_reduce.cuh"

namespace gsw {

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half from_f<__half>(float x) { return __float2half_rn(x); }

// Search-direction storage is padded to 4 entries per node so that one
// 8-byte (FP16) or 16-byte (FP32) load fetches a node.
__device__ __forceinline__ void load3(const float* p, float& a, float& b, float& c) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x;
  b = v.y;
  c = v.z;
}
__device__ __forceinline__ void load3(const __half* p, float& a, float& b, float& c) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __half2 h0 = *reinterpret_cast<const __half2*>(&v.x);
  const __half2 h1 = *reinterpret_cast<const __half2*>(&v.y);
  a = __low2float(h0);
  b = __high2float(h0);
  c = __low2float(h1);
}

__device__ __forceinline__ void store4(float* p, const float (&q)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(q[0], q[1], q[2], q[3]);
}
__device__ __forceinline__ void store4(__half* p, const __half (&q)[4]) {
  const __half2 a = __halves2half2(q[0], q[1]), b = __halves2half2(q[2], q[3]);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
}

// Operator element order inside a block: warp w, lane l processes element
// 6 l + w of the block.  With the 6 Kuhn tetrahedra of each cell stored
// consecutively, a warp then holds congruent tetrahedra of 32 different cells,
// so the 32 lanes of one shared-memory atomic never target the same node.
__host__ __device__ __forceinline__ int lo_elem_of_pos(int p) { return 6 * (p % 32) + p / 32; }

// Packed per-element record of the reduced-precision operator.
struct LoRecH {   // 48 bytes: FP16 gradients
  uint16_t lc[10];
  __half g[9];
  uint16_t pad0;
  float vol;
  uint16_t mat;
  uint16_t pad1;
};
struct LoRecF {   // 64 bytes: FP32 gradients
  uint16_t lc[10];
  float g[9];
  float vol;
  uint16_t mat;
  uint16_t pad1;
};
template <typename SG> struct LoRec;
template <> struct LoRec<__half> { typedef LoRecH type; static constexpr int words = 3; };
template <> struct LoRec<float> { typedef LoRecF type; static constexpr int words = 4; };
static_assert(sizeof(LoRecH) == 48 && sizeof(LoRecF) == 64, "record layout");

constexpr int kSortN = 2048;  // >= 10 * kLoBlock, power of two

// ------------------------------------------------------------------------------
// Element blocks: unique nodes per block via an in-shared-memory bitonic sort
// ------------------------------------------------------------------------------

__device__ void load_sorted_block(const ModelView& m, int b, int* keys) {
  const int64_t e0 = (int64_t)b * kLoBlock;
  const int ne = (int)((m.E - e0) < kLoBlock ? (m.E - e0) : kLoBlock);
  for (int i = threadIdx.x; i < kSortN; i += blockDim.x) {
    int v = 0x7fffffff;
    if (i < 10 * ne) {
      const int k = i / ne, el = i % ne;
      v = m.conn[(int64_t)k * m.E + e0 + el];
    }
    keys[i] = v;
  }
  __syncthreads();
  for (int size = 2; size <= kSortN; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < kSortN / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const int a = keys[lo], c = keys[hi];
        if ((a > c) == up) {
          keys[lo] = c;
          keys[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void block_count_kernel(ModelView m, int32_t* counts) {
  __shared__ int keys[kSortN];
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  load_sorted_block(m, blockIdx.x, keys);
  int c = 0;
  for (int i = threadIdx.x; i < kSortN; i += blockDim.x)
    if (keys[i] != 0x7fffffff && (i == 0 || keys[i] != keys[i - 1])) ++c;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = cnt;
}

__global__ void block_fill_kernel(ModelView m, BlockView bv, int32_t* nodes, uint16_t* lconn,
                                  int32_t* refcount, const int32_t* counts) {
  __shared__ int keys[kSortN];
  __shared__ int flag[kSortN];
  const int b = blockIdx.x;
  load_sorted_block(m, b, keys);
  for (int i = threadIdx.x; i < kSortN; i += blockDim.x)
    flag[i] = (keys[i] != 0x7fffffff && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
  __syncthreads();
  // inclusive scan of flags (Hillis-Steele, in place with a temporary)
  for (int off = 1; off < kSortN; off <<= 1) {
    int v[kSortN / 256];  // blockDim.x == 256
#pragma unroll
    for (int j = 0; j < kSortN / 256; ++j) {
      const int i = threadIdx.x + j * 256;
      v[j] = (i < kSortN && i >= off) ? flag[i - off] : 0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortN / 256; ++j) {
      const int i = threadIdx.x + j * 256;
      if (i < kSortN) flag[i] += v[j];
    }
    __syncthreads();
  }
  const int base = bv.ptr[b];
  const int nu = counts[b];  // unique nodes; entries nu .. ptr[b+1]-base-1 are padding
  for (int i = nu + threadIdx.x; i < bv.ptr[b + 1] - base; i += blockDim.x) nodes[base + i] = (int32_t)m.N;
  for (int i = threadIdx.x; i < kSortN; i += blockDim.x) {
    const bool first = keys[i] != 0x7fffffff && (i == 0 || keys[i] != keys[i - 1]);
    if (first) {
      const int slot = flag[i] - 1;
      nodes[base + slot] = keys[i];
      atomicAdd(refcount + keys[i], 1);
    }
  }
  __syncthreads();
  // compact the unique keys to the front of `keys` (reuse flag as storage)
  for (int i = threadIdx.x; i < nu; i += blockDim.x) flag[i] = nodes[base + i];
  __syncthreads();
  // local indices in the operator's element order: position p = w * 32 + lane
  // of block b holds element b * kLoBlock + 6 * lane + w
  for (int i = threadIdx.x; i < 10 * kLoBlock; i += blockDim.x) {
    const int k = i / kLoBlock, pl = i % kLoBlock;
    const int64_t e = (int64_t)b * kLoBlock + lo_elem_of_pos(pl);
    int lo = 0;
    if (e < m.E) {
      const int g = m.conn[(int64_t)k * m.E + e];
      int hi = nu - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (flag[mid] < g)
          lo = mid + 1;
        else
          hi = mid;
      }
    }
    lconn[(int64_t)k * ((int64_t)bv.n_blk * kLoBlock) + (int64_t)b * kLoBlock + pl] = (uint16_t)lo;
  }
}

__global__ void face_refcount_kernel(ModelView m, int32_t* refcount) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= m.F) return;
  if (m.fgeo[5 * m.F + f] < 0.5) return;  // free surface faces add nothing
  for (int k = 0; k < 6; ++k) atomicAdd(refcount + m.fnode[k * m.F + f], 2);
}

__global__ void block_mark_kernel(int total, int32_t* nodes, const int32_t* refcount) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int g = nodes[i];
  if (refcount[g] == 1) nodes[i] = (int32_t)((uint32_t)g | 0x80000000u);  // the dummy node's count stays 0
}

// Element records in operator order (invalid positions of the last block get
// zero volume, so they contribute nothing) and FP32 face data.
template <typename SG>
__global__ void lo_convert_kernel(ModelView m, int n_blk, const uint16_t* __restrict__ lconn,
                                  typename LoRec<SG>::type* rec, float* fgeo32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t P = (int64_t)n_blk * kLoBlock;
  if (t < P) {
    const int64_t b = t / kLoBlock;
    const int pl = (int)(t % kLoBlock);
    const int64_t e = b * kLoBlock + lo_elem_of_pos(pl);
    typename LoRec<SG>::type r;
    for (int k = 0; k < 10; ++k) r.lc[k] = lconn[(int64_t)k * P + t];
    const bool ok = e < m.E;
    for (int k = 0; k < 9; ++k) r.g[k] = from_f<SG>(ok ? (float)m.geo[k * m.E + e] : 0.f);
    r.vol = ok ? (float)m.geo[9 * m.E + e] : 0.f;
    r.mat = ok ? (uint16_t)m.emat[e] : 0;
    r.pad1 = 0;
    // block b's records are stored as RW planes of kLoBlock 16-byte words, so
    // that consecutive threads read consecutive words
    constexpr int RW = LoRec<SG>::words;
    union {
      typename LoRec<SG>::type r;
      uint4 v[RW];
    } u;
    u.r = r;
    uint4* out = reinterpret_cast<uint4*>(rec) + b * RW * kLoBlock + pl;
#pragma unroll
    for (int q = 0; q < RW; ++q) out[q * kLoBlock] = u.v[q];
  }
  if (t < 6 * m.F) fgeo32[t] = (float)m.fgeo[t];
}

// Mean diagonal entry of D^-1 (sets the inner right-hand-side scale).
__global__ void dinv_mean_kernel(int64_t N, const double* __restrict__ dinv, double* partials, InnerScalars* sc) {
  double s = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    s += dinv[6 * n] + dinv[6 * n + 1] + dinv[6 * n + 2];
  double vals[1] = {s}, out[1];
  if (last_block_reduce<1>(vals, partials, &sc->counter, out) && threadIdx.x == 0) sc->dinv_mean = out[0] / (3.0 * N);
}

// D^-1 in the inner storage type, divided by its mean diagonal entry: entries
// of order one (FP16 keeps them), and the inner PCG iterates do not change
// when the preconditioner is scaled by a constant (the inner right-hand side
// is scaled to match, see inner_init_kernel).
template <typename SD>
__global__ void dinv_lo_kernel(int64_t n6, const double* __restrict__ dinv, const InnerScalars* sc,
                               SD* __restrict__ out) {
  const double dm = ((volatile const InnerScalars*)sc)->dinv_mean;
  const double inv = dm > 0.0 ? 1.0 / dm : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n6; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = from_f<SD>((float)(dinv[i] * inv));
}

// ------------------------------------------------------------------------------
// Reduced-precision element-by-element product w = A d (+ partial d . w)
// ------------------------------------------------------------------------------

// Inside a solve (outer != nullptr) the inner kernels return at entry once the
// outer iteration has converged or the current inner solve has met its
// relative tolerance.
__device__ __forceinline__ bool inner_stopped(const CgScalars* outer, const InnerScalars* sc) {
  return outer != nullptr &&
         (((volatile const CgScalars*)outer)->done || ((volatile const InnerScalars*)sc)->idone);
}

// Per-CTA partial sum of the per-thread d . A d contributions (FP32), stored
// in dw_part[blockIdx.x]; the direction update sums the partials in a fixed
// order (so the operator kernel carries no grid-wide reduction tail).
__device__ __forceinline__ void lo_store_dw(float dot, float* dw_part, InnerScalars* sc) {
  __shared__ float shd[32];
  const float s = block_sum_f(dot, shd);
  if (threadIdx.x == 0) {
    dw_part[blockIdx.x] = s;
    if (blockIdx.x == 0) sc->n_dw = gridDim.x;
  }
}

// One CTA per block of kLoBlock elements: the CTA gathers the block's unique
// nodes into shared memory, each thread applies one element (records are
// loaded as 16-byte vectors before the gather so their latency overlaps it)
// with shared-memory atomics, and the CTA writes each unique node once (a
// plain store when no other block or absorbing face touches it).  CTAs after
// the element blocks apply the absorbing faces with global atomics.
template <typename SG, typename SD, int MINB, bool FUSE = false>
__global__ void __launch_bounds__(kLoBlock, MINB) ebe_lo_kernel(LoView<SG> m, const SD* __restrict__ d,
                                                           float* __restrict__ w, double* partials,
                                                           InnerScalars* sc, const CgScalars* outer,
                                                           const SD* __restrict__ t4 = nullptr,
                                                           SD* __restrict__ dnew = nullptr) {
  if (inner_stopped(outer, sc)) return;
  typedef typename LoRec<SG>::type Rec;
  constexpr int RW = LoRec<SG>::words;
  extern __shared__ float sm[];
  __shared__ float matc[kMaxMat][3];
  if (threadIdx.x < m.n_mat) {
    const float4 c = m.matf[threadIdx.x];
    matc[threadIdx.x][0] = c.x;
    matc[threadIdx.x][1] = c.y;
    matc[threadIdx.x][2] = c.z;
  }
  float dot = 0.f;
  const int b = blockIdx.x;
  if (b < m.blk.n_blk) {
    float* xs = sm;
    float* ys = sm + 3 * m.blk.max_local;
    union {
      uint4 v[RW];
      Rec r;
    } u;
    const uint4* rp = reinterpret_cast<const uint4*>(m.rec) + (int64_t)b * kLoBlock * RW + threadIdx.x;
#pragma unroll
    for (int q = 0; q < RW; ++q) u.v[q] = __ldcs(rp + q * kLoBlock);  // streamed: read once per launch
    // node lists have the fixed stride max_local (padding names the dummy
    // node N), so no offset load precedes the index loads
    const int64_t n0 = (int64_t)b * m.blk.max_local;
    const int nn = m.blk.max_local;
    // each thread owns nodes threadIdx.x + j * kLoBlock (j < kLoNodesPerThread):
    // all index loads first, then all gathers, so their latencies overlap
    int32_t raw[kLoNodesPerThread];
#pragma unroll
    for (int j = 0; j < kLoNodesPerThread; ++j) {
      const int i = threadIdx.x + j * kLoBlock;
      raw[j] = (i < nn) ? __ldcs(m.blk.nodes + n0 + i) : 0;
    }
    float xv[kLoNodesPerThread][3];
    if (FUSE) {
      // the direction recurrence of the previous inner iteration, fused into
      // the gather: d' = t + beta d (rounded to the storage precision), written
      // to the other direction buffer (every block touching a node writes the
      // same value; the buffer read here is not written in this launch)
      const float beta = ((volatile const InnerScalars*)sc)->beta_f;
      float tv[kLoNodesPerThread][3];
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        if (i < nn) {
          const int64_t g = raw[j] & 0x7fffffff;
          load3(d + 4 * g, xv[j][0], xv[j][1], xv[j][2]);
          load3(t4 + 4 * g, tv[j][0], tv[j][1], tv[j][2]);
        }
      }
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        if (i < nn) {
          const int64_t g = raw[j] & 0x7fffffff;
          SD q[4];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            q[c] = from_f<SD>(fmaf(beta, xv[j][c], tv[j][c]));
            xv[j][c] = to_f(q[c]);
          }
          q[3] = from_f<SD>(0.f);
          store4(dnew + 4 * g, q);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        if (i < nn) load3(d + 4 * (int64_t)(raw[j] & 0x7fffffff), xv[j][0], xv[j][1], xv[j][2]);
      }
    }
#pragma unroll
    for (int j = 0; j < kLoNodesPerThread; ++j) {
      const int i = threadIdx.x + j * kLoBlock;
      if (i < nn) {
        xs[3 * i] = xv[j][0];
        xs[3 * i + 1] = xv[j][1];
        xs[3 * i + 2] = xv[j][2];
        ys[3 * i] = 0.f;
        ys[3 * i + 1] = 0.f;
        ys[3 * i + 2] = 0.f;
      }
    }
    __syncthreads();
    {
      float g[3][3];
#pragma unroll
      for (int mm = 0; mm < 3; ++mm)
#pragma unroll
        for (int i = 0; i < 3; ++i) g[mm][i] = to_f(u.r.g[3 * mm + i]);
      const float V = u.r.vol;
      const int mt = u.r.mat;
      const float lamS = matc[mt][0] * V, muS = matc[mt][1] * V, mS = matc[mt][2] * V;
      float wv[10][3], f[10][3];
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) wv[k][i] = xs[3 * u.r.lc[k] + i];
      stiffness_apply<float>(wv, g, lamS, muS, f);
      mass_apply<float>(wv, mS, f);
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          atomicAdd(ys + 3 * u.r.lc[k] + i, f[k][i]);
          dot = fmaf(wv[k][i], f[k][i], dot);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kLoNodesPerThread; ++j) {
      const int i = threadIdx.x + j * kLoBlock;
      const int64_t g = raw[j] & 0x7fffffff;
      if (i < nn && g != m.N) {  // padding entries name the dummy node N: skip them
        if (raw[j] < 0) {
          w[3 * g] = ys[3 * i];
          w[3 * g + 1] = ys[3 * i + 1];
          w[3 * g + 2] = ys[3 * i + 2];
        } else {
          atomicAdd(w + 3 * g, ys[3 * i]);
          atomicAdd(w + 3 * g + 1, ys[3 * i + 1]);
          atomicAdd(w + 3 * g + 2, ys[3 * i + 2]);
        }
      }
    }
  } else {
    // absorbing faces: (2/dt) C_abs d
    const int64_t fc = (int64_t)(b - m.blk.n_blk) * kLoBlock + threadIdx.x;
    if (fc < m.F && m.fgeo[5 * m.F + fc] > 0.5f) {
      const float sc2 = m.face_c;
      const float As = sc2 * m.fgeo[fc], Ad = sc2 * m.fgeo[m.F + fc];
      const float n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
      int64_t nd[6];
      float z[6][3], xin[6][3];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        nd[k] = m.fnode[k * m.F + fc];
        load3(d + 4 * nd[k], xin[k][0], xin[k][1], xin[k][2]);
        if (FUSE) {
          // the same fused direction the element blocks use (rounded alike)
          const float beta = ((volatile const InnerScalars*)sc)->beta_f;
          float tv[3];
          load3(t4 + 4 * nd[k], tv[0], tv[1], tv[2]);
#pragma unroll
          for (int c = 0; c < 3; ++c) xin[k][c] = to_f(from_f<SD>(fmaf(beta, xin[k][c], tv[c])));
        }
        const float dn = n[0] * xin[k][0] + n[1] * xin[k][1] + n[2] * xin[k][2];
#pragma unroll
        for (int i = 0; i < 3; ++i) z[k][i] = fmaf(As, xin[k][i], Ad * dn * n[i]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float Zv = z[0][i] + z[1][i] + z[2][i];
        const float Ze = z[3][i] + z[4][i] + z[5][i];
        float yf[6];
        yf[0] = 7.f * z[0][i] - Zv - 4.f * z[4][i];
        yf[1] = 7.f * z[1][i] - Zv - 4.f * z[5][i];
        yf[2] = 7.f * z[2][i] - Zv - 4.f * z[3][i];
        yf[3] = 16.f * (z[3][i] + Ze) - 4.f * z[2][i];
        yf[4] = 16.f * (z[4][i] + Ze) - 4.f * z[0][i];
        yf[5] = 16.f * (z[5][i] + Ze) - 4.f * z[1][i];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          atomicAdd(w + 3 * nd[k] + i, yf[k]);
          dot = fmaf(xin[k][i], yf[k], dot);
        }
      }
    }
  }
  lo_store_dw(dot, m.dw_part, sc);
}

// The same operator applied to the search directions of up to three inner
// solves at once (the three input directions of one model, advancing in
// lockstep): the element records and the block's node list are read once and
// the element geometry decoded once; each right-hand side has its own
// shared-memory gather/accumulation arrays, result, d . A d partials and
// scalars, and is skipped once its solve has stopped.
template <typename SG, typename SD, int MINB>
__global__ void __launch_bounds__(kLoBlock, MINB) ebe_lo3_kernel(LoView<SG> m, Lo3Args a) {
  // right-hand sides still running (bit r), read once: the flags change only between launches
  const unsigned act = (a.nr > 0 && !inner_stopped(a.outer[0], a.sc[0]) ? 1u : 0u) |
                       (a.nr > 1 && !inner_stopped(a.outer[1], a.sc[1]) ? 2u : 0u) |
                       (a.nr > 2 && !inner_stopped(a.outer[2], a.sc[2]) ? 4u : 0u);
  if (!act) return;
  typedef typename LoRec<SG>::type Rec;
  constexpr int RW = LoRec<SG>::words;
  extern __shared__ float sm[];
  __shared__ float matc[kMaxMat][3];
  if (threadIdx.x < m.n_mat) {
    const float4 c = m.matf[threadIdx.x];
    matc[threadIdx.x][0] = c.x;
    matc[threadIdx.x][1] = c.y;
    matc[threadIdx.x][2] = c.z;
  }
  float dot0 = 0.f, dot1 = 0.f, dot2 = 0.f;
  const int b = blockIdx.x;
  const int nn = m.blk.max_local;
  if (b < m.blk.n_blk) {
    union {
      uint4 v[RW];
      Rec r;
    } u;
    const uint4* rp = reinterpret_cast<const uint4*>(m.rec) + (int64_t)b * kLoBlock * RW + threadIdx.x;
#pragma unroll
    for (int q = 0; q < RW; ++q) u.v[q] = __ldcs(rp + q * kLoBlock);
    const int64_t n0 = (int64_t)b * nn;
    int32_t raw[kLoNodesPerThread];
#pragma unroll
    for (int j = 0; j < kLoNodesPerThread; ++j) {
      const int i = threadIdx.x + j * kLoBlock;
      raw[j] = (i < nn) ? __ldcs(m.blk.nodes + n0 + i) : 0;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!(act & (1u << r))) continue;
      const SD* d = reinterpret_cast<const SD*>(a.d[r]);
      float* xs = sm + 6 * nn * r;
      float* ys = xs + 3 * nn;
      float xv[kLoNodesPerThread][3];
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        if (i < nn) load3(d + 4 * (int64_t)(raw[j] & 0x7fffffff), xv[j][0], xv[j][1], xv[j][2]);
      }
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        if (i < nn) {
          xs[3 * i] = xv[j][0];
          xs[3 * i + 1] = xv[j][1];
          xs[3 * i + 2] = xv[j][2];
          ys[3 * i] = 0.f;
          ys[3 * i + 1] = 0.f;
          ys[3 * i + 2] = 0.f;
        }
      }
    }
    __syncthreads();
    {
      float g[3][3];
#pragma unroll
      for (int mm = 0; mm < 3; ++mm)
#pragma unroll
        for (int i = 0; i < 3; ++i) g[mm][i] = to_f(u.r.g[3 * mm + i]);
      const float V = u.r.vol;
      const int mt = u.r.mat;
      const float lamS = matc[mt][0] * V, muS = matc[mt][1] * V, mS = matc[mt][2] * V;
#pragma unroll 1
      for (int r = 0; r < 3; ++r) {
        if (!(act & (1u << r))) continue;
        const float* xs = sm + 6 * nn * r;
        float* ys = sm + 6 * nn * r + 3 * nn;
        float wv[10][3], f[10][3];
#pragma unroll
        for (int k = 0; k < 10; ++k)
#pragma unroll
          for (int i = 0; i < 3; ++i) wv[k][i] = xs[3 * u.r.lc[k] + i];
        stiffness_apply<float>(wv, g, lamS, muS, f);
        mass_apply<float>(wv, mS, f);
        float dt = 0.f;
#pragma unroll
        for (int k = 0; k < 10; ++k)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            atomicAdd(ys + 3 * u.r.lc[k] + i, f[k][i]);
            dt = fmaf(wv[k][i], f[k][i], dt);
          }
        if (r == 0)
          dot0 = dt;
        else if (r == 1)
          dot1 = dt;
        else
          dot2 = dt;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!(act & (1u << r))) continue;
      const float* ys = sm + 6 * nn * r + 3 * nn;
      float* w = a.w[r];
#pragma unroll
      for (int j = 0; j < kLoNodesPerThread; ++j) {
        const int i = threadIdx.x + j * kLoBlock;
        const int64_t g = raw[j] & 0x7fffffff;
        if (i < nn && g != m.N) {  // padding entries name the dummy node N: skip them
          if (raw[j] < 0) {
            w[3 * g] = ys[3 * i];
            w[3 * g + 1] = ys[3 * i + 1];
            w[3 * g + 2] = ys[3 * i + 2];
          } else {
            atomicAdd(w + 3 * g, ys[3 * i]);
            atomicAdd(w + 3 * g + 1, ys[3 * i + 1]);
            atomicAdd(w + 3 * g + 2, ys[3 * i + 2]);
          }
        }
      }
    }
  } else {
    // absorbing faces: (2/dt) C_abs d, per right-hand side
    const int64_t fc = (int64_t)(b - m.blk.n_blk) * kLoBlock + threadIdx.x;
    if (fc < m.F && m.fgeo[5 * m.F + fc] > 0.5f) {
      const float sc2 = m.face_c;
      const float As = sc2 * m.fgeo[fc], Ad = sc2 * m.fgeo[m.F + fc];
      const float n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
      int64_t nd[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) nd[k] = m.fnode[k * m.F + fc];
#pragma unroll 1
      for (int r = 0; r < 3; ++r) {
        if (!(act & (1u << r))) continue;
        const SD* d = reinterpret_cast<const SD*>(r == 0 ? a.d[0] : (r == 1 ? a.d[1] : a.d[2]));
        float* w = r == 0 ? a.w[0] : (r == 1 ? a.w[1] : a.w[2]);
        float z[6][3], xin[6][3];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          load3(d + 4 * nd[k], xin[k][0], xin[k][1], xin[k][2]);
          const float dn = n[0] * xin[k][0] + n[1] * xin[k][1] + n[2] * xin[k][2];
#pragma unroll
          for (int i = 0; i < 3; ++i) z[k][i] = fmaf(As, xin[k][i], Ad * dn * n[i]);
        }
        float dt = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float Zv = z[0][i] + z[1][i] + z[2][i];
          const float Ze = z[3][i] + z[4][i] + z[5][i];
          float yf[6];
          yf[0] = 7.f * z[0][i] - Zv - 4.f * z[4][i];
          yf[1] = 7.f * z[1][i] - Zv - 4.f * z[5][i];
          yf[2] = 7.f * z[2][i] - Zv - 4.f * z[3][i];
          yf[3] = 16.f * (z[3][i] + Ze) - 4.f * z[2][i];
          yf[4] = 16.f * (z[4][i] + Ze) - 4.f * z[0][i];
          yf[5] = 16.f * (z[5][i] + Ze) - 4.f * z[1][i];
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            atomicAdd(w + 3 * nd[k] + i, yf[k]);
            dt = fmaf(xin[k][i], yf[k], dt);
          }
        }
        if (r == 0)
          dot0 = dt;
        else if (r == 1)
          dot1 = dt;
        else
          dot2 = dt;
      }
    }
  }
  if (act & 1u) lo_store_dw(dot0, a.dw_part[0], a.sc[0]);
  if (act & 2u) lo_store_dw(dot1, a.dw_part[1], a.sc[1]);
  if (act & 4u) lo_store_dw(dot2, a.dw_part[2], a.sc[2]);
}

// ------------------------------------------------------------------------------
// Inner PCG vector kernels (FP32 arithmetic)
// ------------------------------------------------------------------------------

__device__ __forceinline__ void dinv_apply_f(const float* __restrict__ D, const float r[3], float z[3]) {
  z[0] = D[0] * r[0] + D[3] * r[1] + D[4] * r[2];
  z[1] = D[3] * r[0] + D[1] * r[1] + D[5] * r[2];
  z[2] = D[4] * r[0] + D[5] * r[1] + D[2] * r[2];
}

template <typename SD>
__global__ void inner_init_kernel(int64_t N, const double* __restrict__ r, const SD* __restrict__ dinv,
                                  float* __restrict__ s, float* __restrict__ y, SD* __restrict__ t,
                                  SD* __restrict__ d, float* __restrict__ w, double* partials,
                                  InnerScalars* sc, const CgScalars* cg, float rtol, double coarse_rel) {
  if (((volatile const CgScalars*)cg)->done) return;
  // the scale is computed once per block (FP64 division and square root are
  // slow on this GPU) and broadcast through shared memory
  __shared__ double scale_s;
  if (threadIdx.x == 0) {
    // s of RMS one; with D^-1 stored divided by its mean (dinv_lo_kernel), t and d are of order one
    const double rr = ((volatile const CgScalars*)cg)->rr;
    scale_s = rr > 0.0 ? sqrt(3.0 * (double)N / rr) : 1.0;
  }
  __syncthreads();
  const double scale = scale_s;
  float st = 0.f;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    float sn[3], tn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sn[i] = (float)(r[3 * n + i] * scale);
      s[3 * n + i] = sn[i];
      y[3 * n + i] = 0.f;
      w[3 * n + i] = 0.f;
    }
    float Dn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Dn[k] = to_f(dinv[6 * n + k]);
    dinv_apply_f(Dn, sn, tn);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      t[4 * n + i] = from_f<SD>(tn[i]);
      d[4 * n + i] = from_f<SD>(tn[i]);
      st = fmaf(sn[i], tn[i], st);
    }
    t[4 * n + 3] = from_f<SD>(0.f);
    d[4 * n + 3] = from_f<SD>(0.f);
  }
  float vals[1] = {st}, out[1];
  if (last_block_reduce_f<1>(vals, reinterpret_cast<float*>(partials), &sc->counter, out) && threadIdx.x == 0) {
    sc->st = out[0];
    sc->st0 = out[0];
    sc->st_f = out[0];
    sc->scale = scale;
    const volatile CgScalars* vc = cg;
    sc->coarse_on = (coarse_rel <= 0.0 || vc->rr > coarse_rel * coarse_rel * vc->bb) ? 1u : 0u;
    sc->rtol2 = rtol * rtol;
    sc->idone = (rtol > 0.f && !(out[0] > 0.f)) ? 1u : 0u;
  }
}

// Node quads: thread g owns nodes 4g .. 4g+3, whose 3-vectors (12 floats),
// D^-1 blocks (24 floats) and padded 4-entry vectors (the direction d and the
// preconditioned residual t: 16 values) are whole 16-byte words; the N mod 4
// trailing nodes go to thread N/4.
template <int K>
__device__ __forceinline__ void ldq(const float* p, float (&v)[4 * K]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float4 a = q[k];
    v[4 * k] = a.x;
    v[4 * k + 1] = a.y;
    v[4 * k + 2] = a.z;
    v[4 * k + 3] = a.w;
  }
}
template <int K>
__device__ __forceinline__ void stq(float* p, const float (&v)[4 * K]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < K; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
__device__ __forceinline__ void ld_dir(const float* p, float (&v)[16]) { ldq<4>(p, v); }
__device__ __forceinline__ void ld_dir(const __half* p, float (&v)[16]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint4 a = q[k];
    const unsigned u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __half2 x = *reinterpret_cast<const __half2*>(&u[h]);
      v[8 * k + 2 * h] = __low2float(x);
      v[8 * k + 2 * h + 1] = __high2float(x);
    }
  }
}
__device__ __forceinline__ void st_dir(float* p, const float (&v)[16]) { stq<4>(p, v); }
// the four D^-1 blocks of a node quad (24 entries)
__device__ __forceinline__ void ld_dinv(const float* p, float (&v)[24]) { ldq<6>(p, v); }
__device__ __forceinline__ void ld_dinv(const __half* p, float (&v)[24]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 a = q[k];
    const unsigned u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __half2 x = *reinterpret_cast<const __half2*>(&u[h]);
      v[8 * k + 2 * h] = __low2float(x);
      v[8 * k + 2 * h + 1] = __high2float(x);
    }
  }
}
__device__ __forceinline__ void st_dir(__half* p, const float (&v)[16]) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    unsigned u[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __half2 x = __floats2half2_rn(v[8 * k + 2 * h], v[8 * k + 2 * h + 1]);
      u[h] = *reinterpret_cast<const unsigned*>(&x);
    }
    q[k] = make_uint4(u[0], u[1], u[2], u[3]);
  }
}

// d . A d from the operator's per-CTA partials, summed by the calling CTA in
// a fixed order (the result is valid in thread 0).
__device__ __forceinline__ float sum_dw_partials(const float* __restrict__ dw_part, const InnerScalars* sc,
                                                 float* sh_red) {
  const unsigned int G = ((volatile const InnerScalars*)sc)->n_dw, B = blockDim.x;
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 0.f;
  unsigned int i = threadIdx.x;
  for (; i + 7 * B < G; i += 8 * B) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __ldcg(dw_part + i + j * B);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += v[j];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (i + j * B < G) a[j] += __ldcg(dw_part + i + j * B);
  return block_sum_f(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])), sh_red);
}

// alpha = s . t / d . A d from the operator's per-CTA partials (one CTA,
// fixed summation order).
__global__ void inner_alpha_kernel(const float* __restrict__ dw_part, InnerScalars* sc, const CgScalars* outer) {
  if (inner_stopped(outer, sc)) return;
  __shared__ float sh_red[32];
  const float dw = sum_dw_partials(dw_part, sc, sh_red);
  if (threadIdx.x == 0) {
    const double st = ((volatile InnerScalars*)sc)->st;
    sc->dw = dw;
    sc->alpha_f = (dw != 0.f) ? (float)(st / (double)dw) : 0.f;
  }
}

// y += alpha d, s -= alpha w, t = D^-1 s, w = 0, partial s . t; the last
// block forms beta and tests the relative stopping factor.  With PRO (few
// operator partials, i.e. a small model) every CTA forms alpha itself in a
// prologue and no separate alpha kernel is launched.
template <typename SD, bool PRO = false, bool COARSE = false>
__global__ void inner_update_kernel(int64_t N, float* __restrict__ y, float* __restrict__ s, SD* __restrict__ t,
                                    const SD* __restrict__ d, float* __restrict__ w, const SD* __restrict__ dinv,
                                    double* partials, InnerScalars* sc, const CgScalars* outer,
                                    const float* __restrict__ dw_part = nullptr) {
  if (inner_stopped(outer, sc)) return;
  float alpha;
  if (PRO) {
    __shared__ float sh_red[32];
    __shared__ float alpha_s;
    const float dw = sum_dw_partials(dw_part, sc, sh_red);
    if (threadIdx.x == 0) {
      const double st_old = ((volatile const InnerScalars*)sc)->st;
      alpha_s = (dw != 0.f) ? (float)(st_old / (double)dw) : 0.f;
      if (blockIdx.x == 0) {
        sc->dw = dw;
        sc->alpha_f = alpha_s;
      }
    }
    __syncthreads();
    alpha = alpha_s;
  } else {
    alpha = ((volatile const InnerScalars*)sc)->alpha_f;
  }
  float st = 0.f;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t G4 = N >> 2;
  for (int64_t g = g0; g < G4; g += (int64_t)gridDim.x * blockDim.x) {
    float yv[12], sv[12], wv[12], tv[16], dv[16], Dv[24];
    ldq<3>(y + 12 * g, yv);
    ldq<3>(s + 12 * g, sv);
    ldq<3>(w + 12 * g, wv);
    ld_dir(d + 16 * g, dv);
    ld_dinv(dinv + 24 * g, Dv);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        yv[3 * q + i] = fmaf(alpha, dv[4 * q + i], yv[3 * q + i]);
        sv[3 * q + i] = fmaf(-alpha, wv[3 * q + i], sv[3 * q + i]);
      }
      dinv_apply_f(Dv + 6 * q, sv + 3 * q, tv + 4 * q);
      tv[4 * q + 3] = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) st = fmaf(sv[3 * q + i], tv[4 * q + i], st);
    }
    const float zero[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    stq<3>(y + 12 * g, yv);
    stq<3>(s + 12 * g, sv);
    st_dir(t + 16 * g, tv);
    stq<3>(w + 12 * g, zero);
  }
  if (g0 == 0) {  // the last N mod 4 nodes
    for (int64_t n = 4 * G4; n < N; ++n) {
      float sn[3], tn[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t k = 3 * n + i;
        y[k] = fmaf(alpha, to_f(d[4 * n + i]), y[k]);
        sn[i] = fmaf(-alpha, w[k], s[k]);
        s[k] = sn[i];
        w[k] = 0.f;
      }
      float Dn[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) Dn[k] = to_f(dinv[6 * n + k]);
      dinv_apply_f(Dn, sn, tn);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        t[4 * n + i] = from_f<SD>(tn[i]);
        st = fmaf(sn[i], tn[i], st);
      }
      t[4 * n + 3] = from_f<SD>(0.f);
    }
  }
  float vals[1] = {st}, out[1];
  if (last_block_reduce_f<1>(vals, reinterpret_cast<float*>(partials), &sc->counter, out) && threadIdx.x == 0) {
    if (COARSE) {  // s . t, beta and the stopping test follow in the restriction kernel
      sc->st_f = out[0];
      sc->iters += 1ull;
      return;
    }
    const double st_old = ((volatile InnerScalars*)sc)->st;
    const double beta = (st_old != 0.0) ? out[0] / st_old : 0.0;
    sc->beta = beta;
    sc->beta_f = (float)beta;
    sc->st = out[0];
    sc->iters += 1ull;
    const float r2 = ((volatile InnerScalars*)sc)->rtol2;
    if (r2 > 0.f && (double)out[0] <= (double)r2 * ((volatile InnerScalars*)sc)->st0) sc->idone = 1u;
  }
}

// P z_c at fine node n: the mean of its two vertices' coarse values (a vertex
// node names its own vertex twice).
__device__ __forceinline__ void prolong_add(const float4* __restrict__ zc, int a, int b, float* v) {
  const float4 za = __ldg(zc + a), zb = __ldg(zc + b);
  v[0] += 0.5f * (za.x + zb.x);
  v[1] += 0.5f * (za.y + zb.y);
  v[2] += 0.5f * (za.z + zb.z);
}

// d = t + beta d (the padding entry of each node stays 0); with CO (the
// two-level preconditioner) t is the fine part D^-1 s and the coarse part
// P z_c is added on the fly: d = t + P z_c + beta d.
template <typename SD, bool CO = false>
__global__ void inner_dupdate_kernel(int64_t N, const SD* __restrict__ t, SD* __restrict__ d,
                                     const InnerScalars* sc, const CgScalars* outer,
                                     const int2* __restrict__ pair = nullptr, const float4* __restrict__ zc = nullptr) {
  if (inner_stopped(outer, sc)) return;
  const float beta = ((volatile const InnerScalars*)sc)->beta_f;
  const bool co = CO && ((volatile const InnerScalars*)sc)->coarse_on;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t G4 = N >> 2;
  for (int64_t g = g0; g < G4; g += (int64_t)gridDim.x * blockDim.x) {
    float tv[16], dv[16];
    ld_dir(t + 16 * g, tv);
    ld_dir(d + 16 * g, dv);
    if (co) {
      const int4* pp = reinterpret_cast<const int4*>(pair + 4 * g);
      const int4 p01 = __ldg(pp), p23 = __ldg(pp + 1);
      prolong_add(zc, p01.x, p01.y, tv);
      prolong_add(zc, p01.z, p01.w, tv + 4);
      prolong_add(zc, p23.x, p23.y, tv + 8);
      prolong_add(zc, p23.z, p23.w, tv + 12);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 3; ++i) dv[4 * q + i] = fmaf(beta, dv[4 * q + i], tv[4 * q + i]);
    st_dir(d + 16 * g, dv);
  }
  if (g0 == 0) {
    for (int64_t n = 4 * G4; n < N; ++n) {
      float tn[3] = {to_f(t[4 * n]), to_f(t[4 * n + 1]), to_f(t[4 * n + 2])};
      if (co) prolong_add(zc, pair[n].x, pair[n].y, tn);
#pragma unroll
      for (int i = 0; i < 3; ++i) d[4 * n + i] = from_f<SD>(fmaf(beta, to_f(d[4 * n + i]), tn[i]));
    }
  }
}

// ------------------------------------------------------------------------------
// Two-level inner preconditioner: first-order (vertex) coarse level
// ------------------------------------------------------------------------------
//
// t = D^-1 s + omega P D_c^-1 P^T s.  The update kernel forms the fine part
// (t = D^-1 s and s . D^-1 s); this kernel forms z_c = omega D_c^-1 P^T s,
// (P^T s)_v = s_v + 1/2 sum of s over the mid-edge nodes on v's edges (a
// gather over the vertex's CSR row: deterministic, no atomics), and completes
// s . t = s . D^-1 s + (P^T s) . z_c; the direction update adds P z_c.  With
// sc == nullptr it only forms z_c (diagnostics).  first: the start of an inner
// solve (s . t becomes the reference of the stopping test, beta = 0).
__device__ __forceinline__ void coarse_finish(InnerScalars* sc, float rz, int first) {
  const volatile InnerScalars* vs = sc;
  const double st = vs->st_f + (double)rz;
  const float r2 = vs->rtol2;
  if (first) {
    sc->st = st;
    sc->st0 = st;
    sc->beta = 0.0;
    sc->beta_f = 0.f;
    sc->idone = (r2 > 0.f && !(st > 0.0)) ? 1u : 0u;
  } else {
    const double st_old = vs->st;
    const double beta = (st_old != 0.0) ? st / st_old : 0.0;
    sc->beta = beta;
    sc->beta_f = (float)beta;
    sc->st = st;
    if (r2 > 0.f && st <= (double)r2 * vs->st0) sc->idone = 1u;
  }
}

constexpr int kCoarseThreads = 1024;
__global__ void __launch_bounds__(kCoarseThreads) coarse_restrict_kernel(CoarseView c, const float* __restrict__ s,
                                                                        float4* __restrict__ zc, double* partials,
                                                                        InnerScalars* sc, const CgScalars* outer,
                                                                        int first) {
  if (sc != nullptr && inner_stopped(outer, sc)) return;
  if (sc != nullptr && !((volatile const InnerScalars*)sc)->coarse_on) {
    // this inner solve runs on the fine level alone: only the scalars move on
    if (blockIdx.x == 0 && threadIdx.x == 0) coarse_finish(sc, 0.f, first);
    return;
  }
  float acc = 0.f;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < c.Nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = __ldg(c.vnode + v);
    float h[3] = {0.f, 0.f, 0.f};
    const int j1 = __ldg(c.ptr + v + 1);
    for (int j = __ldg(c.ptr + v); j < j1; ++j) {
      const int64_t mnode = __ldg(c.mid + j);
#pragma unroll
      for (int i = 0; i < 3; ++i) h[i] += s[3 * mnode + i];
    }
    float r[3], z[3], D[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = fmaf(0.5f, h[i], s[3 * n + i]);
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] = __ldg(c.dc + 6 * v + k);
    dinv_apply_f(D, r, z);
    zc[v] = make_float4(z[0], z[1], z[2], 0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) acc = fmaf(r[i], z[i], acc);
  }
  if (sc == nullptr) return;
  float vals[1] = {acc}, out[1];
  if (last_block_reduce_f<1>(vals, reinterpret_cast<float*>(partials), &sc->counter, out) && threadIdx.x == 0)
    coarse_finish(sc, out[0], first);
}

// y = scale * P z_c in FP64 (diagnostics).
__global__ void coarse_prolong_kernel(int64_t N, const int2* __restrict__ pair, const float4* __restrict__ zc,
                                      double scale, double* __restrict__ y) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pair[n];
    const float4 a = zc[p.x], b = zc[p.y];
    y[3 * n] = scale * 0.5 * ((double)a.x + (double)b.x);
    y[3 * n + 1] = scale * 0.5 * ((double)a.y + (double)b.y);
    y[3 * n + 2] = scale * 0.5 * ((double)a.z + (double)b.z);
  }
}

// omega D_c^-1 in FP32, divided by the mean diagonal entry of D^-1 like the
// fine blocks (the inner right-hand side is scaled to match).
__global__ void coarse_lo_kernel(int64_t n6, const double* __restrict__ cinv, const InnerScalars* sc, double omega,
                                 float* __restrict__ dc) {
  const double dm = ((volatile const InnerScalars*)sc)->dinv_mean;
  const double f = omega / (dm > 0.0 ? dm : 1.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n6; i += (int64_t)gridDim.x * blockDim.x)
    dc[i] = (float)(cinv[i] * f);
}

__global__ void to_f32_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// ------------------------------------------------------------------------------
// Flexible CG outer kernels (FP64)
// ------------------------------------------------------------------------------

__global__ void fcg_residual_kernel(int64_t N, const double* __restrict__ b, double* __restrict__ q,
                                    double* __restrict__ r, double* partials, CgScalars* cg) {
  if (((volatile CgScalars*)cg)->done) return;
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    q[i] = 0.0;
    rr = fma(ri, ri, rr);
  }
  double vals[1] = {rr}, out[1];
  if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->rr = out[0];
    cg->relres = sqrt(out[0] / cg->bb);
    cg->relres0 = cg->relres;
    if (!isfinite(out[0])) {
      cg->status = -5;
      cg->done = 1;
    } else if (cg->relres <= cg->tol) {
      cg->done = 1;
    }
  }
}

// The flexible CG's search direction p: FP64, or (dwp, double-word outer
// operator) stored as double-word pairs in the same 8 bytes, so that the
// operator reads it without conversion; every reader sees the same value.
__device__ __forceinline__ double ld_p(const double* __restrict__ p, int64_t i, int dwp) {
  if (dwp) {
    const float2 c = reinterpret_cast<const float2*>(p)[i];
    return to_double(dw(c.x, c.y));
  }
  return p[i];
}
__device__ __forceinline__ void st_p(double* __restrict__ p, int64_t i, double v, int dwp) {
  if (dwp) {
    const dw d = to_dw(v);
    reinterpret_cast<float2*>(p)[i] = make_float2(d.hi, d.lo);
  } else {
    p[i] = v;
  }
}

__global__ void fcg_first_kernel(int64_t N, const float* __restrict__ y, const double* __restrict__ r,
                                 double* __restrict__ z, double* __restrict__ p, double* partials, CgScalars* cg,
                                 const InnerScalars* sc, int dwp) {
  if (((volatile CgScalars*)cg)->done) return;
  const double inv = 1.0 / ((volatile const InnerScalars*)sc)->scale;
  double rz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)y[i] * inv;
    z[i] = zi;
    st_p(p, i, zi, dwp);
    rz = fma(r[i], zi, rz);
  }
  double vals[1] = {rz}, out[1];
  if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) cg->rz = out[0];
}

__global__ void fcg_update_kernel(int64_t N, double* __restrict__ x, double* __restrict__ r,
                                  const double* __restrict__ p, const double* __restrict__ q, double* partials,
                                  CgScalars* cg, int dwp) {
  if (((volatile CgScalars*)cg)->done) return;
  const double alpha = ((volatile CgScalars*)cg)->rz / ((volatile CgScalars*)cg)->pq;
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, ld_p(p, i, dwp), x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double vals[1] = {rr}, out[1];
  if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->iter += 1;
    cg->alpha = alpha;
    cg->rr = out[0];
    cg->relres = sqrt(out[0] / cg->bb);
    if (!isfinite(out[0]) || !isfinite(alpha)) {
      cg->status = -5;
      cg->done = 1;
    } else if (cg->relres <= cg->tol) {
      cg->done = 1;
    } else if (cg->iter >= cg->max_iter) {
      cg->status = -4;
      cg->done = 1;
    }
  }
}

__global__ void fcg_zbeta_kernel(int64_t N, const float* __restrict__ y, const double* __restrict__ r,
                                 const double* __restrict__ q, double* __restrict__ z, double* partials,
                                 CgScalars* cg, const InnerScalars* sc) {
  if (((volatile CgScalars*)cg)->done) return;
  const double inv = 1.0 / ((volatile const InnerScalars*)sc)->scale;
  double zq = 0.0, rz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)y[i] * inv;
    z[i] = zi;
    zq = fma(zi, q[i], zq);
    rz = fma(r[i], zi, rz);
  }
  double vals[2] = {zq, rz}, out[2];
  if (last_block_reduce<2>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->beta = -cg->alpha * out[0] / cg->rz;
    cg->rz = out[1];
    if (!isfinite(cg->beta) || !isfinite(out[1])) {
      cg->status = -5;
      cg->done = 1;
    }
  }
}

__global__ void fcg_pupdate_kernel(int64_t N, const double* __restrict__ z, double* __restrict__ p,
                                   double* __restrict__ q, const CgScalars* cg, int dwp) {
  if (((volatile const CgScalars*)cg)->done) return;
  const double beta = ((volatile const CgScalars*)cg)->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    st_p(p, i, fma(beta, ld_p(p, i, dwp), z[i]), dwp);
    q[i] = 0.0;
  }
}

// ------------------------------------------------------------------------------
// Device-driven step bracket (batched, graph-captured stepping)
// ------------------------------------------------------------------------------

__global__ void step_begin_kernel(StepState* ss, CgScalars* cg) {
  const int active = (ss->step < ss->n_steps) && (ss->step < ss->stop_at) && (ss->failed == 0) &&
                     (ss->needs_host == 0);
  ss->active = active;
  ss->commit = 0;
  cg->iter = 0;
  cg->done = active ? 0 : 1;
  cg->status = 0;
  cg->zero_rhs = 0;
  cg->relres = 0.0;
  cg->tol = ss->tol;
  cg->max_iter = ss->max_iter;
}

// After the fixed outer-iteration budget: commit a converged step, record a
// failure (non-finite value, or the outer-iteration cap), or hand a step that
// needs more outer iterations than the budget to the host.
__global__ void step_end_kernel(StepState* ss, const CgScalars* cg) {
  if (!ss->active) return;
  if (cg->status != 0) {
    ss->failed = cg->status;
    ss->fail_step = ss->step;
  } else if (!cg->done) {
    ss->needs_host = 1;
  } else {
    ss->commit = 1;
    ss->iters_last = cg->iter;
    if (cg->iter > ss->iters_max) ss->iters_max = cg->iter;
    ss->iters_total += cg->iter;
    ss->inner_total += (long long)cg->iter * ss->inner_iters;
    ss->relres_last = cg->relres;
  }
}

__global__ void step_advance_kernel(StepState* ss) {
  if (ss->commit) ss->step += 1;
}

template <typename SD>
__global__ void to_lo_kernel(int64_t n, const double* __restrict__ x, SD* __restrict__ d, float* __restrict__ w) {
  for (int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; nd < n / 3; nd += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      d[4 * nd + i] = from_f<SD>((float)x[3 * nd + i]);
      w[3 * nd + i] = 0.f;
    }
    d[4 * nd + 3] = from_f<SD>(0.f);
  }
}
__global__ void from_f32_kernel(int64_t n, const float* __restrict__ w, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)w[i];
}

// ------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------

void launch_step_begin(StepState* ss, CgScalars* cg, cudaStream_t s) { step_begin_kernel<<<1, 1, 0, s>>>(ss, cg); }
void launch_step_end(StepState* ss, const CgScalars* cg, cudaStream_t s) { step_end_kernel<<<1, 1, 0, s>>>(ss, cg); }
void launch_step_advance(StepState* ss, cudaStream_t s) { step_advance_kernel<<<1, 1, 0, s>>>(ss); }

__global__ void loop_open_kernel(cudaGraphConditionalHandle h, LoopSet ls, int cap) {
  bool go = false;
  for (int i = 0; i < ls.n; ++i) {
    ls.ss[i]->loops = 0;
    go = go || (ls.ss[i]->active && !((volatile const CgScalars*)ls.cg[i])->done);
  }
  cudaGraphSetConditional(h, (cap > 0 && go) ? 1u : 0u);
}
__global__ void loop_next_kernel(cudaGraphConditionalHandle h, LoopSet ls, int cap) {
  const int n = ++ls.ss[0]->loops;
  bool go = false;
  for (int i = 0; i < ls.n; ++i) go = go || !((volatile const CgScalars*)ls.cg[i])->done;
  cudaGraphSetConditional(h, (go && n < cap) ? 1u : 0u);
}
void launch_loop_open(cudaGraphConditionalHandle h, const LoopSet& ls, int cap, cudaStream_t s) {
  loop_open_kernel<<<1, 1, 0, s>>>(h, ls, cap);
}
void launch_loop_next(cudaGraphConditionalHandle h, const LoopSet& ls, int cap, cudaStream_t s) {
  loop_next_kernel<<<1, 1, 0, s>>>(h, ls, cap);
}
void launch_to_lo(int64_t N, const double* x, void* d, int half_vec, float* w, cudaStream_t s) {
  if (half_vec)
    to_lo_kernel<__half><<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, x, (__half*)d, w);
  else
    to_lo_kernel<float><<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, x, (float*)d, w);
}
void launch_from_f32(int64_t N, const float* w, double* y, cudaStream_t s) {
  from_f32_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, w, y);
}

int lo_block_elems() { return kLoBlock; }
void launch_block_count(const ModelView& m, int n_blk, int32_t* counts, cudaStream_t s) {
  block_count_kernel<<<n_blk, 256, 0, s>>>(m, counts);
}
void launch_block_fill(const ModelView& m, BlockView b, int32_t* nodes, uint16_t* lconn, int32_t* refcount,
                       cudaStream_t s, const int32_t* counts) {
  block_fill_kernel<<<b.n_blk, 256, 0, s>>>(m, b, nodes, lconn, refcount, counts);  // lconn: [10][n_blk * kLoBlock]
  if (m.F > 0) face_refcount_kernel<<<(unsigned)((m.F + 255) / 256), 256, 0, s>>>(m, refcount);
}
void launch_block_mark(const ModelView& m, BlockView b, int32_t* nodes, int32_t* refcount, int total,
                       cudaStream_t s) {
  (void)m;
  (void)b;
  block_mark_kernel<<<(total + 255) / 256, 256, 0, s>>>(total, nodes, refcount);
}
// FP32 material coefficients of the reduced-precision operator (computed once
// per model so that the operator kernels do no FP64 arithmetic).
// matf[i]: operator A (cK lam/20, cK mu/20, cM rho/420, 0); matf[kMaxMat + 2i]:
// right-hand side (lam/20, mu/20, rho/420, beta); matf[kMaxMat + 2i + 1]:
// (4/dt + alpha, 0, 0, 0).
__global__ void lo_material_kernel(const MatCoef* mat, int n_mat, double dt, float4* matf) {
  const int i = threadIdx.x;
  if (i < n_mat) {
    const MatCoef& c = mat[i];
    matf[i] = make_float4((float)(c.cK * c.lam / 20.0), (float)(c.cK * c.mu / 20.0), (float)(c.cM * c.rho / 420.0),
                          0.f);
    matf[kMaxMat + 2 * i] = make_float4((float)(c.lam / 20.0), (float)(c.mu / 20.0), (float)(c.rho / 420.0),
                                        (float)c.beta);
    matf[kMaxMat + 2 * i + 1] = make_float4((float)(4.0 / dt + c.alpha), 0.f, 0.f, 0.f);
  }
}

void launch_lo_convert(const ModelView& m, int n_blk, const uint16_t* lconn, int half_geo, int half_vec, void* rec,
                       float* fgeo32, const double* dinv, void* dinv_lo, double* partials, InnerScalars* sc,
                       float4* matf, int n_mat, cudaStream_t s) {
  lo_material_kernel<<<1, kMaxMat, 0, s>>>(m.mat, n_mat, m.dt, matf);
  int64_t n = (int64_t)n_blk * kLoBlock;
  if (6 * m.F > n) n = 6 * m.F;
  if (6 * m.N > n) n = 6 * m.N;
  const unsigned g = (unsigned)((n + 255) / 256);
  if (half_geo)
    lo_convert_kernel<__half><<<g, 256, 0, s>>>(m, n_blk, lconn, (LoRecH*)rec, fgeo32);
  else
    lo_convert_kernel<float><<<g, 256, 0, s>>>(m, n_blk, lconn, (LoRecF*)rec, fgeo32);
  dinv_mean_kernel<<<node_blocks(m.N), kNodeThreads, 0, s>>>(m.N, dinv, partials, sc);
  if (half_vec)
    dinv_lo_kernel<__half><<<node_blocks(6 * m.N), kNodeThreads, 0, s>>>(6 * m.N, dinv, sc, (__half*)dinv_lo);
  else
    dinv_lo_kernel<float><<<node_blocks(6 * m.N), kNodeThreads, 0, s>>>(6 * m.N, dinv, sc, (float*)dinv_lo);
}
size_t lo_record_bytes(int half_geo) { return half_geo ? sizeof(LoRecH) : sizeof(LoRecF); }
void launch_inner_init(int64_t N, const double* r, const void* dinv_lo, float* s, float* y, void* t, void* d,
                       int half_vec, float* w, double* partials, InnerScalars* sc, const CgScalars* cg,
                       cudaStream_t st, float rtol, double coarse_rel) {
  if (half_vec)
    inner_init_kernel<__half><<<node_blocks(N), kNodeThreads, 0, st>>>(
        N, r, (const __half*)dinv_lo, s, y, (__half*)t, (__half*)d, w, partials, sc, cg, rtol, coarse_rel);
  else
    inner_init_kernel<float><<<node_blocks(N), kNodeThreads, 0, st>>>(
        N, r, (const float*)dinv_lo, s, y, (float*)t, (float*)d, w, partials, sc, cg, rtol, coarse_rel);
}

// ---- software-pipelined variant ----------------------------------------------
//
// Persistent CTAs walk their element blocks b_i = blockIdx.x + i * gridDim
// with cp.async staging: the packed records and the node-index list of b_{i+2}
// (three stages) and the search-direction gather of b_{i+1} (two stages) are
// in flight while b_i is applied, so the gather latency overlaps arithmetic.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <typename SD>
__device__ __forceinline__ void unpack3(const unsigned char* p, float& a, float& b, float& c) {
  load3(reinterpret_cast<const SD*>(p), a, b, c);
}

template <typename SG, typename SD>
size_t lo_pipe_smem(int max_local) {
  return sizeof(uint4) * 3 * kLoBlock * LoRec<SG>::words + sizeof(int32_t) * 3 * (size_t)max_local +
         sizeof(SD) * 4 * 2 * (size_t)max_local + sizeof(float) * 3 * (size_t)max_local;
}

template <typename SG, typename SD>
__global__ void __launch_bounds__(kLoBlock, 2) ebe_lo_pipe_kernel(LoView<SG> m, const SD* __restrict__ d,
                                                                   float* __restrict__ w, double* partials,
                                                                   InnerScalars* sc, const CgScalars* outer,
                                                                   int n_pipe) {
  if (inner_stopped(outer, sc)) return;
  typedef typename LoRec<SG>::type Rec;
  constexpr int RW = LoRec<SG>::words;
  constexpr int NB = (int)sizeof(SD) * 4;  // bytes per node of the padded search direction
  extern __shared__ __align__(16) unsigned char smem[];
  const int ML = m.blk.max_local;  // padded, a multiple of 4
  uint4* recs = reinterpret_cast<uint4*>(smem);
  int32_t* idx = reinterpret_cast<int32_t*>(recs + 3 * kLoBlock * RW);
  unsigned char* xr = reinterpret_cast<unsigned char*>(idx + 3 * ML);
  float* ys = reinterpret_cast<float*>(xr + (size_t)2 * ML * NB);
  __shared__ float matc[kMaxMat][3];
  if (threadIdx.x < m.n_mat) {
    const float4 c = m.matf[threadIdx.x];
    matc[threadIdx.x][0] = c.x;
    matc[threadIdx.x][1] = c.y;
    matc[threadIdx.x][2] = c.z;
  }
  for (int q = threadIdx.x; q < 3 * ML; q += kLoBlock) ys[q] = 0.f;
  float dot = 0.f;
  const int nb = m.blk.n_blk;
  if ((int)blockIdx.x < n_pipe) {
    const int first = blockIdx.x;
    const int n_my = first < nb ? (nb - first + n_pipe - 1) / n_pipe : 0;
    auto issue_meta = [&](int i) {
      if (i < n_my) {
        const int b = first + i * n_pipe, st = i % 3;
        const uint4* src = reinterpret_cast<const uint4*>(m.rec) + (int64_t)b * kLoBlock * RW;
        for (int q = threadIdx.x; q < kLoBlock * RW; q += kLoBlock) cp_async16(recs + st * kLoBlock * RW + q, src + q);
        const int n0 = m.blk.ptr[b], nn = m.blk.ptr[b + 1] - n0;
        const int4* isrc = reinterpret_cast<const int4*>(m.blk.nodes + n0);
        for (int q = threadIdx.x; q < nn / 4; q += kLoBlock) cp_async16(idx + st * ML + 4 * q, isrc + q);
      }
      cp_async_commit();
    };
    auto issue_gather = [&](int i) {
      if (i < n_my) {
        const int b = first + i * n_pipe, st = i % 3, xb = i & 1;
        const int nn = m.blk.ptr[b + 1] - m.blk.ptr[b];
        for (int q = threadIdx.x; q < nn; q += kLoBlock) {
          const int64_t g = idx[st * ML + q] & 0x7fffffff;
          unsigned char* dst = xr + ((size_t)xb * ML + q) * NB;
          if (NB == 16)
            cp_async16(dst, d + 4 * g);
          else
            cp_async8(dst, d + 4 * g);
        }
      }
      cp_async_commit();
    };
    issue_meta(0);
    issue_meta(1);
    cp_async_wait1();
    __syncthreads();
    issue_gather(0);
    for (int i = 0; i < n_my; ++i) {
      issue_meta(i + 2);
      cp_async_wait1();  // all but the newest group: gather of b_i, meta of b_{i+1}
      __syncthreads();
      issue_gather(i + 1);
      const int b = first + i * n_pipe, st = i % 3, xb = i & 1;
      const int nn = m.blk.ptr[b + 1] - m.blk.ptr[b];
      {
        union {
          uint4 v[RW];
          Rec r;
        } u;
#pragma unroll
        for (int q = 0; q < RW; ++q) u.v[q] = recs[st * kLoBlock * RW + q * kLoBlock + threadIdx.x];
        float g[3][3];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm)
#pragma unroll
          for (int k = 0; k < 3; ++k) g[mm][k] = to_f(u.r.g[3 * mm + k]);
        const float V = u.r.vol;
        const int mt = u.r.mat;
        const float lamS = matc[mt][0] * V, muS = matc[mt][1] * V, mS = matc[mt][2] * V;
        float wv[10][3], f[10][3];
#pragma unroll
        for (int k = 0; k < 10; ++k)
          unpack3<SD>(xr + ((size_t)xb * ML + u.r.lc[k]) * NB, wv[k][0], wv[k][1], wv[k][2]);
        stiffness_apply<float>(wv, g, lamS, muS, f);
        mass_apply<float>(wv, mS, f);
#pragma unroll
        for (int k = 0; k < 10; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            atomicAdd(ys + 3 * u.r.lc[k] + c, f[k][c]);
            dot = fmaf(wv[k][c], f[k][c], dot);
          }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < nn; q += kLoBlock) {
        const int32_t raw = idx[st * ML + q];
        const int64_t g = raw & 0x7fffffff;
        const float y0 = ys[3 * q], y1 = ys[3 * q + 1], y2 = ys[3 * q + 2];
        ys[3 * q] = 0.f;
        ys[3 * q + 1] = 0.f;
        ys[3 * q + 2] = 0.f;
        if (g == m.N) continue;  // padding entry (dummy node N)
        if (raw < 0) {
          w[3 * g] = y0;
          w[3 * g + 1] = y1;
          w[3 * g + 2] = y2;
        } else {
          atomicAdd(w + 3 * g, y0);
          atomicAdd(w + 3 * g + 1, y1);
          atomicAdd(w + 3 * g + 2, y2);
        }
      }
      __syncthreads();
    }
    cp_async_wait0();
  } else {
    __syncthreads();
    // absorbing faces: (2/dt) C_abs d
    const int64_t fc = (int64_t)(blockIdx.x - n_pipe) * kLoBlock + threadIdx.x;
    if (fc < m.F && m.fgeo[5 * m.F + fc] > 0.5f) {
      const float sc2 = m.face_c;
      const float As = sc2 * m.fgeo[fc], Ad = sc2 * m.fgeo[m.F + fc];
      const float n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
      int64_t nd[6];
      float z[6][3], xin[6][3];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        nd[k] = m.fnode[k * m.F + fc];
        load3(d + 4 * nd[k], xin[k][0], xin[k][1], xin[k][2]);
        const float dn = n[0] * xin[k][0] + n[1] * xin[k][1] + n[2] * xin[k][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[k][c] = fmaf(As, xin[k][c], Ad * dn * n[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float Zv = z[0][c] + z[1][c] + z[2][c];
        const float Ze = z[3][c] + z[4][c] + z[5][c];
        float yf[6];
        yf[0] = 7.f * z[0][c] - Zv - 4.f * z[4][c];
        yf[1] = 7.f * z[1][c] - Zv - 4.f * z[5][c];
        yf[2] = 7.f * z[2][c] - Zv - 4.f * z[3][c];
        yf[3] = 16.f * (z[3][c] + Ze) - 4.f * z[2][c];
        yf[4] = 16.f * (z[4][c] + Ze) - 4.f * z[0][c];
        yf[5] = 16.f * (z[5][c] + Ze) - 4.f * z[1][c];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          atomicAdd(w + 3 * nd[k] + c, yf[k]);
          dot = fmaf(xin[k][c], yf[k], dot);
        }
      }
    }
  }
  lo_store_dw(dot, m.dw_part, sc);
}

template <typename SG, typename SD>
static void ebe_lo_pipe_launch(const LoView<SG>& m, const SD* d, float* w, double* partials, InnerScalars* sc,
                               cudaStream_t st, const CgScalars* outer) {
  const size_t smem = lo_pipe_smem<SG, SD>(m.blk.max_local);
  static size_t attr_set = 0;  // per instantiation
  if (smem > attr_set) {
    cudaFuncSetAttribute(ebe_lo_pipe_kernel<SG, SD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = smem;
  }
  int dev = 0, sms = 152, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ebe_lo_pipe_kernel<SG, SD>, kLoBlock, smem);
  if (occ < 1) occ = 1;
  int n_pipe = sms * occ;
  if (n_pipe > m.blk.n_blk) n_pipe = m.blk.n_blk > 0 ? m.blk.n_blk : 1;
  const unsigned g = (unsigned)(n_pipe + (m.F + kLoBlock - 1) / kLoBlock);
  ebe_lo_pipe_kernel<SG, SD><<<g, kLoBlock, smem, st>>>(m, d, w, partials, sc, outer, n_pipe);
}

// ---- warp-specialised variant -------------------------------------------------
//
// Persistent CTAs of 6 consumer warps (one element per thread, as above) and
// one producer warp.  The producer stages element block b_i in a ring of
// kWsStages shared-memory stages: lane 0 issues two bulk asynchronous copies
// (the block's packed records and its node list) that complete on the
// stage's "meta" mbarrier; once they have landed, the 32 lanes gather the
// block's search-direction entries with cp.async, completing on the stage's
// "x" mbarrier.  Metadata runs one block ahead of the gathers, so the
// producer keeps two blocks in flight while the consumers apply a third;
// the consumers release a stage through its "empty" mbarrier.  Every wait is
// bounded: a wait that runs out sets InnerScalars::err (and fails the outer
// solve), and the CTA stops after its copies in flight have landed.

constexpr int kWsStages = 3;
constexpr int kWsThreads = kLoBlock + 32;
constexpr long long kWsSpin = 1ll << 22;  // try_wait attempts (each may suspend briefly)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false if it ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit = kWsSpin) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try(b, parity)) return true;
  return false;
}

// Failure-detection self-test: the bounded wait above on an mbarrier that
// expects one arrival which never comes.  The wait runs out after `limit`
// attempts; out[0] = 1 if it did, out[1] = 1 if it (wrongly) completed.
__global__ void wait_probe_kernel(long long limit, unsigned* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool done = mbar_wait(&bar, 0u, limit);
    out[0] = done ? 0u : 1u;
    out[1] = done ? 1u : 0u;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kLoBlock) : "memory"); }

template <typename SG, typename SD>
size_t lo_ws_smem(int max_local) {
  return (sizeof(uint4) * kLoBlock * LoRec<SG>::words + sizeof(int32_t) * (size_t)max_local +
          sizeof(SD) * 4 * (size_t)max_local) *
             kWsStages +
         sizeof(float) * 3 * (size_t)max_local;
}

template <typename SG, typename SD>
__global__ void __launch_bounds__(kWsThreads, 2) ebe_lo_ws_kernel(LoView<SG> m, const SD* __restrict__ d,
                                                                 float* __restrict__ w, double* partials,
                                                                 InnerScalars* sc, const CgScalars* outer,
                                                                 int n_ws) {
  if (inner_stopped(outer, sc)) return;
  typedef typename LoRec<SG>::type Rec;
  constexpr int RW = LoRec<SG>::words;
  constexpr int NB = (int)sizeof(SD) * 4;  // bytes per node of the padded search direction
  constexpr unsigned kRecBytes = sizeof(uint4) * kLoBlock * RW;
  extern __shared__ __align__(16) unsigned char ws_smem[];
  const int ML = m.blk.max_local;  // a multiple of 4
  uint4* recs = reinterpret_cast<uint4*>(ws_smem);
  int32_t* idx = reinterpret_cast<int32_t*>(ws_smem + (size_t)kRecBytes * kWsStages);
  unsigned char* xr = reinterpret_cast<unsigned char*>(idx + (size_t)kWsStages * ML);
  float* ys = reinterpret_cast<float*>(xr + (size_t)kWsStages * ML * NB);
  __shared__ __align__(8) uint64_t bar_meta[kWsStages], bar_x[kWsStages], bar_empty[kWsStages];
  __shared__ int nn_stage[kWsStages];
  __shared__ int abort_flag;
  __shared__ float matc[kMaxMat][3];
  const int tid = threadIdx.x;
  if (tid < m.n_mat) {
    const float4 c = m.matf[tid];
    matc[tid][0] = c.x;
    matc[tid][1] = c.y;
    matc[tid][2] = c.z;
  }
  if (tid == 0) {
    for (int st = 0; st < kWsStages; ++st) {
      mbar_init(&bar_meta[st], 1);
      mbar_init(&bar_x[st], 32);
      mbar_init(&bar_empty[st], kLoBlock / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  for (int q = tid; q < 3 * ML; q += kWsThreads) ys[q] = 0.f;
  __syncthreads();
  float dot = 0.f;
  const int nb = m.blk.n_blk;
  const int b0 = blockIdx.x;
  if (b0 < n_ws) {
    const int n_my = b0 < nb ? (nb - b0 + n_ws - 1) / n_ws : 0;
    if (tid >= kLoBlock) {
      // ---------------- producer warp ----------------
      const int lane = tid - kLoBlock;
      int issued = 0;  // blocks whose metadata copies were issued
      bool ok = true;
      for (int i = 0; i <= n_my && ok; ++i) {
        if (i < n_my) {
          const int st = i % kWsStages;
          if (i >= kWsStages) ok = mbar_wait(&bar_empty[st], ((i / kWsStages) - 1) & 1);
          if (ok && lane == 0) {
            const int b = b0 + i * n_ws;
            const int n0 = m.blk.ptr[b], nn = m.blk.ptr[b + 1] - n0;
            nn_stage[st] = nn;
            mbar_expect_tx(&bar_meta[st], kRecBytes + 4u * (unsigned)nn);
            bulk_g2s(recs + (size_t)st * kLoBlock * RW,
                     reinterpret_cast<const uint4*>(m.rec) + (int64_t)b * kLoBlock * RW, kRecBytes,
                     &bar_meta[st]);
            if (nn > 0) bulk_g2s(idx + (size_t)st * ML, m.blk.nodes + n0, 4u * (unsigned)nn, &bar_meta[st]);
          }
          if (ok) issued = i + 1;
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        }
        if (ok && i >= 1) {
          const int j = i - 1, st = j % kWsStages;
          ok = mbar_wait(&bar_meta[st], (j / kWsStages) & 1);
          ok = __all_sync(0xffffffffu, ok);
          if (ok) {
            const int nn = nn_stage[st];
            const int32_t* ix = idx + (size_t)st * ML;
            unsigned char* dst = xr + (size_t)st * ML * NB;
            for (int q = lane; q < nn; q += 32) {
              const int64_t g = ix[q] & 0x7fffffff;
              if (NB == 16)
                cp_async16(dst + (size_t)q * NB, d + 4 * g);
              else
                cp_async8(dst + (size_t)q * NB, d + 4 * g);
            }
            cp_async_arrive(&bar_x[st]);
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        sc->err = 1u;
        if (outer != nullptr) {
          ((CgScalars*)outer)->status = kStatusTimeout;
          ((CgScalars*)outer)->done = 1;
        }
      }
      // every copy issued by this warp lands before the CTA may exit
      cp_async_wait0();
      if (lane == 0)
        for (int i = (issued > kWsStages ? issued - kWsStages : 0); i < issued; ++i)
          mbar_wait(&bar_meta[i % kWsStages], (i / kWsStages) & 1);
      __syncwarp();
    } else {
      // ---------------- consumer warps ----------------
      for (int i = 0; i < n_my; ++i) {
        const int st = i % kWsStages;
        const unsigned ph = (i / kWsStages) & 1;
        bool ok = mbar_wait(&bar_meta[st], ph);
        if (ok) ok = mbar_wait(&bar_x[st], ph);
        if (!ok) {
          atomicExch(&abort_flag, 1);
          sc->err = 1u;
          if (outer != nullptr) {
            ((CgScalars*)outer)->status = kStatusTimeout;
            ((CgScalars*)outer)->done = 1;
          }
        }
        consumer_sync();
        if (((volatile int*)&abort_flag)[0]) break;
        const uint4* rs = recs + (size_t)st * kLoBlock * RW;
        const unsigned char* xs = xr + (size_t)st * ML * NB;
        {
          union {
            uint4 v[RW];
            Rec r;
          } u;
#pragma unroll
          for (int q = 0; q < RW; ++q) u.v[q] = rs[q * kLoBlock + tid];
          float g[3][3];
#pragma unroll
          for (int mm = 0; mm < 3; ++mm)
#pragma unroll
            for (int k = 0; k < 3; ++k) g[mm][k] = to_f(u.r.g[3 * mm + k]);
          const float V = u.r.vol;
          const int mt = u.r.mat;
          const float lamS = matc[mt][0] * V, muS = matc[mt][1] * V, mS = matc[mt][2] * V;
          float wv[10][3], f[10][3];
#pragma unroll
          for (int k = 0; k < 10; ++k) unpack3<SD>(xs + (size_t)u.r.lc[k] * NB, wv[k][0], wv[k][1], wv[k][2]);
          stiffness_apply<float>(wv, g, lamS, muS, f);
          mass_apply<float>(wv, mS, f);
#pragma unroll
          for (int k = 0; k < 10; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              atomicAdd(ys + 3 * u.r.lc[k] + c, f[k][c]);
              dot = fmaf(wv[k][c], f[k][c], dot);
            }
        }
        consumer_sync();
        const int nn = nn_stage[st];
        const int32_t* ix = idx + (size_t)st * ML;
        for (int q = tid; q < nn; q += kLoBlock) {
          const int32_t raw = ix[q];
          const int64_t g = raw & 0x7fffffff;
          const float y0 = ys[3 * q], y1 = ys[3 * q + 1], y2 = ys[3 * q + 2];
          ys[3 * q] = 0.f;
          ys[3 * q + 1] = 0.f;
          ys[3 * q + 2] = 0.f;
          if (g == m.N) continue;  // padding entry (dummy node N)
          if (raw < 0) {
            w[3 * g] = y0;
            w[3 * g + 1] = y1;
            w[3 * g + 2] = y2;
          } else {
            atomicAdd(w + 3 * g, y0);
            atomicAdd(w + 3 * g + 1, y1);
            atomicAdd(w + 3 * g + 2, y2);
          }
        }
        consumer_sync();
        if ((tid & 31) == 0) mbar_arrive(&bar_empty[st]);
      }
    }
  } else {
    // absorbing faces: (2/dt) C_abs d
    const int64_t fc = (int64_t)(b0 - n_ws) * kWsThreads + tid;
    if (fc < m.F && m.fgeo[5 * m.F + fc] > 0.5f) {
      const float sc2 = m.face_c;
      const float As = sc2 * m.fgeo[fc], Ad = sc2 * m.fgeo[m.F + fc];
      const float n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
      int64_t nd[6];
      float z[6][3], xin[6][3];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        nd[k] = m.fnode[k * m.F + fc];
        load3(d + 4 * nd[k], xin[k][0], xin[k][1], xin[k][2]);
        const float dn = n[0] * xin[k][0] + n[1] * xin[k][1] + n[2] * xin[k][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[k][c] = fmaf(As, xin[k][c], Ad * dn * n[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float Zv = z[0][c] + z[1][c] + z[2][c];
        const float Ze = z[3][c] + z[4][c] + z[5][c];
        float yf[6];
        yf[0] = 7.f * z[0][c] - Zv - 4.f * z[4][c];
        yf[1] = 7.f * z[1][c] - Zv - 4.f * z[5][c];
        yf[2] = 7.f * z[2][c] - Zv - 4.f * z[3][c];
        yf[3] = 16.f * (z[3][c] + Ze) - 4.f * z[2][c];
        yf[4] = 16.f * (z[4][c] + Ze) - 4.f * z[0][c];
        yf[5] = 16.f * (z[5][c] + Ze) - 4.f * z[1][c];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          atomicAdd(w + 3 * nd[k] + c, yf[k]);
          dot = fmaf(xin[k][c], yf[k], dot);
        }
      }
    }
  }
  lo_store_dw(dot, m.dw_part, sc);
}

template <typename SG, typename SD>
static void ebe_lo_ws_launch(const LoView<SG>& m, const SD* d, float* w, double* partials, InnerScalars* sc,
                             cudaStream_t st, const CgScalars* outer) {
  const size_t smem = lo_ws_smem<SG, SD>(m.blk.max_local);
  static size_t attr_set = 0;  // per instantiation
  static int sms = 0, occ = 0;
  static size_t occ_smem = 0;
  if (smem > attr_set) {
    cudaFuncSetAttribute(ebe_lo_ws_kernel<SG, SD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = smem;
  }
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (occ_smem != smem) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ebe_lo_ws_kernel<SG, SD>, kWsThreads, smem);
    if (occ < 1) occ = 1;
    occ_smem = smem;
  }
  int n_ws = sms * occ;
  if (n_ws > m.blk.n_blk) n_ws = m.blk.n_blk > 0 ? m.blk.n_blk : 1;
  const unsigned g = (unsigned)(n_ws + (m.F + kWsThreads - 1) / kWsThreads);
  ebe_lo_ws_kernel<SG, SD><<<g, kWsThreads, smem, st>>>(m, d, w, partials, sc, outer, n_ws);
}

// variant: 0 -> up to 3 CTAs per SM (no register cap below 96), 1 -> 4 CTAs
// per SM (80 registers), 2 -> the persistent software-pipelined kernel,
// 3 -> the persistent warp-specialised kernel (bulk copies, mbarriers);
// picked per model by the set-up autotuner.
template <typename SG, typename SD>
static void ebe_lo_launch(int variant, const LoView<SG>& m, const SD* d, float* w, double* partials,
                          InnerScalars* sc, cudaStream_t st, const CgScalars* outer) {
  if (variant == 2) {
    ebe_lo_pipe_launch<SG, SD>(m, d, w, partials, sc, st, outer);
    return;
  }
  // bulk copies need 16-byte aligned sources (device allocations are)
  if (variant == 3 && ((reinterpret_cast<uintptr_t>(m.rec) | reinterpret_cast<uintptr_t>(m.blk.nodes)) & 15) == 0) {
    ebe_lo_ws_launch<SG, SD>(m, d, w, partials, sc, st, outer);
    return;
  }
  const unsigned g = (unsigned)(m.blk.n_blk + (m.F + kLoBlock - 1) / kLoBlock);
  const size_t smem = sizeof(float) * 6 * (size_t)m.blk.max_local;
  if (variant == 1)
    ebe_lo_kernel<SG, SD, 4><<<g, kLoBlock, smem, st>>>(m, d, w, partials, sc, outer);
  else
    ebe_lo_kernel<SG, SD, 1><<<g, kLoBlock, smem, st>>>(m, d, w, partials, sc, outer);
}
template <typename SG, typename SD>
static void ebe_lo_fused_launch(int variant, const LoView<SG>& m, const SD* dprev, const SD* t4, SD* dnew,
                                float* w, double* partials, InnerScalars* sc, cudaStream_t st,
                                const CgScalars* outer) {
  const unsigned g = (unsigned)(m.blk.n_blk + (m.F + kLoBlock - 1) / kLoBlock);
  const size_t smem = sizeof(float) * 6 * (size_t)m.blk.max_local;
  if (variant == 1)
    ebe_lo_kernel<SG, SD, 4, true><<<g, kLoBlock, smem, st>>>(m, dprev, w, partials, sc, outer, t4, dnew);
  else
    ebe_lo_kernel<SG, SD, 1, true><<<g, kLoBlock, smem, st>>>(m, dprev, w, partials, sc, outer, t4, dnew);
}
bool lo_variant_fuses(int variant) { return variant == 0 || variant == 1; }
void launch_ebe_lo_fused(int half_geo, int half_vec, const void* lo_view, const void* dprev, const void* t4,
                         void* dnew, float* w, double* partials, InnerScalars* sc, cudaStream_t st, int variant,
                         const CgScalars* outer) {
  if (half_geo) {
    const LoView<__half>& m = *(const LoView<__half>*)lo_view;
    if (half_vec)
      ebe_lo_fused_launch<__half, __half>(variant, m, (const __half*)dprev, (const __half*)t4, (__half*)dnew, w, partials, sc, st,
                                          outer);
    else
      ebe_lo_fused_launch<__half, float>(variant, m, (const float*)dprev, (const float*)t4, (float*)dnew, w, partials, sc, st,
                                         outer);
  } else {
    const LoView<float>& m = *(const LoView<float>*)lo_view;
    if (half_vec)
      ebe_lo_fused_launch<float, __half>(variant, m, (const __half*)dprev, (const __half*)t4, (__half*)dnew, w, partials, sc, st,
                                         outer);
    else
      ebe_lo_fused_launch<float, float>(variant, m, (const float*)dprev, (const float*)t4, (float*)dnew, w, partials, sc, st,
                                        outer);
  }
}
void launch_ebe_lo(int half_geo, int half_vec, const void* lo_view, const void* d, float* w, double* partials,
                   InnerScalars* sc, cudaStream_t st, int variant, const CgScalars* outer) {
  if (half_geo) {
    const LoView<__half>& m = *(const LoView<__half>*)lo_view;
    if (half_vec)
      ebe_lo_launch<__half, __half>(variant, m, (const __half*)d, w, partials, sc, st, outer);
    else
      ebe_lo_launch<__half, float>(variant, m, (const float*)d, w, partials, sc, st, outer);
  } else {
    const LoView<float>& m = *(const LoView<float>*)lo_view;
    if (half_vec)
      ebe_lo_launch<float, __half>(variant, m, (const __half*)d, w, partials, sc, st, outer);
    else
      ebe_lo_launch<float, float>(variant, m, (const float*)d, w, partials, sc, st, outer);
  }
}
template <typename SG, typename SD>
static void ebe_lo3_launch(int variant, const LoView<SG>& m, const Lo3Args& a, cudaStream_t st) {
  const unsigned g = (unsigned)(m.blk.n_blk + (m.F + kLoBlock - 1) / kLoBlock);
  const size_t smem = sizeof(float) * 18 * (size_t)m.blk.max_local;
  static size_t attr[2] = {0, 0};  // per instantiation and occupancy variant
  const int vi = variant == 1 ? 1 : 0;
  if (smem > 48 * 1024 && smem > attr[vi]) {
    if (vi)
      cudaFuncSetAttribute(ebe_lo3_kernel<SG, SD, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
      cudaFuncSetAttribute(ebe_lo3_kernel<SG, SD, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[vi] = smem;
  }
  if (vi)
    ebe_lo3_kernel<SG, SD, 3><<<g, kLoBlock, smem, st>>>(m, a);
  else
    ebe_lo3_kernel<SG, SD, 1><<<g, kLoBlock, smem, st>>>(m, a);
}
void launch_ebe_lo3(int half_geo, int half_vec, const void* lo_view, const Lo3Args& a, cudaStream_t st, int variant) {
  if (half_geo) {
    const LoView<__half>& m = *(const LoView<__half>*)lo_view;
    if (half_vec)
      ebe_lo3_launch<__half, __half>(variant, m, a, st);
    else
      ebe_lo3_launch<__half, float>(variant, m, a, st);
  } else {
    const LoView<float>& m = *(const LoView<float>*)lo_view;
    if (half_vec)
      ebe_lo3_launch<float, __half>(variant, m, a, st);
    else
      ebe_lo3_launch<float, float>(variant, m, a, st);
  }
}

// ------------------------------------------------------------------------------
// FP32 right-hand side (its norm sets the relative-residual scale)
// ------------------------------------------------------------------------------

// u, v, a in FP32, one padded 16-byte word each per node: uva[3n + {0, 1, 2}].
__global__ void uva_f32_kernel(int64_t N, const double* __restrict__ u, const double* __restrict__ v,
                               const double* __restrict__ a, float4* __restrict__ uva, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    uva[3 * n] = make_float4((float)u[3 * n], (float)u[3 * n + 1], (float)u[3 * n + 2], 0.f);
    uva[3 * n + 1] = make_float4((float)v[3 * n], (float)v[3 * n + 1], (float)v[3 * n + 2], 0.f);
    uva[3 * n + 2] = make_float4((float)a[3 * n], (float)a[3 * n + 1], (float)a[3 * n + 2], 0.f);
  }
}

// b = f - K u + C v + M (a + 4/dt v) in FP32 on the reduced-precision
// operator's element blocks (Newmark, the right-hand side of A du = b):
// element stiffness on beta_e v - u, element mass on a + (4/dt + alpha_e) v,
// dashpot faces on v plus the base force 2 p C_base e_dir.  Same block
// assembly as the operator (shared-memory gather and atomics, one write per
// unique node).  b must be zero on entry.  Only ||b|| is taken from it (the
// scale of the relative-residual test), so FP32 accuracy suffices; the FP64
// solve never uses b itself.
template <typename SG>
__global__ void __launch_bounds__(kLoBlock, 3) ebe_lo_rhs_kernel(LoView<SG> m, const float4* __restrict__ uva,
                                                                float* __restrict__ b, float force, int dir,
                                                                Drive dr) {
  if (dr.ss != nullptr) {
    if (!((volatile const StepState*)dr.ss)->active) return;
    force = 2.f * (float)dr.p[dr.ss->step];
  }
  typedef typename LoRec<SG>::type Rec;
  constexpr int RW = LoRec<SG>::words;
  extern __shared__ __align__(16) float rhs_sm[];
  __shared__ float4 mr[2 * kMaxMat];
  if (threadIdx.x < 2 * m.n_mat) mr[threadIdx.x] = m.matf[kMaxMat + threadIdx.x];
  const int b0 = blockIdx.x;
  const int ML = m.blk.max_local;
  if (b0 < m.blk.n_blk) {
    float4* xs = reinterpret_cast<float4*>(rhs_sm);  // [ML][3]: u, v, a
    float* ys = rhs_sm + 12 * ML;
    union {
      uint4 v[RW];
      Rec r;
    } u;
    const uint4* rp = reinterpret_cast<const uint4*>(m.rec) + (int64_t)b0 * kLoBlock * RW + threadIdx.x;
#pragma unroll
    for (int q = 0; q < RW; ++q) u.v[q] = __ldg(rp + q * kLoBlock);
    const int64_t n0 = (int64_t)b0 * ML;
    for (int i = threadIdx.x; i < ML; i += kLoBlock) {
      const int64_t g = m.blk.nodes[n0 + i] & 0x7fffffff;
      xs[3 * i] = uva[3 * g];
      xs[3 * i + 1] = uva[3 * g + 1];
      xs[3 * i + 2] = uva[3 * g + 2];
      ys[3 * i] = 0.f;
      ys[3 * i + 1] = 0.f;
      ys[3 * i + 2] = 0.f;
    }
    __syncthreads();
    {
      float g[3][3];
#pragma unroll
      for (int mm = 0; mm < 3; ++mm)
#pragma unroll
        for (int i = 0; i < 3; ++i) g[mm][i] = to_f(u.r.g[3 * mm + i]);
      const float V = u.r.vol;
      const float4 c0 = mr[2 * u.r.mat], c1 = mr[2 * u.r.mat + 1];
      float w[10][3], f[10][3];
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const float4 uu = xs[3 * u.r.lc[k]], vv = xs[3 * u.r.lc[k] + 1];
        w[k][0] = fmaf(c0.w, vv.x, -uu.x);
        w[k][1] = fmaf(c0.w, vv.y, -uu.y);
        w[k][2] = fmaf(c0.w, vv.z, -uu.z);
      }
      stiffness_apply<float>(w, g, c0.x * V, c0.y * V, f);
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const float4 vv = xs[3 * u.r.lc[k] + 1], aa = xs[3 * u.r.lc[k] + 2];
        w[k][0] = fmaf(c1.x, vv.x, aa.x);
        w[k][1] = fmaf(c1.x, vv.y, aa.y);
        w[k][2] = fmaf(c1.x, vv.z, aa.z);
      }
      mass_apply<float>(w, c0.z * V, f);
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) atomicAdd(ys + 3 * u.r.lc[k] + i, f[k][i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ML; i += kLoBlock) {
      const int32_t raw = m.blk.nodes[n0 + i];
      const int64_t g = raw & 0x7fffffff;
      if (g == m.N) continue;  // padding entry (dummy node N)
      if (raw < 0) {
        b[3 * g] = ys[3 * i];
        b[3 * g + 1] = ys[3 * i + 1];
        b[3 * g + 2] = ys[3 * i + 2];
      } else {
        atomicAdd(b + 3 * g, ys[3 * i]);
        atomicAdd(b + 3 * g + 1, ys[3 * i + 1]);
        atomicAdd(b + 3 * g + 2, ys[3 * i + 2]);
      }
    }
  } else {
    // dashpot faces: C_abs v (face mass pattern A/180 on rho Vs / rho Vp) and,
    // on the base, the input force 2 p C_base e_dir (int N_a dA = A/3 at edge
    // nodes, 0 at vertices)
    const int64_t fc = (int64_t)(b0 - m.blk.n_blk) * kLoBlock + threadIdx.x;
    if (fc < m.F && m.fgeo[5 * m.F + fc] > 0.5f) {
      const float tag = m.fgeo[5 * m.F + fc];
      const float As = m.fgeo[fc] / 180.f, Ad = m.fgeo[m.F + fc] / 180.f;
      const float n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
      int64_t nd[6];
      float z[6][3];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        nd[k] = m.fnode[k * m.F + fc];
        const float4 vv = uva[3 * nd[k] + 1];
        const float dn = n[0] * vv.x + n[1] * vv.y + n[2] * vv.z;
        z[k][0] = fmaf(As, vv.x, Ad * dn * n[0]);
        z[k][1] = fmaf(As, vv.y, Ad * dn * n[1]);
        z[k][2] = fmaf(As, vv.z, Ad * dn * n[2]);
      }
      const float ndir = dir == 0 ? n[0] : (dir == 1 ? n[1] : n[2]);
      float fz[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) fz[i] = (tag < 1.5f) ? force * 60.f * (As * (dir == i) + Ad * ndir * n[i]) : 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float Zv = z[0][i] + z[1][i] + z[2][i];
        const float Ze = z[3][i] + z[4][i] + z[5][i];
        float yf[6];
        yf[0] = 7.f * z[0][i] - Zv - 4.f * z[4][i];
        yf[1] = 7.f * z[1][i] - Zv - 4.f * z[5][i];
        yf[2] = 7.f * z[2][i] - Zv - 4.f * z[3][i];
        yf[3] = 16.f * (z[3][i] + Ze) - 4.f * z[2][i] + fz[i];
        yf[4] = 16.f * (z[4][i] + Ze) - 4.f * z[0][i] + fz[i];
        yf[5] = 16.f * (z[5][i] + Ze) - 4.f * z[1][i] + fz[i];
#pragma unroll
        for (int k = 0; k < 6; ++k) atomicAdd(b + 3 * nd[k] + i, yf[k]);
      }
    }
  }
}

void launch_rhs_lo(int half_geo, const void* lo_view, int64_t N, const double* u, const double* v, const double* a,
                   float4* uva, float* b32, double force, int dir, cudaStream_t st, Drive dr) {
  uva_f32_kernel<<<node_blocks(N), kNodeThreads, 0, st>>>(N, u, v, a, uva, dr.ss);
  if (half_geo) {
    const LoView<__half>& m = *(const LoView<__half>*)lo_view;
    const unsigned g = (unsigned)(m.blk.n_blk + (m.F + kLoBlock - 1) / kLoBlock);
    ebe_lo_rhs_kernel<__half><<<g, kLoBlock, sizeof(float) * 15 * (size_t)m.blk.max_local, st>>>(m, uva, b32,
                                                                                                 (float)force, dir, dr);
  } else {
    const LoView<float>& m = *(const LoView<float>*)lo_view;
    const unsigned g = (unsigned)(m.blk.n_blk + (m.F + kLoBlock - 1) / kLoBlock);
    ebe_lo_rhs_kernel<float><<<g, kLoBlock, sizeof(float) * 15 * (size_t)m.blk.max_local, st>>>(m, uva, b32,
                                                                                                (float)force, dir, dr);
  }
}

static unsigned quad_blocks(int64_t N) { return (unsigned)(((N >> 2) + 1 + kNodeThreads - 1) / kNodeThreads); }
// Persistent grid of the node-quad kernels: the SMs times the CTAs that fit on
// one, so a CTA walks many quads and forms its reduction partial once.
static unsigned persistent_cap(const void* kernel) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kNodeThreads, 0);
  return (unsigned)((sms > 0 ? sms : 1) * (occ > 0 ? occ : 1));
}
static unsigned quad_grid(int64_t N, unsigned cap) {
  const unsigned b = quad_blocks(N);
  return b < cap ? b : cap;
}
void launch_inner_update(int64_t N, float* y, float* s, void* t, const void* d, int half_vec, float* w,
                         const void* dinv_lo, const float* dw_part, double* partials, InnerScalars* sc,
                         cudaStream_t st, const CgScalars* outer, int n_dw_max) {
  if (n_dw_max <= kAlphaPrologueMax) {
    if (half_vec) {
      static const unsigned cap = persistent_cap((const void*)inner_update_kernel<__half, true>);
      inner_update_kernel<__half, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
          N, y, s, (__half*)t, (const __half*)d, w, (const __half*)dinv_lo, partials, sc, outer, dw_part);
    } else {
      static const unsigned cap = persistent_cap((const void*)inner_update_kernel<float, true>);
      inner_update_kernel<float, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
          N, y, s, (float*)t, (const float*)d, w, (const float*)dinv_lo, partials, sc, outer, dw_part);
    }
    return;
  }
  inner_alpha_kernel<<<1, 1024, 0, st>>>(dw_part, sc, outer);
  if (half_vec) {
    static const unsigned cap = persistent_cap((const void*)inner_update_kernel<__half>);
    inner_update_kernel<__half><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
        N, y, s, (__half*)t, (const __half*)d, w, (const __half*)dinv_lo, partials, sc, outer);
  } else {
    static const unsigned cap = persistent_cap((const void*)inner_update_kernel<float>);
    inner_update_kernel<float><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
        N, y, s, (float*)t, (const float*)d, w, (const float*)dinv_lo, partials, sc, outer);
  }
}
void launch_inner_update_coarse(int64_t N, float* y, float* s, void* t, const void* d, int half_vec, float* w,
                                const void* dinv_lo, const float* dw_part, double* partials, InnerScalars* sc,
                                cudaStream_t st, const CgScalars* outer, int n_dw_max) {
  if (n_dw_max <= kAlphaPrologueMax) {
    if (half_vec) {
      static const unsigned cap = persistent_cap((const void*)inner_update_kernel<__half, true, true>);
      inner_update_kernel<__half, true, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
          N, y, s, (__half*)t, (const __half*)d, w, (const __half*)dinv_lo, partials, sc, outer, dw_part);
    } else {
      static const unsigned cap = persistent_cap((const void*)inner_update_kernel<float, true, true>);
      inner_update_kernel<float, true, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
          N, y, s, (float*)t, (const float*)d, w, (const float*)dinv_lo, partials, sc, outer, dw_part);
    }
    return;
  }
  inner_alpha_kernel<<<1, 1024, 0, st>>>(dw_part, sc, outer);
  if (half_vec) {
    static const unsigned cap = persistent_cap((const void*)inner_update_kernel<__half, false, true>);
    inner_update_kernel<__half, false, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
        N, y, s, (__half*)t, (const __half*)d, w, (const __half*)dinv_lo, partials, sc, outer);
  } else {
    static const unsigned cap = persistent_cap((const void*)inner_update_kernel<float, false, true>);
    inner_update_kernel<float, false, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(
        N, y, s, (float*)t, (const float*)d, w, (const float*)dinv_lo, partials, sc, outer);
  }
}
void launch_coarse_restrict(const CoarseView& c, const float* s, float4* zc, double* partials, InnerScalars* sc,
                            const CgScalars* outer, int first, cudaStream_t st) {
  if (c.Nv <= 0) return;
  // one CTA of 1024 threads per SM: a solve whose coarse level is switched off
  // pays only for this small grid's early exit
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int64_t need = (c.Nv + kCoarseThreads - 1) / kCoarseThreads;
  const unsigned grid = (unsigned)(need < sms ? need : sms);
  coarse_restrict_kernel<<<grid, kCoarseThreads, 0, st>>>(c, s, zc, partials, sc, outer, first);
}
void launch_coarse_prolong(int64_t N, const int2* pair, const float4* zc, double scale, double* y, cudaStream_t st) {
  coarse_prolong_kernel<<<node_blocks(N), kNodeThreads, 0, st>>>(N, pair, zc, scale, y);
}
void launch_coarse_lo(int64_t Nv, const double* cinv, const InnerScalars* sc, double omega, float* dc,
                      cudaStream_t st) {
  coarse_lo_kernel<<<node_blocks(6 * Nv), kNodeThreads, 0, st>>>(6 * Nv, cinv, sc, omega, dc);
}
void launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t st) {
  to_f32_kernel<<<node_blocks(n), kNodeThreads, 0, st>>>(n, x, y);
}
void launch_inner_dupdate(int64_t N, const void* t, void* d, int half_vec, const InnerScalars* sc,
                          cudaStream_t st, const CgScalars* outer, const int2* pair, const float4* zc) {
  if (zc != nullptr) {
    if (half_vec) {
      static const unsigned cap = persistent_cap((const void*)inner_dupdate_kernel<__half, true>);
      inner_dupdate_kernel<__half, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(N, (const __half*)t, (__half*)d,
                                                                                   sc, outer, pair, zc);
    } else {
      static const unsigned cap = persistent_cap((const void*)inner_dupdate_kernel<float, true>);
      inner_dupdate_kernel<float, true><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(N, (const float*)t, (float*)d,
                                                                                  sc, outer, pair, zc);
    }
    return;
  }
  if (half_vec) {
    static const unsigned cap = persistent_cap((const void*)inner_dupdate_kernel<__half>);
    inner_dupdate_kernel<__half><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(N, (const __half*)t, (__half*)d, sc,
                                                                             outer);
  } else {
    static const unsigned cap = persistent_cap((const void*)inner_dupdate_kernel<float>);
    inner_dupdate_kernel<float><<<quad_grid(N, cap), kNodeThreads, 0, st>>>(N, (const float*)t, (float*)d, sc,
                                                                            outer);
  }
}
void launch_fcg_residual(const ModelView& m, const double* b, double* q, double* r, double* partials, CgScalars* cg,
                         cudaStream_t s) {
  fcg_residual_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, b, q, r, partials, cg);
}
void launch_fcg_first(const ModelView& m, const float* y, const double* r, double* z, double* p, double* partials,
                      CgScalars* cg, const InnerScalars* sc, cudaStream_t s, int dwp) {
  fcg_first_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, y, r, z, p, partials, cg, sc, dwp);
}
void launch_fcg_update(const ModelView& m, double* x, double* r, const double* p, const double* q, double* partials,
                       CgScalars* cg, cudaStream_t s, int dwp) {
  fcg_update_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, x, r, p, q, partials, cg, dwp);
}
void launch_fcg_zbeta(const ModelView& m, const float* y, const double* r, const double* q, double* z,
                      double* partials, CgScalars* cg, const InnerScalars* sc, cudaStream_t s) {
  fcg_zbeta_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, y, r, q, z, partials, cg, sc);
}
void launch_fcg_pupdate(const ModelView& m, const double* z, double* p, double* q, const CgScalars* cg,
                        cudaStream_t s, int dwp) {
  fcg_pupdate_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, z, p, q, cg, dwp);
}

void launch_wait_probe(long long limit, unsigned* out, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(limit, out);
}

}  // namespace gsw
