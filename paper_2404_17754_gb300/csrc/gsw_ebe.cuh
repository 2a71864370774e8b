// Element-level operators of the second-order tetrahedron, shared by the
// FP64 and the reduced-precision kernels (T = double or float).
//
// For an affine quadratic tetrahedron with barycentric gradients
// g_m = grad L_m, the displacement gradient is linear, grad u = sum_k L_k H_k,
// with H_k (the gradient at vertex k)
//     H_k = 4 [ u_k (x) g_k + sum_{b != k} u_kb (x) g_b ] - sum_a u_a (x) g_a.
// The stress is sigma = sum_k L_k S_k, S_k = lam tr(H_k) I + mu (H_k + H_k^T),
// and exact integration of sigma . grad N (int L_i L_j dV = V (1 + d_ij) / 20)
// gives, with T_km = S_k g_m and T_m = sum_k T_km,
//     vertex a:     f_a  = V/20 (4 T_aa - T_a)
//     edge (a, b):  f_ab = V/5  (T_a + T_b + T_ab + T_ba).
// The consistent mass is the closed-form pattern rho V / 420 {vertex diag 6,
// vertex-vertex 1, vertex-edge -4 (edge contains the vertex) or -6, edge diag
// 32, adjacent edges 16, opposite edges 8}.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace gsw {

// products with an exact float constant (overloaded for double-word values)
template <typename T>
__device__ __forceinline__ T kmul(float c, T x) {
  return T(c) * x;
}
template <typename T>
__device__ __forceinline__ T kfma(float c, T x, T y) {
  return fma(T(c), x, y);
}
// Intermediate results consumed by the next operation at once: plain
// arithmetic for double and float; the double-word overloads skip the final
// renormalisation.
template <typename T>
__device__ __forceinline__ T add_u(T a, T b) {
  return a + b;
}
template <typename T>
__device__ __forceinline__ T sub_u(T a, T b) {
  return a - b;
}
template <typename T>
__device__ __forceinline__ T mul_u(T a, T b) {
  return a * b;
}
template <typename T>
__device__ __forceinline__ T fma_u(T a, T b, T c) {
  return fma(a, b, c);
}
template <typename T>
__device__ __forceinline__ T kfma_u(float c, T x, T y) {
  return fma(T(c), x, y);
}

// edge index of the vertex pair (a, b), VTK order 01, 12, 02, 03, 13, 23
__host__ __device__ constexpr int edge_of(int a, int b) {
  return (a + b == 1) ? 0 : (a + b == 3 ? (a * b == 2 ? 1 : 3) : (a + b == 2 ? 2 : (a + b == 4 ? 4 : 5)));
}
__host__ __device__ constexpr int edge_a(int e) { return e == 0 ? 0 : e == 1 ? 1 : e == 2 ? 0 : e == 3 ? 0 : e == 4 ? 1 : 2; }
__host__ __device__ constexpr int edge_b(int e) { return e == 0 ? 1 : e == 1 ? 2 : e == 2 ? 2 : e == 3 ? 3 : e == 4 ? 3 : 3; }
__host__ __device__ constexpr int edge_opp(int e) { return e == 0 ? 5 : e == 1 ? 3 : e == 2 ? 4 : e == 3 ? 1 : e == 4 ? 2 : 0; }

// T_km = S_k g_m (m = 0..3, g_0 = -(g_1 + g_2 + g_3)) at vertex k, from
// U[b] = u_k (b == k) or u_edge(k, b) and D0[m] = u_{m+1} - u_0:
// H_k = sum_{m=1..3} (4 (U[m] - U[0]) - D0[m-1]) (x) g_m, S_k its stress.
template <typename T>
__device__ __forceinline__ void vertex_traction(const T (&U)[4][3], const T (&D0)[3][3], const T (&g)[3][3],
                                                T lamS, T muS, T mu2S, T (&Tk)[4][3]) {
  T H[3][3];
#pragma unroll
  for (int m = 1; m < 4; ++m) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T E = kfma_u(4.0f, sub_u(U[m][i], U[0][i]), -D0[m - 1][i]);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (m == 1)
          H[i][j] = mul_u(E, g[0][j]);
        else if (m == 2)
          H[i][j] = fma_u(E, g[m - 1][j], H[i][j]);
        else
          H[i][j] = fma_u(E, g[m - 1][j], H[i][j]);
      }
    }
  }
  const T tr = add_u(add_u(H[0][0], H[1][1]), H[2][2]);
  const T lt = mul_u(lamS, tr);
  T S[3][3];
  S[0][0] = fma_u(mu2S, H[0][0], lt);
  S[1][1] = fma_u(mu2S, H[1][1], lt);
  S[2][2] = fma_u(mu2S, H[2][2], lt);
  S[0][1] = S[1][0] = mul_u(muS, add_u(H[0][1], H[1][0]));
  S[0][2] = S[2][0] = mul_u(muS, add_u(H[0][2], H[2][0]));
  S[1][2] = S[2][1] = mul_u(muS, add_u(H[1][2], H[2][1]));
#pragma unroll
  for (int m = 1; m < 4; ++m)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      Tk[m][i] = fma_u(S[i][0], g[m - 1][0], fma_u(S[i][1], g[m - 1][1], mul_u(S[i][2], g[m - 1][2])));
#pragma unroll
  for (int i = 0; i < 3; ++i) Tk[0][i] = -add_u(add_u(Tk[1][i], Tk[2][i]), Tk[3][i]);
}

// y = K' w, K' = the element stiffness with lam, mu pre-scaled (lamS = s lam
// V/20, muS = s mu V/20).  g[m] = grad L_{m+1}; grad L_0 = -(g0 + g1 + g2).
template <typename T>
__device__ __forceinline__ void stiffness_apply(const T (&w)[10][3], const T (&g)[3][3], T lamS, T muS,
                                                T (&y)[10][3]) {
  T D0[3][3];  // u_m - u_0, m = 1..3
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int i = 0; i < 3; ++i) D0[m][i] = w[m + 1][i] - w[0][i];
  T sumT[4][3], diagT[4][3], cross[6][3];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int i = 0; i < 3; ++i) sumT[m][i] = T(0);
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int i = 0; i < 3; ++i) cross[e][i] = T(0);
  const T mu2S = kmul(2.0f, muS);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T U[4][3], Tk[4][3];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int i = 0; i < 3; ++i) U[b][i] = (b == k) ? w[k][i] : w[4 + edge_of(k, b)][i];
    vertex_traction(U, D0, g, lamS, muS, mu2S, Tk);
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int i = 0; i < 3; ++i) sumT[m][i] += Tk[m][i];
#pragma unroll
    for (int i = 0; i < 3; ++i) diagT[k][i] = Tk[k][i];
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (b != k)
#pragma unroll
        for (int i = 0; i < 3; ++i) cross[edge_of(k, b)][i] += Tk[b][i];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) y[a][i] = kfma(4.0f, diagT[a][i], -sumT[a][i]);
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      y[4 + e][i] = kmul(4.0f, sumT[edge_a(e)][i] + sumT[edge_b(e)][i] + cross[e][i]);
}

// One displacement component: y += ms * P w (w, y: the 10 nodes' entries).
template <typename T>
__device__ __forceinline__ void mass_comp(const T (&w)[10], T ms, T (&y)[10]) {
  const T Xv = add_u(add_u(w[0], w[1]), add_u(w[2], w[3]));
  const T Xe = add_u(add_u(add_u(w[4], w[5]), add_u(w[6], w[7])), add_u(w[8], w[9]));
  const T tv = kfma_u(-6.0f, Xe, Xv);
  const T te = kfma_u(16.0f, Xe, kmul(-6.0f, Xv));
  // vertex a: 5 w_a + 2 (edges at a) + Xv - 6 Xe
  const T P0 = kfma_u(5.0f, w[0], kfma_u(2.0f, add_u(add_u(w[4], w[6]), w[7]), tv));
  const T P1 = kfma_u(5.0f, w[1], kfma_u(2.0f, add_u(add_u(w[4], w[5]), w[8]), tv));
  const T P2 = kfma_u(5.0f, w[2], kfma_u(2.0f, add_u(add_u(w[5], w[6]), w[9]), tv));
  const T P3 = kfma_u(5.0f, w[3], kfma_u(2.0f, add_u(add_u(w[7], w[8]), w[9]), tv));
  y[0] = fma_u(ms, P0, y[0]);
  y[1] = fma_u(ms, P1, y[1]);
  y[2] = fma_u(ms, P2, y[2]);
  y[3] = fma_u(ms, P3, y[3]);
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = edge_a(e), b = edge_b(e), o = edge_opp(e);
    const T P = kfma_u(2.0f, add_u(w[a], w[b]), kfma_u(16.0f, w[4 + e], kfma_u(-8.0f, w[4 + o], te)));
    y[4 + e] = fma_u(ms, P, y[4 + e]);
  }
}

// y += ms * P w with P the consistent-mass pattern (ms = s rho V / 420).
template <typename T>
__device__ __forceinline__ void mass_apply(const T (&w)[10][3], T ms, T (&y)[10][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T wi[10], yi[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      wi[k] = w[k][i];
      yi[k] = y[k][i];
    }
    mass_comp(wi, ms, yi);
#pragma unroll
    for (int k = 0; k < 10; ++k) y[k][i] = yi[k];
  }
}

// ---- FP32 specialisations on packed component pairs ------------------------
//
// Blackwell executes two FP32 operations per instruction on a float2
// (fma.rn.f32x2, add, mul).  The FP32 element operators therefore carry each
// 3-vector as (x, y) in a float2 plus z in a float: every component-wise
// operation is one packed and one scalar instruction instead of three.  The
// arithmetic is that of the generic templates above, each operation rounded
// once (round to nearest).
struct V3 {
  float2 xy;
  float z;
};
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ V3 v3_add(V3 a, V3 b) { return V3{__fadd2_rn(a.xy, b.xy), __fadd_rn(a.z, b.z)}; }
__device__ __forceinline__ V3 v3_sub(V3 a, V3 b) {
  return V3{__fadd2_rn(a.xy, make_float2(-b.xy.x, -b.xy.y)), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ V3 v3_scale(float s, V3 a) { return V3{__fmul2_rn(bc2(s), a.xy), __fmul_rn(s, a.z)}; }
// s a + c
__device__ __forceinline__ V3 v3_fma(float s, V3 a, V3 c) {
  return V3{__ffma2_rn(bc2(s), a.xy, c.xy), __fmaf_rn(s, a.z, c.z)};
}
__device__ __forceinline__ V3 v3_neg(V3 a) { return V3{make_float2(-a.xy.x, -a.xy.y), -a.z}; }
__device__ __forceinline__ V3 v3_zero() { return V3{make_float2(0.f, 0.f), 0.f}; }

template <>
__device__ __forceinline__ void stiffness_apply<float>(const float (&w3)[10][3], const float (&g)[3][3], float lamS,
                                                       float muS, float (&y3)[10][3]) {
  V3 w[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) w[k] = V3{make_float2(w3[k][0], w3[k][1]), w3[k][2]};
  V3 D0[3];  // u_m - u_0, m = 1..3
#pragma unroll
  for (int m = 0; m < 3; ++m) D0[m] = v3_sub(w[m + 1], w[0]);
  V3 sumT[4], diagT[4], cross[6];
#pragma unroll
  for (int m = 0; m < 4; ++m) sumT[m] = v3_zero();
#pragma unroll
  for (int e = 0; e < 6; ++e) cross[e] = v3_zero();
  const float mu2S = 2.0f * muS;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    V3 U[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) U[b] = (b == k) ? w[k] : w[4 + edge_of(k, b)];
    // column j of H_k over the displacement component i: Hc[j].i = H[i][j]
    V3 Hc[3];
#pragma unroll
    for (int m = 1; m < 4; ++m) {
      const V3 E = v3_fma(4.0f, v3_sub(U[m], U[0]), v3_neg(D0[m - 1]));
#pragma unroll
      for (int j = 0; j < 3; ++j) Hc[j] = (m == 1) ? v3_scale(g[0][j], E) : v3_fma(g[m - 1][j], E, Hc[j]);
    }
    const float tr = Hc[0].xy.x + Hc[1].xy.y + Hc[2].z;
    const float lt = lamS * tr;
    const float S00 = fmaf(mu2S, Hc[0].xy.x, lt), S11 = fmaf(mu2S, Hc[1].xy.y, lt), S22 = fmaf(mu2S, Hc[2].z, lt);
    const float S01 = muS * (Hc[1].xy.x + Hc[0].xy.y);
    const float S02 = muS * (Hc[2].xy.x + Hc[0].z);
    const float S12 = muS * (Hc[2].xy.y + Hc[1].z);
    // columns of the symmetric stress
    const V3 Sc0{make_float2(S00, S01), S02}, Sc1{make_float2(S01, S11), S12}, Sc2{make_float2(S02, S12), S22};
    V3 Tk[4];
#pragma unroll
    for (int m = 1; m < 4; ++m) Tk[m] = v3_fma(g[m - 1][0], Sc0, v3_fma(g[m - 1][1], Sc1, v3_scale(g[m - 1][2], Sc2)));
    Tk[0] = v3_neg(v3_add(v3_add(Tk[1], Tk[2]), Tk[3]));
#pragma unroll
    for (int m = 0; m < 4; ++m) sumT[m] = v3_add(sumT[m], Tk[m]);
    diagT[k] = Tk[k];
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (b != k) cross[edge_of(k, b)] = v3_add(cross[edge_of(k, b)], Tk[b]);
  }
  V3 y[10];
#pragma unroll
  for (int a = 0; a < 4; ++a) y[a] = v3_fma(4.0f, diagT[a], v3_neg(sumT[a]));
#pragma unroll
  for (int e = 0; e < 6; ++e) y[4 + e] = v3_scale(4.0f, v3_add(v3_add(sumT[edge_a(e)], sumT[edge_b(e)]), cross[e]));
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    y3[k][0] = y[k].xy.x;
    y3[k][1] = y[k].xy.y;
    y3[k][2] = y[k].z;
  }
}

template <>
__device__ __forceinline__ void mass_apply<float>(const float (&w3)[10][3], float ms, float (&y3)[10][3]) {
  V3 w[10], y[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    w[k] = V3{make_float2(w3[k][0], w3[k][1]), w3[k][2]};
    y[k] = V3{make_float2(y3[k][0], y3[k][1]), y3[k][2]};
  }
  const V3 Xv = v3_add(v3_add(w[0], w[1]), v3_add(w[2], w[3]));
  const V3 Xe = v3_add(v3_add(v3_add(w[4], w[5]), v3_add(w[6], w[7])), v3_add(w[8], w[9]));
  const V3 tv = v3_fma(-6.0f, Xe, Xv);
  const V3 te = v3_fma(16.0f, Xe, v3_scale(-6.0f, Xv));
  // vertex a: 5 w_a + 2 (edges at a) + Xv - 6 Xe
  const V3 P0 = v3_fma(5.0f, w[0], v3_fma(2.0f, v3_add(v3_add(w[4], w[6]), w[7]), tv));
  const V3 P1 = v3_fma(5.0f, w[1], v3_fma(2.0f, v3_add(v3_add(w[4], w[5]), w[8]), tv));
  const V3 P2 = v3_fma(5.0f, w[2], v3_fma(2.0f, v3_add(v3_add(w[5], w[6]), w[9]), tv));
  const V3 P3 = v3_fma(5.0f, w[3], v3_fma(2.0f, v3_add(v3_add(w[7], w[8]), w[9]), tv));
  y[0] = v3_fma(ms, P0, y[0]);
  y[1] = v3_fma(ms, P1, y[1]);
  y[2] = v3_fma(ms, P2, y[2]);
  y[3] = v3_fma(ms, P3, y[3]);
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = edge_a(e), b = edge_b(e), o = edge_opp(e);
    const V3 P = v3_fma(2.0f, v3_add(w[a], w[b]), v3_fma(16.0f, w[4 + e], v3_fma(-8.0f, w[4 + o], te)));
    y[4 + e] = v3_fma(ms, P, y[4 + e]);
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    y3[k][0] = y[k].xy.x;
    y3[k][1] = y[k].xy.y;
    y3[k][2] = y[k].z;
  }
}

}  // namespace gsw
