// FP64 kernels of the implicit finite-element wave analysis.
//
// Discretisation (Section 2, Eq. (1); Section 3, computational-cost
// paragraph): second-order (10-node) straight-sided tetrahedra, Newmark
// average acceleration, block-Jacobi preconditioned CG per step, Lysmer
// dashpots on base and sides with the input applied as a base force.
//
// Element-by-element operator.  For an affine quadratic tetrahedron with
// barycentric gradients g_m = grad L_m, the displacement gradient is linear:
// grad u = sum_k L_k H_k, with H_k (the gradient at vertex k)
//     H_k = 4 [ u_k (x) g_k + sum_{b != k} u_kb (x) g_b ] - sum_a u_a (x) g_a,
// so the stress is sigma = sum_k L_k S_k with S_k = lam tr(H_k) I + mu (H_k +
// H_k^T).  Integrating sigma . grad N exactly (int L_i L_j dV = V (1 + d_ij)/20)
// gives, with T_km = S_k g_m and T_m = sum_k T_km,
//     vertex a:     f_a  = V/20 (4 T_aa - T_a)
//     edge (a, b):  f_ab = V/5  (T_a + T_b + T_ab + T_ba).
// This costs ~520 FP64 operations per element instead of the ~1800 of a dense
// 30x30 product, which matters because the FP64 pipe is the bound on GB300.
// The consistent mass uses its closed-form pattern rho V / 420 {vertex diag 6,
// vertex-vertex 1, vertex-edge -4 (edge contains the vertex) or -6, edge diag
// 32, adjacent edges 16, opposite edges 8}.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsw_internal.cuh"
#include "gsw_dword.cuh"
#include "gsw_ebe.cuh"
#include "gsw_reduce.cuh"

namespace gsw {

// ------------------------------------------------------------------------------
// Setup kernels
// ------------------------------------------------------------------------------

__device__ __forceinline__ double unwrap(double x, double x0, double P) {
  return P > 0.0 ? x - P * rint((x - x0) / P) : x;
}

__global__ void geometry_kernel(ModelView m, const double* __restrict__ xyz, double px, double py,
                                double* __restrict__ geo, int* err) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  double X[10][3];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const int64_t n = m.conn[k * m.E + e];
    X[k][0] = xyz[3 * n];
    X[k][1] = xyz[3 * n + 1];
    X[k][2] = xyz[3 * n + 2];
  }
#pragma unroll
  for (int k = 1; k < 10; ++k) {
    X[k][0] = unwrap(X[k][0], X[0][0], px);
    X[k][1] = unwrap(X[k][1], X[0][1], py);
  }
  double c1[3], c2[3], c3[3];
  for (int i = 0; i < 3; ++i) {
    c1[i] = X[1][i] - X[0][i];
    c2[i] = X[2][i] - X[0][i];
    c3[i] = X[3][i] - X[0][i];
  }
  // rows of J^{-1} for J = [c1 c2 c3] are (c2 x c3, c3 x c1, c1 x c2) / det
  double r1[3] = {c2[1] * c3[2] - c2[2] * c3[1], c2[2] * c3[0] - c2[0] * c3[2], c2[0] * c3[1] - c2[1] * c3[0]};
  double r2[3] = {c3[1] * c1[2] - c3[2] * c1[1], c3[2] * c1[0] - c3[0] * c1[2], c3[0] * c1[1] - c3[1] * c1[0]};
  double r3[3] = {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2], c1[0] * c2[1] - c1[1] * c2[0]};
  const double det = c1[0] * r1[0] + c1[1] * r1[1] + c1[2] * r1[2];
  if (!(det > 0.0) || !isfinite(det)) atomicOr(err, 1);
  // straight sides: mid-edge nodes at the edge midpoints
  double hmax = 0.0, dev = 0.0;
#pragma unroll
  for (int ed = 0; ed < 6; ++ed) {
    const int a = edge_a(ed), b = edge_b(ed);
    for (int i = 0; i < 3; ++i) {
      const double mid = 0.5 * (X[a][i] + X[b][i]);
      dev = fmax(dev, fabs(X[4 + ed][i] - mid));
      hmax = fmax(hmax, fabs(X[a][i] - X[b][i]));
    }
  }
  if (!(dev <= 1e-9 * hmax)) atomicOr(err, 2);
  const double inv = 1.0 / det;
  for (int i = 0; i < 3; ++i) {
    geo[(0 + i) * m.E + e] = r1[i] * inv;
    geo[(3 + i) * m.E + e] = r2[i] * inv;
    geo[(6 + i) * m.E + e] = r3[i] * inv;
  }
  geo[9 * m.E + e] = det / 6.0;
}

__global__ void face_geometry_kernel(ModelView m, const double* __restrict__ xyz, double px, double py,
                                     const int32_t* __restrict__ face_elem,
                                     const int32_t* __restrict__ face_tag, double* __restrict__ fgeo,
                                     int* err) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= m.F) return;
  double X[6][3];
  for (int k = 0; k < 6; ++k) {
    const int64_t n = m.fnode[k * m.F + f];
    for (int i = 0; i < 3; ++i) X[k][i] = xyz[3 * n + i];
    X[k][0] = unwrap(X[k][0], X[0][0], px);
    X[k][1] = unwrap(X[k][1], X[0][1], py);
  }
  double a[3], b[3];
  for (int i = 0; i < 3; ++i) {
    a[i] = X[1][i] - X[0][i];
    b[i] = X[2][i] - X[0][i];
  }
  double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const double nrm = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(err, 4);
  const double area = 0.5 * nrm;
  const MatCoef mc = m.mat[m.emat[face_elem[f]]];
  const double zs = mc.rho * mc.Vs, zp = mc.rho * mc.Vp;
  fgeo[0 * m.F + f] = area * zs;
  fgeo[1 * m.F + f] = area * (zp - zs);
  fgeo[2 * m.F + f] = c[0] / nrm;
  fgeo[3 * m.F + f] = c[1] / nrm;
  fgeo[4 * m.F + f] = c[2] / nrm;
  fgeo[5 * m.F + f] = (double)face_tag[f];
}

// Rayleigh coefficients: least-squares fit of alpha/(4 pi f) + beta pi f to h
// over [f1, f2], from the closed-form integrals of the normal equations.
__global__ void material_kernel(MatCoef* mat, const double* raw, int n_mat, double dt, double f1,
                                double f2) {
  const int i = threadIdx.x;
  if (i >= n_mat) return;
  const double Vp = raw[4 * i], Vs = raw[4 * i + 1], rho = raw[4 * i + 2], h = raw[4 * i + 3];
  MatCoef c;
  c.Vp = Vp;
  c.Vs = Vs;
  c.rho = rho;
  c.h = h;
  c.mu = rho * Vs * Vs;
  c.lam = rho * Vp * Vp - 2.0 * c.mu;
  c.alpha = c.beta = 0.0;
  c.cK = c.cM = 0.0;
  if (dt > 0.0) {
    const double pi = 3.14159265358979323846;
    const double g11 = (1.0 / f1 - 1.0 / f2) / (16.0 * pi * pi);
    const double g12 = 0.25 * (f2 - f1);
    const double g22 = pi * pi * (f2 * f2 * f2 - f1 * f1 * f1) / 3.0;
    const double r1 = h * log(f2 / f1) / (4.0 * pi);
    const double r2 = h * pi * (f2 * f2 - f1 * f1) / 2.0;
    const double det = g11 * g22 - g12 * g12;
    c.alpha = (g22 * r1 - g12 * r2) / det;
    c.beta = (g11 * r2 - g12 * r1) / det;
    c.cK = 1.0 + 2.0 * c.beta / dt;
    c.cM = 4.0 / (dt * dt) + 2.0 * c.alpha / dt;
  }
  mat[i] = c;
}

// Diagonal 3x3 nodal blocks of A: per element, K_aa = (lam + mu) G + mu tr(G) I
// with G = int grad N_a grad N_a^T dV (vertex: 3V/5 g_a g_a^T; edge (a,b):
// 8V/5 (g_a g_a^T + g_b g_b^T) + 4V/5 (g_a g_b^T + g_b g_a^T)), M_aa = rho V
// (6 or 32)/420 I; per absorbing face (2/dt) A (6 or 32)/180 T.
__global__ void diag_blocks_kernel(ModelView m, double* __restrict__ dblk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m.E) {
    const int64_t e = t;
    double g[4][3];
    for (int i = 0; i < 3; ++i) {
      g[1][i] = m.geo[(0 + i) * m.E + e];
      g[2][i] = m.geo[(3 + i) * m.E + e];
      g[3][i] = m.geo[(6 + i) * m.E + e];
      g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
    }
    const double V = m.geo[9 * m.E + e];
    const MatCoef mc = m.mat[m.emat[e]];
    const double kl = mc.cK * (mc.lam + mc.mu), km = mc.cK * mc.mu;
    for (int k = 0; k < 10; ++k) {
      double G[3][3];
      if (k < 4) {
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) G[i][j] = 0.6 * V * g[k][i] * g[k][j];
      } else {
        const int a = edge_a(k - 4), b = edge_b(k - 4);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            G[i][j] = 1.6 * V * (g[a][i] * g[a][j] + g[b][i] * g[b][j]) +
                      0.8 * V * (g[a][i] * g[b][j] + g[b][i] * g[a][j]);
      }
      const double tr = G[0][0] + G[1][1] + G[2][2];
      const double md = mc.cM * mc.rho * V * (k < 4 ? 6.0 : 32.0) / 420.0;
      const int64_t n = m.conn[k * m.E + e];
      double* d = dblk + 6 * n;
      atomicAdd(d + 0, kl * G[0][0] + km * tr + md);
      atomicAdd(d + 1, kl * G[1][1] + km * tr + md);
      atomicAdd(d + 2, kl * G[2][2] + km * tr + md);
      atomicAdd(d + 3, kl * G[0][1]);
      atomicAdd(d + 4, kl * G[0][2]);
      atomicAdd(d + 5, kl * G[1][2]);
    }
  } else if (t < m.E + m.F) {
    const int64_t f = t - m.E;
    const double tag = m.fgeo[5 * m.F + f];
    if (tag < 0.5) return;  // free surface
    const double As = m.fgeo[f], Ad = m.fgeo[m.F + f];
    const double n0 = m.fgeo[2 * m.F + f], n1 = m.fgeo[3 * m.F + f], n2 = m.fgeo[4 * m.F + f];
    const double s = 2.0 / m.dt;
    for (int k = 0; k < 6; ++k) {
      const double w = s * (k < 3 ? 6.0 : 32.0) / 180.0;
      const int64_t n = m.fnode[k * m.F + f];
      double* d = dblk + 6 * n;
      atomicAdd(d + 0, w * (As + Ad * n0 * n0));
      atomicAdd(d + 1, w * (As + Ad * n1 * n1));
      atomicAdd(d + 2, w * (As + Ad * n2 * n2));
      atomicAdd(d + 3, w * Ad * n0 * n1);
      atomicAdd(d + 4, w * Ad * n0 * n2);
      atomicAdd(d + 5, w * Ad * n1 * n2);
    }
  }
}

// Diagonal 3x3 blocks of P^T A P at the vertices, P the interpolation from
// vertex values to the quadratic nodes.  On straight-sided elements the
// vertex's linear hat function is N_a + 1/2 sum_b N_ab, so the blocks are those
// of the linear (4-node) tetrahedron: K_aa = (lam + mu) G + mu tr(G) I with
// G = V g_a g_a^T, M_aa = rho V / 10 I, and per absorbing face the linear
// triangle's (2/dt) (area / 6) T.
__global__ void coarse_blocks_kernel(ModelView m, const int32_t* __restrict__ vid, double* __restrict__ cblk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m.E) {
    const int64_t e = t;
    double g[4][3];
    for (int i = 0; i < 3; ++i) {
      g[1][i] = m.geo[(0 + i) * m.E + e];
      g[2][i] = m.geo[(3 + i) * m.E + e];
      g[3][i] = m.geo[(6 + i) * m.E + e];
      g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
    }
    const double V = m.geo[9 * m.E + e];
    const MatCoef mc = m.mat[m.emat[e]];
    const double kl = mc.cK * (mc.lam + mc.mu) * V, km = mc.cK * mc.mu * V;
    const double md = mc.cM * mc.rho * V / 10.0;
    for (int k = 0; k < 4; ++k) {
      const double tr = g[k][0] * g[k][0] + g[k][1] * g[k][1] + g[k][2] * g[k][2];
      double* d = cblk + 6 * (int64_t)vid[m.conn[k * m.E + e]];
      atomicAdd(d + 0, kl * g[k][0] * g[k][0] + km * tr + md);
      atomicAdd(d + 1, kl * g[k][1] * g[k][1] + km * tr + md);
      atomicAdd(d + 2, kl * g[k][2] * g[k][2] + km * tr + md);
      atomicAdd(d + 3, kl * g[k][0] * g[k][1]);
      atomicAdd(d + 4, kl * g[k][0] * g[k][2]);
      atomicAdd(d + 5, kl * g[k][1] * g[k][2]);
    }
  } else if (t < m.E + m.F) {
    const int64_t f = t - m.E;
    if (m.fgeo[5 * m.F + f] < 0.5) return;  // free surface
    const double As = m.fgeo[f], Ad = m.fgeo[m.F + f];
    const double n0 = m.fgeo[2 * m.F + f], n1 = m.fgeo[3 * m.F + f], n2 = m.fgeo[4 * m.F + f];
    const double w = 2.0 / m.dt / 6.0;
    for (int k = 0; k < 3; ++k) {
      double* d = cblk + 6 * (int64_t)vid[m.fnode[k * m.F + f]];
      atomicAdd(d + 0, w * (As + Ad * n0 * n0));
      atomicAdd(d + 1, w * (As + Ad * n1 * n1));
      atomicAdd(d + 2, w * (As + Ad * n2 * n2));
      atomicAdd(d + 3, w * Ad * n0 * n1);
      atomicAdd(d + 4, w * Ad * n0 * n2);
      atomicAdd(d + 5, w * Ad * n1 * n2);
    }
  }
}

__global__ void invert_blocks_kernel(int64_t N, const double* __restrict__ dblk,
                                     double* __restrict__ dinv, int* err) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    const double* d = dblk + 6 * n;
    const double a = d[0], b = d[1], c = d[2], xy = d[3], xz = d[4], yz = d[5];
    const double i00 = b * c - yz * yz, i11 = a * c - xz * xz, i22 = a * b - xy * xy;
    const double i01 = xz * yz - xy * c, i02 = xy * yz - xz * b, i12 = xy * xz - a * yz;
    const double det = a * i00 + xy * i01 + xz * i02;
    if (!(det > 0.0) || !isfinite(det)) atomicOr(err, 8);
    const double s = 1.0 / det;
    double* o = dinv + 6 * n;
    o[0] = i00 * s;
    o[1] = i11 * s;
    o[2] = i22 * s;
    o[3] = i01 * s;
    o[4] = i02 * s;
    o[5] = i12 * s;
  }
}

// Receivers: the lowest-numbered free-surface face whose horizontal projection
// contains the point (barycentric coordinates >= -1e-10), then the 6-node
// triangle's shape functions there.
__global__ void receiver_find_kernel(ModelView m, const double* __restrict__ xyz, double px,
                                     double py, const double* __restrict__ rec_xy,
                                     int32_t* rec_face) {
  const int r = blockIdx.x;
  const double qx0 = rec_xy[2 * r], qy0 = rec_xy[2 * r + 1];
  for (int64_t f = threadIdx.x; f < m.F; f += blockDim.x) {
    if (m.fgeo[5 * m.F + f] != 0.0) continue;
    double x[3], y[3];
    for (int k = 0; k < 3; ++k) {
      const int64_t n = m.fnode[k * m.F + f];
      x[k] = xyz[3 * n];
      y[k] = xyz[3 * n + 1];
    }
    x[1] = unwrap(x[1], x[0], px);
    x[2] = unwrap(x[2], x[0], px);
    y[1] = unwrap(y[1], y[0], py);
    y[2] = unwrap(y[2], y[0], py);
    const double qx = unwrap(qx0, x[0], px), qy = unwrap(qy0, y[0], py);
    const double ax = x[1] - x[0], ay = y[1] - y[0], bx = x[2] - x[0], by = y[2] - y[0];
    const double det = ax * by - bx * ay;
    const double dx = qx - x[0], dy = qy - y[0];
    const double l1 = (dx * by - bx * dy) / det, l2 = (ax * dy - dx * ay) / det;
    const double l0 = 1.0 - l1 - l2;
    if (l0 >= -1e-10 && l1 >= -1e-10 && l2 >= -1e-10) atomicMin(rec_face + r, (int32_t)f);
  }
}

__global__ void receiver_weights_kernel(ModelView m, const double* __restrict__ xyz, double px,
                                        double py, const double* __restrict__ rec_xy, int n_rec,
                                        const int32_t* __restrict__ rec_face, int32_t* rec_node,
                                        double* rec_w, int* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rec) return;
  const int32_t f = rec_face[r];
  if (f < 0 || f >= m.F) {
    atomicOr(err, 16);
    for (int k = 0; k < 6; ++k) {
      rec_node[6 * r + k] = 0;
      rec_w[6 * r + k] = 0.0;
    }
    return;
  }
  double x[3], y[3];
  int64_t nd[6];
  for (int k = 0; k < 6; ++k) nd[k] = m.fnode[k * m.F + f];
  for (int k = 0; k < 3; ++k) {
    x[k] = xyz[3 * nd[k]];
    y[k] = xyz[3 * nd[k] + 1];
  }
  x[1] = unwrap(x[1], x[0], px);
  x[2] = unwrap(x[2], x[0], px);
  y[1] = unwrap(y[1], y[0], py);
  y[2] = unwrap(y[2], y[0], py);
  const double qx = unwrap(rec_xy[2 * r], x[0], px), qy = unwrap(rec_xy[2 * r + 1], y[0], py);
  const double ax = x[1] - x[0], ay = y[1] - y[0], bx = x[2] - x[0], by = y[2] - y[0];
  const double det = ax * by - bx * ay;
  const double dx = qx - x[0], dy = qy - y[0];
  const double L1 = (dx * by - bx * dy) / det, L2 = (ax * dy - dx * ay) / det;
  const double L[3] = {1.0 - L1 - L2, L1, L2};
  double w[6];
  for (int a = 0; a < 3; ++a) w[a] = L[a] * (2.0 * L[a] - 1.0);
  w[3] = 4.0 * L[0] * L[1];
  w[4] = 4.0 * L[1] * L[2];
  w[5] = 4.0 * L[2] * L[0];
  for (int k = 0; k < 6; ++k) {
    rec_node[6 * r + k] = (int32_t)nd[k];
    rec_w[6 * r + k] = w[k];
  }
}

// ------------------------------------------------------------------------------
// Element-by-element operator
// ------------------------------------------------------------------------------

// Dashpot faces (threads E <= t < E + F) of the element-by-element operator,
// FP64: the face term of A (scaled by 2/dt) in kModeA, the damping force of
// the velocity plus the base force in kModeRhs / kModeRes.
template <int MODE, bool DWIN = false>
__device__ __forceinline__ void face_apply(const ModelView& m, int64_t fc, const double* __restrict__ x,
                                           const double* __restrict__ vv, double force, int dir, double* y,
                                           double& dot) {
  const double tag = m.fgeo[5 * m.F + fc];
  if (tag > 0.5) {
    const double sc = (MODE == kModeA) ? 2.0 / m.dt : 1.0;
    const double As = sc * m.fgeo[fc] / 180.0, Ad = sc * m.fgeo[m.F + fc] / 180.0;
    const double n[3] = {m.fgeo[2 * m.F + fc], m.fgeo[3 * m.F + fc], m.fgeo[4 * m.F + fc]};
    int64_t nd[6];
    double z[6][3], xin[6][3];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      nd[k] = m.fnode[k * m.F + fc];
      const double* src = (MODE == kModeRhs || MODE == kModeRes) ? vv : x;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (DWIN) {  // v~ stored as double-word pairs
          const float2 c = reinterpret_cast<const float2*>(src)[3 * nd[k] + i];
          xin[k][i] = to_double(dw(c.x, c.y));
        } else {
          xin[k][i] = src[3 * nd[k] + i];
        }
      }
      const double dn = n[0] * xin[k][0] + n[1] * xin[k][1] + n[2] * xin[k][2];
#pragma unroll
      for (int i = 0; i < 3; ++i) z[k][i] = fma(As, xin[k][i], Ad * dn * n[i]);
    }
    double yf[6][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double Zv = z[0][i] + z[1][i] + z[2][i];
      const double Ze = z[3][i] + z[4][i] + z[5][i];
      // vertex a: 7 z_a - Zv - 4 z_(opposite edge); edge e: 16 z_e + 16 Ze - 4 z_(opposite vertex)
      yf[0][i] = 7.0 * z[0][i] - Zv - 4.0 * z[4][i];
      yf[1][i] = 7.0 * z[1][i] - Zv - 4.0 * z[5][i];
      yf[2][i] = 7.0 * z[2][i] - Zv - 4.0 * z[3][i];
      yf[3][i] = 16.0 * (z[3][i] + Ze) - 4.0 * z[2][i];
      yf[4][i] = 16.0 * (z[4][i] + Ze) - 4.0 * z[0][i];
      yf[5][i] = 16.0 * (z[5][i] + Ze) - 4.0 * z[1][i];
    }
    if ((MODE == kModeRhs || MODE == kModeRes) && tag < 1.5) {
      // base force 2 p C_base e_dir: int N_a dA = A/3 at edge nodes, 0 at vertices
      const double nd_ = dir == 0 ? n[0] : (dir == 1 ? n[1] : n[2]);
      const double Af = m.fgeo[fc] / 180.0, Adf = m.fgeo[m.F + fc] / 180.0;
      const double fz[3] = {Af * (dir == 0) + Adf * nd_ * n[0], Af * (dir == 1) + Adf * nd_ * n[1],
                            Af * (dir == 2) + Adf * nd_ * n[2]};
#pragma unroll
      for (int k = 3; k < 6; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) yf[k][i] += force * 60.0 * fz[i];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        atomicAdd(y + 3 * nd[k] + i, yf[k][i]);
        if (MODE == kModeA) dot = fma(xin[k][i], yf[k][i], dot);
      }
  }
}

// One thread per element (t < E) or boundary face (E <= t < E + F).
//   kModeA   y = A x               (+ partial x.y when partials != nullptr)
//   kModeK   y = K x,  kModeM y = M x,  kModeC y = C x
//   kModeRhs y = f - K u + C v + M (a + (4/dt) v)  with x = u
//   kModeRes y = f - K u~ + C v~ + M a~  with x = u~ = u + du0,
//            vv = v~ = v - (2/dt) du0, aa = a~ = a + (4/dt) v - (4/dt^2) du0:
//            the Newmark residual b - A du0 at an initial guess du0 from a
//            single stiffness application
template <int MODE>
__global__ void __launch_bounds__(kElemThreads) ebe_kernel(ModelView m, const double* __restrict__ x,
                                                            const double* __restrict__ vv,
                                                            const double* __restrict__ aa, double* y,
                                                            double force, int dir, double* partials,
                                                            CgScalars* cg, Drive dr) {
  if (cg != nullptr && ((volatile CgScalars*)cg)->done) return;
  if (dr.ss != nullptr) {
    if (!((volatile StepState*)dr.ss)->active) return;
    force = 2.0 * dr.p[dr.ss->step];
  }
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dot = 0.0;
  if (t < m.E) {
    const int64_t e = t;
    int64_t nd[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) nd[k] = m.conn[k * m.E + e];
    double g[3][3];
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
#pragma unroll
      for (int i = 0; i < 3; ++i) g[mm][i] = __ldg(m.geo + (3 * mm + i) * m.E + e);
    const double V = __ldg(m.geo + 9 * m.E + e);
    const MatCoef mc = m.mat[m.emat[e]];
    double ks, ms;  // stiffness and mass scales
    if (MODE == kModeA) {
      ks = mc.cK;
      ms = mc.cM;
    } else if (MODE == kModeK) {
      ks = 1.0;
      ms = 0.0;
    } else if (MODE == kModeM) {
      ks = 0.0;
      ms = 1.0;
    } else if (MODE == kModeC) {
      ks = mc.beta;
      ms = mc.alpha;
    } else if (MODE == kModeRes) {
      ks = -1.0;
      ms = 1.0;
    } else {
      ks = 1.0;
      ms = 1.0;
    }
    const double lamS = ks * mc.lam * V * (1.0 / 20.0), muS = ks * mc.mu * V * (1.0 / 20.0);
    const double mS = ms * mc.rho * V * (1.0 / 420.0);
    double w[10][3], f[10][3];
    if (MODE == kModeRhs) {
      // stiffness acts on -u + beta v
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[k][i] = fma(mc.beta, vv[3 * nd[k] + i], -x[3 * nd[k] + i]);
    } else if (MODE == kModeRes) {
      // residual at the initial guess: stiffness acts on u~ - beta v~ (x = u~, vv = v~)
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[k][i] = fma(-mc.beta, vv[3 * nd[k] + i], x[3 * nd[k] + i]);
    } else {
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[k][i] = x[3 * nd[k] + i];
    }
    if (MODE != kModeM) {
      stiffness_apply(w, g, lamS, muS, f);
    } else {
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) f[k][i] = 0.0;
    }
    if (MODE == kModeRhs || MODE == kModeRes) {
      // mass acts on a + (4/dt + alpha) v (right-hand side) or a~ + alpha v~ (residual)
      const double cv = (MODE == kModeRhs) ? 4.0 / m.dt + mc.alpha : mc.alpha;
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[k][i] = fma(cv, vv[3 * nd[k] + i], aa[3 * nd[k] + i]);
    }
    if (MODE != kModeK) mass_apply(w, mS, f);
#pragma unroll
    for (int k = 0; k < 10; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        atomicAdd(y + 3 * nd[k] + i, f[k][i]);
        if (MODE == kModeA) dot = fma(w[k][i], f[k][i], dot);
      }
  } else if (t < m.E + m.F && MODE != kModeK && MODE != kModeM) {
    face_apply<MODE>(m, t - m.E, x, vv, force, dir, y, dot);
  }
  if (MODE == kModeA && partials != nullptr) {
    double vals[1] = {dot}, out[1];
    if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) cg->pq = out[0];
  }
}

// The same operator for the flexible CG's outer iteration in double-word
// arithmetic (gsw_dword.cuh): y = A x with the partial x . A x (kModeA), or
// the residual at the initial guess (kModeRes).  Element data and state are
// FP64 in memory; each element converts its inputs to double-word values
// (bit operations), applies the same stiffness and mass formulas on the FP32
// pipe and adds its 30 results to y as doubles.  Dashpot faces stay FP64.
//
// Double-word code is about ten FP32 instructions per FP64 operation, so the
// element is laid out to keep the kernel's code and registers small: the
// element's inputs and its per-vertex sums live in shared memory (one slot
// column per thread), the four vertices run through one loop body (the
// vertex's nodes are picked by index) and so do the three displacement
// components of the output and mass stage.
constexpr int kDwSlotW = 0;      // [30] stiffness input w, node k component i at 3k + i
constexpr int kDwSlotDiag = 30;  // [12] 4 T_aa, vertex a
constexpr int kDwSlotCross = 42; // [18] T_ab + T_ba, edge (a, b)
constexpr int kDwSlots = 60;
constexpr int kDwMinBlocks = 3;
constexpr size_t kDwSmem = sizeof(float2) * kDwSlots * kElemThreads;

template <int MODE, bool DWIN>
__global__ void __launch_bounds__(kElemThreads, kDwMinBlocks)
    ebe_dw_kernel(ModelView m, const double* __restrict__ x, const double* __restrict__ vv,
                  const double* __restrict__ aa, double* y, double force, int dir, double* partials,
                  CgScalars* cg, Drive dr) {
  static_assert(MODE == kModeA || MODE == kModeRes, "double-word operator: kModeA or kModeRes");
  static_assert(MODE == kModeA || DWIN, "the residual pass reads double-word inputs");
  extern __shared__ float2 dsm[];  // [kDwSlots][kElemThreads]
  // DWIN: the inputs arrive as double-word pairs (float2): the search
  // direction (fcg kernels) or u~, v~, a~ (cg_init_mixed_kernel)
  const float2* __restrict__ x2 = reinterpret_cast<const float2*>(x);
  const float2* __restrict__ v2 = reinterpret_cast<const float2*>(vv);
  const float2* __restrict__ a2 = reinterpret_cast<const float2*>(aa);
  if (cg != nullptr && ((volatile CgScalars*)cg)->done) return;
  if (dr.ss != nullptr) {
    if (!((volatile StepState*)dr.ss)->active) return;
    force = 2.0 * dr.p[dr.ss->step];
  }
  float2* sl = dsm + threadIdx.x;
  auto ld = [&](int q) {
    const float2 v = sl[q * kElemThreads];
    return dw(v.x, v.y);
  };
  auto st = [&](int q, dw v) { sl[q * kElemThreads] = make_float2(v.hi, v.lo); };
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dot = 0.0;
  if (t < m.E) {
    const int64_t e = t;
    int32_t nd[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) nd[k] = m.conn[k * m.E + e];
    const MatCoef mc = m.mat[m.emat[e]];
    // stiffness input: x (kModeA) or u~ - beta v~ (kModeRes)
    const dw nbeta = to_dw(-mc.beta);
    // two halves of five nodes: each half's gathers are issued together
#pragma unroll 1
    for (int h = 0; h < 10; h += 5) {
      if (DWIN) {
        float2 xs[5][3], vs[5][3];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int64_t n3 = 3 * (int64_t)m.conn[(h + k) * m.E + e];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            xs[k][i] = x2[n3 + i];
            if (MODE == kModeRes) vs[k][i] = v2[n3 + i];
          }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const dw xd(xs[k][i].x, xs[k][i].y);
            st(kDwSlotW + 3 * (h + k) + i,
               MODE == kModeRes ? fma_u(nbeta, dw(vs[k][i].x, vs[k][i].y), xd) : xd);
          }
      } else {
        double xs[5][3];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int64_t n3 = 3 * (int64_t)m.conn[(h + k) * m.E + e];
#pragma unroll
          for (int i = 0; i < 3; ++i) xs[k][i] = x[n3 + i];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
          for (int i = 0; i < 3; ++i) st(kDwSlotW + 3 * (h + k) + i, to_dw(xs[k][i]));
      }
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) st(kDwSlotCross + q, dw(0));
    dw g[3][3];
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
#pragma unroll
      for (int i = 0; i < 3; ++i) g[mm][i] = to_dw(__ldg(m.geo + (3 * mm + i) * m.E + e));
    const double V = __ldg(m.geo + 9 * m.E + e);
    const double ks = (MODE == kModeA) ? mc.cK : -1.0;
    const double ms = (MODE == kModeA) ? mc.cM : 1.0;
    const dw lamS = to_dw(ks * mc.lam * V * (1.0 / 20.0)), muS = to_dw(ks * mc.mu * V * (1.0 / 20.0));
    const dw mu2S = kmul(2.0f, muS);
    const dw mS = to_dw(ms * mc.rho * V * (1.0 / 420.0));
    dw D0[3][3];
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
#pragma unroll
      for (int i = 0; i < 3; ++i) D0[mm][i] = sub_u(ld(kDwSlotW + 3 * (mm + 1) + i), ld(kDwSlotW + i));
    dw sumT[4][3];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm)
#pragma unroll
      for (int i = 0; i < 3; ++i) sumT[mm][i] = dw(0);
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      dw U[4][3], Tk[4][3];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int nb = (b == k) ? k : 4 + edge_of(k, b);
#pragma unroll
        for (int i = 0; i < 3; ++i) U[b][i] = ld(kDwSlotW + 3 * nb + i);
      }
      vertex_traction(U, D0, g, lamS, muS, mu2S, Tk);
#pragma unroll
      for (int mm = 0; mm < 4; ++mm)
#pragma unroll
        for (int i = 0; i < 3; ++i) sumT[mm][i] = add_u(sumT[mm][i], Tk[mm][i]);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b == k) {
#pragma unroll
          for (int i = 0; i < 3; ++i) st(kDwSlotDiag + 3 * b + i, kmul(4.0f, Tk[b][i]));
        } else {
          const int q = kDwSlotCross + 3 * edge_of(k, b);
#pragma unroll
          for (int i = 0; i < 3; ++i) st(q + i, add_u(ld(q + i), Tk[b][i]));
        }
      }
    }
    // per component: vertex a 4 T_aa - T_a, edge (a, b) 4 (T_a + T_b + T_ab + T_ba), plus the mass
    const dw ca = to_dw(mc.alpha);
    dw dd(0);
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
      dw sT[4], yi[10], wi[10];
#pragma unroll
      for (int a = 0; a < 4; ++a) sT[a] = i == 0 ? sumT[a][0] : (i == 1 ? sumT[a][1] : sumT[a][2]);
#pragma unroll
      for (int a = 0; a < 4; ++a) yi[a] = sub_u(ld(kDwSlotDiag + 3 * a + i), sT[a]);
#pragma unroll
      for (int q = 0; q < 6; ++q)
        yi[4 + q] = kmul(4.0f, add_u(add_u(sT[edge_a(q)], sT[edge_b(q)]), ld(kDwSlotCross + 3 * q + i)));
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        // mass input: x (kModeA) or a~ + alpha v~ (kModeRes)
        const int64_t q = 3 * (int64_t)nd[k] + i;
        if (MODE == kModeRes) {
          const float2 vq = v2[q], aq = a2[q];
          wi[k] = fma_u(ca, dw(vq.x, vq.y), dw(aq.x, aq.y));
        } else {
          wi[k] = ld(kDwSlotW + 3 * k + i);
        }
      }
      mass_comp(wi, mS, yi);
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        atomicAdd(y + 3 * (int64_t)nd[k] + i, to_double(yi[k]));
        if (MODE == kModeA) dd = fma_u(wi[k], yi[k], dd);
      }
    }
    if (MODE == kModeA) dot = to_double(dd);
  } else if (t < m.E + m.F) {
    face_apply<MODE, DWIN>(m, t - m.E, x, vv, force, dir, y, dot);
  }
  if (MODE == kModeA && partials != nullptr) {
    double vals[1] = {dot}, out[1];
    if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) cg->pq = out[0];
  }
}

// ------------------------------------------------------------------------------
// CG vector kernels (node-wise, 3 DOF per thread, grid-stride)
// ------------------------------------------------------------------------------

__device__ __forceinline__ void apply_dinv(const double* __restrict__ d, const double r[3], double z[3]) {
  z[0] = d[0] * r[0] + d[3] * r[1] + d[4] * r[2];
  z[1] = d[3] * r[0] + d[1] * r[1] + d[5] * r[2];
  z[2] = d[4] * r[0] + d[5] * r[1] + d[2] * r[2];
}

__global__ void cg_init_kernel(int64_t N, const double* __restrict__ b, const double* __restrict__ v,
                               const double* __restrict__ a, double dt, double* __restrict__ x,
                               double* __restrict__ q, double* partials, CgScalars* cg, int use_guess,
                               const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  double bb = 0.0;
  const double h = 0.5 * dt * dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    bb = fma(bi, bi, bb);
    double x0 = fma(dt, v[i], h * a[i]);
    if (use_guess) {
      const double g = x[i];
      if (isfinite(g)) x0 = g;  // a non-finite guess falls back to the predictor
    }
    x[i] = x0;
    q[i] = 0.0;
  }
  double vals[1] = {bb}, out[1];
  if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->bb = out[0];
    cg->iter = 0;
    cg->status = 0;
    cg->relres = 0.0;
    cg->zero_rhs = (out[0] == 0.0);
    cg->done = (out[0] == 0.0);
    if (!isfinite(out[0])) {
      cg->status = -5;
      cg->done = 1;
    }
  }
}

// Mixed-mode start of a step: ||b||^2 from the FP32 right-hand side, the
// initial guess du0 (the predictor dt v + dt^2/2 a, or the value already in x),
// and the shifted state u~ = u + du0, v~ = v - (2/dt) du0,
// a~ = a + (4/dt) v - (4/dt^2) du0 read by the single-pass residual; r = q = 0.
// With dw_out the shifted state is stored as double-word pairs (float2, the
// same 8 bytes) for the double-word residual kernel.
__global__ void cg_init_mixed_kernel(int64_t N, const float* __restrict__ b32, const double* __restrict__ u,
                                     const double* __restrict__ v, const double* __restrict__ a, double dt,
                                     double* __restrict__ x, double* __restrict__ ut, double* __restrict__ vt,
                                     double* __restrict__ at, double* __restrict__ r, double* __restrict__ q,
                                     double* partials, CgScalars* cg, const StepState* ss, int use_guess,
                                     int dw_out) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  double bb = 0.0;
  const double h = 0.5 * dt * dt, c2 = 2.0 / dt, c4 = 4.0 / dt, c44 = 4.0 / (dt * dt);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = (double)b32[i];
    bb = fma(bi, bi, bb);
    const double vi = v[i], ai = a[i];
    double x0 = fma(dt, vi, h * ai);
    if (use_guess) {
      const double g = x[i];
      if (isfinite(g)) x0 = g;  // a non-finite guess falls back to the predictor
    }
    x[i] = x0;
    const double uti = u[i] + x0, vti = fma(-c2, x0, vi), ati = fma(-c44, x0, fma(c4, vi, ai));
    if (dw_out) {
      const dw a2 = to_dw(uti), b2 = to_dw(vti), c3 = to_dw(ati);
      reinterpret_cast<float2*>(ut)[i] = make_float2(a2.hi, a2.lo);
      reinterpret_cast<float2*>(vt)[i] = make_float2(b2.hi, b2.lo);
      reinterpret_cast<float2*>(at)[i] = make_float2(c3.hi, c3.lo);
    } else {
      ut[i] = uti;
      vt[i] = vti;
      at[i] = ati;
    }
    r[i] = 0.0;
    q[i] = 0.0;
  }
  double vals[1] = {bb}, out[1];
  if (last_block_reduce<1>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->bb = out[0];
    cg->iter = 0;
    cg->status = 0;
    cg->relres = 0.0;
    cg->zero_rhs = (out[0] == 0.0);
    cg->done = (out[0] == 0.0);
    if (!isfinite(out[0])) {
      cg->status = -5;
      cg->done = 1;
    }
  }
}

// rr = r . r of the residual produced by the single-pass residual kernel.
__global__ void cg_rnorm_kernel(int64_t N, const double* __restrict__ r, double* partials, CgScalars* cg) {
  if (((volatile CgScalars*)cg)->done) return;
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x)
    rr = fma(r[i], r[i], rr);
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

__global__ void cg_residual_kernel(int64_t N, const double* __restrict__ b, double* __restrict__ q,
                                   double* __restrict__ r, double* __restrict__ z,
                                   double* __restrict__ p, const double* __restrict__ dinv,
                                   double* partials, CgScalars* cg) {
  if (((volatile CgScalars*)cg)->done) return;
  double rr = 0.0, rz = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    double rn[3], zn[3];
    for (int i = 0; i < 3; ++i) {
      rn[i] = b[3 * n + i] - q[3 * n + i];
      q[3 * n + i] = 0.0;
      r[3 * n + i] = rn[i];
      rr = fma(rn[i], rn[i], rr);
    }
    apply_dinv(dinv + 6 * n, rn, zn);
    for (int i = 0; i < 3; ++i) {
      z[3 * n + i] = zn[i];
      p[3 * n + i] = zn[i];
      rz = fma(rn[i], zn[i], rz);
    }
  }
  double vals[2] = {rr, rz}, out[2];
  if (last_block_reduce<2>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->rr = out[0];
    cg->rz = out[1];
    cg->relres = sqrt(out[0] / cg->bb);
    cg->relres0 = cg->relres;
    if (!isfinite(out[0]) || !isfinite(out[1])) {
      cg->status = -5;
      cg->done = 1;
    } else if (cg->relres <= cg->tol) {
      cg->done = 1;
    }
  }
}

__global__ void cg_update_kernel(int64_t N, double* __restrict__ x, double* __restrict__ r,
                                 double* __restrict__ z, const double* __restrict__ p,
                                 double* __restrict__ q, const double* __restrict__ dinv,
                                 double* partials, CgScalars* cg) {
  if (((volatile CgScalars*)cg)->done) return;
  const double alpha = ((volatile CgScalars*)cg)->rz / ((volatile CgScalars*)cg)->pq;
  double rr = 0.0, rz = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    double rn[3], zn[3];
    for (int i = 0; i < 3; ++i) {
      const int64_t k = 3 * n + i;
      x[k] = fma(alpha, p[k], x[k]);
      rn[i] = fma(-alpha, q[k], r[k]);
      q[k] = 0.0;
      r[k] = rn[i];
      rr = fma(rn[i], rn[i], rr);
    }
    apply_dinv(dinv + 6 * n, rn, zn);
    for (int i = 0; i < 3; ++i) {
      z[3 * n + i] = zn[i];
      rz = fma(rn[i], zn[i], rz);
    }
  }
  double vals[2] = {rr, rz}, out[2];
  if (last_block_reduce<2>(vals, partials, &cg->counter, out) && threadIdx.x == 0) {
    cg->iter += 1;
    cg->rr = out[0];
    cg->relres = sqrt(out[0] / cg->bb);
    if (!isfinite(out[0]) || !isfinite(out[1]) || !isfinite(alpha)) {
      cg->status = -5;
      cg->done = 1;
    } else if (cg->relres <= cg->tol) {
      cg->done = 1;
    } else if (cg->iter >= cg->max_iter) {
      cg->status = -4;
      cg->done = 1;
    } else {
      cg->beta = out[1] / cg->rz;
      cg->rz = out[1];
    }
  }
}

__global__ void cg_pupdate_kernel(int64_t N, const double* __restrict__ z, double* __restrict__ p,
                                  const CgScalars* cg) {
  if (((volatile const CgScalars*)cg)->done) return;
  const double beta = ((volatile const CgScalars*)cg)->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void newmark_kernel(int64_t N, const double* __restrict__ x, double* __restrict__ u,
                               double* __restrict__ v, double* __restrict__ a, double dt,
                               const CgScalars* cg, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  const bool zero = cg->zero_rhs != 0;
  const double c1 = 2.0 / dt, c2 = 4.0 / (dt * dt), c3 = 4.0 / dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double du = zero ? 0.0 : x[i];
    const double vi = v[i];
    u[i] += du;
    v[i] = fma(c1, du, -vi);
    a[i] = fma(c2, du, fma(-c3, vi, -a[i]));
  }
}

__global__ void record_kernel(const double* __restrict__ v, const int32_t* __restrict__ rec_node,
                              const double* __restrict__ rec_w, int n_rec, double* wave, int n_steps,
                              int step, const StepState* ss) {
  if (ss != nullptr) {
    if (!((volatile const StepState*)ss)->commit) return;
    step = ss->step;
  }
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_rec) return;
  const int r = t / 3, c = t % 3;
  double s = 0.0;
  for (int k = 0; k < 6; ++k) s = fma(rec_w[6 * r + k], v[3 * (int64_t)rec_node[6 * r + k] + c], s);
  wave[(int64_t)(3 * r + c) * n_steps + step] = s;
}

// ------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------

int ebe_blocks(const ModelView& m) {
  return (int)((m.E + m.F + kElemThreads - 1) / kElemThreads);
}
int node_blocks(int64_t n) {
  int64_t b = (n + kNodeThreads - 1) / kNodeThreads;
  return (int)(b < kMaxNodeBlocks ? (b < 1 ? 1 : b) : kMaxNodeBlocks);
}

void launch_geometry(const ModelView& m, const double* xyz, double px, double py, double* geo,
                     int* err, cudaStream_t s) {
  if (m.E == 0) return;
  geometry_kernel<<<(unsigned)((m.E + 127) / 128), 128, 0, s>>>(m, xyz, px, py, geo, err);
}
void launch_face_geometry(const ModelView& m, const double* xyz, double px, double py,
                          const int32_t* face_elem, const int32_t* face_tag, double* fgeo, int* err,
                          cudaStream_t s) {
  if (m.F == 0) return;
  face_geometry_kernel<<<(unsigned)((m.F + 127) / 128), 128, 0, s>>>(m, xyz, px, py, face_elem,
                                                                     face_tag, fgeo, err);
}
void launch_material(MatCoef* mat, const double* raw, int n_mat, double dt, double f1, double f2,
                     cudaStream_t s) {
  material_kernel<<<1, kMaxMat, 0, s>>>(mat, raw, n_mat, dt, f1, f2);
}
void launch_block_jacobi(const ModelView& m, double* dblk, double* dinv, int* err, cudaStream_t s) {
  cudaMemsetAsync(dblk, 0, sizeof(double) * 6 * m.N, s);
  if (m.E + m.F > 0)
    diag_blocks_kernel<<<(unsigned)((m.E + m.F + 127) / 128), 128, 0, s>>>(m, dblk);
  invert_blocks_kernel<<<node_blocks(m.N), kNodeThreads, 0, s>>>(m.N, dblk, dinv, err);
}
void launch_coarse_blocks(const ModelView& m, const int32_t* vid, double* cblk, cudaStream_t s) {
  if (m.E + m.F > 0)
    coarse_blocks_kernel<<<(unsigned)((m.E + m.F + 127) / 128), 128, 0, s>>>(m, vid, cblk);
}
void launch_invert_blocks(int64_t n, const double* blk, double* inv, int* err, cudaStream_t s) {
  invert_blocks_kernel<<<node_blocks(n), kNodeThreads, 0, s>>>(n, blk, inv, err);
}
void launch_receivers(const ModelView& m, const double* xyz, double px, double py,
                      const double* rec_xy, int n_rec, int32_t* rec_face, int32_t* rec_node,
                      double* rec_w, int* err, cudaStream_t s) {
  if (n_rec == 0) return;
  cudaMemsetAsync(rec_face, 0x7f, sizeof(int32_t) * n_rec, s);
  receiver_find_kernel<<<n_rec, 256, 0, s>>>(m, xyz, px, py, rec_xy, rec_face);
  receiver_weights_kernel<<<(n_rec + 127) / 128, 128, 0, s>>>(m, xyz, px, py, rec_xy, n_rec, rec_face,
                                                              rec_node, rec_w, err);
}
void launch_ebe(int mode, const ModelView& m, const double* x, const double* v, const double* a,
                double* y, double force, int dir, double* partials, CgScalars* cg, cudaStream_t s, Drive dr) {
  const int nb = ebe_blocks(m);
  if (nb == 0) return;
  switch (mode) {
    case kModeA:
      ebe_kernel<kModeA><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, partials, cg, dr);
      break;
    case kModeK:
      ebe_kernel<kModeK><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr, dr);
      break;
    case kModeM:
      ebe_kernel<kModeM><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr, dr);
      break;
    case kModeC:
      ebe_kernel<kModeC><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr, dr);
      break;
    case kModeRes:
      ebe_kernel<kModeRes><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr, dr);
      break;
    default:
      ebe_kernel<kModeRhs><<<nb, kElemThreads, 0, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr, dr);
      break;
  }
}
void launch_ebe_dw(int mode, int dw_in, const ModelView& m, const double* x, const double* v, const double* a,
                   double* y, double force, int dir, double* partials, CgScalars* cg, cudaStream_t s, Drive dr) {
  const int nb = ebe_blocks(m);
  if (nb == 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(ebe_dw_kernel<kModeA, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
    cudaFuncSetAttribute(ebe_dw_kernel<kModeA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
    cudaFuncSetAttribute(ebe_dw_kernel<kModeRes, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
    attr_set = true;
  }
  if (mode == kModeA && dw_in)
    ebe_dw_kernel<kModeA, true><<<nb, kElemThreads, kDwSmem, s>>>(m, x, v, a, y, force, dir, partials, cg, dr);
  else if (mode == kModeA)
    ebe_dw_kernel<kModeA, false><<<nb, kElemThreads, kDwSmem, s>>>(m, x, v, a, y, force, dir, partials, cg, dr);
  else
    ebe_dw_kernel<kModeRes, true><<<nb, kElemThreads, kDwSmem, s>>>(m, x, v, a, y, force, dir, nullptr, nullptr,
                                                                     dr);
}
void launch_cg_init(const ModelView& m, const double* b, const double* v, const double* a,
                    double* x, double* q, double* partials, CgScalars* cg, cudaStream_t s, int use_guess,
                    const StepState* ss) {
  cg_init_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, b, v, a, m.dt, x, q, partials, cg, use_guess, ss);
}

// ------------------------------------------------------------------------------
// Initial guess from the increment history
// ------------------------------------------------------------------------------

// du0 = sum_j c_j du_{n-j}, j = 0..k, c_j = (-1)^j C(k+1, j+1): the degree-k
// polynomial through the last k+1 increments, evaluated one step ahead.  ring
// holds S = k+1 increments ([S][3N]); ext = {count, head} (head: next slot).
// Until k+1 increments exist the Newmark predictor dt v + dt^2/2 a is used.
__global__ void guess_extrap_kernel(int64_t n3, const double* __restrict__ ring, int S, const int* ext, int k,
                                    const double* __restrict__ v, const double* __restrict__ a, double dt,
                                    double* __restrict__ x, const StepState* ss, const ProjState* ps) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  if (ps != nullptr && !((volatile const ProjState*)ps)->retired) {
    // the projection guess still acts: du0 = 0, so the residual pass yields b
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
      x[i] = 0.0;
    return;
  }
  const int count = ((volatile const int*)ext)[0], head = ((volatile const int*)ext)[1];
  const bool ok = count >= k + 1;
  double c[kMaxGuessOrder + 1];
  int slot[kMaxGuessOrder + 1];
  double binom = 1.0;  // C(k+1, j+1), built up term by term
  for (int j = 0; j <= k; ++j) {
    binom = binom * (double)(k + 1 - j) / (double)(j + 1);
    c[j] = (j & 1) ? -binom : binom;
    slot[j] = ((head - 1 - j) % S + S) % S;
  }
  const double h = 0.5 * dt * dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    double g;
    if (ok) {
      g = 0.0;
      for (int j = 0; j <= k; ++j) g = fma(c[j], ring[(int64_t)slot[j] * n3 + i], g);
    } else {
      g = fma(dt, v[i], h * a[i]);
    }
    x[i] = g;
  }
}
// After a committed step: ring[head] = du, then (one thread) head, count advance.
__global__ void guess_push_kernel(int64_t n3, const double* __restrict__ du, double* __restrict__ ring, int S,
                                  const int* ext, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  const int head = ((volatile const int*)ext)[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    ring[(int64_t)head * n3 + i] = du[i];
}
__global__ void guess_advance_kernel(int* ext, int S, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  ext[1] = (ext[1] + 1) % S;
  ext[0] = ext[0] < S ? ext[0] + 1 : S;
}
// ------------------------------------------------------------------------------
// Initial guess by Galerkin projection onto the last k converged increments
// ------------------------------------------------------------------------------
//
// W = [du_{n-1} .. du_{n-k}] (ring of slots), Z = A W stored as the converged
// steps' b - r (no operator application), G = (W^T Z + Z^T W) / 2 kept by
// slot.  At a step with right-hand side b: c = G^+ W^T b (eigenvalues below
// 1e-12 of the largest dropped), du0 = W c and r0 = b - Z c: the A-norm
// optimal combination of the past increments.

// Solve of the symmetric positive semi-definite n x n system G c = g (n <=
// kMaxProj) in one thread: Cholesky factorisation of G + ridge I with ridge
// 1e-12 times the largest diagonal entry, so nearly collinear increments give
// a bounded combination instead of a breakdown; a pivot that still vanishes
// drops its direction.
__device__ void proj_solve(const double* G, const double* g, int n, double* c) {
  double L[kMaxProj][kMaxProj], y[kMaxProj];
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = fmax(dmax, G[i * kMaxProj + i]);
  const double ridge = 1e-12 * dmax;
  for (int j = 0; j < n; ++j) {
    double d = G[j * kMaxProj + j] + ridge;
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    L[j][j] = d > ridge ? sqrt(d) : 0.0;
    for (int i = j + 1; i < n; ++i) {
      double v = G[i * kMaxProj + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = L[j][j] > 0.0 ? v / L[j][j] : 0.0;
    }
  }
  for (int i = 0; i < n; ++i) {  // L y = g
    double v = g[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = L[i][i] > 0.0 ? v / L[i][i] : 0.0;
  }
  for (int i = n - 1; i >= 0; --i) {  // L^T c = y
    double v = y[i];
    for (int k = i + 1; k < n; ++k) v -= L[k][i] * c[k];
    c[i] = L[i][i] > 0.0 ? v / L[i][i] : 0.0;
  }
}

// g = W^T b over the filled slots, then c (in ps) by the projection solve.
__global__ void proj_coef_kernel(int64_t n3, const double* __restrict__ W, const double* __restrict__ b,
                                 ProjState* ps, double* partials, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  if (((volatile const ProjState*)ps)->retired) return;
  const int cnt = ((volatile const ProjState*)ps)->count;
  double acc[kMaxProj];
#pragma unroll
  for (int j = 0; j < kMaxProj; ++j) acc[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
#pragma unroll
    for (int j = 0; j < kMaxProj; ++j)
      if (j < cnt) acc[j] = fma(W[(int64_t)j * n3 + i], bi, acc[j]);
  }
  double out[kMaxProj];
  if (last_block_reduce<kMaxProj>(acc, partials, &ps->counter, out) && threadIdx.x == 0) {
    if (cnt > 0) proj_solve(ps->G, out, cnt, ps->c);
    for (int j = cnt; j < kMaxProj; ++j) ps->c[j] = 0.0;
  }
}

// x = W c, keep b, r = b - Z c (r holds b on entry).
__global__ void proj_apply_kernel(int64_t n3, const double* __restrict__ W, const double* __restrict__ Z,
                                  const ProjState* ps, double* __restrict__ x, double* __restrict__ r,
                                  double* __restrict__ bkeep, const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  if (((volatile const ProjState*)ps)->retired) return;
  const int cnt = ((volatile const ProjState*)ps)->count;
  double c[kMaxProj];
#pragma unroll
  for (int j = 0; j < kMaxProj; ++j) c[j] = ((volatile const ProjState*)ps)->c[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    double xi = 0.0, zi = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxProj; ++j)
      if (j < cnt) {
        xi = fma(c[j], W[(int64_t)j * n3 + i], xi);
        zi = fma(c[j], Z[(int64_t)j * n3 + i], zi);
      }
    const double bi = r[i];
    bkeep[i] = bi;
    x[i] = xi;
    r[i] = bi - zi;
  }
}

// x = W c only (the FP64 solver forms its own first residual).
__global__ void proj_guess_kernel(int64_t n3, const double* __restrict__ W, const ProjState* ps, double* __restrict__ x,
                                  const StepState* ss) {
  if (ss != nullptr && !((volatile const StepState*)ss)->active) return;
  if (((volatile const ProjState*)ps)->retired) return;
  const int cnt = ((volatile const ProjState*)ps)->count;
  double c[kMaxProj];
#pragma unroll
  for (int j = 0; j < kMaxProj; ++j) c[j] = ((volatile const ProjState*)ps)->c[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    double xi = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxProj; ++j)
      if (j < cnt) xi = fma(c[j], W[(int64_t)j * n3 + i], xi);
    x[i] = xi;
  }
}

// Push the converged increment: slot `head` of W gets du, of Z gets b - r
// (= A du), and the slot's row and column of G are recomputed from the dots
// with every filled slot; count and head advance.
__global__ void proj_push_kernel(int64_t n3, const double* __restrict__ du, const double* __restrict__ b,
                                 const double* __restrict__ r, double* __restrict__ W, double* __restrict__ Z,
                                 ProjState* ps, int k, double* partials, const StepState* ss,
                                 const CgScalars* cg, double handover) {
  if (ss != nullptr && !((volatile const StepState*)ss)->commit) return;
  if (((volatile const ProjState*)ps)->retired) return;
  const int head = ((volatile const ProjState*)ps)->head;
  const int cnt0 = ((volatile const ProjState*)ps)->count;
  const int cnt = cnt0 < k ? cnt0 + 1 : k;  // slots filled after this push
  double acc[2 * kMaxProj];
#pragma unroll
  for (int j = 0; j < 2 * kMaxProj; ++j) acc[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double di = du[i], zi = b[i] - r[i];
    W[(int64_t)head * n3 + i] = di;
    Z[(int64_t)head * n3 + i] = zi;
#pragma unroll
    for (int j = 0; j < kMaxProj; ++j)
      if (j < cnt) {
        const double wj = j == head ? di : W[(int64_t)j * n3 + i];
        const double zj = j == head ? zi : Z[(int64_t)j * n3 + i];
        acc[j] = fma(di, zj, acc[j]);
        acc[kMaxProj + j] = fma(wj, zi, acc[kMaxProj + j]);
      }
  }
  double out[2 * kMaxProj];
  if (last_block_reduce<2 * kMaxProj>(acc, partials, &ps->counter, out) && threadIdx.x == 0) {
    for (int j = 0; j < kMaxProj; ++j) {
      const double gj = j < cnt ? 0.5 * (out[j] + out[kMaxProj + j]) : 0.0;
      ps->G[head * kMaxProj + j] = gj;
      ps->G[j * kMaxProj + head] = gj;
    }
    ps->count = cnt;
    ps->head = (head + 1) % k;
    // hand over to the extrapolation once a step started close enough
    if (handover > 0.0 && cg != nullptr && ((volatile const CgScalars*)cg)->relres0 < handover) ps->retired = 1;
  }
}

// The W/Z slots are in ring order, but the projection is invariant to the
// order of its basis, so the dots and combinations run over slots 0..count-1.
// The reductions use the projection's own partials buffer (2 * kMaxProj *
// kMaxNodeBlocks doubles), so they run on the full node grid.
static int proj_blocks(int64_t n3) { return node_blocks(n3); }
void launch_proj_coef(int64_t N, const double* W, const double* b, ProjState* ps, double* partials, cudaStream_t s,
                      const StepState* ss) {
  proj_coef_kernel<<<proj_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, W, b, ps, partials, ss);
}
void launch_proj_apply(int64_t N, const double* W, const double* Z, const ProjState* ps, double* x, double* r,
                       double* bkeep, cudaStream_t s, const StepState* ss) {
  proj_apply_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, W, Z, ps, x, r, bkeep, ss);
}
void launch_proj_guess(int64_t N, const double* W, const ProjState* ps, double* x, cudaStream_t s,
                       const StepState* ss) {
  proj_guess_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, W, ps, x, ss);
}
void launch_proj_push(int64_t N, const double* du, const double* b, const double* r, double* W, double* Z,
                      ProjState* ps, int k, double* partials, cudaStream_t s, const StepState* ss,
                      const CgScalars* cg, double handover) {
  proj_push_kernel<<<proj_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, du, b, r, W, Z, ps, k, partials, ss, cg,
                                                               handover);
}

void launch_guess_extrap(int64_t N, const double* ring, int k, const int* ext, const double* v, const double* a,
                         double dt, double* x, cudaStream_t s, const StepState* ss, const ProjState* ps) {
  guess_extrap_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, ring, k + 1, ext, k, v, a, dt, x, ss, ps);
}
void launch_guess_push(int64_t N, const double* du, double* ring, int k, int* ext, cudaStream_t s,
                       const StepState* ss) {
  guess_push_kernel<<<node_blocks(3 * N), kNodeThreads, 0, s>>>(3 * N, du, ring, k + 1, ext, ss);
  guess_advance_kernel<<<1, 1, 0, s>>>(ext, k + 1, ss);
}
void launch_cg_init_mixed(const ModelView& m, const float* b32, const double* u, const double* v, const double* a,
                          double* x, double* ut, double* vt, double* at, double* r, double* q, double* partials,
                          CgScalars* cg, cudaStream_t s, const StepState* ss, int use_guess, int dw_out) {
  cg_init_mixed_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, b32, u, v, a, m.dt, x, ut, vt, at, r, q,
                                                                       partials, cg, ss, use_guess, dw_out);
}
void launch_cg_rnorm(const ModelView& m, const double* r, double* partials, CgScalars* cg, cudaStream_t s) {
  cg_rnorm_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, r, partials, cg);
}
void launch_cg_residual(const ModelView& m, const double* b, double* q, double* r, double* z,
                        double* p, const double* dinv, double* partials, CgScalars* cg,
                        cudaStream_t s) {
  cg_residual_kernel<<<node_blocks(m.N), kNodeThreads, 0, s>>>(m.N, b, q, r, z, p, dinv, partials, cg);
}
void launch_cg_update(const ModelView& m, double* x, double* r, double* z, const double* p,
                      double* q, const double* dinv, double* partials, CgScalars* cg,
                      cudaStream_t s) {
  cg_update_kernel<<<node_blocks(m.N), kNodeThreads, 0, s>>>(m.N, x, r, z, p, q, dinv, partials, cg);
}
void launch_cg_pupdate(const ModelView& m, const double* z, double* p, const CgScalars* cg,
                       cudaStream_t s) {
  cg_pupdate_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, z, p, cg);
}
void launch_newmark(const ModelView& m, const double* x, double* u, double* v, double* a,
                    const CgScalars* cg, cudaStream_t s, const StepState* ss) {
  newmark_kernel<<<node_blocks(3 * m.N), kNodeThreads, 0, s>>>(m.N, x, u, v, a, m.dt, cg, ss);
}
void launch_record(const double* v, const int32_t* rec_node, const double* rec_w, int n_rec,
                   double* wave, int n_steps, int step, cudaStream_t s, const StepState* ss) {
  if (n_rec == 0) return;
  record_kernel<<<(3 * n_rec + 127) / 128, 128, 0, s>>>(v, rec_node, rec_w, n_rec, wave, n_steps, step, ss);
}

}  // namespace gsw
