// Input-wave estimate and misfit ERR on the GPU (Section 2).
//
// With p(t) shifted by l strides (l = 0..L-1) the response at receiver k in
// direction i is U_ki[n] = sum_j sum_l G[k,i,j,n - l s] c_jl (Section 2,
// superposition of Green's functions).  The coefficients minimise the
// weighted least-squares misfit sum_ki w_ki sum_n (U_ki - obs_ki)^2 with
// w_ki = 1 / sum_n obs_ki^2, giving A c = b with
//     A[(j,l),(j',l')] = sum_ki w_ki sum_n G[k,i,j,n-ls] G[k,i,j',n-l's]
//     b[(j,l)]         = sum_ki w_ki sum_n G[k,i,j,n-ls] obs_ki[n].
// A is symmetric positive semi-definite, so its SVD is its eigen
// decomposition, computed here by the cyclic Jacobi method (Golub & Van Loan,
// symmetric Schur rotations) with the round-robin pairing so that P/2
// rotations proceed in parallel; eigenvalues below tau * lambda_max are
// discarded.  ERR follows Eq. (2) over the pairs with non-negligible
// observed energy (>= 1e-12 of the largest).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "gsw_misfit.cuh"

namespace gsw {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum_d(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) v = warp_sum_d(v);
  __syncthreads();
  return v;  // valid in thread 0
}

__global__ void energy_kernel(const double* __restrict__ obs, int n_t, double* energy) {
  const int pair = blockIdx.x;
  double s = 0.0;
  for (int n = threadIdx.x; n < n_t; n += blockDim.x) {
    const double o = obs[(size_t)pair * n_t + n];
    s = fma(o, o, s);
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) energy[pair] = s;
}

__global__ void weights_kernel(const double* __restrict__ energy, int n_pairs, double* w, double* n_kept) {
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n_pairs; ++i) m = fmax(m, energy[i]);
    mx = m;
  }
  __syncthreads();
  double cnt = 0.0;
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x) {
    const bool keep = mx > 0.0 && energy[i] >= 1e-12 * mx;
    w[i] = keep ? 1.0 / energy[i] : 0.0;
    cnt += keep ? 1.0 : 0.0;
  }
  cnt = block_sum_d(cnt);
  if (threadIdx.x == 0) *n_kept = cnt;
}

// One block per upper-triangle entry (r, c) of A.
__global__ void assemble_A_kernel(const double* __restrict__ G, const double* __restrict__ w,
                                  int n_rec, int n_t, int stride, int L, double* A) {
  const int r = blockIdx.y, c = blockIdx.x;
  const int P = 3 * L;
  if (c < r) return;
  const int j = r / L, l = r % L, j2 = c / L, l2 = c % L;
  const int s1 = l * stride, s2 = l2 * stride;
  const int n0 = s1 > s2 ? s1 : s2;
  double acc = 0.0;
  for (int pair = 0; pair < 3 * n_rec; ++pair) {
    const double wk = w[pair];
    if (wk == 0.0) continue;
    const int k = pair / 3, i = pair % 3;
    const double* g1 = G + (((size_t)k * 3 + i) * 3 + j) * n_t;
    const double* g2 = G + (((size_t)k * 3 + i) * 3 + j2) * n_t;
    double part = 0.0;
    for (int n = n0 + threadIdx.x; n < n_t; n += blockDim.x) part = fma(g1[n - s1], g2[n - s2], part);
    acc = fma(wk, part, acc);
  }
  acc = block_sum_d(acc);
  if (threadIdx.x == 0) {
    A[(size_t)r * P + c] = acc;
    A[(size_t)c * P + r] = acc;
  }
}

__global__ void assemble_b_kernel(const double* __restrict__ G, const double* __restrict__ obs,
                                  const double* __restrict__ w, int n_rec, int n_t, int stride, int L,
                                  double* b) {
  const int r = blockIdx.x;
  const int j = r / L, l = r % L;
  const int s1 = l * stride;
  double acc = 0.0;
  for (int pair = 0; pair < 3 * n_rec; ++pair) {
    const double wk = w[pair];
    if (wk == 0.0) continue;
    const int k = pair / 3, i = pair % 3;
    const double* g1 = G + (((size_t)k * 3 + i) * 3 + j) * n_t;
    const double* o = obs + (size_t)pair * n_t;
    double part = 0.0;
    for (int n = s1 + threadIdx.x; n < n_t; n += blockDim.x) part = fma(g1[n - s1], o[n], part);
    acc = fma(wk, part, acc);
  }
  acc = block_sum_d(acc);
  if (threadIdx.x == 0) b[r] = acc;
}

// Cyclic Jacobi eigen decomposition of the symmetric P x P matrix A (in
// place; on exit A is diagonal up to the tolerance) with eigenvectors V.
// Single block; round-robin pairing, P padded to even with a dummy index.
__global__ void __launch_bounds__(1024) jacobi_kernel(double* A, double* V, int P, int max_sweeps,
                                                      int* sweeps_out) {
  __shared__ double cs[kMisfitMaxUnknowns / 2 + 1], sn[kMisfitMaxUnknowns / 2 + 1];
  __shared__ int pp[kMisfitMaxUnknowns / 2 + 1], qq[kMisfitMaxUnknowns / 2 + 1];
  __shared__ int stop;
  const int Pe = P + (P & 1);
  const int half = Pe / 2;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) V[i] = (i / P == i % P) ? 1.0 : 0.0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
      const double a = A[i];
      tot = fma(a, a, tot);
      if (i / P != i % P) off = fma(a, a, off);
    }
    off = block_sum_d(off);
    tot = block_sum_d(tot);
    if (threadIdx.x == 0) stop = !(off > 1e-30 * tot);
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < Pe - 1; ++round) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        const int a = (k == 0) ? 0 : ((k - 1 + round) % (Pe - 1)) + 1;
        const int b = ((Pe - 1 - k - 1 + round) % (Pe - 1)) + 1;
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < P) {
          const double apq = A[(size_t)p * P + q];
          if (apq != 0.0) {
            const double tau = (A[(size_t)q * P + q] - A[(size_t)p * P + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        } else {
          p = q = -1;
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = threadIdx.x; idx < half * P; idx += blockDim.x) {
        const int k = idx / P, col = idx % P;
        const int p = pp[k], q = qq[k];
        if (p < 0) continue;
        const double c = cs[k], s = sn[k];
        const double ap = A[(size_t)p * P + col], aq = A[(size_t)q * P + col];
        A[(size_t)p * P + col] = c * ap - s * aq;
        A[(size_t)q * P + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = threadIdx.x; idx < half * P; idx += blockDim.x) {
        const int k = idx / P, row = idx % P;
        const int p = pp[k], q = qq[k];
        if (p < 0) continue;
        const double c = cs[k], s = sn[k];
        const double ap = A[(size_t)row * P + p], aq = A[(size_t)row * P + q];
        A[(size_t)row * P + p] = c * ap - s * aq;
        A[(size_t)row * P + q] = s * ap + c * aq;
        const double vp = V[(size_t)row * P + p], vq = V[(size_t)row * P + q];
        V[(size_t)row * P + p] = c * vp - s * vq;
        V[(size_t)row * P + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) *sweeps_out = sweep;
}

// c = sum over kept eigenpairs v_i (v_i . b) / lambda_i.
__global__ void pinv_solve_kernel(const double* __restrict__ A, const double* __restrict__ V,
                                  const double* __restrict__ b, int P, double tau, double* c) {
  __shared__ double lmax;
  __shared__ double coef[kMisfitMaxUnknowns];
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < P; ++i) m = fmax(m, A[(size_t)i * P + i]);
    lmax = m;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double lam = A[(size_t)i * P + i];
    double vb = 0.0;
    for (int r = 0; r < P; ++r) vb = fma(V[(size_t)r * P + i], b[r], vb);
    coef[i] = (lmax > 0.0 && lam >= tau * lmax && lam > 0.0) ? vb / lam : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < P; ++i) s = fma(V[(size_t)r * P + i], coef[i], s);
    c[r] = s;
  }
}

// Per (k, i): sqrt(sum (U - obs)^2) / sqrt(sum obs^2) for kept pairs.
__global__ void err_kernel(const double* __restrict__ G, const double* __restrict__ obs,
                           const double* __restrict__ w, const double* __restrict__ c, int n_t, int stride,
                           int L, double* ratio) {
  const int pair = blockIdx.x;
  const int k = pair / 3, i = pair % 3;
  double s = 0.0;
  if (w[pair] != 0.0) {
    for (int n = threadIdx.x; n < n_t; n += blockDim.x) {
      double U = 0.0;
      for (int j = 0; j < 3; ++j) {
        const double* g = G + (((size_t)k * 3 + i) * 3 + j) * n_t;
        for (int l = 0; l < L && l * stride <= n; ++l) U = fma(c[j * L + l], g[n - l * stride], U);
      }
      const double d = U - obs[(size_t)pair * n_t + n];
      s = fma(d, d, s);
    }
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) ratio[pair] = (w[pair] != 0.0) ? sqrt(s) * sqrt(w[pair]) : 0.0;
}

__global__ void err_final_kernel(const double* __restrict__ ratio, int n_pairs, const double* n_kept,
                                 double* err) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x) s += ratio[i];
  s = block_sum_d(s);
  if (threadIdx.x == 0) *err = (*n_kept > 0.0) ? s / *n_kept : 0.0;
}

}  // namespace

// Green's functions from the three directions' receiver histories:
// G[k][i][j][n] = wave_j[k][i][n], n < n_t.
__global__ void gather_green_kernel(int n_rec, int n_t, int n_steps, const double* __restrict__ w0,
                                    const double* __restrict__ w1, const double* __restrict__ w2,
                                    double* __restrict__ G) {
  const int64_t total = (int64_t)n_rec * 9 * n_t;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(t % n_t);
    const int64_t kij = t / n_t;
    const int j = (int)(kij % 3);
    const int64_t ki = kij / 3;
    const double* w = j == 0 ? w0 : (j == 1 ? w1 : w2);
    G[t] = w[ki * n_steps + n];
  }
}

namespace {

int misfit_scratch(MisfitWork& w, cudaStream_t s, size_t need, char* msg, size_t msg_len) {
  if (need * sizeof(double) > w.bytes) {
    if (w.buf) {
      if (w.free_)
        w.free_(w.buf, (void*)s, w.user);
      else
        cudaFreeAsync(w.buf, s);
    }
    w.buf = nullptr;
    w.bytes = 0;
    void* p = nullptr;
    if (w.alloc)
      p = w.alloc(need * sizeof(double), (void*)s, w.user);
    else if (cudaMallocAsync(&p, need * sizeof(double), s) != cudaSuccess)
      p = nullptr;
    if (!p) {
      snprintf(msg, msg_len, "scratch allocation of %zu bytes failed", need * sizeof(double));
      return 2;
    }
    w.buf = (double*)p;
    w.bytes = need * sizeof(double);
  }
  if (!w.host && cudaMallocHost(&w.host, sizeof(double) * (kMisfitMaxUnknowns + 4)) != cudaSuccess) {
    snprintf(msg, msg_len, "pinned allocation failed");
    return 2;
  }
  return 0;
}

// The misfit on device-resident G and obs (inside w.buf): weights, normal
// equations, Jacobi eigen pseudo-inverse, ERR; results to the host.
int misfit_core(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, int stride, int L, double tau, double* err,
                double* c_out, char* msg, size_t msg_len, cudaError_t* ce) {
  const int P = 3 * L;
  const int n_pairs = 3 * n_rec;
  const size_t nG = (size_t)n_rec * 9 * n_t, nO = (size_t)n_rec * 3 * n_t;
  double* dG = w.buf;
  double* dO = dG + nG;
  double* energy = dO + nO;
  double* wt = energy + n_pairs;
  double* ratio = wt + n_pairs;
  double* A = ratio + n_pairs;
  double* V = A + (size_t)P * P;
  double* b = V + (size_t)P * P;
  double* c = b + P;
  double* scal = c + P;  // n_kept, err, sweeps
  cudaError_t e;
#define CKR(call)        \
  if ((e = (call)) != cudaSuccess) { \
    *ce = e;             \
    snprintf(msg, msg_len, "%s", #call); \
    return 1;            \
  }
  energy_kernel<<<n_pairs, kT, 0, s>>>(dO, n_t, energy);
  weights_kernel<<<1, kT, 0, s>>>(energy, n_pairs, wt, scal);
  assemble_A_kernel<<<dim3(P, P), kT, 0, s>>>(dG, wt, n_rec, n_t, stride, L, A);
  assemble_b_kernel<<<P, kT, 0, s>>>(dG, dO, wt, n_rec, n_t, stride, L, b);
  jacobi_kernel<<<1, 1024, 0, s>>>(A, V, P, 60, (int*)(scal + 2));
  pinv_solve_kernel<<<1, kT, 0, s>>>(A, V, b, P, tau, c);
  err_kernel<<<n_pairs, kT, 0, s>>>(dG, dO, wt, c, n_t, stride, L, ratio);
  err_final_kernel<<<1, kT, 0, s>>>(ratio, n_pairs, scal, scal + 1);
  CKR(cudaGetLastError());
  CKR(cudaMemcpyAsync(w.host, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKR(cudaMemcpyAsync(w.host + 1, c, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
  CKR(cudaStreamSynchronize(s));
#undef CKR
  *err = w.host[0];
  if (c_out) memcpy(c_out, w.host + 1, sizeof(double) * P);
  return 0;
}

size_t misfit_need(int n_rec, int n_t, int L) {
  const int P = 3 * L;
  const size_t n_pairs = 3 * (size_t)n_rec;
  return (size_t)n_rec * 9 * n_t + (size_t)n_rec * 3 * n_t + 3 * n_pairs + 2 * (size_t)P * P + 2 * (size_t)P + 4;
}

}  // namespace

int misfit_run(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, const double* G, const double* obs,
               int stride, int L, double tau, double* err, double* c_out, char* msg, size_t msg_len,
               cudaError_t* ce) {
  int rc = misfit_scratch(w, s, misfit_need(n_rec, n_t, L), msg, msg_len);
  if (rc) return rc;
  const size_t nG = (size_t)n_rec * 9 * n_t, nO = (size_t)n_rec * 3 * n_t;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(w.buf, G, nG * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w.buf + nG, obs, nO * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    *ce = e;
    snprintf(msg, msg_len, "input copy");
    return 1;
  }
  return misfit_core(w, s, n_rec, n_t, stride, L, tau, err, c_out, msg, msg_len, ce);
}

int misfit_run_waves(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, int n_steps, const double* const wave[3],
                     const double* obs, int stride, int L, double tau, double* err, double* c_out, char* msg,
                     size_t msg_len, cudaError_t* ce) {
  int rc = misfit_scratch(w, s, misfit_need(n_rec, n_t, L), msg, msg_len);
  if (rc) return rc;
  const size_t nG = (size_t)n_rec * 9 * n_t, nO = (size_t)n_rec * 3 * n_t;
  int64_t blocks = ((int64_t)nG + kT - 1) / kT;
  if (blocks > 152 * 8) blocks = 152 * 8;
  gather_green_kernel<<<(unsigned)blocks, kT, 0, s>>>(n_rec, n_t, n_steps, wave[0], wave[1], wave[2], w.buf);
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(w.buf + nG, obs, nO * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    *ce = e;
    snprintf(msg, msg_len, "Green's function gather");
    return 1;
  }
  return misfit_core(w, s, n_rec, n_t, stride, L, tau, err, c_out, msg, msg_len, ce);
}

// ---- allocation-free variant ---------------------------------------------------
//
// The working memory of gsw_misfit_noalloc lives in this fixed array instead of
// a cudaMalloc'ed buffer.  Host code cannot pass `g_noalloc_scratch` to a
// kernel directly (in host code the name denotes a host-side stand-in), so its
// device address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr int kNoAllocP = 3 * kNoAllocMaxShifts;
constexpr int kNoAllocPairs = 3 * kNoAllocMaxRec;
constexpr size_t kNoAllocDoubles =
    3 * (size_t)kNoAllocPairs + 2 * (size_t)kNoAllocP * kNoAllocP + 2 * (size_t)kNoAllocP + 4;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
constexpr int kMaxDevices = 64;
double* g_noalloc_addr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;
}  // namespace

int misfit_run_noalloc(cudaStream_t s, int device, int n_rec, int n_t, const double* G_dev, const double* obs_dev,
                       int stride, int L, double tau, double* err_dev, double* c_dev, char* msg, size_t msg_len,
                       cudaError_t* ce) {
  if (L > kNoAllocMaxShifts || n_rec > kNoAllocMaxRec) {
    snprintf(msg, msg_len, "n_shifts %d / n_rec %d exceed the fixed working memory (max %d / %d)", L, n_rec,
             kNoAllocMaxShifts, kNoAllocMaxRec);
    return 3;
  }
  if (device < 0 || device >= kMaxDevices) {
    snprintf(msg, msg_len, "device %d out of range", device);
    return 3;
  }
  double* base;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        *ce = e;
        snprintf(msg, msg_len, "cudaGetSymbolAddress of the fixed working memory");
        return 1;
      }
      g_noalloc_addr[device] = (double*)p;
    }
    base = g_noalloc_addr[device];
  }
  const int P = 3 * L;
  const int n_pairs = 3 * n_rec;
  double* energy = base;
  double* wt = energy + n_pairs;
  double* ratio = wt + n_pairs;
  double* A = ratio + n_pairs;
  double* V = A + (size_t)P * P;
  double* b = V + (size_t)P * P;
  double* c = b + P;
  double* scal = c + P;  // n_kept, err, sweeps
  energy_kernel<<<n_pairs, kT, 0, s>>>(obs_dev, n_t, energy);
  weights_kernel<<<1, kT, 0, s>>>(energy, n_pairs, wt, scal);
  assemble_A_kernel<<<dim3(P, P), kT, 0, s>>>(G_dev, wt, n_rec, n_t, stride, L, A);
  assemble_b_kernel<<<P, kT, 0, s>>>(G_dev, obs_dev, wt, n_rec, n_t, stride, L, b);
  jacobi_kernel<<<1, 1024, 0, s>>>(A, V, P, 60, (int*)(scal + 2));
  pinv_solve_kernel<<<1, kT, 0, s>>>(A, V, b, P, tau, c_dev ? c_dev : c);
  err_kernel<<<n_pairs, kT, 0, s>>>(G_dev, obs_dev, wt, c_dev ? c_dev : c, n_t, stride, L, ratio);
  err_final_kernel<<<1, kT, 0, s>>>(ratio, n_pairs, scal, err_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ce = e;
    snprintf(msg, msg_len, "kernel launch");
    return 1;
  }
  return 0;
}

void misfit_free(MisfitWork& w, cudaStream_t s) {
  if (w.buf) {
    if (w.free_)
      w.free_(w.buf, (void*)s, w.user);
    else
      cudaFreeAsync(w.buf, s);
  }
  w.buf = nullptr;
  w.bytes = 0;
  if (w.host) cudaFreeHost(w.host);
  w.host = nullptr;
}

}  // namespace gsw
