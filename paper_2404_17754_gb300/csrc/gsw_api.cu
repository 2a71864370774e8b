// C ABI of the library (declared in include/gsw.h): context, model upload
// and validation, time stepping driver, state access, misfit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gsw.h"
#include "gsw_internal.cuh"
#include "gsw_misfit.cuh"

static_assert(gsw::kStatusTimeout == GSW_E_TIMEOUT, "device timeout status");
#include <cuda_fp16.h>

using namespace gsw;

namespace {

struct Model {
  int64_t N = 0, E = 0, F = 0;
  int n_mat = 0, n_rec = 0;
  double period[2] = {0.0, 0.0};
  std::vector<double> raw_mat;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // device: mesh
  double* xyz = nullptr;
  int32_t* conn = nullptr;
  double* geo = nullptr;
  int32_t* emat = nullptr;
  double* raw_mat_dev = nullptr;
  MatCoef* mat = nullptr;
  int32_t* fnode = nullptr;
  int32_t* face_elem = nullptr;
  int32_t* face_tag = nullptr;
  double* fgeo = nullptr;
  double* rec_xy = nullptr;
  int32_t* rec_face = nullptr;
  int32_t* rec_node = nullptr;
  double* rec_w = nullptr;
  int* err = nullptr;
  // time stepping
  bool time_set = false;
  double dt = 0.0, f1 = 0.0, f2 = 0.0;
  int n_steps = 0;
  double *u = nullptr, *v = nullptr, *a = nullptr, *b = nullptr, *x = nullptr, *r = nullptr,
         *z = nullptr, *p = nullptr, *q = nullptr, *dblk = nullptr, *dinv = nullptr,
         *partials = nullptr, *wave = nullptr;
  CgScalars* cg = nullptr;
  CgScalars* cg_host = nullptr;  // pinned
  std::vector<double> input;
  int dir = 0;
  bool input_set = false;
  gsw_solver_opts opts = {1e-8, 10000, GSW_PREC_FP64, 20, 8, 6, -1, 0.0, 0, 0, 0, 0, 0.0, 0.0, 0.0};
  int64_t step = 0;
  bool failed = false;
  gsw_stats stats = {};
  // reduced-precision inner solve (mixed modes)
  bool lo_ready = false;
  int lo_half = 0;  // 1: FP16 geometry and search direction
  int n_blk = 0, max_local = 0;
  int32_t* blk_ptr = nullptr;
  int32_t* blk_nodes = nullptr;
  uint16_t* lconn = nullptr;
  void* geo_lo = nullptr;  // packed element records of the inner operator
  float* fgeo32 = nullptr;
  float* dinv32 = nullptr;
  float *y32 = nullptr, *s32 = nullptr, *t32 = nullptr, *w32 = nullptr;
  void* d_lo = nullptr;
  void* d_lo2 = nullptr;  // second inner direction buffer (the fused recurrence alternates the two)
  InnerScalars* isc = nullptr;
  float* dw_part = nullptr;    // per-CTA partial sums of the inner operator's d . A d
  double* guess_ring = nullptr;  // [k+1][3N] converged increments (extrapolated initial guess)
  int guess_ring_k = 0;           // degree the ring was sized for
  int* guess_ext = nullptr;       // {count, head} of the ring, on the device
  double* guess_base = nullptr;   // this step's extrapolated guess (base of the learned correction)
  // Galerkin projection guess: W, Z = A W ([k][3N] each), this step's b, state
  double *proj_W = nullptr, *proj_Z = nullptr, *proj_b = nullptr, *proj_part = nullptr;
  ProjState* proj = nullptr;
  int proj_k = 0;
  // two-level inner preconditioner (opts.coarse_weight > 0): the first-order
  // coarse level (structure and blocks shared with the direction instances;
  // zc is each analysis's own)
  int64_t Nv = 0;
  int32_t *cv_node = nullptr, *cv_ptr = nullptr, *cv_mid = nullptr, *c_vid = nullptr;
  int2* c_pair = nullptr;
  double *cblk = nullptr, *cinv = nullptr;  // [Nv][6] coarse diagonal blocks and their inverses
  float* cdc = nullptr;                     // [Nv][6] omega D_c^-1 / mean(D^-1)
  float4* zc = nullptr;                     // [Nv] coarse correction of the current inner iteration
  bool coarse() const { return opts.coarse_weight > 0.0 && opts.precision != GSW_PREC_FP64 && zc != nullptr; }
  CoarseView cview() const { return CoarseView{Nv, cv_node, cv_ptr, cv_mid, c_pair, cdc}; }
  float4* matf = nullptr;      // FP32 material coefficients of the inner operator and the FP32 RHS
  float4* uva = nullptr;       // FP32 copy of u, v, a ([N + 1][3] words) for the FP32 RHS
  unsigned long long iters_mark = 0;   // device inner-iteration counter when timing started
  unsigned long long iters_reset = 0;  // device inner-iteration counter at the last reset
  int lo_variant = 0;          // launch variant of the inner operator (autotuned)
  bool live_tune = false;      // refine the choice inside the next host-driven inner solve
  // learned initial guess
  gsw_learn_opts learn = {0, 0, 0, 0, 0.f, 0u};
  bool mlp_ready = false;
  float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
  uint32_t* packed = nullptr;
  double* hist = nullptr;  // [4][3N] backward differences of the last four increments
  float *nodef = nullptr, *trainX = nullptr, *trainY = nullptr;
  int32_t* node_mat = nullptr;
  MlpScalars* ms = nullptr;
  MlpScalars ms_host = {};
  int hist_head = 3, hist_count = 0, adam_t = 0;
  // referee of the learned guess: initial residuals of the plain predictor
  // (training phase) and of the learned guess (application phase)
  double std_r0_recent[5] = {0, 0, 0, 0, 0}, mlp_r0_recent[5] = {0, 0, 0, 0, 0};
  int64_t std_r0_n = 0, mlp_r0_n = 0, applied = 0;
  bool mlp_off = false;
  // device-driven (batched) stepping
  double* p_dev = nullptr;     // input samples on the device
  int batch = 0;               // id of the batch holding the model (0: none)
  int version = 0;             // bumped when a captured step graph would be stale
  // host-driven steps: the inner solve captured once as a CUDA graph
  cudaGraphExec_t ig_exec = nullptr;
  int ig_version = -1;
  float lo_variant_ms[kLoVariants] = {0.f, 0.f, 0.f};
  LoView<float> lo_f;
  LoView<__half> lo_h;
  // directional analyses of gsw_run's direction mask: one instance per input
  // direction, sharing this model's mesh, element, preconditioner and
  // inner-operator data (read-only, owned here) and holding its own state,
  // solver vectors and receiver history
  Model* parent = nullptr;                      // set on an instance
  Model* inst[3] = {nullptr, nullptr, nullptr};  // instances (parent only)
  int inst_version[3] = {-1, -1, -1};           // parent version each was made for
  std::vector<double> dir_input[3];             // input of each direction (parent only)
  // kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double ebe_ms = 0.0;
  int64_t ebe_count = 0;
  double lo_ms = 0.0;
  int64_t lo_count = 0;
  std::vector<cudaEvent_t> ev_lo;

  ModelView view() const {
    ModelView m;
    m.N = N;
    m.E = E;
    m.F = F;
    m.conn = conn;
    m.geo = geo;
    m.emat = emat;
    m.mat = mat;
    m.fnode = fnode;
    m.fgeo = fgeo;
    m.dt = dt;
    return m;
  }
};

}  // namespace

struct gsw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free_)(void*, void*, void*) = nullptr;
  void* user = nullptr;
  std::map<int, Model*> models;
  int next_id = 1;
  MisfitWork misfit;
  std::map<int, struct Batch*> batches;
  int next_batch = 1;
};

// A set of models advanced together: one CUDA graph per time step holds every
// model's device-driven step on its own stream branch.
// Kernel launches of one captured step, split into the part issued once per
// step and the device-side loop body (issued once per further outer iteration).
// PCG iterations an FP64 member's step may run inside the step graph's
// device-side loop (batch_outer = 0); a step that needs more is finished by
// the host-driven solver.
constexpr int kFp64LoopCap = 1000;

struct StepLaunches {
  int64_t fixed = 0, body = 0;
};

struct Batch {
  std::vector<Model*> members;  // models or direction instances
  std::vector<int> ids;         // model id of each member (for messages)
  std::vector<int> dirs;        // input direction of an instance member, -1 for a model
  // members i .. i + lane[i] - 1 advance in lockstep on stream i (lane[i] = 0:
  // inside an earlier member's lane); 1 = on its own
  std::vector<int> lane;
  std::vector<int> versions;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr, done_ev = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  StepState* ss_dev = nullptr;
  StepState* ss_host = nullptr;  // pinned
  int64_t launches_per_step = 0;
  int outer = 0;
  int fp64_loop = 0;  // device-side loop budget of the FP64 members when captured
  // adaptive budget (members with batch_outer == 0): outer iterations captured
  // per step, and the chunks in a row whose steps needed fewer
  int adapt_outer = 6;
  int lower_streak = 0, lower_max = 0;
  // device-side outer loop (WHILE conditional nodes); off after a failed build
  bool use_while = true;
  cudaStream_t body_stream = nullptr;
  std::vector<StepLaunches> launches;  // per member, of the captured step
};

namespace {

gsw_status fail(gsw_ctx* c, gsw_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, GSW_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                    \
  } while (0)

// NVTX range over a scope (time step, batch step, CG phase) for profilers.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

void* dev_alloc(gsw_ctx* ctx, Model* m, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, (void*)ctx->stream, ctx->user);
  } else if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
    p = nullptr;
  }
  if (p && m) {
    m->allocs.push_back(p);
    m->bytes += bytes;
  }
  return p;
}

void dev_free(gsw_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->free_)
    ctx->free_(p, (void*)ctx->stream, ctx->user);
  else
    cudaFreeAsync(p, ctx->stream);
}

template <class T>
gsw_status alloc_into(gsw_ctx* ctx, Model* m, T** out, size_t count) {
  *out = (T*)dev_alloc(ctx, m, sizeof(T) * count);
  if (!*out) return fail(ctx, GSW_E_NOMEM, "device allocation of %zu bytes failed", sizeof(T) * count);
  return GSW_OK;
}

#define TRY(expr)               \
  do {                          \
    gsw_status s_ = (expr);     \
    if (s_ != GSW_OK) return s_; \
  } while (0)

void free_model(gsw_ctx* ctx, Model* m) {
  for (int d = 0; d < 3; ++d)
    if (m->inst[d]) {
      free_model(ctx, m->inst[d]);
      m->inst[d] = nullptr;
    }
  if (m->ig_exec) cudaGraphExecDestroy(m->ig_exec);
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : m->ev_lo) cudaEventDestroy(e);
  for (void* p : m->allocs) dev_free(ctx, p);
  m->allocs.clear();
  if (m->cg_host) cudaFreeHost(m->cg_host);
  delete m;
}

Model* find(gsw_ctx* ctx, int id) {
  auto it = ctx->models.find(id);
  return it == ctx->models.end() ? nullptr : it->second;
}

gsw_status check_device_err(gsw_ctx* ctx, Model* m, const char* what) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    std::string msg;
    if (h & 1) msg += " non-positive or non-finite element volume;";
    if (h & 2) msg += " curved element (mid-edge node off the edge midpoint);";
    if (h & 4) msg += " degenerate boundary face;";
    if (h & 8) msg += " singular nodal diagonal block;";
    if (h & 16) msg += " receiver outside the free surface;";
    return fail(ctx, GSW_E_INVALID, "%s:%s", what, msg.c_str());
  }
  return GSW_OK;
}

// Structure-of-arrays transpose of a row-major [n][k] int32 table.
std::vector<int32_t> soa(const int32_t* src, int64_t n, int k) {
  std::vector<int32_t> out((size_t)n * k);
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < k; ++j) out[(size_t)j * n + i] = src[(size_t)i * k + j];
  return out;
}

// Step-dependent state of an analysis; own_precond: also the block-Jacobi
// blocks (an instance shares its parent's).
gsw_status model_state_alloc(gsw_ctx* ctx, Model* m, bool own_precond = true) {
  const size_t n3 = 3 * (size_t)m->N;
  TRY(alloc_into(ctx, m, &m->u, n3));
  TRY(alloc_into(ctx, m, &m->v, n3));
  TRY(alloc_into(ctx, m, &m->a, n3));
  TRY(alloc_into(ctx, m, &m->b, n3));
  TRY(alloc_into(ctx, m, &m->x, n3));
  TRY(alloc_into(ctx, m, &m->r, n3));
  TRY(alloc_into(ctx, m, &m->z, n3));
  TRY(alloc_into(ctx, m, &m->p, n3));
  TRY(alloc_into(ctx, m, &m->q, n3));
  if (own_precond) {
    TRY(alloc_into(ctx, m, &m->dblk, 6 * (size_t)m->N));
    TRY(alloc_into(ctx, m, &m->dinv, 6 * (size_t)m->N));
  }
  ModelView mv = m->view();
  size_t np = (size_t)ebe_blocks(mv) + 2;
  if (np < 2 * (size_t)kMaxNodeBlocks) np = 2 * (size_t)kMaxNodeBlocks;
  TRY(alloc_into(ctx, m, &m->partials, np));
  TRY(alloc_into(ctx, m, &m->cg, 1));
  if (!m->cg_host) CK(cudaMallocHost(&m->cg_host, sizeof(CgScalars)));
  TRY(alloc_into(ctx, m, &m->wave, (size_t)m->n_rec * 3 * (size_t)(m->n_steps > 0 ? m->n_steps : 1)));
  return GSW_OK;
}

// The projection guess hands over to the extrapolation of order guess_order
// once a step starts from an initial relative residual below proj_relres.
bool proj_hands_over(const Model* m) {
  return m->opts.proj_dim > 0 && m->opts.proj_relres > 0.0 && m->opts.guess_order > 0;
}

// Buffers of the projection guess (proj_dim > 0): W, Z, the step's b, state.
gsw_status proj_alloc(gsw_ctx* ctx, Model* m, int k) {
  if (k <= 0 || (m->proj && m->proj_k >= k)) return GSW_OK;
  const size_t n3 = 3 * (size_t)m->N;
  TRY(alloc_into(ctx, m, &m->proj_W, (size_t)k * n3));
  TRY(alloc_into(ctx, m, &m->proj_Z, (size_t)k * n3));
  if (!m->proj_b) TRY(alloc_into(ctx, m, &m->proj_b, n3));
  if (!m->proj_part) TRY(alloc_into(ctx, m, &m->proj_part, 2 * (size_t)kMaxProj * kMaxNodeBlocks));
  if (!m->proj) TRY(alloc_into(ctx, m, &m->proj, 1));
  CK(cudaMemsetAsync(m->proj, 0, sizeof(ProjState), ctx->stream));
  m->proj_k = k;
  return GSW_OK;
}

gsw_status model_reset(gsw_ctx* ctx, Model* m) {
  const size_t n3 = 3 * (size_t)m->N;
  CK(cudaMemsetAsync(m->u, 0, sizeof(double) * n3, ctx->stream));
  CK(cudaMemsetAsync(m->v, 0, sizeof(double) * n3, ctx->stream));
  CK(cudaMemsetAsync(m->a, 0, sizeof(double) * n3, ctx->stream));
  CK(cudaMemsetAsync(m->wave, 0, sizeof(double) * (size_t)m->n_rec * 3 * (size_t)m->n_steps, ctx->stream));
  CK(cudaMemsetAsync(m->cg, 0, sizeof(CgScalars), ctx->stream));
  m->step = 0;
  m->failed = false;
  m->stats = gsw_stats{};
  if (m->guess_ext) CK(cudaMemsetAsync(m->guess_ext, 0, 2 * sizeof(int), ctx->stream));  // no increment history
  if (m->proj) CK(cudaMemsetAsync(m->proj, 0, sizeof(ProjState), ctx->stream));
  if (m->lo_ready) {
    // a wait of the inner operator that ran out failed the run; a reset clears it
    CK(cudaMemsetAsync(&m->isc->err, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemcpyAsync(&m->iters_reset, &m->isc->iters, sizeof(m->iters_reset), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  m->hist_head = 3;
  m->hist_count = 0;
  return GSW_OK;
}

// One Newmark step: RHS (one EBE pass), PCG from the predictor, update, record.
// The CG's (outer) element-by-element operator: hardware FP64, or double-word
// arithmetic on the FP32 pipe (gsw_solver_opts.outer_op; by default the mixed
// modes use double-word, the FP64 mode FP64).
bool outer_dword(const Model* m) {
  return m->opts.outer_op == GSW_OUTER_DWORD || (m->opts.outer_op == GSW_OUTER_AUTO && m->opts.precision != GSW_PREC_FP64);
}
void launch_outer(const Model* m, int mode, const ModelView& mv, const double* x, const double* v, const double* a,
                  double* y, double force, int dir, double* partials, CgScalars* cg, cudaStream_t s,
                  Drive dr = Drive{nullptr, nullptr}) {
  // the mixed modes keep the search direction and the shifted state as double-word pairs
  if (outer_dword(m))
    launch_ebe_dw(mode, m->opts.precision != GSW_PREC_FP64 ? 1 : 0, mv, x, v, a, y, force, dir, partials, cg, s, dr);
  else
    launch_ebe(mode, mv, x, v, a, y, force, dir, partials, cg, s, dr);
}

gsw_status step_fp64(gsw_ctx* ctx, Model* m) {
  NvtxRange nv("gsw step (FP64 PCG)");
  cudaStream_t s = ctx->stream;
  ModelView mv = m->view();
  const double force = 2.0 * m->input[(size_t)m->step];
  CK(cudaMemsetAsync(m->b, 0, sizeof(double) * 3 * (size_t)m->N, s));
  launch_ebe(kModeRhs, mv, m->u, m->v, m->a, m->b, force, m->dir, nullptr, nullptr, s);
  // scalars: tol / max_iter travel with the state
  CgScalars init = {};
  init.tol = m->opts.tol;
  init.max_iter = m->opts.max_iter;
  CK(cudaMemcpyAsync(m->cg, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
  const int k_guess = m->opts.guess_order;
  const bool proj = m->opts.proj_dim > 0;
  if (proj) {
    // the successor guess first; the projection kernels overwrite it until they retire
    if (proj_hands_over(m))
      launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s);
    launch_proj_coef(m->N, m->proj_W, m->b, m->proj, m->proj_part, s);
    launch_proj_guess(m->N, m->proj_W, m->proj, m->x, s);
  } else if (k_guess > 0) {
    launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s);
  }
  launch_cg_init(mv, m->b, m->v, m->a, m->x, m->q, m->partials, m->cg, s, (k_guess > 0 || proj) ? 1 : 0);
  launch_outer(m, kModeA, mv, m->x, nullptr, nullptr, m->q, 0.0, 0, nullptr, m->cg, s);
  launch_cg_residual(mv, m->b, m->q, m->r, m->z, m->p, m->dinv, m->partials, m->cg, s);
  const int chunk = m->opts.check_every > 0 ? m->opts.check_every : 8;
  int64_t launches = 5;  // rhs, init, A x0, residual (+ newmark and record below)
  if (m->timing && (int)m->ev.size() < 2 * chunk) {
    for (int i = (int)m->ev.size(); i < 2 * chunk; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      m->ev.push_back(e);
    }
  }
  int prev_iter = 0;
  for (;;) {
    m->ev_used = 0;
    for (int k = 0; k < chunk; ++k) {
      if (m->timing) CK(cudaEventRecord(m->ev[2 * k], s));
      launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, s);
      if (m->timing) {
        CK(cudaEventRecord(m->ev[2 * k + 1], s));
        m->ev_used = k + 1;
      }
      launch_cg_update(mv, m->x, m->r, m->z, m->p, m->q, m->dinv, m->partials, m->cg, s);
      launch_cg_pupdate(mv, m->z, m->p, m->cg, s);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(m->cg_host, m->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    launches += 3 * chunk;
    if (m->timing) {
      // time only the launches that did work: one operator product per
      // iteration counted since the previous check (later launches in the
      // chunk returned at entry once the solve had converged)
      const int worked = m->cg_host->iter - prev_iter;
      for (int k = 0; k < worked && k < m->ev_used; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, m->ev[2 * k], m->ev[2 * k + 1]));
        m->ebe_ms += ms;
      }
    }
    prev_iter = m->cg_host->iter;
    if (m->cg_host->done) break;
  }
  const CgScalars& h = *m->cg_host;
  if (h.status != 0) {
    m->failed = true;
    if (h.status == GSW_E_NOCONV)
      return fail(ctx, GSW_E_NOCONV, "step %lld: CG did not reach %g in %d iterations (at %g)",
                  (long long)m->step, m->opts.tol, h.iter, h.relres);
    return fail(ctx, GSW_E_NAN, "step %lld: non-finite CG residual", (long long)m->step);
  }
  if (proj)
    launch_proj_push(m->N, m->x, m->b, m->r, m->proj_W, m->proj_Z, m->proj, m->opts.proj_dim, m->proj_part, s,
                     nullptr, m->cg, m->opts.proj_relres);
  if ((!proj || proj_hands_over(m)) && m->opts.guess_order > 0)
    launch_guess_push(m->N, m->x, m->guess_ring, m->opts.guess_order, m->guess_ext, s);
  launch_newmark(mv, m->x, m->u, m->v, m->a, m->cg, s);
  launch_record(m->v, m->rec_node, m->rec_w, m->n_rec, m->wave, m->n_steps, (int)m->step, s);
  CK(cudaGetLastError());
  m->stats.steps_done += 1;
  m->stats.cg_iters_total += h.iter;
  m->stats.cg_iters_last = h.iter;
  if (h.iter > m->stats.cg_iters_max) m->stats.cg_iters_max = h.iter;
  m->stats.relres_last = h.relres;
  m->stats.kernel_launches += launches + 2;
  if (m->timing) m->ebe_count += h.iter;
  m->step += 1;
  return GSW_OK;
}

// Set-up autotuner of the inner operator: times every launch variant on this
// model's own data (search direction = the state u, zero after a reset) and
// keeps the fastest.
gsw_status autotune_lo(gsw_ctx* ctx, Model* m) {
  cudaStream_t s = ctx->stream;
  const void* view = m->lo_half ? (const void*)&m->lo_h : (const void*)&m->lo_f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch_to_lo(m->N, m->u, m->d_lo, m->lo_half, m->w32, s);
  CK(cudaMemsetAsync(&m->isc->err, 0, sizeof(unsigned int), s));
  // rounds interleave the variants so none profits from a cache warmed by
  // another; each variant keeps the median of its rounds
  constexpr int kRounds = 5;
  float t[kLoVariants][kRounds] = {};
  for (int v = 0; v < kLoVariants; ++v)  // warm-up (and the pipelined kernel's attributes)
    launch_ebe_lo(m->lo_half, m->lo_half, view, m->d_lo, m->w32, m->partials, m->isc, s, v);
  for (int rnd = 0; rnd < kRounds; ++rnd) {
    for (int v = 0; v < kLoVariants; ++v) {
      if (m->opts.inner_variant >= 0 && v != m->opts.inner_variant) continue;
      CK(cudaEventRecord(e0, s));
      launch_ebe_lo(m->lo_half, m->lo_half, view, m->d_lo, m->w32, m->partials, m->isc, s, v);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&t[v][rnd], e0, e1));
    }
  }
  float best = 1e30f;
  for (int v = 0; v < kLoVariants; ++v) {
    if (m->opts.inner_variant >= 0 && v != m->opts.inner_variant) continue;
    std::sort(t[v], t[v] + kRounds);
    m->lo_variant_ms[v] = t[v][kRounds / 2];
    if (t[v][kRounds / 2] < best) {
      best = t[v][kRounds / 2];
      m->lo_variant = v;
    }
  }
  CK(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  unsigned int err = 0;
  CK(cudaMemcpyAsync(&err, &m->isc->err, sizeof(err), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err) return fail(ctx, GSW_E_TIMEOUT, "inner operator: a bounded device-side wait ran out");
  return GSW_OK;
}

// Element blocks with local numbering and the reduced-precision copies of the
// operator data and preconditioner (built once per model; the conversion is
// redone when dt changes).
// First-order coarse level of the two-level inner preconditioner: the
// vertices (the first four nodes of each element), the vertex pair each fine
// node interpolates and, per vertex, the mid-edge nodes of its edges (CSR, in
// ascending node order) are built on first use from the connectivity; the
// blocks of P^T A P and omega D_c^-1 again with every rebuild of the inner
// operator (they depend on dt, the materials and omega).
gsw_status build_coarse(gsw_ctx* ctx, Model* m) {
  cudaStream_t s = ctx->stream;
  if (!m->cv_node) {
    static const int ea[6] = {0, 1, 0, 0, 1, 2}, eb[6] = {1, 2, 2, 3, 3, 3};  // the element's edge order
    const int64_t N = m->N, E = m->E;
    std::vector<int32_t> conn((size_t)10 * E);  // [10][E]
    CK(cudaMemcpyAsync(conn.data(), m->conn, sizeof(int32_t) * conn.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int32_t> vid((size_t)N, -1), vnode;
    for (int k = 0; k < 4; ++k)
      for (int64_t e = 0; e < E; ++e) vid[(size_t)conn[(size_t)(k * E + e)]] = 0;
    int32_t nv = 0;
    for (int64_t n = 0; n < N; ++n)
      if (vid[(size_t)n] == 0) {
        vid[(size_t)n] = nv++;
        vnode.push_back((int32_t)n);
      }
    std::vector<int2> pair((size_t)N, make_int2(-1, -1));
    for (int64_t n = 0; n < N; ++n)
      if (vid[(size_t)n] >= 0) pair[(size_t)n] = make_int2(vid[(size_t)n], vid[(size_t)n]);
    for (int k = 0; k < 6; ++k)
      for (int64_t e = 0; e < E; ++e) {
        const int32_t mn = conn[(size_t)((4 + k) * E + e)];
        int32_t a = vid[(size_t)conn[(size_t)(ea[k] * E + e)]], b = vid[(size_t)conn[(size_t)(eb[k] * E + e)]];
        if (a > b) std::swap(a, b);
        if (vid[(size_t)mn] >= 0)
          return fail(ctx, GSW_E_INVALID, "node %d is both a vertex and a mid-edge node", mn);
        int2& p = pair[(size_t)mn];
        if (p.x < 0)
          p = make_int2(a, b);
        else if (p.x != a || p.y != b)
          return fail(ctx, GSW_E_INVALID, "mid-edge node %d lies on two different edges", mn);
      }
    std::vector<int32_t> ptr((size_t)nv + 1, 0);
    for (int64_t n = 0; n < N; ++n) {
      const int2 p = pair[(size_t)n];
      if (p.x < 0) return fail(ctx, GSW_E_INVALID, "node %lld belongs to no element", (long long)n);
      if (p.x != p.y) {
        ptr[(size_t)p.x + 1] += 1;
        ptr[(size_t)p.y + 1] += 1;
      }
    }
    for (int32_t v = 0; v < nv; ++v) ptr[(size_t)v + 1] += ptr[(size_t)v];
    std::vector<int32_t> mid((size_t)std::max(ptr[(size_t)nv], 1), 0), fill(ptr.begin(), ptr.end() - 1);
    for (int64_t n = 0; n < N; ++n) {
      const int2 p = pair[(size_t)n];
      if (p.x != p.y) {
        mid[(size_t)fill[(size_t)p.x]++] = (int32_t)n;
        mid[(size_t)fill[(size_t)p.y]++] = (int32_t)n;
      }
    }
    const size_t nvs = (size_t)std::max(nv, 1);
    TRY(alloc_into(ctx, m, &m->cv_node, nvs));
    TRY(alloc_into(ctx, m, &m->cv_ptr, (size_t)nv + 1));
    TRY(alloc_into(ctx, m, &m->cv_mid, mid.size()));
    TRY(alloc_into(ctx, m, &m->c_pair, (size_t)N));
    TRY(alloc_into(ctx, m, &m->c_vid, (size_t)N));
    TRY(alloc_into(ctx, m, &m->cblk, 6 * nvs));
    TRY(alloc_into(ctx, m, &m->cinv, 6 * nvs));
    TRY(alloc_into(ctx, m, &m->cdc, 6 * nvs));
    TRY(alloc_into(ctx, m, &m->zc, nvs));
    CK(cudaMemcpyAsync(m->cv_node, vnode.data(), sizeof(int32_t) * (size_t)nv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->cv_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->cv_mid, mid.data(), sizeof(int32_t) * mid.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->c_pair, pair.data(), sizeof(int2) * (size_t)N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->c_vid, vid.data(), sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(m->zc, 0, sizeof(float4) * nvs, s));
    CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
    m->Nv = nv;
  }
  CK(cudaMemsetAsync(m->cblk, 0, sizeof(double) * 6 * (size_t)m->Nv, s));
  CK(cudaMemsetAsync(m->err, 0, sizeof(int), s));
  launch_coarse_blocks(m->view(), m->c_vid, m->cblk, s);
  launch_invert_blocks(m->Nv, m->cblk, m->cinv, m->err, s);
  launch_coarse_lo(m->Nv, m->cinv, m->isc, m->opts.coarse_weight, m->cdc, s);
  CK(cudaGetLastError());
  return check_device_err(ctx, m, "coarse preconditioner");
}

gsw_status build_lo(gsw_ctx* ctx, Model* m, int half) {
  cudaStream_t s = ctx->stream;
  ModelView mv = m->view();
  if (!m->lo_ready) {
    m->n_blk = (int)((m->E + kLoBlock - 1) / kLoBlock);
    int32_t* counts = nullptr;
    TRY(alloc_into(ctx, m, &counts, (size_t)m->n_blk));
    launch_block_count(mv, m->n_blk, counts, s);
    std::vector<int32_t> h((size_t)m->n_blk), ptr((size_t)m->n_blk + 1);
    CK(cudaMemcpyAsync(h.data(), counts, sizeof(int32_t) * m->n_blk, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // node lists at the fixed stride max_local (a multiple of 4 entries, so
    // 16-byte aligned starts); padding entries name the dummy node N (zero
    // contribution)
    int mx = 4;
    for (int b = 0; b < m->n_blk; ++b) mx = std::max(mx, (h[b] + 3) & ~3);
    for (int b = 0; b <= m->n_blk; ++b) ptr[b] = b * mx;
    m->max_local = mx;
    if ((int64_t)m->n_blk * mx > (int64_t)INT32_MAX)
      return fail(ctx, GSW_E_INVALID, "mesh too large for 32-bit element-block node lists");
    if (mx > kLoBlock * kLoNodesPerThread)
      return fail(ctx, GSW_E_INVALID, "element block with %d unique nodes exceeds %d (mesh ordering too scattered)", mx,
                  kLoBlock * kLoNodesPerThread);
    const int total = ptr[m->n_blk];
    int32_t* refcount = nullptr;
    TRY(alloc_into(ctx, m, &m->blk_ptr, (size_t)m->n_blk + 1));
    TRY(alloc_into(ctx, m, &m->blk_nodes, (size_t)total));
    TRY(alloc_into(ctx, m, &m->lconn, 10 * (size_t)m->n_blk * kLoBlock));
    TRY(alloc_into(ctx, m, &refcount, (size_t)m->N + 1));
    CK(cudaMemcpyAsync(m->blk_ptr, ptr.data(), sizeof(int32_t) * (m->n_blk + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(refcount, 0, sizeof(int32_t) * (m->N + 1), s));
    BlockView bv = {m->n_blk, m->max_local, m->blk_ptr, m->blk_nodes};
    launch_block_fill(mv, bv, m->blk_nodes, m->lconn, refcount, s, counts);
    launch_block_mark(mv, bv, m->blk_nodes, refcount, total, s);
    CK(cudaGetLastError());
    const size_t n3 = 3 * (size_t)m->N;
    TRY(alloc_into(ctx, m, &m->fgeo32, 6 * (size_t)(m->F > 0 ? m->F : 1)));
    TRY(alloc_into(ctx, m, &m->dinv32, 6 * (size_t)m->N));
    TRY(alloc_into(ctx, m, &m->y32, n3));
    TRY(alloc_into(ctx, m, &m->s32, n3));
    TRY(alloc_into(ctx, m, &m->t32, 4 * ((size_t)m->N + 1)));  // padded: 4 entries per node
    CK(cudaMemsetAsync(m->t32, 0, sizeof(float) * 4 * ((size_t)m->N + 1), s));  // the dummy node's row stays 0
    TRY(alloc_into(ctx, m, &m->w32, n3 + 4));  // + the dummy node's row
    TRY(alloc_into(ctx, m, &m->isc, 1));
    TRY(alloc_into(ctx, m, &m->dw_part, (size_t)m->n_blk + (size_t)((m->F + kLoBlock - 1) / kLoBlock) + 1));
    TRY(alloc_into(ctx, m, &m->matf, (size_t)3 * kMaxMat));
    TRY(alloc_into(ctx, m, &m->uva, 3 * ((size_t)m->N + 1)));
    CK(cudaMemsetAsync(m->uva, 0, sizeof(float4) * 3 * ((size_t)m->N + 1), s));
    CK(cudaMemsetAsync(m->isc, 0, sizeof(InnerScalars), s));
    m->lo_ready = true;
    m->geo_lo = nullptr;
    m->d_lo = nullptr;
    m->d_lo2 = nullptr;
  }
  if (m->geo_lo == nullptr || m->lo_half != half) {
    // (re)allocate the precision-dependent buffers; the old ones stay owned by the model
    m->geo_lo = dev_alloc(ctx, m, lo_record_bytes(half) * (size_t)m->n_blk * kLoBlock);
    const size_t dbytes = (half ? sizeof(__half) : sizeof(float)) * 4 * ((size_t)m->N + 1);
    m->d_lo = dev_alloc(ctx, m, dbytes);
    m->d_lo2 = dev_alloc(ctx, m, dbytes);
    if (!m->geo_lo || !m->d_lo || !m->d_lo2) return fail(ctx, GSW_E_NOMEM, "device allocation failed (inner solve)");
    CK(cudaMemsetAsync(m->d_lo, 0, dbytes, s));
    CK(cudaMemsetAsync(m->d_lo2, 0, dbytes, s));
    m->lo_half = half;
  }
  launch_lo_convert(mv, m->n_blk, m->lconn, half, half, m->geo_lo, m->fgeo32, m->dinv, m->dinv32, m->partials, m->isc,
                    m->matf, m->n_mat, s);
  CK(cudaGetLastError());
  BlockView bv = {m->n_blk, m->max_local, m->blk_ptr, m->blk_nodes};
  const float face_c = (float)(2.0 / m->dt / 180.0);
  m->lo_f = LoView<float>{m->N, m->E, m->F, m->n_mat, bv, m->geo_lo, m->matf, m->fnode, m->fgeo32, m->dt,
                          m->dw_part, face_c};
  m->lo_h = LoView<__half>{m->N, m->E, m->F, m->n_mat, bv, m->geo_lo, m->matf, m->fnode, m->fgeo32, m->dt,
                           m->dw_part, face_c};
  if (m->opts.coarse_weight > 0.0) TRY(build_coarse(ctx, m));
  m->live_tune = (m->opts.inner_variant < 0);
  return autotune_lo(ctx, m);
}

// The analysis of input direction d of model m, sharing m's mesh, element,
// preconditioner and inner-operator data; its own state, CG and inner
// vectors, increment history and receiver history; at rest.
gsw_status make_instance(gsw_ctx* ctx, Model* m, int d, Model** out) {
  Model* c = new Model();
  c->parent = m;
  c->N = m->N;
  c->E = m->E;
  c->F = m->F;
  c->n_mat = m->n_mat;
  c->n_rec = m->n_rec;
  c->period[0] = m->period[0];
  c->period[1] = m->period[1];
  c->raw_mat = m->raw_mat;
  c->xyz = m->xyz;
  c->conn = m->conn;
  c->geo = m->geo;
  c->emat = m->emat;
  c->raw_mat_dev = m->raw_mat_dev;
  c->mat = m->mat;
  c->fnode = m->fnode;
  c->face_elem = m->face_elem;
  c->face_tag = m->face_tag;
  c->fgeo = m->fgeo;
  c->rec_xy = m->rec_xy;
  c->rec_face = m->rec_face;
  c->rec_node = m->rec_node;
  c->rec_w = m->rec_w;
  c->err = m->err;
  c->time_set = true;
  c->dt = m->dt;
  c->f1 = m->f1;
  c->f2 = m->f2;
  c->n_steps = m->n_steps;
  c->dblk = m->dblk;
  c->dinv = m->dinv;
  c->opts = m->opts;
  c->dir = d;
  c->input = m->dir_input[d];
  c->input_set = true;
  cudaStream_t s = ctx->stream;
  auto bail = [&](gsw_status st) {
    cudaStreamSynchronize(s);
    free_model(ctx, c);
    return st;
  };
#define TRYI(expr)                   \
  do {                               \
    gsw_status s_ = (expr);          \
    if (s_ != GSW_OK) return bail(s_); \
  } while (0)
  TRYI(model_state_alloc(ctx, c, false));
  if (c->opts.guess_order > 0) {
    TRYI(alloc_into(ctx, c, &c->guess_ext, 2));
    TRYI(alloc_into(ctx, c, &c->guess_ring, (size_t)(c->opts.guess_order + 1) * 3 * (size_t)c->N));
    c->guess_ring_k = c->opts.guess_order;
  }
  TRYI(proj_alloc(ctx, c, c->opts.proj_dim));
  if (m->lo_ready && m->opts.precision != GSW_PREC_FP64) {
    c->lo_half = m->lo_half;
    c->n_blk = m->n_blk;
    c->max_local = m->max_local;
    c->blk_ptr = m->blk_ptr;
    c->blk_nodes = m->blk_nodes;
    c->lconn = m->lconn;
    c->geo_lo = m->geo_lo;
    c->fgeo32 = m->fgeo32;
    c->dinv32 = m->dinv32;
    c->matf = m->matf;
    if (m->zc) {
      c->Nv = m->Nv;
      c->cv_node = m->cv_node;
      c->cv_ptr = m->cv_ptr;
      c->cv_mid = m->cv_mid;
      c->c_pair = m->c_pair;
      c->cdc = m->cdc;
      TRYI(alloc_into(ctx, c, &c->zc, (size_t)std::max<int64_t>(m->Nv, 1)));
    }
    c->lo_variant = m->lo_variant;
    for (int v = 0; v < kLoVariants; ++v) c->lo_variant_ms[v] = m->lo_variant_ms[v];
    const size_t n3 = 3 * (size_t)c->N;
    TRYI(alloc_into(ctx, c, &c->y32, n3));
    TRYI(alloc_into(ctx, c, &c->s32, n3));
    TRYI(alloc_into(ctx, c, &c->t32, 4 * ((size_t)c->N + 1)));
    TRYI(alloc_into(ctx, c, &c->w32, n3 + 4));
    TRYI(alloc_into(ctx, c, &c->isc, 1));
    TRYI(alloc_into(ctx, c, &c->dw_part, (size_t)c->n_blk + (size_t)((c->F + kLoBlock - 1) / kLoBlock) + 1));
    TRYI(alloc_into(ctx, c, &c->uva, 3 * ((size_t)c->N + 1)));
    const size_t dbytes = (c->lo_half ? sizeof(__half) : sizeof(float)) * 4 * ((size_t)c->N + 1);
    c->d_lo = dev_alloc(ctx, c, dbytes);
    c->d_lo2 = dev_alloc(ctx, c, dbytes);
    if (!c->d_lo || !c->d_lo2) return bail(fail(ctx, GSW_E_NOMEM, "device allocation failed (inner solve)"));
    if (cudaMemsetAsync(c->t32, 0, sizeof(float) * 4 * ((size_t)c->N + 1), s) != cudaSuccess ||
        cudaMemsetAsync(c->uva, 0, sizeof(float4) * 3 * ((size_t)c->N + 1), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_lo, 0, dbytes, s) != cudaSuccess || cudaMemsetAsync(c->d_lo2, 0, dbytes, s) != cudaSuccess ||
        cudaMemcpyAsync(c->isc, m->isc, sizeof(InnerScalars), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return bail(fail(ctx, GSW_E_CUDA, "instance set-up copies failed"));
    BlockView bv = {c->n_blk, c->max_local, c->blk_ptr, c->blk_nodes};
    const float face_c = (float)(2.0 / c->dt / 180.0);
    c->lo_f = LoView<float>{c->N, c->E, c->F, c->n_mat, bv, c->geo_lo, c->matf, c->fnode, c->fgeo32, c->dt,
                            c->dw_part, face_c};
    c->lo_h = LoView<__half>{c->N, c->E, c->F, c->n_mat, bv, c->geo_lo, c->matf, c->fnode, c->fgeo32, c->dt,
                             c->dw_part, face_c};
    c->lo_ready = true;
    c->live_tune = false;
  }
  TRYI(model_reset(ctx, c));
#undef TRYI
  *out = c;
  return GSW_OK;
}

// The up-to-date instance of direction d (made, or re-made after the parent's
// time, input or solver set-up changed).
gsw_status get_instance(gsw_ctx* ctx, Model* m, int d, Model** out) {
  if (m->dir_input[d].empty()) return fail(ctx, GSW_E_STATE, "no input set for direction %d", d);
  if (m->inst[d] && m->inst_version[d] == m->version && m->inst[d]->input == m->dir_input[d]) {
    *out = m->inst[d];
    return GSW_OK;
  }
  if (m->inst[d]) {
    cudaStreamSynchronize(ctx->stream);
    free_model(ctx, m->inst[d]);
    m->inst[d] = nullptr;
  }
  TRY(make_instance(ctx, m, d, &m->inst[d]));
  m->inst_version[d] = m->version;
  *out = m->inst[d];
  return GSW_OK;
}

// ---- learned initial guess ----------------------------------------------------

// Reproducible uniform(-1, 1) from a counter (same on every host).
double hash_uniform(uint32_t seed, uint32_t i) {
  uint64_t z = ((uint64_t)seed << 32) ^ (uint64_t)i;
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) / 9007199254740992.0) - 1.0;
}

gsw_status mlp_alloc(gsw_ctx* ctx, Model* m) {
  if (m->mlp_ready) return GSW_OK;
  TRY(alloc_into(ctx, m, &m->theta, kMlpParams));
  TRY(alloc_into(ctx, m, &m->adam_m, kMlpParams));
  TRY(alloc_into(ctx, m, &m->adam_v, kMlpParams));
  TRY(alloc_into(ctx, m, &m->grad, kMlpParams));
  TRY(alloc_into(ctx, m, &m->packed, (size_t)mlp_packed_words()));
  TRY(alloc_into(ctx, m, &m->hist, 4 * 3 * (size_t)m->N));
  TRY(alloc_into(ctx, m, &m->nodef, 4 * (size_t)m->N));
  TRY(alloc_into(ctx, m, &m->node_mat, (size_t)m->N));
  TRY(alloc_into(ctx, m, &m->trainX, 16 * (size_t)65536));
  TRY(alloc_into(ctx, m, &m->trainY, 3 * (size_t)65536));
  TRY(alloc_into(ctx, m, &m->ms, 1));
  CK(cudaMemsetAsync(m->ms, 0, sizeof(MlpScalars), ctx->stream));
  launch_node_features(m->view(), m->n_mat, m->node_mat, m->nodef, ctx->stream);
  m->mlp_ready = true;
  return GSW_OK;
}

// He-uniform weights (fan-in) with a 100x smaller last layer, zero biases,
// Adam moments and gradients cleared, history emptied.
gsw_status mlp_init(gsw_ctx* ctx, Model* m, uint32_t seed) {
  std::vector<float> th(kMlpParams, 0.f);
  const int offs[3] = {0, 1088, 5248}, fan_in[3] = {16, 64, 64}, count[3] = {1024, 4096, 192};
  for (int l = 0; l < 3; ++l) {
    const double lim = sqrt(6.0 / fan_in[l]) * (l == 2 ? 0.01 : 1.0);
    for (int i = 0; i < count[l]; ++i) th[offs[l] + i] = (float)(lim * hash_uniform(seed + 17u * l, (uint32_t)i));
  }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(m->theta, th.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(m->adam_m, 0, sizeof(float) * kMlpParams, s));
  CK(cudaMemsetAsync(m->adam_v, 0, sizeof(float) * kMlpParams, s));
  CK(cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpParams, s));
  CK(cudaMemsetAsync(m->hist, 0, sizeof(double) * 12 * (size_t)m->N, s));
  launch_mlp_pack(m->theta, m->packed, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  m->hist_head = 3;
  m->hist_count = 0;
  m->adam_t = 0;
  for (int k = 0; k < 5; ++k) m->std_r0_recent[k] = m->mlp_r0_recent[k] = 0.0;
  m->std_r0_n = m->mlp_r0_n = m->applied = 0;
  m->mlp_off = false;
  return GSW_OK;
}

// Before a step: write the learned guess into x when it applies.
bool mlp_use_guess(gsw_ctx* ctx, Model* m, cudaStream_t s, const double* base) {
  (void)ctx;
  if (!m->learn.enable || !m->mlp_ready || m->mlp_off || m->hist_count < 4 || m->step < m->learn.train_steps)
    return false;
  // every 10th step of the application phase is a probe with the plain
  // predictor, keeping the referee's baseline current
  if ((m->applied++ % 10) == 9) return false;
  launch_mlp_sigma(m->N, m->hist, m->partials, m->ms, s);
  launch_mlp_infer(m->N, m->hist, m->nodef, m->packed, m->ms, m->x, nullptr, nullptr, s, base);
  m->stats.kernel_launches += 2;
  return true;
}

// After a converged step (before the Newmark update overwrites v, a): train on
// the converged increment, then push it into the history.
gsw_status mlp_after_step(gsw_ctx* ctx, Model* m, cudaStream_t s, const double* base) {
  if (!m->learn.enable || !m->mlp_ready) return GSW_OK;
  // the scale of the correction to the base guess: this step's targets and
  // the next step's output use it
  launch_mlp_sigma_e(m->N, m->x, base, m->partials, m->ms, s);
  if (m->step < m->learn.train_steps && m->hist_count >= 4 && !m->cg_host->zero_rhs) {
    launch_mlp_sigma(m->N, m->hist, m->partials, m->ms, s);
    CK(cudaMemsetAsync(&m->ms->loss, 0, sizeof(double), s));
    const int B = m->learn.batch;
    for (int it = 0; it < m->learn.iters_per_step; ++it) {
      launch_mlp_sample(m->N, B, m->learn.seed, (int)m->step, it, m->hist, m->nodef, m->x, base, m->ms, m->trainX,
                        m->trainY, s);
      if (launch_mlp_fwdbwd(B, m->trainX, m->trainY, m->theta, m->grad, &m->ms->loss, s))
        return fail(ctx, GSW_E_CUDA, "training kernel configuration failed");
      m->adam_t += 1;
      launch_mlp_adam(m->theta, m->grad, m->adam_m, m->adam_v, m->adam_t, m->learn.lr, s);
    }
    launch_mlp_pack(m->theta, m->packed, s);
    m->stats.kernel_launches += 2 + 3 * m->learn.iters_per_step;
  }
  launch_hist_push(m->N, m->x, m->hist, m->cg, s);
  if (m->hist_count < 4) m->hist_count += 1;
  m->stats.kernel_launches += 1;
  CK(cudaGetLastError());
  return GSW_OK;
}

// Upper bound of the inner operator's grid (element blocks + face CTAs).
int lo_grid_max(const Model* m) { return m->n_blk + (int)((m->F + kLoBlock - 1) / kLoBlock); }
// The direction recurrence is fused into the operator (variants 0, 1) only on
// small models, where launches dominate: on the 2.42 M-element model the fused
// operator costs more than the recurrence kernel it replaces.
bool inner_fuses(const Model* m, int variant) {
  return !m->coarse() && lo_variant_fuses(variant) && lo_grid_max(m) <= kAlphaPrologueMax;
}
// Kernel launches of one inner solve: initialisation, then per iteration the
// operator, the update (+ a one-CTA alpha kernel for large models) and,
// unless the operator fuses it, the direction recurrence (not after the last).
int64_t inner_solve_launches(const Model* m, bool fuse) {
  const int64_t it = m->opts.inner_iters > 0 ? m->opts.inner_iters : 1;
  const int64_t per = (lo_grid_max(m) <= kAlphaPrologueMax ? 2 : 3);
  if (m->coarse()) return 3 + per * it + 2 * (it - 1);  // + restriction and recurrence at the start and per iteration
  return 1 + per * it + (fuse ? 0 : it - 1);
}
// Start of an inner solve: s (the scaled outer residual), y = 0, t = D^-1 s,
// d = t; with the two-level preconditioner also z_c and d = t + P z_c.
void inner_begin(Model* m, cudaStream_t s, float rtol) {
  launch_inner_init(m->N, m->r, m->dinv32, m->s32, m->y32, m->t32, m->d_lo, m->lo_half, m->w32, m->partials, m->isc,
                    m->cg, s, rtol, m->opts.coarse_relres);
  if (m->coarse()) {
    launch_coarse_restrict(m->cview(), m->s32, m->zc, m->partials, m->isc, m->cg, 1, s);
    launch_inner_dupdate(m->N, m->t32, m->d_lo, m->lo_half, m->isc, s, m->cg, m->c_pair, m->zc);
  }
}
// After inner iteration k's operator product (d_k in dk): y, s and t, then,
// except after the last iteration, the next direction (unless the operator
// fuses the recurrence).
void inner_after_op(Model* m, cudaStream_t s, const void* dk, int k, int it, bool fuse) {
  const int half = m->lo_half;
  if (m->coarse()) {
    launch_inner_update_coarse(m->N, m->y32, m->s32, m->t32, dk, half, m->w32, m->dinv32, m->dw_part, m->partials,
                               m->isc, s, m->cg, lo_grid_max(m));
    if (k + 1 < it) {
      launch_coarse_restrict(m->cview(), m->s32, m->zc, m->partials, m->isc, m->cg, 0, s);
      launch_inner_dupdate(m->N, m->t32, m->d_lo, half, m->isc, s, m->cg, m->c_pair, m->zc);
    }
    return;
  }
  launch_inner_update(m->N, m->y32, m->s32, m->t32, dk, half, m->w32, m->dinv32, m->dw_part, m->partials, m->isc, s,
                      m->cg, lo_grid_max(m));
  if (!fuse && k + 1 < it) launch_inner_dupdate(m->N, m->t32, m->d_lo, half, m->isc, s, m->cg);
}
// Operator product of inner iteration k; returns the direction buffer that
// holds d_k.  With a fusing variant, iteration k > 0 forms d_k = t + beta
// d_{k-1} in its gather and writes it to the other of the two direction
// buffers (no separate recurrence kernel).
void* inner_operator_step(Model* m, cudaStream_t s, const void* view, int k, int variant, bool fuse) {
  const int half = m->lo_half;
  void* dk = (fuse && (k & 1)) ? m->d_lo2 : m->d_lo;
  if (fuse && k > 0) {
    void* dprev = (k & 1) ? m->d_lo : m->d_lo2;
    launch_ebe_lo_fused(half, half, view, dprev, m->t32, dk, m->w32, m->partials, m->isc, s, variant, m->cg);
  } else {
    launch_ebe_lo(half, half, view, dk, m->w32, m->partials, m->isc, s, variant, m->cg);
  }
  return dk;
}

// Inner preconditioner: inner_iters block-Jacobi PCG iterations in reduced
// precision on the scaled outer residual; result in y32 (scaled).
int64_t inner_solve(Model* m, cudaStream_t s) {
  const int half = m->lo_half;
  const void* view = half ? (const void*)&m->lo_h : (const void*)&m->lo_f;
  const int it = m->opts.inner_iters > 0 ? m->opts.inner_iters : 1;
  // live tuning: inside the first host-driven inner solve the launch variants
  // take turns (in the cache state of a real solve) and the fastest median
  // wins; that solve runs all inner_iters iterations
  const bool tune = m->live_tune && it >= 2 * kLoVariants && (int)m->ev_lo.size() >= 2 * it;
  inner_begin(m, s, tune ? 0.f : (float)m->opts.inner_rtol);
  const bool timed = (m->timing || tune) && (int)m->ev_lo.size() >= 2 * it;
  const bool fuse = !tune && inner_fuses(m, m->lo_variant);
  for (int k = 0; k < it; ++k) {
    const int variant = tune ? k % kLoVariants : m->lo_variant;
    if (timed) cudaEventRecord(m->ev_lo[2 * k], s);
    void* dk = inner_operator_step(m, s, view, k, variant, fuse);
    if (timed) cudaEventRecord(m->ev_lo[2 * k + 1], s);
    inner_after_op(m, s, dk, k, it, fuse);
  }
  m->stats.inner_iters_total += it;
  if (timed) {
    cudaEventSynchronize(m->ev_lo[2 * it - 1]);
    std::vector<float> per[kLoVariants], msv((size_t)it, 0.f);
    for (int k = 0; k < it; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, m->ev_lo[2 * k], m->ev_lo[2 * k + 1]) != cudaSuccess) continue;
      msv[(size_t)k] = ms;
      if (tune && k >= kLoVariants) per[k % kLoVariants].push_back(ms);  // the first round warms up
    }
    if (m->timing) {
      // executed iterations: a solve that met inner_rtol returns at entry from the
      // remaining launches, which are not operator applications and are not counted
      unsigned long long n = 0;
      if (cudaMemcpyAsync(&n, &m->isc->iters, sizeof(n), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          cudaStreamSynchronize(s) == cudaSuccess) {
        const int64_t done = (int64_t)(n - m->iters_mark);
        for (int64_t k = 0; k < done && k < it; ++k) m->lo_ms += msv[(size_t)k];
        m->lo_count += done;
        m->iters_mark = n;
      }
    }
    if (tune) {
      float best = 1e30f;
      for (int v = 0; v < kLoVariants; ++v) {
        if (per[v].empty()) continue;
        std::sort(per[v].begin(), per[v].end());
        const float med = per[v][per[v].size() / 2];
        m->lo_variant_ms[v] = med;
        if (med < best) {
          best = med;
          m->lo_variant = v;
        }
      }
      m->live_tune = false;
      m->version += 1;  // a captured batch graph must pick up the choice
    }
  }
  return inner_solve_launches(m, fuse);
}

// Host-driven steps after the live tuning: the inner solve's launches (about
// four per inner iteration) are captured once into a CUDA graph, re-captured
// when the model's version changes (solver options, time step, tuning
// choice), and launched as one graph per outer iteration.  With kernel timing
// on, or where the stream cannot be captured, the launches are issued directly.
void inner_solve_dev(Model* m, cudaStream_t s);
int64_t inner_solve_step(Model* m, cudaStream_t s) {
  NvtxRange nv("gsw inner solve");
  if (m->timing || m->live_tune) return inner_solve(m, s);
  if (m->ig_version != m->version) {
    if (m->ig_exec) cudaGraphExecDestroy(m->ig_exec);
    m->ig_exec = nullptr;
    m->ig_version = m->version;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      inner_solve_dev(m, s);
      if (cudaStreamEndCapture(s, &g) == cudaSuccess && g != nullptr) {
        if (cudaGraphInstantiate(&m->ig_exec, g, 0) != cudaSuccess) m->ig_exec = nullptr;
        cudaGraphDestroy(g);
      }
    }
    cudaGetLastError();  // a failed capture leaves the direct launches
  }
  if (!m->ig_exec || cudaGraphLaunch(m->ig_exec, s) != cudaSuccess) return inner_solve(m, s);
  m->stats.inner_iters_total += m->opts.inner_iters > 0 ? m->opts.inner_iters : 1;
  return inner_solve_launches(m, inner_fuses(m, m->lo_variant));
}

// One Newmark step with flexible CG (FP64) preconditioned by the inner solve.
gsw_status step_mixed(gsw_ctx* ctx, Model* m) {
  NvtxRange nv("gsw step (flexible CG)");
  cudaStream_t s = ctx->stream;
  ModelView mv = m->view();
  const double force = 2.0 * m->input[(size_t)m->step];
  // ||b|| from an FP32 right-hand side (w32 is free scratch between solves)
  CK(cudaMemsetAsync(m->w32, 0, sizeof(float) * 3 * (size_t)m->N, s));
  launch_rhs_lo(m->lo_half, m->lo_half ? (const void*)&m->lo_h : (const void*)&m->lo_f, m->N, m->u, m->v, m->a,
                m->uva, m->w32, force, m->dir, s);
  CgScalars init = {};
  init.tol = m->opts.tol;
  init.max_iter = m->opts.max_iter;
  CK(cudaMemcpyAsync(m->cg, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
  // initial guess (predictor, extrapolation or learned) and the shifted state (u~ in p, v~ in z, a~ in b),
  // r = q = 0; with learning the network corrects the step's base guess (the
  // extrapolation at guess order > 0, else the predictor), kept in guess_base
  double* base = nullptr;
  if (m->learn.enable) {
    if (!m->guess_base) TRY(alloc_into(ctx, m, &m->guess_base, 3 * (size_t)m->N));
    base = m->guess_base;
    if (m->opts.guess_order > 0)
      launch_guess_extrap(m->N, m->guess_ring, m->opts.guess_order, m->guess_ext, m->v, m->a, m->dt, base, s);
    else
      launch_predictor(m->N, m->v, m->a, m->dt, base, s);
  }
  const bool learned = mlp_use_guess(ctx, m, s, base);
  const bool proj = m->opts.proj_dim > 0;
  const bool extrap = !learned && !proj && m->opts.guess_order > 0;
  if (extrap && base)
    CK(cudaMemcpyAsync(m->x, base, sizeof(double) * 3 * (size_t)m->N, cudaMemcpyDeviceToDevice, s));
  else if (extrap)
    launch_guess_extrap(m->N, m->guess_ring, m->opts.guess_order, m->guess_ext, m->v, m->a, m->dt, m->x, s);
  // the projection guess: the residual pass at du0 = 0 gives b exactly, then du0 = W c and r = b - Z c
  // (once it has handed over, the extrapolation kernel writes the extrapolated guess instead of 0)
  if (proj && proj_hands_over(m))
    launch_guess_extrap(m->N, m->guess_ring, m->opts.guess_order, m->guess_ext, m->v, m->a, m->dt, m->x, s, nullptr,
                        m->proj);
  else if (proj)
    CK(cudaMemsetAsync(m->x, 0, sizeof(double) * 3 * (size_t)m->N, s));
  launch_cg_init_mixed(mv, m->w32, m->u, m->v, m->a, m->x, m->p, m->z, m->b, m->r, m->q, m->partials, m->cg, s,
                       nullptr, (learned || extrap || proj) ? 1 : 0, outer_dword(m) ? 1 : 0);
  // FP64 residual at the initial guess in one element-by-element pass
  launch_outer(m, kModeRes, mv, m->p, m->z, m->b, m->r, force, m->dir, nullptr, m->cg, s);
  if (proj) {
    launch_proj_coef(m->N, m->proj_W, m->r, m->proj, m->proj_part, s);
    launch_proj_apply(m->N, m->proj_W, m->proj_Z, m->proj, m->x, m->r, m->proj_b, s);
  }
  launch_cg_rnorm(mv, m->r, m->partials, m->cg, s);
  int64_t launches = proj ? (proj_hands_over(m) ? 7 : 6) : 4;
  if ((m->timing || m->live_tune) && (int)m->ev_lo.size() < 2 * m->opts.inner_iters) {
    for (int i = (int)m->ev_lo.size(); i < 2 * m->opts.inner_iters; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      m->ev_lo.push_back(e);
    }
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(m->cg_host, m->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  m->stats.init_relres_sum += m->cg_host->relres;
  if (m->learn.enable && !m->cg_host->zero_rhs) {
    // referee: the learned guess stays while the mean initial residual of its
    // last 5 steps beats that of the plain predictor's last 5 steps (the last
    // training steps, then the probe steps)
    double* buf = learned ? m->mlp_r0_recent : m->std_r0_recent;
    int64_t& cnt = learned ? m->mlp_r0_n : m->std_r0_n;
    buf[cnt % 5] = m->cg_host->relres;
    cnt += 1;
    if (learned && m->mlp_r0_n >= 5 && m->std_r0_n >= 1) {
      const int64_t ks = m->std_r0_n < 5 ? m->std_r0_n : 5;
      double ml = 0.0, sl = 0.0;
      for (int k = 0; k < 5; ++k) ml += m->mlp_r0_recent[k] / 5.0;
      for (int64_t k = 0; k < ks; ++k) sl += m->std_r0_recent[k] / (double)ks;
      if (ml > sl) m->mlp_off = true;
    }
  }
  if (!m->cg_host->done) {
    launches += inner_solve_step(m, s);
    launch_fcg_first(mv, m->y32, m->r, m->z, m->p, m->partials, m->cg, m->isc, s, outer_dword(m) ? 1 : 0);
    launches += 1;
    if (m->timing && m->ev.size() < 2) {
      for (int i = (int)m->ev.size(); i < 2; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        m->ev.push_back(e);
      }
    }
    if (m->timing && (int)m->ev_lo.size() < 2 * m->opts.inner_iters) {
      for (int i = (int)m->ev_lo.size(); i < 2 * m->opts.inner_iters; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        m->ev_lo.push_back(e);
      }
    }
    for (;;) {
      if (m->timing) CK(cudaEventRecord(m->ev[0], s));
      launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, s);
      if (m->timing) CK(cudaEventRecord(m->ev[1], s));
      launch_fcg_update(mv, m->x, m->r, m->p, m->q, m->partials, m->cg, s, outer_dword(m) ? 1 : 0);
      launches += 2;
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(m->cg_host, m->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (m->timing) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, m->ev[0], m->ev[1]));
        m->ebe_ms += ms;
        m->ebe_count += 1;
      }
      if (m->cg_host->done) break;
      launches += inner_solve_step(m, s);
      launch_fcg_zbeta(mv, m->y32, m->r, m->q, m->z, m->partials, m->cg, m->isc, s);
      launch_fcg_pupdate(mv, m->z, m->p, m->q, m->cg, s, outer_dword(m) ? 1 : 0);
      launches += 2;
    }
  }
  const CgScalars& h = *m->cg_host;
  if (h.status != 0) {
    m->failed = true;
    if (h.status == GSW_E_NOCONV)
      return fail(ctx, GSW_E_NOCONV, "step %lld: flexible CG did not reach %g in %d iterations (at %g)",
                  (long long)m->step, m->opts.tol, h.iter, h.relres);
    if (h.status == GSW_E_TIMEOUT)
      return fail(ctx, GSW_E_TIMEOUT, "step %lld: a bounded wait of the inner operator ran out", (long long)m->step);
    return fail(ctx, GSW_E_NAN, "step %lld: non-finite CG residual", (long long)m->step);
  }
  TRY(mlp_after_step(ctx, m, s, base));
  if (proj)
    launch_proj_push(m->N, m->x, m->proj_b, m->r, m->proj_W, m->proj_Z, m->proj, m->opts.proj_dim, m->proj_part, s,
                     nullptr, m->cg, m->opts.proj_relres);
  if ((!proj || proj_hands_over(m)) && m->opts.guess_order > 0)
    launch_guess_push(m->N, m->x, m->guess_ring, m->opts.guess_order, m->guess_ext, s);
  launch_newmark(mv, m->x, m->u, m->v, m->a, m->cg, s);
  launch_record(m->v, m->rec_node, m->rec_w, m->n_rec, m->wave, m->n_steps, (int)m->step, s);
  CK(cudaGetLastError());
  m->stats.steps_done += 1;
  m->stats.cg_iters_total += h.iter;
  m->stats.cg_iters_last = h.iter;
  if (h.iter > m->stats.cg_iters_max) m->stats.cg_iters_max = h.iter;
  m->stats.relres_last = h.relres;
  m->stats.kernel_launches += launches + 2;
  m->step += 1;
  return GSW_OK;
}

// Device-driven inner solve (no timing, no host bookkeeping).
void inner_solve_dev(Model* m, cudaStream_t s) {
  const int half = m->lo_half;
  const void* view = half ? (const void*)&m->lo_h : (const void*)&m->lo_f;
  inner_begin(m, s, (float)m->opts.inner_rtol);
  const int it = m->opts.inner_iters > 0 ? m->opts.inner_iters : 1;
  const bool fuse = inner_fuses(m, m->lo_variant);
  for (int k = 0; k < it; ++k) {
    void* dk = inner_operator_step(m, s, view, k, m->lo_variant, fuse);
    inner_after_op(m, s, dk, k, it, fuse);
  }
}

// Iterations 2.. of a captured step's solve.  With a body stream, they run in
// a WHILE conditional node of the graph (device-side loop: the body runs while
// the step has not converged, at most outer - 1 times); otherwise they are
// unrolled `outer` - 1 times (kernels of a converged step return at entry).
// Returns false if the conditional node could not be built.
bool issue_loop(cudaStream_t s, const LoopSet& ls, int outer, cudaStream_t bs, StepLaunches* n,
                int64_t per_iter, const std::function<void(cudaStream_t)>& body) {
  if (bs == nullptr) {
    for (int k = 1; k < outer; ++k) body(s);
    n->fixed += per_iter * (outer - 1);
    return true;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g) != cudaSuccess || cs != cudaStreamCaptureStatusActive) return false;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) return false;
  launch_loop_open(h, ls, outer - 1, s);
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd) != cudaSuccess) return false;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, edges, nd, &p) != cudaSuccess) return false;
  if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return false;
  cudaGraph_t bg = p.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(bs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return false;
  body(bs);
  launch_loop_next(h, ls, outer - 1, bs);
  if (cudaStreamEndCapture(bs, &bg) != cudaSuccess) return false;
  n->fixed += 1;
  n->body += per_iter + 1;
  return true;
}

// Outer (flexible-CG) iterations 2.. of a captured mixed step.
bool issue_outer_loop(Model* m, cudaStream_t s, StepState* ss, int outer, cudaStream_t bs, StepLaunches* n) {
  ModelView mv = m->view();
  const int64_t per_iter = inner_solve_launches(m, inner_fuses(m, m->lo_variant)) + 4;  // + zbeta, pupdate, A p, update
  return issue_loop(s, LoopSet{{ss, nullptr, nullptr}, {m->cg, nullptr, nullptr}, 1}, outer, bs, n, per_iter,
                    [&](cudaStream_t st) {
    inner_solve_dev(m, st);
    launch_fcg_zbeta(mv, m->y32, m->r, m->q, m->z, m->partials, m->cg, m->isc, st);
    launch_fcg_pupdate(mv, m->z, m->p, m->q, m->cg, st, outer_dword(m) ? 1 : 0);
    launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, st);
    launch_fcg_update(mv, m->x, m->r, m->p, m->q, m->partials, m->cg, st, outer_dword(m) ? 1 : 0);
  });
}

// Issues one plain FP64 time step (block-Jacobi PCG) of model m on stream s
// with no host synchronisation: step_begin, right-hand side, initial guess,
// A x0 and the first residual, the PCG iterations in a device-side loop (at
// most `outer` - 1 body runs of one iteration each: A p, update, direction),
// step_end, Newmark update, receivers and step advance.
bool issue_device_step_fp64(Model* m, cudaStream_t s, StepState* ss, int outer, cudaStream_t bs, StepLaunches* n) {
  ModelView mv = m->view();
  Drive dr{m->p_dev, ss};
  launch_step_begin(ss, m->cg, s);
  cudaMemsetAsync(m->b, 0, sizeof(double) * 3 * (size_t)m->N, s);
  launch_ebe(kModeRhs, mv, m->u, m->v, m->a, m->b, 0.0, m->dir, nullptr, nullptr, s, dr);
  const int k_guess = m->opts.guess_order;
  const bool proj = m->opts.proj_dim > 0;
  if (proj) {
    if (proj_hands_over(m))
      launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s, ss);
    launch_proj_coef(m->N, m->proj_W, m->b, m->proj, m->proj_part, s, ss);
    launch_proj_guess(m->N, m->proj_W, m->proj, m->x, s, ss);
  } else if (k_guess > 0) {
    launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s, ss);
  }
  launch_cg_init(mv, m->b, m->v, m->a, m->x, m->q, m->partials, m->cg, s, (k_guess > 0 || proj) ? 1 : 0, ss);
  launch_outer(m, kModeA, mv, m->x, nullptr, nullptr, m->q, 0.0, 0, nullptr, m->cg, s);
  launch_cg_residual(mv, m->b, m->q, m->r, m->z, m->p, m->dinv, m->partials, m->cg, s);
  n->fixed += 6 + (proj ? (proj_hands_over(m) ? 3 : 2) : (k_guess > 0 ? 1 : 0));
  // the first residual may already meet the tolerance; every PCG iteration is a loop body
  if (!issue_loop(s, LoopSet{{ss, nullptr, nullptr}, {m->cg, nullptr, nullptr}, 1}, outer + 1, bs, n, 3,
                  [&](cudaStream_t st) {
        launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, st);
        launch_cg_update(mv, m->x, m->r, m->z, m->p, m->q, m->dinv, m->partials, m->cg, st);
        launch_cg_pupdate(mv, m->z, m->p, m->cg, st);
      }))
    return false;
  launch_step_end(ss, m->cg, s);
  if (proj)
    launch_proj_push(m->N, m->x, m->b, m->r, m->proj_W, m->proj_Z, m->proj, m->opts.proj_dim, m->proj_part, s, ss,
                     m->cg, m->opts.proj_relres);
  if ((!proj || proj_hands_over(m)) && k_guess > 0)
    launch_guess_push(m->N, m->x, m->guess_ring, k_guess, m->guess_ext, s, ss);
  launch_newmark(mv, m->x, m->u, m->v, m->a, m->cg, s, ss);
  launch_record(m->v, m->rec_node, m->rec_w, m->n_rec, m->wave, m->n_steps, 0, s, ss);
  launch_step_advance(ss, s);
  n->fixed += 5;
  return true;
}

// Device-driven start of a mixed step: the initial guess (extrapolation,
// projection or predictor), the shifted state and the FP64 residual at the
// guess in one element-by-element pass, and its norm.
void issue_guess_and_residual(Model* m, cudaStream_t s, StepState* ss, Drive dr, StepLaunches* n) {
  ModelView mv = m->view();
  const int k_guess = m->opts.guess_order;
  const bool proj = m->opts.proj_dim > 0;
  if (proj && proj_hands_over(m))
    launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s, ss, m->proj);
  else if (proj)
    cudaMemsetAsync(m->x, 0, sizeof(double) * 3 * (size_t)m->N, s);
  else if (k_guess > 0)
    launch_guess_extrap(m->N, m->guess_ring, k_guess, m->guess_ext, m->v, m->a, m->dt, m->x, s, ss);
  launch_cg_init_mixed(mv, m->w32, m->u, m->v, m->a, m->x, m->p, m->z, m->b, m->r, m->q, m->partials, m->cg, s, ss,
                       (k_guess > 0 || proj) ? 1 : 0, outer_dword(m) ? 1 : 0);
  launch_outer(m, kModeRes, mv, m->p, m->z, m->b, m->r, 0.0, m->dir, nullptr, m->cg, s, dr);
  if (proj) {
    launch_proj_coef(m->N, m->proj_W, m->r, m->proj, m->proj_part, s, ss);
    launch_proj_apply(m->N, m->proj_W, m->proj_Z, m->proj, m->x, m->r, m->proj_b, s, ss);
  }
  launch_cg_rnorm(mv, m->r, m->partials, m->cg, s);
  n->fixed += 3 + (proj ? (proj_hands_over(m) ? 4 : 3) : (k_guess > 0 ? 1 : 0));
}
// On commit: the converged increment into the guess history.
void issue_history_push(Model* m, cudaStream_t s, StepState* ss, StepLaunches* n) {
  const bool proj = m->opts.proj_dim > 0;
  if (proj) {
    launch_proj_push(m->N, m->x, m->proj_b, m->r, m->proj_W, m->proj_Z, m->proj, m->opts.proj_dim, m->proj_part, s,
                     ss, m->cg, m->opts.proj_relres);
    n->fixed += 1;
  }
  if ((!proj || proj_hands_over(m)) && m->opts.guess_order > 0) {
    launch_guess_push(m->N, m->x, m->guess_ring, m->opts.guess_order, m->guess_ext, s, ss);
    n->fixed += 2;
  }
}

// Issues one mixed time step of model m on stream s with no host
// synchronisation (device-side step counter, input samples and stopping):
// step_begin, FP32 right-hand side, shifted state and FP64 residual, the
// first outer iteration, the remaining ones (see issue_outer_loop), and
// step_end (commit or pause for the host), Newmark update, receivers and
// step advance.  Kernels return at entry once the solve has converged.
bool issue_device_step(Model* m, cudaStream_t s, StepState* ss, int outer, cudaStream_t bs, StepLaunches* n) {
  ModelView mv = m->view();
  Drive dr{m->p_dev, ss};
  const int64_t inner_launches = inner_solve_launches(m, inner_fuses(m, m->lo_variant));
  launch_step_begin(ss, m->cg, s);
  cudaMemsetAsync(m->w32, 0, sizeof(float) * 3 * (size_t)m->N, s);
  launch_rhs_lo(m->lo_half, m->lo_half ? (const void*)&m->lo_h : (const void*)&m->lo_f, m->N, m->u, m->v, m->a,
                m->uva, m->w32, 0.0, m->dir, s, dr);
  issue_guess_and_residual(m, s, ss, dr, n);
  inner_solve_dev(m, s);
  launch_fcg_first(mv, m->y32, m->r, m->z, m->p, m->partials, m->cg, m->isc, s, outer_dword(m) ? 1 : 0);
  launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, s);
  launch_fcg_update(mv, m->x, m->r, m->p, m->q, m->partials, m->cg, s, outer_dword(m) ? 1 : 0);
  n->fixed += 3 + inner_launches + 3;
  if (!issue_outer_loop(m, s, ss, outer, bs, n)) return false;
  launch_step_end(ss, m->cg, s);
  issue_history_push(m, s, ss, n);  // on commit
  launch_newmark(mv, m->x, m->u, m->v, m->a, m->cg, s, ss);
  launch_record(m->v, m->rec_node, m->rec_w, m->n_rec, m->wave, m->n_steps, 0, s, ss);
  launch_step_advance(ss, s);
  n->fixed += 4;
  return true;
}

// Inner solves of a set of direction analyses of one model in lockstep: each
// keeps its own vectors and scalars, and every iteration applies the operator
// to all their search directions in one pass over the shared element data.
void inner_solve_group_dev(Model* const* g, int n, cudaStream_t s) {
  Model* m0 = g[0];
  const int half = m0->lo_half;
  const void* view = half ? (const void*)&m0->lo_h : (const void*)&m0->lo_f;
  for (int i = 0; i < n; ++i) inner_begin(g[i], s, (float)g[i]->opts.inner_rtol);
  Lo3Args a = {};
  a.nr = n;
  for (int i = 0; i < n; ++i) {
    a.d[i] = g[i]->d_lo;
    a.w[i] = g[i]->w32;
    a.dw_part[i] = g[i]->dw_part;
    a.sc[i] = g[i]->isc;
    a.outer[i] = g[i]->cg;
  }
  const int variant = m0->lo_variant == 0 ? 0 : 1;  // the one-CTA-per-block occupancy variants
  const int it = m0->opts.inner_iters > 0 ? m0->opts.inner_iters : 1;
  for (int k = 0; k < it; ++k) {
    launch_ebe_lo3(half, half, view, a, s, variant);
    for (int i = 0; i < n; ++i) inner_after_op(g[i], s, g[i]->d_lo, k, it, false);
  }
}
int64_t inner_group_launches(const Model* m0, int n) {
  const int64_t it = m0->opts.inner_iters > 0 ? m0->opts.inner_iters : 1;
  const int64_t per = (lo_grid_max(m0) <= kAlphaPrologueMax ? 1 : 2);
  if (m0->coarse()) return 3 * n + it * (1 + n * per) + 2 * n * (it - 1);
  return n + it * (1 + n * per) + n * (it - 1);
}

// One mixed time step of the n direction analyses g[0..n) of one model in
// lockstep on stream s (their step states at ss[0..n)): each analysis's
// right-hand side, guess and residual, the shared inner solves, and the
// flexible-CG iterations in one device-side loop that runs while any of the
// analyses has not converged; then each commits (or is handed to the host).
bool issue_device_step_group(Model* const* g, int n, cudaStream_t s, StepState* ss, int outer, cudaStream_t bs,
                             StepLaunches* nl) {
  for (int i = 0; i < n; ++i) {
    Model* m = g[i];
    ModelView mv = m->view();
    Drive dr{m->p_dev, ss + i};
    launch_step_begin(ss + i, m->cg, s);
    cudaMemsetAsync(m->w32, 0, sizeof(float) * 3 * (size_t)m->N, s);
    launch_rhs_lo(m->lo_half, m->lo_half ? (const void*)&m->lo_h : (const void*)&m->lo_f, m->N, m->u, m->v, m->a,
                  m->uva, m->w32, 0.0, m->dir, s, dr);
    issue_guess_and_residual(m, s, ss + i, dr, nl);
    nl->fixed += 3;
  }
  inner_solve_group_dev(g, n, s);
  for (int i = 0; i < n; ++i) {
    Model* m = g[i];
    ModelView mv = m->view();
    launch_fcg_first(mv, m->y32, m->r, m->z, m->p, m->partials, m->cg, m->isc, s, outer_dword(m) ? 1 : 0);
    launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, s);
    launch_fcg_update(mv, m->x, m->r, m->p, m->q, m->partials, m->cg, s, outer_dword(m) ? 1 : 0);
  }
  nl->fixed += inner_group_launches(g[0], n) + 3 * n;
  LoopSet ls = {};
  ls.n = n;
  for (int i = 0; i < n; ++i) {
    ls.ss[i] = ss + i;
    ls.cg[i] = g[i]->cg;
  }
  const int64_t per_iter = inner_group_launches(g[0], n) + 4 * n;
  if (!issue_loop(s, ls, outer, bs, nl, per_iter, [&](cudaStream_t st) {
        inner_solve_group_dev(g, n, st);
        for (int i = 0; i < n; ++i) {
          Model* m = g[i];
          ModelView mv = m->view();
          launch_fcg_zbeta(mv, m->y32, m->r, m->q, m->z, m->partials, m->cg, m->isc, st);
          launch_fcg_pupdate(mv, m->z, m->p, m->q, m->cg, st, outer_dword(m) ? 1 : 0);
          launch_outer(m, kModeA, mv, m->p, nullptr, nullptr, m->q, 0.0, 0, m->partials, m->cg, st);
          launch_fcg_update(mv, m->x, m->r, m->p, m->q, m->partials, m->cg, st, outer_dword(m) ? 1 : 0);
        }
      }))
    return false;
  for (int i = 0; i < n; ++i) {
    Model* m = g[i];
    ModelView mv = m->view();
    launch_step_end(ss + i, m->cg, s);
    issue_history_push(m, s, ss + i, nl);
    launch_newmark(mv, m->x, m->u, m->v, m->a, m->cg, s, ss + i);
    launch_record(m->v, m->rec_node, m->rec_w, m->n_rec, m->wave, m->n_steps, 0, s, ss + i);
    launch_step_advance(ss + i, s);
  }
  nl->fixed += 4 * n;
  return true;
}

void batch_free(gsw_ctx* ctx, Batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->body_stream) cudaStreamDestroy(b->body_stream);
  if (b->ss_dev) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, b->ss_dev);
  }
  if (b->ss_host) cudaFreeHost(b->ss_host);
  delete b;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(p[i])) return false;
  return true;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================

extern "C" {

gsw_status gsw_create(gsw_ctx** out, int device, void* cuda_stream) {
  if (!out) return GSW_E_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GSW_E_CUDA;
  gsw_ctx* ctx = new gsw_ctx();
  ctx->device = device;
  DeviceGuard g(device);
  ctx->stream = (cudaStream_t)cuda_stream;  // NULL: the default stream
  *out = ctx;
  return GSW_OK;
}

void gsw_destroy(gsw_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->batches) batch_free(ctx, kv.second);
  ctx->batches.clear();
  for (auto& kv : ctx->models) free_model(ctx, kv.second);
  ctx->models.clear();
  misfit_free(ctx->misfit, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

const char* gsw_last_error(const gsw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

gsw_status gsw_set_allocator(gsw_ctx* ctx, void* (*alloc)(size_t, void*, void*),
                             void (*free_)(void*, void*, void*), void* user) {
  if (!ctx) return GSW_E_INVALID;
  if (!ctx->models.empty()) return fail(ctx, GSW_E_STATE, "set the allocator before uploading models");
  if ((alloc == nullptr) != (free_ == nullptr))
    return fail(ctx, GSW_E_INVALID, "alloc and free must both be set or both be NULL");
  if (ctx->misfit.buf) {
    misfit_free(ctx->misfit, ctx->stream);  // scratch of the previous allocator
    cudaStreamSynchronize(ctx->stream);
  }
  ctx->alloc = alloc;
  ctx->free_ = free_;
  ctx->user = user;
  ctx->misfit.alloc = alloc;
  ctx->misfit.free_ = free_;
  ctx->misfit.user = user;
  return GSW_OK;
}

gsw_status gsw_model_upload(gsw_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_elem,
                            const int32_t* conn, const int32_t* elem_mat, int32_t n_mat,
                            const double* mat, int64_t n_faces, const int32_t* faces,
                            const int32_t* face_elem, const int32_t* face_tag, const double* period,
                            int32_t n_rec, const double* rec_xy, int32_t* model_id) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  if (!model_id) return fail(ctx, GSW_E_INVALID, "model_id is NULL");
  if (n_nodes <= 0 || n_elem <= 0 || n_faces < 0 || n_rec < 0)
    return fail(ctx, GSW_E_INVALID, "sizes must be positive (n_nodes %lld, n_elem %lld)",
                (long long)n_nodes, (long long)n_elem);
  if (n_nodes > (int64_t)INT32_MAX || n_elem > (int64_t)INT32_MAX / 10)
    return fail(ctx, GSW_E_INVALID, "mesh too large for 32-bit node indices");
  if (!xyz || !conn || !elem_mat || !mat || (n_faces > 0 && (!faces || !face_elem || !face_tag)) ||
      (n_rec > 0 && !rec_xy))
    return fail(ctx, GSW_E_INVALID, "NULL array argument");
  if (n_mat <= 0 || n_mat > kMaxMat) return fail(ctx, GSW_E_INVALID, "n_mat must be 1..%d", kMaxMat);
  if (!finite_all(xyz, 3 * (size_t)n_nodes)) return fail(ctx, GSW_E_INVALID, "non-finite node coordinate");
  for (int i = 0; i < n_mat; ++i) {
    const double Vp = mat[4 * i], Vs = mat[4 * i + 1], rho = mat[4 * i + 2], h = mat[4 * i + 3];
    if (!(Vs > 0.0 && Vp > Vs && rho > 0.0 && h >= 0.0 && isfinite(Vp) && isfinite(rho) && isfinite(h)))
      return fail(ctx, GSW_E_INVALID, "material %d must satisfy Vp > Vs > 0, rho > 0, h >= 0", i);
  }
  for (int64_t i = 0; i < 10 * n_elem; ++i)
    if (conn[i] < 0 || conn[i] >= n_nodes)
      return fail(ctx, GSW_E_INVALID, "element %lld references node %d outside [0, %lld)",
                  (long long)(i / 10), conn[i], (long long)n_nodes);
  for (int64_t i = 0; i < n_elem; ++i)
    if (elem_mat[i] < 0 || elem_mat[i] >= n_mat)
      return fail(ctx, GSW_E_INVALID, "element %lld has material %d outside [0, %d)", (long long)i,
                  elem_mat[i], n_mat);
  for (int64_t i = 0; i < n_faces; ++i) {
    if (face_elem[i] < 0 || face_elem[i] >= n_elem)
      return fail(ctx, GSW_E_INVALID, "face %lld owner element out of range", (long long)i);
    if (face_tag[i] < 0 || face_tag[i] > 2)
      return fail(ctx, GSW_E_INVALID, "face %lld tag %d not in {0, 1, 2}", (long long)i, face_tag[i]);
    for (int k = 0; k < 6; ++k)
      if (faces[6 * i + k] < 0 || faces[6 * i + k] >= n_nodes)
        return fail(ctx, GSW_E_INVALID, "face %lld references a node out of range", (long long)i);
  }
  if (n_rec > 0 && !finite_all(rec_xy, 2 * (size_t)n_rec))
    return fail(ctx, GSW_E_INVALID, "non-finite receiver position");
  double px = period ? period[0] : 0.0, py = period ? period[1] : 0.0;
  if (!(px >= 0.0 && py >= 0.0)) return fail(ctx, GSW_E_INVALID, "periods must be >= 0");

  Model* m = new Model();
  m->N = n_nodes;
  m->E = n_elem;
  m->F = n_faces;
  m->n_mat = n_mat;
  m->n_rec = n_rec;
  m->period[0] = px;
  m->period[1] = py;
  m->raw_mat.assign(mat, mat + 4 * n_mat);
  cudaStream_t s = ctx->stream;
  gsw_status st = GSW_OK;
  auto bail = [&](gsw_status code) {
    cudaStreamSynchronize(s);
    free_model(ctx, m);
    return code;
  };
#define TRYM(expr)                  \
  do {                              \
    st = (expr);                    \
    if (st != GSW_OK) return bail(st); \
  } while (0)
#define CKM(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bail(fail(ctx, GSW_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));       \
  } while (0)
  TRYM(alloc_into(ctx, m, &m->xyz, 3 * (size_t)n_nodes));
  TRYM(alloc_into(ctx, m, &m->conn, 10 * (size_t)n_elem));
  TRYM(alloc_into(ctx, m, &m->geo, 10 * (size_t)n_elem));
  TRYM(alloc_into(ctx, m, &m->emat, (size_t)n_elem));
  TRYM(alloc_into(ctx, m, &m->raw_mat_dev, 4 * (size_t)n_mat));
  TRYM(alloc_into(ctx, m, &m->mat, (size_t)kMaxMat));
  TRYM(alloc_into(ctx, m, &m->fnode, 6 * (size_t)(n_faces > 0 ? n_faces : 1)));
  TRYM(alloc_into(ctx, m, &m->face_elem, (size_t)(n_faces > 0 ? n_faces : 1)));
  TRYM(alloc_into(ctx, m, &m->face_tag, (size_t)(n_faces > 0 ? n_faces : 1)));
  TRYM(alloc_into(ctx, m, &m->fgeo, 6 * (size_t)(n_faces > 0 ? n_faces : 1)));
  TRYM(alloc_into(ctx, m, &m->rec_xy, 2 * (size_t)(n_rec > 0 ? n_rec : 1)));
  TRYM(alloc_into(ctx, m, &m->rec_face, (size_t)(n_rec > 0 ? n_rec : 1)));
  TRYM(alloc_into(ctx, m, &m->rec_node, 6 * (size_t)(n_rec > 0 ? n_rec : 1)));
  TRYM(alloc_into(ctx, m, &m->rec_w, 6 * (size_t)(n_rec > 0 ? n_rec : 1)));
  TRYM(alloc_into(ctx, m, &m->err, 1));
  std::vector<int32_t> conn_soa = soa(conn, n_elem, 10);
  std::vector<int32_t> face_soa = n_faces > 0 ? soa(faces, n_faces, 6) : std::vector<int32_t>();
  CKM(cudaMemcpyAsync(m->xyz, xyz, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, s));
  CKM(cudaMemcpyAsync(m->conn, conn_soa.data(), sizeof(int32_t) * 10 * n_elem, cudaMemcpyHostToDevice, s));
  CKM(cudaMemcpyAsync(m->emat, elem_mat, sizeof(int32_t) * n_elem, cudaMemcpyHostToDevice, s));
  CKM(cudaMemcpyAsync(m->raw_mat_dev, mat, sizeof(double) * 4 * n_mat, cudaMemcpyHostToDevice, s));
  if (n_faces > 0) {
    CKM(cudaMemcpyAsync(m->fnode, face_soa.data(), sizeof(int32_t) * 6 * n_faces, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(m->face_elem, face_elem, sizeof(int32_t) * n_faces, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(m->face_tag, face_tag, sizeof(int32_t) * n_faces, cudaMemcpyHostToDevice, s));
  }
  if (n_rec > 0)
    CKM(cudaMemcpyAsync(m->rec_xy, rec_xy, sizeof(double) * 2 * n_rec, cudaMemcpyHostToDevice, s));
  CKM(cudaMemsetAsync(m->err, 0, sizeof(int), s));
  launch_material(m->mat, m->raw_mat_dev, n_mat, 0.0, 0.0, 0.0, s);
  ModelView mv = m->view();
  launch_geometry(mv, m->xyz, px, py, m->geo, m->err, s);
  launch_face_geometry(mv, m->xyz, px, py, m->face_elem, m->face_tag, m->fgeo, m->err, s);
  launch_receivers(mv, m->xyz, px, py, m->rec_xy, n_rec, m->rec_face, m->rec_node, m->rec_w, m->err, s);
  CKM(cudaGetLastError());
  st = check_device_err(ctx, m, "model rejected");
  if (st != GSW_OK) return bail(st);
  const int id = ctx->next_id++;
  ctx->models[id] = m;
  *model_id = id;
  return GSW_OK;
#undef TRYM
#undef CKM
}

gsw_status gsw_model_free(gsw_ctx* ctx, int32_t model_id) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (m->batch) return fail(ctx, GSW_E_STATE, "model %d belongs to batch %d; destroy the batch first", model_id, m->batch);
  cudaStreamSynchronize(ctx->stream);
  free_model(ctx, m);
  ctx->models.erase(model_id);
  return GSW_OK;
}

gsw_status gsw_model_info(gsw_ctx* ctx, int32_t model_id, int64_t* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  out[0] = m->N;
  out[1] = m->E;
  out[2] = m->F;
  out[3] = m->n_rec;
  size_t bytes = m->bytes;
  for (int d = 0; d < 3; ++d)
    if (m->inst[d]) bytes += m->inst[d]->bytes;
  out[4] = (int64_t)bytes;
  out[5] = m->lo_ready ? m->lo_variant : -1;
  return GSW_OK;
}

gsw_status gsw_set_time(gsw_ctx* ctx, int32_t model_id, double dt, int32_t n_steps, double f1,
                        double f2) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!(dt > 0.0) || !isfinite(dt) || n_steps <= 0 || !(f1 > 0.0) || !(f2 > f1) || !isfinite(f2))
    return fail(ctx, GSW_E_INVALID, "need dt > 0, n_steps > 0, 0 < f1 < f2");
  if (m->time_set && n_steps != m->n_steps) {
    // re-size the receiver history
    dev_free(ctx, m->wave);
    for (auto& p : m->allocs)
      if (p == m->wave) p = nullptr;
    m->n_steps = n_steps;
    TRY(alloc_into(ctx, m, &m->wave, (size_t)m->n_rec * 3 * (size_t)n_steps));
    m->p_dev = nullptr;  // reallocated at the next batch creation
  }
  m->dt = dt;
  m->f1 = f1;
  m->f2 = f2;
  if (!m->time_set) {
    m->n_steps = n_steps;
    TRY(model_state_alloc(ctx, m));
  }
  m->time_set = true;
  m->input_set = false;
  m->version += 1;
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(m->err, 0, sizeof(int), s));
  launch_material(m->mat, m->raw_mat_dev, m->n_mat, dt, f1, f2, s);
  launch_block_jacobi(m->view(), m->dblk, m->dinv, m->err, s);
  CK(cudaGetLastError());
  TRY(check_device_err(ctx, m, "preconditioner"));
  TRY(model_reset(ctx, m));
  if (m->opts.precision != GSW_PREC_FP64) TRY(build_lo(ctx, m, m->opts.precision == GSW_PREC_FP16));
  return GSW_OK;
}

gsw_status gsw_set_input(gsw_ctx* ctx, int32_t model_id, int32_t dir, const double* p, int32_t n) {
  if (!ctx) return GSW_E_INVALID;
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (dir < 0 || dir > 2) return fail(ctx, GSW_E_INVALID, "dir must be 0, 1 or 2");
  if (!p || n != m->n_steps) return fail(ctx, GSW_E_INVALID, "input length %d != n_steps %d", n, m->n_steps);
  if (!finite_all(p, (size_t)n)) return fail(ctx, GSW_E_INVALID, "non-finite input sample");
  m->input.assign(p, p + n);
  m->dir_input[dir].assign(p, p + n);
  if (m->dir != dir) m->version += 1;
  m->dir = dir;
  m->input_set = true;
  if (m->p_dev) {
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(m->p_dev, p, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return GSW_OK;
}

gsw_status gsw_set_solver(gsw_ctx* ctx, int32_t model_id, const gsw_solver_opts* opts) {
  if (!ctx || !opts) return GSW_E_INVALID;
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!(opts->tol > 0.0) || opts->max_iter <= 0)
    return fail(ctx, GSW_E_INVALID, "need tol > 0 and max_iter > 0");
  if (opts->precision < GSW_PREC_FP64 || opts->precision > GSW_PREC_FP16)
    return fail(ctx, GSW_E_INVALID, "precision mode %d is not one of FP64, FP32, FP16", opts->precision);
  if (opts->precision != GSW_PREC_FP64 && (opts->inner_iters <= 0 || opts->inner_iters > 10000))
    return fail(ctx, GSW_E_INVALID, "inner_iters must be 1..10000");
  if (!(opts->inner_rtol >= 0.0 && opts->inner_rtol < 1.0))
    return fail(ctx, GSW_E_INVALID, "inner_rtol must be in [0, 1)");
  if (opts->inner_variant < -1 || opts->inner_variant >= kLoVariants)
    return fail(ctx, GSW_E_INVALID, "inner_variant must be -1 (autotune) or 0..%d", kLoVariants - 1);
  if (opts->guess_order < 0 || opts->guess_order > kMaxGuessOrder)
    return fail(ctx, GSW_E_INVALID, "guess_order must be 0..%d", kMaxGuessOrder);
  if (opts->outer_op < GSW_OUTER_AUTO || opts->outer_op > GSW_OUTER_DWORD)
    return fail(ctx, GSW_E_INVALID, "outer_op must be 0 (auto), 1 (FP64) or 2 (double-word)");
  if (!(opts->coarse_weight >= 0.0 && opts->coarse_weight <= 4.0))
    return fail(ctx, GSW_E_INVALID, "coarse_weight must be in [0, 4]");
  if (!(opts->coarse_relres >= 0.0 && opts->coarse_relres < 1.0))
    return fail(ctx, GSW_E_INVALID, "coarse_relres must be in [0, 1)");
  if (opts->proj_dim != 0 && (opts->proj_dim < 2 || opts->proj_dim > kMaxProj))
    return fail(ctx, GSW_E_INVALID, "proj_dim must be 0 or 2..%d", kMaxProj);
  if (!(opts->proj_relres >= 0.0 && opts->proj_relres < 1.0))
    return fail(ctx, GSW_E_INVALID, "proj_relres must be in [0, 1)");
  if (opts->proj_relres > 0.0 && (opts->proj_dim == 0 || opts->guess_order == 0))
    return fail(ctx, GSW_E_INVALID, "proj_relres hands the projection guess over to the extrapolation: it needs "
                                    "proj_dim > 0 and guess_order > 0");
  if (opts->proj_dim > 0 && m->learn.enable)
    return fail(ctx, GSW_E_STATE, "the projection guess and the learned guess exclude each other");
  if (opts->proj_dim > 0) {
    DeviceGuard g(ctx->device);
    if (opts->proj_dim != m->opts.proj_dim && m->proj)
      CK(cudaMemsetAsync(m->proj, 0, sizeof(ProjState), ctx->stream));  // the history restarts
    TRY(proj_alloc(ctx, m, opts->proj_dim));
  }
  if (opts->guess_order > 0) {
    DeviceGuard g(ctx->device);
    if (!m->guess_ext) TRY(alloc_into(ctx, m, &m->guess_ext, 2));
    if (!m->guess_ring || m->guess_ring_k < opts->guess_order) {
      TRY(alloc_into(ctx, m, &m->guess_ring, (size_t)(opts->guess_order + 1) * 3 * (size_t)m->N));
      m->guess_ring_k = opts->guess_order;
    }
    if (opts->guess_order != m->opts.guess_order || m->opts.guess_order == 0)
      CK(cudaMemsetAsync(m->guess_ext, 0, 2 * sizeof(int), ctx->stream));  // the history restarts
  }
  m->opts = *opts;
  m->version += 1;
  if (m->opts.precision != GSW_PREC_FP64 && m->time_set) {
    DeviceGuard g(ctx->device);
    TRY(build_lo(ctx, m, m->opts.precision == GSW_PREC_FP16));
  }
  return GSW_OK;
}

gsw_status gsw_reset(gsw_ctx* ctx, int32_t model_id) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  return model_reset(ctx, m);
}

gsw_status gsw_step(gsw_ctx* ctx, int32_t model_id, int32_t n) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set || !m->input_set) return fail(ctx, GSW_E_STATE, "set the time and the input first");
  if (m->failed) return fail(ctx, GSW_E_STATE, "model failed at step %lld; reset it", (long long)m->step);
  if (n < 0 || m->step + n > m->n_steps)
    return fail(ctx, GSW_E_INVALID, "cannot step %d from %lld of %d", n, (long long)m->step, m->n_steps);
  for (int i = 0; i < n; ++i) {
    if (m->opts.precision == GSW_PREC_FP64)
      TRY(step_fp64(ctx, m));
    else
      TRY(step_mixed(ctx, m));
  }
  return GSW_OK;
}

static gsw_status batch_make(gsw_ctx* ctx, const std::vector<Model*>& ms, const std::vector<int>& model_ids,
                             const std::vector<int>& dirs, int32_t* batch_id, const std::vector<int>* lanes = nullptr);

gsw_status gsw_run(gsw_ctx* ctx, const int32_t* model_ids, int32_t n_models, int32_t dirs_mask) {
  if (!ctx || (!model_ids && n_models > 0)) return GSW_E_INVALID;
  if (dirs_mask < 0 || dirs_mask > 7) return fail(ctx, GSW_E_INVALID, "dirs_mask must be 0..7");
  DeviceGuard g(ctx->device);
  std::vector<Model*> members;
  std::vector<int> ids, dirs, lanes;
  int max_steps = 0;
  for (int i = 0; i < n_models; ++i) {
    Model* m = find(ctx, model_ids[i]);
    if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_ids[i]);
    for (int j = 0; j < i; ++j)
      if (model_ids[j] == model_ids[i]) return fail(ctx, GSW_E_INVALID, "model %d listed twice", model_ids[i]);
    if (!m->time_set) return fail(ctx, GSW_E_STATE, "model %d: call gsw_set_time first", model_ids[i]);
    if (m->batch) return fail(ctx, GSW_E_STATE, "model %d belongs to batch %d", model_ids[i], m->batch);
    if (dirs_mask == 0) {
      TRY(gsw_reset(ctx, model_ids[i]));
      if (m->learn.enable) {
        TRY(gsw_step(ctx, model_ids[i], m->n_steps));
        continue;
      }
      if (!m->input_set) return fail(ctx, GSW_E_STATE, "model %d: set the input first", model_ids[i]);
      members.push_back(m);
      ids.push_back(model_ids[i]);
      dirs.push_back(-1);
      lanes.push_back(1);
    } else {
      const size_t first = members.size();
      for (int d = 0; d < 3; ++d) {
        if (!(dirs_mask & (1 << d))) continue;
        Model* c = nullptr;
        TRY(get_instance(ctx, m, d, &c));
        TRY(model_reset(ctx, c));
        members.push_back(c);
        ids.push_back(model_ids[i]);
        dirs.push_back(d);
        lanes.push_back(1);
      }
      // the direction analyses share each inner-operator pass (lockstep)
      const int cnt = (int)(members.size() - first);
      if (m->opts.share_dirs && m->opts.precision != GSW_PREC_FP64 && cnt > 1) {
        lanes[first] = cnt;
        for (int k = 1; k < cnt; ++k) lanes[first + k] = 0;
      }
    }
    max_steps = std::max(max_steps, m->n_steps);
  }
  if (members.empty()) return GSW_OK;
  int32_t bid = 0;
  TRY(batch_make(ctx, members, ids, dirs, &bid, &lanes));
  gsw_status st = gsw_batch_step(ctx, bid, max_steps);
  std::string msg = ctx->err;
  gsw_batch_destroy(ctx, bid);
  if (st != GSW_OK) ctx->err = msg;
  return st;
}

// A batch over models or direction instances (the members).
static gsw_status batch_make(gsw_ctx* ctx, const std::vector<Model*>& ms, const std::vector<int>& model_ids,
                             const std::vector<int>& dirs, int32_t* batch_id, const std::vector<int>* lanes) {
  DeviceGuard g(ctx->device);
  const int n_models = (int)ms.size();
  for (int i = 0; i < n_models; ++i) {
    Model* m = ms[i];
    if (!m->time_set || !m->input_set) return fail(ctx, GSW_E_STATE, "model %d: set the time and the input first", model_ids[i]);
    if (m->opts.precision != GSW_PREC_FP64 && !m->lo_ready)
      return fail(ctx, GSW_E_STATE, "model %d: the inner solve of the mixed mode is not set up", model_ids[i]);
    if (m->batch) return fail(ctx, GSW_E_STATE, "model %d already belongs to batch %d", model_ids[i], m->batch);
    if (m->learn.enable)
      return fail(ctx, GSW_E_STATE, "model %d: the learned guess runs with host-driven stepping only", model_ids[i]);
  }
  Batch* b = new Batch();
  auto bail = [&](const char* what, cudaError_t e) {
    batch_free(ctx, b);
    return fail(ctx, GSW_E_CUDA, "batch creation: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
  if ((e = cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
  if ((e = cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
  b->ss_dev = (StepState*)dev_alloc(ctx, nullptr, sizeof(StepState) * n_models);
  if (!b->ss_dev) {
    batch_free(ctx, b);
    return fail(ctx, GSW_E_NOMEM, "device allocation failed (batch step states)");
  }
  if ((e = cudaMallocHost(&b->ss_host, sizeof(StepState) * n_models)) != cudaSuccess) return bail("state", e);
  for (int i = 0; i < n_models; ++i) {
    Model* m = ms[i];
    cudaStream_t s;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
    b->streams.push_back(s);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
    b->joins.push_back(ev);
    if (!m->p_dev) {
      m->p_dev = (double*)dev_alloc(ctx, m, sizeof(double) * m->n_steps);
      if (!m->p_dev) {
        batch_free(ctx, b);
        return fail(ctx, GSW_E_NOMEM, "device allocation failed (input samples)");
      }
    }
    if ((e = cudaMemcpyAsync(m->p_dev, m->input.data(), sizeof(double) * m->n_steps, cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
      return bail("input copy", e);
    b->members.push_back(m);
    b->ids.push_back(model_ids[i]);
    b->dirs.push_back(dirs[i]);
    b->lane.push_back(lanes ? (*lanes)[i] : 1);
    b->versions.push_back(-1);
  }
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail("synchronise", e);
  const int id = ctx->next_batch++;
  for (int i = 0; i < n_models; ++i) ms[i]->batch = id;
  ctx->batches[id] = b;
  *batch_id = id;
  return GSW_OK;
}

gsw_status gsw_batch_create(gsw_ctx* ctx, const int32_t* model_ids, int32_t n_models, int32_t* batch_id) {
  if (!ctx || !model_ids || n_models <= 0 || !batch_id) return GSW_E_INVALID;
  std::vector<Model*> ms;
  std::vector<int> ids, dirs;
  for (int i = 0; i < n_models; ++i) {
    Model* m = find(ctx, model_ids[i]);
    if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_ids[i]);
    for (int j = 0; j < i; ++j)
      if (model_ids[j] == model_ids[i]) return fail(ctx, GSW_E_INVALID, "model %d listed twice", model_ids[i]);
    ms.push_back(m);
    ids.push_back(model_ids[i]);
    dirs.push_back(-1);
  }
  return batch_make(ctx, ms, ids, dirs, batch_id);
}

gsw_status gsw_batch_step(gsw_ctx* ctx, int32_t batch_id, int32_t n_steps) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  auto it = ctx->batches.find(batch_id);
  if (it == ctx->batches.end()) return fail(ctx, GSW_E_INVALID, "unknown batch %d", batch_id);
  Batch* b = it->second;
  if (n_steps < 0) return fail(ctx, GSW_E_INVALID, "n_steps must be >= 0");
  const int nm = (int)b->ids.size();
  int outer = 0;
  bool stale = (b->exec == nullptr);
  bool adaptive = false;
  int outer_loop = 0;  // budget of the device-side loop (adaptive members: 32)
  int remaining = 0;
  int fp64_loop = 0;  // budget of the device-side loop of FP64 members (PCG iterations)
  for (int i = 0; i < nm; ++i) {
    Model* m = b->members[i];
    if (m->opts.precision == GSW_PREC_FP64) {
      fp64_loop = std::max(fp64_loop, m->opts.batch_outer > 0 ? m->opts.batch_outer : kFp64LoopCap);
    } else {
      const int o = m->opts.batch_outer > 0 ? m->opts.batch_outer : b->adapt_outer;
      if (m->opts.batch_outer <= 0) adaptive = true;
      if (o > outer) outer = o;
      outer_loop = std::max(outer_loop, m->opts.batch_outer > 0 ? m->opts.batch_outer : 32);
    }
    if (b->versions[i] != m->version) stale = true;
    StepState& h = b->ss_host[i];
    memset(&h, 0, sizeof(StepState));
    h.step = (int)m->step;
    h.n_steps = m->n_steps;
    h.stop_at = (int)std::min<int64_t>((int64_t)m->n_steps, m->step + n_steps);
    h.failed = m->failed ? GSW_E_STATE : 0;
    h.tol = m->opts.tol;
    h.max_iter = m->opts.max_iter;
    h.inner_iters = m->opts.precision == GSW_PREC_FP64 ? 0 : (m->opts.inner_iters > 0 ? m->opts.inner_iters : 1);
    if (!m->failed) remaining = std::max(remaining, h.stop_at - h.step);
  }
  if ((b->use_while ? outer_loop : outer) != b->outer || fp64_loop != b->fp64_loop) stale = true;
  CK(cudaEventRecord(b->fork, ctx->stream));
  CK(cudaStreamWaitEvent(b->origin, b->fork, 0));
  CK(cudaMemcpyAsync(b->ss_dev, b->ss_host, sizeof(StepState) * nm, cudaMemcpyHostToDevice, b->origin));
  // (re)capture the step graph: the outer iterations after the first run in a
  // device-side WHILE loop per member (budget outer_loop), or, if that cannot
  // be built, unrolled (budget outer)
  auto capture = [&]() -> gsw_status {
    for (;;) {
      const bool wl = b->use_while;
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      CK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
      CK(cudaEventRecord(b->fork, b->origin));
      bool ok = true;
      b->launches.assign(nm, StepLaunches());
      for (int i = 0; i < nm && ok; ++i) {
        if (b->lane[i] == 0) continue;  // advanced by the lane that holds it
        Model* m = b->members[i];
        const bool fp64 = m->opts.precision == GSW_PREC_FP64;
        ok = cudaStreamWaitEvent(b->streams[i], b->fork, 0) == cudaSuccess &&
             (b->lane[i] > 1 ? issue_device_step_group(&b->members[i], b->lane[i], b->streams[i], b->ss_dev + i,
                                                       wl ? outer_loop : outer, wl ? b->body_stream : nullptr,
                                                       &b->launches[i])
              : fp64 ? issue_device_step_fp64(m, b->streams[i], b->ss_dev + i, wl ? fp64_loop : outer,
                                              wl ? b->body_stream : nullptr, &b->launches[i])
                     : issue_device_step(m, b->streams[i], b->ss_dev + i, wl ? outer_loop : outer,
                                         wl ? b->body_stream : nullptr, &b->launches[i])) &&
             cudaEventRecord(b->joins[i], b->streams[i]) == cudaSuccess &&
             cudaStreamWaitEvent(b->origin, b->joins[i], 0) == cudaSuccess;
      }
      cudaError_t ce = cudaStreamEndCapture(b->origin, &b->graph);
      if (ok && ce == cudaSuccess && cudaGraphInstantiate(&b->exec, b->graph, 0) == cudaSuccess) break;
      cudaGetLastError();
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      if (!wl) return fail(ctx, GSW_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
      b->use_while = false;  // retry with the unrolled loop
    }
    int64_t launches = 0;
    for (const StepLaunches& l : b->launches) launches += l.fixed + l.body;
    b->launches_per_step = launches;
    b->outer = b->use_while ? outer_loop : outer;
    b->fp64_loop = fp64_loop;
    for (int i = 0; i < nm; ++i) b->versions[i] = b->members[i]->version;
    return GSW_OK;
  };
  if (stale && remaining > 0) {
    NvtxRange nvc("gsw batch graph capture");
    TRY(capture());
  }
  gsw_status st = GSW_OK;
  const int chunk = 8;
  NvtxRange nv("gsw batch steps");
  while (remaining > 0) {
    const int launch_n = std::min(remaining, chunk);
    for (int s = 0; s < launch_n; ++s) CK(cudaGraphLaunch(b->exec, b->origin));
    CK(cudaMemcpyAsync(b->ss_host, b->ss_dev, sizeof(StepState) * nm, cudaMemcpyDeviceToHost, b->origin));
    CK(cudaStreamSynchronize(b->origin));
    remaining = 0;
    bool rewrite = false;
    int need = 0;  // most outer iterations a step of this chunk needed
    for (int i = 0; i < nm; ++i) {
      Model* m = b->members[i];
      StepState& h = b->ss_host[i];
      const int advanced = h.step - (int)m->step;
      m->step = h.step;
      m->stats.steps_done += advanced;
      m->stats.cg_iters_total += h.iters_total;
      m->stats.inner_iters_total += h.inner_total;
      {
        // launches issued for this member: the fixed part of every graph
        // launch, plus one loop body per outer iteration after a step's first
        // (an FP64 member runs every PCG iteration in the loop)
        const StepLaunches& l = b->launches[i];
        const bool fp64 = m->opts.precision == GSW_PREC_FP64;
        const int64_t extra = fp64 ? h.iters_total : std::max<int64_t>(0, h.iters_total - advanced);
        m->stats.kernel_launches += (int64_t)launch_n * l.fixed + (b->use_while ? extra * l.body : 0);
      }
      if (advanced > 0) {
        m->stats.cg_iters_last = h.iters_last;
        m->stats.relres_last = h.relres_last;
      }
      if (h.iters_max > m->stats.cg_iters_max) m->stats.cg_iters_max = h.iters_max;
      if (m->opts.precision != GSW_PREC_FP64) need = std::max(need, h.iters_max);
      h.iters_total = h.inner_total = h.iters_max = 0;
      rewrite = true;
      if (h.failed && !m->failed) {
        m->failed = true;
        if (st == GSW_OK) {
          st = (h.failed == GSW_E_NOCONV || h.failed == GSW_E_NAN || h.failed == GSW_E_TIMEOUT) ? (gsw_status)h.failed
                                                                                                 : GSW_E_STATE;
          fail(ctx, st, "model %d%s failed at step %d (%s)", b->ids[i],
               b->dirs[i] == 0 ? " (direction x1)" : (b->dirs[i] == 1 ? " (direction x2)" :
                                                      (b->dirs[i] == 2 ? " (direction x3)" : "")),
               h.fail_step, h.failed == GSW_E_NAN ? "non-finite residual"
                            : (h.failed == GSW_E_TIMEOUT ? "a bounded wait of the inner operator ran out"
                                                         : "no convergence"));
        }
      }
      if (h.needs_host && !m->failed) {
        // more outer iterations than the captured budget: finish this step on
        // the host-driven path (same algorithm, iteration cap max_iter)
        CK(cudaEventRecord(b->done_ev, b->origin));
        CK(cudaStreamWaitEvent(ctx->stream, b->done_ev, 0));
        gsw_status hs = m->opts.precision == GSW_PREC_FP64 ? step_fp64(ctx, m) : step_mixed(ctx, m);
        if (hs != GSW_OK) {
          h.failed = hs;
          h.fail_step = h.step;
          if (st == GSW_OK) st = hs;  // message set by step_mixed
        } else {
          h.step = (int)m->step;
          h.needs_host = 0;
          if (m->opts.precision != GSW_PREC_FP64) need = std::max(need, m->stats.cg_iters_last);
        }
        CK(cudaEventRecord(b->fork, ctx->stream));
        CK(cudaStreamWaitEvent(b->origin, b->fork, 0));
      }
      if (!m->failed && !h.failed) remaining = std::max(remaining, h.stop_at - h.step);
    }
    if (rewrite) CK(cudaMemcpyAsync(b->ss_dev, b->ss_host, sizeof(StepState) * nm, cudaMemcpyHostToDevice, b->origin));
    if (adaptive && !b->use_while && need > 0 && st == GSW_OK) {
      // the captured budget follows the steps: one more than the most outer
      // iterations a step of the chunk needed (2..16); raised at once (steps
      // beyond it were finished by the host), lowered after two chunks in a
      // row that needed less
      const int target = std::min(16, std::max(2, need + 1));
      int next = b->adapt_outer;
      if (target > b->adapt_outer) {
        next = target;
        b->lower_streak = b->lower_max = 0;
      } else if (target < b->adapt_outer) {
        b->lower_max = std::max(b->lower_max, target);
        if (++b->lower_streak >= 2) {
          next = b->lower_max;
          b->lower_streak = b->lower_max = 0;
        }
      } else {
        b->lower_streak = b->lower_max = 0;
      }
      if (next != b->adapt_outer) {
        b->adapt_outer = next;
        outer = 0;
        for (int i = 0; i < nm; ++i) {
          Model* m = b->members[i];
          outer = std::max(outer, m->opts.batch_outer > 0 ? m->opts.batch_outer : b->adapt_outer);
        }
        if (outer != b->outer && remaining > 0) TRY(capture());
      }
    }
  }
  CK(cudaEventRecord(b->done_ev, b->origin));
  CK(cudaStreamWaitEvent(ctx->stream, b->done_ev, 0));
  CK(cudaStreamSynchronize(b->origin));
  return st;
}

gsw_status gsw_batch_destroy(gsw_ctx* ctx, int32_t batch_id) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  auto it = ctx->batches.find(batch_id);
  if (it == ctx->batches.end()) return fail(ctx, GSW_E_INVALID, "unknown batch %d", batch_id);
  cudaStreamSynchronize(it->second->origin);
  for (Model* m : it->second->members) m->batch = 0;
  batch_free(ctx, it->second);
  ctx->batches.erase(it);
  return GSW_OK;
}

gsw_status gsw_batch_launches(gsw_ctx* ctx, int32_t batch_id, int64_t* per_step) {
  if (!ctx || !per_step) return GSW_E_INVALID;
  auto it = ctx->batches.find(batch_id);
  if (it == ctx->batches.end()) return fail(ctx, GSW_E_INVALID, "unknown batch %d", batch_id);
  *per_step = it->second->launches_per_step;
  return GSW_OK;
}

// The analysis selected by dir: -1 the model's own (the direction of its last
// gsw_set_input), 0..2 the instance of that input direction run by gsw_run.
gsw_status analysis_of(gsw_ctx* ctx, int32_t model_id, int32_t dir, Model** out, bool need_time = true) {
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (dir < -1 || dir > 2) return fail(ctx, GSW_E_INVALID, "dir must be -1, 0, 1 or 2");
  if (need_time && !m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (dir >= 0) {
    m = m->inst[dir];
    if (!m)
      return fail(ctx, GSW_E_STATE, "direction %d of model %d has not been run (gsw_run with its bit in dirs_mask)",
                  dir, model_id);
  }
  *out = m;
  return GSW_OK;
}

gsw_status gsw_read_waveforms(gsw_ctx* ctx, int32_t model_id, int32_t dir, double* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = nullptr;
  TRY(analysis_of(ctx, model_id, dir, &m));
  CK(cudaMemcpyAsync(out, m->wave, sizeof(double) * (size_t)m->n_rec * 3 * m->n_steps,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSW_OK;
}

gsw_status gsw_read_waveform_steps(gsw_ctx* ctx, int32_t model_id, int32_t step0, int32_t count,
                                   double* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (step0 < 0 || count <= 0 || step0 + count > m->n_steps)
    return fail(ctx, GSW_E_INVALID, "steps [%d, %d) outside [0, %d)", step0, step0 + count, m->n_steps);
  if (m->n_rec == 0) return GSW_OK;
  CK(cudaMemcpy2DAsync(out, sizeof(double) * count, m->wave + step0, sizeof(double) * m->n_steps,
                       sizeof(double) * count, 3 * (size_t)m->n_rec, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSW_OK;
}

gsw_status gsw_timing(gsw_ctx* ctx, int32_t model_id, int32_t enable, double* ms, int64_t* launches) {
  if (!ctx) return GSW_E_INVALID;
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (enable == 1) {
    m->timing = true;
    m->ebe_ms = m->lo_ms = 0.0;
    m->ebe_count = m->lo_count = 0;
    m->iters_mark = 0;
    if (m->lo_ready) {
      DeviceGuard g(ctx->device);
      CK(cudaMemcpyAsync(&m->iters_mark, &m->isc->iters, sizeof(m->iters_mark), cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
  } else if (enable == 0) {
    m->timing = false;
  }
  if (ms) {
    ms[0] = m->ebe_ms;
    ms[1] = m->lo_ms;
  }
  if (launches) {
    launches[0] = m->ebe_count;
    launches[1] = m->lo_count;
  }
  return GSW_OK;
}

gsw_status gsw_stats_get(gsw_ctx* ctx, int32_t model_id, int32_t dir, gsw_stats* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  Model* m = nullptr;
  TRY(analysis_of(ctx, model_id, dir, &m, false));
  *out = m->stats;
  if (m->lo_ready && m->opts.precision != GSW_PREC_FP64) {
    // inner iterations actually executed since the last reset (device counter)
    DeviceGuard g(ctx->device);
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, &m->isc->iters, sizeof(n), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->inner_iters_total = (int64_t)(n - m->iters_reset);
  }
  return GSW_OK;
}

gsw_status gsw_get_state(gsw_ctx* ctx, int32_t model_id, double* u, double* v, double* a, int64_t* step) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  const size_t bytes = sizeof(double) * 3 * (size_t)m->N;
  if (u) CK(cudaMemcpyAsync(u, m->u, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (v) CK(cudaMemcpyAsync(v, m->v, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (a) CK(cudaMemcpyAsync(a, m->a, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (step) *step = m->step;
  return GSW_OK;
}

gsw_status gsw_set_state(gsw_ctx* ctx, int32_t model_id, const double* u, const double* v,
                         const double* a, int64_t step) {
  if (!ctx || !u || !v || !a) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (step < 0 || step > m->n_steps) return fail(ctx, GSW_E_INVALID, "step out of range");
  const size_t n3 = 3 * (size_t)m->N;
  if (!finite_all(u, n3) || !finite_all(v, n3) || !finite_all(a, n3))
    return fail(ctx, GSW_E_INVALID, "non-finite state");
  const size_t bytes = sizeof(double) * n3;
  CK(cudaMemcpyAsync(m->u, u, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(m->v, v, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(m->a, a, bytes, cudaMemcpyHostToDevice, ctx->stream));
  if (m->guess_ext) CK(cudaMemsetAsync(m->guess_ext, 0, 2 * sizeof(int), ctx->stream));  // no increment history
  if (m->proj) CK(cudaMemsetAsync(m->proj, 0, sizeof(ProjState), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  m->step = step;
  m->failed = false;
  return GSW_OK;
}

// Checkpoint layout: a fixed header, then u, v, a [3N] doubles, the receiver
// history [n_rec][3][n_steps] doubles, the increment ring [(k+1)][3N] doubles
// (guess order k > 0), and with the learned guess its parameters, Adam
// moments ([5443] floats each) and increment history ([4][3N] floats).
namespace {
constexpr uint64_t kCkptMagic = 0x31544b5057534737ULL;  // "7GSWPKT1"
struct CkptHeader {
  uint64_t magic;
  int64_t n_nodes, n_steps, n_rec, step;
  int32_t dir, guess_order, ring_count, ring_head;
  int32_t has_mlp, hist_head, hist_count, adam_t;
  int32_t mlp_off, failed;
  int32_t proj_dim, pad_;
  int64_t std_r0_n, mlp_r0_n, applied, inner_done;
  double std_r0[5], mlp_r0[5];
  gsw_stats stats;
  MlpScalars ms;
  gsw_learn_opts learn;
  uint64_t bytes;
};
size_t ckpt_bytes(const Model* m, bool mlp) {
  const size_t n3 = 3 * (size_t)m->N;
  size_t b = sizeof(CkptHeader) + 3 * n3 * sizeof(double) + (size_t)m->n_rec * 3 * m->n_steps * sizeof(double);
  if (m->opts.guess_order > 0) b += (size_t)(m->opts.guess_order + 1) * n3 * sizeof(double);
  if (m->opts.proj_dim > 0) b += 2 * (size_t)m->opts.proj_dim * n3 * sizeof(double) + sizeof(ProjState);
  if (mlp) b += 3 * (size_t)kMlpParams * sizeof(float) + 4 * n3 * sizeof(double);
  return b;
}
}  // namespace

gsw_status gsw_checkpoint(gsw_ctx* ctx, int32_t model_id, void* buf, size_t* bytes) {
  if (!ctx || !bytes) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  const bool mlp = m->mlp_ready && m->learn.enable;
  const size_t need = ckpt_bytes(m, mlp);
  if (!buf) {
    *bytes = need;
    return GSW_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return fail(ctx, GSW_E_INVALID, "checkpoint buffer of %zu bytes is smaller than %zu", *bytes, need);
  }
  cudaStream_t s = ctx->stream;
  CkptHeader h = {};
  h.magic = kCkptMagic;
  h.n_nodes = m->N;
  h.n_steps = m->n_steps;
  h.n_rec = m->n_rec;
  h.step = m->step;
  h.dir = m->dir;
  h.guess_order = m->opts.guess_order;
  h.proj_dim = m->opts.proj_dim;
  h.has_mlp = mlp ? 1 : 0;
  h.hist_head = m->hist_head;
  h.hist_count = m->hist_count;
  h.adam_t = m->adam_t;
  h.mlp_off = m->mlp_off ? 1 : 0;
  h.failed = m->failed ? 1 : 0;
  h.std_r0_n = m->std_r0_n;
  h.mlp_r0_n = m->mlp_r0_n;
  h.applied = m->applied;
  for (int k = 0; k < 5; ++k) {
    h.std_r0[k] = m->std_r0_recent[k];
    h.mlp_r0[k] = m->mlp_r0_recent[k];
  }
  TRY(gsw_stats_get(ctx, model_id, -1, &h.stats));
  h.bytes = need;
  if (m->guess_ext) {
    int ext[2] = {0, 0};
    CK(cudaMemcpyAsync(ext, m->guess_ext, sizeof(ext), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h.ring_count = ext[0];
    h.ring_head = ext[1];
  }
  if (mlp) {
    h.learn = m->learn;
    CK(cudaMemcpyAsync(&h.ms, m->ms, sizeof(MlpScalars), cudaMemcpyDeviceToHost, s));
  }
  char* p = (char*)buf + sizeof(CkptHeader);
  const size_t n3 = 3 * (size_t)m->N;
  auto d2h = [&](const void* src, size_t nb) {
    cudaError_t e = cudaMemcpyAsync(p, src, nb, cudaMemcpyDeviceToHost, s);
    p += nb;
    return e;
  };
  CK(d2h(m->u, n3 * sizeof(double)));
  CK(d2h(m->v, n3 * sizeof(double)));
  CK(d2h(m->a, n3 * sizeof(double)));
  CK(d2h(m->wave, (size_t)m->n_rec * 3 * m->n_steps * sizeof(double)));
  if (m->opts.guess_order > 0) CK(d2h(m->guess_ring, (size_t)(m->opts.guess_order + 1) * n3 * sizeof(double)));
  if (m->opts.proj_dim > 0) {
    CK(d2h(m->proj_W, (size_t)m->opts.proj_dim * n3 * sizeof(double)));
    CK(d2h(m->proj_Z, (size_t)m->opts.proj_dim * n3 * sizeof(double)));
    CK(d2h(m->proj, sizeof(ProjState)));
  }
  if (mlp) {
    CK(d2h(m->theta, kMlpParams * sizeof(float)));
    CK(d2h(m->adam_m, kMlpParams * sizeof(float)));
    CK(d2h(m->adam_v, kMlpParams * sizeof(float)));
    CK(d2h(m->hist, 4 * n3 * sizeof(double)));
  }
  CK(cudaStreamSynchronize(s));
  memcpy(buf, &h, sizeof(h));
  *bytes = need;
  return GSW_OK;
}

gsw_status gsw_restore(gsw_ctx* ctx, int32_t model_id, const void* buf, size_t bytes) {
  if (!ctx || !buf) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (m->batch) return fail(ctx, GSW_E_STATE, "model %d belongs to a batch", model_id);
  CkptHeader h;
  if (bytes < sizeof(h)) return fail(ctx, GSW_E_INVALID, "checkpoint too short");
  memcpy(&h, buf, sizeof(h));
  if (h.magic != kCkptMagic) return fail(ctx, GSW_E_INVALID, "not a checkpoint of this library");
  if (h.n_nodes != m->N || h.n_steps != m->n_steps || h.n_rec != m->n_rec)
    return fail(ctx, GSW_E_INVALID, "checkpoint of a different model or time set-up");
  if (h.dir != m->dir)
    return fail(ctx, GSW_E_INVALID, "checkpoint of input direction %d, model set to direction %d", h.dir, m->dir);
  if (h.guess_order != m->opts.guess_order || h.proj_dim != m->opts.proj_dim)
    return fail(ctx, GSW_E_INVALID, "checkpoint taken with guess_order %d / proj_dim %d, model set to %d / %d",
                h.guess_order, h.proj_dim, m->opts.guess_order, m->opts.proj_dim);
  if (h.has_mlp && !(m->learn.enable && m->mlp_ready))
    return fail(ctx, GSW_E_STATE, "checkpoint holds a learned guess: enable learning on the model first");
  if (h.step < 0 || h.step > m->n_steps || h.bytes != bytes || bytes != ckpt_bytes(m, h.has_mlp != 0))
    return fail(ctx, GSW_E_INVALID, "checkpoint size or step inconsistent");
  cudaStream_t s = ctx->stream;
  const char* p = (const char*)buf + sizeof(CkptHeader);
  const size_t n3 = 3 * (size_t)m->N;
  if (!finite_all((const double*)p, 3 * n3)) return fail(ctx, GSW_E_INVALID, "non-finite state in checkpoint");
  auto h2d = [&](void* dst, size_t nb) {
    cudaError_t e = cudaMemcpyAsync(dst, p, nb, cudaMemcpyHostToDevice, s);
    p += nb;
    return e;
  };
  CK(h2d(m->u, n3 * sizeof(double)));
  CK(h2d(m->v, n3 * sizeof(double)));
  CK(h2d(m->a, n3 * sizeof(double)));
  CK(h2d(m->wave, (size_t)m->n_rec * 3 * m->n_steps * sizeof(double)));
  if (m->opts.guess_order > 0) {
    CK(h2d(m->guess_ring, (size_t)(m->opts.guess_order + 1) * n3 * sizeof(double)));
    const int ext[2] = {h.ring_count, h.ring_head};
    CK(cudaMemcpyAsync(m->guess_ext, ext, sizeof(ext), cudaMemcpyHostToDevice, s));
  }
  if (m->opts.proj_dim > 0) {
    CK(h2d(m->proj_W, (size_t)m->opts.proj_dim * n3 * sizeof(double)));
    CK(h2d(m->proj_Z, (size_t)m->opts.proj_dim * n3 * sizeof(double)));
    CK(h2d(m->proj, sizeof(ProjState)));
  }
  if (h.has_mlp) {
    CK(h2d(m->theta, kMlpParams * sizeof(float)));
    CK(h2d(m->adam_m, kMlpParams * sizeof(float)));
    CK(h2d(m->adam_v, kMlpParams * sizeof(float)));
    CK(h2d(m->hist, 4 * n3 * sizeof(double)));
    CK(cudaMemcpyAsync(m->ms, &h.ms, sizeof(MlpScalars), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpParams, s));
    launch_mlp_pack(m->theta, m->packed, s);
    CK(cudaGetLastError());
    m->learn = h.learn;
    m->hist_head = h.hist_head;
    m->hist_count = h.hist_count;
    m->adam_t = h.adam_t;
    m->mlp_off = h.mlp_off != 0;
    m->std_r0_n = h.std_r0_n;
    m->mlp_r0_n = h.mlp_r0_n;
    m->applied = h.applied;
    for (int k = 0; k < 5; ++k) {
      m->std_r0_recent[k] = h.std_r0[k];
      m->mlp_r0_recent[k] = h.mlp_r0[k];
    }
  }
  if (m->lo_ready) {
    // inner iterations since the reset continue from the checkpoint's count
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, &m->isc->iters, sizeof(n), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    m->iters_reset = n - (unsigned long long)h.stats.inner_iters_total;
  }
  CK(cudaStreamSynchronize(s));
  m->stats = h.stats;
  m->step = h.step;
  m->failed = h.failed != 0;
  return GSW_OK;
}

gsw_status gsw_apply(gsw_ctx* ctx, int32_t model_id, int32_t which, const double* x_dev, double* y_dev) {
  if (!ctx || !x_dev || !y_dev) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (which < 0 || which > 6) return fail(ctx, GSW_E_INVALID, "which must be 0..6");
  if (which == 6) {
    if (!m->coarse() || !m->lo_ready)
      return fail(ctx, GSW_E_STATE, "the coarse correction needs a mixed precision mode with coarse_weight > 0");
    double dm = 0.0;
    CK(cudaMemcpyAsync(&dm, &m->isc->dinv_mean, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    launch_to_f32(3 * m->N, x_dev, m->s32, ctx->stream);
    launch_coarse_restrict(m->cview(), m->s32, m->zc, nullptr, nullptr, nullptr, 0, ctx->stream);
    launch_coarse_prolong(m->N, m->c_pair, m->zc, dm / m->opts.coarse_weight, y_dev, ctx->stream);
    CK(cudaGetLastError());
    return GSW_OK;
  }
  if (which == 4) {
    if (m->opts.precision == GSW_PREC_FP64 || !m->lo_ready)
      return fail(ctx, GSW_E_STATE, "the reduced-precision operator needs a mixed precision mode");
    launch_to_lo(m->N, x_dev, m->d_lo, m->lo_half, m->w32, ctx->stream);
    const void* view = m->lo_half ? (const void*)&m->lo_h : (const void*)&m->lo_f;
    launch_ebe_lo(m->lo_half, m->lo_half, view, m->d_lo, m->w32, m->partials, m->isc, ctx->stream, m->lo_variant);
    launch_from_f32(m->N, m->w32, y_dev, ctx->stream);
    CK(cudaGetLastError());
    return GSW_OK;
  }
  CK(cudaMemsetAsync(y_dev, 0, sizeof(double) * 3 * (size_t)m->N, ctx->stream));
  if (which == 5) {
    launch_ebe_dw(kModeA, 0, m->view(), x_dev, nullptr, nullptr, y_dev, 0.0, 0, nullptr, nullptr, ctx->stream);
    CK(cudaGetLastError());
    return GSW_OK;
  }
  const int mode = which == 0 ? kModeA : which == 1 ? kModeK : which == 2 ? kModeM : kModeC;
  launch_ebe(mode, m->view(), x_dev, nullptr, nullptr, y_dev, 0.0, 0, nullptr, nullptr, ctx->stream);
  CK(cudaGetLastError());
  return GSW_OK;
}

gsw_status gsw_read_preconditioner(gsw_ctx* ctx, int32_t model_id, double* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  CK(cudaMemcpyAsync(out, m->dinv, sizeof(double) * 6 * (size_t)m->N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSW_OK;
}

gsw_status gsw_wait_probe(gsw_ctx* ctx, int64_t limit) {
  if (!ctx) return GSW_E_INVALID;
  if (limit < 1 || limit > (int64_t)1 << 22) return fail(ctx, GSW_E_INVALID, "limit must be 1 .. 2^22");
  DeviceGuard g(ctx->device);
  unsigned* out = (unsigned*)dev_alloc(ctx, nullptr, 2 * sizeof(unsigned));
  if (!out) return fail(ctx, GSW_E_NOMEM, "device allocation failed (wait probe)");
  unsigned h[2] = {0u, 0u};
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    launch_wait_probe((long long)limit, out, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(ctx, out);
  if (e != cudaSuccess) return fail(ctx, GSW_E_CUDA, "wait probe: %s", cudaGetErrorString(e));
  if (h[0] == 1u) return fail(ctx, GSW_E_TIMEOUT, "bounded wait ran out after %lld attempts (expected)",
                              (long long)limit);
  return GSW_OK;
}

gsw_status gsw_read_receivers(gsw_ctx* ctx, int32_t model_id, int32_t* nodes, double* weights) {
  if (!ctx || !nodes || !weights) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (m->n_rec == 0) return GSW_OK;
  CK(cudaMemcpyAsync(nodes, m->rec_node, sizeof(int32_t) * 6 * m->n_rec, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(weights, m->rec_w, sizeof(double) * 6 * m->n_rec, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSW_OK;
}

gsw_status gsw_misfit(gsw_ctx* ctx, int32_t model_id, const double* obs, int32_t stride, int32_t n_shifts,
                      double tau, double* err, double* c_out) {
  if (!ctx || !obs || !err) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (stride <= 0 || n_shifts <= 0 || !(tau >= 0.0))
    return fail(ctx, GSW_E_INVALID, "need stride, n_shifts > 0 and tau >= 0");
  if (3 * n_shifts > kMisfitMaxUnknowns)
    return fail(ctx, GSW_E_INVALID, "3 * n_shifts must be <= %d", kMisfitMaxUnknowns);
  if (m->n_rec <= 0) return fail(ctx, GSW_E_STATE, "model %d has no receivers", model_id);
  const double* waves[3];
  for (int d = 0; d < 3; ++d) {
    Model* c = m->inst[d];
    if (!c || c->failed || c->step != c->n_steps || m->inst_version[d] != m->version || c->input != m->dir_input[d])
      return fail(ctx, GSW_E_STATE, "model %d: run all three input directions to the end first (gsw_run with "
                  "dirs_mask 7)", model_id);
    waves[d] = c->wave;
  }
  if (!finite_all(obs, (size_t)m->n_rec * 3 * m->n_steps))
    return fail(ctx, GSW_E_INVALID, "non-finite observation");
  char msg[256] = {0};
  cudaError_t ce = cudaSuccess;
  int rc = misfit_run_waves(ctx->misfit, ctx->stream, m->n_rec, m->n_steps, m->n_steps, waves, obs, stride,
                            n_shifts, tau, err, c_out, msg, sizeof msg, &ce);
  if (rc == 1) return fail(ctx, GSW_E_CUDA, "misfit: %s (%s)", msg, cudaGetErrorString(ce));
  if (rc == 2) return fail(ctx, GSW_E_NOMEM, "misfit: %s", msg);
  if (rc == 3) return fail(ctx, GSW_E_INVALID, "misfit: %s", msg);
  return GSW_OK;
}

gsw_status gsw_misfit_green(gsw_ctx* ctx, int32_t n_rec, int32_t n_t, const double* G, const double* obs,
                            int32_t stride, int32_t n_shifts, double tau, double* err, double* c_out) {
  if (!ctx || !G || !obs || !err) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  if (n_rec <= 0 || n_t <= 0 || stride <= 0 || n_shifts <= 0 || !(tau >= 0.0))
    return fail(ctx, GSW_E_INVALID, "need n_rec, n_t, stride, n_shifts > 0 and tau >= 0");
  if (3 * n_shifts > kMisfitMaxUnknowns)
    return fail(ctx, GSW_E_INVALID, "3 * n_shifts must be <= %d", kMisfitMaxUnknowns);
  if (!finite_all(G, (size_t)n_rec * 9 * n_t) || !finite_all(obs, (size_t)n_rec * 3 * n_t))
    return fail(ctx, GSW_E_INVALID, "non-finite Green's function or observation");
  char msg[256] = {0};
  cudaError_t ce = cudaSuccess;
  int rc = misfit_run(ctx->misfit, ctx->stream, n_rec, n_t, G, obs, stride, n_shifts, tau, err, c_out,
                      msg, sizeof msg, &ce);
  if (rc == 1) return fail(ctx, GSW_E_CUDA, "misfit: %s (%s)", msg, cudaGetErrorString(ce));
  if (rc == 2) return fail(ctx, GSW_E_NOMEM, "misfit: %s", msg);
  if (rc == 3) return fail(ctx, GSW_E_INVALID, "misfit: %s", msg);
  return GSW_OK;
}

gsw_status gsw_set_learning(gsw_ctx* ctx, int32_t model_id, const gsw_learn_opts* opts) {
  if (!ctx || !opts) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  if (m->batch) return fail(ctx, GSW_E_STATE, "model %d belongs to a batch", model_id);
  if (opts->enable) {
    if (m->opts.precision == GSW_PREC_FP64)
      return fail(ctx, GSW_E_STATE, "the learned guess runs with the mixed-precision solver");
    if (m->opts.proj_dim > 0)
      return fail(ctx, GSW_E_STATE, "the projection guess and the learned guess exclude each other");
    if (opts->train_steps < 5 || opts->batch < 64 || opts->batch > 65536 || opts->iters_per_step < 0 ||
        !(opts->lr > 0.f))
      return fail(ctx, GSW_E_INVALID, "need train_steps >= 5, 64 <= batch <= 65536, iters_per_step >= 0, lr > 0");
  }
  m->learn = *opts;
  if (opts->enable) {
    TRY(mlp_alloc(ctx, m));
    TRY(mlp_init(ctx, m, opts->seed));
  }
  return GSW_OK;
}

gsw_status gsw_mlp_train(gsw_ctx* ctx, int32_t model_id, int32_t n_train_steps, const gsw_learn_opts* opts) {
  if (!ctx || !opts) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set || !m->input_set) return fail(ctx, GSW_E_STATE, "set the time and the input first");
  if (m->batch) return fail(ctx, GSW_E_STATE, "model %d belongs to a batch", model_id);
  if (m->opts.precision == GSW_PREC_FP64)
    return fail(ctx, GSW_E_STATE, "the learned guess runs with the mixed-precision solver");
  if (!opts->enable) return fail(ctx, GSW_E_INVALID, "opts->enable must be 1");
  if (m->opts.proj_dim > 0)
    return fail(ctx, GSW_E_STATE, "the projection guess and the learned guess exclude each other");
  if (n_train_steps < 5 || m->step + n_train_steps > m->n_steps)
    return fail(ctx, GSW_E_INVALID, "need 5 <= n_train_steps <= the steps left (%lld)",
                (long long)(m->n_steps - m->step));
  if (opts->batch < 64 || opts->batch > 65536 || opts->iters_per_step < 0 || !(opts->lr > 0.f))
    return fail(ctx, GSW_E_INVALID, "need 64 <= batch <= 65536, iters_per_step >= 0, lr > 0");
  const bool fresh = !(m->learn.enable && m->mlp_ready);
  m->learn = *opts;
  m->learn.train_steps = (int32_t)(m->step + n_train_steps);
  if (fresh) {
    TRY(mlp_alloc(ctx, m));
    TRY(mlp_init(ctx, m, opts->seed));
  }
  return gsw_step(ctx, model_id, n_train_steps);
}

gsw_status gsw_mlp_params(gsw_ctx* ctx, int32_t model_id, double* get, const double* set) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->time_set) return fail(ctx, GSW_E_STATE, "call gsw_set_time first");
  TRY(mlp_alloc(ctx, m));
  std::vector<float> th(kMlpParams);
  if (get) {
    CK(cudaMemcpyAsync(th.data(), m->theta, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < kMlpParams; ++i) get[i] = th[i];
  }
  if (set) {
    if (!finite_all(set, kMlpParams)) return fail(ctx, GSW_E_INVALID, "non-finite parameter");
    for (int i = 0; i < kMlpParams; ++i) th[i] = (float)set[i];
    CK(cudaMemcpyAsync(m->theta, th.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, ctx->stream));
    launch_mlp_pack(m->theta, m->packed, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return GSW_OK;
}

gsw_status gsw_mlp_forward(gsw_ctx* ctx, int32_t model_id, int32_t n, const float* x, float* out) {
  if (!ctx || !x || !out) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->mlp_ready) return fail(ctx, GSW_E_STATE, "no MLP: call gsw_set_learning or gsw_mlp_params first");
  if (n <= 0 || n > 65536) return fail(ctx, GSW_E_INVALID, "n must be 1..65536");
  CK(cudaMemcpyAsync(m->trainX, x, sizeof(float) * 16 * n, cudaMemcpyHostToDevice, ctx->stream));
  launch_mlp_infer(n, nullptr, nullptr, m->packed, nullptr, nullptr, m->trainX, m->trainY, ctx->stream, nullptr);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, m->trainY, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSW_OK;
}

gsw_status gsw_mlp_grad(gsw_ctx* ctx, int32_t model_id, int32_t n, const float* x, const float* y, double* loss,
                        double* grad) {
  if (!ctx || !x || !y || !grad || !loss) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->mlp_ready) return fail(ctx, GSW_E_STATE, "no MLP: call gsw_set_learning or gsw_mlp_params first");
  if (n <= 0 || n > 65536) return fail(ctx, GSW_E_INVALID, "n must be 1..65536");
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(m->trainX, x, sizeof(float) * 16 * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m->trainY, y, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpParams, s));
  CK(cudaMemsetAsync(&m->ms->loss, 0, sizeof(double), s));
  if (launch_mlp_fwdbwd(n, m->trainX, m->trainY, m->theta, m->grad, &m->ms->loss, s))
    return fail(ctx, GSW_E_CUDA, "training kernel configuration failed");
  CK(cudaGetLastError());
  std::vector<float> gh(kMlpParams);
  CK(cudaMemcpyAsync(gh.data(), m->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(loss, &m->ms->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpParams, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < kMlpParams; ++i) grad[i] = gh[i];
  return GSW_OK;
}

gsw_status gsw_mlp_state(gsw_ctx* ctx, int32_t model_id, double* out) {
  if (!ctx || !out) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  for (int i = 0; i < 5; ++i) out[i] = 0.0;
  if (m->mlp_ready) {
    CK(cudaMemcpyAsync(out, &m->ms->loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  out[1] = (m->learn.enable && !m->mlp_off) ? 1.0 : 0.0;
  double mean = 0.0;
  const int64_t ks = m->std_r0_n < 5 ? m->std_r0_n : 5;
  for (int64_t i = 0; i < ks; ++i) mean += m->std_r0_recent[i];
  out[2] = ks ? mean / (double)ks : 0.0;
  mean = 0.0;
  const int64_t k = m->mlp_r0_n < 5 ? m->mlp_r0_n : 5;
  for (int64_t i = 0; i < k; ++i) mean += m->mlp_r0_recent[i];
  out[3] = k ? mean / (double)k : 0.0;
  out[4] = (double)m->mlp_r0_n;
  return GSW_OK;
}

gsw_status gsw_mlp_inputs(gsw_ctx* ctx, int32_t model_id, float* x_train, float* y_train, int32_t n,
                          const int32_t* nodes, float* x, double* base, double* scale) {
  if (!ctx) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  Model* m = find(ctx, model_id);
  if (!m) return fail(ctx, GSW_E_INVALID, "unknown model %d", model_id);
  if (!m->learn.enable || !m->mlp_ready) return fail(ctx, GSW_E_STATE, "the learned guess is not enabled");
  if (n < 0 || n > 65536 || (n > 0 && (!nodes || !x || !base)))
    return fail(ctx, GSW_E_INVALID, "need 0 <= n <= 65536 and node, feature and base arrays");
  for (int i = 0; i < n; ++i)
    if (nodes[i] < 0 || nodes[i] >= m->N) return fail(ctx, GSW_E_INVALID, "node %d out of range", nodes[i]);
  if ((n > 0 || scale) && m->hist_count < 1) return fail(ctx, GSW_E_STATE, "no converged step yet");
  cudaStream_t s = ctx->stream;
  const int B = m->learn.batch;
  if (x_train) CK(cudaMemcpyAsync(x_train, m->trainX, sizeof(float) * 16 * (size_t)B, cudaMemcpyDeviceToHost, s));
  if (y_train) CK(cudaMemcpyAsync(y_train, m->trainY, sizeof(float) * 3 * (size_t)B, cudaMemcpyDeviceToHost, s));
  if (n > 0 || scale) {
    // the next step's inputs: the difference scales, the base guess
    launch_mlp_sigma(m->N, m->hist, m->partials, m->ms, s);
    if (!m->guess_base) TRY(alloc_into(ctx, m, &m->guess_base, 3 * (size_t)m->N));
    const double* xb = m->guess_base;
    if (m->opts.guess_order > 0)
      launch_guess_extrap(m->N, m->guess_ring, m->opts.guess_order, m->guess_ext, m->v, m->a, m->dt, m->guess_base, s);
    else
      launch_predictor(m->N, m->v, m->a, m->dt, m->guess_base, s);
    if (n > 0) {
      int32_t* nd = (int32_t*)dev_alloc(ctx, nullptr, sizeof(int32_t) * n);
      float* xd = (float*)dev_alloc(ctx, nullptr, sizeof(float) * 16 * (size_t)n);
      double* bd = (double*)dev_alloc(ctx, nullptr, sizeof(double) * 3 * (size_t)n);
      gsw_status st = GSW_OK;
      if (!nd || !xd || !bd) {
        st = fail(ctx, GSW_E_NOMEM, "device allocation failed (diagnostics)");
      } else if (cudaMemcpyAsync(nd, nodes, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(ctx, GSW_E_CUDA, "node list copy failed");
      } else {
        launch_mlp_inputs(n, nd, m->N, m->hist, m->nodef, m->ms, xb, xd, bd, s);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(x, xd, sizeof(float) * 16 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(base, bd, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
          st = fail(ctx, GSW_E_CUDA, "diagnostic read-back failed");
      }
      cudaStreamSynchronize(s);
      dev_free(ctx, nd);
      dev_free(ctx, xd);
      dev_free(ctx, bd);
      TRY(st);
    }
    if (scale) {
      MlpScalars h = {};
      CK(cudaMemcpyAsync(&h, m->ms, sizeof(MlpScalars), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      scale[0] = h.sigma[0];
      scale[1] = h.sigma_e;
    }
  }
  CK(cudaStreamSynchronize(s));
  return GSW_OK;
}

gsw_status gsw_misfit_noalloc(gsw_ctx* ctx, int32_t n_rec, int32_t n_t, const double* G_dev,
                              const double* obs_dev, int32_t stride, int32_t n_shifts, double tau, double* err_dev,
                              double* c_dev) {
  if (!ctx || !G_dev || !obs_dev || !err_dev) return GSW_E_INVALID;
  DeviceGuard g(ctx->device);
  if (n_rec <= 0 || n_t <= 0 || stride <= 0 || n_shifts <= 0 || !(tau >= 0.0))
    return fail(ctx, GSW_E_INVALID, "need n_rec, n_t, stride, n_shifts > 0 and tau >= 0");
  char msg[256] = {0};
  cudaError_t ce = cudaSuccess;
  int rc = misfit_run_noalloc(ctx->stream, ctx->device, n_rec, n_t, G_dev, obs_dev, stride, n_shifts, tau,
                              err_dev, c_dev, msg, sizeof msg, &ce);
  if (rc == 1) return fail(ctx, GSW_E_CUDA, "misfit (no allocation): %s (%s)", msg, cudaGetErrorString(ce));
  if (rc == 3) return fail(ctx, GSW_E_INVALID, "misfit (no allocation): %s", msg);
  return GSW_OK;
}

}  // extern "C"
