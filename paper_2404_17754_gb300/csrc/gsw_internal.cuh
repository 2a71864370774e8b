// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsw {

constexpr int kMaxMat = 32;        // materials (layers) per model
constexpr int kStatusTimeout = -6;  // GSW_E_TIMEOUT: a bounded device-side wait ran out
constexpr int kNodeThreads = 256;  // node-wise kernels
constexpr int kElemThreads = 128;  // element-by-element kernels
constexpr int kMaxNodeBlocks = 152 * 8;
constexpr int kLoBlock = 192;  // elements (and threads) per CTA of the reduced-precision operator
constexpr int kLoNodesPerThread = 6;  // unique nodes of a block <= kLoBlock * this (checked at set-up)

// Per-material coefficients. lam, mu, rho from (Vp, Vs, rho); alpha, beta the
// Rayleigh fit; cK = 1 + 2 beta/dt and cM = 4/dt^2 + 2 alpha/dt scale the
// element stiffness and mass inside A = K + (2/dt) C + (4/dt^2) M.
struct MatCoef {
  double lam, mu, rho, alpha, beta, Vp, Vs, h, cK, cM;
};

// Device-side scalars of one CG solve (one per model and right-hand side).
struct CgScalars {
  double bb;      // ||b||^2
  double rz;      // r . z of the current iterate
  double pq;      // p . A p
  double rr;      // r . r
  double relres;  // ||r|| / ||b||
  double tol;
  double beta;    // p <- z + beta p
  double alpha;   // step length of the last update
  int iter;
  int max_iter;
  int done;       // 1 once converged or failed
  int status;     // 0, or a gsw_status error code
  int zero_rhs;   // b == 0: the solution is exactly 0
  int pad1;
  unsigned int counter;  // arrival counter of the last-block reductions
  unsigned int pad2;
  double relres0;  // ||r|| / ||b|| at the step's initial guess
};

// Scalars of the learned initial guess (one set per model).
constexpr int kMlpParams = 5443;  // 16-64-64-3 MLP
struct MlpScalars {
  double sigma[4];  // RMS of the backward differences D_0..D_3 of the latest increments
  double loss;      // training loss accumulator
  unsigned int counter;
  unsigned int pad;
  double sigma_e;   // RMS of the last step's correction du - base (the output scale)
};
void launch_mlp_sigma_e(int64_t N, const double* du, const double* base, double* partials, MlpScalars* ms,
                        cudaStream_t s);

// Step counter and status of a model advanced on the device (batched,
// graph-captured stepping): the host reads it only between steps.
struct StepState {
  int step;        // index of the next step to compute
  int n_steps;
  int active;      // this step runs (step < n_steps and no earlier failure)
  int failed;      // sticky: status of the first failure (0 = none)
  int fail_step;
  int commit;      // this step converged: apply the Newmark update and record
  int stop_at;     // the batch call advances the model up to this step
  int needs_host;  // the outer budget ran out: the host completes this step
  int iters_last, iters_max;
  long long iters_total;
  long long inner_total;
  double relres_last;
  double tol;
  int max_iter;
  int inner_iters;
  int loops;       // body runs of the device-side outer-iteration loop in this step
  int pad_;
};

// Device-driven inputs of a step (null pointers: the host drives the step).
struct Drive {
  const double* p;  // [n_steps] input samples
  StepState* ss;
};

// Element / face / node data of one uploaded model (device pointers).
struct ModelView {
  int64_t N;                // nodes
  int64_t E;                // elements
  int64_t F;                // boundary faces (all tags)
  const int32_t* conn;      // [10][E] (structure of arrays)
  const double* geo;        // [10][E]: grad L1 (3), grad L2 (3), grad L3 (3), V
  const int32_t* emat;      // [E]
  const MatCoef* mat;       // [n_mat]
  const int32_t* fnode;     // [6][F]
  const double* fgeo;       // [6][F]: A rho Vs, A (rho Vp - rho Vs), n (3), tag
  double dt;
};

// Scalars of the reduced-precision inner solve (the variable preconditioner).
struct InnerScalars {
  double st;     // s . t  (t = D^-1 s)
  double dw;     // d . A d
  double beta;
  double scale;  // inner right-hand side = scale * outer residual
  double dinv_mean;  // mean diagonal entry of D^-1 (set once per model)
  unsigned int counter;
  unsigned int pad;
  float alpha_f;  // s . t / d . A d, set by the last block of the operator kernel
  float beta_f;   // FP32 copy of beta for the direction update
  unsigned int err;   // nonzero: a bounded wait of the operator kernel ran out
  unsigned int n_dw;  // grid size of the last operator launch (entries of LoView::dw_part)
  double st0;         // s . t at the start of the current inner solve
  float rtol2;        // squared relative stopping factor (0: fixed iteration count)
  unsigned int idone; // 1 once the current inner solve has met rtol
  unsigned long long iters;  // inner iterations executed (all solves)
  double st_f;        // s . D^-1 s, the fine part of s . t (two-level preconditioner)
  unsigned int coarse_on;  // two-level: this inner solve applies the coarse correction
  unsigned int pad2;
};

// First-order (vertex) coarse level of the two-level inner preconditioner
// t = D^-1 s + omega P D_c^-1 P^T s: P interpolates vertex values to the
// quadratic nodes (a vertex node takes its vertex's value, a mid-edge node the
// mean of its edge's two vertices), D_c are the 3x3 nodal diagonal blocks of
// P^T A P (the linear-tetrahedron operator on the same vertices).
struct CoarseView {
  int64_t Nv;            // vertices
  const int32_t* vnode;  // [Nv] fine node of each vertex
  const int32_t* ptr;    // [Nv + 1] CSR: the mid-edge nodes on each vertex's edges
  const int32_t* mid;    // [ptr[Nv]]
  const int2* pair;      // [N] the two vertices a fine node interpolates (a vertex node: its own twice)
  const float* dc;       // [Nv][6] omega D_c^-1 / mean(D^-1) (xx yy zz xy xz yz)
};

// Element blocks with local node numbering: block b holds elements
// [b * kLoBlock, (b + 1) * kLoBlock); its unique nodes are
// nodes[ptr[b] .. ptr[b+1]) (bit 31 set: no other block and no absorbing face
// touches the node).  Local connectivity lives in the packed element records.
struct BlockView {
  int n_blk;
  int max_local;
  const int32_t* ptr;
  const int32_t* nodes;
};

// Reduced-precision copy of a model for the inner solve.  SG: storage type of
// the element geometry (float or __half).
template <typename SG>
struct LoView {
  int64_t N, E, F;
  int n_mat;
  BlockView blk;
  const void* rec;          // [n_blk * kLoBlock] packed element records (operator order)
  const float4* matf;       // [n_mat] (cK lam / 20, cK mu / 20, cM rho / 420, 0) in FP32
  const int32_t* fnode;     // [6][F]
  const float* fgeo;        // [6][F]
  double dt;
  float* dw_part;           // [operator grid] per-CTA partial sums of d . A d
  float face_c;             // (2 / dt) / 180: dashpot face-mass scale
};

enum EbeMode { kModeA = 0, kModeK = 1, kModeM = 2, kModeC = 3, kModeRhs = 4, kModeRes = 5 };

// ---- kernels (gsw_kernels.cu) -------------------------------------------------
void launch_geometry(const ModelView& m, const double* xyz, double px, double py, double* geo,
                     int* err, cudaStream_t s);
void launch_face_geometry(const ModelView& m, const double* xyz, double px, double py,
                          const int32_t* face_elem, const int32_t* face_tag, double* fgeo,
                          int* err, cudaStream_t s);
void launch_material(MatCoef* mat, const double* raw, int n_mat, double dt, double f1, double f2,
                     cudaStream_t s);
void launch_block_jacobi(const ModelView& m, double* dblk, double* dinv, int* err,
                         cudaStream_t s);
// 3x3 nodal diagonal blocks of P^T A P on the vertices (vid: vertex index of
// each fine node, -1 elsewhere; cblk zeroed by the caller) and their inverses
void launch_coarse_blocks(const ModelView& m, const int32_t* vid, double* cblk, cudaStream_t s);
void launch_invert_blocks(int64_t n, const double* blk, double* inv, int* err, cudaStream_t s);
void launch_receivers(const ModelView& m, const double* xyz, double px, double py,
                      const double* rec_xy, int n_rec, int32_t* rec_face, int32_t* rec_node,
                      double* rec_w, int* err, cudaStream_t s);
void launch_ebe(int mode, const ModelView& m, const double* x, const double* v, const double* a,
                double* y, double force, int dir, double* partials, CgScalars* cg,
                cudaStream_t s, Drive dr = Drive{nullptr, nullptr});
// The flexible CG's outer operator in double-word (paired FP32) arithmetic:
// mode kModeA (with partials / cg as launch_ebe) or kModeRes.  dw_in: the
// input vectors are stored as double-word pairs (always so for kModeRes).
void launch_ebe_dw(int mode, int dw_in, const ModelView& m, const double* x, const double* v, const double* a,
                   double* y, double force, int dir, double* partials, CgScalars* cg,
                   cudaStream_t s, Drive dr = Drive{nullptr, nullptr});
// Initial guess from the last k+1 increments (degree-k extrapolation), k <=
// kMaxGuessOrder; ring: [k+1][3N] doubles, ext: {count, head} on the device.
constexpr int kMaxGuessOrder = 6;
struct ProjState;
// ps: a projection guess that hands over to the extrapolation; while it has not
// retired the kernel writes du0 = 0 (the residual pass then yields b for it)
void launch_guess_extrap(int64_t N, const double* ring, int k, const int* ext, const double* v, const double* a,
                         double dt, double* x, cudaStream_t s, const StepState* ss = nullptr,
                         const ProjState* ps = nullptr);
void launch_guess_push(int64_t N, const double* du, double* ring, int k, int* ext, cudaStream_t s,
                       const StepState* ss = nullptr);
// Initial guess by Galerkin projection onto the last k <= kMaxProj converged
// increments W with Z = A W (kept from each step's b - r): c = G^+ W^T b,
// G = W^T Z, du0 = W c.  W, Z: [k][3N] doubles.
constexpr int kMaxProj = 8;
struct ProjState {
  int count, head;          // filled slots, next slot
  unsigned int counter;     // arrival counter of the last-block reductions
  unsigned int pad;
  double G[kMaxProj * kMaxProj];  // by slot
  double c[kMaxProj];             // coefficients of the current step
  int retired;                    // 1: the extrapolated guess has taken over for the rest of the run
  int pad2;
};
void launch_proj_coef(int64_t N, const double* W, const double* b, ProjState* ps, double* partials, cudaStream_t s,
                      const StepState* ss = nullptr);
// x = W c; r (holding b on entry) -> b - Z c; bkeep <- b
void launch_proj_apply(int64_t N, const double* W, const double* Z, const ProjState* ps, double* x, double* r,
                       double* bkeep, cudaStream_t s, const StepState* ss = nullptr);
void launch_proj_guess(int64_t N, const double* W, const ProjState* ps, double* x, cudaStream_t s,
                       const StepState* ss = nullptr);
// on commit: W[head] = du, Z[head] = b - r, G row/column of head, advance; with
// handover > 0 the projection retires once a step started from an initial
// relative residual (cg->relres0) below handover.  All projection kernels
// return at entry once it has retired.
void launch_proj_push(int64_t N, const double* du, const double* b, const double* r, double* W, double* Z,
                      ProjState* ps, int k, double* partials, cudaStream_t s, const StepState* ss = nullptr,
                      const CgScalars* cg = nullptr, double handover = 0.0);
void launch_cg_init(const ModelView& m, const double* b, const double* v, const double* a,
                    double* x, double* q, double* partials, CgScalars* cg, cudaStream_t s, int use_guess = 0,
                    const StepState* ss = nullptr);
// FP32 right-hand side on the reduced-precision operator's element blocks
// (uva: [N + 1][3] float4 scratch for the FP32 state; b32 zero on entry).
void launch_rhs_lo(int half_geo, const void* lo_view, int64_t N, const double* u, const double* v, const double* a,
                   float4* uva, float* b32, double force, int dir, cudaStream_t st, Drive dr = Drive{nullptr, nullptr});
// x0 = x (use_guess) or the predictor dt v + dt^2/2 a; writes u~ = u + x0,
// v~ = v - (2/dt) x0, a~ = a + (4/dt) v - (4/dt^2) x0 for the one-pass residual
void launch_cg_init_mixed(const ModelView& m, const float* b32, const double* u, const double* v, const double* a,
                          double* x, double* ut, double* vt, double* at, double* r, double* q, double* partials,
                          CgScalars* cg, cudaStream_t s, const StepState* ss = nullptr, int use_guess = 0,
                          int dw_out = 0);
// device-driven step bracket (batched stepping)
void launch_step_begin(StepState* ss, CgScalars* cg, cudaStream_t s);
void launch_step_end(StepState* ss, const CgScalars* cg, cudaStream_t s);
void launch_step_advance(StepState* ss, cudaStream_t s);
// Device-side iteration loop of a captured step (a WHILE conditional node)
// over a set of up to three solves that advance together: `open` sets the
// loop condition before the node (run the body unless every step is inactive
// or already converged); `next`, the body's last kernel, keeps it set while a
// solve of the set has not converged and the body has run fewer than `cap`
// times, so the loop always ends.
struct LoopSet {
  StepState* ss[3];
  const CgScalars* cg[3];
  int n;
};
void launch_loop_open(cudaGraphConditionalHandle h, const LoopSet& ls, int cap, cudaStream_t s);
void launch_loop_next(cudaGraphConditionalHandle h, const LoopSet& ls, int cap, cudaStream_t s);
void launch_cg_rnorm(const ModelView& m, const double* r, double* partials, CgScalars* cg, cudaStream_t s);
void launch_cg_residual(const ModelView& m, const double* b, double* q, double* r, double* z,
                        double* p, const double* dinv, double* partials, CgScalars* cg,
                        cudaStream_t s);
void launch_cg_update(const ModelView& m, double* x, double* r, double* z, const double* p,
                      double* q, const double* dinv, double* partials, CgScalars* cg,
                      cudaStream_t s);
void launch_cg_pupdate(const ModelView& m, const double* z, double* p, const CgScalars* cg,
                       cudaStream_t s);
void launch_newmark(const ModelView& m, const double* x, double* u, double* v, double* a,
                    const CgScalars* cg, cudaStream_t s, const StepState* ss = nullptr);
void launch_record(const double* v, const int32_t* rec_node, const double* rec_w, int n_rec,
                   double* wave, int n_steps, int step, cudaStream_t s, const StepState* ss = nullptr);
int ebe_blocks(const ModelView& m);

// ---- mixed precision (gsw_mixed.cu) -------------------------------------------
// Element blocks: counts[b] of unique nodes per block (pass 1), then fill
// nodes / lconn / refcount given ptr (pass 2), then mark exclusive nodes.
void launch_block_count(const ModelView& m, int n_blk, int32_t* counts, cudaStream_t s);
void launch_block_fill(const ModelView& m, BlockView b, int32_t* nodes, uint16_t* lconn,
                       int32_t* refcount, cudaStream_t s, const int32_t* counts);
void launch_block_mark(const ModelView& m, BlockView b, int32_t* nodes, int32_t* refcount,
                       int total, cudaStream_t s);
// dinv_lo: D^-1 divided by its mean diagonal entry, in the inner storage type (half_vec)
void launch_lo_convert(const ModelView& m, int n_blk, const uint16_t* lconn, int half_geo, int half_vec, void* rec,
                       float* fgeo32, const double* dinv, void* dinv_lo, double* partials, InnerScalars* sc,
                       float4* matf, int n_mat, cudaStream_t s);
size_t lo_record_bytes(int half_geo);
// inner solve: half_vec selects __half storage of the search direction d, of
// t = D^-1 s (both padded to 4 entries per node) and of the scaled D^-1
// coarse_rel: two-level preconditioner, the solve applies the coarse correction
// while the outer relative residual ||r|| / ||b|| it starts from exceeds
// coarse_rel (<= 0: always)
void launch_inner_init(int64_t N, const double* r, const void* dinv_lo, float* s, float* y,
                       void* t, void* d, int half_vec, float* w, double* partials,
                       InnerScalars* sc, const CgScalars* cg, cudaStream_t st, float rtol,
                       double coarse_rel = 0.0);
void launch_ebe_lo(int half_geo, int half_vec, const void* lo_view, const void* d, float* w,
                   double* partials, InnerScalars* sc, cudaStream_t st, int variant,
                   const CgScalars* outer = nullptr);
constexpr int kLoVariants = 4;
// The inner operator on the search directions of up to three inner solves
// that share one model's element data (the three input directions advancing
// in lockstep): one read of the records and node lists for all of them.
struct Lo3Args {
  const void* d[3];          // search directions (inner storage type, 4 entries per node)
  float* w[3];               // results A d
  float* dw_part[3];         // per-CTA partials of d . A d
  InnerScalars* sc[3];
  const CgScalars* outer[3];
  int nr;                    // right-hand sides in use (1..3)
};
void launch_ebe_lo3(int half_geo, int half_vec, const void* lo_view, const Lo3Args& a, cudaStream_t st, int variant);
// Variants 0 and 1 can fuse the previous inner iteration's direction
// recurrence d' = t + beta d into their gather (t padded to 4 entries per
// node; d' goes to the other direction buffer).
bool lo_variant_fuses(int variant);
void launch_ebe_lo_fused(int half_geo, int half_vec, const void* lo_view, const void* dprev, const void* t4,
                         void* dnew, float* w, double* partials, InnerScalars* sc, cudaStream_t st, int variant,
                         const CgScalars* outer);
// n_dw_max: an upper bound of the operator's grid size; up to
// kAlphaPrologueMax partials the update forms alpha itself (one launch less).
constexpr int kAlphaPrologueMax = 2048;
void launch_inner_update(int64_t N, float* y, float* s, void* t, const void* d, int half_vec,
                         float* w, const void* dinv_lo, const float* dw_part, double* partials,
                         InnerScalars* sc, cudaStream_t st, const CgScalars* outer, int n_dw_max);
void launch_inner_dupdate(int64_t N, const void* t, void* d, int half_vec, const InnerScalars* sc,
                          cudaStream_t st, const CgScalars* outer, const int2* pair = nullptr,
                          const float4* zc = nullptr);
// Two-level inner preconditioner.  With coarse = 1 the update kernel leaves
// s . t, beta and the stopping test to the restriction kernel (it stores the
// fine part s . D^-1 s in st_f); the restriction forms z_c = omega D_c^-1 P^T s
// and completes s . t (first = 1: at the start of an inner solve, beta = 0);
// the direction update (pair, zc) adds P z_c to t.
void launch_inner_update_coarse(int64_t N, float* y, float* s, void* t, const void* d, int half_vec, float* w,
                                const void* dinv_lo, const float* dw_part, double* partials, InnerScalars* sc,
                                cudaStream_t st, const CgScalars* outer, int n_dw_max);
void launch_coarse_restrict(const CoarseView& c, const float* s, float4* zc, double* partials, InnerScalars* sc,
                            const CgScalars* outer, int first, cudaStream_t st);
// y = scale * P z_c (FP64 output, diagnostics)
void launch_coarse_prolong(int64_t N, const int2* pair, const float4* zc, double scale, double* y, cudaStream_t st);
// dc = omega * cinv / mean(D^-1) in FP32
void launch_coarse_lo(int64_t Nv, const double* cinv, const InnerScalars* sc, double omega, float* dc,
                      cudaStream_t st);
void launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t st);
// failure-detection self-test of the bounded mbarrier wait (out[2] on the device)
void launch_wait_probe(long long limit, unsigned* out, cudaStream_t st);
// conversions for the standalone reduced-precision operator (tests)
void launch_to_lo(int64_t N, const double* x, void* d, int half_vec, float* w, cudaStream_t s);
void launch_from_f32(int64_t N, const float* w, double* y, cudaStream_t s);
// flexible CG outer iteration (FP64)
void launch_fcg_residual(const ModelView& m, const double* b, double* q, double* r, double* partials,
                         CgScalars* cg, cudaStream_t s);
void launch_fcg_first(const ModelView& m, const float* y, const double* r, double* z, double* p,
                      double* partials, CgScalars* cg, const InnerScalars* sc, cudaStream_t s, int dwp = 0);
void launch_fcg_update(const ModelView& m, double* x, double* r, const double* p, const double* q,
                       double* partials, CgScalars* cg, cudaStream_t s, int dwp = 0);
void launch_fcg_zbeta(const ModelView& m, const float* y, const double* r, const double* q,
                      double* z, double* partials, CgScalars* cg, const InnerScalars* sc,
                      cudaStream_t s);
void launch_fcg_pupdate(const ModelView& m, const double* z, double* p, double* q,
                        const CgScalars* cg, cudaStream_t s, int dwp = 0);
int node_blocks(int64_t n);

// ---- learned initial guess (gsw_mlp.cu) ------------------------------------------
void launch_mlp_pack(const float* theta, uint32_t* packed, cudaStream_t s);
void launch_node_features(const ModelView& m, int n_mat, int32_t* node_mat, float* nodef, cudaStream_t s);
// hist: [4][3N] doubles, the backward differences D_0..D_3 of the last four
// converged increments (D_k = sum_j (-1)^j C(k, j) du_{s-1-j}).
void launch_mlp_sigma(int64_t N, const double* hist, double* partials, MlpScalars* ms, cudaStream_t s);
// x <- base + sigma_e * MLP(features) over all nodes (xin / yout: explicit
// features and raw outputs, diagnostics)
void launch_mlp_infer(int64_t N, const double* hist, const float* nodef, const uint32_t* packed, const MlpScalars* ms,
                      double* x, const float* xin, float* yout, cudaStream_t s, const double* x_base);
void launch_mlp_sample(int64_t N, int B, uint32_t seed, int step, int iter, const double* hist, const float* nodef,
                       const double* du, const double* base, const MlpScalars* ms, float* X, float* Y, cudaStream_t s);
int launch_mlp_fwdbwd(int B, const float* X, const float* Y, const float* theta, float* grad, double* loss,
                      cudaStream_t s);
void launch_mlp_adam(float* theta, float* grad, float* m, float* v, int t, float lr, cudaStream_t s);
void launch_hist_push(int64_t N, const double* du, double* hist, const CgScalars* cg, cudaStream_t s,
                      const StepState* ss = nullptr);
void launch_predictor(int64_t N, const double* v, const double* a, double dt, double* x, cudaStream_t s);
void launch_mlp_inputs(int n, const int32_t* nodes, int64_t N, const double* hist, const float* nodef,
                       const MlpScalars* ms, const double* base, float* X, double* base_out, cudaStream_t s);
int mlp_packed_words();

}  // namespace gsw
