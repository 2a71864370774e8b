// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsw {

constexpr int kMaxMat = 32;        // materials (layers) per model
constexpr int kNodeThreads = 256;  // node-wise kernels
constexpr int kElemThreads = 128;  // element-by-element kernels
constexpr int kMaxNodeBlocks = 152 * 8;
constexpr int kLoBlock = 32;   // elements per block of the reduced-precision operator (one warp)
constexpr int kLoWarps = 4;    // blocks (warps) per CTA
constexpr int kLoThreads = kLoBlock * kLoWarps;

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
};

// Element blocks with local node numbering: block b holds elements
// [b * kLoBlock, (b + 1) * kLoBlock); its unique nodes are
// nodes[ptr[b] .. ptr[b+1]) (bit 31 set: no other block and no absorbing face
// touches the node), and lconn[k * E + e] is the local index of node k of e.
struct BlockView {
  int n_blk;
  int max_local;
  const int32_t* ptr;
  const int32_t* nodes;
  const uint16_t* lconn;
};

// Reduced-precision copy of a model for the inner solve.  SG: storage type of
// the element geometry (float or __half).
template <typename SG>
struct LoView {
  int64_t N, E, F;
  int n_mat;
  BlockView blk;
  const SG* geo;            // [9][E] barycentric gradients
  const float* vol;         // [E] element volumes
  const int32_t* emat;
  const MatCoef* mat;
  const int32_t* fnode;     // [6][F]
  const float* fgeo;        // [6][F]
  double dt;
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
void launch_receivers(const ModelView& m, const double* xyz, double px, double py,
                      const double* rec_xy, int n_rec, int32_t* rec_face, int32_t* rec_node,
                      double* rec_w, int* err, cudaStream_t s);
void launch_ebe(int mode, const ModelView& m, const double* x, const double* v, const double* a,
                double* y, double force, int dir, double* partials, CgScalars* cg,
                cudaStream_t s);
void launch_cg_init(const ModelView& m, const double* b, const double* v, const double* a,
                    double* x, double* q, double* partials, CgScalars* cg, cudaStream_t s);
void launch_rhs_f32(const ModelView& m, const double* u, const double* v, const double* a, float* b32,
                    double force, int dir, cudaStream_t s);
void launch_cg_init_mixed(const ModelView& m, const float* b32, const double* u, const double* v, const double* a,
                          double* x, double* ut, double* vt, double* r, double* q, double* partials, CgScalars* cg,
                          cudaStream_t s);
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
                    const CgScalars* cg, cudaStream_t s);
void launch_record(const double* v, const int32_t* rec_node, const double* rec_w, int n_rec,
                   double* wave, int n_steps, int step, cudaStream_t s);
int ebe_blocks(const ModelView& m);

// ---- mixed precision (gsw_mixed.cu) -------------------------------------------
// Element blocks: counts[b] of unique nodes per block (pass 1), then fill
// nodes / lconn / refcount given ptr (pass 2), then mark exclusive nodes.
void launch_block_count(const ModelView& m, int n_blk, int32_t* counts, cudaStream_t s);
void launch_block_fill(const ModelView& m, BlockView b, int32_t* nodes, uint16_t* lconn,
                       int32_t* refcount, cudaStream_t s);
void launch_block_mark(const ModelView& m, BlockView b, int32_t* nodes, int32_t* refcount,
                       int total, cudaStream_t s);
void launch_lo_convert(const ModelView& m, int half_geo, void* geo_lo, float* vol32, float* fgeo32,
                       const double* dinv, float* dinv32, double* partials, InnerScalars* sc,
                       cudaStream_t s);
// inner solve: half_vec selects __half storage of the search direction d
// (padded to 4 entries per node)
void launch_inner_init(int64_t N, const double* r, const float* dinv32, float* s, float* y,
                       float* t, void* d, int half_vec, float* w, double* partials,
                       InnerScalars* sc, const CgScalars* cg, cudaStream_t st);
void launch_ebe_lo(int half_geo, int half_vec, const void* lo_view, const void* d, float* w,
                   double* partials, InnerScalars* sc, cudaStream_t st);
void launch_inner_update(int64_t N, float* y, float* s, float* t, const void* d, int half_vec,
                         float* w, const float* dinv32, double* partials, InnerScalars* sc,
                         cudaStream_t st);
void launch_inner_dupdate(int64_t N, const float* t, void* d, int half_vec, const InnerScalars* sc,
                          cudaStream_t st);
// conversions for the standalone reduced-precision operator (tests)
void launch_to_lo(int64_t N, const double* x, void* d, int half_vec, float* w, cudaStream_t s);
void launch_from_f32(int64_t N, const float* w, double* y, cudaStream_t s);
// flexible CG outer iteration (FP64)
void launch_fcg_residual(const ModelView& m, const double* b, double* q, double* r, double* partials,
                         CgScalars* cg, cudaStream_t s);
void launch_fcg_first(const ModelView& m, const float* y, const double* r, double* z, double* p,
                      double* partials, CgScalars* cg, const InnerScalars* sc, cudaStream_t s);
void launch_fcg_update(const ModelView& m, double* x, double* r, const double* p, const double* q,
                       double* partials, CgScalars* cg, cudaStream_t s);
void launch_fcg_zbeta(const ModelView& m, const float* y, const double* r, const double* q,
                      double* z, double* partials, CgScalars* cg, const InnerScalars* sc,
                      cudaStream_t s);
void launch_fcg_pupdate(const ModelView& m, const double* z, double* p, double* q,
                        const CgScalars* cg, cudaStream_t s);
int node_blocks(int64_t n);

}  // namespace gsw
