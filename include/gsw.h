/*
 * gsw.h -- C ABI of the GB300 implicit finite-element seismic-wave library.
 *
 * The library runs the per-candidate 3D wave-propagation analysis of
 * Ichimura et al., "Development of an Estimation Method for the Seismic Motion
 * Reproducibility of a Three-dimensional Ground Structure Model ..."
 * (arXiv 2404.17754): Eq. (1) (linear elastodynamics) discretised with
 * second-order tetrahedra, Newmark-beta implicit time integration solved by
 * preconditioned conjugate gradients every step (Section 3, computational-cost
 * paragraph), absorbing base and sides driven by the input velocity at the
 * base (Section 2), surface receivers, and the input-wave estimate and misfit
 * ERR of Section 2, Eq. (2).
 *
 * Conventions (all entry points):
 *  - Every call returns a gsw_status.  No C++ exception crosses the ABI.
 *    gsw_last_error() returns a message describing the last failing call on
 *    that context.  A failed call leaves the context usable.
 *  - Pointers are HOST pointers unless the argument name ends in "_dev"
 *    (device memory on the context's GPU).  The library copies what it needs
 *    from host arrays during the call; the caller keeps ownership.
 *  - Arrays are C-contiguous.  Node-major vectors are [n_nodes][3] float64.
 *  - Device memory (model data, batch step states, misfit scratch) is
 *    allocated through the allocator set by gsw_set_allocator (default:
 *    cudaMallocAsync on the context's stream); gsw_misfit_noalloc allocates
 *    none.
 *  - All GPU work is issued on the stream given to gsw_create.  Calls that
 *    return host data synchronise that stream.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef GSW_H
#define GSW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsw_ctx gsw_ctx;

typedef enum {
  GSW_OK = 0,
  GSW_E_INVALID = -1,  /* bad argument or malformed mesh (message says which) */
  GSW_E_CUDA = -2,     /* CUDA runtime error */
  GSW_E_NOMEM = -3,    /* device allocation failed */
  GSW_E_NOCONV = -4,   /* CG did not reach the tolerance within max_iter */
  GSW_E_NAN = -5,      /* non-finite residual or state */
  GSW_E_TIMEOUT = -6,  /* a bounded device-side wait gave up */
  GSW_E_STATE = -7     /* call not valid in the model's current state */
} gsw_status;

/* Solver precision of the preconditioner's inner products (the outer CG
 * vectors, its dot products and the Newmark update are FP64 in every mode;
 * the arithmetic of the outer operator is set by gsw_outer_op). */
typedef enum {
  GSW_PREC_FP64 = 0,   /* plain block-Jacobi PCG, everything FP64 */
  GSW_PREC_FP32 = 1,   /* flexible CG; inner preconditioner EBE in FP32 */
  GSW_PREC_FP16 = 2    /* flexible CG; inner vectors FP16, FP32 EBE arithmetic */
} gsw_precision;

/* Arithmetic of the CG's (outer) operator A = K + (2/dt) C + (4/dt^2) M.
 * Double-word: each FP64 value is carried as an unevaluated sum of two floats
 * (about 48 significant bits) and every operation is an error-free
 * transformation on the FP32 pipe (TwoSum, Fast2Sum, TwoProd with a fused
 * multiply-add); element data, vectors and the accumulation of A x stay FP64
 * in memory.  Relative error of A x about 2^-46 times the cancellation of the
 * element sums, far below the 1e-8 residual target; on GB300, whose FP64 pipe
 * retires 2 fused multiply-adds per clock per SM against 128 in FP32, the
 * double-word operator is the faster one. */
typedef enum {
  GSW_OUTER_AUTO = 0,   /* double-word in the mixed modes, FP64 in GSW_PREC_FP64 */
  GSW_OUTER_FP64 = 1,   /* hardware FP64 */
  GSW_OUTER_DWORD = 2   /* double-word arithmetic */
} gsw_outer_op;

typedef struct {
  double tol;           /* relative residual ||b - A x|| / ||b|| target (1e-8) */
  int32_t max_iter;     /* outer CG iteration cap per step -> GSW_E_NOCONV */
  int32_t precision;    /* gsw_precision */
  int32_t inner_iters;  /* inner preconditioner iterations (mixed modes) */
  int32_t check_every;  /* CG iterations issued between host convergence checks */
  int32_t batch_outer;  /* batched stepping: flexible-CG iterations a step may use
                           inside the step graph; a step that needs more is
                           completed by the host-driven solver (up to max_iter)
                           and the model then rejoins the graph.  0 = 32 in the
                           device-side loop; with the unrolled fallback, 0 =
                           a budget that starts at 6 and follows the steps (one
                           more than the most iterations a step of the last
                           8-step chunk needed; raised at once, lowered after
                           two lower chunks; the graph is re-captured) */
  int32_t inner_variant; /* launch variant of the inner operator: -1 lets the set-up
                            autotuner time all and keep the fastest; 0, 1 one CTA
                            per element block (3 or 4 CTAs per SM); 2 persistent,
                            cp.async-pipelined CTAs; 3 persistent warp-specialised
                            CTAs (a producer warp stages element blocks with bulk
                            asynchronous copies and mbarriers) */
  double inner_rtol;     /* mixed modes: the inner PCG stops once its preconditioned
                            residual norm has dropped by this factor (0 = always run
                            inner_iters iterations, which stay the cap); must be in [0, 1) */
  int32_t guess_order;   /* initial guess of each step's solve: 0 = the Newmark
                            predictor dt v + dt^2/2 a; k = 1..6 = the degree-k
                            polynomial through the last k+1 converged increments,
                            one step ahead (the predictor until k+1 exist; the
                            history restarts at gsw_reset / gsw_set_state).  Any
                            guess converges to the same tolerance. */
  int32_t outer_op;      /* arithmetic of the CG's element-by-element operator (the
                            FP64 residual at the initial guess and A p): gsw_outer_op */
  int32_t share_dirs;    /* mixed modes, gsw_run with a direction mask: 1 = the model's
                            direction analyses advance in lockstep and share every
                            inner-operator pass (the element records and node lists
                            are read once for all directions; a direction whose solve
                            has converged skips its share); 0 = each advances on its own */
  int32_t proj_dim;      /* 0, or k = 2..8: each step's initial guess is the Galerkin
                            projection of its solution onto the last k converged
                            increments W, du0 = W c with (W^T A W) c = W^T b; A W is kept
                            from each converged step (b - r, no extra operator pass)
                            and, in the mixed modes, b comes from the residual pass at
                            du0 = 0.  Takes precedence over guess_order; excludes the
                            learned guess.  The history restarts at gsw_reset /
                            gsw_set_state. */
  double coarse_weight;  /* mixed modes: 0 = the inner PCG's preconditioner is the
                            3x3 nodal block Jacobi D^-1; omega > 0 = the two-level
                            preconditioner D^-1 + omega P D_c^-1 P^T, with P the
                            interpolation from the vertices (first-order coarse
                            level, Section 3's multi-level solver) to the quadratic
                            nodes and D_c the nodal diagonal blocks of P^T A P;
                            must be finite and in [0, 4] */
  double coarse_relres;  /* two-level preconditioner: an inner solve applies the coarse
                            correction only while the outer relative residual ||r|| / ||b||
                            it starts from exceeds this (0 = in every inner solve); the
                            coarse level removes smooth error, which a poor initial guess
                            leaves and a good one does not */
  double proj_relres;    /* 0, or with proj_dim > 0 and guess_order > 0: the projection
                            guess hands over, for the rest of the run, to the degree-
                            guess_order extrapolation once a step starts from an initial
                            relative residual below this (the projection pays while the
                            motion is young and the extrapolation is poor); the history
                            restarts, and the projection with it, at gsw_reset /
                            gsw_set_state */
} gsw_solver_opts;

typedef struct {
  int64_t steps_done;     /* time steps completed since the last reset */
  int64_t cg_iters_total; /* outer CG iterations summed over those steps */
  int32_t cg_iters_last;  /* outer CG iterations of the last step */
  int32_t cg_iters_max;   /* largest per-step count so far */
  double relres_last;     /* final recursive relative residual of the last step */
  int64_t inner_iters_total; /* inner preconditioner iterations (mixed modes) */
  int64_t kernel_launches;   /* library kernels launched by gsw_step since the last reset */
  double init_relres_sum;    /* sum over host-driven mixed steps of the relative residual
                                of the initial guess (measures the guess quality) */
} gsw_stats;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the CUDA default stream, as in the runtime API). */
gsw_status gsw_create(gsw_ctx **out, int device, void *cuda_stream);
void gsw_destroy(gsw_ctx *ctx);
const char *gsw_last_error(const gsw_ctx *ctx);

/* Route device allocations through caller callbacks (for example a framework's
 * caching allocator).  alloc(bytes, stream, user) returns device memory or
 * NULL; free_(ptr, stream, user) releases it.  Pass NULLs to restore the
 * default.  Must be called before any model is uploaded. */
gsw_status gsw_set_allocator(gsw_ctx *ctx, void *(*alloc)(size_t, void *, void *),
                             void (*free_)(void *, void *, void *), void *user);

/* ---- model -------------------------------------------------------------- */

/* Upload one candidate ground model (Section 3: second-order tetrahedra).
 *  xyz       [n_nodes][3] node coordinates (m); x3 is elevation, surface z = 0.
 *  conn      [n_elem][10] node indices, VTK quadratic-tetrahedron order
 *            (vertices 0..3, then mid-edge nodes of edges 01,12,02,03,13,23);
 *            det[x1-x0, x2-x0, x3-x0] > 0; straight-sided (mid-edge nodes at
 *            edge midpoints).
 *  elem_mat  [n_elem] layer index into mat.
 *  mat       [n_mat][4] rows (Vp, Vs, rho, h): P/S velocity, density, damping
 *            ratio; requires Vp > Vs > 0, rho > 0, h >= 0.
 *  faces     [n_faces][6] 6-node boundary triangles (3 vertices, then the
 *            mid-edge nodes of edges 01, 12, 20), face_elem [n_faces] owning
 *            element, face_tag [n_faces]: 0 free surface, 1 absorbing base
 *            (carries the input), 2 absorbing side.
 *  period    [2] lateral periods for laterally periodic meshes, 0 = none.
 *  rec_xy    [n_rec][2] receiver positions on the free surface.
 * Validation (index ranges, finiteness, material order, positive volumes,
 * straight sides, receivers on the surface) rejects the model with
 * GSW_E_INVALID.  On success *model_id receives a handle. */
gsw_status gsw_model_upload(gsw_ctx *ctx, int64_t n_nodes, const double *xyz, int64_t n_elem,
                            const int32_t *conn, const int32_t *elem_mat, int32_t n_mat,
                            const double *mat, int64_t n_faces, const int32_t *faces,
                            const int32_t *face_elem, const int32_t *face_tag,
                            const double *period, int32_t n_rec, const double *rec_xy,
                            int32_t *model_id);
gsw_status gsw_model_free(gsw_ctx *ctx, int32_t model_id);
/* Sizes of an uploaded model: out[0]=n_nodes, out[1]=n_elem, out[2]=n_faces,
 * out[3]=n_rec, out[4]=device bytes held, out[5]=launch variant of the inner
 * reduced-precision operator chosen by the set-up autotuner (-1 before a
 * mixed precision mode is set). */
gsw_status gsw_model_info(gsw_ctx *ctx, int32_t model_id, int64_t *out);

/* Time integration (Section 3: Newmark-beta, average acceleration
 * beta = 1/4, gamma = 1/2) with increment dt and Rayleigh damping fitted to
 * each layer's h over [f1, f2] Hz.  Allocates the step-dependent state,
 * builds the block-Jacobi preconditioner and resets the model to rest. */
gsw_status gsw_set_time(gsw_ctx *ctx, int32_t model_id, double dt, int32_t n_steps, double f1,
                        double f2);

/* Input velocity (Section 2: force at the base): p[n] is the incident
 * velocity at t_{n+1} = (n+1) dt in direction dir (0 = x1, 1 = x2, 2 = x3);
 * the base load is 2 C_base (p e_dir).  n must equal the model's n_steps.
 * The model keeps the input of each direction (for gsw_run's direction mask);
 * its own analysis, advanced by gsw_step, follows the direction of the last
 * call. */
gsw_status gsw_set_input(gsw_ctx *ctx, int32_t model_id, int32_t dir, const double *p, int32_t n);

gsw_status gsw_set_solver(gsw_ctx *ctx, int32_t model_id, const gsw_solver_opts *opts);

/* Reset the model to rest (u = v = a = 0, step 0, receivers cleared). */
gsw_status gsw_reset(gsw_ctx *ctx, int32_t model_id);

/* Advance n time steps.  On GSW_E_NOCONV / GSW_E_NAN the model stays at the
 * last completed step and further steps return GSW_E_STATE until reset. */
gsw_status gsw_step(gsw_ctx *ctx, int32_t model_id, int32_t n);

/* Run analyses from rest through all their steps (Section 2: the Green's
 * functions of a candidate are three analyses, one per input direction; one
 * candidate analysis in the sense of Section 3's cost paragraph is all three).
 *  dirs_mask = 0: each listed model's own analysis (its last gsw_set_input
 *    direction);
 *  dirs_mask bits 0..2 (x1, x2, x3): for every listed model, the analysis of
 *    each direction whose bit is set, from the input last set for that
 *    direction (GSW_E_STATE if none).  These analyses share the model's mesh,
 *    element, preconditioner and inner-operator data and hold their own state
 *    and receiver history (read with gsw_read_waveforms(..., dir, ...)); they
 *    are re-made after gsw_set_time or gsw_set_solver.
 * All analyses run together as one batch (see gsw_batch_create), except a
 * model's own analysis with the learned guess enabled, which runs first with
 * host-driven steps. */
gsw_status gsw_run(gsw_ctx *ctx, const int32_t *model_ids, int32_t n_models, int32_t dirs_mask);

/* ---- batched stepping ------------------------------------------------------
 * A batch advances several models (uneven sizes and any mix of precision
 * modes allowed) together: every time step of every model runs on the device
 * without host synchronisation (device-side step counter and input samples;
 * the CG iterations run in a device-side loop of the graph, a WHILE
 * conditional node, until the step converges or the budget is used up: in the
 * mixed modes the flexible-CG iterations after a step's first, at most
 * solver_opts.batch_outer; in GSW_PREC_FP64 every block-Jacobi PCG iteration,
 * at most batch_outer, or 1000 when batch_outer = 0), each model on its own
 * stream, all captured into one CUDA graph that is launched once per time
 * step.  Where
 * the conditional node cannot be built, the budget is unrolled into the
 * graph (kernels of a converged step return at entry).  Models that reach their
 * n_steps stop advancing; a step that needs more outer iterations than the
 * budget is finished by the host-driven solver; a model that fails stops at
 * the failing step while the others continue, and gsw_batch_step reports the
 * first failure.  Member models keep their own state, waveforms and
 * statistics. */
gsw_status gsw_batch_create(gsw_ctx *ctx, const int32_t *model_ids, int32_t n_models,
                            int32_t *batch_id);
/* Advance every member by n_steps time steps (members already at their end
 * stay there).  The step graph is (re)captured when a member's solver
 * options or time set-up changed since the last capture. */
gsw_status gsw_batch_step(gsw_ctx *ctx, int32_t batch_id, int32_t n_steps);
gsw_status gsw_batch_destroy(gsw_ctx *ctx, int32_t batch_id);
/* Kernel launches captured in the batch's step graph (per time step). */
gsw_status gsw_batch_launches(gsw_ctx *ctx, int32_t batch_id, int64_t *per_step);

/* Receiver velocity history: out [n_rec][3][n_steps] (entries of steps not
 * yet run are zero) of the model's own analysis (dir = -1) or of the
 * analysis of input direction dir = 0..2 run by gsw_run (GSW_E_STATE if it
 * has not been run). */
gsw_status gsw_read_waveforms(gsw_ctx *ctx, int32_t model_id, int32_t dir, double *out);
/* Receiver velocities of steps step0 .. step0+count-1 only:
 * out [n_rec][3][count] (host; pinned memory gives an asynchronous copy). */
gsw_status gsw_read_waveform_steps(gsw_ctx *ctx, int32_t model_id, int32_t step0, int32_t count,
                                   double *out);
/* Statistics of the model's own analysis (dir = -1) or of the analysis of
 * input direction dir = 0..2 run by gsw_run. */
gsw_status gsw_stats_get(gsw_ctx *ctx, int32_t model_id, int32_t dir, gsw_stats *out);

/* Checkpoint / restore of the time-stepping state: u, v, a [n_nodes][3] and
 * the step counter (receiver history up to that step is kept by the caller
 * via gsw_read_waveforms).  Host arrays. */
gsw_status gsw_get_state(gsw_ctx *ctx, int32_t model_id, double *u, double *v, double *a,
                         int64_t *step);
gsw_status gsw_set_state(gsw_ctx *ctx, int32_t model_id, const double *u, const double *v,
                         const double *a, int64_t step);

/* Full checkpoint of the model's own analysis, for resuming a run exactly:
 * u, v, a, the step counter and statistics, the receiver history, the
 * increment history of the extrapolated or projected initial guess and,
 * with the learned guess enabled, the network's parameters, its Adam moments
 * and step count, its increment history, its training schedule and the
 * referee's state.  buf is a
 * host buffer of *bytes bytes; buf = NULL returns the size needed in *bytes.
 * gsw_restore needs the same model sizes, n_steps, input direction and
 * guess_order (and learning enabled when the checkpoint holds a network);
 * otherwise GSW_E_INVALID / GSW_E_STATE and the model is unchanged. */
gsw_status gsw_checkpoint(gsw_ctx *ctx, int32_t model_id, void *buf, size_t *bytes);
gsw_status gsw_restore(gsw_ctx *ctx, int32_t model_id, const void *buf, size_t bytes);

/* Kernel timing: enable = 1 clears the counters and brackets every operator
 * launch of subsequent steps with CUDA events on the context's stream;
 * enable = 0 stops; any other value only reads.  ms[2] and launches[2]
 * (either may be NULL) receive the summed device time and the number of
 * timed launches of [0] the element-by-element A p product of the CG
 * iteration (FP64 or double-word, gsw_outer_op) and [1] the reduced-precision
 * element-by-element product of the inner preconditioner (mixed modes; an
 * inner solve that met inner_rtol returns at entry from its remaining
 * launches, which are not counted). */
gsw_status gsw_timing(gsw_ctx *ctx, int32_t model_id, int32_t enable, double *ms,
                      int64_t *launches);

/* Operator application on device vectors [n_nodes][3] (diagnostics, tests):
 *  which = 0: y = A x, A = K + (2/dt) C + (4/dt^2) M (the CG operator);
 *  which = 1: y = K x;  which = 2: y = M x;  which = 3: y = C x;
 *  which = 4: y = A x by the reduced-precision inner operator of the model's
 *  current mixed precision mode (x rounded to the inner storage type,
 *  FP32 arithmetic and accumulation); GSW_E_STATE in FP64 mode;
 *  which = 5: y = A x in double-word arithmetic (GSW_OUTER_DWORD);
 *  which = 6: y = P D_c^-1 P^T x, the coarse correction of the two-level inner
 *  preconditioner (FP32 arithmetic; GSW_E_STATE unless a mixed mode with
 *  coarse_weight > 0 is set).
 * x_dev, y_dev device pointers; y is overwritten. */
gsw_status gsw_apply(gsw_ctx *ctx, int32_t model_id, int32_t which, const double *x_dev,
                     double *y_dev);

/* Inverted 3x3 nodal diagonal blocks of A (the block-Jacobi preconditioner),
 * host out [n_nodes][6] symmetric entries (xx, yy, zz, xy, xz, yz). */
gsw_status gsw_read_preconditioner(gsw_ctx *ctx, int32_t model_id, double *out);

/* Receiver interpolation: nodes [n_rec][6] and weights [n_rec][6] of the
 * 6-node surface triangle containing each receiver. */
gsw_status gsw_read_receivers(gsw_ctx *ctx, int32_t model_id, int32_t *nodes, double *weights);

/* Failure-detection self-test (no counterpart in the paper).  Runs the bounded
 * mbarrier wait that guards the warp-specialised inner operator's pipeline
 * stages on a barrier that expects one arrival which never comes, with `limit`
 * attempts (1 .. 2^22; each attempt may suspend the thread for a short,
 * hardware-bounded time).  The wait must run out: the call returns
 * GSW_E_TIMEOUT, the status a solve whose wait ran out reports, and the context
 * stays usable.  GSW_OK would mean the wait completed without an arrival;
 * GSW_E_INVALID for a limit outside the range. */
gsw_status gsw_wait_probe(gsw_ctx *ctx, int64_t limit);

/* ---- learned initial guess ------------------------------------------------
 * A per-node MLP (16 -> 64 -> 64 -> 3, ReLU) corrects the step's base guess
 * (the Newmark predictor dt v + dt^2/2 a, or the guess_order extrapolation):
 * features = the backward differences D_0..D_3 of the last four displacement
 * increments (D_k = sum_j (-1)^j C(k, j) du_{s-1-j}), each divided by its RMS
 * over all DOF (12 values), and the node's layer properties (Vs/1000, Vp/3000,
 * rho/2000, h/0.05); du0 = base + sigma_e * MLP(features), sigma_e the RMS of
 * the previous step's correction du - base.  During the first train_steps
 * steps the CG starts from the base guess and, after each converged step, the
 * network takes iters_per_step Adam steps on a batch of random nodes (target:
 * (du - base) / RMS(du - base)); the training's products run on the tensor
 * cores (BF16 operands, FP32 accumulation), as does the inference that
 * supplies the initial guess afterwards.  The CG always iterates to the same
 * relative-residual tolerance; a non-finite guess falls back to the
 * predictor, and the plain base guess stays the referee (see gsw_mlp_state).
 * Host-driven stepping (gsw_step) only. */
typedef struct {
  int32_t enable;          /* 0: plain predictor; 1: learned guess */
  int32_t train_steps;     /* steps used for training (the guess is applied after them) */
  int32_t batch;           /* training samples per Adam step (<= 65536) */
  int32_t iters_per_step;  /* Adam steps after each training step */
  float lr;                /* Adam learning rate */
  uint32_t seed;           /* weight initialisation and node sampling */
} gsw_learn_opts;
gsw_status gsw_set_learning(gsw_ctx *ctx, int32_t model_id, const gsw_learn_opts *opts);
/* Train the learned guess on the model's next n_train_steps steps and advance
 * them (host-driven): each converged step's solution trains the network
 * (opts->iters_per_step Adam steps on opts->batch random nodes); afterwards
 * gsw_step applies the learned guess.  opts->train_steps is ignored (training
 * ends n_train_steps from the current step).  A network already enabled on
 * the model keeps training; otherwise it is initialised from opts->seed.
 * GSW_E_STATE in GSW_PREC_FP64 or for a batch member. */
gsw_status gsw_mlp_train(gsw_ctx *ctx, int32_t model_id, int32_t n_train_steps, const gsw_learn_opts *opts);
/* MLP parameters (5443 doubles: W1[16][64], b1[64], W2[64][64], b2[64],
 * W3[64][3], b3[3], row-major): read into get (if not NULL), then replace
 * from set (if not NULL). */
gsw_status gsw_mlp_params(gsw_ctx *ctx, int32_t model_id, double *get, const double *set);
/* Diagnostics: network outputs out[n][3] for explicit features x[n][16] with
 * the tensor-core inference kernel; loss and gradient grad[5443] of the mean
 * squared error against y[n][3] with the training kernels.  Host arrays. */
gsw_status gsw_mlp_forward(gsw_ctx *ctx, int32_t model_id, int32_t n, const float *x, float *out);
gsw_status gsw_mlp_grad(gsw_ctx *ctx, int32_t model_id, int32_t n, const float *x, const float *y,
                        double *loss, double *grad);
/* State of the learned guess, out[5]: [0] mean training loss of the last
 * training step, [1] 1 while the guess is applied (0 once the referee has
 * reverted to the predictor, or when disabled), [2] mean initial relative
 * residual of the plain predictor over its last (up to 5) steps, [3] the same
 * for the learned guess, [4] number of steps that used the learned guess.
 * After training, every 10th step is a probe with the plain predictor; the
 * referee reverts to the predictor for good when [3] (over 5 steps) exceeds [2]. */
gsw_status gsw_mlp_state(gsw_ctx *ctx, int32_t model_id, double *out);

/* Diagnostics of the learned guess's data path (tests), between steps of a
 * model with learning enabled.
 *  x_train [batch][16], y_train [batch][3] (either may be NULL): the last
 *    training batch -- features and targets of the last Adam step of the last
 *    training step.  Sample j of Adam step i of step s is node
 *    H(seed ^ H(s * 0x9E3779B9 ^ H(i * 0x85EBCA6B ^ j))) mod n_nodes, with H
 *    Wellons' "lowbias32" 32-bit hash and products modulo 2^32.
 *  nodes [n]: for these nodes, x [n][16] receives the features and base [n][3]
 *    the base guess (predictor, or the guess_order extrapolation) that the
 *    next step's inference would use.
 *  scale [2] (may be NULL): the RMS of the latest increment and the output
 *    scale of the next step's correction (the RMS of the last correction).
 * Host arrays.  GSW_E_STATE before the first converged step or without learning. */
gsw_status gsw_mlp_inputs(gsw_ctx *ctx, int32_t model_id, float *x_train, float *y_train, int32_t n,
                          const int32_t *nodes, float *x, double *base, double *scale);

/* ---- misfit (Section 2, Eq. (2)) ----------------------------------------- */

/* Input-wave estimate and ERR for one candidate model and one event, from
 * the model's device-resident Green's functions: the receiver histories of
 * its three input-direction analyses (gsw_run with dirs_mask 7, run to the
 * end since the last set-up; GSW_E_STATE otherwise), each driven by the unit
 * pulse p(t) of the basis.
 *  obs  [n_rec][3][n_steps] observed surface velocity (host).
 *  stride, n_shifts: pulse shifts l * stride steps, l = 0..n_shifts-1
 *       (3 * n_shifts <= 384).
 *  tau  relative eigenvalue cut of the truncated pseudo-inverse.
 * Outputs: *err (Eq. (2)) and c_out [3][n_shifts] (may be NULL), host.
 * Pairs (k, i) whose observed energy is below 1e-12 of the largest are
 * dropped from the weights and from n_obs.  Model selection is the caller's
 * argmin over the candidates' err (ties: lowest index). */
gsw_status gsw_misfit(gsw_ctx *ctx, int32_t model_id, const double *obs, int32_t stride, int32_t n_shifts,
                      double tau, double *err, double *c_out);

/* The same for Green's functions given by the caller (host arrays):
 *  G    [n_rec][3 (i)][3 (j)][n_t]: velocity in direction i at receiver k for
 *       the unit pulse input in direction j;
 *  obs  [n_rec][3][n_t]. */
gsw_status gsw_misfit_green(gsw_ctx *ctx, int32_t n_rec, int32_t n_t, const double *G,
                            const double *obs, int32_t stride, int32_t n_shifts, double tau,
                            double *err, double *c_out);

/* ---- misfit without device allocation ------------------------------------ */

/* Same computation as gsw_misfit_green, for callers that cannot allocate device
 * memory: for example code whose GPU memory is wholly owned by another
 * allocator (a framework's caching pool or a fixed arena reserved at start-up),
 * or a latency-critical loop where cudaMalloc / cudaFree would synchronise the
 * device.  This paper has no counterpart of this entry point; it is a service
 * of the library.
 *
 * All five array arguments are DEVICE pointers owned by the caller:
 *  G_dev   [n_rec][3][3][n_t] and obs_dev [n_rec][3][n_t] (inputs, as in
 *          gsw_misfit);
 *  err_dev one double (output, Eq. (2));
 *  c_dev   [3][n_shifts] doubles (output; may be NULL).
 * The call only launches kernels on the context's stream and returns without
 * waiting for them.  It calls no cudaMalloc / cudaFree and no allocating
 * library routine: its working memory is one fixed array of about 0.67 MB
 * (file-scope __device__ storage) that every GPU loading the library holds
 * until the process exits.  Limits: n_shifts <= 64 (3 * n_shifts <= 192
 * unknowns) and n_rec <= 1024; larger sizes return GSW_E_INVALID.
 * The first call on each device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call on a device shares the one array and leaves its
 * contents behind; the kernels overwrite every entry they read, so nothing is
 * cleared between calls.  Calls that overlap on the GPU (other streams or
 * other contexts on the same device) race on the array: serialise them. */
gsw_status gsw_misfit_noalloc(gsw_ctx *ctx, int32_t n_rec, int32_t n_t, const double *G_dev,
                              const double *obs_dev, int32_t stride, int32_t n_shifts,
                              double tau, double *err_dev, double *c_dev);

#ifdef __cplusplus
}
#endif
#endif /* GSW_H */
