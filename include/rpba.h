/*
 * rpba.h -- C ABI of the GB300 (sm_103a) implementation of the RPBA hot path:
 * covariance-weighted parallel bundle adjustment by sub-blocks (Mayer,
 * "RPBA - Robust Parallel Bundle Adjustment Based on Covariance Information").
 *
 * Problem statement (Sec. 2; Sec. 4, sub-block split): M cameras P_i (pose:
 * angle-axis omega and translation t, X_c = R(omega) X + t; fixed pinhole
 * intrinsics f, cx, cy), N 3D points X_j, K image observations x_k of point j
 * in camera i with 2x2 weight C_k^-1. Every camera belongs to exactly one
 * sub-block; a point observed from cameras of several sub-blocks is a tie
 * point (TP). The method alternates the adjustment of every sub-block with its
 * TPs as weighted control points (Eq. bact) and the intersection of the TPs
 * with all cameras fixed (Eq. bars), which yields the TP positions, their
 * covariances and the per-sub-block weights W^l (Sec. 5.1).
 *
 * Conventions for every call
 *   - All array arguments are HOST pointers owned by the caller; the library
 *     copies what it needs and never keeps a caller pointer past the call.
 *   - Row-major, tightly packed; indices are 0-based int32.
 *   - sym3 = 6 doubles (a00, a01, a02, a11, a12, a22).
 *   - Every call returns an rpba_status; on error the context keeps a message
 *     (rpba_last_error) and the state is left as it was before the failing
 *     kernel (device state may be partially updated after RPBA_ERR_CUDA).
 *   - The library owns all device memory (cudaMalloc, or the caller's
 *     allocator hook in rpba_options) and runs every kernel on the stream
 *     given at creation. Calls on one context must not overlap.
 *   - No CPU fallback: without a usable sm_103a device rpba_create fails with
 *     RPBA_ERR_CUDA.
 */
#ifndef RPBA_H
#define RPBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpba_ctx rpba_ctx;

typedef enum {
  RPBA_OK = 0,
  RPBA_ERR_INVALID_ARG = 1,   /* bad size, index out of range, NULL where required */
  RPBA_ERR_OOM = 2,           /* device allocation failed */
  RPBA_ERR_CUDA = 3,          /* a CUDA runtime error (message has the CUDA text) */
  RPBA_ERR_NOT_CONVERGED = 4, /* iteration cap reached (state is still valid) */
  RPBA_ERR_DEVICE_TIMEOUT = 5,/* a bounded device-side wait ran out */
  RPBA_ERR_NUMERIC = 6,       /* non-finite values where finite ones are required */
  RPBA_ERR_STATE = 7          /* call out of order (e.g. sub-block index >= L) */
} rpba_status;

/* Input block (Sec. 2). cam_pose n_cams x 6 (omega rad, t); cam_intr
 * n_cams x 3 (f, cx, cy); points n_points x 3; obs_cam/obs_point n_obs;
 * obs_xy n_obs x 2 pixels; obs_winv n_obs x 3 (w11, w12, w22) of C_k^-1 or
 * NULL for identity; cam_subblock n_cams (global sub-block ids 0..L-1, every
 * id used); cam_block n_cams or NULL: id of the independent block a camera
 * belongs to (only used for reporting; independent blocks are simply
 * sub-blocks that share no point). A point needs two observations to be
 * estimated; points with fewer stay inactive. */
typedef struct {
  int32_t n_cams, n_points, n_obs;
  const double *cam_pose;
  const double *cam_intr;
  const double *points;
  const int32_t *obs_cam;
  const int32_t *obs_point;
  const double *obs_xy;
  const double *obs_winv;
  const int32_t *cam_subblock;
  const int32_t *cam_block;
  const double *cam_k1;  /* n_cams initial radial parameters, read with options.intrinsics = 1
                            (NULL: 0) */
} rpba_problem;

/* solver 4 (auto) starts with block-Jacobi PCG for at most this many
 * sub-blocks (else the direct FP32 Cholesky with FP64 refinement), and moves
 * to the direct solver for good once a PCG solve needs more than this many
 * lock-step iterations (one iteration costs ~1/50 of a direct solve) */
#define RPBA_AUTO_PCG_MAX_SUBBLOCKS 64
#define RPBA_AUTO_PCG_MAX_ITER 48
#define RPBA_AUTO_PCG_MAX_ITER_FP32 80 /* precision 1: its CG steps cost about half as much */

/* Options; rpba_default_options fills the paper's values (Sec. 5.3, 5.5). */
typedef struct {
  double lambda0;        /* LM damping N + lambda diag(N), 1e-4 (Sec. 5.5) */
  double t_v;            /* robust threshold on sqrt(v^T C^-1 v)/sigma_cam, 4 (Sec. 5.3) */
  double downweight;     /* weight of a detected outlier, 1e-4 (Sec. 5.3) */
  double stop_ratio;     /* best/current ratio that ends a loop, 1.01 (Sec. 5.5) */
  int32_t grace;         /* iterations allowed below the ratio, 1 (Sec. 5.5) */
  int32_t max_outer;     /* cap on bact/bars iterations, 30 */
  int32_t max_inner;     /* cap on LM iterations per sub-block per bact, 20 */
  int32_t max_reject;    /* rejected LM steps in a row that end a bact, 6 */
  int32_t robust;        /* 1: robust stage (Sec. 5.3, parallel variant) */
  int32_t robust_from_start; /* 1: robust weights from the first intersection on */
  int32_t weight_mode;   /* the TPs' weight W^l in the other sub-blocks: 0 the refined weight of
                            Sec. 5.1 (the point's normal matrix without sub-block l), 1 the
                            normal matrix of all cameras, 2 a scalar rho I with rho = rho0 at
                            the first intersection, times 1.01 per outer iteration (the
                            ablation variants of Sec. 6.4) */
  double rho0;           /* weight_mode 2: the first rho, 200 (Sec. 6.3, simulated data) */
  int32_t robust_serial; /* end of the robust stage: 0 the parallel variant (eliminate every
                            point with a down-weighted observation), 1 the serial variant of
                            Sec. 5.3 (delete the down-weighted observations: weight 0, then
                            eliminate points left with fewer than two; use with t_v = 3) */
  int32_t isect_max_iter;/* Gauss-Newton iterations of the intersection, 10 */
  double isect_tol;      /* ||dX|| <= tol (1 + ||X||) ends it, 1e-10 */
  double isect_px_tol;   /* ... or a step that moves the image residuals by less than this per
                            observation (dX^T N dX <= px_tol^2 n_obs), 1e-3 px */
  double cond_max;       /* Frobenius condition number that drops a point, 1e12 */
  int32_t precision;     /* 0: all FP64 ("plain"); 1: FP32 bulk (float-float residuals for
                            the cost, sigma_0 and robust tests), FP64 reductions */
  int32_t solver;        /* RCS solve: 0 FP64 Cholesky; 1 PCG with block-Jacobi
                            preconditioning (Sec. 5.5) to pcg_tol (FP64 vectors; with
                            precision 1, for sub-blocks of up to 2048 unknowns, FP32 CG
                            stages on S rounded to FP32, each refined by the float-float
                            residual y - S x, FP64 above); 2 FP32 Cholesky of the
                            Jacobi-scaled RCS with FP64 iterative refinement; 3 FP64 PCG
                            with the learned preconditioner (rpba_set_gnn_weights),
                            block-Jacobi PCG again for a sub-block it leaves above pcg_tol;
                            4 auto: 1 for at most RPBA_AUTO_PCG_MAX_SUBBLOCKS sub-blocks,
                            else 2; 1 becomes 2 after a solve of more than
                            RPBA_AUTO_PCG_MAX_ITER iterations (RPBA_AUTO_PCG_MAX_ITER_FP32
                            with precision 1) (rpba_get_options) */
  double pcg_tol;        /* relative residual of the PCG solve, 1e-8 */
  int32_t pcg_max_iter;  /* PCG iteration cap, 500 */
  int32_t ir_steps;      /* refinement passes of solver 2 after the first solve, 2 */
  int32_t chol_tc;       /* solver 2's FP32 factorisation: 0 (default) right-looking on the
                            CUDA cores; left-looking with its updates on the tensor cores
                            (tcgen05.mma kind::tf32, each factor entry split into three TF32
                            pieces, six products: FP32 accuracy), operands staged by TMA, as
                            2 one persistent launch over every step of every sub-block or 1
                            one launch per step. Same results to rounding; rpba_tune picks
                            the fastest for a workload */
  int32_t intrinsics;    /* 1: per-camera intrinsics as in the Final data sets of Sec. 6: the
                            focal length f (cam_intr[0]) and the first radial parameter k1
                            (cam_k1) of every camera are estimated with its pose, 8 unknowns
                            per camera; the projection applies 1 + k1 |p|^2 to the normalised
                            coordinates p = (x_c, y_c)/z_c; the principal point stays fixed.
                            Solvers 0, 1, 2 and 4; 3 (the learned preconditioner, built on
                            6 x 6 camera blocks) gives INVALID_ARG.
                            0 (default): intrinsics known, pinhole, 6 unknowns per camera */
  const char *tune_cache; /* NULL, or a file of tuned launch shapes (JSON lines, one object per
                            workload: cameras, points, observations, sub-blocks, precision,
                            solver and SM count): the entry of this workload, if any, is
                            applied at create; rpba_tune writes it (the string is copied) */
  /* optional device allocator (NULL: cudaMalloc / cudaFree) */
  void *(*dev_alloc)(size_t bytes, void *user);
  void (*dev_free)(void *ptr, void *user);
  void *alloc_user;
} rpba_options;

typedef struct {
  double sigma0;          /* final sigma_0 (Eq. sigma0, weights C^-1) */
  double rms;             /* RMS image residual [px] over active, not down-weighted obs */
  double sigma0_initial;  /* sigma_0 after the initial intersection */
  int32_t outer;          /* bact/bars iterations done */
  int32_t inner_total;    /* LM iterations summed over sub-blocks */
  int32_t lm_launches;    /* lock-step LM iterations (all sub-blocks together) */
  int32_t deleted_points; /* points eliminated or dropped since creation */
  int32_t active_points;
  int32_t active_obs;
  int32_t robust_started_at; /* outer iteration where the robust stage began, -1 never */
  double sigma0_hist[128];
} rpba_report;

void rpba_default_options(rpba_options *opt);

/* Creates a context: validates and copies the block to the device, builds the
 * sub-block topology (point instances, CSR orders by instance and by camera,
 * RCS layout). `cuda_stream` is a cudaStream_t (NULL = default stream).
 * Errors: INVALID_ARG (sizes, ids out of range, a duplicate (camera, point)
 * observation), OOM, CUDA. */
rpba_status rpba_create(const rpba_problem *prob, const rpba_options *opt, void *cuda_stream,
                        rpba_ctx **out);
void rpba_destroy(rpba_ctx *ctx);
const char *rpba_last_error(const rpba_ctx *ctx);

/* Intersection of every active point with all cameras fixed (Eq. bars, the
 * start values for the first bact): Gauss-Newton on X_j, then W^l_j = N_j -
 * N_j^(l) for every instance (Sec. 5.1). Points that do not converge are
 * dropped (Sec. 5.5). Runs in FP64 whatever options.precision says: it runs
 * once, from the raw input, and both forms start from the same point set. */
rpba_status rpba_intersect(rpba_ctx *ctx);

/* The RPBA iteration (Sec. 5): up to max_outer (<= 0: options.max_outer)
 * alternations of the LM adjustment of every sub-block (Eq. bact; all
 * sub-blocks advance together, one launch per step) and the TP intersection
 * (Eq. bars), with the robust stage of Sec. 5.3 when enabled. Runs
 * rpba_intersect first if it has not been run. `report` may be NULL. */
rpba_status rpba_iterate(rpba_ctx *ctx, int32_t max_outer, rpba_report *report);

/* Autotuner: times candidate launch shapes on the context's own data with
 * CUDA events (5 runs each after one untimed run) and keeps the fastest: the
 * CTA sizes of the intersection (64/128/256 points), the linearisation and the
 * back-substitution (64/128/256 instances) and the robust weights (128/256/512
 * observations), and, for the direct solver, the tensor-core factorisation's
 * launch form (chol_tc 1 or 2). These kernels give every thread one
 * independent item, so the choice changes timing, not results. The state is
 * unchanged (the intersection's timing restores it). With cache_path (or the
 * context's tune_cache when NULL) the choice is written there for the
 * workload. chosen (nullable, 5 values): isect, lin, backsub, robust,
 * chol_tc. Not a step of the paper's method. Errors: INVALID_ARG for an
 * unwritable cache, CUDA. */
rpba_status rpba_tune(rpba_ctx *ctx, const char *cache_path, int32_t *chosen);

/* One outer iteration of the RPBA loop (Sec. 5) in steady state: the LM
 * adjustment of every sub-block (Eq. bact, up to options.max_inner lock-step
 * LM iterations), the exchange of cameras and single-sub-block points, the
 * robust weights from the per-camera scale when `robust` is nonzero (Sec.
 * 5.3), the intersection of the tie points with their refined weights (Eq.
 * bars, Sec. 5.1) and sigma_0 (Eq. sigma0). Unlike rpba_iterate it evaluates
 * no start or final sigma_0, applies no stop rule and eliminates no point: the
 * caller owns the loop. Runs rpba_intersect first if it has not been run.
 * Outputs (nullable): sigma0 after the iteration, lm_launches = lock-step LM
 * iterations it ran. Errors: NOT_CONVERGED if the LM loop does not end,
 * CUDA. */
rpba_status rpba_outer_iteration(rpba_ctx *ctx, int32_t robust, double *sigma0, int32_t *lm_launches);

/* Sharded runs (the sub-blocks of one block spread over processes, each with
 * its own context holding the whole block; Sec. 5's exchange between them).
 * rpba_set_subblock_mask: the LM adjustment of rpba_bact, rpba_iterate and
 * rpba_outer_iteration moves only the sub-blocks l with mask[l] != 0
 * (n_subblocks bytes, host, read during the call; NULL restores all, the
 * default). rpba_set_point_mask: the intersections (rpba_intersect_points
 * and those inside the iteration) handle only the points j with mask[j] != 0
 * (n_points bytes in the caller's numbering; NULL: all). Both persist until
 * changed. Errors: CUDA. */
rpba_status rpba_set_subblock_mask(rpba_ctx *ctx, const uint8_t *mask);
rpba_status rpba_set_point_mask(rpba_ctx *ctx, const uint8_t *mask);

/* C_j = N_j^-1 of the listed points at the current state (Eq. bars), out is
 * n x 9 row-major; inactive points give NaN. */
rpba_status rpba_covariance(rpba_ctx *ctx, const int32_t *point_ids, int32_t n, double *out9);

rpba_status rpba_get_cameras(rpba_ctx *ctx, double *pose /* n_cams x 6 */);
rpba_status rpba_get_points(rpba_ctx *ctx, double *X /* n_points x 3 */, uint8_t *active /* nullable */);

/* ---- state access and single steps (used by the parity tests) ---------- */

rpba_status rpba_info(rpba_ctx *ctx, int32_t *n_subblocks, int32_t *n_instances);
/* the context's options, with solver 4 (auto) resolved to the solver the next
 * LM step uses */
rpba_status rpba_get_options(rpba_ctx *ctx, rpba_options *out);
/* cameras of sub-block l in RCS row order (ascending global id); n_out = count */
rpba_status rpba_sub_cameras(rpba_ctx *ctx, int32_t l, int32_t *cams, int32_t *n_out);
rpba_status rpba_set_cameras(rpba_ctx *ctx, const double *pose);
/* the camera state as held, without the angle-axis conversion: R (n_cams x 9,
 * row-major, X_c = R X + t) and t (n_cams x 3), host buffers. A sharded run's
 * exchange moves cameras through these, bit for bit. Errors: INVALID_ARG for
 * a NULL buffer, CUDA. */
rpba_status rpba_get_camera_rt(rpba_ctx *ctx, double *R, double *t);
rpba_status rpba_set_camera_rt(rpba_ctx *ctx, const double *R, const double *t);
rpba_status rpba_set_points(rpba_ctx *ctx, const double *X, const uint8_t *active /* nullable */);
/* per-camera intrinsics (options.intrinsics = 1): fk is n_cams x 2, the focal
 * length and the radial parameter k1 of every camera (Sec. 6, Final data
 * sets), host buffer. Without intrinsics get returns (f, 0) and set accepts
 * only (f, 0) with the creation's f: anything else gives INVALID_ARG. */
rpba_status rpba_get_intrinsics(rpba_ctx *ctx, double *fk);
rpba_status rpba_set_intrinsics(rpba_ctx *ctx, const double *fk);
/* instances sorted by (sub-block, point): point id, sub-block id, X^l (P x 3),
 * W^l (P x 6 sym3); any output may be NULL */
rpba_status rpba_get_instances(rpba_ctx *ctx, int32_t *inst_point, int32_t *inst_sub, double *Xl,
                               double *Wl);
rpba_status rpba_set_instances(rpba_ctx *ctx, const double *Xl, const double *Wl);
/* robust weights w_k, in the caller's observation order */
rpba_status rpba_get_weights(rpba_ctx *ctx, double *w);
rpba_status rpba_set_weights(rpba_ctx *ctx, const double *w);
/* v_k = g_k(P_i, X_j) - x_k at the global state (Sec. 2), n_obs x 2 */
rpba_status rpba_residuals(rpba_ctx *ctx, double *v);
/* Jc (n_obs x 2 x 6, d/d(dw, dt), dw left-multiplied; n_obs x 2 x 8 with
 * intrinsics, d/d(dw, dt, df, dk1)) and Jx (n_obs x 2 x 3) (Eq. ta) */
rpba_status rpba_jacobians(rpba_ctx *ctx, double *Jc, double *Jx);
/* sigma_0 (Eq. sigma0) and RMS at the global state */
rpba_status rpba_sigma0(rpba_ctx *ctx, double *sigma0, double *rms);
/* per-camera 1.4826 * MAD of the whitened residual components (Sec. 5.3) */
rpba_status rpba_camera_scale(rpba_ctx *ctx, double *sigma /* n_cams */);
/* robust weights from that scale; n_down = number down-weighted (Sec. 5.3) */
rpba_status rpba_robust_weights(rpba_ctx *ctx, int32_t *n_down);
/* intersection of all active points (tp_only = 0) or of the TPs only */
rpba_status rpba_intersect_points(rpba_ctx *ctx, int32_t tp_only, int32_t *n_dropped);
/* F_l of every sub-block at the current state (Eq. bact), n_subblocks values */
rpba_status rpba_sub_costs(rpba_ctx *ctx, double *F);
/* damped RCS of sub-block l (Sec. 2, 5.5): S (n x n, symmetric, row-major;
 * n = 6 x cameras of l, 8 x with intrinsics) and y (n), at the current state */
rpba_status rpba_rcs(rpba_ctx *ctx, int32_t l, double lambda, double *S, double *y);
/* one LM step of every sub-block with damping lambda: solve, trial, accept
 * if F_l decreases. Outputs per sub-block (nullable): accepted (1/0/-1 solve
 * failed), F before, F of the trial; dc = camera updates in RCS order of all
 * sub-blocks concatenated (6 x n_cams, 8 x with intrinsics), dx = instance
 * updates (P x 3). */
rpba_status rpba_lm_step(rpba_ctx *ctx, double lambda, int32_t *accepted, double *F_before,
                         double *F_trial, double *dc, double *dx);
/* the LM adjustment of every sub-block to its own stop (Eq. bact, with the
 * damping and stop rules of Sec. 5.5) from the current state, the tie points
 * held by their current X_TP and W^l: all sub-blocks advance in lock step,
 * each with its own lambda. iters (nullable, n_subblocks) receives each
 * sub-block's LM iterations. This is the first stage of every outer
 * iteration of rpba_iterate. Errors: NOT_CONVERGED if the loop does not end,
 * CUDA. */
rpba_status rpba_bact(rpba_ctx *ctx, int32_t *iters);

/* PCG solvers (solver = 1, 3, or 4 while or after it used PCG): iterations
 * and final relative residual ||r|| / ||y|| of every sub-block in the last PCG
 * pass (n_subblocks values each, nullable; with precision 1 the CG steps of
 * all refinement stages and the float-float residual of the returned
 * solution). Errors: STATE when the context has no PCG state. */
rpba_status rpba_solver_stats(rpba_ctx *ctx, int32_t *iters, double *relres);
/* precision 1 with block-Jacobi PCG: the refinement stages of every
 * sub-block in the last solve (n_subblocks values; each stage is one FP32 CG
 * run and one float-float product S x); zeros for the other solvers and
 * forms. Errors: INVALID_ARG for a NULL stages. */
rpba_status rpba_solver_stages(rpba_ctx *ctx, int32_t *stages);
/* solver 3: number of sub-block solves, since create, that the learned
 * preconditioner left above pcg_tol and block-Jacobi PCG solved again */
rpba_status rpba_solver_fallbacks(rpba_ctx *ctx, int64_t *n);

/* ---- learned preconditioner (solver 3) ------------------------------------
 * The paper preconditions CG on the RCS with the inverses of the 6x6 camera
 * blocks S_ii (block-Jacobi, Sec. 5.5). A graph network over the cameras of a
 * sub-block (edge i-j where S_ij != 0, i.e. the cameras share a point)
 * predicts a correction of every camera block and a gain for every camera
 * pair; the paper has no such network.
 *   features x_i (21): log S_ii[k,k] minus its mean over the sub-block (6),
 *     S_ii[k,l] / sqrt(S_ii[k,k] S_ii[l,l]) for k > l, row by row (15)
 *   edge weight e_ij = ||S_ij||_F / sqrt(||S_ii||_F ||S_jj||_F)
 *   h0 = relu(W0 x + b0); h_t = relu(A_t h_{t-1} + B_t sum_j e_ij h_{t-1,j} + c_t),
 *   t = 1..3 (width 64); C_i = Wo h3_i + bo (21 entries of a lower-triangular
 *   6x6, row by row); q_ij = ws.(h3_i + h3_j) + wp.(h3_i * h3_j) + we e_ij + bq
 *   M_i = I + 0.5 tanh(C_i), L_i = chol(S_ii), N_ij = tanh(q_ij) L_i^-1 S_ij L_j^-T
 *   (i > j in the sub-block's camera order), G = M^-1 (I - N) L^-1,
 *   P^-1 = G^T G: SPD, and block-Jacobi when both output heads are zero.
 * Parameters: one FP32 vector of rpba_gnn_param_count() values in the order
 * W0 (64x21), b0, then for t = 1..3 A_t (64x64), B_t (64x64), c_t, then Wo
 * (21x64), bo, ws (64), wp (64), we, bq; matrices row-major. The matrices
 * W0, A_t, B_t, Wo are applied in BF16, activations accumulate in FP32; the
 * factor G is formed in FP64 and applied in FP32; PCG vectors are FP64. */
#define RPBA_GNN_FEATURES 21
#define RPBA_GNN_HIDDEN 64
#define RPBA_GNN_LAYERS 3
int32_t rpba_gnn_param_count(void);
/* copies the parameters (host, rpba_gnn_param_count() floats) into a context
 * created with solver = 3. Errors: INVALID_ARG (count), STATE (other solver). */
rpba_status rpba_set_gnn_weights(rpba_ctx *ctx, const float *w, int32_t n);

/* Trainer: a network, a dataset of systems and Adam, on the current device.
 * Loss: the mean over the systems of Kaporin's condition number of
 * A = G S G^T per unit of dimension d, less its constant log det S / d:
 *   log(T / d) + (2 / d) sum_i log det(M_i L_i),  T = (1/n_p) sum_p v_p^T S v_p,
 *   v_p = G^T z_p, with the system's Gaussian probe vectors z_p (T estimates
 *   tr A). Block-Jacobi minimises it among block-diagonal preconditioners. */
typedef struct rpba_gnn rpba_gnn;
/* He-normal hidden layers from `seed` (splitmix64, Box-Muller), zero output
 * layer: the new network is block-Jacobi. */
rpba_status rpba_gnn_create(uint64_t seed, rpba_gnn **out);
void rpba_gnn_destroy(rpba_gnn *g);
const char *rpba_gnn_last_error(const rpba_gnn *g);
rpba_status rpba_gnn_get_weights(rpba_gnn *g, float *w);
/* also resets the Adam moments */
rpba_status rpba_gnn_set_weights(rpba_gnn *g, const float *w);
/* adds one system: S (HOST, n_cams*6 rows of leading dimension ld >= 6 n_cams,
 * row-major; only the lower triangle is read), z (HOST, n_probes x 6 n_cams).
 * Every system of a dataset has the same n_probes. Errors: INVALID_ARG,
 * NUMERIC when a diagonal camera block is not positive definite. */
rpba_status rpba_gnn_add_system(rpba_gnn *g, int32_t n_cams, const double *S, int32_t ld, int32_t n_probes,
                                const double *z);
/* adds the damped RCS (damping lambda) of every sub-block of a context at its
 * current state, with n_probes probes drawn from `seed`. The context must be
 * on the trainer's device. */
rpba_status rpba_gnn_add_rcs(rpba_gnn *g, rpba_ctx *ctx, double lambda, int32_t n_probes, uint64_t seed);
rpba_status rpba_gnn_dataset_size(rpba_gnn *g, int32_t *n_nodes, int32_t *n_edges, int32_t *n_systems);
/* the dataset's graph: x n_nodes x 21, ptr n_nodes + 1, adj and e n_edges
 * (nodes of all systems numbered consecutively); HOST, nullable */
rpba_status rpba_gnn_graph(rpba_gnn *g, float *x, int32_t *ptr, int32_t *adj, float *e);
/* z = P^-1 r for every dataset system at the current weights (HOST, r and z
 * n_nodes x 6: the systems' vectors one after another) */
rpba_status rpba_gnn_precondition(rpba_gnn *g, const double *r, double *z);
/* loss and its gradient (HOST, rpba_gnn_param_count() floats, nullable) */
rpba_status rpba_gnn_loss_grad(rpba_gnn *g, double *loss, float *grad);
/* `steps` Adam steps (beta 0.9, 0.999, eps 1e-8) with learning rate lr over
 * the whole dataset; loss_hist (nullable, steps values) the loss before each.
 * probe_seed != 0 draws new probe vectors before every step (splitmix64 of
 * (probe_seed, Adam step, element), Box-Muller), so that the network cannot
 * fit a fixed set of probes; 0 keeps the dataset's probes. */
rpba_status rpba_gnn_train(rpba_gnn *g, int32_t steps, float lr, uint64_t probe_seed, double *loss_hist);

/* ---- measurement ------------------------------------------------------- */

/* Resets the per-kernel counters; enable != 0 also times every kernel launch
 * with a pair of CUDA events on the context stream (adds two event records
 * per launch; leave it off outside measurements). */
rpba_status rpba_profile_enable(rpba_ctx *ctx, int32_t enable);
/* While profiling is enabled, time only the launches of the kernel named
 * `kernel` (NULL or "": all kernels); every launch is still counted. Timing
 * one kernel keeps the event records out of the rest of the step. */
rpba_status rpba_profile_select(rpba_ctx *ctx, const char *kernel);
/* Kernel launches since the last rpba_profile_enable, per kernel name (names:
 * max_kernels slots of 48 chars), their summed event time in ms (0 when
 * timing was off), the number of distinct kernels and of launches. */
rpba_status rpba_profile_read(rpba_ctx *ctx, int32_t max_kernels, char *names, double *ms,
                              int64_t *launches, int32_t *n_kernels, int64_t *total_launches);

/* ---- format checks (tests) ----------------------------------------------- */

/* Runs the FP32 form's format changes on the device (default stream) over n
 * host values: x[e] split into hi[e] + lo[e] (hi: x truncated to 24
 * significant bits, lo: the remaining bits rounded to float; values below
 * 2^-74 or at or above 2^128 in magnitude take the FP64 conversion, zeros
 * give 0 + 0), back[e] = hi[e] + lo[e] summed in FP64, and f[e] widened to
 * double (fd[e]; subnormal floats give a signed zero). x and f are read
 * when their outputs are asked for; every output may be NULL. Allocates and
 * frees its own device buffers. Errors: INVALID_ARG (n < 0, or an output
 * without its input), OOM, CUDA. */
rpba_status rpba_check_formats(const double *x, const float *f, int32_t n, float *hi, float *lo, double *back,
                               double *fd);

/* ---- sub-block construction ----------------------------------------------- */

/* Sub-blocks from the visibility graph (Sec. 5.2): the cameras are split into
 * n_parts parts by recursive bisection of the graph whose nodes are the
 * cameras and whose edges join cameras that observe a common point (weight:
 * the number of such points), each camera weighted by the cube root of the sum,
 * over the points it sees, of their observation counts; every bisection
 * balances the weight (each side within 2 % of its share) and keeps the cut
 * weight small (greedy
 * graph growing, then Fiduccia-Mattheyses passes). The paper uses METIS here;
 * this partitioner is the library's own. Host computation, no GPU.
 *   obs_cam / obs_point: n_obs observations (host), as in rpba_problem.
 *   cam_subblock: n_cams outputs in [0, n_parts), usable as
 *   rpba_problem.cam_subblock. node_weight (nullable, n_cams): the weights
 *   used. edge_cut (nullable): the total weight of the edges between parts.
 * Deterministic for the same input. Errors: INVALID_ARG for sizes out of range
 * (1 <= n_parts <= n_cams) or an index outside the cameras or points. */
rpba_status rpba_partition(int32_t n_cams, int32_t n_points, int32_t n_obs, const int32_t *obs_cam,
                           const int32_t *obs_point, int32_t n_parts, int32_t *cam_subblock,
                           double *node_weight, double *edge_cut);

/* ---- a variant that allocates no device memory --------------------------- */

/* Largest block rpba_sigma0_noalloc accepts (its fixed scratch: 8192 partial
 * sums of observations and 8192 of points, about 330 KB on every device that
 * loads the library, held until the process exits). */
#define RPBA_NOALLOC_MAX_OBS (8192 * 256)
#define RPBA_NOALLOC_MAX_POINTS (8192 * 256)

/* sigma_0 and RMS as rpba_sigma0 computes them (sigma_0 squared: the sum of
 * w v^T C^-1 v over the observations of active points, divided by
 * 2 K - 6 M - 3 N + 7 with K active observations, M cameras and N active
 * points; RMS: the root mean square of the residual components over the
 * observations with w == 1), for a block given entirely in caller-owned DEVICE
 * memory, without allocating any device memory. The paper has no counterpart
 * to this entry point; it exists for callers that cannot allocate device
 * memory per call (a fixed device-memory budget, an allocator owned by another
 * framework).
 *   R n_cams x 9 (row-major rotation, X_c = R X + t), t n_cams x 3, intr
 *   n_cams x 3 (f, cx, cy), X n_points x 3, active n_points (NULL: all),
 *   obs_cam / obs_point n_obs, obs_xy n_obs x 2, obs_winv n_obs x 3 (NULL:
 *   identity), obs_w n_obs (NULL: 1). All on the current device.
 * Outputs (HOST, nullable): sums5 = {sum w v^T C^-1 v, active observations,
 * sum |v|^2 (w == 1), observations with w == 1, active points}, sigma0, rms.
 * Runs on `cuda_stream` and synchronizes it before returning.
 * Scratch: one file-scope device array shared by every call; its device
 * address is looked up on the first call on each device (make that first call
 * before any stream capture). Calls that overlap on the GPU race on it.
 * Errors: INVALID_ARG for negative sizes, sizes above the limits, missing
 * arrays, or observations without any camera or point; CUDA for a failed
 * launch or copy. */
rpba_status rpba_sigma0_noalloc(int32_t n_cams, int32_t n_points, int32_t n_obs, const double *R,
                                const double *t, const double *intr, const double *X,
                                const uint8_t *active, const int32_t *obs_cam,
                                const int32_t *obs_point, const double *obs_xy,
                                const double *obs_winv, const double *obs_w, void *cuda_stream,
                                double *sums5, double *sigma0, double *rms);

#ifdef __cplusplus
}
#endif
#endif
