// rpba_internal.cuh -- device data layout and shared device helpers of the
// GB300 RPBA library. Everything here is GPU-side code of the library; the
// CPU oracle used by the tests is separate and shares nothing with it.
//
// Data layout in HBM (all arrays device-resident for the life of a context):
//   cameras (M):   R (9 f64), t (3 f64), intrinsics (3 f64), trial R/t,
//                  sub-block id, position inside the sub-block (RCS row / 6)
//   points (N):    X (3 f64), active flag (u8), CSR point -> instances;
//                  numbered internally by (sub-block of the first camera,
//                  first camera, caller's id), translated at the boundary
//   instances (P): sorted by (sub-block l, point j); X^l (3 f64), trial X^l,
//                  W^l (sym3 f64), damped inverse point block Ninv (sym3),
//                  point gradient gX (3), TP flag = point has >= 2 instances
//   observations (K): sorted by instance (so every instance and every
//                  sub-block is a contiguous segment), structure of arrays:
//                  cam (i32), inst (i32), xy (2 f64), C^-1 (3 f64), robust
//                  weight w (f64), user index (i32); FP64 form: per-LM-step
//                  N_XC (3x6) and Z = Ninv N_XC (3x6)
//   FP32 form:     camera records (R, C, f as hi + lo, t; 128 B each) of the
//                  current and trial state, X, X^l and trial X^l as hi + lo
//                  words, observations relative to the principal point as
//                  hi + lo, C^-1, w and W^l in FP32
//   camera order:  CSR camera -> observation positions (gather list)
//   Schur pairs:   (a, b) observation positions of one instance whose cameras
//                  differ, local(cam a) > local(cam b): lower-triangle blocks;
//                  FP32 form: sorted by (camera of a, camera of b, a) with
//                  their instance and camera-pair segment
//   RCS:           per sub-block a dense n_pad x n_pad f64 matrix (row-major,
//                  n_pad = 32 * ceil(6 M_l / 32), padding = identity), rhs;
//                  inverted 32 x 32 diagonal tiles of the factor; for the
//                  mixed solver an FP32 copy of the scaled RCS and FP64
//                  refinement vectors
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/rpba.h"
#include "ffloat.cuh"

#define RPBA_TILE 32

namespace rpba {

// ---------------------------------------------------------------------------
// small device math (sym3 = a00 a01 a02 a11 a12 a22)
// ---------------------------------------------------------------------------
__host__ __device__ inline int s3idx(int r, int c) {
  return (r == c) ? (r == 0 ? 0 : (r == 1 ? 3 : 5)) : (r + c == 1 ? 1 : (r + c == 2 ? 2 : 4));
}

template <typename T>
__device__ inline T sym3_inv(const T a[6], T inv[6]) {
  T c00 = a[3] * a[5] - a[4] * a[4];
  T c01 = a[2] * a[4] - a[1] * a[5];
  T c02 = a[1] * a[4] - a[2] * a[3];
  T c11 = a[0] * a[5] - a[2] * a[2];
  T c12 = a[1] * a[2] - a[0] * a[4];
  T c22 = a[0] * a[3] - a[1] * a[1];
  T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  T id = T(1) / det;
  inv[0] = c00 * id; inv[1] = c01 * id; inv[2] = c02 * id;
  inv[3] = c11 * id; inv[4] = c12 * id; inv[5] = c22 * id;
  return det;
}

template <typename T>
__device__ inline T sym3_frob(const T a[6]) {
  return sqrt(a[0] * a[0] + a[3] * a[3] + a[5] * a[5] + T(2) * (a[1] * a[1] + a[2] * a[2] + a[4] * a[4]));
}

// R = exp([w]x), Rodrigues formula with a series for small angles
__device__ inline void rodrigues(const double w[3], double R[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (th2 < 1e-8) {
    a = 1.0 - th2 * (1.0 / 6.0) + th2 * th2 * (1.0 / 120.0);
    b = 0.5 - th2 * (1.0 / 24.0) + th2 * th2 * (1.0 / 720.0);
  } else {
    double th = sqrt(th2);
    double s, c;
    sincos(th, &s, &c);
    a = s / th;
    b = (1.0 - c) / th2;
  }
  // R = I + a K + b K^2, K = [w]x, K^2 = w w^T - th2 I
  R[0] = 1.0 + b * (w[0] * w[0] - th2);
  R[4] = 1.0 + b * (w[1] * w[1] - th2);
  R[8] = 1.0 + b * (w[2] * w[2] - th2);
  R[1] = -a * w[2] + b * w[0] * w[1];
  R[3] = a * w[2] + b * w[0] * w[1];
  R[2] = a * w[1] + b * w[0] * w[2];
  R[6] = -a * w[1] + b * w[0] * w[2];
  R[5] = -a * w[0] + b * w[1] * w[2];
  R[7] = a * w[0] + b * w[1] * w[2];
}

// Projection g_k (Sec. 2) of a camera-frame point Xc and its Jacobians.
// RX = R X (camera frame before the translation) enters the rotation part:
// d Xc / d dw = -[R X]x for R' = exp([dw]x) R; d Xc / dt = I; d Xc / dX = R.
// CD = 6: pinhole, camera unknowns (dw, dt). CD = 8: per-camera intrinsics
// (the Final data sets of Sec. 6), the first radial parameter on the
// normalised coordinates p = (x_c, y_c)/z_c, (u, v) = f (1 + k1 |p|^2) p +
// (cx, cy), camera unknowns (dw, dt, df, dk1). Jc is 2 x CD row-major.
template <typename T, int CD = 6>
struct ProjJac {
  T u, v;          // projection
  T Jc[2 * CD];    // 2 x CD
  T Jx[6];         // 2 x 3
};

template <typename T, int CD = 6>
__device__ inline void project_jac(const T R[9], const T Xc[3], const T RX[3], T f, T k1, T cx, T cy,
                                   ProjJac<T, CD> &o) {
  T iz = T(1) / Xc[2];
  T px = Xc[0] * iz, py = Xc[1] * iz;
  T a0 = RX[0], a1 = RX[1], a2 = RX[2];
  if constexpr (CD == 6) {
    T fx = f * iz;
    o.u = fx * Xc[0] + cx;
    o.v = fx * Xc[1] + cy;
    // P = d(u,v)/dXc = fx [[1, 0, -px], [0, 1, -py]]
    // Jx = P R
    for (int c = 0; c < 3; c++) {
      o.Jx[c] = fx * (R[c] - px * R[6 + c]);
      o.Jx[3 + c] = fx * (R[3 + c] - py * R[6 + c]);
    }
    // rotation part: P * (-[RX]x); -[a]x = [[0, a2, -a1], [-a2, 0, a0], [a1, -a0, 0]]
    o.Jc[0] = fx * (0 - px * a1);
    o.Jc[1] = fx * (a2 + px * a0);
    o.Jc[2] = fx * (-a1);
    o.Jc[6] = fx * (-a2 - py * a1);
    o.Jc[7] = fx * (py * a0);
    o.Jc[8] = fx * (a0);
    // translation part: P
    o.Jc[3] = fx; o.Jc[4] = 0; o.Jc[5] = -fx * px;
    o.Jc[9] = 0; o.Jc[10] = fx; o.Jc[11] = -fx * py;
  } else {
    T r2 = px * px + py * py;
    T d = T(1) + k1 * r2;
    T fd = f * d;
    o.u = fd * px + cx;
    o.v = fd * py + cy;
    // d(u,v)/dp = f (d I + 2 k1 p p^T) = [[D00, D01], [D01, D11]]
    T a = T(2) * k1 * f;
    T D00 = fd + a * px * px, D01 = a * px * py, D11 = fd + a * py * py;
    // P = d(u,v)/dXc = D (1/z) [[1, 0, -px], [0, 1, -py]]
    T P[6] = {iz * D00, iz * D01, -iz * (D00 * px + D01 * py),
              iz * D01, iz * D11, -iz * (D01 * px + D11 * py)};
    for (int r = 0; r < 2; r++) {
      const T *Pr = P + 3 * r;
      for (int c = 0; c < 3; c++) o.Jx[3 * r + c] = Pr[0] * R[c] + Pr[1] * R[3 + c] + Pr[2] * R[6 + c];
      T *J = o.Jc + CD * r;
      J[0] = Pr[1] * (-a2) + Pr[2] * a1;
      J[1] = Pr[0] * a2 - Pr[2] * a0;
      J[2] = -Pr[0] * a1 + Pr[1] * a0;
      J[3] = Pr[0]; J[4] = Pr[1]; J[5] = Pr[2];
      T pr = r == 0 ? px : py;
      J[6] = d * pr;       // d/df
      J[7] = f * r2 * pr;  // d/dk1
    }
  }
}

// FP64 projection of X by camera (R, t, f, k1, cx, cy); returns z_c. With
// k1 = 0 the pinhole expression (f x_c / z_c + cx) as written everywhere else.
__device__ inline double proj64(const double *R, const double *t, double f, double k1, double cx, double cy,
                                const double *X, double &u, double &v) {
  double Xc[3];
  for (int r = 0; r < 3; r++) Xc[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
  double iz = 1.0 / Xc[2];
  if (k1 == 0.0) {
    u = f * Xc[0] * iz + cx;
    v = f * Xc[1] * iz + cy;
  } else {
    double px = Xc[0] * iz, py = Xc[1] * iz;
    double fd = f * (1.0 + k1 * (px * px + py * py));
    u = fd * px + cx;
    v = fd * py + cy;
  }
  return Xc[2];
}

// ---------------------------------------------------------------------------
// learned preconditioner: z = G^T G r, G = M^-1 (I - N) L^-1 block lower
// triangular over the camera graph, applied in FP32 (a preconditioner needs no
// FP64; the PCG vectors stay FP64). Per camera g: D = M^-1 L^-1 and Li = L^-1
// (36 floats each, row-major); per CSR entry a = (row v, column u < v):
// F = M_v^-1 N_vu (36 floats); mir[a] = position of the reverse entry.
//   pass 1  rh_c = Li_c r_c
//   pass 2  y_i = D_i r_i - sum_{j<i} F_ij rh_j                     (y = G r)
//   pass 3  z_j = D_j^T y_j - Li_j^T sum_{i>j} F_ij^T y_i           (z = G^T y)
// ---------------------------------------------------------------------------
struct FsaiView {
  const int *ptr, *adj, *mir;
  const float *D, *Li, *F;
};

struct FsaiApply {
  int M = 0;                       // cameras
  const int *node_sys = nullptr;   // camera -> system (sub-block), for the live mask
  const int *nvo = nullptr;        // camera -> offset of its 6 entries in r and z
  FsaiView P{};
  float *rh = nullptr, *y = nullptr;  // 6 floats per camera each
  cudaStream_t stream = nullptr;      // used when no context is given
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct GraphRec;

// launch shapes the autotuner picks (rpba_tune): block sizes of kernels that
// give every thread one independent item, so they change timing, not results
// the FP32 Schur kernel's pairs per thread (consecutive pairs of one segment)
#define SC_ITEM 8

struct Tuning {
  int isect = 128;    // k_isect_fused_f: points per CTA
  int lin = 128;      // k_linearize: instances per CTA
  int backsub = 128;  // k_backsub: instances per CTA
  int robust = 256;   // k_robust_weights(_f): observations per CTA
};

struct Ctx {
  rpba_options opt;
  Tuning tune;
  std::string tune_cache_path;  // the context's copy of opt.tune_cache
  cudaStream_t stream = nullptr;
  std::string err;
  int dev = 0;

  int M = 0, N = 0, K = 0, L = 0, P = 0;
  long long n_pairs = 0;
  bool has_winv = false;
  bool intersected = false;
  int max_cam_obs = 0;  // largest observation count of one camera
  int max_tiles = 0;    // largest RCS tile count of a sub-block

  // host copies of the topology
  std::vector<int> h_sub_cam_ptr;   // L+1 (cameras sorted by (sub, id))
  std::vector<int> h_sub_cam;       // M
  std::vector<int> h_sub_inst_ptr;  // L+1
  std::vector<int> h_inst_pt, h_inst_sub;
  std::vector<int> h_obs_user;      // K: GPU position -> user index
  std::vector<int> h_pt_nobs;       // N: observations per point
  // internal point numbering (see build): caller's id -> internal, and back;
  // canonical instance order (sub-block, caller's id) -> internal instance
  std::vector<int> h_pt_perm, h_pt_inv, h_inst_canon;
  int *d_pt_inv = nullptr, *d_inst_canon = nullptr;  // the same maps on the device
  double *perm_scratch = nullptr;                      // one per-point or per-instance array
  size_t perm_scratch_n = 0;                           // its length in doubles
  int n_active_start = 0;
  std::vector<long long> h_S_off;   // L: offset (doubles) of the RCS of l
  std::vector<int> h_npad;          // L: padded RCS size
  long long S_total = 0;

  // every device allocation, freed at destroy
  std::vector<void *> allocs;

  // cameras
  double *R = nullptr, *t = nullptr, *intr = nullptr, *Rt = nullptr, *tt = nullptr;
  // per-camera intrinsics (opt.intrinsics): cd = 8 camera unknowns, the
  // radial parameter k1 (and f in intr) estimated, trial f and k1
  int cd = 6;
  double *k1 = nullptr, *ft = nullptr, *k1t = nullptr;
  int *cam_sub = nullptr, *cam_local = nullptr, *sub_cam_ptr = nullptr, *sub_cam = nullptr;
  int *cam_obs_ptr = nullptr, *cam_obs = nullptr;
  double *cam_sigma = nullptr;
  // points
  double *X = nullptr;
  uint8_t *active = nullptr;
  int *pt_inst_ptr = nullptr, *pt_inst = nullptr;
  int *tp_list = nullptr;  // the tie points (>= 2 instances), internal numbering
  int n_tp = 0;
  // instances
  int *inst_pt = nullptr, *inst_sub = nullptr, *inst_obs_ptr = nullptr, *sub_inst_ptr = nullptr;
  double *Xl = nullptr, *Xlt = nullptr, *Wl = nullptr, *inst_cost = nullptr;
  void *Ninv = nullptr, *gX = nullptr;  // compute precision
  // intersection scratch
  double *isect_N = nullptr;  // P x 9 (sym3 + gradient)
  int *isect_state = nullptr; // N: 0 idle, 1 running, 2 converged, 3 failed
  int *isect_iter = nullptr;
  // observations
  int *obs_cam = nullptr, *obs_inst = nullptr, *obs_user = nullptr, *obs_pt = nullptr;
  uint16_t *obs_camloc = nullptr;  // camera of each observation within its sub-block (staged cost kernels)
  // FP32 form: the static observation streams in camera-major order (the
  // order of cam_obs), for the per-camera kernels (MAD, camera blocks): point,
  // instance, position (hi, lo), C^-1 and its upper Cholesky factor
  int *cm_pt = nullptr, *cm_inst = nullptr;
  float *cm_xy32 = nullptr, *cm_xylo = nullptr, *cm_winv32 = nullptr, *cm_whiten32 = nullptr;
  double *obs_xy = nullptr, *obs_winv = nullptr, *obs_w = nullptr;
  void *NXC = nullptr, *Z = nullptr;  // compute precision, K x 18 each
  // Schur pairs
  int *pair_a = nullptr, *pair_b = nullptr;
  // FP32 form: Schur pairs sorted by (camera of a, camera of b, a): the two
  // observation positions, the instance and the segment (camera pair) of each
  // pair; the two cameras of each segment
  int *spair_a = nullptr, *spair_b = nullptr, *spair_q = nullptr, *spair_seg = nullptr;
  int *seg_cam = nullptr, *seg_nb = nullptr;
  long long n_segs = 0;
  // items: runs of at most SC_ITEM consecutive pairs of one segment, one per
  // thread of the Schur kernel (first pair of each item, then n_pairs)
  int *sitem = nullptr;
  long long n_items = 0;
  // FP32 form, block-Jacobi PCG by refinement: the RCS as hi and lo planes
  // (the layout of S), the solution X in float-float, the FP32 CG vectors of
  // a stage (x, r, z, p) and its product q, M^-1 in FP32, per-sub-block stage
  // words and the active flags (stage number + 1 while the solve runs)
  float *pcg_Shi = nullptr, *pcg_Slo = nullptr;
  float2 *pcg_fx = nullptr;
  float *pcg_x32 = nullptr, *pcg_r32 = nullptr, *pcg_z32 = nullptr, *pcg_p32 = nullptr;
  unsigned long long *pcg_qi = nullptr;  // the CG product S_hi p in 64-bit fixed point
  int2 *pcg_tile_map = nullptr;           // per lower tile of the running RCS: (sub-block, a << 16 | b)
  float *pcg_Minv32 = nullptr, *pcg_s32 = nullptr;
  int *pcg_act = nullptr;
  size_t pcg_ff_smem = 0;  // the FP32 step's shared memory: r and z of the largest sub-block
  int pcg_pred = 8;        // CG iterations of the previous solve: the first convergence read
  int pcg_pred_stage[8] = {8, 8, 8, 8, 8, 8, 8, 8};  // the same per refinement stage
  // the loop as conditional graph nodes: two streams on which its bodies are
  // captured, and the list that receives the body kernels' names meanwhile
  cudaStream_t pcg_body_stream[2] = {nullptr, nullptr};
  std::vector<const char *> *capture_list = nullptr;
  bool pcg_no_device_loop = false;  // its capture failed once: the host-driven loop
  // RCS
  double *S = nullptr, *y = nullptr, *dC = nullptr;  // y, dC: sum of n_pad over l
  long long *S_off = nullptr;
  int *npad = nullptr, *ycam_off = nullptr, *sub_ntiles = nullptr, *linv_off = nullptr;
  int ytot = 0;
  // PCG on the RCS
  double *pcg_Minv = nullptr, *pcg_x = nullptr, *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr,
         *pcg_q = nullptr, *pcg_st = nullptr, *pcg_pq = nullptr;
  int *pcg_live = nullptr, *pcg_tiles = nullptr;
  int pcg_tiles_total = 0;
  double *obs_cost = nullptr, *seg_part = nullptr;
  double *obs_whiten = nullptr;  // per observation upper Cholesky factor of C^-1 (when given)
  float *obs_xy32 = nullptr, *obs_winv32 = nullptr, *obs_w32 = nullptr;
  float *Xl_hi = nullptr, *Xl_lo = nullptr, *X_hi = nullptr,
        *X_lo = nullptr, *dC32 = nullptr;
  // FP32 form, float-float residuals: camera records (FF_CAM floats) of the
  // current and the trial state, the low words of the observations relative
  // to the principal point, trial copies X^l as hi + lo, W^l and the
  // whitening factors in FP32, and the per-camera robust scale in FP32
  float *camff = nullptr, *camff_t = nullptr, *obs_xylo = nullptr, *Xlt_hi = nullptr, *Xlt_lo = nullptr,
        *Wl32 = nullptr, *obs_whiten32 = nullptr, *cam_sigma32 = nullptr;
  int *sub_obs_ptr = nullptr;
  // chunks of <= 256 observations inside one sub-block: sub-block, first
  // observation, chunks per sub-block (CSR), one partial cost per chunk
  int *chunk_sub = nullptr, *chunk_start = nullptr, *sub_chunk_ptr = nullptr;
  int n_chunks = 0;
  // groups of up to COST_GROUP chunks of one sub-block (first chunk of each)
  // for the cost kernels that stage the sub-block's camera records in shared
  // memory (cost_smem bytes per CTA; 0: the records are read from global memory)
  int *group_chunk = nullptr;
  int n_groups = 0;
  size_t cost_smem = 0;
  double *chunk_part = nullptr;
  // FP32 form: the outer iteration's tail evaluates the sub-block costs with
  // the sigma_0 sums in one pass (every X^l equals its X there); the next
  // bact starts from these costs while no entry point has changed the state
  // since. sigma0_part: 5 sums per chunk, then per sub-block, then the total
  double *f0_cache = nullptr, *sigma0_part = nullptr;
  bool f0_valid = false;
  std::vector<int> h_sched;  // per factorisation step: prefix sums of panel and update tiles
  int *sched = nullptr;
  double *Linv64 = nullptr;
  float *S32 = nullptr, *Linv32 = nullptr, *ir_r32 = nullptr;
  long long *S32_off = nullptr;
  double *ir_d = nullptr, *ir_rs = nullptr, *ir_x = nullptr, *ir_t = nullptr;
  // FP32 factorisation on the tensor cores (chol_tc): the factor's block
  // columns of 32 as three TF32 pieces in panel-major order (block column k
  // of sub-block l is npad_l rows of 32 floats from row tc_prow[l] + k npad_l),
  // a TMA tensor map per piece, per step the CTA prefix sums over the
  // sub-blocks, and a flag that a bounded wait gave up
  float *tc_panel[3] = {nullptr, nullptr, nullptr};
  long long *tc_prow = nullptr;
  int *tc_sched = nullptr;
  std::vector<int> h_tc_ctas;  // CTAs of each step
  CUtensorMap tc_map[3];
  int *tc_err = nullptr;
  bool tc_ready = false;
  // persistent form: the task queue, tasks per (sub-block, step), the queue
  // head and finished-task counters, the grid (resident CTAs)
  int4 *tc_tasks = nullptr;
  int *tc_need = nullptr, *tc_count = nullptr;
  int tc_n_tasks = 0, tc_grid = 0;
  // which sub-blocks the LM adjustment moves and which points the
  // intersection handles (all by default; a share of them in sharded runs)
  uint8_t *sub_mask = nullptr, *pt_mask = nullptr;
  // the scalar TP weight's rho (weight_mode 2) on the device, and the outer
  // iterations run so far (rho = rho0 1.01^t)
  double *wrho = nullptr;
  int outer_done = 0;
  // LM control per sub-block
  double *lm_lambda = nullptr, *lm_F = nullptr, *lm_Ft = nullptr, *lm_best = nullptr;
  int *lm_grace = nullptr, *lm_rej = nullptr, *lm_it = nullptr, *lm_run = nullptr;
  int *lm_acc = nullptr, *lm_cholfail = nullptr;
  // reductions
  double *red = nullptr;   // scratch for block partials
  int red_blocks = 0;
  int *counters = nullptr; // small device counters
  // profiling: kernel launch counts (always) and event-timed phases (when enabled)
  long long launches = 0;
  std::map<std::string, long long> launch_by_name;
  bool prof_enabled = false;
  std::string prof_only;  // when set, only launches of this kernel are timed
  struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_recs;
  std::map<std::string, double> prof_ms;
  // CUDA graph of one lock-step LM iteration (captured on first use)
  GraphRec *capture = nullptr;  // non-null while capturing
  GraphRec *lm_graph = nullptr;
  GraphRec *lm_graph_pre = nullptr, *lm_graph_post = nullptr;  // PCG solvers: around the CG loop
  GraphRec *outer_graph[2] = {nullptr, nullptr};  // one outer iteration's tail (without / with robust weights)
  bool use_graphs = true;
  cudaStream_t own_stream = nullptr;  // created when the caller passes the legacy default stream
  int *h_pinned_counter = nullptr;
  double *h_pinned_d = nullptr;
  // learned block preconditioner (solver 3): camera graph in sub-block order,
  // network parameters (FP32 and BF16) and per-camera work arrays
  std::vector<int> h_nadj_ptr, h_nadj, h_nadj_mir, h_nadj_row;
  int *node_sys = nullptr, *nadj_ptr = nullptr, *nadj = nullptr, *nadj_mir = nullptr, *nadj_row = nullptr;
  float *gnn_w = nullptr;
  void *gnn_wb = nullptr;
  float *gnn_x = nullptr, *gnn_e = nullptr, *gnn_h = nullptr, *gnn_C = nullptr;
  double *gnn_L = nullptr, *gnn_nrm = nullptr, *gnn_shat = nullptr, *gnn_gam = nullptr;
  float *pcg_D32 = nullptr, *pcg_Li32 = nullptr, *pcg_F32 = nullptr;  // factor of the learned P^-1
  float *gnn_rh = nullptr, *gnn_y = nullptr;                            // apply scratch, 6 per camera
  int *node_voff = nullptr;                                             // camera -> RCS vector offset
  int *gnn_ok = nullptr, *pcg_run2 = nullptr, *pcg_fail2 = nullptr;
  bool gnn_ready = false;
  long long gnn_fallbacks = 0;  // sub-block solves re-done by block-Jacobi PCG
  FsaiApply fsai;               // the learned factor of the current LM iteration
  bool auto_solver = false;     // solver 4: PCG until a solve needs too many iterations
  bool auto_switch = false;     // ... then the direct solver from the next LM step
};

// device allocation through the context's allocator (freed at destroy)
rpba_status ctx_alloc(Ctx *ctx, void **p, size_t bytes);

// error helpers
#define RPBA_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return RPBA_ERR_CUDA;                                                          \
    }                                                                                \
  } while (0)

#define RPBA_TRY(call)                \
  do {                                \
    rpba_status s_ = (call);          \
    if (s_ != RPBA_OK) return s_;     \
  } while (0)

rpba_status check_launch(Ctx *ctx, const char *what);

// A captured CUDA graph with the names of its kernels and, per kernel, a pair
// of event-record nodes, so that replays can be counted and timed per kernel.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  bool with_events = false;  // captured with per-kernel event-record nodes
  std::string prof_only;     // ... for this kernel only (empty: all)
  std::vector<const char *> kernels;
  // the FP32-form PCG loop as conditional while nodes: the kernels of the
  // inner (CG step) and outer (refinement stage) bodies, counted per replay
  // from the loop's device counters
  bool pcg_loop = false;
  std::vector<const char *> loop_inner, loop_outer;
  struct Ev {
    const char *name;
    cudaEvent_t a, b;
  };
  std::vector<Ev> events;
};

// times the kernel launched in its scope with CUDA events on the context
// stream; while a graph is being captured the events become record nodes of
// the graph (timed on every replay)
struct PhaseTimer {
  Ctx *ctx;
  const char *name;
  cudaEvent_t a = nullptr, b = nullptr;
  PhaseTimer(Ctx *c, const char *n) : ctx(c), name(n) {
    if (ctx->capture && !ctx->capture->with_events) return;
    if (!ctx->prof_only.empty() && ctx->prof_only != name) return;
    if (ctx->capture) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecordWithFlags(a, ctx->stream, cudaEventRecordExternal);
    } else if (ctx->prof_enabled) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~PhaseTimer() {
    if (!a) return;
    if (ctx->capture) {
      cudaEventRecordWithFlags(b, ctx->stream, cudaEventRecordExternal);
      ctx->capture->events.push_back({name, a, b});
    } else {
      cudaEventRecord(b, ctx->stream);
      ctx->prof_recs.push_back({name, a, b});
    }
  }
};

// after every kernel launch: count it and check the launch status
inline rpba_status post_launch(Ctx *ctx, const char *name) {
  if (ctx->capture_list) {
    ctx->capture_list->push_back(name);
  } else if (ctx->capture) {
    ctx->capture->kernels.push_back(name);
  } else {
    ctx->launches++;
    ctx->launch_by_name[name]++;
  }
  return check_launch(ctx, name);
}

#define RPBA_KERNEL(ctx, name, ...)      \
  do {                                   \
    {                                    \
      PhaseTimer pt_(ctx, name);         \
      __VA_ARGS__;                       \
    }                                    \
    RPBA_TRY(post_launch(ctx, name));    \
  } while (0)

// kernels (host launchers), see kernels_*.cu
rpba_status launch_residuals(Ctx *ctx, double *v_dev /* K x 2, GPU order */);
rpba_status launch_jacobians(Ctx *ctx, double *Jc_dev, double *Jx_dev);
// sigma_0 in two halves: the sums into pinned memory (capturable), and the
// values from them after a synchronisation
rpba_status sigma0_launch(Ctx *ctx);
rpba_status cost_sigma0_launch(Ctx *ctx);
// the cost kernels with staged camera records: chunks per CTA, bytes per
// staged record, the largest staging they take (else the global-memory form)
#define RPBA_COST_GROUP 4
#define RPBA_CAM_STAGE_BYTES 144
#define RPBA_COST_STAGE_MAX_SMEM (96 * 1024)  // 682 cameras: local indices fit 16 bits
rpba_status cost_groups_setup(Ctx *ctx);
// the camera-major copies (FP32 form), from the observation-order arrays
rpba_status camera_major_setup(Ctx *ctx);
void sigma0_finish(const Ctx *ctx, double *sigma0, double *rms, long long *n_obs, long long *n_points);
rpba_status launch_sigma0(Ctx *ctx, double *sigma0, double *rms, long long *n_obs = nullptr,
                          long long *n_points = nullptr);
// Eq. bars for all points (tp_only = 0) or the tie points; fp64 forces the
// FP64 kernels in the FP32 form. tp_copies: the FP32 form's TP intersection
// also restarts the converged TPs' copies X^l at X_TP (a later
// launch_tp_copies is then not needed for them)
rpba_status launch_intersect(Ctx *ctx, int tp_only, int *n_dropped, bool fp64 = false, bool tp_copies = false);
rpba_status launch_exchange(Ctx *ctx);
rpba_status launch_tp_copies(Ctx *ctx, int tp_only);
rpba_status launch_camera_scale(Ctx *ctx);
// FP32 form: rebuild the camera records and the hi + lo words of X and X^l
// from the FP64 state (after the host sets it)
rpba_status sync_mirrors(Ctx *ctx);
rpba_status launch_robust_weights(Ctx *ctx, int *n_down);
rpba_status launch_eliminate(Ctx *ctx);
rpba_status launch_sub_costs(Ctx *ctx, int trial, double *F_dev);
rpba_status launch_build_rcs(Ctx *ctx, const double *lambda_dev, const int *run_dev);
rpba_status launch_solve_rcs(Ctx *ctx, const int *run_dev, int *fail_dev);
rpba_status tc_chol_setup(Ctx *ctx);
rpba_status launch_pcg_blockjacobi(Ctx *ctx, const int *run_dev, int *fail_dev);
rpba_status launch_pcg_learned(Ctx *ctx, const int *run_dev, int *fail_dev);
void build_camera_graph(Ctx *ctx, const std::vector<int> &inst_obs_ptr, const std::vector<int> &obs_cam_sorted,
                        const std::vector<int> &inst_sub, const std::vector<int> &cam_local);
rpba_status pcg_iterate(Ctx *ctx, const int *run_dev, int *fail_dev, const FsaiApply *fsai);
// the phases of pcg_iterate, and the preconditioner set-ups
rpba_status pcg_init(Ctx *ctx, const int *run_dev, int *fail_dev, const FsaiApply *fsai);
// the FP32 form's block-Jacobi PCG runs as FP32 CG stages refined by
// float-float residuals (solver 1, also when chosen by solver 4) when no
// sub-block has more than RPBA_PCG_FF_MAX_N unknowns (256 threads x 8
// elements in registers; r and z, 4 B each, then take at most 16 KB of shared
// memory). A stage stops at RPBA_PCG_INNER_TOL of its right-hand side (or
// sooner, where the final tolerance asks for less); at most
// RPBA_PCG_MAX_STAGES stages per solve.
#define RPBA_PCG_FF_MAX_N 2048
#define RPBA_PCG_INNER_TOL 1e-4
#define RPBA_PCG_MAX_STAGES 8
#define PCG_S32_WORDS 8  // per-sub-block FP32 words of the refinement (pcg_s32)
#define PCG_S32_STAGES 4 // the word counting the stages of the last solve
inline bool ff_pcg(const Ctx *ctx) { return ctx->pcg_Shi != nullptr && ctx->opt.solver == 1; }
rpba_status pcg_loop(Ctx *ctx, const FsaiApply *fsai, int *iters /* lock-step iterations run, nullable */);
// counters of the device-driven FP32-form loop: lock-step CG steps and
// refinement stages of the last solve (device counters[12, 14), copied to
// h_pinned_counter[12, 14) by the captured graph)
#define PCG_LOOP_COUNTERS 12
// the FP32-form PCG loop runs as conditional graph nodes when the LM step is
// captured (the context's body streams exist and no loop kernel is timed)
bool pcg_device_loop(const Ctx *ctx);
rpba_status pcg_out(Ctx *ctx, const int *run_dev, const int *fail_dev);
rpba_status pcg_bj_setup(Ctx *ctx, const int *run_dev, int *fail_dev);
rpba_status learned_setup(Ctx *ctx, const int *run_dev, int *fail_dev, FsaiApply *F);
rpba_status learned_fallback(Ctx *ctx, const int *run_dev, int *fail_dev);
// z = P^-1 r with the learned factor over the cameras of the live systems
// (live NULL: all); counted on ctx when given, else launched on F.stream
rpba_status fsai_apply(Ctx *ctx, const FsaiApply &F, const int *live, const double *r, double *z,
                       bool skip_first = false);
rpba_status launch_backsub_trial(Ctx *ctx, const int *run_dev);
rpba_status launch_lm_decide(Ctx *ctx);
rpba_status launch_lm_apply(Ctx *ctx, const int *acc_dev);
rpba_status launch_lm_init(Ctx *ctx);
rpba_status launch_fill_int(Ctx *ctx, int *p, int n, int v);
rpba_status launch_fill_double(Ctx *ctx, double *p, long long n, double v);

}  // namespace rpba

// the opaque handle of the C ABI
struct rpba_ctx {
  rpba::Ctx c;
};

