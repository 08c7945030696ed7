// kernels_obs.cu -- observation-, instance-, point- and camera-level kernels
// of the RPBA hot path on sm_103a:
//   residuals and Jacobians (Sec. 2, Eq. ta), weighted cost and sigma_0
//   (Eq. v2, normalw, sigma0), intersection of points with the cameras fixed
//   and the refined TP weights (Eq. bars, Sec. 5.1), normal equations of a
//   sub-block with the TP control term and LM damping (Eq. bact, Sec. 5.5),
//   Schur complement onto the cameras (Sec. 2, 5.5), back-substitution and
//   trial update, robust weights (Sec. 5.3).
//
// Compute precision T is double for the all-FP64 form and float for the
// FP32 form; the FP64 master state (positions, rotations) and the RCS stay
// double. The FP32 form runs no FP64 arithmetic per observation, point or
// instance: residuals for the cost, sigma_0, the MAD and the robust test in
// float-float (ffloat.cuh), Jacobians and normal equations in FP32 on hi + lo
// position words, the per-observation N_XC and Z blocks in registers only,
// format changes by integer bit operations, and FP64 only for sums over
// blocks of terms and for the rare ill-conditioned 3x3 point systems.
#include <cuda_runtime.h>
#include <math.h>

#include "rpba_internal.cuh"

namespace rpba {

// ---------------------------------------------------------------------------
// views
// ---------------------------------------------------------------------------
struct View {
  int M, N, K, L, P, has_winv;
  const double *R, *t;
  double *intr;
  double *Rt, *tt;
  // per-camera intrinsics: cd = 8 camera unknowns, k1 (NULL without), trial
  // f and k1; k1on: the projections include the radial term
  int cd, k1on;
  double *k1, *ft, *k1t;
  const int *cam_sub, *cam_local, *sub_cam_ptr, *sub_cam, *cam_obs_ptr, *cam_obs;
  const uint16_t *obs_camloc;
  const int *cm_pt, *cm_inst;
  const float *cm_xy32, *cm_winv32;
  double *X;
  uint8_t *active;
  const int *pt_inst_ptr, *pt_inst;
  const int *inst_pt, *inst_sub, *inst_obs_ptr, *sub_inst_ptr;
  double *Xl, *Xlt, *Wl, *inst_cost;
  const int *obs_cam, *obs_inst, *obs_user, *obs_pt;
  const double *obs_xy, *obs_winv;
  double *obs_w;
  double *S, *y, *dC;
  const long long *S_off;
  const int *npad, *ycam_off;
  // FP32 form: inputs rounded once, positions as float hi + lo pairs
  const float *obs_xy32;   // (x - cx, y - cy)
  const float *obs_winv32;
  float *obs_w32;
  float *Xl_hi, *Xl_lo;    // sub-block copies X^l
  float *X_hi, *X_lo;      // points X
  float *dC32;             // camera updates
  // float-float residuals: camera records, observation low words, trial X^l
  float *camff, *camff_t;
  const float *obs_xylo;
  float *Xlt_hi, *Xlt_lo;
  float *Wl32;
  // the TPs' weight: 0 refined (Sec. 5.1), 1 all cameras, 2 rho I with rho
  // read from device memory (it grows per outer iteration: graphs replay)
  int wmode;
  const double *wrho;
};

// the weight W^l written for a TP instance under the weight mode (the
// ablations of Sec. 6.4): element e of the sym3 from the refined value and
// the point's full normal matrix
__device__ inline double tp_weight(const View &v, int e, double refined, double full) {
  if (v.wmode == 1) return full;
  if (v.wmode == 2) return (e == 0 || e == 3 || e == 5) ? *v.wrho : 0.0;
  return refined;
}

static View make_view(Ctx *c) {
  View v;
  v.M = c->M; v.N = c->N; v.K = c->K; v.L = c->L; v.P = c->P; v.has_winv = c->has_winv;
  v.R = c->R; v.t = c->t; v.intr = c->intr; v.Rt = c->Rt; v.tt = c->tt;
  v.cam_sub = c->cam_sub; v.cam_local = c->cam_local; v.sub_cam_ptr = c->sub_cam_ptr;
  v.obs_camloc = c->obs_camloc;
  v.cm_pt = c->cm_pt; v.cm_inst = c->cm_inst; v.cm_xy32 = c->cm_xy32; v.cm_winv32 = c->cm_winv32;
  v.sub_cam = c->sub_cam; v.cam_obs_ptr = c->cam_obs_ptr; v.cam_obs = c->cam_obs;
  v.X = c->X; v.active = c->active; v.pt_inst_ptr = c->pt_inst_ptr; v.pt_inst = c->pt_inst;
  v.inst_pt = c->inst_pt; v.inst_sub = c->inst_sub; v.inst_obs_ptr = c->inst_obs_ptr;
  v.sub_inst_ptr = c->sub_inst_ptr; v.Xl = c->Xl; v.Xlt = c->Xlt; v.Wl = c->Wl;
  v.inst_cost = c->inst_cost; v.obs_cam = c->obs_cam; v.obs_inst = c->obs_inst;
  v.obs_user = c->obs_user; v.obs_pt = c->obs_pt; v.obs_xy = c->obs_xy; v.obs_winv = c->obs_winv;
  v.obs_w = c->obs_w; v.S = c->S; v.y = c->y; v.dC = c->dC; v.S_off = c->S_off; v.npad = c->npad;
  v.ycam_off = c->ycam_off;
  v.obs_xy32 = c->obs_xy32; v.obs_winv32 = c->obs_winv32; v.obs_w32 = c->obs_w32;
  v.Xl_hi = c->Xl_hi; v.Xl_lo = c->Xl_lo; v.X_hi = c->X_hi; v.X_lo = c->X_lo;
  v.dC32 = c->dC32;
  v.camff = c->camff; v.camff_t = c->camff_t; v.obs_xylo = c->obs_xylo;
  v.Xlt_hi = c->Xlt_hi; v.Xlt_lo = c->Xlt_lo; v.Wl32 = c->Wl32;
  v.wmode = c->opt.weight_mode;
  v.wrho = c->wrho;
  v.cd = c->cd; v.k1on = c->cd == 8; v.k1 = c->k1; v.ft = c->ft; v.k1t = c->k1t;
  return v;
}

rpba_status check_launch(Ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return RPBA_ERR_CUDA;
  }
  return RPBA_OK;
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// camera i and a point in the compute precision.
// FP64: Xc = R X + t exactly as written (cam_point_d).
// FP32 (cam_point_f): Xc = R (X - C) with the camera centre C and the point X
// both held as float pairs hi + lo (hi = fl(x), lo = fl(x - hi)), so that
// d = (X_hi - C_hi) + (X_lo - C_lo) keeps large coordinates exact to FP32
// precision without any FP64 instruction per observation; RX = Xc - t. On
// this GPU FP64 instructions, conversions included, issue at 1/64 of the
// FP32 rate, so the FP32 form rounds every input once per pass instead.
template <typename T>
struct CamPt {
  T R[9], Xc[3], RX[3], f, k1, cx, cy;
};

__device__ inline void cam_point_d(const View &v, int i, const double X[3], CamPt<double> &o) {
  const double *R = v.R + 9 * i, *t = v.t + 3 * i;
  for (int r = 0; r < 3; r++) {
    double rx = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2];
    o.RX[r] = rx;
    o.Xc[r] = rx + t[r];
  }
  for (int e = 0; e < 9; e++) o.R[e] = R[e];
  o.f = v.intr[3 * i]; o.cx = v.intr[3 * i + 1]; o.cy = v.intr[3 * i + 2];
  o.k1 = v.k1 ? v.k1[i] : 0.0;
}

__device__ inline void cam_point_f(const View &v, int i, const float *Xh, const float *Xlw, CamPt<float> &o) {
  const float4 *p = reinterpret_cast<const float4 *>(v.camff + FF_CAM * (size_t)i);
  float c[16];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    float4 a = __ldg(p + e);
    c[4 * e] = a.x; c[4 * e + 1] = a.y; c[4 * e + 2] = a.z; c[4 * e + 3] = a.w;
  }
  float4 tt = __ldg(p + 7);
  float d[3];
  for (int r = 0; r < 3; r++) d[r] = (Xh[r] - c[9 + r]) + (Xlw[r] - c[12 + r]);
  for (int e = 0; e < 9; e++) o.R[e] = c[e];
  float t[3] = {tt.y, tt.z, tt.w};
  for (int r = 0; r < 3; r++) {
    o.Xc[r] = o.R[3 * r] * d[0] + o.R[3 * r + 1] * d[1] + o.R[3 * r + 2] * d[2];
    o.RX[r] = o.Xc[r] - t[r];
  }
  o.f = c[15]; o.cx = 0.f; o.cy = 0.f;
  o.k1 = v.k1on ? __ldg(p + 6).z : 0.f;  // record float 26
}

// the FP32 projection's words of a camera record held in registers (R, C hi
// and lo, f; t; k1), for a thread that projects many points into one camera
struct CamRecF {
  float c[16], t[3], k1;
};

__device__ inline void load_cam_rec(const View &v, int i, CamRecF &r) {
  const float4 *p = reinterpret_cast<const float4 *>(v.camff + FF_CAM * (size_t)i);
#pragma unroll
  for (int e = 0; e < 4; e++) {
    float4 a = __ldg(p + e);
    r.c[4 * e] = a.x; r.c[4 * e + 1] = a.y; r.c[4 * e + 2] = a.z; r.c[4 * e + 3] = a.w;
  }
  float4 tt = __ldg(p + 7);
  r.t[0] = tt.y; r.t[1] = tt.z; r.t[2] = tt.w;
  r.k1 = v.k1on ? __ldg(p + 6).z : 0.f;  // record float 26
}

// cam_point_f's arithmetic on a record in registers
__device__ inline void cam_point_rec(const CamRecF &r, const float *Xh, const float *Xlw, CamPt<float> &o) {
  float d[3];
  for (int k = 0; k < 3; k++) d[k] = (Xh[k] - r.c[9 + k]) + (Xlw[k] - r.c[12 + k]);
  for (int e = 0; e < 9; e++) o.R[e] = r.c[e];
  for (int k = 0; k < 3; k++) {
    o.Xc[k] = o.R[3 * k] * d[0] + o.R[3 * k + 1] * d[1] + o.R[3 * k + 2] * d[2];
    o.RX[k] = o.Xc[k] - r.t[k];
  }
  o.f = r.c[15]; o.cx = 0.f; o.cy = 0.f;
  o.k1 = r.k1;
}

__device__ inline void split(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// FP32 form: camera records of the current state
__global__ void k_cam_prep(View v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.M) return;
  ff_camera_record(v.R + 9 * i, v.t + 3 * i, v.intr[3 * i], v.k1 ? v.k1[i] : 0.0, v.camff + FF_CAM * (size_t)i);
}

// hi/lo pairs of the sub-block copies (which = 0) or of the points (which = 1)
__global__ void k_split_points(View v, int which) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int n = which ? v.N : v.P;
  if (q >= n) return;
  const double *X = (which ? v.X : v.Xl) + 3 * (size_t)q;
  float *hi = (which ? v.X_hi : v.Xl_hi) + 3 * (size_t)q;
  float *lo = (which ? v.X_lo : v.Xl_lo) + 3 * (size_t)q;
  for (int e = 0; e < 3; e++) split(X[e], hi[e], lo[e]);
}

static rpba_status cam_prep(Ctx *ctx) {
  if (ctx->opt.precision != 1 || ctx->M == 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_cam_prep", k_cam_prep<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(make_view(ctx)));
  return RPBA_OK;
}

static rpba_status split_points(Ctx *ctx, int which) {
  int n = which ? ctx->N : ctx->P;
  if (ctx->opt.precision != 1 || n == 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_split_points", k_split_points<<<nblk(n, 256), 256, 0, ctx->stream>>>(make_view(ctx), which));
  return RPBA_OK;
}

// FP32 form: the camera records and the hi + lo words of X and X^l follow
// the FP64 state. Kernels that change that state keep them current
// (intersection, exchange, TP copies, LM apply); this rebuilds all of them
// after the host sets the state.
rpba_status sync_mirrors(Ctx *ctx) {
  RPBA_TRY(cam_prep(ctx));
  RPBA_TRY(split_points(ctx, 0));
  return split_points(ctx, 1);
}

// observation k in the compute precision: residual-relevant data
template <typename T>
struct ObsT {
  T x, y;    // observation minus principal point
  T W[3];    // C^-1
  T w;       // robust weight
};

template <typename T>
__device__ inline void load_obs(const View &v, int k, ObsT<T> &o) {
  if constexpr (sizeof(T) == sizeof(float)) {
    o.x = v.obs_xy32[2 * k]; o.y = v.obs_xy32[2 * k + 1];
    if (v.has_winv) { o.W[0] = v.obs_winv32[3 * k]; o.W[1] = v.obs_winv32[3 * k + 1]; o.W[2] = v.obs_winv32[3 * k + 2]; }
    else { o.W[0] = 1; o.W[1] = 0; o.W[2] = 1; }
    o.w = v.obs_w32[k];
  } else {
    int i = v.obs_cam[k];
    o.x = v.obs_xy[2 * k] - v.intr[3 * i + 1];
    o.y = v.obs_xy[2 * k + 1] - v.intr[3 * i + 2];
    if (v.has_winv) { o.W[0] = v.obs_winv[3 * k]; o.W[1] = v.obs_winv[3 * k + 1]; o.W[2] = v.obs_winv[3 * k + 2]; }
    else { o.W[0] = 1; o.W[1] = 0; o.W[2] = 1; }
    o.w = v.obs_w[k];
  }
}

// projection (relative to the principal point) and Jacobians of camera i at
// a point given in FP64 (Xd) or as FP32 hi/lo pairs (Xh, Xlw); CD = 8 with
// per-camera intrinsics (camera Jacobian 2 x 8), else 6
template <typename T, int CD>
__device__ inline void obs_proj(const View &v, int i, const double *Xd, const float *Xh, const float *Xlw,
                                ProjJac<T, CD> &pj, T &z) {
  CamPt<T> cp;
  if constexpr (sizeof(T) == sizeof(float)) cam_point_f(v, i, Xh, Xlw, cp);
  else cam_point_d(v, i, Xd, cp);
  z = cp.Xc[2];
  project_jac<T, CD>(cp.R, cp.Xc, cp.RX, cp.f, cp.k1, T(0), T(0), pj);
}

// the projection and the point Jacobian only (intersection, point blocks),
// with or without the radial term
template <typename T>
struct ProjX {
  T u, v, Jx[6];
};

template <typename T>
__device__ inline void proj_x(const View &v, int i, const double *Xd, const float *Xh, const float *Xlw,
                              ProjX<T> &o, T &z) {
  if (v.k1on) {
    ProjJac<T, 8> pj;
    obs_proj<T, 8>(v, i, Xd, Xh, Xlw, pj, z);
    o.u = pj.u; o.v = pj.v;
    for (int e = 0; e < 6; e++) o.Jx[e] = pj.Jx[e];
  } else {
    ProjJac<T, 6> pj;
    obs_proj<T, 6>(v, i, Xd, Xh, Xlw, pj, z);
    o.u = pj.u; o.v = pj.v;
    for (int e = 0; e < 6; e++) o.Jx[e] = pj.Jx[e];
  }
}

// ---------------------------------------------------------------------------
// residuals, Jacobians (diagnostics / parity) at the global state
// ---------------------------------------------------------------------------
__global__ void k_residuals(View v, double *out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  int i = v.obs_cam[k], j = v.obs_pt[k];
  double pu, pv;
  proj64(v.R + 9 * i, v.t + 3 * i, v.intr[3 * i], v.k1 ? v.k1[i] : 0.0, v.intr[3 * i + 1], v.intr[3 * i + 2],
         v.X + 3 * j, pu, pv);
  int u = v.obs_user[k];
  out[2 * u] = pu - v.obs_xy[2 * k];
  out[2 * u + 1] = pv - v.obs_xy[2 * k + 1];
}

template <typename T, int CD>
__global__ void k_jacobians(View v, double *Jc, double *Jx) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  int i = v.obs_cam[k], j = v.obs_pt[k];
  ProjJac<T, CD> pj;
  T z;
  obs_proj<T, CD>(v, i, v.X + 3 * j, v.X_hi + 3 * j, v.X_lo + 3 * j, pj, z);
  int u = v.obs_user[k];
  for (int e = 0; e < 2 * CD; e++) Jc[2 * CD * (size_t)u + e] = (double)pj.Jc[e];
  for (int e = 0; e < 6; e++) Jx[6 * u + e] = (double)pj.Jx[e];
}

rpba_status launch_residuals(Ctx *ctx, double *v_dev) {
  if (ctx->K == 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_residuals", k_residuals<<<nblk(ctx->K, 256), 256, 0, ctx->stream>>>(make_view(ctx), v_dev));
  return RPBA_OK;
}

rpba_status launch_jacobians(Ctx *ctx, double *Jc, double *Jx) {
  if (ctx->K == 0) return RPBA_OK;
  dim3 g(nblk(ctx->K, 256)), b(256);
  if (ctx->opt.precision == 1 && ctx->cd == 8)
    RPBA_KERNEL(ctx, "k_jacobians", k_jacobians<float, 8><<<g, b, 0, ctx->stream>>>(make_view(ctx), Jc, Jx));
  else if (ctx->opt.precision == 1)
    RPBA_KERNEL(ctx, "k_jacobians", k_jacobians<float, 6><<<g, b, 0, ctx->stream>>>(make_view(ctx), Jc, Jx));
  else if (ctx->cd == 8)
    RPBA_KERNEL(ctx, "k_jacobians", k_jacobians<double, 8><<<g, b, 0, ctx->stream>>>(make_view(ctx), Jc, Jx));
  else
    RPBA_KERNEL(ctx, "k_jacobians", k_jacobians<double, 6><<<g, b, 0, ctx->stream>>>(make_view(ctx), Jc, Jx));
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// deterministic block reductions
// ---------------------------------------------------------------------------
template <int NV>
__device__ inline void block_reduce_store(double (&val)[NV], double *out_block) {
  __shared__ double sh[NV][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < NV; e++) {
    double x = val[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[e][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int e = 0; e < NV; e++) {
      double x = lane < nw ? sh[e][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out_block[e] = x;
    }
  }
}

// sum of `nb` rows of NV partials, one block
template <int NV>
__global__ void k_sum_partials(const double *part, int nb, double *out) {
  double acc[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) acc[e] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int e = 0; e < NV; e++) acc[e] += part[(size_t)b * NV + e];
  block_reduce_store<NV>(acc, out);
}

// sigma_0 / RMS sums: [sum w v^T W v, n_active_obs, sum |v|^2 (w == 1), n (w == 1),
// n_active_points]
__global__ void k_obs_sigma(View v, double *part) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.N; j += gridDim.x * blockDim.x)
    acc[4] += v.active[j] ? 1.0 : 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < v.K; k += gridDim.x * blockDim.x) {
    int j = v.obs_pt[k];
    if (!v.active[j]) continue;
    int i = v.obs_cam[k];
    double pu, pv;
    proj64(v.R + 9 * i, v.t + 3 * i, v.intr[3 * i], v.k1 ? v.k1[i] : 0.0, v.intr[3 * i + 1], v.intr[3 * i + 2],
           v.X + 3 * j, pu, pv);
    double r0 = pu - v.obs_xy[2 * k];
    double r1 = pv - v.obs_xy[2 * k + 1];
    double W0 = 1, W1 = 0, W2 = 1;
    if (v.has_winv) { W0 = v.obs_winv[3 * k]; W1 = v.obs_winv[3 * k + 1]; W2 = v.obs_winv[3 * k + 2]; }
    double w = v.obs_w[k];
    if (w == 0.0) continue;  // deleted by the serial robust variant
    acc[0] += w * (W0 * r0 * r0 + 2.0 * W1 * r0 * r1 + W2 * r1 * r1);
    acc[1] += 1.0;
    if (w == 1.0) {
      acc[2] += r0 * r0 + r1 * r1;
      acc[3] += 1.0;
    }
  }
  block_reduce_store<5>(acc, part + 5 * blockIdx.x);
}

// FP32 form: the same sums from float-float residuals (Eq. ta) formed in
// FP32, each thread accumulating float-float (TwoSum), the blocks in FP64
__device__ void sigma_cta_sums(float sh, float sl, float rh, float rl, int n1, int n3, int np, double *o);

// one observation's sigma_0 terms from its float-float residual (FP32 form)
template <bool K1>
__device__ inline void sigma_obs_terms(const View &v, int k, int i, int j, float &sh, float &sl, float &rh,
                                       float &rl, int &n1, int &n3) {
  if (v.obs_w32[k] == 0.f) return;  // deleted by the serial robust variant
  float r0, r1;
  ff_residual(v.camff + FF_CAM * (size_t)i, v.X_hi + 3 * (size_t)j, v.X_lo + 3 * (size_t)j, v.obs_xy32[2 * k],
              v.obs_xylo[2 * k], v.obs_xy32[2 * k + 1], v.obs_xylo[2 * k + 1], r0, r1, K1);
  float W0 = 1.f, W1 = 0.f, W2 = 1.f;
  if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
  float w = v.obs_w32[k], e;
  sh = ff_two_sum(sh, w * (W0 * r0 * r0 + 2.f * W1 * r0 * r1 + W2 * r1 * r1), e);
  sl += e;
  n1++;
  if (w == 1.f) {
    rh = ff_two_sum(rh, r0 * r0 + r1 * r1, e);
    rl += e;
    n3++;
  }
}

template <bool K1>
__global__ void k_obs_sigma_f(View v, double *part) {
  float sh = 0.f, sl = 0.f, rh = 0.f, rl = 0.f;
  int n1 = 0, n3 = 0, np = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.N; j += gridDim.x * blockDim.x) np += v.active[j] ? 1 : 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < v.K; k += gridDim.x * blockDim.x) {
    int j = v.obs_pt[k];
    if (!v.active[j]) continue;
    sigma_obs_terms<K1>(v, k, v.obs_cam[k], j, sh, sl, rh, rl, n1, n3);
  }
  sigma_cta_sums(sh, sl, rh, rl, n1, n3, np, part + 5 * blockIdx.x);
}

// the sigma_0 sums of a CTA in float-float and integers (off the FP64 pipe):
// sum w v^T W v, active observations, sum |v|^2 and count of w == 1, active
// points; thread 0 writes them as 5 doubles to o
__device__ void sigma_cta_sums(float sh, float sl, float rh, float rl, int n1, int n3, int np, double *o) {
  __shared__ float2 wf[2][32];
  __shared__ int wi[3][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float e;
    float oh = __shfl_down_sync(0xffffffffu, sh, o), ol = __shfl_down_sync(0xffffffffu, sl, o);
    sh = ff_two_sum(sh, oh, e);
    sl = __fadd_rn(sl, __fadd_rn(e, ol));
    oh = __shfl_down_sync(0xffffffffu, rh, o);
    ol = __shfl_down_sync(0xffffffffu, rl, o);
    rh = ff_two_sum(rh, oh, e);
    rl = __fadd_rn(rl, __fadd_rn(e, ol));
    n1 += __shfl_down_sync(0xffffffffu, n1, o);
    n3 += __shfl_down_sync(0xffffffffu, n3, o);
    np += __shfl_down_sync(0xffffffffu, np, o);
  }
  if (lane == 0) {
    wf[0][wid] = make_float2(sh, sl);
    wf[1][wid] = make_float2(rh, rl);
    wi[0][wid] = n1; wi[1][wid] = n3; wi[2][wid] = np;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 a = wf[0][0], b = wf[1][0];
    long long c1 = wi[0][0], c3 = wi[1][0], cp = wi[2][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      a = ff_add(a, wf[0][w]);
      b = ff_add(b, wf[1][w]);
      c1 += wi[0][w]; c3 += wi[1][w]; cp += wi[2][w];
    }
    o[0] = ff_to_double(a);
    o[1] = (double)c1;
    o[2] = ff_to_double(b);
    o[3] = (double)c3;
    o[4] = (double)cp;
  }
}

// the sigma_0 sums of the current state into pinned host memory (no
// synchronisation; capturable): 5 doubles at ctx->h_pinned_d
rpba_status sigma0_launch(Ctx *ctx) {
  View v = make_view(ctx);
  int nb = ctx->red_blocks;
  if (ctx->opt.precision == 1) {
    if (ctx->cd == 8) RPBA_KERNEL(ctx, "k_obs_sigma_f", k_obs_sigma_f<true><<<nb, 256, 0, ctx->stream>>>(v, ctx->red));
    else RPBA_KERNEL(ctx, "k_obs_sigma_f", k_obs_sigma_f<false><<<nb, 256, 0, ctx->stream>>>(v, ctx->red));
  } else {
    RPBA_KERNEL(ctx, "k_obs_sigma", k_obs_sigma<<<nb, 256, 0, ctx->stream>>>(v, ctx->red));
  }
  RPBA_KERNEL(ctx, "k_sum_partials", k_sum_partials<5><<<1, 256, 0, ctx->stream>>>(ctx->red, nb, ctx->red + 5 * nb));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_d, ctx->red + 5 * nb, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
  return RPBA_OK;
}

// sigma_0 (Eq. sigma0), RMS and the active counts from the sums of
// sigma0_launch, after the stream has been synchronised
void sigma0_finish(const Ctx *ctx, double *sigma0, double *rms, long long *n_obs, long long *n_points) {
  const double *h = ctx->h_pinned_d;
  double red = 2.0 * h[1] - (double)ctx->cd * ctx->M - 3.0 * h[4] + 7.0;
  if (red < 1.0) red = 1.0;
  if (sigma0) *sigma0 = sqrt(h[0] / red);
  if (rms) *rms = h[3] > 0 ? sqrt(h[2] / (2.0 * h[3])) : 0.0;
  if (n_obs) *n_obs = (long long)h[1];
  if (n_points) *n_points = (long long)h[4];
}

rpba_status launch_sigma0(Ctx *ctx, double *sigma0, double *rms, long long *n_obs, long long *n_points) {
  RPBA_TRY(sigma0_launch(ctx));
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  sigma0_finish(ctx, sigma0, rms, n_obs, n_points);
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// intersection (Eq. bars) and refined weights (Sec. 5.1)
// ---------------------------------------------------------------------------
// N_j and g_j of point j over all its observations in FP64 at the FP64 X_j
// (Eq. bars); false when an observation lies behind its camera
__device__ __noinline__ bool point_normal_fp64(const View &v, int j, double *N, double *g) {
  for (int e = 0; e < 6; e++) N[e] = 0.0;
  for (int e = 0; e < 3; e++) g[e] = 0.0;
  bool ok = true;
  for (int a = v.pt_inst_ptr[j]; a < v.pt_inst_ptr[j + 1]; a++) {
    int q = v.pt_inst[a];
    for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) {
      ProjX<double> pj;
      double z;
      proj_x<double>(v, v.obs_cam[k], v.X + 3 * (size_t)j, nullptr, nullptr, pj, z);
      if (!(z > 0.0)) { ok = false; continue; }
      ObsT<double> ob;
      load_obs<double>(v, k, ob);
      double r0 = pj.u - ob.x, r1 = pj.v - ob.y, a0[3], a1[3];
      for (int c = 0; c < 3; c++) {
        a0[c] = ob.w * (ob.W[0] * pj.Jx[c] + ob.W[1] * pj.Jx[3 + c]);
        a1[c] = ob.w * (ob.W[1] * pj.Jx[c] + ob.W[2] * pj.Jx[3 + c]);
      }
      for (int r = 0; r < 3; r++) {
        for (int c = r; c < 3; c++) N[s3idx(r, c)] += pj.Jx[r] * a0[c] + pj.Jx[3 + r] * a1[c];
        g[r] += a0[r] * r0 + a1[r] * r1;
      }
    }
  }
  return ok;
}

// per instance of a running point: partial normal matrix N^(l) (sym3) and
// gradient g^(l) at the current X_j, cameras fixed. flag bit: behind camera.
template <typename T>
__global__ void k_isect_inst(View v, const int *state, T *part) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= v.P) return;
  int j = v.inst_pt[q];
  if (state[j] != 1) return;
  T N[6] = {0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
  bool behind = false;
  for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) {
    int i = v.obs_cam[k];
    ProjX<T> pj;
    T z;
    proj_x<T>(v, i, v.X + 3 * j, v.X_hi + 3 * j, v.X_lo + 3 * j, pj, z);
    if (!(z > T(0))) { behind = true; continue; }
    ObsT<T> ob;
    load_obs<T>(v, k, ob);
    T r0 = pj.u - ob.x, r1 = pj.v - ob.y;
    // w W Jx (2x3)
    T a0[3], a1[3];
    for (int c = 0; c < 3; c++) {
      a0[c] = ob.w * (ob.W[0] * pj.Jx[c] + ob.W[1] * pj.Jx[3 + c]);
      a1[c] = ob.w * (ob.W[1] * pj.Jx[c] + ob.W[2] * pj.Jx[3 + c]);
    }
    for (int r = 0; r < 3; r++) {
      for (int c = r; c < 3; c++) N[s3idx(r, c)] += pj.Jx[r] * a0[c] + pj.Jx[3 + r] * a1[c];
      g[r] += a0[r] * r0 + a1[r] * r1;
    }
  }
  T *o = part + 10 * (size_t)q;
  for (int e = 0; e < 6; e++) o[e] = N[e];
  for (int e = 0; e < 3; e++) o[6 + e] = g[e];
  o[9] = behind ? T(-1) : T(v.inst_obs_ptr[q + 1] - v.inst_obs_ptr[q]);  // observation count
}

// per running point: sum the instance parts, Gauss-Newton update, checks,
// and on convergence W^l = N - N^(l) for every instance. Converged when
// ||dX|| <= tol (1 + ||X||) or when the step moves the point's image
// residuals by less than px_tol per observation: dX^T N dX <= px_tol^2 n_obs
// (reachable in FP32, whose residuals carry ~1e-4 px rounding).
// FP32 form: the 3x3 system is solved in FP32; when its Frobenius condition
// number exceeds 1e6, N_j and g_j are formed again in FP64 from the
// observations, and the cond_max test and the solve use those.
template <typename T>
__global__ void k_isect_point(View v, int *state, int *iter, const T *part, int max_iter, double tol,
                              double px_tol, double cond_max, int last) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.N || state[j] != 1) return;
  int q0 = v.pt_inst_ptr[j], q1 = v.pt_inst_ptr[j + 1];
  T N[6] = {0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
  bool behind = false;
  T nobs = 0;
  for (int a = q0; a < q1; a++) {
    const T *o = part + 10 * (size_t)v.pt_inst[a];
    for (int e = 0; e < 6; e++) N[e] += o[e];
    for (int e = 0; e < 3; e++) g[e] += o[6 + e];
    behind |= o[9] < T(0);
    nobs += o[9];
  }
  bool fail = behind;
  double d[3] = {0, 0, 0};
  float df[3] = {0.f, 0.f, 0.f};  // FP32 form: the step in FP32
  double nd2_img = 0.0;           // d^T N d (FP64 re-formation)
  T nd2T = T(-1);                 // d^T N d in the compute precision (else)
  if (!fail) {
    T inv[6];
    T det = sym3_inv<T>(N, inv);
    T cond = sym3_frob<T>(N) * sym3_frob<T>(inv);
    double Nimg[6];
    if (sizeof(T) == sizeof(float) && !(cond <= T(1e6))) {
      // FP32 sums round a nearly singular N_j into a better conditioned one,
      // so the cond_max test cannot be taken on them: N_j and g_j again in FP64
      double gd[3], invd[6];
      fail = !point_normal_fp64(v, j, Nimg, gd);
      double detd = sym3_inv<double>(Nimg, invd);
      fail = fail || !(detd > 0.0) || !(sym3_frob<double>(Nimg) * sym3_frob<double>(invd) <= cond_max);
      for (int r = 0; r < 3; r++) {
        d[r] = invd[s3idx(r, 0)] * gd[0] + invd[s3idx(r, 1)] * gd[1] + invd[s3idx(r, 2)] * gd[2];
        df[r] = (float)d[r];
      }
      if (px_tol > 0.0) {
        double Nd3[3];
        for (int r = 0; r < 3; r++) Nd3[r] = Nimg[s3idx(r, 0)] * d[0] + Nimg[s3idx(r, 1)] * d[1] + Nimg[s3idx(r, 2)] * d[2];
        nd2_img = d[0] * Nd3[0] + d[1] * Nd3[1] + d[2] * Nd3[2];
      }
    } else {
      // the step and its image-space size in the compute precision; only the
      // position update below is FP64
      fail = !(det > T(0)) || !(cond <= (T)cond_max);
      T dT[3];
      for (int r = 0; r < 3; r++) dT[r] = inv[s3idx(r, 0)] * g[0] + inv[s3idx(r, 1)] * g[1] + inv[s3idx(r, 2)] * g[2];
      if (px_tol > 0.0) {
        T Nd3[3];
        for (int r = 0; r < 3; r++) Nd3[r] = N[s3idx(r, 0)] * dT[0] + N[s3idx(r, 1)] * dT[1] + N[s3idx(r, 2)] * dT[2];
        nd2T = dT[0] * Nd3[0] + dT[1] * Nd3[1] + dT[2] * Nd3[2];
      }
      if constexpr (sizeof(T) == sizeof(float))
        for (int r = 0; r < 3; r++) df[r] = (float)dT[r];
      else
        for (int r = 0; r < 3; r++) d[r] = (double)dT[r];
    }
  }
  bool conv = false;
  if (!fail) {
    if constexpr (sizeof(T) == sizeof(float)) {
      // X - d on the hi + lo words in float-float; the FP64 copy from them
      float *xh = v.X_hi + 3 * j, *xl = v.X_lo + 3 * j;
      for (int r = 0; r < 3; r++) {
        float2 xn = ff_add(make_float2(xh[r], xl[r]), make_float2(-df[r], 0.f));
        xh[r] = xn.x;
        xl[r] = xn.y;
        v.X[3 * j + r] = ff_to_double(xn);
      }
      float nd = sqrtf(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
      float nx = sqrtf(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
      conv = nd <= (float)tol * (1.f + nx);
    } else {
      double Xn[3];
      for (int r = 0; r < 3; r++) Xn[r] = v.X[3 * j + r] - d[r];
      for (int r = 0; r < 3; r++) v.X[3 * j + r] = Xn[r];
      if (v.X_hi)  // FP32 form under its FP64 first intersection: the hi + lo mirror
        for (int r = 0; r < 3; r++) split(Xn[r], v.X_hi[3 * j + r], v.X_lo[3 * j + r]);
      double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double nx = sqrt(Xn[0] * Xn[0] + Xn[1] * Xn[1] + Xn[2] * Xn[2]);
      conv = nd <= tol * (1.0 + nx);
    }
    if (!conv && px_tol > 0.0)
      conv = nd2T >= T(0) ? nd2T <= (T)(px_tol * px_tol) * nobs : nd2_img <= px_tol * px_tol * (double)nobs;
  }
  int it = ++iter[j];
  if (!fail && !conv && (it >= max_iter || last)) fail = true;
  if (fail) {
    state[j] = 3;
    v.active[j] = 0;
    for (int a = q0; a < q1; a++)
      for (int e = 0; e < 6; e++) {
        v.Wl[6 * (size_t)v.pt_inst[a] + e] = 0.0;
        if (v.Wl32) v.Wl32[6 * (size_t)v.pt_inst[a] + e] = 0.f;
      }
  } else if (conv) {
    state[j] = 2;
    bool tp = (q1 - q0) >= 2;
    for (int a = q0; a < q1; a++) {
      int q = v.pt_inst[a];
      const T *o = part + 10 * (size_t)q;
      if constexpr (sizeof(T) == sizeof(float)) {
        // FP32 form: W^l as the float-float sum of the other instances' parts.
        // N - N^(l) in FP32 cancels when the other sub-blocks' observations are
        // down-weighted (w = 1e-4), and can lose positive semi-definiteness.
        float Wh[6] = {0, 0, 0, 0, 0, 0}, Wlo[6] = {0, 0, 0, 0, 0, 0};
        for (int b = q0; b < q1; b++) {
          if (b == a) continue;
          const T *ob = part + 10 * (size_t)v.pt_inst[b];
          for (int e = 0; e < 6; e++) ff_acc(Wh[e], Wlo[e], ob[e]);
        }
        for (int e = 0; e < 6; e++) {
          float2 w = make_float2(Wh[e], Wlo[e]);
          double wd = tp_weight(v, e, ff_to_double(w), (double)N[e]);
          v.Wl[6 * (size_t)q + e] = tp ? wd : 0.0;
          v.Wl32[6 * (size_t)q + e] = tp ? (v.wmode ? (float)wd : __fadd_rn(Wh[e], Wlo[e])) : 0.f;
        }
      } else {
        for (int e = 0; e < 6; e++)
          v.Wl[6 * (size_t)q + e] = tp ? tp_weight(v, e, (double)(N[e] - o[e]), (double)N[e]) : 0.0;
        if (v.Wl32)
          for (int e = 0; e < 6; e++)
            v.Wl32[6 * (size_t)q + e] = tp ? (float)tp_weight(v, e, (double)(N[e] - o[e]), (double)N[e]) : 0.f;
      }
    }
  }
}

// FP32 form, one Gauss-Newton iteration of Eq. bars for one point (the
// kernel below runs them all in one launch): N_j and g_j over all the point's observations at the
// current X_j (hi + lo), the FP32 solve with the same checks, FP64
// re-formation and convergence tests as k_isect_point, the position update
// in float-float. On convergence the refined weights W^l = N_j - N_j^(l):
// N_j is also summed in float-float, each instance's part N_j^(l) formed again
// from its observations, and the difference taken in float-float (the FP32
// difference would cancel when the other sub-blocks' observations are
// down-weighted).
__device__ inline void isect_obs_acc(const View &v, int j, int k, float N[6], float g[3], bool &behind) {
  ProjX<float> pj;
  float z;
  proj_x<float>(v, v.obs_cam[k], nullptr, v.X_hi + 3 * (size_t)j, v.X_lo + 3 * (size_t)j, pj, z);
  if (!(z > 0.f)) { behind = true; return; }
  ObsT<float> ob;
  load_obs<float>(v, k, ob);
  float r0 = pj.u - ob.x, r1 = pj.v - ob.y, a0[3], a1[3];
  for (int c = 0; c < 3; c++) {
    a0[c] = ob.w * (ob.W[0] * pj.Jx[c] + ob.W[1] * pj.Jx[3 + c]);
    a1[c] = ob.w * (ob.W[1] * pj.Jx[c] + ob.W[2] * pj.Jx[3 + c]);
  }
  for (int r = 0; r < 3; r++) {
    for (int c = r; c < 3; c++) N[s3idx(r, c)] += pj.Jx[r] * a0[c] + pj.Jx[3 + r] * a1[c];
    g[r] += a0[r] * r0 + a1[r] * r1;
  }
}

__device__ static void isect_fused_step(const View &v, int j, int *state, int *iter, int max_iter, double tol,
                                        double px_tol, double cond_max, int last, int copies) {
  int q0 = v.pt_inst_ptr[j], q1 = v.pt_inst_ptr[j + 1];
  float N[6] = {0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
  float Nh[6] = {0, 0, 0, 0, 0, 0}, Nl[6] = {0, 0, 0, 0, 0, 0};  // N_j in float-float
  bool behind = false;
  float nobs = 0.f;
  const bool tp = (q1 - q0) >= 2;
  for (int a = q0; a < q1; a++) {
    int q = v.pt_inst[a];
    float Nq[6] = {0, 0, 0, 0, 0, 0};
    for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) isect_obs_acc(v, j, k, Nq, g, behind);
    for (int e = 0; e < 6; e++) { N[e] += Nq[e]; ff_acc(Nh[e], Nl[e], Nq[e]); }
    // each instance's part N_j^(l) waits in its W^l slot (this point's thread
    // alone touches it) until the refined weight is formed at convergence;
    // every point leaves the launch converged or failed, which overwrites it
    if (tp)
      for (int e = 0; e < 6; e++) v.Wl32[6 * (size_t)q + e] = Nq[e];
    nobs += (float)(v.inst_obs_ptr[q + 1] - v.inst_obs_ptr[q]);
  }
  bool fail = behind;
  float df[3] = {0.f, 0.f, 0.f};
  float nd2 = -1.f;        // d^T N d (FP32 solve)
  double nd2_img = 0.0;    // d^T N d (FP64 re-formation)
  if (!fail) {
    float inv[6];
    float det = sym3_inv<float>(N, inv);
    float cond = sym3_frob<float>(N) * sym3_frob<float>(inv);
    if (!(cond <= 1e6f)) {
      double Nimg[6], gd[3], invd[6];
      fail = !point_normal_fp64(v, j, Nimg, gd);
      double detd = sym3_inv<double>(Nimg, invd);
      fail = fail || !(detd > 0.0) || !(sym3_frob<double>(Nimg) * sym3_frob<double>(invd) <= cond_max);
      double d[3];
      for (int r = 0; r < 3; r++) {
        d[r] = invd[s3idx(r, 0)] * gd[0] + invd[s3idx(r, 1)] * gd[1] + invd[s3idx(r, 2)] * gd[2];
        df[r] = (float)d[r];
      }
      if (px_tol > 0.0) {
        double Nd3[3];
        for (int r = 0; r < 3; r++) Nd3[r] = Nimg[s3idx(r, 0)] * d[0] + Nimg[s3idx(r, 1)] * d[1] + Nimg[s3idx(r, 2)] * d[2];
        nd2_img = d[0] * Nd3[0] + d[1] * Nd3[1] + d[2] * Nd3[2];
      }
    } else {
      fail = !(det > 0.f) || !(cond <= (float)cond_max);
      for (int r = 0; r < 3; r++) df[r] = inv[s3idx(r, 0)] * g[0] + inv[s3idx(r, 1)] * g[1] + inv[s3idx(r, 2)] * g[2];
      if (px_tol > 0.0) {
        float Nd3[3];
        for (int r = 0; r < 3; r++) Nd3[r] = N[s3idx(r, 0)] * df[0] + N[s3idx(r, 1)] * df[1] + N[s3idx(r, 2)] * df[2];
        nd2 = df[0] * Nd3[0] + df[1] * Nd3[1] + df[2] * Nd3[2];
      }
    }
  }
  bool conv = false;
  if (!fail) {
    float *xh = v.X_hi + 3 * (size_t)j, *xl = v.X_lo + 3 * (size_t)j;
    for (int r = 0; r < 3; r++) {
      float2 xn = ff_add(make_float2(xh[r], xl[r]), make_float2(-df[r], 0.f));
      xh[r] = xn.x;
      xl[r] = xn.y;
      v.X[3 * (size_t)j + r] = ff_to_double(xn);
    }
    float nd = sqrtf(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
    float nx = sqrtf(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
    conv = nd <= (float)tol * (1.f + nx);
    if (!conv && px_tol > 0.0)
      conv = nd2 >= 0.f ? nd2 <= (float)(px_tol * px_tol) * nobs : nd2_img <= px_tol * px_tol * (double)nobs;
  }
  int it = ++iter[j];
  if (!fail && !conv && (it >= max_iter || last)) fail = true;
  if (fail) {
    state[j] = 3;
    v.active[j] = 0;
    for (int a = q0; a < q1; a++)
      for (int e = 0; e < 6; e++) {
        v.Wl[6 * (size_t)v.pt_inst[a] + e] = 0.0;
        v.Wl32[6 * (size_t)v.pt_inst[a] + e] = 0.f;
      }
  } else if (conv) {
    state[j] = 2;
    for (int a = q0; a < q1; a++) {
      int q = v.pt_inst[a];
      if (!tp) {
        for (int e = 0; e < 6; e++) { v.Wl[6 * (size_t)q + e] = 0.0; v.Wl32[6 * (size_t)q + e] = 0.f; }
        continue;
      }
      // this instance's part at the same (pre-step) X as N_j: the one this
      // pass left in the W^l slot
      float Nq[6];
      for (int e = 0; e < 6; e++) Nq[e] = v.Wl32[6 * (size_t)q + e];
      for (int e = 0; e < 6; e++) {
        float2 w = ff_add(make_float2(Nh[e], Nl[e]), make_float2(-Nq[e], 0.f));
        if (v.wmode) {
          double wd = tp_weight(v, e, 0.0, ff_to_double(make_float2(Nh[e], Nl[e])));
          v.Wl[6 * (size_t)q + e] = wd;
          v.Wl32[6 * (size_t)q + e] = (float)wd;
        } else {
          v.Wl[6 * (size_t)q + e] = ff_to_double(w);
          v.Wl32[6 * (size_t)q + e] = __fadd_rn(w.x, w.y);
        }
      }
      if (copies)  // the TP copies restart at X_TP (as k_tp_copies writes them)
        for (int e = 0; e < 3; e++) {
          v.Xl[3 * (size_t)q + e] = v.X[3 * (size_t)j + e];
          v.Xl_hi[3 * (size_t)q + e] = v.X_hi[3 * (size_t)j + e];
          v.Xl_lo[3 * (size_t)q + e] = v.X_lo[3 * (size_t)j + e];
        }
    }
  }
}

// the points are independent (cameras fixed): each thread runs its point's
// Gauss-Newton iterations to convergence or failure in one launch. With a
// list (the TP intersection) the threads cover the listed points only, so no
// warp lane idles on a point that is not intersected; pt_mask given: the
// listed points (all TPs) set their own start state, in place of
// k_isect_start. copies: a converged TP also restarts its sub-block copies
// X^l at X_TP, in place of k_tp_copies.
__global__ void k_isect_fused_f(View v, const int *list, int n, const uint8_t *pt_mask, int copies, int *state,
                                int *iter, int max_iter, double tol, double px_tol, double cond_max) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int j = list ? list[t] : t;
  if (pt_mask) {
    state[j] = (v.active[j] && pt_mask[j]) ? 1 : 0;
    iter[j] = 0;
  }
  for (int pass = 0; pass < max_iter && state[j] == 1; pass++)
    isect_fused_step(v, j, state, iter, max_iter, tol, px_tol, cond_max, pass == max_iter - 1, copies);
}

__global__ void k_isect_start(View v, const uint8_t *pt_mask, int *state, int *iter, int tp_only, int *count) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.N) return;
  int nq = v.pt_inst_ptr[j + 1] - v.pt_inst_ptr[j];
  int s = (v.active[j] && (!tp_only || nq >= 2) && pt_mask[j]) ? 1 : 0;
  state[j] = s;
  iter[j] = 0;
  if (s) atomicAdd(count, 1);
}

__global__ void k_isect_count(const int *state, int n, int *running, int *failed) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (state[j] == 1) atomicAdd(running, 1);
  if (state[j] == 3) atomicAdd(failed, 1);
}

rpba_status launch_intersect(Ctx *ctx, int tp_only, int *n_dropped, bool fp64, bool tp_copies) {
  View v = make_view(ctx);
  if (ctx->N == 0) { if (n_dropped) *n_dropped = 0; return RPBA_OK; }
  const bool fused = ctx->opt.precision == 1 && !fp64;
  // the TP list launch sets its points' start states itself unless the
  // dropped points are counted afterwards (that count reads every state)
  const bool own_start = fused && tp_only && !n_dropped;
  if (!own_start) {
    RPBA_CUDA(cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(int), ctx->stream));
    RPBA_KERNEL(ctx, "k_isect_start", k_isect_start<<<nblk(ctx->N, 256), 256, 0, ctx->stream>>>(
                                          v, ctx->pt_mask, ctx->isect_state, ctx->isect_iter, tp_only, ctx->counters));
  }
  int maxit = ctx->opt.isect_max_iter;
  double tol = ctx->opt.isect_tol;
  double px_tol = ctx->opt.isect_px_tol;
  if (fused) {  // FP32 form: every point's iterations in one launch
    const int *list = tp_only ? ctx->tp_list : nullptr;
    int n = tp_only ? ctx->n_tp : ctx->N;
    if (n)
      RPBA_KERNEL(ctx, "k_isect_fused_f", k_isect_fused_f<<<nblk(n, ctx->tune.isect), ctx->tune.isect, 0, ctx->stream>>>(
                                            v, list, n, own_start ? ctx->pt_mask : nullptr, tp_copies && tp_only ? 1 : 0,
                                            ctx->isect_state, ctx->isect_iter, maxit, tol, px_tol,
                                            ctx->opt.cond_max));
  } else {
    for (int it = 0; it < maxit; it++) {
      RPBA_KERNEL(ctx, "k_isect_inst", k_isect_inst<double><<<nblk(ctx->P, 128), 128, 0, ctx->stream>>>(
                                           v, ctx->isect_state, ctx->isect_N));
      RPBA_KERNEL(ctx, "k_isect_point", k_isect_point<double><<<nblk(ctx->N, 256), 256, 0, ctx->stream>>>(
                                            v, ctx->isect_state, ctx->isect_iter, ctx->isect_N, maxit, tol, px_tol,
                                            ctx->opt.cond_max, it == maxit - 1));
    }
  }
  if (!n_dropped) return RPBA_OK;  // no count wanted: no host synchronisation
  RPBA_CUDA(cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(int), ctx->stream));
  RPBA_KERNEL(ctx, "k_isect_count", k_isect_count<<<nblk(ctx->N, 256), 256, 0, ctx->stream>>>(
                                        ctx->isect_state, ctx->N, ctx->counters, ctx->counters + 1));
  int h[2];
  RPBA_CUDA(cudaMemcpyAsync(h, ctx->counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  *n_dropped = h[1];
  return RPBA_OK;
}

// exchange after bact: points seen in one sub-block take that sub-block's copy
__global__ void k_exchange(View v) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.N || !v.active[j]) return;
  int q0 = v.pt_inst_ptr[j];
  if (v.pt_inst_ptr[j + 1] - q0 != 1) return;
  int q = v.pt_inst[q0];
  for (int e = 0; e < 3; e++) v.X[3 * j + e] = v.Xl[3 * (size_t)q + e];
  if (v.X_hi)
    for (int e = 0; e < 3; e++) {
      v.X_hi[3 * j + e] = v.Xl_hi[3 * (size_t)q + e];
      v.X_lo[3 * j + e] = v.Xl_lo[3 * (size_t)q + e];
    }
}

// sub-block copies restart at the intersected position
__global__ void k_tp_copies(View v, int tp_only) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= v.P) return;
  int j = v.inst_pt[q];
  if (tp_only && v.pt_inst_ptr[j + 1] - v.pt_inst_ptr[j] < 2) return;
  for (int e = 0; e < 3; e++) v.Xl[3 * (size_t)q + e] = v.X[3 * j + e];
  if (v.Xl_hi)
    for (int e = 0; e < 3; e++) {
      v.Xl_hi[3 * (size_t)q + e] = v.X_hi[3 * j + e];
      v.Xl_lo[3 * (size_t)q + e] = v.X_lo[3 * j + e];
    }
}

rpba_status launch_exchange(Ctx *ctx) {
  if (ctx->N == 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_exchange", k_exchange<<<nblk(ctx->N, 256), 256, 0, ctx->stream>>>(make_view(ctx)));
  return RPBA_OK;
}

rpba_status launch_tp_copies(Ctx *ctx, int tp_only) {
  if (ctx->P == 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_tp_copies", k_tp_copies<<<nblk(ctx->P, 256), 256, 0, ctx->stream>>>(make_view(ctx), tp_only));
  return RPBA_OK;
}

// robust weights from the per-camera scale (Sec. 5.3)
__global__ void k_robust_weights(View v, const double *sigma, double t_v, double dw, int *count) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  int j = v.obs_pt[k];
  if (!v.active[j]) return;
  int i = v.obs_cam[k];
  double pu, pv;
  proj64(v.R + 9 * i, v.t + 3 * i, v.intr[3 * i], v.k1 ? v.k1[i] : 0.0, v.intr[3 * i + 1], v.intr[3 * i + 2],
         v.X + 3 * j, pu, pv);
  double r0 = pu - v.obs_xy[2 * k];
  double r1 = pv - v.obs_xy[2 * k + 1];
  double W0 = 1, W1 = 0, W2 = 1;
  if (v.has_winv) { W0 = v.obs_winv[3 * k]; W1 = v.obs_winv[3 * k + 1]; W2 = v.obs_winv[3 * k + 2]; }
  double nr = sqrt(W0 * r0 * r0 + 2.0 * W1 * r0 * r1 + W2 * r1 * r1);
  double s = sigma[i];
  bool out = (s > 0.0) && (nr / s > t_v);
  v.obs_w[k] = out ? dw : 1.0;
  if (v.obs_w32) v.obs_w32[k] = out ? (float)dw : 1.0f;
  if (out) atomicAdd(count, 1);
}

// FP32 form: float-float residual, the test |v|_W > t_v sigma_i in FP32.
// A separate pass in observation order: written from the per-camera scale
// kernel the weights would scatter over the observation-ordered arrays
// (measured slower on the 20M-observation block).
template <bool K1>
__global__ void k_robust_weights_f(View v, const float *sigma, float t_v, double dw, int *count) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  int j = v.obs_pt[k];
  int i = v.obs_cam[k];
  const bool act = v.active[j] != 0;  // read beside the residual's gathers, not before them
  float r0, r1;
  ff_residual(v.camff + FF_CAM * (size_t)i, v.X_hi + 3 * (size_t)j, v.X_lo + 3 * (size_t)j, v.obs_xy32[2 * k],
              v.obs_xylo[2 * k], v.obs_xy32[2 * k + 1], v.obs_xylo[2 * k + 1], r0, r1, K1);
  if (!act) return;
  float W0 = 1.f, W1 = 0.f, W2 = 1.f;
  if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
  float nr = sqrtf(W0 * r0 * r0 + 2.f * W1 * r0 * r1 + W2 * r1 * r1);
  float s = sigma[i];
  bool out = (s > 0.f) && (nr > t_v * s);
  v.obs_w[k] = out ? dw : 1.0;
  v.obs_w32[k] = out ? (float)dw : 1.0f;
  if (out) atomicAdd(count, 1);
}

rpba_status launch_robust_weights(Ctx *ctx, int *n_down) {
  RPBA_TRY(launch_camera_scale(ctx));
  RPBA_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(int), ctx->stream));
  if (ctx->K && ctx->opt.precision == 1) {
    dim3 g(nblk(ctx->K, ctx->tune.robust)), b(ctx->tune.robust);
    if (ctx->cd == 8)
      RPBA_KERNEL(ctx, "k_robust_weights_f", k_robust_weights_f<true><<<g, b, 0, ctx->stream>>>(
                                               make_view(ctx), ctx->cam_sigma32, (float)ctx->opt.t_v,
                                               ctx->opt.downweight, ctx->counters));
    else
      RPBA_KERNEL(ctx, "k_robust_weights_f", k_robust_weights_f<false><<<g, b, 0, ctx->stream>>>(
                                               make_view(ctx), ctx->cam_sigma32, (float)ctx->opt.t_v,
                                               ctx->opt.downweight, ctx->counters));
  }
  else if (ctx->K)
    RPBA_KERNEL(ctx, "k_robust_weights", k_robust_weights<<<nblk(ctx->K, ctx->tune.robust), ctx->tune.robust, 0, ctx->stream>>>(make_view(ctx), ctx->cam_sigma, ctx->opt.t_v,
                                                                ctx->opt.downweight, ctx->counters));
  if (n_down) {
    RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter, ctx->counters, sizeof(int), cudaMemcpyDeviceToHost,
                              ctx->stream));
    RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
    *n_down = ctx->h_pinned_counter[0];
  }
  return RPBA_OK;
}

__global__ void k_eliminate(View v) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  if (v.obs_w[k] != 1.0) v.active[v.obs_pt[k]] = 0;
}

// serial robust variant (Sec. 5.3): the down-weighted observations are
// deleted (weight 0)
__global__ void k_delete_obs(View v) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  if (v.obs_w[k] != 1.0) {
    v.obs_w[k] = 0.0;
    if (v.obs_w32) v.obs_w32[k] = 0.f;
  }
}

// ... and a point seen by fewer than two cameras afterwards is eliminated
__global__ void k_eliminate_thin(View v) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= v.N || !v.active[j]) return;
  int kept = 0;
  for (int a = v.pt_inst_ptr[j]; a < v.pt_inst_ptr[j + 1]; a++) {
    int q = v.pt_inst[a];
    for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) kept += v.obs_w[k] == 1.0 ? 1 : 0;
  }
  if (kept < 2) v.active[j] = 0;
}

rpba_status launch_eliminate(Ctx *ctx) {
  if (!ctx->K) return RPBA_OK;
  if (ctx->opt.robust_serial) {
    RPBA_KERNEL(ctx, "k_delete_obs", k_delete_obs<<<nblk(ctx->K, 256), 256, 0, ctx->stream>>>(make_view(ctx)));
    if (ctx->N)
      RPBA_KERNEL(ctx, "k_eliminate_thin",
                  k_eliminate_thin<<<nblk(ctx->N, 256), 256, 0, ctx->stream>>>(make_view(ctx)));
    return RPBA_OK;
  }
  RPBA_KERNEL(ctx, "k_eliminate", k_eliminate<<<nblk(ctx->K, 256), 256, 0, ctx->stream>>>(make_view(ctx)));
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// sub-block cost F_l (Eq. bact): one thread per observation (its weighted
// squared residual; the first observation of an instance adds the TP control
// term), then a deterministic two-stage sum over each sub-block's contiguous
// observation range. An observation behind its camera contributes +inf, so
// the trial is rejected.
// ---------------------------------------------------------------------------
// trial = 1 evaluates the trial cameras/instances of running sub-blocks
__global__ void k_obs_cost(View v, int trial, const int *run, double *cost) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.K) return;
  int q = v.obs_inst[k];
  int l = v.inst_sub[q];
  int j = v.inst_pt[q];
  if ((run && !run[l]) || !v.active[j]) { cost[k] = 0.0; return; }
  int i = v.obs_cam[k];
  const double *R = (trial ? v.Rt : v.R) + 9 * i;
  const double *t = (trial ? v.tt : v.t) + 3 * i;
  const double *Xq = (trial ? v.Xlt : v.Xl) + 3 * (size_t)q;
  double f = (trial && v.ft) ? v.ft[i] : v.intr[3 * i];
  double k1 = v.k1 ? (trial ? v.k1t[i] : v.k1[i]) : 0.0;
  double pu, pv;
  double zc = proj64(R, t, f, k1, v.intr[3 * i + 1], v.intr[3 * i + 2], Xq, pu, pv);
  double F;
  if (!(zc > 0.0)) {
    F = INFINITY;
  } else {
    double r0 = pu - v.obs_xy[2 * k];
    double r1 = pv - v.obs_xy[2 * k + 1];
    double W0 = 1, W1 = 0, W2 = 1;
    if (v.has_winv) { W0 = v.obs_winv[3 * k]; W1 = v.obs_winv[3 * k + 1]; W2 = v.obs_winv[3 * k + 2]; }
    F = v.obs_w[k] * (W0 * r0 * r0 + 2.0 * W1 * r0 * r1 + W2 * r1 * r1);
  }
  if (k == v.inst_obs_ptr[q]) {
    // TP control term (X^l - X_TP)^T W^l (X^l - X_TP)
    const double *W = v.Wl + 6 * (size_t)q;
    double d[3] = {Xq[0] - v.X[3 * j], Xq[1] - v.X[3 * j + 1], Xq[2] - v.X[3 * j + 2]};
    F += W[0] * d[0] * d[0] + W[3] * d[1] * d[1] + W[5] * d[2] * d[2] +
         2.0 * (W[1] * d[0] * d[1] + W[2] * d[0] * d[2] + W[4] * d[1] * d[2]);
  }
  cost[k] = F;
}

// the sigma_0 sums of one thread (FP32 form): sum w v^T W v and sum |v|^2
// (w == 1) in float-float, the counts of active and of w == 1 observations
struct SigmaAcc {
  float sh = 0.f, sl = 0.f, rh = 0.f, rl = 0.f;
  int n1 = 0, n3 = 0;
};

// FP32 form: the observation's term from its float-float residual, formed
// in FP32 and stored in FP64 for the FP64 sum; the TP control term from the
// float-float difference X^l - X_TP and W^l in FP32. With SIG the same
// residual also feeds the observation's sigma_0 terms (Eq. sigma0: every
// observation of an active point that is not deleted, whatever its depth)
// The loads do not wait for the point's active flag: the observation's point,
// camera and instance come from its own streams, so every gather of the term
// issues after one dependent load; an inactive point's term is dropped at the
// end.
template <bool SIG, bool K1>
__device__ inline float obs_cost_term_f(const View &v, int trial, int k, SigmaAcc *sig = nullptr,
                                       const float4 *cam_s = nullptr) {
  int q = v.obs_inst[k];
  int j = v.obs_pt[k];  // = inst_pt[q]
  const bool act = v.active[j] != 0;
  const float *Xh = (trial ? v.Xlt_hi : v.Xl_hi) + 3 * (size_t)q;
  const float *Xw = (trial ? v.Xlt_lo : v.Xl_lo) + 3 * (size_t)q;
  float c[28];
  if (cam_s)  // the sub-block's records staged in shared memory
    ff_load_record_s(cam_s + FF_CAM_S * (int)v.obs_camloc[k], c);
  else
    ff_load_record<7>((trial ? v.camff_t : v.camff) + FF_CAM * (size_t)v.obs_cam[k], c);
  float r0, r1;
  float F;
  bool front = ff_residual_rec(c, Xh, Xw, v.obs_xy32[2 * k], v.obs_xylo[2 * k], v.obs_xy32[2 * k + 1],
                               v.obs_xylo[2 * k + 1], r0, r1, K1);
  if (!front && !SIG) {
    F = INFINITY;
  } else {
    float W0 = 1.f, W1 = 0.f, W2 = 1.f;
    if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
    float w = v.obs_w32[k];
    F = w * (W0 * r0 * r0 + 2.f * W1 * r0 * r1 + W2 * r1 * r1);
    if constexpr (SIG) {
      if (act && w != 0.f) {  // w = 0: deleted by the serial robust variant
        float e;
        sig->sh = ff_two_sum(sig->sh, F, e);
        sig->sl += e;
        sig->n1++;
        if (w == 1.f) {
          sig->rh = ff_two_sum(sig->rh, r0 * r0 + r1 * r1, e);
          sig->rl += e;
          sig->n3++;
        }
      }
      if (!front) F = INFINITY;
    }
  }
  if (k == v.inst_obs_ptr[q]) {
    const float *W = v.Wl32 + 6 * (size_t)q;
    float d[3];
    for (int e = 0; e < 3; e++)
      d[e] = __fadd_rn(__fsub_rn(Xh[e], v.X_hi[3 * (size_t)j + e]), __fsub_rn(Xw[e], v.X_lo[3 * (size_t)j + e]));
    F += W[0] * d[0] * d[0] + W[3] * d[1] * d[1] + W[5] * d[2] * d[2] +
         2.f * (W[1] * d[0] * d[1] + W[2] * d[0] * d[2] + W[4] * d[1] * d[2]);
  }
  return act ? F : 0.f;
}

// FP32 form, F_l in two deterministic stages without a per-observation array:
// one CTA per chunk (<= 256 observations of one sub-block, one per thread)
// writes its sum, then one CTA per sub-block adds its chunks' sums in order.
// With SIG (at a state where every X^l equals its X) the chunk also writes
// its 5 sigma_0 sums to sig (the active points counted over a grid stride)
template <bool SIG, bool K1>
__global__ void __launch_bounds__(256) k_cost_chunks_f(View v, int trial, const int *run, const int *chunk_sub,
                                                       const int *chunk_start, const int *sub_obs_ptr, double *part,
                                                       double *sig) {
  __shared__ float2 ws[8];
  int c = blockIdx.x, l = chunk_sub[c];
  if (run && !run[l]) return;
  int k = chunk_start[c] + threadIdx.x;
  SigmaAcc acc;
  float F = k < sub_obs_ptr[l + 1] ? obs_cost_term_f<SIG, K1>(v, trial, k, &acc) : 0.f;
  // a point behind its camera makes the sum +inf (TwoSum would turn it into NaN)
  int any_inf = __syncthreads_or(isinf(F));
  float h = any_inf ? 0.f : F, lo = 0.f;  // float-float sum: off the FP64 pipe
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, lo, o);
    float e;
    h = ff_two_sum(h, oh, e);
    lo = __fadd_rn(lo, __fadd_rn(e, ol));
  }
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_float2(h, lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = ws[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) t = ff_add(t, ws[w]);
    part[c] = any_inf ? (double)INFINITY : ff_to_double(t);
  }
  if constexpr (SIG) {
    int np = 0;
    for (int j = c * blockDim.x + threadIdx.x; j < v.N; j += gridDim.x * blockDim.x) np += v.active[j] ? 1 : 0;
    sigma_cta_sums(acc.sh, acc.sl, acc.rh, acc.rl, acc.n1, acc.n3, np, sig + 5 * (size_t)c);
  }
}

// The same sums with the sub-block's camera records staged in shared memory
// once per CTA: a CTA takes up to RPBA_COST_GROUP consecutive chunks of one
// sub-block (group_chunk: the first chunk of each group) and writes every
// chunk's sums as k_cost_chunks_f does, so the results are the same. In the
// observations' (sub-block, point) order the 32 lanes of a warp read ~32
// different cameras: gathered from global memory each camera-record load
// touches 32 cache lines, staged it is one coalesced copy of the sub-block's
// records (~112 B per camera) per group.
static_assert(FF_CAM_S * 16 == RPBA_CAM_STAGE_BYTES, "staged camera record size");
template <bool SIG, bool K1>
__global__ void __launch_bounds__(256) k_cost_groups_f(View v, int trial, const int *run, const int *group_chunk,
                                                       const int *chunk_sub, const int *chunk_start,
                                                       const int *sub_obs_ptr, const int *sub_chunk_ptr,
                                                       int n_chunks, double *part, double *sig) {
  extern __shared__ float4 cam_s[];  // the sub-block's records, FF_CAM_S float4 each
  __shared__ float2 ws[8];
  int c0 = group_chunk[blockIdx.x], l = chunk_sub[c0];
  if (run && !run[l]) return;
  int c1 = min(c0 + RPBA_COST_GROUP, sub_chunk_ptr[l + 1]);
  int g0 = v.sub_cam_ptr[l], nl = v.sub_cam_ptr[l + 1] - g0;
  const float *rec = trial ? v.camff_t : v.camff;
  for (int e = threadIdx.x; e < 7 * nl; e += blockDim.x) {
    int r = e / 7, p = e - 7 * r;
    cam_s[FF_CAM_S * r + p] = __ldg(reinterpret_cast<const float4 *>(rec + FF_CAM * (size_t)v.sub_cam[g0 + r]) + p);
  }
  __syncthreads();
  for (int c = c0; c < c1; c++) {
    int k = chunk_start[c] + threadIdx.x;
    SigmaAcc acc;
    float F = k < sub_obs_ptr[l + 1] ? obs_cost_term_f<SIG, K1>(v, trial, k, &acc, cam_s) : 0.f;
    int any_inf = __syncthreads_or(isinf(F));
    float h = any_inf ? 0.f : F, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, lo, o);
      float e;
      h = ff_two_sum(h, oh, e);
      lo = __fadd_rn(lo, __fadd_rn(e, ol));
    }
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_float2(h, lo);
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 t = ws[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) t = ff_add(t, ws[w]);
      part[c] = any_inf ? (double)INFINITY : ff_to_double(t);
    }
    if constexpr (SIG) {
      int np = 0;
      for (int j = c * 256 + threadIdx.x; j < v.N; j += n_chunks * 256) np += v.active[j] ? 1 : 0;
      sigma_cta_sums(acc.sh, acc.sl, acc.rh, acc.rl, acc.n1, acc.n3, np, sig + 5 * (size_t)c);
    } else {
      __syncthreads();  // ws is written again by the next chunk
    }
  }
}

// F_l from its chunks in order; with SIG also its chunks' sigma_0 sums
template <bool SIG>
__global__ void k_cost_sub_f(int L, const int *run, const int *sub_chunk_ptr, const double *part, double *F,
                             const double *sig, double *sig_sub) {
  int l = blockIdx.x;
  if (l >= L || (run && !run[l])) return;
  double acc[1] = {0.0};
  for (int c = sub_chunk_ptr[l] + threadIdx.x; c < sub_chunk_ptr[l + 1]; c += blockDim.x) acc[0] += part[c];
  block_reduce_store<1>(acc, F + l);
  if constexpr (SIG) {
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = sub_chunk_ptr[l] + threadIdx.x; c < sub_chunk_ptr[l + 1]; c += blockDim.x)
#pragma unroll
      for (int e = 0; e < 5; e++) s[e] += sig[5 * (size_t)c + e];
    block_reduce_store<5>(s, sig_sub + 5 * (size_t)l);
  }
}

#define SEG_CHUNKS 32
// stage 1: chunk g of sub-block l's observation range -> part[l][g]
__global__ void k_seg_partial(const int *seg_ptr, const int *run, const double *val, double *part) {
  int l = blockIdx.y, g = blockIdx.x;
  if (run && !run[l]) return;
  int a = seg_ptr[l], b = seg_ptr[l + 1];
  long long len = b - a;
  int c0 = a + (int)(len * g / SEG_CHUNKS), c1 = a + (int)(len * (g + 1) / SEG_CHUNKS);
  double acc[1] = {0.0};
  for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) acc[0] += val[k];
  block_reduce_store<1>(acc, part + (size_t)l * SEG_CHUNKS + g);
}

// stage 2: F[l] = sum of its chunks in order
__global__ void k_seg_final(int L, const int *run, const double *part, double *F) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L || (run && !run[l])) return;
  double s = 0.0;
  for (int g = 0; g < SEG_CHUNKS; g++) s += part[(size_t)l * SEG_CHUNKS + g];
  F[l] = s;
}

// The cost that decides acceptance needs residuals far more accurate than
// FP32 image coordinates give: FP32 residuals of ~1000 px coordinates carry
// ~1e-4 px rounding, which hides the last LM improvements. The FP64 form
// evaluates them in FP64; the FP32 form in float-float on the FP32 pipes
// (~1e-10 px), with each term then formed in FP32 and all sums in FP64.
// dst[p] = src[list[p]] for rows of w words
template <typename T>
__global__ void k_gather_rows(long long n, int w, const int *list, const T *src, T *dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * w) return;
  long long r = e / w;
  dst[e] = src[(long long)list[r] * w + (e - r * w)];
}

rpba_status camera_major_setup(Ctx *ctx) {
  long long K = ctx->K;
  if (ctx->opt.precision != 1 || K == 0) return RPBA_OK;
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_pt, K * sizeof(int)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_inst, K * sizeof(int)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_xy32, 2 * K * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_xylo, 2 * K * sizeof(float)));
  auto g = [&](auto *src, auto *dst, int w, const char *what) -> rpba_status {
    RPBA_KERNEL(ctx, what, (k_gather_rows<<<nblk(K * w, 256), 256, 0, ctx->stream>>>(K, w, ctx->cam_obs, src, dst)));
    return RPBA_OK;
  };
  RPBA_TRY(g(ctx->obs_pt, ctx->cm_pt, 1, "k_gather_rows"));
  RPBA_TRY(g(ctx->obs_inst, ctx->cm_inst, 1, "k_gather_rows"));
  RPBA_TRY(g(ctx->obs_xy32, ctx->cm_xy32, 2, "k_gather_rows"));
  RPBA_TRY(g(ctx->obs_xylo, ctx->cm_xylo, 2, "k_gather_rows"));
  if (ctx->has_winv) {
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_winv32, 3 * K * sizeof(float)));
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->cm_whiten32, 3 * K * sizeof(float)));
    RPBA_TRY(g(ctx->obs_winv32, ctx->cm_winv32, 3, "k_gather_rows"));
    RPBA_TRY(g(ctx->obs_whiten32, ctx->cm_whiten32, 3, "k_gather_rows"));
  }
  return RPBA_OK;
}

rpba_status cost_groups_setup(Ctx *ctx) {
  if (ctx->cost_smem > 48 * 1024) {
    int b = (int)ctx->cost_smem;
    RPBA_CUDA(cudaFuncSetAttribute(k_cost_groups_f<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    RPBA_CUDA(cudaFuncSetAttribute(k_cost_groups_f<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    RPBA_CUDA(cudaFuncSetAttribute(k_cost_groups_f<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    RPBA_CUDA(cudaFuncSetAttribute(k_cost_groups_f<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
  }
  return RPBA_OK;
}

template <bool SIG>
static rpba_status cost_groups_launch(Ctx *ctx, const View &v, int trial, const int *run, double *sig) {
  auto kern = ctx->cd == 8 ? k_cost_groups_f<SIG, true> : k_cost_groups_f<SIG, false>;
  RPBA_KERNEL(ctx, "k_cost_groups_f", kern<<<ctx->n_groups, 256, ctx->cost_smem, ctx->stream>>>(
                                         v, trial, run, ctx->group_chunk, ctx->chunk_sub, ctx->chunk_start,
                                         ctx->sub_obs_ptr, ctx->sub_chunk_ptr, ctx->n_chunks, ctx->chunk_part, sig));
  return RPBA_OK;
}

static rpba_status sub_costs_impl(Ctx *ctx, int trial, const int *run, double *F_dev) {
  View v = make_view(ctx);
  if (ctx->opt.precision == 1) {
    if (ctx->n_groups)
      RPBA_TRY(cost_groups_launch<false>(ctx, v, trial, run, nullptr));
    else if (ctx->n_chunks && ctx->cd == 8)
      RPBA_KERNEL(ctx, "k_cost_chunks_f", k_cost_chunks_f<false, true><<<ctx->n_chunks, 256, 0, ctx->stream>>>(
                                         v, trial, run, ctx->chunk_sub, ctx->chunk_start, ctx->sub_obs_ptr,
                                         ctx->chunk_part, nullptr));
    else if (ctx->n_chunks)
      RPBA_KERNEL(ctx, "k_cost_chunks_f", k_cost_chunks_f<false, false><<<ctx->n_chunks, 256, 0, ctx->stream>>>(
                                         v, trial, run, ctx->chunk_sub, ctx->chunk_start, ctx->sub_obs_ptr,
                                         ctx->chunk_part, nullptr));
    if (ctx->L)
      RPBA_KERNEL(ctx, "k_cost_sub_f", k_cost_sub_f<false><<<ctx->L, 256, 0, ctx->stream>>>(
                                        ctx->L, run, ctx->sub_chunk_ptr, ctx->chunk_part, F_dev, nullptr, nullptr));
    return RPBA_OK;
  }
  if (ctx->K) {
    RPBA_KERNEL(ctx, "k_obs_cost", k_obs_cost<<<nblk(ctx->K, 256), 256, 0, ctx->stream>>>(v, trial, run, ctx->obs_cost));
  }
  RPBA_KERNEL(ctx, "k_seg_partial", k_seg_partial<<<dim3(SEG_CHUNKS, ctx->L), 256, 0, ctx->stream>>>(
                                        ctx->sub_obs_ptr, run, ctx->obs_cost, ctx->seg_part));
  RPBA_KERNEL(ctx, "k_seg_final", k_seg_final<<<nblk(ctx->L, 128), 128, 0, ctx->stream>>>(ctx->L, run, ctx->seg_part, F_dev));
  return RPBA_OK;
}

rpba_status launch_sub_costs(Ctx *ctx, int trial, double *F_dev) {
  return sub_costs_impl(ctx, trial, trial ? ctx->lm_run : nullptr, F_dev);
}

// FP32 form, at the end of the outer iteration's tail (after the exchange
// and the TP copies every instance's X^l equals its point's X, so the TP
// control terms vanish and F_l is the image part of sigma_0's sum over the
// sub-block): one pass over the observations gives every sub-block's cost
// (into f0_cache, for the next bact's start) and the sigma_0 sums (5 doubles
// into pinned host memory, like sigma0_launch). Capturable, no synchronisation.
rpba_status cost_sigma0_launch(Ctx *ctx) {
  if (ctx->opt.precision != 1 || !ctx->n_chunks || !ctx->L) return sigma0_launch(ctx);
  View v = make_view(ctx);
  double *sig_chunk = ctx->sigma0_part, *sig_sub = sig_chunk + 5 * (size_t)ctx->n_chunks;
  double *sig_tot = sig_sub + 5 * (size_t)ctx->L;
  if (ctx->n_groups)
    RPBA_TRY(cost_groups_launch<true>(ctx, v, 0, nullptr, sig_chunk));
  else if (ctx->cd == 8)
    RPBA_KERNEL(ctx, "k_cost_chunks_f", k_cost_chunks_f<true, true><<<ctx->n_chunks, 256, 0, ctx->stream>>>(
                                         v, 0, nullptr, ctx->chunk_sub, ctx->chunk_start, ctx->sub_obs_ptr,
                                         ctx->chunk_part, sig_chunk));
  else
    RPBA_KERNEL(ctx, "k_cost_chunks_f", k_cost_chunks_f<true, false><<<ctx->n_chunks, 256, 0, ctx->stream>>>(
                                         v, 0, nullptr, ctx->chunk_sub, ctx->chunk_start, ctx->sub_obs_ptr,
                                         ctx->chunk_part, sig_chunk));
  RPBA_KERNEL(ctx, "k_cost_sub_f", k_cost_sub_f<true><<<ctx->L, 256, 0, ctx->stream>>>(
                                    ctx->L, nullptr, ctx->sub_chunk_ptr, ctx->chunk_part, ctx->f0_cache, sig_chunk,
                                    sig_sub));
  RPBA_KERNEL(ctx, "k_sum_partials", k_sum_partials<5><<<1, 256, 0, ctx->stream>>>(sig_sub, ctx->L, sig_tot));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_d, sig_tot, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// normal equations of the sub-blocks and the Schur complement (Sec. 2, 5.5)
// ---------------------------------------------------------------------------
// N_XX (+ W^l, damped) and g_X of instance q in FP64 at its FP64 position
__device__ __noinline__ void instance_normal_fp64(const View &v, int q, double lam, double *N, double *g) {
  int j = v.inst_pt[q];
  const double *Xd = v.Xl + 3 * (size_t)q;
  for (int e = 0; e < 6; e++) N[e] = 0.0;
  for (int e = 0; e < 3; e++) g[e] = 0.0;
  for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) {
    ProjX<double> pj;
    double z;
    proj_x<double>(v, v.obs_cam[k], Xd, nullptr, nullptr, pj, z);
    ObsT<double> ob;
    load_obs<double>(v, k, ob);
    double r0 = pj.u - ob.x, r1 = pj.v - ob.y, a0[3], a1[3];
    for (int c = 0; c < 3; c++) {
      a0[c] = ob.w * (ob.W[0] * pj.Jx[c] + ob.W[1] * pj.Jx[3 + c]);
      a1[c] = ob.w * (ob.W[1] * pj.Jx[c] + ob.W[2] * pj.Jx[3 + c]);
    }
    for (int r = 0; r < 3; r++) {
      for (int c = r; c < 3; c++) N[s3idx(r, c)] += pj.Jx[r] * a0[c] + pj.Jx[3 + r] * a1[c];
      g[r] += a0[r] * r0 + a1[r] * r1;
    }
  }
  const double *Wq = v.Wl + 6 * (size_t)q;
  double d[3] = {Xd[0] - v.X[3 * j], Xd[1] - v.X[3 * j + 1], Xd[2] - v.X[3 * j + 2]};
  for (int e = 0; e < 6; e++) N[e] += Wq[e];
  for (int r = 0; r < 3; r++) g[r] += Wq[s3idx(r, 0)] * d[0] + Wq[s3idx(r, 1)] * d[1] + Wq[s3idx(r, 2)] * d[2];
  N[0] += lam * N[0]; N[3] += lam * N[3]; N[5] += lam * N[5];
}

// per instance: N_XX (+ W^l, damped), g_X, Ninv. FP64 form: also per
// observation N_XC = w A_X^T W A_C and Z = Ninv N_XC (both 3x6 row-major),
// read by the camera and Schur kernels. The FP32 form stores nothing per
// observation: its consumers form those blocks again in registers. FP32
// form: when the FP32 N_XX has a Frobenius condition number above 1e5, N_XX
// and g_X are formed again in FP64 and the FP64 inverse is rounded to FP32 (an
// FP32 inverse would be wrong in the weak direction).
template <typename T, int CD>
__global__ void k_linearize(View v, const double *lambda, const int *run, T *NXC, T *Z, T *Ninv_out,
                            T *gX_out) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= v.P) return;
  int l = v.inst_sub[q];
  if (!run[l]) return;
  int j = v.inst_pt[q];
  int k0 = v.inst_obs_ptr[q], k1 = v.inst_obs_ptr[q + 1];
  constexpr bool kStore = sizeof(T) == sizeof(double);
  if (!v.active[j]) {
    for (int e = 0; e < 6; e++) Ninv_out[6 * (size_t)q + e] = 0;
    for (int e = 0; e < 3; e++) gX_out[3 * (size_t)q + e] = 0;
    if (kStore)
      for (int k = k0; k < k1; k++)
        for (int e = 0; e < 3 * CD; e++) { NXC[3 * CD * (size_t)k + e] = 0; Z[3 * CD * (size_t)k + e] = 0; }
    return;
  }
  const double *Xd = v.Xl + 3 * (size_t)q;
  const float *Xh = v.Xl_hi + 3 * (size_t)q, *Xw = v.Xl_lo + 3 * (size_t)q;
  T N[6] = {0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
  for (int k = k0; k < k1; k++) {
    int i = v.obs_cam[k];
    ProjJac<T, CD> pj;
    T z;
    obs_proj<T, CD>(v, i, Xd, Xh, Xw, pj, z);
    ObsT<T> ob;
    load_obs<T>(v, k, ob);
    T r0 = pj.u - ob.x, r1 = pj.v - ob.y;
    T a0[3], a1[3];  // rows of w W A_X, transposed use
    for (int c = 0; c < 3; c++) {
      a0[c] = ob.w * (ob.W[0] * pj.Jx[c] + ob.W[1] * pj.Jx[3 + c]);
      a1[c] = ob.w * (ob.W[1] * pj.Jx[c] + ob.W[2] * pj.Jx[3 + c]);
    }
    for (int r = 0; r < 3; r++) {
      for (int c = r; c < 3; c++) N[s3idx(r, c)] += pj.Jx[r] * a0[c] + pj.Jx[3 + r] * a1[c];
      g[r] += a0[r] * r0 + a1[r] * r1;
    }
    if (kStore) {
      // N_XC = (w W A_X)^T A_C : row r (point coord) = a0[r] Jc[0,:] + a1[r] Jc[1,:]
      T *o = NXC + 3 * CD * (size_t)k;
      for (int r = 0; r < 3; r++)
        for (int c = 0; c < CD; c++) o[CD * r + c] = a0[r] * pj.Jc[c] + a1[r] * pj.Jc[CD + c];
    }
  }
  // TP control term
  if constexpr (sizeof(T) == sizeof(float)) {
    // X^l - X_TP from the hi + lo words (the leading parts cancel exactly), W^l in FP32
    const float *Wq = v.Wl32 + 6 * (size_t)q;
    float d[3];
    for (int e = 0; e < 3; e++)
      d[e] = __fadd_rn(__fsub_rn(Xh[e], v.X_hi[3 * (size_t)j + e]), __fsub_rn(Xw[e], v.X_lo[3 * (size_t)j + e]));
    for (int e = 0; e < 6; e++) N[e] += Wq[e];
    for (int r = 0; r < 3; r++) g[r] += Wq[s3idx(r, 0)] * d[0] + Wq[s3idx(r, 1)] * d[1] + Wq[s3idx(r, 2)] * d[2];
  } else {
    const double *Wq = v.Wl + 6 * (size_t)q;
    double d[3] = {Xd[0] - v.X[3 * j], Xd[1] - v.X[3 * j + 1], Xd[2] - v.X[3 * j + 2]};
    for (int e = 0; e < 6; e++) N[e] += Wq[e];
    for (int r = 0; r < 3; r++) g[r] += Wq[s3idx(r, 0)] * d[0] + Wq[s3idx(r, 1)] * d[1] + Wq[s3idx(r, 2)] * d[2];
  }
  // damping of the point block
  T lam = (T)lambda[l];
  N[0] += lam * N[0]; N[3] += lam * N[3]; N[5] += lam * N[5];
  T inv[6];
  T det = sym3_inv<T>(N, inv);
  if constexpr (sizeof(T) == sizeof(float)) {
    if (!(det > T(0)) || !(sym3_frob<T>(N) * sym3_frob<T>(inv) <= T(1e5))) {
      double Nd[6], gd[3], invd[6];
      instance_normal_fp64(v, q, lambda[l], Nd, gd);
      sym3_inv<double>(Nd, invd);
      for (int e = 0; e < 6; e++) inv[e] = (T)invd[e];
      for (int e = 0; e < 3; e++) g[e] = (T)gd[e];
    }
  }
  for (int e = 0; e < 6; e++) Ninv_out[6 * (size_t)q + e] = inv[e];
  for (int e = 0; e < 3; e++) gX_out[3 * (size_t)q + e] = g[e];
  if (kStore)
  for (int k = k0; k < k1; k++) {
    const T *B = NXC + 3 * CD * (size_t)k;
    T *o = Z + 3 * CD * (size_t)k;
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < CD; c++)
        o[CD * r + c] = inv[s3idx(r, 0)] * B[c] + inv[s3idx(r, 1)] * B[CD + c] + inv[s3idx(r, 2)] * B[2 * CD + c];
  }
}

// FP32 form: N_XC = (w W A_X)^T A_C of observation k (camera i, instance q)
// in registers, with the projection at the instance's X^l
template <int CD>
__device__ inline void nxc_f(const View &v, int i, int k, int q, float B[3 * CD]) {
  ProjJac<float, CD> pj;
  float z;
  obs_proj<float, CD>(v, i, nullptr, v.Xl_hi + 3 * (size_t)q, v.Xl_lo + 3 * (size_t)q, pj, z);
  float w = v.obs_w32[k], W0 = 1.f, W1 = 0.f, W2 = 1.f;
  if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
#pragma unroll
  for (int r = 0; r < 3; r++) {
    float a0 = w * (W0 * pj.Jx[r] + W1 * pj.Jx[3 + r]);
    float a1 = w * (W1 * pj.Jx[r] + W2 * pj.Jx[3 + r]);
#pragma unroll
    for (int c = 0; c < CD; c++) B[CD * r + c] = a0 * pj.Jc[c] + a1 * pj.Jc[CD + c];
  }
}

// the same with the camera's record in registers
template <int CD>
__device__ inline void nxc_f_rec(const View &v, const CamRecF &rec, int k, int q, float B[3 * CD]) {
  ProjJac<float, CD> pj;
  CamPt<float> cp;
  cam_point_rec(rec, v.Xl_hi + 3 * (size_t)q, v.Xl_lo + 3 * (size_t)q, cp);
  project_jac<float, CD>(cp.R, cp.Xc, cp.RX, cp.f, cp.k1, 0.f, 0.f, pj);
  float w = v.obs_w32[k], W0 = 1.f, W1 = 0.f, W2 = 1.f;
  if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
#pragma unroll
  for (int r = 0; r < 3; r++) {
    float a0 = w * (W0 * pj.Jx[r] + W1 * pj.Jx[3 + r]);
    float a1 = w * (W1 * pj.Jx[r] + W2 * pj.Jx[3 + r]);
#pragma unroll
    for (int c = 0; c < CD; c++) B[CD * r + c] = a0 * pj.Jc[c] + a1 * pj.Jc[CD + c];
  }
}

// Z = Ninv N_XC (3 x CD) with Ninv a packed symmetric 3x3
template <int CD>
__device__ inline void z_of(const float inv[6], const float B[3 * CD], float Zk[3 * CD]) {
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int c = 0; c < CD; c++)
      Zk[CD * r + c] = inv[s3idx(r, 0)] * B[c] + inv[s3idx(r, 1)] * B[CD + c] + inv[s3idx(r, 2)] * B[2 * CD + c];
}

// one CTA (CB_THREADS threads) per camera of a running sub-block: diagonal RCS block
//   S_ii = U_ii + lambda diag(U_ii) - sum_k N_XC,k^T Z_k,  U_ii = sum_k w A_C^T W A_C
// and right-hand side y_i = -sum_k w A_C^T W v + sum_k Z_k^T g_X
#define CB_THREADS 128
// one observation k (instance q) of camera i: its terms of U, SZ, gc and yz
// added to acc when act (the point is active)
template <typename T, int CD>
__device__ __forceinline__ void cb_obs_body(const View &v, int i, int k, int q, bool act, const ObsT<T> &ob,
                                            const T *NXC, const T *Z, const T *gX, const T *Ninv, T *acc);

template <typename T, int CD>
__device__ __forceinline__ void cb_obs(const View &v, int i, int k, int q, bool act, const T *NXC, const T *Z,
                                       const T *gX, const T *Ninv, T *acc) {
  ObsT<T> ob;
  load_obs<T>(v, k, ob);
  cb_obs_body<T, CD>(v, i, k, q, act, ob, NXC, Z, gX, Ninv, acc);
}

// FP32 form: the observation already loaded (from the camera-major streams)
template <typename T, int CD>
__device__ __forceinline__ void cb_obs_ob(const View &v, int i, int q, bool act, const ObsT<T> &ob, const T *Ninv,
                                          const T *gX, T *acc) {
  cb_obs_body<T, CD>(v, i, 0, q, act, ob, nullptr, nullptr, gX, Ninv, acc);
}

template <typename T, int CD>
__device__ __forceinline__ void cb_obs_body(const View &v, int i, int k, int q, bool act, const ObsT<T> &ob,
                                            const T *NXC, const T *Z, const T *gX, const T *Ninv, T *acc) {
  constexpr int NU = CD * (CD + 1) / 2;
  ProjJac<T, CD> pj;
  T z;
  obs_proj<T, CD>(v, i, v.Xl + 3 * (size_t)q, v.Xl_hi + 3 * (size_t)q, v.Xl_lo + 3 * (size_t)q, pj, z);
  T r0 = pj.u - ob.x, r1 = pj.v - ob.y;
  T b0[CD], b1[CD];  // w W A_C
#pragma unroll
  for (int c = 0; c < CD; c++) {
    b0[c] = ob.w * (ob.W[0] * pj.Jc[c] + ob.W[1] * pj.Jc[CD + c]);
    b1[c] = ob.w * (ob.W[1] * pj.Jc[c] + ob.W[2] * pj.Jc[CD + c]);
  }
  const T *gq = gX + 3 * (size_t)q;
  T Bl[3 * CD], Zl[3 * CD], g3[3] = {gq[0], gq[1], gq[2]};
  if constexpr (sizeof(T) == sizeof(float)) {  // N_XC and Z in registers
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < CD; c++) {
        T a0 = ob.w * (ob.W[0] * pj.Jx[r] + ob.W[1] * pj.Jx[3 + r]);
        T a1 = ob.w * (ob.W[1] * pj.Jx[r] + ob.W[2] * pj.Jx[3 + r]);
        Bl[CD * r + c] = a0 * pj.Jc[c] + a1 * pj.Jc[CD + c];
      }
    const float *iv = Ninv + 6 * (size_t)q;
    float inv[6] = {iv[0], iv[1], iv[2], iv[3], iv[4], iv[5]};
    z_of<CD>(inv, Bl, Zl);
  } else {
    const T *B = NXC + 3 * CD * (size_t)k, *Zk = Z + 3 * CD * (size_t)k;
#pragma unroll
    for (int e = 0; e < 3 * CD; e++) { Bl[e] = B[e]; Zl[e] = Zk[e]; }
  }
  if (!act) return;
  int e = 0;
#pragma unroll
  for (int r = 0; r < CD; r++) {
    acc[2 * NU + r] += b0[r] * r0 + b1[r] * r1;
    acc[2 * NU + CD + r] += Zl[r] * g3[0] + Zl[CD + r] * g3[1] + Zl[2 * CD + r] * g3[2];
#pragma unroll
    for (int c = r; c < CD; c++, e++) {
      acc[e] += pj.Jc[r] * b0[c] + pj.Jc[CD + r] * b1[c];
      acc[NU + e] += Bl[r] * Zl[c] + Bl[CD + r] * Zl[CD + c] + Bl[2 * CD + r] * Zl[2 * CD + c];
    }
  }
}

template <typename T, int CD>
__global__ void __launch_bounds__(CB_THREADS) k_camera_blocks(View v, const double *lambda, const int *run,
                                                              const T *NXC, const T *Z, const T *gX,
                                                              const T *Ninv) {
  constexpr int NU = CD * (CD + 1) / 2;  // upper triangle of a CD x CD block
  constexpr int NA = 2 * NU + 2 * CD;    // U, SZ, gc, yz
  int i = blockIdx.x;
  if (i >= v.M) return;
  int l = v.cam_sub[i];
  if (!run[l]) return;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T acc[NA];
#pragma unroll
  for (int e = 0; e < NA; e++) acc[e] = 0;
  const int p1 = v.cam_obs_ptr[i + 1];
  if constexpr (sizeof(T) == sizeof(float)) {
    // the camera's observations from the camera-major streams (coalesced);
    // only the robust weight (it changes) is gathered by observation, and the
    // point's active flag is read beside the other gathers, not before them
    for (int p = v.cam_obs_ptr[i] + threadIdx.x; p < p1; p += CB_THREADS) {
      int q = v.cm_inst[p];
      const bool act = v.active[v.cm_pt[p]] != 0;
      ObsT<float> ob;
      ob.x = v.cm_xy32[2 * (size_t)p];
      ob.y = v.cm_xy32[2 * (size_t)p + 1];
      if (v.has_winv) {
        ob.W[0] = v.cm_winv32[3 * (size_t)p]; ob.W[1] = v.cm_winv32[3 * (size_t)p + 1];
        ob.W[2] = v.cm_winv32[3 * (size_t)p + 2];
      } else {
        ob.W[0] = 1.f; ob.W[1] = 0.f; ob.W[2] = 1.f;
      }
      ob.w = v.obs_w32[v.cam_obs[p]];
      cb_obs_ob<T, CD>(v, i, q, act, ob, Ninv, gX, acc);
    }
  } else {
    for (int p = v.cam_obs_ptr[i] + threadIdx.x; p < p1; p += CB_THREADS) {
      int k = v.cam_obs[p];
      int q = v.obs_inst[k];
      if (!v.active[v.inst_pt[q]]) continue;
      cb_obs<T, CD>(v, i, k, q, true, NXC, Z, gX, Ninv, acc);
    }
  }
  // warp reduction, then across the CTA's warps
  __shared__ T red[CB_THREADS / 32][NA];
#pragma unroll
  for (int e = 0; e < NA; e++) {
    T x = acc[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][e] = x;
  }
  __syncthreads();
  if (threadIdx.x < NA) {
    T x = 0;
    for (int w = 0; w < CB_THREADS / 32; w++) x += red[w][threadIdx.x];
    red[0][threadIdx.x] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const T *U = red[0], *SZ = red[0] + NU, *gc = red[0] + 2 * NU, *yz = red[0] + 2 * NU + CD;
    double lam = lambda[l];
    int li = v.cam_local[i];
    int np = v.npad[l];
    double *S = v.S + v.S_off[l];
    int e = 0;
    for (int r = 0; r < CD; r++)
      for (int c = r; c < CD; c++, e++) {
        double val = (double)U[e] - (double)SZ[e];
        if (r == c) val += lam * (double)U[e];
        S[(size_t)(CD * li + r) * np + CD * li + c] = val;
        S[(size_t)(CD * li + c) * np + CD * li + r] = val;
      }
    double *yv = v.y + v.ycam_off[l];
    for (int r = 0; r < CD; r++) yv[CD * li + r] = -(double)gc[r] + (double)yz[r];
  }
}

// off-diagonal Schur blocks: one thread per (pair, row r):
//   S[(CD ia + r), CD ib + c] -= sum_e N_XC,a[e][r] Z_b[e][c]    (ia > ib)
template <typename T, int CD>
__global__ void k_schur_pairs(View v, const int *run, const int *pa, const int *pb, long long npairs,
                              const T *NXC, const T *Z) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= npairs * CD) return;
  long long p = tid / CD;
  int r = (int)(tid - p * CD);
  int a = pa[p], b = pb[p];
  int q = v.obs_inst[a];
  int l = v.inst_sub[q];
  if (!run[l] || !v.active[v.inst_pt[q]]) return;
  int ia = v.cam_local[v.obs_cam[a]], ib = v.cam_local[v.obs_cam[b]];
  const T *A = NXC + 3 * CD * (size_t)a, *Zb = Z + 3 * CD * (size_t)b;
  T x0 = A[r], x1 = A[CD + r], x2 = A[2 * CD + r];
  double *row = v.S + v.S_off[l] + (size_t)(CD * ia + r) * v.npad[l] + CD * ib;
#pragma unroll
  for (int c = 0; c < CD; c++) {
    T val = x0 * Zb[c] + x1 * Zb[CD + c] + x2 * Zb[2 * CD + c];
    atomicAdd(row + c, -(double)val);
  }
}

// FP32 form, off-diagonal Schur blocks: point pairs (a seen by camera i, b
// seen by camera i', the same instance, local(i) > local(i')),
//   S[6 li + r, 6 li' + c] -= sum_e N_XC,a[e][r] Z_b[e][c],
// the blocks formed in FP32 registers. The pairs are sorted by camera pair
// (segment) and cut into items of at most SC_ITEM consecutive pairs of one
// segment; a thread sums its item's blocks in registers, then a segmented
// warp reduction (items sorted, so a segment is a run of lanes) sums each
// segment's part and its first lane adds the CD x CD values to S (FP64 atomics,
// one set per segment piece instead of one per pair).
#define SC_THREADS 256
template <int CD>
__global__ void __launch_bounds__(SC_THREADS, CD == 6 ? 2 : 1) k_schur_seg(View v, const int *run, long long nitems,
                                                             const int *item, const int *spa, const int *spb,
                                                             const int *spq, const int *sps, const int *seg_cam,
                                                             const int *seg_nb, const float *Ninv) {
  long long it = (long long)blockIdx.x * SC_THREADS + threadIdx.x;
  int lane = threadIdx.x & 31;
  int sg = -1;
  float acc[CD * CD];
#pragma unroll
  for (int e = 0; e < CD * CD; e++) acc[e] = 0.f;
  if (it < nitems) {
    int t0 = item[it], t1 = item[it + 1];
    sg = sps[t0];
    int i = seg_cam[sg], ib = seg_nb[sg];
    if (run[v.cam_sub[i]]) {
      // the item's two cameras, read once for its pairs (a warp's lanes read
      // ~32 different records: per pair that was twice five gathered loads)
      CamRecF ra, rb;
      load_cam_rec(v, i, ra);
      load_cam_rec(v, ib, rb);
      for (int t = t0; t < t1; t++) {
        int q = spq[t];
        if (!v.active[v.inst_pt[q]]) continue;
        float A[3 * CD], B[3 * CD], Zb[3 * CD];
        nxc_f_rec<CD>(v, ra, spa[t], q, A);
        nxc_f_rec<CD>(v, rb, spb[t], q, B);
        const float *iv = Ninv + 6 * (size_t)q;
        float inv[6] = {iv[0], iv[1], iv[2], iv[3], iv[4], iv[5]};
        z_of<CD>(inv, B, Zb);
#pragma unroll
        for (int r = 0; r < CD; r++)
#pragma unroll
          for (int c = 0; c < CD; c++)
            acc[CD * r + c] += A[r] * Zb[c] + A[CD + r] * Zb[CD + c] + A[2 * CD + r] * Zb[2 * CD + c];
      }
    }
  }
  // segments are contiguous runs of lanes: after the steps, a lane holds the
  // sum over itself and the following lanes of its run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int so = __shfl_down_sync(0xffffffffu, sg, o);
    bool take = (lane + o < 32) && so == sg;
#pragma unroll
    for (int e = 0; e < CD * CD; e++) {
      float y = __shfl_down_sync(0xffffffffu, acc[e], o);
      if (take) acc[e] += y;
    }
  }
  int sprev = __shfl_up_sync(0xffffffffu, sg, 1);
  if (sg < 0 || (lane > 0 && sprev == sg)) return;
  int i = seg_cam[sg], ib = seg_nb[sg];
  int l = v.cam_sub[i];
  if (!run[l]) return;
  int np = v.npad[l];
  double *row = v.S + v.S_off[l] + (size_t)(CD * v.cam_local[i]) * np + CD * v.cam_local[ib];
#pragma unroll
  for (int r = 0; r < CD; r++)
#pragma unroll
    for (int c = 0; c < CD; c++) atomicAdd(row + (size_t)r * np + c, f2d(-acc[CD * r + c]));
}

// zero the lower 32 x 32 tiles of the RCS of running sub-blocks, identity on
// the padding. The strictly upper tiles are left as they are: every reader of
// S (the factorisations, the products, the preconditioners, rpba_rcs) takes
// the matrix from its lower triangle, and the Schur kernels write the upper
// triangle only inside the diagonal camera blocks. One CTA per row, the row
// through the end of its diagonal tile (np is a multiple of 32).
__global__ void k_rcs_clear(View v, const int *run, int L) {
  int l = blockIdx.y;
  if (l >= L || !run[l]) return;
  int np = v.npad[l];
  int n = v.cd * (v.sub_cam_ptr[l + 1] - v.sub_cam_ptr[l]);
  double *S = v.S + v.S_off[l];
  for (int r = blockIdx.x; r < np; r += gridDim.x) {
    double *row = S + (size_t)r * np;
    int lim = (r | 31) + 1;
    for (int c = threadIdx.x; c < lim; c += blockDim.x) row[c] = (r == c && r >= n) ? 1.0 : 0.0;
  }
  double *yv = v.y + v.ycam_off[l];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np; e += gridDim.x * blockDim.x)
    if (e >= n) yv[e] = 0.0;
}

template <int CD>
static rpba_status build_rcs_cd(Ctx *ctx, const View &v, const double *lambda_dev, const int *run_dev);

rpba_status launch_build_rcs(Ctx *ctx, const double *lambda_dev, const int *run_dev) {
  View v = make_view(ctx);
  dim3 gclr(256, ctx->L);
  RPBA_KERNEL(ctx, "k_rcs_clear", k_rcs_clear<<<gclr, 128, 0, ctx->stream>>>(v, run_dev, ctx->L));
  if (ctx->P == 0) return RPBA_OK;
  if (ctx->cd == 8) return build_rcs_cd<8>(ctx, v, lambda_dev, run_dev);
  return build_rcs_cd<6>(ctx, v, lambda_dev, run_dev);
}

template <int CD>
static rpba_status build_rcs_cd(Ctx *ctx, const View &v, const double *lambda_dev, const int *run_dev) {
  if (ctx->opt.precision == 1) {
    RPBA_KERNEL(ctx, "k_linearize_f32", k_linearize<float, CD><<<nblk(ctx->P, ctx->tune.lin), ctx->tune.lin, 0, ctx->stream>>>(
                                        v, lambda_dev, run_dev, nullptr, nullptr, (float *)ctx->Ninv, (float *)ctx->gX));
    RPBA_KERNEL(ctx, "k_camera_blocks_f32", k_camera_blocks<float, CD><<<ctx->M, CB_THREADS, 0, ctx->stream>>>(
        v, lambda_dev, run_dev, nullptr, nullptr, (const float *)ctx->gX, (const float *)ctx->Ninv));
    if (ctx->n_pairs)
      RPBA_KERNEL(ctx, "k_schur_seg", k_schur_seg<CD><<<nblk(ctx->n_items, SC_THREADS), SC_THREADS, 0, ctx->stream>>>(
                                          v, run_dev, ctx->n_items, ctx->sitem, ctx->spair_a, ctx->spair_b,
                                          ctx->spair_q, ctx->spair_seg, ctx->seg_cam, ctx->seg_nb,
                                          (const float *)ctx->Ninv));
  } else {
    double *NXC = (double *)ctx->NXC, *Z = (double *)ctx->Z;
    RPBA_KERNEL(ctx, "k_linearize_f64", k_linearize<double, CD><<<nblk(ctx->P, ctx->tune.lin), ctx->tune.lin, 0, ctx->stream>>>(v, lambda_dev, run_dev, NXC, Z,
                                                                    (double *)ctx->Ninv, (double *)ctx->gX));
    RPBA_KERNEL(ctx, "k_camera_blocks_f64", k_camera_blocks<double, CD><<<ctx->M, CB_THREADS, 0, ctx->stream>>>(
        v, lambda_dev, run_dev, NXC, Z, (const double *)ctx->gX, (const double *)ctx->Ninv));
    if (ctx->n_pairs)
      RPBA_KERNEL(ctx, "k_schur_pairs", k_schur_pairs<double, CD><<<nblk(ctx->n_pairs * CD, 256), 256, 0, ctx->stream>>>(
          v, run_dev, ctx->pair_a, ctx->pair_b, ctx->n_pairs, NXC, Z));
  }
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// back-substitution, trial state
// ---------------------------------------------------------------------------
// dX = Ninv (-g_X - sum_k N_XC,k dC_i(k)); X^l trial = X^l + dX
template <typename T, int CD>
__global__ void k_backsub(View v, const int *run, const T *NXC, const T *Ninv, const T *gX) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= v.P) return;
  int l = v.inst_sub[q];
  if (!run[l]) return;
  const double *Xq = v.Xl + 3 * (size_t)q;
  double *Xt = v.Xlt + 3 * (size_t)q;
  if (!v.active[v.inst_pt[q]]) {
    for (int e = 0; e < 3; e++) Xt[e] = Xq[e];
    if constexpr (sizeof(T) == sizeof(float))
      for (int e = 0; e < 3; e++) {
        v.Xlt_hi[3 * (size_t)q + e] = v.Xl_hi[3 * (size_t)q + e];
        v.Xlt_lo[3 * (size_t)q + e] = v.Xl_lo[3 * (size_t)q + e];
      }
    return;
  }
  T rhs[3] = {-gX[3 * (size_t)q], -gX[3 * (size_t)q + 1], -gX[3 * (size_t)q + 2]};
  for (int k = v.inst_obs_ptr[q]; k < v.inst_obs_ptr[q + 1]; k++) {
    int i = v.obs_cam[k];
    int off = v.ycam_off[l] + CD * v.cam_local[i];
    if constexpr (sizeof(T) == sizeof(float)) {
      // N_XC dC = (w W A_X)^T (A_C dC), the Jacobians formed again in registers
      float dc[CD];
      for (int c = 0; c < CD; c++) dc[c] = v.dC32[off + c];
      ProjJac<float, CD> pj;
      float z;
      obs_proj<float, CD>(v, i, nullptr, v.Xl_hi + 3 * (size_t)q, v.Xl_lo + 3 * (size_t)q, pj, z);
      float w = v.obs_w32[k], W0 = 1.f, W1 = 0.f, W2 = 1.f;
      if (v.has_winv) { W0 = v.obs_winv32[3 * k]; W1 = v.obs_winv32[3 * k + 1]; W2 = v.obs_winv32[3 * k + 2]; }
      float u0 = 0.f, u1 = 0.f;
      for (int c = 0; c < CD; c++) { u0 += pj.Jc[c] * dc[c]; u1 += pj.Jc[CD + c] * dc[c]; }
      float e0 = w * (W0 * u0 + W1 * u1), e1 = w * (W1 * u0 + W2 * u1);
      for (int r = 0; r < 3; r++) rhs[r] -= pj.Jx[r] * e0 + pj.Jx[3 + r] * e1;
    } else {
      T dc[CD];
      for (int c = 0; c < CD; c++) dc[c] = v.dC[off + c];
      const T *B = NXC + 3 * CD * (size_t)k;
      for (int r = 0; r < 3; r++) {
        T s = 0;
        for (int c = 0; c < CD; c++) s += B[CD * r + c] * dc[c];
        rhs[r] -= s;
      }
    }
  }
  const T *iv = Ninv + 6 * (size_t)q;
  for (int r = 0; r < 3; r++) {
    T dx = iv[s3idx(r, 0)] * rhs[0] + iv[s3idx(r, 1)] * rhs[1] + iv[s3idx(r, 2)] * rhs[2];
    if constexpr (sizeof(T) == sizeof(float)) {
      // the trial position in float-float from the hi + lo words (one FP64 add for the FP64 copy)
      float2 xn = ff_add(make_float2(v.Xl_hi[3 * (size_t)q + r], v.Xl_lo[3 * (size_t)q + r]), make_float2(dx, 0.f));
      v.Xlt_hi[3 * (size_t)q + r] = xn.x;
      v.Xlt_lo[3 * (size_t)q + r] = xn.y;
      Xt[r] = ff_to_double(xn);
    } else {
      Xt[r] = Xq[r] + dx;
    }
  }
}

// trial cameras: R' = exp([dw]x) R, t' = t + dt; with per-camera
// intrinsics f' = f + df, k1' = k1 + dk1
__global__ void k_cam_trial(View v, const int *run) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.M) return;
  int l = v.cam_sub[i];
  const double *R = v.R + 9 * i;
  double *Rt = v.Rt + 9 * i;
  double f = v.intr[3 * i], k1 = v.k1 ? v.k1[i] : 0.0;
  if (!run[l]) {
    for (int e = 0; e < 9; e++) Rt[e] = R[e];
    for (int e = 0; e < 3; e++) v.tt[3 * i + e] = v.t[3 * i + e];
  } else {
    const double *dc = v.dC + v.ycam_off[l] + v.cd * v.cam_local[i];
    double dR[9];
    rodrigues(dc, dR);
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++)
        Rt[3 * r + c] = dR[3 * r] * R[c] + dR[3 * r + 1] * R[3 + c] + dR[3 * r + 2] * R[6 + c];
    for (int e = 0; e < 3; e++) v.tt[3 * i + e] = v.t[3 * i + e] + dc[3 + e];
    if (v.cd == 8) {
      f += dc[6];
      k1 += dc[7];
    }
  }
  if (v.ft) {
    v.ft[i] = f;
    v.k1t[i] = k1;
  }
  if (v.camff_t) ff_camera_record(Rt, v.tt + 3 * i, f, k1, v.camff_t + FF_CAM * (size_t)i);
}

__global__ void k_to_float(const double *a, float *b, int n) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

rpba_status launch_backsub_trial(Ctx *ctx, const int *run_dev) {
  View v = make_view(ctx);
  if (ctx->opt.precision == 1 && ctx->ytot)
    RPBA_KERNEL(ctx, "k_to_float", k_to_float<<<nblk(ctx->ytot, 256), 256, 0, ctx->stream>>>(ctx->dC, ctx->dC32, ctx->ytot));
  if (ctx->P) {
    dim3 g(nblk(ctx->P, ctx->tune.backsub)), b(ctx->tune.backsub);
    const double *nxc = (const double *)ctx->NXC, *ninv = (const double *)ctx->Ninv, *gx = (const double *)ctx->gX;
    const float *ninv32 = (const float *)ctx->Ninv, *gx32 = (const float *)ctx->gX;
    if (ctx->opt.precision == 1 && ctx->cd == 8)
      RPBA_KERNEL(ctx, "k_backsub_f32", k_backsub<float, 8><<<g, b, 0, ctx->stream>>>(v, run_dev, nullptr, ninv32, gx32));
    else if (ctx->opt.precision == 1)
      RPBA_KERNEL(ctx, "k_backsub_f32", k_backsub<float, 6><<<g, b, 0, ctx->stream>>>(v, run_dev, nullptr, ninv32, gx32));
    else if (ctx->cd == 8)
      RPBA_KERNEL(ctx, "k_backsub_f64", k_backsub<double, 8><<<g, b, 0, ctx->stream>>>(v, run_dev, nxc, ninv, gx));
    else
      RPBA_KERNEL(ctx, "k_backsub_f64", k_backsub<double, 6><<<g, b, 0, ctx->stream>>>(v, run_dev, nxc, ninv, gx));
  }
  if (ctx->M) RPBA_KERNEL(ctx, "k_cam_trial", k_cam_trial<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(v, run_dev));
  return sub_costs_impl(ctx, 1, run_dev, ctx->lm_Ft);
}

// ---------------------------------------------------------------------------
// LM control per sub-block (Sec. 5.5 and the stopping reading)
// ---------------------------------------------------------------------------
__global__ void k_lm_init(View v, const uint8_t *sub_mask, double lambda0, int grace, double *lam, double *F,
                          double *best, int *gr, int *rej, int *it, int *run, const double *F0) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= v.L) return;
  lam[l] = lambda0;
  F[l] = F0[l];
  best[l] = F0[l];
  gr[l] = grace;
  rej[l] = 0;
  it[l] = 0;
  run[l] = (v.sub_cam_ptr[l + 1] - v.sub_cam_ptr[l]) > 0 && sub_mask[l];
}

__global__ void k_lm_decide(int L, double lambda0, double stop_ratio, int max_inner, int max_reject,
                            double *lam, double *F, const double *Ft, double *best, int *gr, int *rej, int *it,
                            int *run, int *acc, const int *fail, int *n_running) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  acc[l] = 0;
  if (!run[l]) return;
  it[l] += 1;
  double ft = Ft[l];
  bool ok = !fail[l] && isfinite(ft) && ft < F[l];
  bool stop = false;
  if (!ok) {
    lam[l] *= 10.0;
    if (++rej[l] > max_reject) stop = true;
  } else {
    acc[l] = 1;
    rej[l] = 0;
    double ratio = best[l] / (ft > 1e-300 ? ft : 1e-300);
    F[l] = ft;
    double nl = lam[l] / 10.0;
    lam[l] = nl > lambda0 ? nl : lambda0;
    if (ft < best[l]) best[l] = ft;
    if (ratio < stop_ratio) {
      if (gr[l] > 0) gr[l] -= 1;
      else stop = true;
    }
  }
  if (it[l] >= max_inner) stop = true;
  if (stop) run[l] = 0;
  else atomicAdd(n_running, 1);
}

// copy the trial state of accepted sub-blocks
__global__ void k_lm_apply_cams(View v, const int *acc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.M || !acc[v.cam_sub[i]]) return;
  double *R = const_cast<double *>(v.R) + 9 * i;
  double *t = const_cast<double *>(v.t) + 3 * i;
  for (int e = 0; e < 9; e++) R[e] = v.Rt[9 * i + e];
  for (int e = 0; e < 3; e++) t[e] = v.tt[3 * i + e];
  if (v.ft) {
    v.intr[3 * i] = v.ft[i];
    v.k1[i] = v.k1t[i];
  }
  if (v.camff)
    for (int e = 0; e < FF_CAM; e++) v.camff[FF_CAM * (size_t)i + e] = v.camff_t[FF_CAM * (size_t)i + e];
}

__global__ void k_lm_apply_inst(View v, const int *acc) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= v.P || !acc[v.inst_sub[q]]) return;
  for (int e = 0; e < 3; e++) v.Xl[3 * (size_t)q + e] = v.Xlt[3 * (size_t)q + e];
  if (v.Xl_hi)
    for (int e = 0; e < 3; e++) {
      v.Xl_hi[3 * (size_t)q + e] = v.Xlt_hi[3 * (size_t)q + e];
      v.Xl_lo[3 * (size_t)q + e] = v.Xlt_lo[3 * (size_t)q + e];
    }
}

rpba_status launch_lm_apply(Ctx *ctx, const int *acc_dev) {
  View v = make_view(ctx);
  if (ctx->M) RPBA_KERNEL(ctx, "k_lm_apply_cams", k_lm_apply_cams<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(v, acc_dev));
  if (ctx->P) RPBA_KERNEL(ctx, "k_lm_apply_inst", k_lm_apply_inst<<<nblk(ctx->P, 256), 256, 0, ctx->stream>>>(v, acc_dev));
  return RPBA_OK;
}

// the costs F_l at the start of a bact: those the outer iteration's tail left
// when nothing has changed the state since (cost_sigma0_launch), else
// evaluated here
rpba_status launch_lm_init(Ctx *ctx) {
  const double *F0 = ctx->lm_Ft;
  if (ctx->f0_valid) F0 = ctx->f0_cache;
  else RPBA_TRY(sub_costs_impl(ctx, 0, nullptr, ctx->lm_Ft));
  ctx->f0_valid = false;  // the bact changes the state
  RPBA_KERNEL(ctx, "k_lm_init", k_lm_init<<<nblk(ctx->L, 128), 128, 0, ctx->stream>>>(make_view(ctx), ctx->sub_mask, ctx->opt.lambda0, ctx->opt.grace,
                                                        ctx->lm_lambda, ctx->lm_F, ctx->lm_best, ctx->lm_grace,
                                                        ctx->lm_rej, ctx->lm_it, ctx->lm_run, F0));
  return RPBA_OK;
}

rpba_status launch_lm_decide(Ctx *ctx) {
  RPBA_KERNEL(ctx, "k_lm_decide", k_lm_decide<<<nblk(ctx->L, 128), 128, 0, ctx->stream>>>(
      ctx->L, ctx->opt.lambda0, ctx->opt.stop_ratio, ctx->opt.max_inner, ctx->opt.max_reject, ctx->lm_lambda,
      ctx->lm_F, ctx->lm_Ft, ctx->lm_best, ctx->lm_grace, ctx->lm_rej, ctx->lm_it, ctx->lm_run, ctx->lm_acc,
      ctx->lm_cholfail, ctx->counters));
  return RPBA_OK;
}

__global__ void k_fill_int(int *p, int n, int val) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) p[e] = val;
}
__global__ void k_fill_double(double *p, long long n, double val) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) p[e] = val;
}
rpba_status launch_fill_int(Ctx *ctx, int *p, int n, int v) {
  if (n <= 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_fill_int", k_fill_int<<<nblk(n, 256), 256, 0, ctx->stream>>>(p, n, v));
  return RPBA_OK;
}
rpba_status launch_fill_double(Ctx *ctx, double *p, long long n, double v) {
  if (n <= 0) return RPBA_OK;
  RPBA_KERNEL(ctx, "k_fill_double", k_fill_double<<<nblk(n, 256), 256, 0, ctx->stream>>>(p, n, v));
  return RPBA_OK;
}

}  // namespace rpba
