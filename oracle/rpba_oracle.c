/*
 * rpba_oracle.c -- plain, slow FP64 CPU oracle of the RPBA iteration.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the timed
 * CPU baseline of the benchmark to check the CUDA path. It shares no code with
 * that path. Everything is double precision, single threaded, and written as
 * directly as the method allows: one loop per sum of the paper's equations,
 * dense matrices, textbook Cholesky, qsort medians.
 *
 * Readings of the paper where it is silent or ambiguous (also listed with the
 * design notes of the repository):
 *  - sigma_0 and the normalised residual use v^T C^-1 v (Eq. normalw), not the
 *    C_x printed in Eq. sigma0.
 *  - ||.||_W in Eq. batp / bact is the squared Mahalanobis distance.
 *  - damping multiplies the diagonal of the whole normal matrix (camera and
 *    point blocks, TP control term included): N + lambda diag(N) (Sec. 5.5).
 *  - a rejected LM step multiplies lambda by 10, an accepted one divides it
 *    by 10 but not below lambda0 (the paper keeps lambda fixed and says nothing
 *    about rejected steps).
 *  - convergence (Sec. 5.5), for the LM loop of a sub-block (cost F_l) and for
 *    the outer loop (sigma_0) alike: ratio = best-so-far / value after this
 *    iteration; ratio < 1.01 ends the loop unless the grace iteration is still
 *    unused, in which case it is used up.
 *  - initial intersection of all points before the first bact gives the
 *    starting TP weights; later intersections run for the TPs only, starting
 *    from the previous X_TP; the sub-block copies X^l of TPs restart at X_TP.
 *  - intersection is undamped Gauss-Newton, at most 10 iterations, converged
 *    when the step moves the point's image residuals by less than 1e-3 px per
 *    observation (dX^T N_j dX <= (1e-3)^2 n_obs) or when ||dX|| <= 1e-10
 *    (1 + ||X||); it drops the point when it does not converge, when an
 *    observation lies behind its camera (z_c <= 0), or when the Frobenius
 *    condition number of N_j exceeds 1e12 (Sec. 5.5, last paragraph). W^l and
 *    N_j are those of the last Gauss-Newton iteration.
 *  - refined weight (Sec. 5.1): W^l_j = N_j - N_j^(l), the normal matrix of
 *    point j without the observations from cameras of sub-block l; zero for a
 *    point seen in one sub-block only.
 *  - robust stage (Sec. 5.3, parallel variant): starts after the first outer
 *    convergence (option robust_from_start: already at the first intersection
 *    after the first bact, for blocks with gross outliers); before every TP intersection from then on the per-camera
 *    scale is 1.4826 * MAD of the whitened residual components and an
 *    observation whose sqrt(v^T C^-1 v) / scale exceeds t_v = 4 gets weight
 *    1e-4, otherwise 1; the weights enter every cost. At the end every point
 *    with a down-weighted observation is eliminated.
 *  - an LM trial with any observation behind its camera is rejected.
 *  - redundancy of sigma_0: 2 K - 6 M - 3 N + 7 over the active observations
 *    and points (free network); with per-camera intrinsics 2 K - 8 M - 3 N + 7.
 *  - per-camera intrinsics (the Final data sets of Sec. 6: focal length and
 *    the first radial distortion parameter estimated per camera): the radial
 *    polynomial acts on the normalised image coordinates p = (x_c/z_c, y_c/z_c),
 *    u = f (1 + k1 |p|^2) p_x + cx, v = f (1 + k1 |p|^2) p_y + cy, with the
 *    principal point fixed; the camera unknowns are (dw, dt, df, dk1), f and
 *    k1 updated additively.
 */
#include "rpba_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_ctx {
  int M, N, K, L, P;
  int cd;       /* camera unknowns: 6 (pose) or 8 (pose, f, k1) */
  double *intr; /* (f, cx, cy) per camera; f is estimated when cd = 8 */
  double *k1;   /* radial parameter per camera (0 unless cd = 8) */
  int *cam_sub;
  int *obs_cam, *obs_pt;
  double *obs_xy, *obs_winv;
  /* topology */
  int *obs_inst;
  int *inst_pt, *inst_sub;
  int *inst_obs_ptr, *inst_obs;
  int *pt_inst_ptr, *pt_inst;
  int *pt_obs_ptr, *pt_obs;
  int *cam_obs_ptr, *cam_obs;
  int *sub_inst_ptr;
  int *sub_cam_ptr, *sub_cam;
  int *cam_local;
  int max_inst_obs;
  /* state */
  double *R, *t, *X, *Xl, *Wl, *w;
  unsigned char *active;
};

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                      */
/* ------------------------------------------------------------------------ */

/* sym3 index of (r, c) */
static int s3(int r, int c) {
  static const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return idx[r][c];
}

/* inverse of a symmetric 3x3 by cofactors; returns the determinant */
static double sym3_inverse(const double a[6], double inv[6]) {
  double c00 = a[3] * a[5] - a[4] * a[4];
  double c01 = a[2] * a[4] - a[1] * a[5];
  double c02 = a[1] * a[4] - a[2] * a[3];
  double c11 = a[0] * a[5] - a[2] * a[2];
  double c12 = a[1] * a[2] - a[0] * a[4];
  double c22 = a[0] * a[3] - a[1] * a[1];
  double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  inv[0] = c00 / det; inv[1] = c01 / det; inv[2] = c02 / det;
  inv[3] = c11 / det; inv[4] = c12 / det; inv[5] = c22 / det;
  return det;
}

static double sym3_frob(const double a[6]) {
  return sqrt(a[0] * a[0] + a[3] * a[3] + a[5] * a[5] +
              2.0 * (a[1] * a[1] + a[2] * a[2] + a[4] * a[4]));
}

static void sym3_mul_vec(const double a[6], const double x[3], double y[3]) {
  for (int r = 0; r < 3; r++) {
    y[r] = 0.0;
    for (int c = 0; c < 3; c++) y[r] += a[s3(r, c)] * x[c];
  }
}

/* out += s * A^T W B with A (2 x p), B (2 x q) row-major, W sym2 (w11, w12, w22);
 * out is p x q row-major */
static void add_AtWB(const double *A, int p, const double *B, int q, const double W[3],
                     double s, double *out) {
  double Wf[2][2] = {{W[0], W[1]}, {W[1], W[2]}};
  for (int a = 0; a < p; a++)
    for (int b = 0; b < q; b++) {
      double acc = 0.0;
      for (int r = 0; r < 2; r++)
        for (int u = 0; u < 2; u++) acc += A[r * p + a] * Wf[r][u] * B[u * q + b];
      out[a * q + b] += s * acc;
    }
}

/* textbook dense Cholesky, lower, in place (row-major n x n); 0 on failure */
static int cholesky(double *A, int n) {
  for (int j = 0; j < n; j++) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; k++) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return 0;
    d = sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; k++) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / d;
    }
  }
  return 1;
}

/* solve L L^T x = b with the lower factor in A; b overwritten by x */
static void cholesky_solve(const double *A, int n, double *b) {
  for (int i = 0; i < n; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= A[(size_t)i * n + k] * b[k];
    b[i] = s / A[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = b[i];
    for (int k = i + 1; k < n; k++) s -= A[(size_t)k * n + i] * b[k];
    b[i] = s / A[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------------------ */
/* rotations and projection (Sec. 2, Sec. 5.5)                              */
/* ------------------------------------------------------------------------ */

/* R = exp([w]x) by the Rodrigues formula */
void orc_rodrigues(const double w[3], double R[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double a, b; /* sin(th)/th, (1 - cos(th))/th^2 */
  if (th < 1e-4) {
    a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
  }
  double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) {
      double kk = 0.0;
      for (int m = 0; m < 3; m++) kk += K[r * 3 + m] * K[m * 3 + c];
      R[r * 3 + c] = (r == c ? 1.0 : 0.0) + a * K[r * 3 + c] + b * kk;
    }
}

/* angle-axis vector of a rotation matrix: theta = atan2(sin, cos) with
 * sin(theta) = |v| / 2, v = (R32 - R23, R13 - R31, R21 - R12) = 2 sin(theta) axis;
 * near theta = pi the axis comes from the symmetric part
 * cos(theta) I + (1 - cos(theta)) a a^T instead of v */
void orc_rotation_log(const double R[9], double w[3]) {
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
  double s = 0.5 * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double th = atan2(s, c);
  if (th < 1e-6) {
    for (int i = 0; i < 3; i++) w[i] = 0.5 * v[i] * (1.0 + th * th / 6.0);
    return;
  }
  if (th < 3.14159265358979323846 - 1e-3) {
    for (int i = 0; i < 3; i++) w[i] = th / (2.0 * s) * v[i];
    return;
  }
  double B[3] = {(R[0] - c) / (1.0 - c), (R[4] - c) / (1.0 - c), (R[8] - c) / (1.0 - c)};
  int k = 0;
  if (B[1] > B[k]) k = 1;
  if (B[2] > B[k]) k = 2;
  double a[3];
  a[k] = sqrt(B[k] > 0.0 ? B[k] : 0.0);
  for (int i = 0; i < 3; i++)
    if (i != k) a[i] = (R[k * 3 + i] + R[i * 3 + k]) / (2.0 * (1.0 - c) * a[k]);
  double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double sgn = (a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) < 0.0 ? -1.0 : 1.0;
  for (int i = 0; i < 3; i++) w[i] = sgn * th * a[i] / n;
}

/* g_k: pinhole projection of X by camera (R, t, f, cx, cy) and its Jacobians.
 * Jc = d(u,v)/d(dw, dt) for R' = exp([dw]x) R, t' = t + dt; Jx = d(u,v)/dX. */
double orc_project(const double R[9], const double t[3], const double intr[3],
                   const double X[3], double uv[2], double Jc[12], double Jx[6]) {
  double RX[3], Xc[3];
  for (int r = 0; r < 3; r++) {
    RX[r] = R[r * 3 + 0] * X[0] + R[r * 3 + 1] * X[1] + R[r * 3 + 2] * X[2];
    Xc[r] = RX[r] + t[r];
  }
  double f = intr[0];
  double iz = 1.0 / Xc[2];
  if (uv) {
    uv[0] = f * Xc[0] * iz + intr[1];
    uv[1] = f * Xc[1] * iz + intr[2];
  }
  if (Jc || Jx) {
    /* d(u,v)/dXc */
    double P[6] = {f * iz, 0.0, -f * Xc[0] * iz * iz, 0.0, f * iz, -f * Xc[1] * iz * iz};
    if (Jx)
      for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
          Jx[r * 3 + c] = P[r * 3 + 0] * R[0 * 3 + c] + P[r * 3 + 1] * R[1 * 3 + c] +
                          P[r * 3 + 2] * R[2 * 3 + c];
    if (Jc) {
      /* dXc/d(dw) = -[RX]x ; dXc/dt = I */
      double M[9] = {0.0, RX[2], -RX[1], -RX[2], 0.0, RX[0], RX[1], -RX[0], 0.0};
      for (int r = 0; r < 2; r++) {
        for (int c = 0; c < 3; c++) {
          Jc[r * 6 + c] = P[r * 3 + 0] * M[0 * 3 + c] + P[r * 3 + 1] * M[1 * 3 + c] +
                          P[r * 3 + 2] * M[2 * 3 + c];
          Jc[r * 6 + 3 + c] = P[r * 3 + c];
        }
      }
    }
  }
  return Xc[2];
}

/* g_k with the first radial distortion parameter (the Final data sets of
 * Sec. 6): p = (x_c/z_c, y_c/z_c), d = 1 + k1 |p|^2, (u, v) = f d p + (cx, cy).
 * Jc (2 x 8) = d(u,v)/d(dw, dt, df, dk1) with the rotation convention of
 * orc_project; Jx = d(u,v)/dX. */
double orc_project_k1(const double R[9], const double t[3], const double intr[3], double k1,
                      const double X[3], double uv[2], double Jc[16], double Jx[6]) {
  double RX[3], Xc[3];
  for (int r = 0; r < 3; r++) {
    RX[r] = R[r * 3 + 0] * X[0] + R[r * 3 + 1] * X[1] + R[r * 3 + 2] * X[2];
    Xc[r] = RX[r] + t[r];
  }
  double f = intr[0];
  double iz = 1.0 / Xc[2];
  double px = Xc[0] * iz, py = Xc[1] * iz;
  double r2 = px * px + py * py;
  double d = 1.0 + k1 * r2;
  if (uv) {
    uv[0] = f * d * px + intr[1];
    uv[1] = f * d * py + intr[2];
  }
  if (Jc || Jx) {
    /* d(u,v)/dp = f (d I + 2 k1 p p^T); dp/dXc = (1/z) [I2 | -p] */
    double D[4] = {f * (d + 2.0 * k1 * px * px), f * 2.0 * k1 * px * py,
                   f * 2.0 * k1 * px * py, f * (d + 2.0 * k1 * py * py)};
    double Q[6] = {iz, 0.0, -px * iz, 0.0, iz, -py * iz};
    double P[6]; /* d(u,v)/dXc = D Q */
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 3; c++) P[r * 3 + c] = D[r * 2 + 0] * Q[c] + D[r * 2 + 1] * Q[3 + c];
    if (Jx)
      for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
          Jx[r * 3 + c] = P[r * 3 + 0] * R[0 * 3 + c] + P[r * 3 + 1] * R[1 * 3 + c] +
                          P[r * 3 + 2] * R[2 * 3 + c];
    if (Jc) {
      double M[9] = {0.0, RX[2], -RX[1], -RX[2], 0.0, RX[0], RX[1], -RX[0], 0.0};
      double pp[2] = {px, py};
      for (int r = 0; r < 2; r++) {
        for (int c = 0; c < 3; c++) {
          Jc[r * 8 + c] = P[r * 3 + 0] * M[0 * 3 + c] + P[r * 3 + 1] * M[1 * 3 + c] +
                          P[r * 3 + 2] * M[2 * 3 + c];
          Jc[r * 8 + 3 + c] = P[r * 3 + c];
        }
        Jc[r * 8 + 6] = d * pp[r];      /* d/df */
        Jc[r * 8 + 7] = f * r2 * pp[r]; /* d/dk1 */
      }
    }
  }
  return Xc[2];
}

/* ------------------------------------------------------------------------ */
/* construction                                                              */
/* ------------------------------------------------------------------------ */

void orc_default_options(orc_options *o) {
  o->lambda0 = 1e-4;
  o->t_v = 4.0;
  o->downweight = 1e-4;
  o->stop_ratio = 1.01;
  o->grace = 1;
  o->max_outer = 30;
  o->max_inner = 20;
  o->max_reject = 6;
  o->robust = 0;
  o->robust_from_start = 0;
  o->isect_max_iter = 10;
  o->isect_tol = 1e-10;
  o->isect_px_tol = 1e-3;
  o->cond_max = 1e12;
  o->robust_serial = 0;
  o->weight_mode = 0;
  o->rho0 = 200.0;
  o->rho = 200.0;
}

static int cmp_ll(const void *a, const void *b) {
  long long x = *(const long long *)a, y = *(const long long *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int cmp_d(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* stable grouping of items 0..n-1 by key[] in 0..nk-1 into CSR (ptr, list) */
static void group_by(const int *key, int n, int nk, int **ptr_out, int **list_out) {
  int *ptr = (int *)calloc((size_t)nk + 1, sizeof(int));
  int *list = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; i++) ptr[key[i] + 1]++;
  for (int k = 0; k < nk; k++) ptr[k + 1] += ptr[k];
  int *fill = (int *)malloc(sizeof(int) * (size_t)(nk > 0 ? nk : 1));
  for (int k = 0; k < nk; k++) fill[k] = ptr[k];
  for (int i = 0; i < n; i++) list[fill[key[i]]++] = i;
  free(fill);
  *ptr_out = ptr;
  *list_out = list;
}

orc_ctx *orc_create(int M, int N, int K, const double *cam_pose, const double *cam_intr,
                    const double *points, const int *obs_cam, const int *obs_point,
                    const double *obs_xy, const double *obs_winv, const int *cam_sub) {
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->M = M; c->N = N; c->K = K;
  c->cd = 6;
  c->intr = (double *)malloc(sizeof(double) * 3 * (M > 0 ? M : 1));
  memcpy(c->intr, cam_intr, sizeof(double) * 3 * M);
  c->k1 = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
  c->cam_sub = (int *)malloc(sizeof(int) * M);
  memcpy(c->cam_sub, cam_sub, sizeof(int) * M);
  int L = 0;
  for (int i = 0; i < M; i++) if (cam_sub[i] + 1 > L) L = cam_sub[i] + 1;
  c->L = L;
  c->obs_cam = (int *)malloc(sizeof(int) * K);
  c->obs_pt = (int *)malloc(sizeof(int) * K);
  c->obs_xy = (double *)malloc(sizeof(double) * 2 * K);
  c->obs_winv = (double *)malloc(sizeof(double) * 3 * K);
  memcpy(c->obs_cam, obs_cam, sizeof(int) * K);
  memcpy(c->obs_pt, obs_point, sizeof(int) * K);
  memcpy(c->obs_xy, obs_xy, sizeof(double) * 2 * K);
  for (int k = 0; k < K; k++) {
    if (obs_winv) {
      for (int e = 0; e < 3; e++) c->obs_winv[3 * k + e] = obs_winv[3 * k + e];
    } else {
      c->obs_winv[3 * k + 0] = 1.0; c->obs_winv[3 * k + 1] = 0.0; c->obs_winv[3 * k + 2] = 1.0;
    }
  }
  /* instances: unique (l, j) over the observations, sorted by (l, j) */
  long long *keys = (long long *)malloc(sizeof(long long) * (size_t)(K > 0 ? K : 1));
  for (int k = 0; k < K; k++) keys[k] = (long long)cam_sub[obs_cam[k]] * N + obs_point[k];
  qsort(keys, (size_t)K, sizeof(long long), cmp_ll);
  int P = 0;
  for (int k = 0; k < K; k++) if (k == 0 || keys[k] != keys[k - 1]) keys[P++] = keys[k];
  c->P = P;
  c->inst_pt = (int *)malloc(sizeof(int) * (P > 0 ? P : 1));
  c->inst_sub = (int *)malloc(sizeof(int) * (P > 0 ? P : 1));
  for (int q = 0; q < P; q++) {
    c->inst_sub[q] = (int)(keys[q] / N);
    c->inst_pt[q] = (int)(keys[q] % N);
  }
  c->obs_inst = (int *)malloc(sizeof(int) * (K > 0 ? K : 1));
  for (int k = 0; k < K; k++) {
    long long key = (long long)cam_sub[obs_cam[k]] * N + obs_point[k];
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      int mid = (lo + hi) / 2;
      if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    c->obs_inst[k] = lo;
  }
  free(keys);
  group_by(c->obs_inst, K, P, &c->inst_obs_ptr, &c->inst_obs);
  group_by(c->inst_pt, P, N, &c->pt_inst_ptr, &c->pt_inst);
  group_by(c->obs_pt, K, N, &c->pt_obs_ptr, &c->pt_obs);
  group_by(c->obs_cam, K, M, &c->cam_obs_ptr, &c->cam_obs);
  group_by(c->cam_sub, M, L, &c->sub_cam_ptr, &c->sub_cam);
  {
    int *dummy;
    group_by(c->inst_sub, P, L, &c->sub_inst_ptr, &dummy);
    free(dummy); /* instances are already sorted by l */
  }
  c->cam_local = (int *)malloc(sizeof(int) * M);
  for (int l = 0; l < L; l++)
    for (int p = c->sub_cam_ptr[l]; p < c->sub_cam_ptr[l + 1]; p++)
      c->cam_local[c->sub_cam[p]] = p - c->sub_cam_ptr[l];
  c->max_inst_obs = 1;
  for (int q = 0; q < P; q++) {
    int m = c->inst_obs_ptr[q + 1] - c->inst_obs_ptr[q];
    if (m > c->max_inst_obs) c->max_inst_obs = m;
  }
  /* state */
  c->R = (double *)malloc(sizeof(double) * 9 * M);
  c->t = (double *)malloc(sizeof(double) * 3 * M);
  c->X = (double *)malloc(sizeof(double) * 3 * N);
  c->Xl = (double *)calloc((size_t)3 * (P > 0 ? P : 1), sizeof(double));
  c->Wl = (double *)calloc((size_t)6 * (P > 0 ? P : 1), sizeof(double));
  c->w = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
  c->active = (unsigned char *)malloc((size_t)(N > 0 ? N : 1));
  orc_set_cameras(c, cam_pose);
  memcpy(c->X, points, sizeof(double) * 3 * N);
  for (int k = 0; k < K; k++) c->w[k] = 1.0;
  /* a point needs two observations to be determined */
  for (int j = 0; j < N; j++) c->active[j] = (c->pt_obs_ptr[j + 1] - c->pt_obs_ptr[j]) >= 2;
  for (int q = 0; q < P; q++)
    for (int e = 0; e < 3; e++) c->Xl[3 * q + e] = c->X[3 * c->inst_pt[q] + e];
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->intr); free(c->k1); free(c->cam_sub); free(c->obs_cam); free(c->obs_pt); free(c->obs_xy);
  free(c->obs_winv); free(c->obs_inst); free(c->inst_pt); free(c->inst_sub);
  free(c->inst_obs_ptr); free(c->inst_obs); free(c->pt_inst_ptr); free(c->pt_inst);
  free(c->pt_obs_ptr); free(c->pt_obs); free(c->cam_obs_ptr); free(c->cam_obs);
  free(c->sub_inst_ptr); free(c->sub_cam_ptr); free(c->sub_cam); free(c->cam_local);
  free(c->R); free(c->t); free(c->X); free(c->Xl); free(c->Wl); free(c->w); free(c->active);
  free(c);
}

int orc_num_subblocks(const orc_ctx *c) { return c->L; }
int orc_num_instances(const orc_ctx *c) { return c->P; }

void orc_instances(const orc_ctx *c, int *inst_point, int *inst_sub) {
  for (int q = 0; q < c->P; q++) {
    inst_point[q] = c->inst_pt[q];
    inst_sub[q] = c->inst_sub[q];
  }
}

int orc_sub_cameras(const orc_ctx *c, int l, int *cams) {
  int n = c->sub_cam_ptr[l + 1] - c->sub_cam_ptr[l];
  if (cams)
    for (int p = 0; p < n; p++) cams[p] = c->sub_cam[c->sub_cam_ptr[l] + p];
  return n;
}

void orc_get_cameras(const orc_ctx *c, double *pose) {
  for (int i = 0; i < c->M; i++) {
    orc_rotation_log(c->R + 9 * i, pose + 6 * i);
    for (int e = 0; e < 3; e++) pose[6 * i + 3 + e] = c->t[3 * i + e];
  }
}

void orc_set_cameras(orc_ctx *c, const double *pose) {
  for (int i = 0; i < c->M; i++) {
    orc_rodrigues(pose + 6 * i, c->R + 9 * i);
    for (int e = 0; e < 3; e++) c->t[3 * i + e] = pose[6 * i + 3 + e];
  }
}

void orc_get_camera_rt(const orc_ctx *c, double *R, double *t) {
  memcpy(R, c->R, sizeof(double) * 9 * c->M);
  memcpy(t, c->t, sizeof(double) * 3 * c->M);
}

void orc_set_camera_rt(orc_ctx *c, const double *R, const double *t) {
  memcpy(c->R, R, sizeof(double) * 9 * c->M);
  memcpy(c->t, t, sizeof(double) * 3 * c->M);
}

void orc_enable_intrinsics(orc_ctx *c, const double *k1) {
  c->cd = 8;
  for (int i = 0; i < c->M; i++) c->k1[i] = k1 ? k1[i] : 0.0;
}

int orc_camera_dim(const orc_ctx *c) { return c->cd; }

void orc_get_intrinsics(const orc_ctx *c, double *fk) {
  for (int i = 0; i < c->M; i++) {
    fk[2 * i] = c->intr[3 * i];
    fk[2 * i + 1] = c->k1[i];
  }
}

void orc_set_intrinsics(orc_ctx *c, const double *fk) {
  for (int i = 0; i < c->M; i++) {
    c->intr[3 * i] = fk[2 * i];
    c->k1[i] = fk[2 * i + 1];
  }
}

void orc_get_points(const orc_ctx *c, double *X, unsigned char *active) {
  if (X) memcpy(X, c->X, sizeof(double) * 3 * c->N);
  if (active) memcpy(active, c->active, (size_t)c->N);
}

void orc_set_points(orc_ctx *c, const double *X, const unsigned char *active) {
  if (X) memcpy(c->X, X, sizeof(double) * 3 * c->N);
  if (active) memcpy(c->active, active, (size_t)c->N);
}

void orc_get_instances(const orc_ctx *c, double *Xl, double *Wl) {
  if (Xl) memcpy(Xl, c->Xl, sizeof(double) * 3 * c->P);
  if (Wl) memcpy(Wl, c->Wl, sizeof(double) * 6 * c->P);
}

void orc_set_instances(orc_ctx *c, const double *Xl, const double *Wl) {
  if (Xl) memcpy(c->Xl, Xl, sizeof(double) * 3 * c->P);
  if (Wl) memcpy(c->Wl, Wl, sizeof(double) * 6 * c->P);
}

void orc_get_weights(const orc_ctx *c, double *w) { memcpy(w, c->w, sizeof(double) * c->K); }
void orc_set_weights(orc_ctx *c, const double *w) { memcpy(c->w, w, sizeof(double) * c->K); }

/* ------------------------------------------------------------------------ */
/* evaluations at the global state                                          */
/* ------------------------------------------------------------------------ */

/* residual of observation k for the camera arrays R, t, intr, k1 (global
 * indexing); Jc is 2 x cd */
static double obs_residual_at(const orc_ctx *c, int k, const double *R, const double *t,
                              const double *intr, const double *k1, const double *X, double v[2],
                              double *Jc, double Jx[6]) {
  int i = c->obs_cam[k];
  double uv[2];
  double z = c->cd == 8 ? orc_project_k1(R + 9 * i, t + 3 * i, intr + 3 * i, k1[i], X, uv, Jc, Jx)
                        : orc_project(R + 9 * i, t + 3 * i, intr + 3 * i, X, uv, Jc, Jx);
  v[0] = uv[0] - c->obs_xy[2 * k + 0];
  v[1] = uv[1] - c->obs_xy[2 * k + 1];
  return z;
}

static double obs_residual(const orc_ctx *c, int k, const double *R, const double *t,
                           const double *X, double v[2], double *Jc, double Jx[6]) {
  return obs_residual_at(c, k, R, t, c->intr, c->k1, X, v, Jc, Jx);
}

static double quad_w(const double W[3], const double v[2]) {
  return W[0] * v[0] * v[0] + 2.0 * W[1] * v[0] * v[1] + W[2] * v[1] * v[1];
}

void orc_residuals(const orc_ctx *c, double *v) {
  for (int k = 0; k < c->K; k++)
    obs_residual(c, k, c->R, c->t, c->X + 3 * c->obs_pt[k], v + 2 * k, NULL, NULL);
}

void orc_jacobians(const orc_ctx *c, double *Jc, double *Jx) {
  double v[2];
  for (int k = 0; k < c->K; k++)
    obs_residual(c, k, c->R, c->t, c->X + 3 * c->obs_pt[k], v, Jc + 2 * (size_t)c->cd * k, Jx + 6 * k);
}

/* sigma_0 (Eq. sigma0, with C^-1 as in Eq. normalw) over the active points */
double orc_sigma0(const orc_ctx *c) {
  double sum = 0.0;
  long long kact = 0, nact = 0;
  double v[2];
  for (int j = 0; j < c->N; j++) nact += c->active[j];
  for (int k = 0; k < c->K; k++) {
    int j = c->obs_pt[k];
    if (!c->active[j] || c->w[k] == 0.0) continue;  /* w = 0: deleted (serial robust variant) */
    obs_residual(c, k, c->R, c->t, c->X + 3 * j, v, NULL, NULL);
    sum += c->w[k] * quad_w(c->obs_winv + 3 * k, v);
    kact++;
  }
  double red = 2.0 * (double)kact - (double)c->cd * c->M - 3.0 * (double)nact + 7.0;
  if (red < 1.0) red = 1.0;
  return sqrt(sum / red);
}

/* RMS image residual [px] over active observations that are not down-weighted */
double orc_rms(const orc_ctx *c) {
  double sum = 0.0;
  long long n = 0;
  double v[2];
  for (int k = 0; k < c->K; k++) {
    int j = c->obs_pt[k];
    if (!c->active[j] || c->w[k] != 1.0) continue;
    obs_residual(c, k, c->R, c->t, c->X + 3 * j, v, NULL, NULL);
    sum += v[0] * v[0] + v[1] * v[1];
    n++;
  }
  return n ? sqrt(sum / (2.0 * (double)n)) : 0.0;
}

/* normal matrix of point j (cameras fixed) at position X: N = sum w A_X^T W A_X */
static int point_normal(const orc_ctx *c, int j, const double X[3], double N6[6]) {
  double v[2], Jx[6], full[9];
  memset(full, 0, sizeof(full));
  for (int p = c->pt_obs_ptr[j]; p < c->pt_obs_ptr[j + 1]; p++) {
    int k = c->pt_obs[p];
    double z = obs_residual(c, k, c->R, c->t, X, v, NULL, Jx);
    if (!(z > 0.0)) return 0;
    add_AtWB(Jx, 3, Jx, 3, c->obs_winv + 3 * k, c->w[k], full);
  }
  for (int r = 0; r < 3; r++)
    for (int s = r; s < 3; s++) N6[s3(r, s)] = full[r * 3 + s];
  return 1;
}

/* covariance C_j = N_j^-1 of the point with the cameras fixed (Eq. bars) */
void orc_covariance(const orc_ctx *c, const int *ids, int n, double *out9) {
  for (int a = 0; a < n; a++) {
    int j = ids[a];
    double N6[6], C6[6];
    int ok = (j >= 0 && j < c->N && c->active[j]) ? point_normal(c, j, c->X + 3 * j, N6) : 0;
    if (ok) ok = sym3_inverse(N6, C6) > 0.0;
    for (int r = 0; r < 3; r++)
      for (int s = 0; s < 3; s++) out9[9 * a + 3 * r + s] = ok ? C6[s3(r, s)] : NAN;
  }
}

double orc_median(double *a, int n) {
  if (n <= 0) return 0.0;
  qsort(a, (size_t)n, sizeof(double), cmp_d);
  return (n % 2) ? a[n / 2] : 0.5 * (a[n / 2 - 1] + a[n / 2]);
}

/* whitened residual components e with e^T e = v^T W v (upper Cholesky factor of W) */
static void whiten(const double W[3], const double v[2], double e[2]) {
  double a = sqrt(W[0]);
  e[0] = a * v[0] + (W[1] / a) * v[1];
  e[1] = sqrt(W[2] - W[1] * W[1] / W[0]) * v[1];
}

/* camera i: 1.4826 * median |e - median(e)| over its whitened components
 * (Sec. 5.3); buf holds at least 2 K_i doubles */
static double camera_scale_one(const orc_ctx *c, int i, double *buf) {
  double v[2], e[2];
  int n = 0;
  for (int p = c->cam_obs_ptr[i]; p < c->cam_obs_ptr[i + 1]; p++) {
    int k = c->cam_obs[p];
    int j = c->obs_pt[k];
    if (!c->active[j]) continue;
    obs_residual(c, k, c->R, c->t, c->X + 3 * j, v, NULL, NULL);
    whiten(c->obs_winv + 3 * k, v, e);
    buf[n++] = e[0];
    buf[n++] = e[1];
  }
  if (n == 0) return 0.0;
  double med = orc_median(buf, n);
  for (int a = 0; a < n; a++) buf[a] = fabs(buf[a] - med);
  return 1.4826 * orc_median(buf, n);
}

void orc_camera_scale(const orc_ctx *c, double *sigma) {
  double *buf = (double *)malloc(sizeof(double) * (size_t)(2 * c->K + 2));
  for (int i = 0; i < c->M; i++) sigma[i] = camera_scale_one(c, i, buf);
  free(buf);
}

/* observation k's robust weight from its camera's scale s: down-weighted when
 * sqrt(v^T C^-1 v) / s > t_v (Sec. 5.3); returns 1 when down-weighted */
static int robust_weight_one(orc_ctx *c, int k, double s, double t_v, double downweight) {
  double v[2];
  int j = c->obs_pt[k];
  obs_residual(c, k, c->R, c->t, c->X + 3 * j, v, NULL, NULL);
  double nr = sqrt(quad_w(c->obs_winv + 3 * k, v));
  int out = (s > 0.0) && (nr / s > t_v);
  c->w[k] = out ? downweight : 1.0;
  return out;
}

int orc_robust_weights(orc_ctx *c, double t_v, double downweight) {
  double *sigma = (double *)malloc(sizeof(double) * (size_t)(c->M > 0 ? c->M : 1));
  orc_camera_scale(c, sigma);
  int nd = 0;
  for (int k = 0; k < c->K; k++) {
    if (!c->active[c->obs_pt[k]]) continue;
    nd += robust_weight_one(c, k, sigma[c->obs_cam[k]], t_v, downweight);
  }
  free(sigma);
  return nd;
}

int orc_robust_weights_cams(orc_ctx *c, const int *cams, int n, double t_v, double downweight) {
  double *buf = (double *)malloc(sizeof(double) * (size_t)(2 * c->K + 2));
  int nd = 0;
  for (int a = 0; a < n; a++) {
    int i = cams[a];
    double s = camera_scale_one(c, i, buf);
    for (int p = c->cam_obs_ptr[i]; p < c->cam_obs_ptr[i + 1]; p++) {
      int k = c->cam_obs[p];
      if (!c->active[c->obs_pt[k]]) continue;
      nd += robust_weight_one(c, k, s, t_v, downweight);
    }
  }
  free(buf);
  return nd;
}

/* ------------------------------------------------------------------------ */
/* intersection, Eq. bars, and refined weights, Sec. 5.1                     */
/* ------------------------------------------------------------------------ */

/* Gauss-Newton on X_j with all cameras fixed. On success X is the new
 * position, Ntot the normal matrix of the last iteration and Nl (one sym3 per
 * instance of j, in the point's instance order) its per-sub-block parts. */
static int intersect_point(const orc_ctx *c, const orc_options *o, int j, double X[3],
                           double Ntot[6], double *Nl) {
  int q0 = c->pt_inst_ptr[j], nq = c->pt_inst_ptr[j + 1] - q0;
  double v[2], Jx[6];
  for (int it = 0; it < o->isect_max_iter; it++) {
    double full[9], g[3] = {0.0, 0.0, 0.0};
    memset(full, 0, sizeof(full));
    memset(Nl, 0, sizeof(double) * 6 * nq);
    for (int p = c->pt_obs_ptr[j]; p < c->pt_obs_ptr[j + 1]; p++) {
      int k = c->pt_obs[p];
      double z = obs_residual(c, k, c->R, c->t, X, v, NULL, Jx);
      if (!(z > 0.0)) return 0;
      const double *W = c->obs_winv + 3 * k;
      double part[9];
      memset(part, 0, sizeof(part));
      add_AtWB(Jx, 3, Jx, 3, W, c->w[k], part);
      for (int e = 0; e < 9; e++) full[e] += part[e];
      add_AtWB(Jx, 3, v, 1, W, c->w[k], g);
      int qi = 0;
      while (c->pt_inst[q0 + qi] != c->obs_inst[k]) qi++;
      for (int r = 0; r < 3; r++)
        for (int s = r; s < 3; s++) Nl[6 * qi + s3(r, s)] += part[r * 3 + s];
    }
    for (int r = 0; r < 3; r++)
      for (int s = r; s < 3; s++) Ntot[s3(r, s)] = full[r * 3 + s];
    double inv[6];
    double det = sym3_inverse(Ntot, inv);
    if (!(det > 0.0)) return 0;
    if (!(sym3_frob(Ntot) * sym3_frob(inv) <= o->cond_max)) return 0;
    double d[3], Nd[3];
    sym3_mul_vec(inv, g, d);
    for (int e = 0; e < 3; e++) X[e] -= d[e];
    double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double nx = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    if (nd <= o->isect_tol * (1.0 + nx)) return 1;
    /* image-space size of the step: dX^T N dX = sum_k w ||W^1/2 A_X,k dX||^2 */
    sym3_mul_vec(Ntot, d, Nd);
    int nobs = c->pt_obs_ptr[j + 1] - c->pt_obs_ptr[j];
    if (d[0] * Nd[0] + d[1] * Nd[1] + d[2] * Nd[2] <= o->isect_px_tol * o->isect_px_tol * nobs) return 1;
  }
  return 0;
}

/* Eq. bars for point j (skipped when inactive, or a single-instance point
 * with tp_only): X_j, or the point dropped; W^l of its instances (Sec. 5.1).
 * Returns 1 when it drops the point. */
static int intersect_one(orc_ctx *c, const orc_options *o, int j, int tp_only, double *Nl) {
  if (!c->active[j]) return 0;
  int q0 = c->pt_inst_ptr[j], nq = c->pt_inst_ptr[j + 1] - q0;
  if (tp_only && nq < 2) return 0;
  double X[3] = {c->X[3 * j], c->X[3 * j + 1], c->X[3 * j + 2]};
  double Ntot[6];
  if (!intersect_point(c, o, j, X, Ntot, Nl)) {
    c->active[j] = 0;
    for (int qi = 0; qi < nq; qi++) memset(c->Wl + 6 * c->pt_inst[q0 + qi], 0, 6 * sizeof(double));
    return 1;
  }
  for (int e = 0; e < 3; e++) c->X[3 * j + e] = X[e];
  for (int qi = 0; qi < nq; qi++) {
    double *W = c->Wl + 6 * c->pt_inst[q0 + qi];
    for (int e = 0; e < 6; e++) {
      double refined = Ntot[e] - Nl[6 * qi + e];           /* Sec. 5.1 */
      double all = Ntot[e];                                /* all cameras (Sec. 6.4) */
      double scalar = (e == 0 || e == 3 || e == 5) ? o->rho : 0.0;  /* rho I (Sec. 6.4) */
      double val = o->weight_mode == 1 ? all : (o->weight_mode == 2 ? scalar : refined);
      W[e] = (nq >= 2) ? val : 0.0;
    }
  }
  return 0;
}

static double *instance_scratch(const orc_ctx *c) {
  int maxq = 1;
  for (int j = 0; j < c->N; j++) {
    int nq = c->pt_inst_ptr[j + 1] - c->pt_inst_ptr[j];
    if (nq > maxq) maxq = nq;
  }
  return (double *)malloc(sizeof(double) * 6 * (size_t)maxq);
}

int orc_intersect(orc_ctx *c, const orc_options *o, int tp_only) {
  int dropped = 0;
  double *Nl = instance_scratch(c);
  for (int j = 0; j < c->N; j++) dropped += intersect_one(c, o, j, tp_only, Nl);
  free(Nl);
  return dropped;
}

int orc_intersect_points(orc_ctx *c, const orc_options *o, const int *ids, int n, int tp_only) {
  int dropped = 0;
  double *Nl = instance_scratch(c);
  for (int a = 0; a < n; a++) dropped += intersect_one(c, o, ids[a], tp_only, Nl);
  free(Nl);
  return dropped;
}

/* ------------------------------------------------------------------------ */
/* sub-block adjustment with TPs as control points, Eq. batp / bact          */
/* ------------------------------------------------------------------------ */

/* F_l for given camera arrays (global indexing) and instance positions */
static double sub_cost_at(const orc_ctx *c, int l, const double *R, const double *t,
                          const double *intr, const double *k1, const double *Xl) {
  double F = 0.0, v[2];
  for (int q = c->sub_inst_ptr[l]; q < c->sub_inst_ptr[l + 1]; q++) {
    int j = c->inst_pt[q];
    if (!c->active[j]) continue;
    for (int p = c->inst_obs_ptr[q]; p < c->inst_obs_ptr[q + 1]; p++) {
      int k = c->inst_obs[p];
      double z = obs_residual_at(c, k, R, t, intr, k1, Xl + 3 * q, v, NULL, NULL);
      if (!(z > 0.0)) return INFINITY;
      F += c->w[k] * quad_w(c->obs_winv + 3 * k, v);
    }
    double d[3], Wd[3];
    for (int e = 0; e < 3; e++) d[e] = Xl[3 * q + e] - c->X[3 * j + e];
    sym3_mul_vec(c->Wl + 6 * q, d, Wd);
    F += d[0] * Wd[0] + d[1] * Wd[1] + d[2] * Wd[2];
  }
  return F;
}

double orc_sub_cost(const orc_ctx *c, int l) { return sub_cost_at(c, l, c->R, c->t, c->intr, c->k1, c->Xl); }

/* Normal equations of sub-block l, damped, reduced to the cameras (Sec. 2,
 * Sec. 5.5). For every instance q of l also returns Ninv (inverse of the
 * damped point block, sym3) and gX (the point gradient). */
static int rcs_build(const orc_ctx *c, int l, double lambda, double *S, double *y,
                     double *Ninv, double *gX) {
  const int cd = c->cd;
  int c0 = c->sub_cam_ptr[l], Ml = c->sub_cam_ptr[l + 1] - c0;
  int n = cd * Ml;
  memset(S, 0, sizeof(double) * (size_t)n * n);
  memset(y, 0, sizeof(double) * n);
  double *NCC = (double *)calloc((size_t)cd * cd * (Ml > 0 ? Ml : 1), sizeof(double));
  double *gC = (double *)calloc((size_t)cd * (Ml > 0 ? Ml : 1), sizeof(double));
  int mmax = c->max_inst_obs;
  double *NXC = (double *)malloc(sizeof(double) * 3 * cd * mmax);
  int *loc = (int *)malloc(sizeof(int) * mmax);
  double v[2], Jc[16], Jx[6];
  int q0 = c->sub_inst_ptr[l];
  for (int q = q0; q < c->sub_inst_ptr[l + 1]; q++) {
    int j = c->inst_pt[q];
    double *Ni = Ninv + 6 * (q - q0), *g = gX + 3 * (q - q0);
    memset(Ni, 0, 6 * sizeof(double));
    memset(g, 0, 3 * sizeof(double));
    if (!c->active[j]) continue;
    double NXX[9];
    memset(NXX, 0, sizeof(NXX));
    int m = 0;
    for (int p = c->inst_obs_ptr[q]; p < c->inst_obs_ptr[q + 1]; p++, m++) {
      int k = c->inst_obs[p];
      int li = c->cam_local[c->obs_cam[k]];
      loc[m] = li;
      obs_residual(c, k, c->R, c->t, c->Xl + 3 * q, v, Jc, Jx);
      const double *W = c->obs_winv + 3 * k;
      double wk = c->w[k];
      add_AtWB(Jc, cd, Jc, cd, W, wk, NCC + cd * cd * li); /* N_CC block of camera i */
      add_AtWB(Jc, cd, v, 1, W, wk, gC + cd * li);         /* camera gradient */
      add_AtWB(Jx, 3, Jx, 3, W, wk, NXX);                  /* N_XX */
      add_AtWB(Jx, 3, v, 1, W, wk, g);                     /* point gradient */
      memset(NXC + 3 * cd * m, 0, 3 * cd * sizeof(double));
      add_AtWB(Jx, 3, Jc, cd, W, wk, NXC + 3 * cd * m);    /* N_XC block (3 x cd) */
    }
    /* TP as control point: + (X^l - X_TP)^T W^l (X^l - X_TP) */
    const double *Wl = c->Wl + 6 * q;
    double d[3], Wd[3];
    for (int e = 0; e < 3; e++) d[e] = c->Xl[3 * q + e] - c->X[3 * j + e];
    sym3_mul_vec(Wl, d, Wd);
    for (int r = 0; r < 3; r++) {
      g[r] += Wd[r];
      for (int s = 0; s < 3; s++) NXX[r * 3 + s] += Wl[s3(r, s)];
    }
    /* damping of the point block */
    double N6[6];
    for (int r = 0; r < 3; r++)
      for (int s = r; s < 3; s++) N6[s3(r, s)] = NXX[r * 3 + s] + (r == s ? lambda * NXX[r * 3 + s] : 0.0);
    sym3_inverse(N6, Ni);
    /* Schur complement: S_ab -= N_XC,a^T Ninv N_XC,b ; y_a += N_XC,a^T Ninv g */
    double Ng[3];
    sym3_mul_vec(Ni, g, Ng);
    for (int a = 0; a < m; a++) {
      const double *Ba = NXC + 3 * cd * a;
      for (int r = 0; r < cd; r++) {
        double acc = 0.0;
        for (int e = 0; e < 3; e++) acc += Ba[e * cd + r] * Ng[e];
        y[cd * loc[a] + r] += acc;
      }
      for (int b = 0; b < m; b++) {
        const double *Bb = NXC + 3 * cd * b;
        double NB[24]; /* Ninv * N_XC,b */
        for (int e = 0; e < 3; e++)
          for (int s = 0; s < cd; s++) {
            double acc = 0.0;
            for (int f = 0; f < 3; f++) acc += Ni[s3(e, f)] * Bb[f * cd + s];
            NB[e * cd + s] = acc;
          }
        for (int r = 0; r < cd; r++)
          for (int s = 0; s < cd; s++) {
            double acc = 0.0;
            for (int e = 0; e < 3; e++) acc += Ba[e * cd + r] * NB[e * cd + s];
            S[(size_t)(cd * loc[a] + r) * n + cd * loc[b] + s] -= acc;
          }
      }
    }
  }
  /* camera blocks, damped, and the camera gradient */
  for (int li = 0; li < Ml; li++)
    for (int r = 0; r < cd; r++) {
      y[cd * li + r] -= gC[cd * li + r];
      for (int s = 0; s < cd; s++) {
        double nv = NCC[cd * cd * li + r * cd + s];
        S[(size_t)(cd * li + r) * n + cd * li + s] += nv + (r == s ? lambda * nv : 0.0);
      }
    }
  free(NCC); free(gC); free(NXC); free(loc);
  return n;
}

int orc_rcs(const orc_ctx *c, int l, double lambda, double *S, double *y) {
  int nP = c->sub_inst_ptr[l + 1] - c->sub_inst_ptr[l];
  double *Ninv = (double *)malloc(sizeof(double) * 6 * (size_t)(nP > 0 ? nP : 1));
  double *gX = (double *)malloc(sizeof(double) * 3 * (size_t)(nP > 0 ? nP : 1));
  int n = rcs_build(c, l, lambda, S, y, Ninv, gX);
  free(Ninv); free(gX);
  return n;
}

int orc_lm_step(orc_ctx *c, int l, double lambda, double *F_before, double *F_trial,
                double *dc_out, double *dx_out) {
  const int cd = c->cd;
  int c0 = c->sub_cam_ptr[l], Ml = c->sub_cam_ptr[l + 1] - c0;
  int q0 = c->sub_inst_ptr[l], nP = c->sub_inst_ptr[l + 1] - q0;
  int n = cd * Ml;
  double F0 = orc_sub_cost(c, l);
  if (F_before) *F_before = F0;
  if (F_trial) *F_trial = F0;
  if (Ml == 0) return 0;
  double *S = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *y = (double *)malloc(sizeof(double) * n);
  double *Ninv = (double *)malloc(sizeof(double) * 6 * (size_t)(nP > 0 ? nP : 1));
  double *gX = (double *)malloc(sizeof(double) * 3 * (size_t)(nP > 0 ? nP : 1));
  double *dx = (double *)calloc((size_t)3 * (nP > 0 ? nP : 1), sizeof(double));
  rcs_build(c, l, lambda, S, y, Ninv, gX);
  int result = -1;
  if (cholesky(S, n)) {
    cholesky_solve(S, n, y); /* y now holds the camera update d_C */
    /* back-substitution: dX = Ninv (-g_X - sum_k N_XC,k dC_i(k)) */
    double v[2], Jc[16], Jx[6];
    for (int q = q0; q < q0 + nP; q++) {
      int j = c->inst_pt[q];
      if (!c->active[j]) continue;
      double rhs[3];
      for (int e = 0; e < 3; e++) rhs[e] = -gX[3 * (q - q0) + e];
      for (int p = c->inst_obs_ptr[q]; p < c->inst_obs_ptr[q + 1]; p++) {
        int k = c->inst_obs[p];
        int li = c->cam_local[c->obs_cam[k]];
        obs_residual(c, k, c->R, c->t, c->Xl + 3 * q, v, Jc, Jx);
        double B[24];
        memset(B, 0, sizeof(B));
        add_AtWB(Jx, 3, Jc, cd, c->obs_winv + 3 * k, c->w[k], B);
        for (int e = 0; e < 3; e++)
          for (int s = 0; s < cd; s++) rhs[e] -= B[e * cd + s] * y[cd * li + s];
      }
      sym3_mul_vec(Ninv + 6 * (q - q0), rhs, dx + 3 * (q - q0));
    }
    /* trial state: only the cameras and instances of sub-block l are set and
     * read (its observations see only its cameras), so sub-blocks can take
     * their steps on separate threads */
    double *Rt = (double *)malloc(sizeof(double) * 9 * c->M);
    double *tt = (double *)malloc(sizeof(double) * 3 * c->M);
    double *it = (double *)malloc(sizeof(double) * 3 * c->M);
    double *kt = (double *)malloc(sizeof(double) * (c->M > 0 ? c->M : 1));
    double *Xt = (double *)malloc(sizeof(double) * 3 * (size_t)(c->P > 0 ? c->P : 1));
    for (int li = 0; li < Ml; li++) {
      int i = c->sub_cam[c0 + li];
      double dR[9];
      orc_rodrigues(y + cd * li, dR);
      for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
          double acc = 0.0;
          for (int m = 0; m < 3; m++) acc += dR[r * 3 + m] * c->R[9 * i + m * 3 + s];
          Rt[9 * i + r * 3 + s] = acc;
        }
      for (int e = 0; e < 3; e++) tt[3 * i + e] = c->t[3 * i + e] + y[cd * li + 3 + e];
      for (int e = 0; e < 3; e++) it[3 * i + e] = c->intr[3 * i + e];
      kt[i] = c->k1[i];
      if (cd == 8) {
        it[3 * i] += y[cd * li + 6];
        kt[i] += y[cd * li + 7];
      }
    }
    for (int q = q0; q < q0 + nP; q++)
      for (int e = 0; e < 3; e++) Xt[3 * q + e] = c->Xl[3 * q + e] + dx[3 * (q - q0) + e];
    double F1 = sub_cost_at(c, l, Rt, tt, it, kt, Xt);
    if (F_trial) *F_trial = F1;
    if (dc_out) memcpy(dc_out, y, sizeof(double) * n);
    if (dx_out) memcpy(dx_out, dx, sizeof(double) * 3 * nP);
    if (F1 < F0) {
      for (int li = 0; li < Ml; li++) {
        int i = c->sub_cam[c0 + li];
        memcpy(c->R + 9 * i, Rt + 9 * i, sizeof(double) * 9);
        memcpy(c->t + 3 * i, tt + 3 * i, sizeof(double) * 3);
        c->intr[3 * i] = it[3 * i];
        c->k1[i] = kt[i];
      }
      memcpy(c->Xl + 3 * (size_t)q0, Xt + 3 * (size_t)q0, sizeof(double) * 3 * nP);
      result = 1;
    } else {
      result = 0;
    }
    free(Rt); free(tt); free(it); free(kt); free(Xt);
  }
  free(S); free(y); free(Ninv); free(gX); free(dx);
  return result;
}

/* LM damping after a step. The paper keeps lambda fixed (Sec. 5.5) and is
 * silent on a rejected step; the reading taken here: x10 after a rejected
 * step, /10 floored at lambda0 after an accepted one. */
double orc_lambda_next(double lambda, int accepted, double lambda0) {
  if (!accepted) return lambda * 10.0;
  return lambda / 10.0 > lambda0 ? lambda / 10.0 : lambda0;
}

/* The stop rule of the inner (F_l) and the outer (sigma_0) loop (Sec. 5.5):
 * after a new value v, ratio = best / v with best the smallest value before
 * v; best then becomes min(best, v). A ratio below stop_ratio uses up one
 * grace iteration if one is left, and otherwise ends the loop (returns 1). */
int orc_ratio_rule(double *best, double v, double stop_ratio, int *grace) {
  double ratio = *best / (v > 1e-300 ? v : 1e-300);
  if (v < *best) *best = v;
  if (ratio >= stop_ratio) return 0;
  if (*grace > 0) {
    (*grace)--;
    return 0;
  }
  return 1;
}

/* the LM loop of one sub-block (one solution of Eq. bact). A rejected step
 * raises lambda and retries; the best/current ratio rule (Sec. 5.5) is
 * applied to accepted steps; more than max_reject rejections in a row end the
 * loop. With a trace (cap > 0), iteration it records the damping it used,
 * whether its step was accepted and the cost F_l after it. */
int orc_sub_lm_trace(orc_ctx *c, int l, const orc_options *o, double *F_hist, double *lambda_hist,
                     int *acc_hist, int cap) {
  if (c->sub_cam_ptr[l + 1] == c->sub_cam_ptr[l]) return 0;
  double lambda = o->lambda0;
  double F = orc_sub_cost(c, l);
  double best = F;
  int grace = o->grace;
  int rejects = 0;
  int it = 0;
  while (it < o->max_inner) {
    double Fb, Ft;
    int r = orc_lm_step(c, l, lambda, &Fb, &Ft, NULL, NULL);
    if (it < cap) {
      lambda_hist[it] = lambda;
      acc_hist[it] = r;
      F_hist[it] = r == 1 ? Ft : F;
    }
    it++;
    if (r != 1) {
      lambda = orc_lambda_next(lambda, 0, o->lambda0);
      if (++rejects > o->max_reject) break;
      continue;
    }
    rejects = 0;
    F = Ft;
    lambda = orc_lambda_next(lambda, 1, o->lambda0);
    if (orc_ratio_rule(&best, F, o->stop_ratio, &grace)) break;
  }
  return it;
}

int orc_sub_lm(orc_ctx *c, int l, const orc_options *o) {
  return orc_sub_lm_trace(c, l, o, NULL, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* the whole method                                                          */
/* ------------------------------------------------------------------------ */

static void tp_copies_from_points(orc_ctx *c, int tp_only) {
  for (int q = 0; q < c->P; q++) {
    int j = c->inst_pt[q];
    int nq = c->pt_inst_ptr[j + 1] - c->pt_inst_ptr[j];
    if (tp_only && nq < 2) continue;
    for (int e = 0; e < 3; e++) c->Xl[3 * q + e] = c->X[3 * j + e];
  }
}

void orc_run(orc_ctx *c, const orc_options *o_in, orc_report *r) {
  /* rho of the scalar weight: rho0 at the first intersection, times 1.01
   * for every outer iteration after it */
  orc_options oo = *o_in;
  orc_options *o = &oo;
  o->rho = o->rho0;
  memset(r, 0, sizeof(*r));
  r->robust_started_at = -1;
  int n_start = 0;
  for (int j = 0; j < c->N; j++) n_start += c->active[j];
  /* initial intersection of all points gives X_TP and W^l for the first bact */
  orc_intersect(c, o, 0);
  tp_copies_from_points(c, 0);
  double s = orc_sigma0(c);
  r->sigma0_initial = s;
  double best = s;
  int grace = o->grace;
  int robust_on = 0;
  for (int outer = 0; outer < o->max_outer; outer++) {
    /* bact: every sub-block independently */
    for (int l = 0; l < c->L; l++) r->inner_total += orc_sub_lm(c, l, o);
    /* exchange: cameras are unique to their sub-block and already global;
     * points seen in one sub-block take that sub-block's position */
    for (int j = 0; j < c->N; j++) {
      int q0 = c->pt_inst_ptr[j];
      if (c->active[j] && c->pt_inst_ptr[j + 1] - q0 == 1)
        for (int e = 0; e < 3; e++) c->X[3 * j + e] = c->Xl[3 * c->pt_inst[q0] + e];
    }
    if (o->robust && o->robust_from_start && !robust_on) {
      robust_on = 1;
      r->robust_started_at = r->outer;
    }
    if (robust_on) orc_robust_weights(c, o->t_v, o->downweight);
    /* bars: intersection of the TPs with all cameras fixed */
    o->rho *= 1.01;
    orc_intersect(c, o, 1);
    tp_copies_from_points(c, 1);
    s = orc_sigma0(c);
    if (r->outer < 128) r->sigma0_hist[r->outer] = s;
    r->outer++;
    if (orc_ratio_rule(&best, s, o->stop_ratio, &grace)) {
      if (o->robust && !robust_on) {
        robust_on = 1;
        r->robust_started_at = r->outer;
        orc_robust_weights(c, o->t_v, o->downweight);
        orc_intersect(c, o, 1);
        tp_copies_from_points(c, 1);
        best = orc_sigma0(c);
        grace = o->grace;
        continue;
      }
      break;
    }
  }
  if (robust_on && o->robust_serial) {
    /* serial variant (Sec. 5.3): the down-weighted observations are deleted
     * (weight 0); a point seen by fewer than two cameras afterwards is
     * eliminated */
    int *cnt = (int *)calloc((size_t)(c->N > 0 ? c->N : 1), sizeof(int));
    for (int k = 0; k < c->K; k++) {
      if (c->w[k] != 1.0) c->w[k] = 0.0;
      else cnt[c->obs_pt[k]]++;
    }
    for (int j = 0; j < c->N; j++)
      if (cnt[j] < 2) c->active[j] = 0;
    free(cnt);
  } else if (robust_on) {
    /* parallel variant: eliminate every point with a down-weighted
     * observation (Sec. 5.3) */
    for (int k = 0; k < c->K; k++)
      if (c->w[k] != 1.0) c->active[c->obs_pt[k]] = 0;
  }
  r->sigma0 = orc_sigma0(c);
  r->rms = orc_rms(c);
  int n_act = 0, k_act = 0;
  for (int j = 0; j < c->N; j++) n_act += c->active[j];
  for (int k = 0; k < c->K; k++) k_act += c->active[c->obs_pt[k]];
  r->active_points = n_act;
  r->active_obs = k_act;
  r->deleted_points = n_start - n_act;
}
