/*
 * rpba_oracle.h -- plain, slow FP64 CPU oracle of the RPBA iteration.
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA path; it is
 * used by the tests, by the smoke check and by the timed CPU-baseline leg of
 * the benchmark, and by nothing else. It shares no code with the CUDA path.
 *
 * What it computes (Mayer, "RPBA - Robust Parallel Bundle Adjustment Based on
 * Covariance Information"):
 *   - projection g_k and residual v_k = g_k(P_i, X_j) - x_k          (Sec. 2)
 *   - weighted cost sum_k w_k v_k^T C_k^-1 v_k                        (Eq. v2, normalw)
 *   - linearisation, normal equations, Schur reduced camera system   (Eq. ta, normal, normalw; Sec. 2)
 *   - LM damping N + lambda diag(N)                                  (Sec. 5.5)
 *   - sub-block adjustment with tie points as weighted control points (Eq. batp, bact)
 *   - intersection of each point with the cameras fixed, its normal
 *     matrix, covariance, refined per-sub-block weights              (Eq. bars; Sec. 5.1)
 *   - sigma_0, per-camera MAD scale, robust down-weighting,
 *     elimination of points                                          (Eq. sigma0; Sec. 5.3)
 *   - convergence by best/current ratio below 1.01 with one grace
 *     iteration                                                      (Sec. 5.5)
 *
 * Storage conventions
 *   pose    : (omega[3], t[3]) per camera, X_c = R(omega) X + t
 *   intr    : (f, cx, cy) per camera, u = f x_c/z_c + cx, v = f y_c/z_c + cy
 *   sym3    : 6 doubles (a00, a01, a02, a11, a12, a22)
 *   winv    : (w11, w12, w22) of C_k^-1 per observation (NULL = identity)
 *   Jc      : 2x6 row-major d(u,v)/d(dw, dt), dw a left-multiplied incremental rotation
 *             (2x8 with per-camera intrinsics: (dw, dt, df, dk1))
 *   Jx      : 2x3 row-major d(u,v)/dX
 *   instance: a (point j, sub-block l) pair for every sub-block l whose cameras
 *             observe j, in canonical order sorted by (l, j). A tie point (TP) is
 *             a point with two or more instances.
 */
#ifndef RPBA_ORACLE_H
#define RPBA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

typedef struct {
  double lambda0;      /* LM damping factor, 1e-4 (Sec. 5.5) */
  double t_v;          /* robust threshold on the normalised residual, 4 (Sec. 5.3) */
  double downweight;   /* weight of a detected outlier, 1e-4 (Sec. 5.3) */
  double stop_ratio;   /* best/current ratio that ends an iteration loop, 1.01 (Sec. 5.5) */
  int grace;           /* non-improving iterations allowed, 1 (Sec. 5.5) */
  int max_outer;       /* cap on bact/bars iterations */
  int max_inner;       /* cap on LM iterations per sub-block and outer iteration */
  int max_reject;      /* rejected LM steps in a row that end the LM loop */
  int robust;          /* 1: robust stage after first convergence (Sec. 5.3) */
  int robust_from_start; /* 1: robust weights from the first intersection after the first bact */
  int isect_max_iter;  /* Gauss-Newton iterations of the intersection, 10 */
  double isect_tol;    /* ||dX|| <= tol (1 + ||X||) ends the intersection, 1e-10 */
  double isect_px_tol; /* or a step moving the image residuals by < this per observation, 1e-3 px */
  double cond_max;     /* Frobenius condition number above which a point is dropped, 1e12 */
  int robust_serial;   /* 1: the serial variant of Sec. 5.3 at the end of the robust stage
                          (delete the down-weighted observations, eliminate points left with
                          fewer than two); 0: the parallel variant (eliminate every point with a
                          down-weighted observation) */
  int weight_mode;     /* the TPs' weight W^l in the other sub-blocks: 0 the refined weight of
                          Sec. 5.1 (normal matrix without sub-block l), 1 the normal matrix of all
                          cameras, 2 a scalar rho I (the ablations of Sec. 6.4) */
  double rho0;         /* weight_mode 2: rho of the first intersection, times 1.01 per outer
                          iteration (the plain approach's schedule, Sec. 6.3; 200) */
  double rho;          /* the rho in effect (set by orc_run; for a direct orc_intersect, rho0) */
} orc_options;

typedef struct {
  double sigma0;       /* final sigma_0 (Eq. sigma0) */
  double rms;          /* final RMS reprojection error over active, unweighted-down obs [px] */
  double sigma0_initial;
  int outer;           /* bact/bars iterations done */
  int inner_total;     /* LM iterations summed over sub-blocks */
  int deleted_points;  /* points eliminated (robust stage + failed intersections) */
  int active_points;
  int active_obs;
  int robust_started_at; /* outer iteration at which the robust stage began, -1 if never */
  double sigma0_hist[128];
} orc_report;

void orc_default_options(orc_options *o);

/* All arrays are copied. cam_sub: sub-block id per camera (0..L-1, each used). */
orc_ctx *orc_create(int n_cams, int n_points, int n_obs, const double *cam_pose,
                    const double *cam_intr, const double *points, const int *obs_cam,
                    const int *obs_point, const double *obs_xy, const double *obs_winv,
                    const int *cam_sub);
void orc_destroy(orc_ctx *c);

int orc_num_subblocks(const orc_ctx *c);
int orc_num_instances(const orc_ctx *c);
void orc_instances(const orc_ctx *c, int *inst_point, int *inst_sub);
/* cameras of sub-block l in the order of the RCS rows (ascending global id) */
int orc_sub_cameras(const orc_ctx *c, int l, int *cams);

/* state */
void orc_get_cameras(const orc_ctx *c, double *pose);
void orc_set_cameras(orc_ctx *c, const double *pose);
/* the rotation matrices (9 per camera, row-major) and translations as held */
void orc_get_camera_rt(const orc_ctx *c, double *R, double *t);
void orc_set_camera_rt(orc_ctx *c, const double *R, const double *t);
void orc_get_points(const orc_ctx *c, double *X, unsigned char *active);
void orc_set_points(orc_ctx *c, const double *X, const unsigned char *active);
void orc_get_instances(const orc_ctx *c, double *Xl, double *Wl);
void orc_set_instances(orc_ctx *c, const double *Xl, const double *Wl);
void orc_get_weights(const orc_ctx *c, double *w);
void orc_set_weights(orc_ctx *c, const double *w);

/* geometry */
void orc_rodrigues(const double w[3], double R[9]);
void orc_rotation_log(const double R[9], double w[3]);
/* returns depth z_c; uv, Jc, Jx may be NULL */
double orc_project(const double R[9], const double t[3], const double intr[3],
                   const double X[3], double uv[2], double Jc[12], double Jx[6]);

/* the same with the first radial distortion parameter k1 (Sec. 6, the Final
 * data sets): p = (x_c, y_c)/z_c, (u, v) = f (1 + k1 |p|^2) p + (cx, cy);
 * Jc is 2x8 row-major d(u,v)/d(dw, dt, df, dk1) */
double orc_project_k1(const double R[9], const double t[3], const double intr[3], double k1,
                      const double X[3], double uv[2], double Jc[16], double Jx[6]);

/* per-camera intrinsics: from this call on, f and k1 of every camera are
 * unknowns (8 per camera) and the projection includes k1 (initial values k1,
 * or 0 when NULL) */
void orc_enable_intrinsics(orc_ctx *c, const double *k1);
int orc_camera_dim(const orc_ctx *c); /* 6, or 8 with intrinsics */
void orc_get_intrinsics(const orc_ctx *c, double *fk); /* (f, k1) per camera */
void orc_set_intrinsics(orc_ctx *c, const double *fk);

/* evaluations at the global state (cameras, points X) */
void orc_residuals(const orc_ctx *c, double *v);
void orc_jacobians(const orc_ctx *c, double *Jc, double *Jx);
double orc_sigma0(const orc_ctx *c);
double orc_rms(const orc_ctx *c);
void orc_covariance(const orc_ctx *c, const int *ids, int n, double *out9);
/* per-camera robust scale 1.4826 * MAD of the whitened residual components */
void orc_camera_scale(const orc_ctx *c, double *sigma);
double orc_median(double *a, int n); /* sorts a */
/* robust weights from the per-camera scale; returns the number down-weighted */
int orc_robust_weights(orc_ctx *c, double t_v, double downweight);
/* the same for the observations of the listed cameras only */
int orc_robust_weights_cams(orc_ctx *c, const int *cams, int n, double t_v, double downweight);

/* intersection (Eq. bars) of all active points (tp_only = 0) or of the tie
 * points only (tp_only = 1), starting at the current X. Writes X, the
 * per-instance weights W^l (Sec. 5.1) and drops points that fail. Returns the
 * number of points dropped. */
int orc_intersect(orc_ctx *c, const orc_options *o, int tp_only);
/* the same for the listed points only */
int orc_intersect_points(orc_ctx *c, const orc_options *o, const int *ids, int n, int tp_only);

/* sub-block l: cost F_l (Eq. bact) at the current sub-block state */
double orc_sub_cost(const orc_ctx *c, int l);
/* damped reduced camera system of sub-block l at the current state;
 * S is n x n row-major (n = 6 * cameras in l, 8 * with intrinsics), y has n
 * entries. Returns n. */
int orc_rcs(const orc_ctx *c, int l, double lambda, double *S, double *y);
/* one LM iteration of sub-block l with damping lambda: solve, trial, accept if
 * the cost decreases. Returns 1 accepted, 0 rejected, -1 solve failed.
 * dc (n) and dx (instances of l x 3) may be NULL. */
int orc_lm_step(orc_ctx *c, int l, double lambda, double *F_before, double *F_trial,
                double *dc, double *dx);
/* the LM loop of sub-block l (one bact); returns the number of iterations */
int orc_sub_lm(orc_ctx *c, int l, const orc_options *o);
/* the same loop; iteration it < cap records the damping it used, its result
 * (as orc_lm_step) and the cost F_l after it */
int orc_sub_lm_trace(orc_ctx *c, int l, const orc_options *o, double *F_hist, double *lambda_hist,
                     int *acc_hist, int cap);
/* the damping after a step: x10 after a rejection, /10 floored at lambda0
 * after an acceptance (reading of Sec. 5.5) */
double orc_lambda_next(double lambda, int accepted, double lambda0);
/* the stop rule of both loops (Sec. 5.5): ratio = best / v, best = min(best,
 * v); below stop_ratio one grace iteration, then stop (returns 1) */
int orc_ratio_rule(double *best, double v, double stop_ratio, int *grace);

/* whole method: initial intersection, bact/bars iterations, robust stage */
void orc_run(orc_ctx *c, const orc_options *o, orc_report *r);

#ifdef __cplusplus
}
#endif
#endif
