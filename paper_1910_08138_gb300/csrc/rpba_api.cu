// rpba_api.cu -- C ABI of the GB300 RPBA library (include/rpba.h): context
// creation (validation, sub-block topology, device layout), state access, and
// the host driver of the iteration of Sec. 5 (bact of all sub-blocks in lock
// step, exchange, bars, convergence, robust stage).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>

#include "rpba_internal.cuh"

using namespace rpba;


namespace rpba {

// ---------------------------------------------------------------------------
// pose <-> rotation, covariance
// ---------------------------------------------------------------------------
__global__ void k_pose_to_R(int M, const double *pose, double *R, double *t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double w[3] = {pose[6 * i], pose[6 * i + 1], pose[6 * i + 2]};
  rodrigues(w, R + 9 * i);
  for (int e = 0; e < 3; e++) t[3 * i + e] = pose[6 * i + 3 + e];
}

// angle-axis vector of R: theta = atan2(|v| / 2, (tr R - 1) / 2) with v the
// skew part (2 sin(theta) axis); close to theta = pi the axis is taken from
// the symmetric part, whose conditioning does not degrade there
__global__ void k_R_to_pose(int M, const double *R, const double *t, double *pose) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double *Q = R + 9 * i;
  double c = 0.5 * (Q[0] + Q[4] + Q[8] - 1.0);
  double v[3] = {Q[7] - Q[5], Q[2] - Q[6], Q[3] - Q[1]};
  double sn = 0.5 * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double th = atan2(sn, c);
  double w[3];
  if (th < 1e-6) {
    double f = 0.5 * (1.0 + th * th / 6.0);
    for (int e = 0; e < 3; e++) w[e] = f * v[e];
  } else if (th < 3.14159265358979323846 - 1e-3) {
    double f = th / (2.0 * sn);
    for (int e = 0; e < 3; e++) w[e] = f * v[e];
  } else {
    double B[3] = {(Q[0] - c) / (1.0 - c), (Q[4] - c) / (1.0 - c), (Q[8] - c) / (1.0 - c)};
    int k = 0;
    if (B[1] > B[k]) k = 1;
    if (B[2] > B[k]) k = 2;
    double a[3];
    a[k] = sqrt(fmax(B[k], 0.0));
    for (int e = 0; e < 3; e++)
      if (e != k) a[e] = (Q[3 * k + e] + Q[3 * e + k]) / (2.0 * (1.0 - c) * a[k]);
    double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double sg = (a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) < 0.0 ? -1.0 : 1.0;
    for (int e = 0; e < 3; e++) w[e] = sg * th * a[e] / n;
  }
  for (int e = 0; e < 3; e++) {
    pose[6 * i + e] = w[e];
    pose[6 * i + 3 + e] = t[3 * i + e];
  }
}

// C_j = N_j^-1 with N_j = sum_k w A_X^T W A_X over all observations of j
__global__ void k_covariance(int n, const int *ids, const double *R, const double *t, const double *intr,
                             const double *k1, const double *X, const uint8_t *active, const int *pt_inst_ptr, const int *pt_inst,
                             const int *inst_obs_ptr, const int *obs_cam, const double *obs_winv, int has_winv,
                             const double *obs_w, int N, double *out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  int j = ids[a];
  bool ok = j >= 0 && j < N && active[j];
  double Nm[6] = {0, 0, 0, 0, 0, 0};
  if (ok) {
    const double *Xj = X + 3 * j;
    for (int s = pt_inst_ptr[j]; s < pt_inst_ptr[j + 1] && ok; s++) {
      int q = pt_inst[s];
      for (int k = inst_obs_ptr[q]; k < inst_obs_ptr[q + 1]; k++) {
        int i = obs_cam[k];
        double Rl[9], Xc[3], RX[3];
        for (int e = 0; e < 9; e++) Rl[e] = R[9 * i + e];
        for (int r = 0; r < 3; r++) {
          RX[r] = Rl[3 * r] * Xj[0] + Rl[3 * r + 1] * Xj[1] + Rl[3 * r + 2] * Xj[2];
          Xc[r] = RX[r] + t[3 * i + r];
        }
        if (!(Xc[2] > 0.0)) { ok = false; break; }
        double Jx[6];
        if (k1) {  // per-camera intrinsics: the radial term
          ProjJac<double, 8> pj;
          project_jac<double, 8>(Rl, Xc, RX, intr[3 * i], k1[i], intr[3 * i + 1], intr[3 * i + 2], pj);
          for (int e = 0; e < 6; e++) Jx[e] = pj.Jx[e];
        } else {
          ProjJac<double, 6> pj;
          project_jac<double, 6>(Rl, Xc, RX, intr[3 * i], 0.0, intr[3 * i + 1], intr[3 * i + 2], pj);
          for (int e = 0; e < 6; e++) Jx[e] = pj.Jx[e];
        }
        double W0 = 1, W1 = 0, W2 = 1;
        if (has_winv) { W0 = obs_winv[3 * k]; W1 = obs_winv[3 * k + 1]; W2 = obs_winv[3 * k + 2]; }
        double w = obs_w[k];
        for (int r = 0; r < 3; r++)
          for (int c = r; c < 3; c++) {
            double a0 = W0 * Jx[c] + W1 * Jx[3 + c], a1 = W1 * Jx[c] + W2 * Jx[3 + c];
            Nm[s3idx(r, c)] += w * (Jx[r] * a0 + Jx[3 + r] * a1);
          }
      }
    }
  }
  double inv[6];
  if (ok) ok = sym3_inv<double>(Nm, inv) > 0.0;
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) out[9 * a + 3 * r + c] = ok ? inv[s3idx(r, c)] : NAN;
}

}  // namespace rpba

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static void free_graph(GraphRec *g);
static bool tune_load(Ctx *ctx, const char *path);
static rpba_status dev_alloc(Ctx *ctx, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *q = nullptr;
  if (ctx->opt.dev_alloc) {
    q = ctx->opt.dev_alloc(bytes, ctx->opt.alloc_user);
    if (!q) {
      ctx->err = "device allocator hook returned NULL";
      return RPBA_ERR_OOM;
    }
  } else {
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? RPBA_ERR_OOM : RPBA_ERR_CUDA;
    }
  }
  ctx->allocs.push_back(q);
  *p = q;
  return RPBA_OK;
}

rpba_status rpba::ctx_alloc(Ctx *ctx, void **p, size_t bytes) { return dev_alloc(ctx, p, bytes); }

template <typename T>
static rpba_status alloc_n(Ctx *ctx, T **p, size_t n) {
  return dev_alloc(ctx, (void **)p, n * sizeof(T));
}

template <typename T>
static rpba_status upload(Ctx *ctx, T **p, const T *host, size_t n) {
  RPBA_TRY(alloc_n(ctx, p, n));
  if (n) RPBA_CUDA(cudaMemcpyAsync(*p, host, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return RPBA_OK;
}

static rpba_status sync(Ctx *ctx) {
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  return RPBA_OK;
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

extern "C" void rpba_default_options(rpba_options *o) {
  memset(o, 0, sizeof(*o));
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
  o->weight_mode = 0;
  o->rho0 = 200.0;
  o->isect_max_iter = 10;
  o->isect_tol = 1e-10;
  o->isect_px_tol = 1e-3;
  o->cond_max = 1e12;
  o->precision = 0;
  o->solver = 0;
  o->pcg_tol = 1e-8;
  o->pcg_max_iter = 500;
  o->ir_steps = 2;
  o->chol_tc = 0;
}

extern "C" const char *rpba_last_error(const rpba_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

extern "C" void rpba_destroy(rpba_ctx *h) {
  if (!h) return;
  Ctx *ctx = &h->c;
  cudaStreamSynchronize(ctx->stream);
  for (void *p : ctx->allocs) {
    if (ctx->opt.dev_free) ctx->opt.dev_free(p, ctx->opt.alloc_user);
    else cudaFree(p);
  }
  if (ctx->h_pinned_counter) cudaFreeHost(ctx->h_pinned_counter);
  if (ctx->h_pinned_d) cudaFreeHost(ctx->h_pinned_d);
  free_graph(ctx->lm_graph);
  free_graph(ctx->lm_graph_pre);
  free_graph(ctx->lm_graph_post);
  for (auto &r : ctx->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  for (cudaStream_t bs : ctx->pcg_body_stream)
    if (bs) cudaStreamDestroy(bs);
  delete h;
}

// ---------------------------------------------------------------------------
// creation: validation and topology
// ---------------------------------------------------------------------------
static rpba_status build(Ctx *ctx, const rpba_problem *pb) {
  const int M = pb->n_cams, N = pb->n_points, K = pb->n_obs;
  ctx->M = M; ctx->N = N; ctx->K = K;
  if (M < 0 || N < 0 || K < 0 || (M && (!pb->cam_pose || !pb->cam_intr || !pb->cam_subblock)) ||
      (N && !pb->points) || (K && (!pb->obs_cam || !pb->obs_point || !pb->obs_xy))) {
    ctx->err = "invalid sizes or NULL input arrays";
    return RPBA_ERR_INVALID_ARG;
  }
  int L = 0;
  for (int i = 0; i < M; i++) {
    int s = pb->cam_subblock[i];
    if (s < 0 || s >= (1 << 20)) { ctx->err = "cam_subblock out of range"; return RPBA_ERR_INVALID_ARG; }
    L = std::max(L, s + 1);
  }
  ctx->L = L;
  // solver 4 (auto): lock-step PCG runs as many iterations as its slowest
  // sub-block needs, a maximum that grows with the number of sub-blocks; the
  // direct solve's critical path is set by the largest sub-block alone
  ctx->cd = ctx->opt.intrinsics ? 8 : 6;
  if (ctx->opt.solver == 4) {
    ctx->auto_solver = true;
    ctx->opt.solver = L <= RPBA_AUTO_PCG_MAX_SUBBLOCKS ? 1 : 2;
  }
  for (int k = 0; k < K; k++) {
    if (pb->obs_cam[k] < 0 || pb->obs_cam[k] >= M || pb->obs_point[k] < 0 || pb->obs_point[k] >= N) {
      ctx->err = "observation index out of range";
      return RPBA_ERR_INVALID_ARG;
    }
  }
  for (long long e = 0; e < 6LL * M; e++)
    if (!isfinite(pb->cam_pose[e])) { ctx->err = "non-finite camera pose"; return RPBA_ERR_NUMERIC; }
  for (long long e = 0; e < 3LL * N; e++)
    if (!isfinite(pb->points[e])) { ctx->err = "non-finite point"; return RPBA_ERR_NUMERIC; }
  for (long long e = 0; e < 2LL * K; e++)
    if (!isfinite(pb->obs_xy[e])) { ctx->err = "non-finite observation"; return RPBA_ERR_NUMERIC; }
  ctx->has_winv = pb->obs_winv != nullptr;
  if (ctx->has_winv)
    for (int k = 0; k < K; k++) {
      const double *W = pb->obs_winv + 3 * k;
      if (!(W[0] > 0.0) || !(W[0] * W[2] - W[1] * W[1] > 0.0)) {
        ctx->err = "obs_winv not positive definite";
        return RPBA_ERR_INVALID_ARG;
      }
    }
  // Internal point numbering: points sorted by (sub-block of their first
  // camera, first camera, id). The observations and point instances follow
  // the point order inside each sub-block, so neighbouring threads then see
  // the same cameras and nearby points; with the caller's numbering (often
  // unrelated to geometry) every observation gathers its camera record and
  // point words from a random line. Every entry point translates: points and
  // covariance ids use the caller's numbering, instances the canonical order
  // (sub-block, caller's point id).
  std::vector<int> &pperm = ctx->h_pt_perm, &pinv = ctx->h_pt_inv;
  std::vector<double> Xperm(3 * (size_t)N);
  std::vector<int32_t> operm(K);
  rpba_problem pbi = *pb;
  {
    std::vector<int> first(N, M);
    for (int k = 0; k < K; k++) first[pb->obs_point[k]] = std::min(first[pb->obs_point[k]], pb->obs_cam[k]);
    std::vector<long long> key(N);
    for (int j = 0; j < N; j++) {
      long long sub = first[j] < M ? pb->cam_subblock[first[j]] : (1 << 20);
      key[j] = (sub << 32) | (long long)first[j];
    }
    pinv.resize(N);
    std::iota(pinv.begin(), pinv.end(), 0);
    std::stable_sort(pinv.begin(), pinv.end(), [&](int a, int b) { return key[a] < key[b]; });
    pperm.resize(N);
    for (int n = 0; n < N; n++) pperm[pinv[n]] = n;
    for (int n = 0; n < N; n++)
      for (int e = 0; e < 3; e++) Xperm[3 * (size_t)n + e] = pb->points[3 * (size_t)pinv[n] + e];
    for (int k = 0; k < K; k++) operm[k] = pperm[pb->obs_point[k]];
    pbi.points = Xperm.data();
    pbi.obs_point = operm.data();
    pb = &pbi;
  }
  // cameras by (sub-block, id)
  std::vector<int> &scp = ctx->h_sub_cam_ptr, &sc = ctx->h_sub_cam;
  scp.assign(L + 1, 0);
  for (int i = 0; i < M; i++) scp[pb->cam_subblock[i] + 1]++;
  for (int l = 0; l < L; l++) scp[l + 1] += scp[l];
  sc.resize(M);
  std::vector<int> cam_local(M), fill(scp.begin(), scp.end() - 1);
  for (int i = 0; i < M; i++) {
    int p = fill[pb->cam_subblock[i]]++;
    sc[p] = i;
    cam_local[i] = p - scp[pb->cam_subblock[i]];
  }
  // observations sorted by (sub-block, point), stable: two counting sorts
  std::vector<int> by_pt(K), order(K);
  {
    std::vector<int> cnt(N + 1, 0);
    for (int k = 0; k < K; k++) cnt[pb->obs_point[k] + 1]++;
    for (int j = 0; j < N; j++) cnt[j + 1] += cnt[j];
    for (int k = 0; k < K; k++) by_pt[cnt[pb->obs_point[k]]++] = k;
  }
  // duplicate (camera, point) check on the point-sorted list
  {
    std::vector<int> seen(M, -1);
    for (int p = 0; p < K; p++) {
      int k = by_pt[p];
      int i = pb->obs_cam[k], j = pb->obs_point[k];
      if (seen[i] == j) { ctx->err = "duplicate (camera, point) observation"; return RPBA_ERR_INVALID_ARG; }
      seen[i] = j;
    }
  }
  {
    std::vector<int> cnt(L + 1, 0);
    for (int k = 0; k < K; k++) cnt[pb->cam_subblock[pb->obs_cam[k]] + 1]++;
    for (int l = 0; l < L; l++) cnt[l + 1] += cnt[l];
    for (int p = 0; p < K; p++) {
      int k = by_pt[p];
      order[cnt[pb->cam_subblock[pb->obs_cam[k]]]++] = k;
    }
  }
  // instances
  std::vector<int> obs_inst(K), inst_obs_ptr(1, 0), inst_pt, inst_sub;
  for (int p = 0; p < K; p++) {
    int k = order[p];
    int l = pb->cam_subblock[pb->obs_cam[k]], j = pb->obs_point[k];
    if (inst_pt.empty() || inst_pt.back() != j || inst_sub.back() != l) {
      if (!inst_pt.empty()) inst_obs_ptr.push_back(p);
      inst_pt.push_back(j);
      inst_sub.push_back(l);
    }
    obs_inst[p] = (int)inst_pt.size() - 1;
  }
  int P = (int)inst_pt.size();
  inst_obs_ptr.push_back(K);
  if (P == 0) inst_obs_ptr.assign(1, 0);
  ctx->P = P;
  ctx->h_inst_pt = inst_pt;
  ctx->h_inst_sub = inst_sub;
  {  // canonical instance order: (sub-block, caller's point id)
    std::vector<int> &canon = ctx->h_inst_canon;
    canon.resize(P);
    std::iota(canon.begin(), canon.end(), 0);
    std::sort(canon.begin(), canon.end(), [&](int a, int b) {
      if (inst_sub[a] != inst_sub[b]) return inst_sub[a] < inst_sub[b];
      return pinv[inst_pt[a]] < pinv[inst_pt[b]];
    });
  }
  ctx->h_obs_user = order;
  std::vector<int> sip(L + 1, 0);
  for (int q = 0; q < P; q++) sip[inst_sub[q] + 1]++;
  for (int l = 0; l < L; l++) sip[l + 1] += sip[l];
  ctx->h_sub_inst_ptr = sip;
  // point -> instances
  std::vector<int> pip(N + 1, 0), pin(P);
  for (int q = 0; q < P; q++) pip[inst_pt[q] + 1]++;
  for (int j = 0; j < N; j++) pip[j + 1] += pip[j];
  {
    std::vector<int> f(pip.begin(), pip.end() - 1);
    for (int q = 0; q < P; q++) pin[f[inst_pt[q]]++] = q;
  }
  // camera -> observation positions
  std::vector<int> cop(M + 1, 0), cob(K);
  for (int p = 0; p < K; p++) cop[pb->obs_cam[order[p]] + 1]++;
  for (int i = 0; i < M; i++) cop[i + 1] += cop[i];
  {
    std::vector<int> f(cop.begin(), cop.end() - 1);
    for (int p = 0; p < K; p++) cob[f[pb->obs_cam[order[p]]]++] = p;
  }
  int mco = 0;
  for (int i = 0; i < M; i++) mco = std::max(mco, cop[i + 1] - cop[i]);
  ctx->max_cam_obs = mco;
  // Schur pairs inside each instance: local(cam a) > local(cam b)
  std::vector<int> pa, pb_;
  for (int q = 0; q < P; q++)
    for (int a = inst_obs_ptr[q]; a < inst_obs_ptr[q + 1]; a++)
      for (int b = inst_obs_ptr[q]; b < inst_obs_ptr[q + 1]; b++) {
        int la = cam_local[pb->obs_cam[order[a]]], lb = cam_local[pb->obs_cam[order[b]]];
        if (la > lb) { pa.push_back(a); pb_.push_back(b); }
      }
  ctx->n_pairs = (long long)pa.size();
  // FP32 form: the pairs grouped by camera of a, then by camera of b (a
  // segment per camera pair (i, i')), then by position: camera i owns the
  // off-diagonal blocks S_{i,i'} with local(i) > local(i'), each the sum over
  // one segment
  std::vector<int> spa, spb, spq, sps, seg_cam, seg_nb, sitem;
  if (ctx->opt.precision == 1) {
    long long np = ctx->n_pairs;
    if (np >= INT_MAX) {  // pair positions and items are 32-bit
      ctx->err = "more than 2^31 - 1 Schur pairs";
      return RPBA_ERR_INVALID_ARG;
    }
    std::vector<long long> by_b(np), cnt(M + 1, 0);
    auto cam_of = [&](int pos) { return pb->obs_cam[order[pos]]; };
    for (long long e = 0; e < np; e++) cnt[cam_of(pb_[e]) + 1]++;
    for (int i = 0; i < M; i++) cnt[i + 1] += cnt[i];
    for (long long e = 0; e < np; e++) by_b[cnt[cam_of(pb_[e])]++] = e;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (long long e = 0; e < np; e++) cnt[cam_of(pa[e]) + 1]++;
    for (int i = 0; i < M; i++) cnt[i + 1] += cnt[i];
    std::vector<long long> srt(np);
    for (long long t = 0; t < np; t++) {
      long long e = by_b[t];
      srt[cnt[cam_of(pa[e])]++] = e;
    }
    spa.resize(np);
    spb.resize(np);
    spq.resize(np);
    sps.resize(np);
    int last_a = -1, last_b = -1;
    for (long long t = 0; t < np; t++) {
      long long e = srt[t];
      spa[t] = pa[e];
      spb[t] = pb_[e];
      spq[t] = obs_inst[pa[e]];
      int ia = cam_of(pa[e]), ib = cam_of(pb_[e]);
      if (ia != last_a || ib != last_b) {
        seg_cam.push_back(ia);
        seg_nb.push_back(ib);
        last_a = ia;
        last_b = ib;
      }
      sps[t] = (int)seg_cam.size() - 1;
    }
    ctx->n_segs = (long long)seg_nb.size();
    for (long long t = 0; t < np;) {  // items: up to SC_ITEM pairs of one segment
      sitem.push_back((int)t);
      long long e = t + 1;
      while (e < np && e - t < SC_ITEM && sps[e] == sps[t]) e++;
      t = e;
    }
    ctx->n_items = (long long)sitem.size();
    sitem.push_back((int)np);
    pa.clear(); pa.shrink_to_fit();
    pb_.clear(); pb_.shrink_to_fit();
  }
  if (ctx->opt.solver == 3) {
    std::vector<int> oc(K);
    for (int p = 0; p < K; p++) oc[p] = pb->obs_cam[order[p]];
    build_camera_graph(ctx, inst_obs_ptr, oc, inst_sub, cam_local);
  }
  // RCS layout
  std::vector<long long> soff(L);
  std::vector<int> npad(L), yoff(L), ntiles(L);
  long long stot = 0;
  int yt = 0, maxT = 0;
  for (int l = 0; l < L; l++) {
    int n = ctx->cd * (scp[l + 1] - scp[l]);
    int T = (n + RPBA_TILE - 1) / RPBA_TILE;
    npad[l] = T * RPBA_TILE;
    ntiles[l] = T;
    maxT = std::max(maxT, T);
    soff[l] = stot;
    stot += (long long)npad[l] * npad[l];
    yoff[l] = yt;
    yt += npad[l];
  }
  ctx->h_S_off = soff;
  ctx->h_npad = npad;
  ctx->S_total = stot;
  ctx->max_tiles = maxT;
  ctx->ytot = yt;
  // factorisation schedule: for step k the tiles of every sub-block, as
  // prefix sums (panel: T_l - k - 1 tiles; trailing update: its triangle)
  {
    int steps = std::max(maxT - 1, 1);
    ctx->h_sched.assign((size_t)steps * 2 * (L + 1), 0);
    for (int k = 0; k < steps; k++) {
      int *pb = &ctx->h_sched[(size_t)k * 2 * (L + 1)];
      int *ub = pb + (L + 1);
      for (int l = 0; l < L; l++) {
        int rem = std::max(ntiles[l] - k - 1, 0);
        pb[l + 1] = pb[l] + rem;
        ub[l + 1] = ub[l] + rem * (rem + 1) / 2;
      }
    }
  }
  std::vector<int> loff(L);
  int ltot = 0;
  for (int l = 0; l < L; l++) {
    loff[l] = ltot;
    ltot += ntiles[l] * RPBA_TILE * RPBA_TILE;
  }
  // per-observation arrays in GPU order
  std::vector<int> ocam(K), opt(K);
  std::vector<double> oxy(2 * (size_t)K), ow(3 * (size_t)(ctx->has_winv ? K : 0));
  for (int p = 0; p < K; p++) {
    int k = order[p];
    ocam[p] = pb->obs_cam[k];
    opt[p] = pb->obs_point[k];
    oxy[2 * p] = pb->obs_xy[2 * k];
    oxy[2 * p + 1] = pb->obs_xy[2 * k + 1];
    if (ctx->has_winv)
      for (int e = 0; e < 3; e++) ow[3 * (size_t)p + e] = pb->obs_winv[3 * (size_t)k + e];
  }
  std::vector<uint8_t> active(N);
  int nact = 0;
  {
    std::vector<int> cnt(N, 0);
    for (int k = 0; k < K; k++) cnt[pb->obs_point[k]]++;
    for (int j = 0; j < N; j++) { active[j] = cnt[j] >= 2; nact += active[j]; }
    ctx->h_pt_nobs = cnt;
  }
  ctx->h_pinned_d = nullptr;
  // device uploads
  double *pose_d = nullptr;
  RPBA_TRY(upload(ctx, &pose_d, pb->cam_pose, 6 * (size_t)M));
  RPBA_TRY(alloc_n(ctx, &ctx->R, 9 * (size_t)M));
  RPBA_TRY(alloc_n(ctx, &ctx->t, 3 * (size_t)M));
  RPBA_TRY(alloc_n(ctx, &ctx->Rt, 9 * (size_t)M));
  RPBA_TRY(alloc_n(ctx, &ctx->tt, 3 * (size_t)M));
  RPBA_TRY(upload(ctx, &ctx->intr, pb->cam_intr, 3 * (size_t)M));
  if (ctx->cd == 8) {  // per-camera intrinsics: k1 and the trial f, k1
    std::vector<double> k1(std::max(M, 1), 0.0);
    if (pb->cam_k1)
      for (int i = 0; i < M; i++) k1[i] = pb->cam_k1[i];
    RPBA_TRY(upload(ctx, &ctx->k1, k1.data(), k1.size()));
    RPBA_TRY(alloc_n(ctx, &ctx->ft, (size_t)std::max(M, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->k1t, (size_t)std::max(M, 1)));
  }
  RPBA_TRY(upload(ctx, &ctx->cam_sub, pb->cam_subblock, (size_t)M));
  RPBA_TRY(upload(ctx, &ctx->cam_local, cam_local.data(), (size_t)M));
  RPBA_TRY(upload(ctx, &ctx->sub_cam_ptr, scp.data(), (size_t)L + 1));
  RPBA_TRY(upload(ctx, &ctx->sub_cam, sc.data(), (size_t)M));
  RPBA_TRY(upload(ctx, &ctx->cam_obs_ptr, cop.data(), (size_t)M + 1));
  RPBA_TRY(upload(ctx, &ctx->cam_obs, cob.data(), (size_t)K));
  RPBA_TRY(alloc_n(ctx, &ctx->cam_sigma, (size_t)M));
  RPBA_TRY(upload(ctx, &ctx->X, pb->points, 3 * (size_t)N));
  RPBA_TRY(upload(ctx, &ctx->active, active.data(), (size_t)N));
  RPBA_TRY(upload(ctx, &ctx->pt_inst_ptr, pip.data(), (size_t)N + 1));
  {  // the tie points (points in two or more sub-blocks), for the TP intersection's launch
    std::vector<int> tps;
    for (int j = 0; j < N; j++)
      if (pip[j + 1] - pip[j] >= 2) tps.push_back(j);
    ctx->n_tp = (int)tps.size();
    if (tps.empty()) tps.push_back(0);  // a one-element buffer; the launch covers n_tp = 0 items
    RPBA_TRY(upload(ctx, &ctx->tp_list, tps.data(), tps.size()));
  }
  // index maps of the boundary translation and their scratch (one per-point
  // or per-instance array at a time)
  RPBA_TRY(upload(ctx, &ctx->d_pt_inv, ctx->h_pt_inv.data(), (size_t)N));
  RPBA_TRY(upload(ctx, &ctx->d_inst_canon, ctx->h_inst_canon.data(), (size_t)P));
  ctx->perm_scratch_n = std::max<size_t>(std::max(3 * (size_t)N, 6 * (size_t)P), 1);
  RPBA_TRY(alloc_n(ctx, &ctx->perm_scratch, ctx->perm_scratch_n));
  RPBA_TRY(upload(ctx, &ctx->pt_inst, pin.data(), (size_t)P));
  RPBA_TRY(upload(ctx, &ctx->inst_pt, inst_pt.data(), (size_t)P));
  RPBA_TRY(upload(ctx, &ctx->inst_sub, inst_sub.data(), (size_t)P));
  RPBA_TRY(upload(ctx, &ctx->inst_obs_ptr, inst_obs_ptr.data(), (size_t)P + 1));
  RPBA_TRY(upload(ctx, &ctx->sub_inst_ptr, sip.data(), (size_t)L + 1));
  {
    std::vector<int> sop(L + 1);
    for (int l = 0; l <= L; l++) sop[l] = inst_obs_ptr[sip[l]];
    RPBA_TRY(upload(ctx, &ctx->sub_obs_ptr, sop.data(), (size_t)L + 1));
    // chunks of at most 256 observations that never straddle two sub-blocks
    // (the sub-block cost: one CTA per chunk, one thread per observation)
    std::vector<int> cs, cst, cp(L + 1, 0);
    for (int l = 0; l < L; l++) {
      for (int k = sop[l]; k < sop[l + 1]; k += 256) { cs.push_back(l); cst.push_back(k); }
      cp[l + 1] = (int)cs.size();
    }
    ctx->n_chunks = (int)cs.size();
    RPBA_TRY(upload(ctx, &ctx->chunk_sub, cs.data(), cs.size()));
    RPBA_TRY(upload(ctx, &ctx->chunk_start, cst.data(), cst.size()));
    RPBA_TRY(upload(ctx, &ctx->sub_chunk_ptr, cp.data(), cp.size()));
    RPBA_TRY(alloc_n(ctx, &ctx->chunk_part, (size_t)std::max(ctx->n_chunks, 1)));
    if (ctx->opt.precision == 1) {
      // camera records of the largest sub-block staged per CTA (144 B each)
      int max_cams = 0;
      for (int l = 0; l < L; l++) max_cams = std::max(max_cams, scp[l + 1] - scp[l]);
      size_t smem = (size_t)max_cams * RPBA_CAM_STAGE_BYTES;
      if (smem <= RPBA_COST_STAGE_MAX_SMEM) {
        std::vector<int> gc;
        for (int l = 0; l < L; l++)
          for (int c = cp[l]; c < cp[l + 1]; c += RPBA_COST_GROUP) gc.push_back(c);
        ctx->n_groups = (int)gc.size();
        ctx->cost_smem = std::max<size_t>(smem, 16);
        RPBA_TRY(upload(ctx, &ctx->group_chunk, gc.data(), gc.size()));
        RPBA_TRY(cost_groups_setup(ctx));
      }
      RPBA_TRY(alloc_n(ctx, &ctx->f0_cache, (size_t)std::max(L, 1)));
      RPBA_TRY(alloc_n(ctx, &ctx->sigma0_part, 5 * ((size_t)ctx->n_chunks + L + 1)));
    }
  }
  if (ctx->opt.precision != 1)  // the FP32 form sums its cost terms per chunk
    RPBA_TRY(alloc_n(ctx, &ctx->obs_cost, (size_t)K));
  if (ctx->opt.precision == 1) {
    // FP32 form: inputs rounded once (observations relative to the principal point)
    std::vector<float> xy32(2 * (size_t)K), w32((size_t)K, 1.0f), wi32(ctx->has_winv ? 3 * (size_t)K : 0);
    for (int p = 0; p < K; p++) {
      int i = ocam[p];
      xy32[2 * (size_t)p] = (float)(oxy[2 * (size_t)p] - pb->cam_intr[3 * (size_t)i + 1]);
      xy32[2 * (size_t)p + 1] = (float)(oxy[2 * (size_t)p + 1] - pb->cam_intr[3 * (size_t)i + 2]);
      if (ctx->has_winv)
        for (int e = 0; e < 3; e++) wi32[3 * (size_t)p + e] = (float)ow[3 * (size_t)p + e];
    }
    std::vector<float> xylo(2 * (size_t)K);
    for (size_t e = 0; e < xy32.size(); e++) {
      int i = ocam[e / 2];
      double rel = oxy[e] - pb->cam_intr[3 * (size_t)i + 1 + (e & 1)];
      xylo[e] = (float)(rel - (double)xy32[e]);
    }
    RPBA_TRY(upload(ctx, &ctx->obs_xy32, xy32.data(), xy32.size()));
    RPBA_TRY(upload(ctx, &ctx->obs_xylo, xylo.data(), xylo.size()));
    RPBA_TRY(upload(ctx, &ctx->obs_w32, w32.data(), w32.size()));
    if (ctx->has_winv) RPBA_TRY(upload(ctx, &ctx->obs_winv32, wi32.data(), wi32.size()));
    RPBA_TRY(alloc_n(ctx, &ctx->Xl_hi, 3 * (size_t)P));
    RPBA_TRY(alloc_n(ctx, &ctx->Xl_lo, 3 * (size_t)P));
    RPBA_TRY(alloc_n(ctx, &ctx->X_hi, 3 * (size_t)N));
    RPBA_TRY(alloc_n(ctx, &ctx->X_lo, 3 * (size_t)N));
    RPBA_TRY(alloc_n(ctx, &ctx->dC32, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->camff, FF_CAM * (size_t)M));
    RPBA_TRY(alloc_n(ctx, &ctx->camff_t, FF_CAM * (size_t)M));
    RPBA_TRY(alloc_n(ctx, &ctx->Xlt_hi, 3 * (size_t)P));
    RPBA_TRY(alloc_n(ctx, &ctx->Xlt_lo, 3 * (size_t)P));
    RPBA_TRY(alloc_n(ctx, &ctx->Wl32, 6 * (size_t)P));
    RPBA_TRY(alloc_n(ctx, &ctx->cam_sigma32, (size_t)M));
    if (P) RPBA_CUDA(cudaMemsetAsync(ctx->Wl32, 0, 6 * (size_t)P * sizeof(float), ctx->stream));
  }
  RPBA_TRY(alloc_n(ctx, &ctx->seg_part, (size_t)L * 32));
  RPBA_TRY(alloc_n(ctx, &ctx->Xl, 3 * (size_t)P));
  RPBA_TRY(alloc_n(ctx, &ctx->Xlt, 3 * (size_t)P));
  RPBA_TRY(alloc_n(ctx, &ctx->Wl, 6 * (size_t)P));
  RPBA_TRY(alloc_n(ctx, &ctx->inst_cost, (size_t)P));
  size_t rs = ctx->opt.precision == 1 ? sizeof(float) : sizeof(double);
  RPBA_TRY(dev_alloc(ctx, &ctx->Ninv, 6 * (size_t)P * rs));
  RPBA_TRY(dev_alloc(ctx, &ctx->gX, 3 * (size_t)P * rs));
  RPBA_TRY(alloc_n(ctx, &ctx->isect_N, 10 * (size_t)P));
  RPBA_TRY(alloc_n(ctx, &ctx->isect_state, (size_t)N));
  RPBA_TRY(alloc_n(ctx, &ctx->isect_iter, (size_t)N));
  RPBA_TRY(upload(ctx, &ctx->obs_cam, ocam.data(), (size_t)K));
  if (ctx->n_groups) {  // the staged cost kernels index the sub-block's records by local camera
    std::vector<uint16_t> ocl(K);
    for (int k = 0; k < K; k++) ocl[k] = (uint16_t)cam_local[ocam[k]];
    RPBA_TRY(upload(ctx, &ctx->obs_camloc, ocl.data(), (size_t)K));
  }
  RPBA_TRY(upload(ctx, &ctx->obs_inst, obs_inst.data(), (size_t)K));
  RPBA_TRY(upload(ctx, &ctx->obs_user, order.data(), (size_t)K));
  RPBA_TRY(upload(ctx, &ctx->obs_pt, opt.data(), (size_t)K));
  RPBA_TRY(upload(ctx, &ctx->obs_xy, oxy.data(), 2 * (size_t)K));
  if (ctx->has_winv) {
    RPBA_TRY(upload(ctx, &ctx->obs_winv, ow.data(), 3 * (size_t)K));
    std::vector<double> wf(3 * (size_t)K);
    for (int p = 0; p < K; p++) {
      const double *W = &ow[3 * (size_t)p];
      double a = sqrt(W[0]);
      wf[3 * (size_t)p] = a;
      wf[3 * (size_t)p + 1] = W[1] / a;
      wf[3 * (size_t)p + 2] = sqrt(W[2] - W[1] * W[1] / W[0]);
    }
    RPBA_TRY(upload(ctx, &ctx->obs_whiten, wf.data(), wf.size()));
    if (ctx->opt.precision == 1) {
      std::vector<float> wf32(wf.begin(), wf.end());
      RPBA_TRY(upload(ctx, &ctx->obs_whiten32, wf32.data(), wf32.size()));
    }
  }
  RPBA_TRY(alloc_n(ctx, &ctx->obs_w, (size_t)K));
  if (ctx->opt.precision != 1) {  // the FP32 form keeps the Jacobian blocks in registers
    RPBA_TRY(dev_alloc(ctx, &ctx->NXC, 3 * (size_t)ctx->cd * K * rs));
    RPBA_TRY(dev_alloc(ctx, &ctx->Z, 3 * (size_t)ctx->cd * K * rs));
  }
  if (ctx->opt.precision == 1) {
    RPBA_TRY(upload(ctx, &ctx->spair_a, spa.data(), spa.size()));
    RPBA_TRY(upload(ctx, &ctx->spair_b, spb.data(), spb.size()));
    RPBA_TRY(upload(ctx, &ctx->spair_q, spq.data(), spq.size()));
    RPBA_TRY(upload(ctx, &ctx->spair_seg, sps.data(), sps.size()));
    RPBA_TRY(upload(ctx, &ctx->seg_cam, seg_cam.data(), seg_cam.size()));
    RPBA_TRY(upload(ctx, &ctx->seg_nb, seg_nb.data(), seg_nb.size()));
    RPBA_TRY(upload(ctx, &ctx->sitem, sitem.data(), sitem.size()));
  } else {
    RPBA_TRY(upload(ctx, &ctx->pair_a, pa.data(), pa.size()));
    RPBA_TRY(upload(ctx, &ctx->pair_b, pb_.data(), pb_.size()));
  }
  RPBA_TRY(alloc_n(ctx, &ctx->S, (size_t)std::max(stot, 1LL)));
  RPBA_TRY(alloc_n(ctx, &ctx->y, (size_t)std::max(yt, 1)));
  RPBA_TRY(alloc_n(ctx, &ctx->dC, (size_t)std::max(yt, 1)));
  RPBA_TRY(upload(ctx, &ctx->S_off, soff.data(), (size_t)L));
  RPBA_TRY(upload(ctx, &ctx->npad, npad.data(), (size_t)L));
  RPBA_TRY(upload(ctx, &ctx->ycam_off, yoff.data(), (size_t)L));
  RPBA_TRY(upload(ctx, &ctx->sub_ntiles, ntiles.data(), (size_t)L));
  RPBA_TRY(upload(ctx, &ctx->linv_off, loff.data(), (size_t)L));
  RPBA_TRY(upload(ctx, &ctx->sched, ctx->h_sched.data(), ctx->h_sched.size()));
  RPBA_TRY(alloc_n(ctx, &ctx->Linv64, (size_t)std::max(ltot, 1)));
  if (ctx->opt.solver == 1 || ctx->opt.solver == 3 || ctx->auto_solver) {
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_Minv, (size_t)ctx->cd * ctx->cd * std::max(M, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_x, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_r, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_z, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_p, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_q, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_st, 4 * (size_t)std::max(L, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_pq, (size_t)std::max(L, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->pcg_live, (size_t)std::max(L, 1)));
    int max_n = 0;
    for (int l = 0; l < L; l++) max_n = std::max(max_n, ctx->cd * (scp[l + 1] - scp[l]));
    // solver 1 or auto's PCG in the FP32 form: float-float, for sub-blocks of
    // up to RPBA_PCG_FF_MAX_N unknowns (the step kernel's register batches)
    if (ctx->opt.precision == 1 && ctx->opt.solver == 1 && max_n <= RPBA_PCG_FF_MAX_N) {
      ctx->pcg_ff_smem = (size_t)std::max(max_n, 1) * 2 * sizeof(float);
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_Shi, (size_t)std::max(stot, 1LL)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_Slo, (size_t)std::max(stot, 1LL)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_fx, (size_t)std::max(yt, 1)));
      for (float **v : {&ctx->pcg_x32, &ctx->pcg_r32, &ctx->pcg_z32, &ctx->pcg_p32})
        RPBA_TRY(alloc_n(ctx, v, (size_t)std::max(yt, 1)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_qi, (size_t)std::max(yt, 1)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_s32, (size_t)PCG_S32_WORDS * std::max(L, 1)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_act, (size_t)std::max(L, 1)));
      RPBA_TRY(alloc_n(ctx, &ctx->pcg_Minv32, (size_t)ctx->cd * ctx->cd * std::max(M, 1)));
      // streams on which the device-driven loop's bodies are captured (none:
      // the host-driven loop)
      for (cudaStream_t &bs : ctx->pcg_body_stream)
        if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          bs = nullptr;
        }
    }
    std::vector<int> pt(L + 1, 0);
    for (int l = 0; l < L; l++) pt[l + 1] = pt[l] + ntiles[l] * (ntiles[l] + 1) / 2;
    ctx->pcg_tiles_total = pt[L];
    RPBA_TRY(upload(ctx, &ctx->pcg_tiles, pt.data(), (size_t)L + 1));
    if (ctx->pcg_Shi) {  // the FP32 CG product's tile table: (sub-block, a << 16 | b) per lower tile
      std::vector<int2> tm((size_t)std::max(pt[L], 1));
      for (int l = 0; l < L; l++)
        for (int a = 0, t = pt[l]; a < ntiles[l]; a++)
          for (int b = 0; b <= a; b++, t++) tm[t] = make_int2(l, (a << 16) | b);
      RPBA_TRY(upload(ctx, &ctx->pcg_tile_map, tm.data(), tm.size()));
    }
  }
  if (ctx->opt.solver == 2 || ctx->auto_solver) {
    RPBA_TRY(alloc_n(ctx, &ctx->S32, (size_t)std::max(stot, 1LL)));
    RPBA_TRY(upload(ctx, &ctx->S32_off, soff.data(), (size_t)L));
    RPBA_TRY(alloc_n(ctx, &ctx->Linv32, (size_t)std::max(ltot, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->ir_r32, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->ir_d, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->ir_rs, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->ir_x, (size_t)std::max(yt, 1)));
    RPBA_TRY(alloc_n(ctx, &ctx->ir_t, (size_t)std::max(yt, 1)));
    RPBA_TRY(tc_chol_setup(ctx));  // the tensor-core forms, for chol_tc and the autotuner
  }
  RPBA_TRY(camera_major_setup(ctx));
  RPBA_TRY(alloc_n(ctx, &ctx->wrho, 1));
  RPBA_CUDA(cudaMemcpyAsync(ctx->wrho, &ctx->opt.rho0, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_TRY(alloc_n(ctx, &ctx->sub_mask, (size_t)std::max(L, 1)));
  RPBA_CUDA(cudaMemsetAsync(ctx->sub_mask, 1, (size_t)std::max(L, 1), ctx->stream));
  RPBA_TRY(alloc_n(ctx, &ctx->pt_mask, (size_t)std::max(N, 1)));
  RPBA_CUDA(cudaMemsetAsync(ctx->pt_mask, 1, (size_t)std::max(N, 1), ctx->stream));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_lambda, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_F, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_Ft, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_best, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_grace, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_rej, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_it, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_run, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_acc, (size_t)L));
  RPBA_TRY(alloc_n(ctx, &ctx->lm_cholfail, (size_t)L));
  {  // grid-stride reductions (sigma_0): ~8 observations per thread, at most
     // 8 CTAs of 256 threads per SM
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 152;
    ctx->red_blocks = (int)std::max(1LL, std::min<long long>(8LL * sms, ((long long)K + 2047) / 2048));
  }
  RPBA_TRY(alloc_n(ctx, &ctx->red, (size_t)ctx->red_blocks * 6 + 16));
  RPBA_TRY(alloc_n(ctx, &ctx->counters, 16));
  RPBA_CUDA(cudaMallocHost((void **)&ctx->h_pinned_counter, 16 * sizeof(int)));
  RPBA_CUDA(cudaMallocHost((void **)&ctx->h_pinned_d, 16 * sizeof(double)));
  // state: rotations from the poses, unit weights, instance copies at X
  if (M) RPBA_KERNEL(ctx, "k_pose_to_R", k_pose_to_R<<<nblk(M, 128), 128, 0, ctx->stream>>>(M, pose_d, ctx->R, ctx->t));
  RPBA_TRY(launch_fill_double(ctx, ctx->obs_w, K, 1.0));
  RPBA_TRY(launch_fill_double(ctx, ctx->Wl, 6LL * P, 0.0));
  RPBA_TRY(sync_mirrors(ctx));
  RPBA_TRY(launch_tp_copies(ctx, 0));
  RPBA_TRY(sync(ctx));
  ctx->n_active_start = nact;
  return RPBA_OK;
}

extern "C" rpba_status rpba_create(const rpba_problem *prob, const rpba_options *opt, void *stream,
                                   rpba_ctx **out) {
  if (!out) return RPBA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!prob) return RPBA_ERR_INVALID_ARG;
  rpba_ctx *h = new (std::nothrow) rpba_ctx();
  if (!h) return RPBA_ERR_OOM;
  Ctx *ctx = &h->c;
  if (opt) ctx->opt = *opt;
  else rpba_default_options(&ctx->opt);
  if ((ctx->opt.precision != 0 && ctx->opt.precision != 1) || ctx->opt.solver < 0 || ctx->opt.solver > 4 ||
      ctx->opt.ir_steps < 0 || ctx->opt.ir_steps > 20 || ctx->opt.pcg_max_iter < 1 || !(ctx->opt.pcg_tol > 0.0) ||
      ctx->opt.chol_tc < 0 || ctx->opt.chol_tc > 2 || ctx->opt.weight_mode < 0 || ctx->opt.weight_mode > 2 ||
      !(ctx->opt.rho0 > 0.0) || ctx->opt.intrinsics < 0 || ctx->opt.intrinsics > 1 ||
      (ctx->opt.intrinsics && ctx->opt.solver == 3)) {
    ctx->err = "invalid precision / solver / ir_steps / intrinsics option";
    *out = h;
    return RPBA_ERR_INVALID_ARG;
  }
  ctx->stream = (cudaStream_t)stream;
  *out = h;
  if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy) {
    // the legacy default stream cannot be captured into a graph: use a blocking
    // stream of our own, which stays ordered with the legacy stream
    cudaError_t es = cudaStreamCreate(&ctx->own_stream);
    if (es == cudaSuccess) ctx->stream = ctx->own_stream;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    ctx->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return RPBA_ERR_CUDA;
  }
  RPBA_CUDA(cudaGetDevice(&ctx->dev));
  if (ctx->opt.tune_cache) {  // kept by the context: the caller's string may go
    ctx->tune_cache_path = ctx->opt.tune_cache;
    ctx->opt.tune_cache = ctx->tune_cache_path.c_str();
  }
  RPBA_TRY(build(ctx, prob));
  if (ctx->opt.tune_cache && *ctx->opt.tune_cache) tune_load(ctx, ctx->opt.tune_cache);
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
// every entry point may change the state, which ends the validity of the
// sub-block costs the outer iteration's tail left (f0_valid); those that only
// read it, and rpba_outer_iteration, which uses them, take CTX_KEEP_COSTS
#define CTX_KEEP_COSTS                       \
  if (!h) return RPBA_ERR_INVALID_ARG;       \
  Ctx *ctx = &h->c;
#define CTX_OR_FAIL \
  CTX_KEEP_COSTS    \
  ctx->f0_valid = false;

// temporary device buffer for host transfers (freed at return)
struct Tmp {
  Ctx *ctx;
  void *p = nullptr;
  Tmp(Ctx *c) : ctx(c) {}
  ~Tmp() {
    if (p) {
      cudaStreamSynchronize(ctx->stream);
      if (ctx->opt.dev_free) ctx->opt.dev_free(p, ctx->opt.alloc_user);
      else cudaFree(p);
    }
  }
  rpba_status alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (ctx->opt.dev_alloc) {
      p = ctx->opt.dev_alloc(bytes, ctx->opt.alloc_user);
      if (!p) { ctx->err = "allocator hook returned NULL"; return RPBA_ERR_OOM; }
      return RPBA_OK;
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { p = nullptr; ctx->err = cudaGetErrorString(e); return RPBA_ERR_OOM; }
    return RPBA_OK;
  }
};

extern "C" rpba_status rpba_info(rpba_ctx *h, int32_t *L, int32_t *P) {
  CTX_KEEP_COSTS;
  if (L) *L = ctx->L;
  if (P) *P = ctx->P;
  return RPBA_OK;
}

extern "C" rpba_status rpba_sub_cameras(rpba_ctx *h, int32_t l, int32_t *cams, int32_t *n) {
  CTX_KEEP_COSTS;
  if (l < 0 || l >= ctx->L) { ctx->err = "sub-block index out of range"; return RPBA_ERR_STATE; }
  int a = ctx->h_sub_cam_ptr[l], b = ctx->h_sub_cam_ptr[l + 1];
  if (cams) for (int p = a; p < b; p++) cams[p - a] = ctx->h_sub_cam[p];
  if (n) *n = b - a;
  return RPBA_OK;
}

// device staging for n doubles: the persistent permutation scratch when it is
// large enough (no allocation per call), else a temporary buffer
static rpba_status staging(Ctx *ctx, Tmp &d, size_t n, double **out) {
  if (n <= ctx->perm_scratch_n) {
    *out = ctx->perm_scratch;
    return RPBA_OK;
  }
  RPBA_TRY(d.alloc(n * sizeof(double)));
  *out = (double *)d.p;
  return RPBA_OK;
}

extern "C" rpba_status rpba_set_cameras(rpba_ctx *h, const double *pose) {
  CTX_OR_FAIL;
  if (!pose) return RPBA_ERR_INVALID_ARG;
  Tmp d(ctx);
  double *buf = nullptr;
  RPBA_TRY(staging(ctx, d, 6 * (size_t)ctx->M, &buf));
  RPBA_CUDA(cudaMemcpyAsync(buf, pose, 6 * (size_t)ctx->M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->M) RPBA_KERNEL(ctx, "k_pose_to_R", k_pose_to_R<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(ctx->M, buf, ctx->R, ctx->t));
  RPBA_TRY(sync_mirrors(ctx));
  return sync(ctx);
}

extern "C" rpba_status rpba_get_camera_rt(rpba_ctx *h, double *R, double *t) {
  CTX_KEEP_COSTS;
  if (!R || !t) return RPBA_ERR_INVALID_ARG;
  RPBA_CUDA(cudaMemcpyAsync(R, ctx->R, 9 * (size_t)ctx->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(t, ctx->t, 3 * (size_t)ctx->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}
extern "C" rpba_status rpba_set_camera_rt(rpba_ctx *h, const double *R, const double *t) {
  CTX_OR_FAIL;
  if (!R || !t) return RPBA_ERR_INVALID_ARG;
  RPBA_CUDA(cudaMemcpyAsync(ctx->R, R, 9 * (size_t)ctx->M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(ctx->t, t, 3 * (size_t)ctx->M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_TRY(sync_mirrors(ctx));
  return sync(ctx);
}
extern "C" rpba_status rpba_get_cameras(rpba_ctx *h, double *pose) {
  CTX_KEEP_COSTS;
  if (!pose) return RPBA_ERR_INVALID_ARG;
  Tmp d(ctx);
  double *buf = nullptr;
  RPBA_TRY(staging(ctx, d, 6 * (size_t)ctx->M, &buf));
  if (ctx->M) RPBA_KERNEL(ctx, "k_R_to_pose", k_R_to_pose<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(ctx->M, ctx->R, ctx->t, buf));
  RPBA_CUDA(cudaMemcpyAsync(pose, buf, 6 * (size_t)ctx->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

// rows of width w permuted by an index map: dst[r] = src[map[r]] (gather)
// or dst[map[r]] = src[r] (scatter)
template <typename T>
__global__ void k_permute_rows(long long n, int w, const int *map, const T *src, T *dst, int gather) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * w) return;
  long long r = e / w;
  int c = (int)(e - r * w);
  long long m = map[r];
  if (gather) dst[r * w + c] = src[m * w + c];
  else dst[m * w + c] = src[r * w + c];
}

// host rows (caller's order) -> device array (internal order), through the scratch
template <typename T>
static rpba_status rows_in(Ctx *ctx, const T *host, T *dev, long long n, int w, const int *map) {
  if (n == 0) return RPBA_OK;
  T *tmp = reinterpret_cast<T *>(ctx->perm_scratch);
  RPBA_CUDA(cudaMemcpyAsync(tmp, host, (size_t)n * w * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_KERNEL(ctx, "k_permute_rows", (k_permute_rows<T><<<nblk(n * w, 256), 256, 0, ctx->stream>>>(n, w, map, tmp, dev, 1)));
  return RPBA_OK;
}

// device array (internal order) -> host rows (caller's order)
template <typename T>
static rpba_status rows_out(Ctx *ctx, const T *dev, T *host, long long n, int w, const int *map) {
  if (n == 0) return RPBA_OK;
  T *tmp = reinterpret_cast<T *>(ctx->perm_scratch);
  RPBA_KERNEL(ctx, "k_permute_rows", (k_permute_rows<T><<<nblk(n * w, 256), 256, 0, ctx->stream>>>(n, w, map, dev, tmp, 0)));
  RPBA_CUDA(cudaMemcpyAsync(host, tmp, (size_t)n * w * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

// instance rows: map[c] = internal row of canonical row c.
// host (canonical) -> device (internal): internal[map[c]] = host[c]
template <typename T>
static rpba_status rows_in_scatter(Ctx *ctx, const T *host, T *dev, long long n, int w, const int *map) {
  if (n == 0) return RPBA_OK;
  T *tmp = reinterpret_cast<T *>(ctx->perm_scratch);
  RPBA_CUDA(cudaMemcpyAsync(tmp, host, (size_t)n * w * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_KERNEL(ctx, "k_permute_rows", (k_permute_rows<T><<<nblk(n * w, 256), 256, 0, ctx->stream>>>(n, w, map, tmp, dev, 0)));
  return RPBA_OK;
}

// device (internal) -> host (canonical): host[c] = internal[map[c]]
template <typename T>
static rpba_status rows_out_gather(Ctx *ctx, const T *dev, T *host, long long n, int w, const int *map) {
  if (n == 0) return RPBA_OK;
  T *tmp = reinterpret_cast<T *>(ctx->perm_scratch);
  RPBA_KERNEL(ctx, "k_permute_rows", (k_permute_rows<T><<<nblk(n * w, 256), 256, 0, ctx->stream>>>(n, w, map, dev, tmp, 1)));
  RPBA_CUDA(cudaMemcpyAsync(host, tmp, (size_t)n * w * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

__global__ void k_to_float32(long long n, const double *a, float *b) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

extern "C" rpba_status rpba_set_points(rpba_ctx *h, const double *X, const uint8_t *active) {
  CTX_OR_FAIL;
  if (X) RPBA_TRY(rows_in(ctx, X, ctx->X, ctx->N, 3, ctx->d_pt_inv));
  if (active) RPBA_TRY(rows_in(ctx, active, ctx->active, ctx->N, 1, ctx->d_pt_inv));
  RPBA_TRY(sync_mirrors(ctx));
  return sync(ctx);
}

extern "C" rpba_status rpba_get_intrinsics(rpba_ctx *h, double *fk) {
  CTX_KEEP_COSTS;
  if (!fk) return RPBA_ERR_INVALID_ARG;
  const int M = ctx->M;
  std::vector<double> intr(3 * (size_t)M), k1(M, 0.0);
  if (M) RPBA_CUDA(cudaMemcpyAsync(intr.data(), ctx->intr, intr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  if (M && ctx->k1)
    RPBA_CUDA(cudaMemcpyAsync(k1.data(), ctx->k1, M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  for (int i = 0; i < M; i++) {
    fk[2 * i] = intr[3 * (size_t)i];
    fk[2 * i + 1] = k1[i];
  }
  return RPBA_OK;
}

// sets f and k1 of every camera; the FP32 form's camera records follow
extern "C" rpba_status rpba_set_intrinsics(rpba_ctx *h, const double *fk) {
  CTX_OR_FAIL;
  if (!fk) return RPBA_ERR_INVALID_ARG;
  const int M = ctx->M;
  std::vector<double> intr(3 * (size_t)M), k1(M);
  if (M) RPBA_CUDA(cudaMemcpyAsync(intr.data(), ctx->intr, intr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  RPBA_TRY(sync(ctx));
  for (int i = 0; i < M; i++) {
    if (!(fk[2 * i] > 0.0) || !isfinite(fk[2 * i + 1]) ||
        (ctx->cd == 6 && (fk[2 * i] != intr[3 * (size_t)i] || fk[2 * i + 1] != 0.0))) {
      ctx->err = "intrinsics: f must be positive and k1 finite; without the intrinsics option they are fixed";
      return RPBA_ERR_INVALID_ARG;
    }
    intr[3 * (size_t)i] = fk[2 * i];
    k1[i] = fk[2 * i + 1];
  }
  if (M) RPBA_CUDA(cudaMemcpyAsync(ctx->intr, intr.data(), intr.size() * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
  if (M && ctx->k1)
    RPBA_CUDA(cudaMemcpyAsync(ctx->k1, k1.data(), M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_TRY(sync_mirrors(ctx));
  return sync(ctx);
}

extern "C" rpba_status rpba_get_points(rpba_ctx *h, double *X, uint8_t *active) {
  CTX_KEEP_COSTS;
  if (X) RPBA_TRY(rows_out(ctx, ctx->X, X, ctx->N, 3, ctx->d_pt_inv));
  if (active) RPBA_TRY(rows_out(ctx, ctx->active, active, ctx->N, 1, ctx->d_pt_inv));
  return sync(ctx);
}

// instances leave and enter in the canonical order (sub-block, caller's point id)
extern "C" rpba_status rpba_get_instances(rpba_ctx *h, int32_t *ip, int32_t *is, double *Xl, double *Wl) {
  CTX_KEEP_COSTS;
  const std::vector<int> &canon = ctx->h_inst_canon;
  for (size_t c = 0; c < (size_t)ctx->P; c++) {
    int q = canon[c];
    if (ip) ip[c] = ctx->h_pt_inv[ctx->h_inst_pt[q]];
    if (is) is[c] = ctx->h_inst_sub[q];
  }
  // canonical c <- internal canon[c]: the caller's order is the canonical one
  if (Xl) RPBA_TRY(rows_out_gather(ctx, ctx->Xl, Xl, ctx->P, 3, ctx->d_inst_canon));
  if (Wl) RPBA_TRY(rows_out_gather(ctx, ctx->Wl, Wl, ctx->P, 6, ctx->d_inst_canon));
  return sync(ctx);
}

extern "C" rpba_status rpba_set_instances(rpba_ctx *h, const double *Xl, const double *Wl) {
  CTX_OR_FAIL;
  if (Xl) RPBA_TRY(rows_in_scatter(ctx, Xl, ctx->Xl, ctx->P, 3, ctx->d_inst_canon));
  if (Wl) {
    RPBA_TRY(rows_in_scatter(ctx, Wl, ctx->Wl, ctx->P, 6, ctx->d_inst_canon));
    if (ctx->Wl32 && ctx->P)
      RPBA_KERNEL(ctx, "k_to_float32", k_to_float32<<<nblk(6LL * ctx->P, 256), 256, 0, ctx->stream>>>(
                                           6LL * ctx->P, ctx->Wl, ctx->Wl32));
  }
  RPBA_TRY(sync_mirrors(ctx));
  return sync(ctx);
}

extern "C" rpba_status rpba_get_weights(rpba_ctx *h, double *w) {
  CTX_KEEP_COSTS;
  if (!w) return RPBA_ERR_INVALID_ARG;
  std::vector<double> g(ctx->K);
  if (ctx->K) RPBA_CUDA(cudaMemcpyAsync(g.data(), ctx->obs_w, ctx->K * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  for (int p = 0; p < ctx->K; p++) w[ctx->h_obs_user[p]] = g[p];
  return RPBA_OK;
}

extern "C" rpba_status rpba_set_weights(rpba_ctx *h, const double *w) {
  CTX_OR_FAIL;
  if (!w) return RPBA_ERR_INVALID_ARG;
  std::vector<double> g(ctx->K);
  for (int p = 0; p < ctx->K; p++) g[p] = w[ctx->h_obs_user[p]];
  if (ctx->K) RPBA_CUDA(cudaMemcpyAsync(ctx->obs_w, g.data(), ctx->K * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->obs_w32 && ctx->K) {
    std::vector<float> g32(g.begin(), g.end());
    RPBA_CUDA(cudaMemcpyAsync(ctx->obs_w32, g32.data(), ctx->K * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    return sync(ctx);
  }
  return sync(ctx);
}

extern "C" rpba_status rpba_residuals(rpba_ctx *h, double *v) {
  CTX_OR_FAIL;
  if (!v) return RPBA_ERR_INVALID_ARG;
  Tmp d(ctx);
  RPBA_TRY(d.alloc(2 * (size_t)ctx->K * sizeof(double)));
  RPBA_TRY(launch_residuals(ctx, (double *)d.p));
  RPBA_CUDA(cudaMemcpyAsync(v, d.p, 2 * (size_t)ctx->K * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

extern "C" rpba_status rpba_jacobians(rpba_ctx *h, double *Jc, double *Jx) {
  CTX_OR_FAIL;
  if (!Jc || !Jx) return RPBA_ERR_INVALID_ARG;
  Tmp a(ctx), b(ctx);
  RPBA_TRY(a.alloc(2 * (size_t)ctx->cd * ctx->K * sizeof(double)));
  RPBA_TRY(b.alloc(6 * (size_t)ctx->K * sizeof(double)));
  RPBA_TRY(launch_jacobians(ctx, (double *)a.p, (double *)b.p));
  RPBA_CUDA(cudaMemcpyAsync(Jc, a.p, 2 * (size_t)ctx->cd * ctx->K * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(Jx, b.p, 6 * (size_t)ctx->K * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

extern "C" rpba_status rpba_sigma0(rpba_ctx *h, double *s0, double *rms) {
  CTX_KEEP_COSTS;
  return launch_sigma0(ctx, s0, rms);
}

extern "C" rpba_status rpba_camera_scale(rpba_ctx *h, double *sigma) {
  CTX_OR_FAIL;
  RPBA_TRY(launch_camera_scale(ctx));
  if (sigma && ctx->M)
    RPBA_CUDA(cudaMemcpyAsync(sigma, ctx->cam_sigma, ctx->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

extern "C" rpba_status rpba_robust_weights(rpba_ctx *h, int32_t *n_down) {
  CTX_OR_FAIL;
  int nd = 0;
  RPBA_TRY(launch_robust_weights(ctx, &nd));
  if (n_down) *n_down = nd;
  return RPBA_OK;
}

extern "C" rpba_status rpba_intersect_points(rpba_ctx *h, int32_t tp_only, int32_t *n_dropped) {
  CTX_OR_FAIL;
  int nd = 0;
  RPBA_TRY(launch_intersect(ctx, tp_only ? 1 : 0, &nd));
  if (n_dropped) *n_dropped = nd;
  return RPBA_OK;
}

extern "C" rpba_status rpba_intersect(rpba_ctx *h) {
  CTX_OR_FAIL;
  // The first intersection starts from the raw input, far from the solution,
  // where a point's fate (kept or dropped) decides which local minimum the
  // blocks descend to. It runs once per run, in FP64 in every form, so that
  // both forms start from the same point set.
  RPBA_TRY(launch_intersect(ctx, 0, nullptr, true));
  RPBA_TRY(launch_tp_copies(ctx, 0));
  ctx->intersected = true;
  return sync(ctx);
}

extern "C" rpba_status rpba_covariance(rpba_ctx *h, const int32_t *ids, int32_t n, double *out9) {
  CTX_OR_FAIL;
  if (n < 0 || (n && (!ids || !out9))) return RPBA_ERR_INVALID_ARG;
  if (n == 0) return RPBA_OK;
  Tmp di(ctx), dout(ctx);
  RPBA_TRY(di.alloc((size_t)n * sizeof(int)));
  RPBA_TRY(dout.alloc(9 * (size_t)n * sizeof(double)));
  std::vector<int> idi(n);  // the internal numbering of the points asked for
  for (int e = 0; e < n; e++) {
    if (ids[e] < 0 || ids[e] >= ctx->N) { ctx->err = "point id out of range"; return RPBA_ERR_INVALID_ARG; }
    idi[e] = ctx->h_pt_perm[ids[e]];
  }
  RPBA_CUDA(cudaMemcpyAsync(di.p, idi.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_KERNEL(ctx, "k_covariance", k_covariance<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, (const int *)di.p, ctx->R, ctx->t, ctx->intr, ctx->cd == 8 ? ctx->k1 : nullptr, ctx->X,
                                                     ctx->active, ctx->pt_inst_ptr, ctx->pt_inst, ctx->inst_obs_ptr,
                                                     ctx->obs_cam, ctx->obs_winv, ctx->has_winv, ctx->obs_w, ctx->N,
                                                     (double *)dout.p));
  RPBA_CUDA(cudaMemcpyAsync(out9, dout.p, 9 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);  // before idi goes
}

extern "C" rpba_status rpba_sub_costs(rpba_ctx *h, double *F) {
  CTX_OR_FAIL;
  RPBA_TRY(launch_sub_costs(ctx, 0, ctx->lm_F));
  if (F && ctx->L) RPBA_CUDA(cudaMemcpyAsync(F, ctx->lm_F, ctx->L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

extern "C" rpba_status rpba_rcs(rpba_ctx *h, int32_t l, double lambda, double *S, double *y) {
  CTX_OR_FAIL;
  if (l < 0 || l >= ctx->L) { ctx->err = "sub-block index out of range"; return RPBA_ERR_STATE; }
  RPBA_TRY(launch_fill_double(ctx, ctx->lm_lambda, ctx->L, lambda));
  RPBA_TRY(launch_fill_int(ctx, ctx->lm_run, ctx->L, 0));
  RPBA_TRY(launch_fill_int(ctx, ctx->lm_run + l, 1, 1));
  RPBA_TRY(launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run));
  int n = ctx->cd * (ctx->h_sub_cam_ptr[l + 1] - ctx->h_sub_cam_ptr[l]);
  int np = ctx->h_npad[l];
  std::vector<double> full((size_t)np * np), yf(np);
  if (np) {
    RPBA_CUDA(cudaMemcpyAsync(full.data(), ctx->S + ctx->h_S_off[l], (size_t)np * np * sizeof(double),
                              cudaMemcpyDeviceToHost, ctx->stream));
    int yoff = 0;
    for (int a = 0; a < l; a++) yoff += ctx->h_npad[a];
    RPBA_CUDA(cudaMemcpyAsync(yf.data(), ctx->y + yoff, np * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  RPBA_TRY(sync(ctx));
  // the device keeps the lower triangle; the caller gets the symmetric matrix
  for (int r = 0; r < n; r++) {
    if (S)
      for (int c = 0; c < n; c++) S[(size_t)r * n + c] = c <= r ? full[(size_t)r * np + c] : full[(size_t)c * np + r];
    if (y) y[r] = yf[r];
  }
  return RPBA_OK;
}

// one lock-step LM iteration of the running sub-blocks
static rpba_status lm_iteration(Ctx *ctx) {
  RPBA_TRY(launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run));
  RPBA_TRY(launch_solve_rcs(ctx, ctx->lm_run, ctx->lm_cholfail));
  RPBA_TRY(launch_backsub_trial(ctx, ctx->lm_run));
  return RPBA_OK;
}

extern "C" rpba_status rpba_lm_step(rpba_ctx *h, double lambda, int32_t *accepted, double *Fb, double *Ft,
                                    double *dc, double *dx) {
  CTX_OR_FAIL;
  int L = ctx->L;
  RPBA_TRY(launch_lm_init(ctx));
  RPBA_TRY(launch_fill_double(ctx, ctx->lm_lambda, L, lambda));
  RPBA_TRY(lm_iteration(ctx));
  std::vector<double> F(L), Fn(L);
  std::vector<int> fail(L), run(L);
  RPBA_CUDA(cudaMemcpyAsync(F.data(), ctx->lm_F, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(Fn.data(), ctx->lm_Ft, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(fail.data(), ctx->lm_cholfail, L * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaMemcpyAsync(run.data(), ctx->lm_run, L * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> Xl(3 * (size_t)ctx->P), Xlt(3 * (size_t)ctx->P);
  if (dx && ctx->P) {
    RPBA_CUDA(cudaMemcpyAsync(Xl.data(), ctx->Xl, Xl.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RPBA_CUDA(cudaMemcpyAsync(Xlt.data(), ctx->Xlt, Xlt.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  int ytot = 0;
  for (int l = 0; l < L; l++) ytot += ctx->h_npad[l];
  std::vector<double> dCh(ytot);
  if (dc && ytot)
    RPBA_CUDA(cudaMemcpyAsync(dCh.data(), ctx->dC, ytot * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  std::vector<int> acc(L);
  for (int l = 0; l < L; l++) {
    if (!run[l]) acc[l] = 0;
    else if (fail[l]) acc[l] = -1;
    else acc[l] = (isfinite(Fn[l]) && Fn[l] < F[l]) ? 1 : 0;
    if (accepted) accepted[l] = acc[l];
    if (Fb) Fb[l] = F[l];
    if (Ft) Ft[l] = (run[l] && !fail[l]) ? Fn[l] : F[l];
  }
  if (dc) {
    int o = 0, yo = 0;
    for (int l = 0; l < L; l++) {
      int n = ctx->cd * (ctx->h_sub_cam_ptr[l + 1] - ctx->h_sub_cam_ptr[l]);
      for (int r = 0; r < n; r++) dc[o + r] = dCh[yo + r];
      o += n;
      yo += ctx->h_npad[l];
    }
  }
  if (dx)  // instances in the canonical order
    for (size_t c = 0; c < (size_t)ctx->P; c++) {
      size_t q = ctx->h_inst_canon[c];
      for (int e = 0; e < 3; e++) dx[3 * c + e] = Xlt[3 * q + e] - Xl[3 * q + e];
    }
  std::vector<int> accp(L);
  for (int l = 0; l < L; l++) accp[l] = acc[l] == 1;
  RPBA_CUDA(cudaMemcpyAsync(ctx->lm_acc, accp.data(), L * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  RPBA_TRY(launch_lm_apply(ctx, ctx->lm_acc));
  return sync(ctx);
}

// ---------------------------------------------------------------------------
// the iteration (Sec. 5)
// ---------------------------------------------------------------------------
// after the RCS solve: back-substitution, trial cost, LM decision and update,
// and the running count for the host
static rpba_status lm_post(Ctx *ctx) {
  RPBA_TRY(launch_backsub_trial(ctx, ctx->lm_run));
  RPBA_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(int), ctx->stream));
  RPBA_TRY(launch_lm_decide(ctx));
  RPBA_TRY(launch_lm_apply(ctx, ctx->lm_acc));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter, ctx->counters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  return RPBA_OK;
}

static bool pcg_solver(const Ctx *ctx) { return ctx->opt.solver == 1 || ctx->opt.solver == 3; }

// PCG solvers: RCS assembly, preconditioner set-up and CG start (the part
// before the host-driven CG loop)
static rpba_status lm_pre_pcg(Ctx *ctx) {
  RPBA_TRY(launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run));
  if (ctx->opt.solver == 3) {
    RPBA_TRY(learned_setup(ctx, ctx->lm_run, ctx->lm_cholfail, &ctx->fsai));
    return pcg_init(ctx, ctx->lm_run, ctx->lm_cholfail, &ctx->fsai);
  }
  RPBA_TRY(pcg_bj_setup(ctx, ctx->lm_run, ctx->lm_cholfail));
  return pcg_init(ctx, ctx->lm_run, ctx->lm_cholfail, nullptr);
}

// PCG solvers: the CG loop and the solution (and solver 3's block-Jacobi check)
static rpba_status lm_cg(Ctx *ctx) {
  const FsaiApply *f = ctx->opt.solver == 3 ? &ctx->fsai : nullptr;
  int iters = 0;
  RPBA_TRY(pcg_loop(ctx, f, &iters));
  // solver 4 (auto): a solve that needed more lock-step iterations than the
  // direct solve is worth moves the context to the direct solver, from the
  // next LM step on
  if (!ctx->capture && ctx->auto_solver &&
      iters > (ff_pcg(ctx) ? RPBA_AUTO_PCG_MAX_ITER_FP32 : RPBA_AUTO_PCG_MAX_ITER))
    ctx->auto_switch = true;
  RPBA_TRY(pcg_out(ctx, ctx->lm_run, ctx->lm_cholfail));
  if (ctx->opt.solver == 3) RPBA_TRY(learned_fallback(ctx, ctx->lm_run, ctx->lm_cholfail));
  return RPBA_OK;
}

// the work of one lock-step LM iteration after the LM inputs are set: build,
// solve, trial, decide, apply, and the running count to pinned memory
static rpba_status lm_step_body(Ctx *ctx) {
  if (pcg_solver(ctx)) {
    RPBA_TRY(lm_pre_pcg(ctx));
    RPBA_TRY(lm_cg(ctx));
    return lm_post(ctx);
  }
  RPBA_TRY(launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run));
  RPBA_TRY(launch_solve_rcs(ctx, ctx->lm_run, ctx->lm_cholfail));
  return lm_post(ctx);
}

static void free_graph(GraphRec *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto &e : g->events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  delete g;
}

static void free_lm_graphs(Ctx *ctx) {
  free_graph(ctx->lm_graph);
  free_graph(ctx->lm_graph_pre);
  free_graph(ctx->lm_graph_post);
  ctx->lm_graph = ctx->lm_graph_pre = ctx->lm_graph_post = nullptr;
  for (GraphRec *&g : ctx->outer_graph) {
    free_graph(g);
    g = nullptr;
  }
}

// capture fn's launches into a graph (all launch parameters are fixed per
// context). *out stays NULL when the stream cannot be captured (e.g. the
// legacy default stream) or the capture fails: the caller then runs eagerly.
template <class F>
static rpba_status capture_graph(Ctx *ctx, GraphRec **out, F fn) {
  *out = nullptr;
  GraphRec *g = new GraphRec();
  g->with_events = ctx->prof_enabled;
  g->prof_only = ctx->prof_only;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    delete g;
    cudaGetLastError();
    return RPBA_OK;
  }
  ctx->capture = g;
  rpba_status st = fn();
  ctx->capture = nullptr;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(ctx->stream, &graph);
  if (st != RPBA_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    free_graph(g);
    cudaGetLastError();  // clear the capture error; run eagerly from now on
    ctx->err.clear();
    return RPBA_OK;
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    free_graph(g);
    ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
    return RPBA_ERR_CUDA;
  }
  *out = g;
  return RPBA_OK;
}

// count a replayed graph's kernels (and add their event times while
// profiling); the stream has been synchronised
static rpba_status account(Ctx *ctx, GraphRec *g) {
  for (const char *k : g->kernels) {
    ctx->launches++;
    ctx->launch_by_name[k]++;
  }
  if (g->pcg_loop) {  // the loop bodies ran as often as their counters say
    long long steps = ctx->h_pinned_counter[PCG_LOOP_COUNTERS], stages = ctx->h_pinned_counter[PCG_LOOP_COUNTERS + 1];
    for (const char *k : g->loop_inner) {
      ctx->launches += steps;
      ctx->launch_by_name[k] += steps;
    }
    for (const char *k : g->loop_outer) {
      ctx->launches += stages;
      ctx->launch_by_name[k] += stages;
    }
  }
  if (ctx->prof_enabled)
    for (auto &ev : g->events) {
      float t = 0.f;
      RPBA_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
      ctx->prof_ms[ev.name] += t;
    }
  return RPBA_OK;
}

// one lock-step LM iteration, then the host reads the running count. Direct
// solvers, and the FP32 form's block-Jacobi PCG (its loop as conditional
// graph nodes): one captured graph. Other PCG solvers, or a timed loop
// kernel: a graph up to the CG start, the CG loop run from the host (it
// stops on count reads), and a graph from the back-substitution on.
static rpba_status lm_step_exec(Ctx *ctx) {
  GraphRec *any = ctx->lm_graph ? ctx->lm_graph : ctx->lm_graph_pre;
  if (any && (any->with_events != ctx->prof_enabled || any->prof_only != ctx->prof_only))
    free_lm_graphs(ctx);  // timing nodes only while profiling
  if (pcg_solver(ctx)) {
    // FP32 form: the whole step, CG loop included, as one graph
    if (ctx->use_graphs && pcg_device_loop(ctx)) {
      if (!ctx->lm_graph) {
        RPBA_TRY(capture_graph(ctx, &ctx->lm_graph, [&] { return lm_step_body(ctx); }));
        if (!ctx->lm_graph) ctx->pcg_no_device_loop = true;  // the host-driven loop from now on
      }
      if (ctx->lm_graph) {
        RPBA_CUDA(cudaGraphLaunch(ctx->lm_graph->exec, ctx->stream));
        RPBA_TRY(sync(ctx));
        if (ctx->auto_solver && ctx->h_pinned_counter[PCG_LOOP_COUNTERS] > RPBA_AUTO_PCG_MAX_ITER_FP32)
          ctx->auto_switch = true;
        return account(ctx, ctx->lm_graph);
      }
    }
    if (ctx->use_graphs && !ctx->lm_graph_pre) {
      RPBA_TRY(capture_graph(ctx, &ctx->lm_graph_pre, [&] { return lm_pre_pcg(ctx); }));
      if (ctx->lm_graph_pre) RPBA_TRY(capture_graph(ctx, &ctx->lm_graph_post, [&] { return lm_post(ctx); }));
      if (!ctx->lm_graph_pre || !ctx->lm_graph_post) {
        free_lm_graphs(ctx);
        ctx->use_graphs = false;
      }
    }
    if (ctx->use_graphs) {
      RPBA_CUDA(cudaGraphLaunch(ctx->lm_graph_pre->exec, ctx->stream));
      RPBA_TRY(lm_cg(ctx));
      RPBA_CUDA(cudaGraphLaunch(ctx->lm_graph_post->exec, ctx->stream));
      RPBA_TRY(sync(ctx));
      RPBA_TRY(account(ctx, ctx->lm_graph_pre));
      return account(ctx, ctx->lm_graph_post);
    }
    RPBA_TRY(lm_step_body(ctx));
    return sync(ctx);
  }
  if (ctx->use_graphs && !ctx->lm_graph) {
    RPBA_TRY(capture_graph(ctx, &ctx->lm_graph, [&] { return lm_step_body(ctx); }));
    if (!ctx->lm_graph) ctx->use_graphs = false;
  }
  if (ctx->use_graphs && ctx->lm_graph) {
    RPBA_CUDA(cudaGraphLaunch(ctx->lm_graph->exec, ctx->stream));
    RPBA_TRY(sync(ctx));
    return account(ctx, ctx->lm_graph);
  }
  RPBA_TRY(lm_step_body(ctx));
  return sync(ctx);
}

static rpba_status lm_step_run(Ctx *ctx) {
  RPBA_TRY(lm_step_exec(ctx));
  if (ctx->auto_switch) {  // the step is complete: its graphs can go
    ctx->auto_switch = false;
    ctx->opt.solver = 2;
    free_lm_graphs(ctx);
  }
  return RPBA_OK;
}

// the tail of one outer iteration: exchange, robust weights (when on), TP
// intersection, TP copies and the sigma_0 sums. Nothing in it needs a host
// read, so it runs as one captured graph; then the host reads sigma_0.
static rpba_status outer_tail_body(Ctx *ctx, bool robust) {
  RPBA_TRY(launch_exchange(ctx));
  if (robust) RPBA_TRY(launch_robust_weights(ctx, nullptr));
  // the FP32 form's TP intersection restarts the converged TPs' copies itself
  const bool fused_copies = ctx->opt.precision == 1;
  RPBA_TRY(launch_intersect(ctx, 1, nullptr, false, fused_copies));
  if (!fused_copies) RPBA_TRY(launch_tp_copies(ctx, 1));
  return cost_sigma0_launch(ctx);
}

static rpba_status outer_tail(Ctx *ctx, bool robust, double *sigma0) {
  // the scalar TP weight's rho for this outer iteration's intersection
  ctx->outer_done++;
  if (ctx->opt.weight_mode == 2) {
    ctx->h_pinned_d[8] = ctx->opt.rho0 * pow(1.01, (double)ctx->outer_done);
    RPBA_CUDA(cudaMemcpyAsync(ctx->wrho, ctx->h_pinned_d + 8, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  }
  GraphRec *&g = ctx->outer_graph[robust ? 1 : 0];
  if (g && (g->with_events != ctx->prof_enabled || g->prof_only != ctx->prof_only)) {
    free_graph(g);  // timing nodes only while profiling
    g = nullptr;
  }
  if (ctx->use_graphs && !g) RPBA_TRY(capture_graph(ctx, &g, [&] { return outer_tail_body(ctx, robust); }));
  if (g) {
    RPBA_CUDA(cudaGraphLaunch(g->exec, ctx->stream));
    RPBA_TRY(sync(ctx));
    RPBA_TRY(account(ctx, g));
  } else {
    RPBA_TRY(outer_tail_body(ctx, robust));
    RPBA_TRY(sync(ctx));
  }
  sigma0_finish(ctx, sigma0, nullptr, nullptr, nullptr);
  // the FP32 form's tail left the sub-block costs of this state for the next bact
  ctx->f0_valid = ctx->opt.precision == 1 && ctx->n_chunks > 0 && ctx->L > 0;
  return RPBA_OK;
}

// bact of all sub-blocks in lock step; returns LM iterations summed over
// sub-blocks and the lock-step count
static rpba_status run_bact(Ctx *ctx, int *inner_total, int *launches) {
  RPBA_TRY(launch_lm_init(ctx));
  int n = 0;
  for (;;) {
    RPBA_TRY(lm_step_run(ctx));
    n++;
    if (ctx->h_pinned_counter[0] == 0) break;
    if (n > 100000) { ctx->err = "LM loop did not terminate"; return RPBA_ERR_NOT_CONVERGED; }
  }
  std::vector<int> it(ctx->L);
  if (ctx->L) RPBA_CUDA(cudaMemcpyAsync(it.data(), ctx->lm_it, ctx->L * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  *inner_total += std::accumulate(it.begin(), it.end(), 0);
  *launches += n;
  return RPBA_OK;
}

extern "C" rpba_status rpba_bact(rpba_ctx *h, int32_t *iters) {
  CTX_OR_FAIL;
  int tot = 0, launches = 0;
  RPBA_TRY(run_bact(ctx, &tot, &launches));
  if (iters && ctx->L) {
    RPBA_CUDA(cudaMemcpyAsync(iters, ctx->lm_it, ctx->L * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RPBA_TRY(sync(ctx));
  }
  return RPBA_OK;
}

extern "C" rpba_status rpba_set_subblock_mask(rpba_ctx *h, const uint8_t *mask) {
  CTX_OR_FAIL;
  if (ctx->L == 0) return RPBA_OK;
  std::vector<uint8_t> m(ctx->L, 1);
  if (mask)
    for (int l = 0; l < ctx->L; l++) m[l] = mask[l] ? 1 : 0;
  RPBA_CUDA(cudaMemcpyAsync(ctx->sub_mask, m.data(), m.size(), cudaMemcpyHostToDevice, ctx->stream));
  return sync(ctx);
}

extern "C" rpba_status rpba_set_point_mask(rpba_ctx *h, const uint8_t *mask) {
  CTX_OR_FAIL;
  if (ctx->N == 0) return RPBA_OK;
  std::vector<uint8_t> m(ctx->N, 1);
  if (mask)  // caller's numbering -> internal
    for (int j = 0; j < ctx->N; j++) m[ctx->h_pt_perm[j]] = mask[j] ? 1 : 0;
  RPBA_CUDA(cudaMemcpyAsync(ctx->pt_mask, m.data(), m.size(), cudaMemcpyHostToDevice, ctx->stream));
  return sync(ctx);
}

// ---------------------------------------------------------------------------
// autotuner: launch shapes timed on the context's own data, cached per workload
// ---------------------------------------------------------------------------
static std::string tune_signature(const Ctx *ctx) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  char b[160];
  snprintf(b, sizeof(b), "M%d_N%d_K%d_L%d_P%d_prec%d_solver%d_cd%d_sm%d", ctx->M, ctx->N, ctx->K, ctx->L,
           ctx->P, ctx->opt.precision, ctx->opt.solver, ctx->cd, sms);
  return b;
}

// one cache line (JSON object): {"sig": "...", "isect": 128, "lin": 128, "backsub": 128, "robust": 256, "chol_tc": 2}
static std::string tune_line(const Ctx *ctx) {
  char b[320];
  snprintf(b, sizeof(b), "{\"sig\": \"%s\", \"isect\": %d, \"lin\": %d, \"backsub\": %d, \"robust\": %d, \"chol_tc\": %d}",
           tune_signature(ctx).c_str(), ctx->tune.isect, ctx->tune.lin, ctx->tune.backsub, ctx->tune.robust,
           ctx->opt.chol_tc);
  return b;
}

static bool json_int(const std::string &line, const char *key, int *out) {
  std::string k = std::string("\"") + key + "\":";
  size_t p = line.find(k);
  if (p == std::string::npos) return false;
  return sscanf(line.c_str() + p + k.size(), " %d", out) == 1;
}

static bool tune_valid(int threads) { return threads >= 32 && threads <= 1024 && threads % 32 == 0; }

// the context's workload in the cache: applies its values; false if absent
static bool tune_load(Ctx *ctx, const char *path) {
  FILE *f = fopen(path, "r");
  if (!f) return false;
  std::string want = "\"sig\": \"" + tune_signature(ctx) + "\"";
  char buf[1024];
  bool found = false;
  while (fgets(buf, sizeof(buf), f)) {
    std::string line(buf);
    if (line.find(want) == std::string::npos) continue;
    Tuning t;
    int chol = ctx->opt.chol_tc;
    bool ok = json_int(line, "isect", &t.isect) && json_int(line, "lin", &t.lin) &&
              json_int(line, "backsub", &t.backsub) && json_int(line, "robust", &t.robust) &&
              json_int(line, "chol_tc", &chol);
    if (ok && tune_valid(t.isect) && tune_valid(t.lin) && tune_valid(t.backsub) && tune_valid(t.robust) &&
        chol >= 0 && chol <= 2) {
      ctx->tune = t;
      if (ctx->tc_ready || chol == 0) ctx->opt.chol_tc = chol;
      found = true;
    }
  }
  fclose(f);
  return found;
}

// rewrite the cache with this workload's line replaced (or appended)
static rpba_status tune_store(Ctx *ctx, const char *path) {
  std::vector<std::string> keep;
  std::string want = "\"sig\": \"" + tune_signature(ctx) + "\"";
  if (FILE *f = fopen(path, "r")) {
    char buf[1024];
    while (fgets(buf, sizeof(buf), f)) {
      std::string line(buf);
      if (line.find(want) == std::string::npos && line.find("\"sig\"") != std::string::npos) keep.push_back(line);
    }
    fclose(f);
  }
  FILE *f = fopen(path, "w");
  if (!f) {
    ctx->err = std::string("cannot write the tune cache ") + path;
    return RPBA_ERR_INVALID_ARG;
  }
  for (auto &l : keep) fputs(l.c_str(), f);
  fprintf(f, "%s\n", tune_line(ctx).c_str());
  fclose(f);
  return RPBA_OK;
}

// mean time of reps calls of fn after one untimed call (CUDA events on the
// context's stream)
template <class F>
static rpba_status time_phase(Ctx *ctx, int reps, float *ms, F fn) {
  RPBA_TRY(fn());
  cudaEvent_t a, b;
  RPBA_CUDA(cudaEventCreate(&a));
  RPBA_CUDA(cudaEventCreate(&b));
  RPBA_CUDA(cudaEventRecord(a, ctx->stream));
  for (int r = 0; r < reps; r++) RPBA_TRY(fn());
  RPBA_CUDA(cudaEventRecord(b, ctx->stream));
  RPBA_CUDA(cudaEventSynchronize(b));
  float t = 0.f;
  RPBA_CUDA(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / (float)reps;
  return RPBA_OK;
}

template <class F>
static rpba_status pick(Ctx *ctx, int *param, const std::vector<int> &cand, F fn) {
  int best = *param;
  float best_ms = 1e30f;
  for (int c : cand) {
    *param = c;
    float ms = 0.f;
    RPBA_TRY(time_phase(ctx, 5, &ms, fn));
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  *param = best;
  return RPBA_OK;
}

extern "C" rpba_status rpba_tune(rpba_ctx *h, const char *cache_path, int32_t *chosen) {
  CTX_OR_FAIL;
  if (!ctx->intersected) RPBA_TRY(rpba_intersect(h));
  bool saved_graphs = ctx->use_graphs, saved_prof = ctx->prof_enabled;
  ctx->prof_enabled = false;
  // the robust weights and the TP intersection change the state: it is saved
  // here and restored after their timings
  std::vector<double> X(3 * (size_t)ctx->N), Xl(3 * (size_t)ctx->P), Wl(6 * (size_t)ctx->P), w(ctx->K);
  std::vector<uint8_t> act(ctx->N);
  RPBA_TRY(rpba_get_points(h, X.data(), act.data()));
  RPBA_TRY(rpba_get_instances(h, nullptr, nullptr, Xl.data(), Wl.data()));
  RPBA_TRY(rpba_get_weights(h, w.data()));
  auto restore = [&]() -> rpba_status {
    RPBA_TRY(rpba_set_points(h, X.data(), act.data()));
    RPBA_TRY(rpba_set_instances(h, Xl.data(), Wl.data()));
    return rpba_set_weights(h, w.data());
  };
  RPBA_TRY(pick(ctx, &ctx->tune.robust, {128, 256, 512}, [&] { return launch_robust_weights(ctx, nullptr); }));
  RPBA_TRY(restore());
  // the RCS assembly (linearisation), then the back-substitution with trial:
  // per-LM-step scratch only, the state is unchanged
  RPBA_TRY(launch_lm_init(ctx));
  RPBA_TRY(pick(ctx, &ctx->tune.lin, {64, 128, 256},
                [&] { return launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run); }));
  RPBA_TRY(launch_solve_rcs(ctx, ctx->lm_run, ctx->lm_cholfail));
  RPBA_TRY(pick(ctx, &ctx->tune.backsub, {64, 128, 256}, [&] { return launch_backsub_trial(ctx, ctx->lm_run); }));
  // the direct solve's factorisation: persistent or one launch per step
  if ((ctx->opt.solver == 2 || ctx->auto_solver) && ctx->tc_ready) {
    int s = ctx->opt.solver;
    ctx->opt.solver = 2;
    rpba_status st = pick(ctx, &ctx->opt.chol_tc, {0, 1, 2}, [&] { return launch_solve_rcs(ctx, ctx->lm_run, ctx->lm_cholfail); });
    ctx->opt.solver = s;
    RPBA_TRY(st);
  }
  // the TP intersection from the saved state every time
  {
    rpba_status st = pick(ctx, &ctx->tune.isect, {64, 128, 256}, [&]() -> rpba_status {
      RPBA_TRY(restore());
      return launch_intersect(ctx, 1, nullptr);
    });
    RPBA_TRY(restore());
    RPBA_TRY(st);
  }
  ctx->use_graphs = saved_graphs;
  ctx->prof_enabled = saved_prof;
  free_lm_graphs(ctx);  // captured graphs carry the old launch shapes
  for (auto &g : ctx->outer_graph)
    if (g) {
      free_graph(g);
      g = nullptr;
    }
  RPBA_TRY(sync(ctx));
  if (chosen) {
    chosen[0] = ctx->tune.isect;
    chosen[1] = ctx->tune.lin;
    chosen[2] = ctx->tune.backsub;
    chosen[3] = ctx->tune.robust;
    chosen[4] = ctx->opt.chol_tc;
  }
  const char *path = cache_path ? cache_path : ctx->opt.tune_cache;
  if (path && *path) RPBA_TRY(tune_store(ctx, path));
  return RPBA_OK;
}

extern "C" rpba_status rpba_outer_iteration(rpba_ctx *h, int32_t robust, double *sigma0, int32_t *lm_launches) {
  CTX_KEEP_COSTS;
  if (!ctx->intersected) RPBA_TRY(rpba_intersect(h));
  int inner = 0, launches = 0;
  RPBA_TRY(run_bact(ctx, &inner, &launches));
  double s = 0.0;
  RPBA_TRY(outer_tail(ctx, robust != 0, &s));
  if (sigma0) *sigma0 = s;
  if (lm_launches) *lm_launches = launches;
  return RPBA_OK;
}

extern "C" rpba_status rpba_iterate(rpba_ctx *h, int32_t max_outer, rpba_report *rep) {
  CTX_OR_FAIL;
  const rpba_options &o = ctx->opt;
  if (max_outer <= 0) max_outer = o.max_outer;
  rpba_report r;
  memset(&r, 0, sizeof(r));
  r.robust_started_at = -1;
  if (!ctx->intersected) RPBA_TRY(rpba_intersect(h));
  double s = 0.0;
  RPBA_TRY(launch_sigma0(ctx, &s, nullptr));
  r.sigma0_initial = s;
  double best = s;
  int grace = o.grace;
  bool robust_on = false;
  for (int outer = 0; outer < max_outer; outer++) {
    RPBA_TRY(run_bact(ctx, &r.inner_total, &r.lm_launches));
    if (o.robust && o.robust_from_start && !robust_on) {
      robust_on = true;
      r.robust_started_at = r.outer;
    }
    RPBA_TRY(outer_tail(ctx, robust_on, &s));
    if (r.outer < 128) r.sigma0_hist[r.outer] = s;
    r.outer++;
    double ratio = best / (s > 1e-300 ? s : 1e-300);
    if (s < best) best = s;
    if (ratio < o.stop_ratio) {
      if (grace > 0) { grace--; continue; }
      if (o.robust && !robust_on) {
        robust_on = true;
        r.robust_started_at = r.outer;
        ctx->f0_valid = false;
        RPBA_TRY(launch_robust_weights(ctx, nullptr));
        RPBA_TRY(launch_intersect(ctx, 1, nullptr));
        RPBA_TRY(launch_tp_copies(ctx, 1));
        RPBA_TRY(launch_sigma0(ctx, &best, nullptr));
        grace = o.grace;
        continue;
      }
      break;
    }
  }
  if (robust_on) RPBA_TRY(launch_eliminate(ctx));
  // sigma_0, RMS and the active counts of the final state, all from one reduction
  long long ka = 0, na = 0;
  RPBA_TRY(launch_sigma0(ctx, &r.sigma0, &r.rms, &ka, &na));
  r.active_points = (int)na;
  r.deleted_points = ctx->n_active_start - (int)na;
  r.active_obs = (int)ka;
  if (rep) *rep = r;
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// profiling
// ---------------------------------------------------------------------------
extern "C" rpba_status rpba_profile_enable(rpba_ctx *h, int32_t enable) {
  CTX_KEEP_COSTS;
  RPBA_TRY(sync(ctx));
  for (auto &r : ctx->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->prof_recs.clear();
  ctx->prof_ms.clear();
  ctx->launch_by_name.clear();
  ctx->launches = 0;
  ctx->prof_enabled = enable != 0;
  return RPBA_OK;
}

extern "C" rpba_status rpba_profile_read(rpba_ctx *h, int32_t max_kernels, char *names, double *ms,
                                         int64_t *launches, int32_t *n_kernels, int64_t *total_launches) {
  CTX_KEEP_COSTS;
  RPBA_TRY(sync(ctx));
  for (auto &r : ctx->prof_recs) {
    float t = 0.f;
    RPBA_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ctx->prof_ms[r.name] += t;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->prof_recs.clear();
  int n = 0;
  for (auto &kv : ctx->launch_by_name) {
    if (n < max_kernels) {
      if (names) {
        strncpy(names + 48 * n, kv.first.c_str(), 47);
        names[48 * n + 47] = 0;
      }
      if (ms) ms[n] = ctx->prof_ms.count(kv.first) ? ctx->prof_ms[kv.first] : 0.0;
      if (launches) launches[n] = kv.second;
    }
    n++;
  }
  if (n_kernels) *n_kernels = n;
  if (total_launches) *total_launches = ctx->launches;
  return RPBA_OK;
}

extern "C" rpba_status rpba_solver_stats(rpba_ctx *h, int32_t *iters, double *relres) {
  CTX_KEEP_COSTS;
  if (!ctx->pcg_st) {
    ctx->err = "solver statistics exist for the PCG solvers only";
    return RPBA_ERR_STATE;
  }
  std::vector<double> st(4 * (size_t)ctx->L);
  if (ctx->L) RPBA_CUDA(cudaMemcpyAsync(st.data(), ctx->pcg_st, st.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  for (int l = 0; l < ctx->L; l++) {
    if (iters) iters[l] = (int32_t)st[4 * l + 3];
    if (relres) relres[l] = st[4 * l + 2];
  }
  return RPBA_OK;
}

extern "C" rpba_status rpba_solver_stages(rpba_ctx *h, int32_t *stages) {
  CTX_KEEP_COSTS;
  if (!stages) return RPBA_ERR_INVALID_ARG;
  if (!ff_pcg(ctx)) {
    for (int l = 0; l < ctx->L; l++) stages[l] = 0;
    return RPBA_OK;
  }
  std::vector<float> w((size_t)PCG_S32_WORDS * ctx->L);
  if (ctx->L)
    RPBA_CUDA(cudaMemcpyAsync(w.data(), ctx->pcg_s32, w.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_TRY(sync(ctx));
  for (int l = 0; l < ctx->L; l++) stages[l] = (int32_t)w[(size_t)PCG_S32_WORDS * l + PCG_S32_STAGES];
  return RPBA_OK;
}

extern "C" rpba_status rpba_solver_fallbacks(rpba_ctx *h, int64_t *n) {
  CTX_KEEP_COSTS;
  if (!n) return RPBA_ERR_INVALID_ARG;
  *n = ctx->gnn_fallbacks;
  return RPBA_OK;
}

extern "C" rpba_status rpba_profile_select(rpba_ctx *h, const char *kernel) {
  CTX_KEEP_COSTS;
  ctx->prof_only = kernel ? std::string(kernel) : std::string();
  return RPBA_OK;
}

__global__ void k_check_formats(const double *x, const float *f, int n, float *hi, float *lo, double *back,
                                double *fd) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (x) {
    float2 s = ff_split_bits(x[e]);
    hi[e] = s.x;
    lo[e] = s.y;
    back[e] = ff_to_double(s);
  }
  if (f) fd[e] = f2d(f[e]);
}

extern "C" rpba_status rpba_check_formats(const double *x, const float *f, int32_t n, float *hi, float *lo,
                                          double *back, double *fd) {
  if (n < 0 || ((hi || lo || back) && !x) || (fd && !f)) return RPBA_ERR_INVALID_ARG;
  if (n == 0) return RPBA_OK;
  bool wx = hi || lo || back, wf = fd != nullptr;
  char *buf = nullptr;
  size_t nb = (size_t)n * (wx ? 8 + 4 + 4 + 8 : 0) + (size_t)n * (wf ? 4 + 8 : 0);
  if (cudaMalloc((void **)&buf, nb) != cudaSuccess) return RPBA_ERR_OOM;
  char *c = buf;
  auto take = [&](size_t bytes) { char *p = c; c += bytes; return p; };
  double *dx = wx ? (double *)take(8 * (size_t)n) : nullptr, *dback = wx ? (double *)take(8 * (size_t)n) : nullptr;
  double *dfd = wf ? (double *)take(8 * (size_t)n) : nullptr;
  float *dhi = wx ? (float *)take(4 * (size_t)n) : nullptr, *dlo = wx ? (float *)take(4 * (size_t)n) : nullptr;
  float *df = wf ? (float *)take(4 * (size_t)n) : nullptr;
  cudaError_t e = cudaSuccess;
  if (wx && e == cudaSuccess) e = cudaMemcpy(dx, x, 8 * (size_t)n, cudaMemcpyHostToDevice);
  if (wf && e == cudaSuccess) e = cudaMemcpy(df, f, 4 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_check_formats<<<nblk(n, 256), 256>>>(dx, df, n, dhi, dlo, dback, dfd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && hi) e = cudaMemcpy(hi, dhi, 4 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && lo) e = cudaMemcpy(lo, dlo, 4 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && back) e = cudaMemcpy(back, dback, 8 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fd) e = cudaMemcpy(fd, dfd, 8 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  return e == cudaSuccess ? RPBA_OK : RPBA_ERR_CUDA;
}

extern "C" rpba_status rpba_get_options(rpba_ctx *h, rpba_options *out) {
  CTX_KEEP_COSTS;
  if (!out) return RPBA_ERR_INVALID_ARG;
  *out = ctx->opt;
  return RPBA_OK;
}
