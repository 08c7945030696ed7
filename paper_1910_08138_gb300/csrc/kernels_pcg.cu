// kernels_pcg.cu -- preconditioned conjugate gradients on the reduced camera
// systems S_l dC_l = y_l of all running sub-blocks at once (Sec. 5.5: the RCS
// is solved by CG with block-Jacobi preconditioning, i.e. the inverses of the
// diagonal camera blocks, 6x6 or 8x8 with per-camera intrinsics). FP64 vectors
// and FP64 matrix-vector products,
// so that the relative residual can reach 1e-8.
//
// Per iteration: k_pcg_symv (one CTA per 32x32 lower tile of every running
// sub-block, q += S p and p^T S p with FP64 atomics) and k_pcg_step (one CTA
// per sub-block: alpha = rz / p.Sp, x += alpha p, r -= alpha q, z = M^-1 r,
// beta = rz' / rz, p = z + beta p, convergence ||r|| <= tol ||y||). Two other
// step designs were slower: an 8-CTA cluster per sub-block (the 64-block
// workload's 304 small sub-blocks then need 2432 cluster CTAs) and three
// grid-wide kernels with one thread per camera (three launch latencies for
// ~1000 threads of work).
// The preconditioner is the inverse of the diagonal camera blocks
// (block-Jacobi), or the learned factorised inverse G^T G (solver 3).
//
// FP32 form, block-Jacobi: the same iteration without FP64 arithmetic in the
// loop. Once per solve the RCS is split into hi + lo float pairs (2^-48
// relative); the product S p runs in float-float on the FP32 pipes (TwoProduct
// and TwoSum per entry), x, r and p are float-float vectors, and the
// preconditioner is applied in FP32 (it needs no more). The product keeps
// ~1e-13 relative accuracy, far below the 1e-8 residual the loop stops at; on
// this GPU the FP64 pipe runs at 1/64 of the FP32 rate, so the FP64 loop is
// bound by its FP64 instructions and this one by memory and latency. The
// float-float step forms p.Sp itself (p . q), keeps its block sums in
// float-float, runs the scalar FP64 arithmetic in one thread and zeroes the q
// it has read; the product uses 128-thread CTAs (two threads per row and per
// column of a tile).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "rpba_internal.cuh"

namespace rpba {

#define PT 32
#define PLD (PT + 1)
#define PCG_THREADS 256  // per-sub-block kernels: one CTA

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// M_i^-1 for every camera of a running sub-block: inverse of S_ii (CD x CD,
// CD = 6, or 8 with per-camera intrinsics; FP64 Gauss-Jordan on the SPD
// block); stored row-major, CD^2 per camera
template <int CD>
__global__ void k_pcg_bj_setup(int M, const int *cam_sub, const int *cam_local, const int *sub_cam_ptr, const int *run,
                               const double *S, const long long *S_off, const int *npad, double *Minv, int *fail,
                               float *Minv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int l = cam_sub[i];
  if (!run[l]) return;
  int np = npad[l], li = cam_local[i];
  const double *A = S + S_off[l];
  double a[CD][2 * CD];
  for (int r = 0; r < CD; r++)
    for (int c = 0; c < CD; c++) {
      int rr = r >= c ? r : c, cc = r >= c ? c : r;  // lower triangle holds the block
      a[r][c] = A[(size_t)(CD * li + rr) * np + CD * li + cc];
      a[r][CD + c] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < CD; c++) {
    double piv = a[c][c];
    if (!(piv > 0.0)) {
      atomicExch(fail + l, 1);
      return;
    }
    double ip = 1.0 / piv;
    for (int e = 0; e < 2 * CD; e++) a[c][e] *= ip;
    for (int r = 0; r < CD; r++) {
      if (r == c) continue;
      double f = a[r][c];
      for (int e = 0; e < 2 * CD; e++) a[r][e] -= f * a[c][e];
    }
  }
  double *o = Minv + CD * CD * (size_t)(sub_cam_ptr[l] + li);  // cameras in sub-block order
  for (int r = 0; r < CD; r++)
    for (int c = 0; c < CD; c++) o[CD * r + c] = a[r][CD + c];
  if (Minv32) {
    float *o32 = Minv32 + CD * CD * (size_t)(sub_cam_ptr[l] + li);
    for (int r = 0; r < CD; r++)
      for (int c = 0; c < CD; c++) o32[CD * r + c] = (float)a[r][CD + c];
  }
}

// q += S p over the lower 32x32 tiles of the running, unconverged sub-blocks
__global__ void __launch_bounds__(256) k_pcg_symv(const double *S, const long long *S_off, const int *npad,
                                                  const int *voff, const int *live, const int *sched_tiles, int L,
                                                  const double *p, double *q, double *pq) {
  // CTA -> (sub-block, tile) through prefix sums of the per-sub-block tile counts
  int idx = blockIdx.x;
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sched_tiles[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  int l = lo;
  if (!live[l]) return;
  int loc = idx - sched_tiles[l];
  int a = (int)((sqrtf(8.0f * (float)loc + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= loc) a++;
  while (a * (a + 1) / 2 > loc) a--;
  int b = loc - a * (a + 1) / 2;
  int np = npad[l];
  const double *A = S + S_off[l];
  const double *pl = p + voff[l];
  double *ql = q + voff[l];
  __shared__ double blk[PT][PLD];
  __shared__ double pI[PT], pJ[PT];
  int tid = threadIdx.x;
  if (tid < PT) {
    pI[tid] = pl[a * PT + tid];
    pJ[tid] = pl[b * PT + tid];
  }
  for (int e = tid; e < PT * PT; e += blockDim.x) {
    int r = e / PT, c = e - r * PT;
    double v = A[(size_t)(a * PT + r) * np + b * PT + c];
    if (a == b && c > r) v = A[(size_t)(a * PT + c) * np + b * PT + r];
    blk[r][c] = v;
  }
  __syncthreads();
  if (tid < PT) {
    double s = 0.0;
    for (int c = 0; c < PT; c++) s += blk[tid][c] * pJ[c];
    atomicAdd(ql + a * PT + tid, s);
    // p^T S p: p_I^T S_IJ p_J, twice for an off-diagonal tile
    double t = pI[tid] * s * (a == b ? 1.0 : 2.0);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (tid == 0) atomicAdd(pq + l, t);
  } else if (tid < 2 * PT && a != b) {
    int c = tid - PT;
    double s = 0.0;
    for (int r = 0; r < PT; r++) s += blk[r][c] * pI[r];
    atomicAdd(ql + b * PT + c, s);
  }
}

template <int NV>
__device__ inline void cta_sum(double (&v)[NV], double (&out)[NV]) {
  __shared__ double sh[NV][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < NV; e++) {
    double x = v[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[e][wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < NV; e++) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[e][w];
    out[e] = s;
  }
  __syncthreads();
}

// CTA -> (sub-block l, lower tile (a, b)) through prefix sums of the
// per-sub-block tile counts
__device__ inline void tile_of(int idx, const int *sched_tiles, int L, int &l, int &a, int &b) {
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sched_tiles[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  l = lo;
  int loc = idx - sched_tiles[l];
  a = (int)((sqrtf(8.0f * (float)loc + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= loc) a++;
  while (a * (a + 1) / 2 > loc) a--;
  b = loc - a * (a + 1) / 2;
}

// FP32 form: the lower tiles of the live sub-blocks as hi + lo pairs
__global__ void __launch_bounds__(256) k_pcg_split(const double *S, const long long *S_off, const int *npad,
                                                   const int *live, const int *sched_tiles, int L, float2 *Sff) {
  int l, a, b;
  tile_of(blockIdx.x, sched_tiles, L, l, a, b);
  if (!live[l]) return;
  int np = npad[l];
  for (int e = threadIdx.x; e < PT * PT; e += blockDim.x) {
    int r = e / PT, c = e - r * PT;
    size_t idx = (size_t)S_off[l] + (size_t)(a * PT + r) * np + b * PT + c;
    Sff[idx] = ff_split_bits(S[idx]);
  }
}

// FP32 form: q += S p in float-float, summed over the tiles with FP64
// atomics. p^T S p is left to the step kernel (p . q over the sub-block):
// one atomic per tile on a single per-sub-block word serialises hundreds of
// CTAs. 128 threads: warps 0-1 form the row sums, warps 2-3 the column sums
// (off-diagonal tiles), two threads per row or column with 16 entries each.
#define SYMV_THREADS 128
__global__ void __launch_bounds__(SYMV_THREADS) k_pcg_symv_ff(const float2 *__restrict__ Sff, const long long *S_off,
                                                              const int *npad, const int *voff, const int *live,
                                                              const int *sched_tiles, int L,
                                                              const float2 *__restrict__ p, double *q) {
  int l, a, b;
  tile_of(blockIdx.x, sched_tiles, L, l, a, b);
  if (!live[l]) return;
  int np = npad[l];
  const float2 *A = Sff + S_off[l];
  const float2 *pl = p + voff[l];
  double *ql = q + voff[l];
  __shared__ float2 blk[PT][PLD];
  __shared__ float2 pI[PT], pJ[PT];
  int tid = threadIdx.x;
  if (tid < PT) pI[tid] = pl[a * PT + tid];
  else if (tid < 2 * PT) pJ[tid - PT] = pl[b * PT + tid - PT];
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    int e = tid + SYMV_THREADS * k, r = e / PT, c = e - r * PT;
    v[k] = (a == b && c > r) ? A[(size_t)(a * PT + c) * np + b * PT + r] : A[(size_t)(a * PT + r) * np + b * PT + c];
  }
#pragma unroll
  for (int k = 0; k < 8; k++) {
    int e = tid + SYMV_THREADS * k, r = e / PT, c = e - r * PT;
    blk[r][c] = v[k];
  }
  __syncthreads();
  bool col = tid >= 2 * PT;
  int u = tid & 63, t = u >> 1, h = u & 1;  // row (or column) t, entries 16h .. 16h+15
  if (col && a == b) return;                // the diagonal tile's columns are its rows
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int k = 16 * h; k < 16 * h + 16; k++) {
    float2 m = col ? blk[k][t] : blk[t][k];
    float2 x = col ? pI[k] : pJ[k];
    float e;
    float pr = ff_two_prod(m.x, x.x, e);
    ff_acc(sh, sl, pr);
    sl = __fadd_rn(sl, __fmaf_rn(m.y, x.x, __fmaf_rn(m.x, x.y, e)));
  }
  float oh = __shfl_xor_sync(0xffffffffu, sh, 1), ol = __shfl_xor_sync(0xffffffffu, sl, 1);
  float e;
  sh = ff_two_sum(sh, oh, e);
  sl = __fadd_rn(sl, __fadd_rn(e, ol));
  if (h == 0) atomicAdd(ql + (col ? b : a) * PT + t, ff_to_double(make_float2(sh, sl)));
}

// FP32 form start: x = 0, r = y, z = M^-1 r (FP32), p = z; rz, |y|
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_init_ff(const int *run, const int *fail, const int *sub_cam_ptr,
                                                             const int *voff, const int *npad, const float *Minv32,
                                                             const double *y, float2 *x, float2 *r, float *z,
                                                             float2 *p, double *st, int *live) {
  int l = blockIdx.x;
  int ok = run[l] && !fail[l];
  if (threadIdx.x == 0) {
    live[l] = ok;
    if (!ok) st[4 * l + 3] = 0.0;  // no iterations in this solve
  }
  if (!ok) return;
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = CD * ncam, o = voff[l];
  double v[2] = {0.0, 0.0};
  const float2 zero = make_float2(0.f, 0.f);
  for (int e = threadIdx.x; e < npad[l]; e += blockDim.x) {  // padding stays zero
    x[o + e] = zero;
    r[o + e] = e < n ? ff_split_bits(y[o + e]) : zero;
    z[o + e] = 0.f;
    p[o + e] = zero;
    if (e < n) v[1] += y[o + e] * y[o + e];
  }
  __syncthreads();
  float rzh = 0.f, rzl = 0.f;
  for (int c = threadIdx.x; c < ncam; c += blockDim.x) {
    const float *Mi = Minv32 + CD * CD * (size_t)(g0 + c);
    const float2 *rc = r + o + CD * c;
    for (int a = 0; a < CD; a++) {
      float t = 0.f;
      for (int b = 0; b < CD; b++) t += Mi[CD * a + b] * rc[b].x;
      z[o + CD * c + a] = t;
      p[o + CD * c + a] = make_float2(t, 0.f);
      float e;
      float pr = ff_two_prod(rc[a].x, t, e);
      ff_acc(rzh, rzl, pr);
      rzl = __fadd_rn(rzl, __fmaf_rn(rc[a].y, t, e));
    }
  }
  v[0] = (double)rzh + (double)rzl;
  double s[2];
  cta_sum<2>(v, s);
  if (threadIdx.x == 0) {
    st[4 * l + 0] = s[0];                    // rz
    st[4 * l + 1] = sqrt(s[1]);              // |y|
    st[4 * l + 2] = s[1] > 0.0 ? 1.0 : 0.0;  // relative residual
    st[4 * l + 3] = 0.0;                     // iterations
    if (!(s[1] > 0.0)) live[l] = 0;
  }
}

// float-float sum over a warp (lane 0 holds the result)
__device__ inline void ff_warp_sum(float &h, float &l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
    float e;
    h = ff_two_sum(h, oh, e);
    l = __fadd_rn(l, __fadd_rn(e, ol));
  }
}

// float-float sums of NV values over the CTA; thread 0 gets the totals (as
// doubles). sh: [NV][32] float2 scratch
template <int NV>
__device__ inline void ff_cta_sum(float (&h)[NV], float (&l)[NV], float2 (*sh)[32], double (&tot)[NV]) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    ff_warp_sum(h[k], l[k]);
    if (lane == 0) sh[k][wid] = make_float2(h[k], l[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; k++) {
      float2 t = sh[k][0];
      for (int w = 1; w < nw; w++) t = ff_add(t, sh[k][w]);
      tot[k] = ff_to_double(t);
    }
}

// FP32 form step: p.Sp = p.q, alpha = rz / p.Sp, x += alpha p, r -= alpha q
// (float-float), z = M^-1 r (FP32), rz' = r.z, beta = rz' / rz, p = z + beta p.
// Each thread loads all of its elements at once (up to PCGF_PER) so that each
// phase waits for one memory latency; r and z pass between the phases in
// shared memory. The block sums are float-float and the scalar FP64
// arithmetic (alpha, beta, the statistics) runs in thread 0 alone: on this GPU
// one SM's FP64 unit would serialise it across the block.
#define PCGF_PER 8
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_step_ff(const int *sub_cam_ptr, const int *voff,
                                                             const float *__restrict__ Minv32, double tol,
                                                             float2 *__restrict__ x, float2 *__restrict__ r,
                                                             float2 *__restrict__ p, double *__restrict__ q,
                                                             double *st, int *live) {
  extern __shared__ float2 rs[];  // r (n), then z as floats (n)
  __shared__ float2 red[2][32];
  __shared__ float2 bc;           // broadcast scalar (alpha, then beta) as a pair
  __shared__ int stop;
  int l = blockIdx.x;
  if (!live[l]) return;
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = CD * ncam, o = voff[l];
  float *zs = reinterpret_cast<float *>(rs + n);
  // the thread's inverse block, independent of this iteration's data
  constexpr int M4 = CD * CD / 4;
  float m[CD * CD];
  int c0 = threadIdx.x;
  if (c0 < ncam) {
    const float4 *Mi = reinterpret_cast<const float4 *>(Minv32 + CD * CD * (size_t)(g0 + c0));
#pragma unroll
    for (int k = 0; k < M4; k++) {
      float4 w = __ldg(Mi + k);
      m[4 * k] = w.x; m[4 * k + 1] = w.y; m[4 * k + 2] = w.z; m[4 * k + 3] = w.w;
    }
  }
  float2 pv[PCGF_PER], xv[PCGF_PER], rv[PCGF_PER], qv[PCGF_PER];
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) { pv[k] = p[o + e]; xv[k] = x[o + e]; rv[k] = r[o + e]; qv[k] = ff_split_bits(q[o + e]); }
  }
  // q is consumed: zero it for the next product (padding rows only ever get +0)
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) q[o + e] = 0.0;
  }
  float ph[1] = {0.f}, pl[1] = {0.f};  // p . q
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) {
      float er;
      float pr = ff_two_prod(pv[k].x, qv[k].x, er);
      ff_acc(ph[0], pl[0], pr);
      pl[0] = __fadd_rn(pl[0], __fmaf_rn(pv[k].y, qv[k].x, __fmaf_rn(pv[k].x, qv[k].y, er)));
    }
  }
  double pqt[1];
  ff_cta_sum<1>(ph, pl, red, pqt);
  if (threadIdx.x == 0) {
    stop = !(pqt[0] > 0.0);  // breakdown: keep the current iterate
    if (stop) live[l] = 0;
    else bc = ff_of(st[4 * l] / pqt[0]);
  }
  __syncthreads();
  if (stop) return;
  float2 af = bc, naf = make_float2(-af.x, -af.y);
  float rr = 0.f;
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) {
      x[o + e] = ff_add(xv[k], ff_mul(af, pv[k]));
      float2 re = ff_add(rv[k], ff_mul(naf, qv[k]));
      r[o + e] = re;
      rs[e] = re;
      rr += re.x * re.x;
    }
  }
  __syncthreads();
  float vh[2] = {rr, 0.f}, vl[2] = {0.f, 0.f};  // r.r (FP32 is enough for the test), r.z
  for (int c = threadIdx.x; c < ncam; c += PCG_THREADS) {
    if (c != c0) {  // more cameras than threads: load this block too
      const float4 *Mi = reinterpret_cast<const float4 *>(Minv32 + CD * CD * (size_t)(g0 + c));
#pragma unroll
      for (int k = 0; k < M4; k++) {
        float4 w = __ldg(Mi + k);
        m[4 * k] = w.x; m[4 * k + 1] = w.y; m[4 * k + 2] = w.z; m[4 * k + 3] = w.w;
      }
    }
    float rh[CD], rl[CD];
#pragma unroll
    for (int b2 = 0; b2 < CD; b2++) { rh[b2] = rs[CD * c + b2].x; rl[b2] = rs[CD * c + b2].y; }
#pragma unroll
    for (int a2 = 0; a2 < CD; a2++) {
      float t = 0.f;
#pragma unroll
      for (int b2 = 0; b2 < CD; b2++) t += m[CD * a2 + b2] * rh[b2];
      zs[CD * c + a2] = t;
      float e;
      float pr = ff_two_prod(rh[a2], t, e);
      ff_acc(vh[1], vl[1], pr);
      vl[1] = __fadd_rn(vl[1], __fmaf_rn(rl[a2], t, e));
    }
  }
  double tot[2];
  ff_cta_sum<2>(vh, vl, red, tot);  // its barrier also orders the z writes before the reads below
  if (threadIdx.x == 0) {
    bc = ff_of(tot[1] / st[4 * l]);
    st[4 * l] = tot[1];
    double rel = sqrt(tot[0]) / st[4 * l + 1];
    st[4 * l + 2] = rel;
    st[4 * l + 3] += 1.0;
    if (rel <= tol) live[l] = 0;
  }
  __syncthreads();
  float2 bf = bc;
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) p[o + e] = ff_add(make_float2(zs[e], 0.f), ff_mul(bf, pv[k]));
  }
}

// FP32 form: dC = x
__global__ void k_pcg_out_ff(const int *run, const int *fail, const int *voff, const int *npad, int L,
                             const float2 *x, double *dC) {
  int l = blockIdx.y;
  if (l >= L || !run[l] || fail[l]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npad[l]; e += gridDim.x * blockDim.x)
    dC[voff[l] + e] = ff_to_double(x[voff[l] + e]);
}

// z = M^-1 r for the cameras of sub-block l (block rows of CD)
template <int CD>
__device__ inline void apply_precond(int n_cam, const double *Minv_l, const double *r, double *z) {
  for (int c = threadIdx.x; c < n_cam; c += blockDim.x) {
    const double *Mi = Minv_l + CD * CD * (size_t)c;
    for (int a = 0; a < CD; a++) {
      double s = 0.0;
      for (int b = 0; b < CD; b++) s += Mi[CD * a + b] * r[CD * c + b];
      z[CD * c + a] = s;
    }
  }
}

// start: x = 0, r = y, z = M^-1 r, p = z; rz, |y|
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_init(const int *run, const int *fail, const int *sub_cam_ptr,
                                                  const int *voff, const int *npad, const double *Minv_sub,
                                                  const double *y, double *x, double *r, double *z, double *p,
                                                  double *st, int *live) {
  int l = blockIdx.x;
  int ok = run[l] && !fail[l];
  if (threadIdx.x == 0) {
    live[l] = ok;
    if (!ok) st[4 * l + 3] = 0.0;  // no iterations in this solve
  }
  if (!ok) return;
  int ncam = sub_cam_ptr[l + 1] - sub_cam_ptr[l];
  int n = CD * ncam;
  int o = voff[l];
  for (int e = threadIdx.x; e < npad[l]; e += blockDim.x) {  // padding stays zero
    x[o + e] = 0.0;
    r[o + e] = e < n ? y[o + e] : 0.0;
    z[o + e] = 0.0;
    p[o + e] = 0.0;
  }
  __syncthreads();
  apply_precond<CD>(ncam, Minv_sub + CD * CD * (size_t)sub_cam_ptr[l], r + o, z + o);
  __syncthreads();
  double v[2] = {0.0, 0.0};
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    p[o + e] = z[o + e];
    v[0] += r[o + e] * z[o + e];
    v[1] += y[o + e] * y[o + e];
  }
  double s[2];
  cta_sum<2>(v, s);
  if (threadIdx.x == 0) {
    st[4 * l + 0] = s[0];               // rz
    st[4 * l + 1] = sqrt(s[1]);         // |y|
    st[4 * l + 2] = s[1] > 0.0 ? 1.0 : 0.0;  // relative residual
    st[4 * l + 3] = 0.0;                // iterations
    if (!(s[1] > 0.0)) live[l] = 0;
  }
}

// ---- learned preconditioner: the PCG step split around a grid-wide apply ----
// start without the preconditioner: x = 0, r = y, z = p = 0, |y|
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_init_a(const int *run, const int *fail, const int *sub_cam_ptr,
                                                    const int *voff, const int *npad, const double *y, double *x,
                                                    double *r, double *z, double *p, double *st, int *live) {
  int l = blockIdx.x;
  int ok = run[l] && !fail[l];
  if (threadIdx.x == 0) {
    live[l] = ok;
    if (!ok) st[4 * l + 3] = 0.0;  // no iterations in this solve
  }
  if (!ok) return;
  int n = 6 * (sub_cam_ptr[l + 1] - sub_cam_ptr[l]);
  int o = voff[l];
  double v1[1] = {0.0};
  for (int e = threadIdx.x; e < npad[l]; e += blockDim.x) {
    x[o + e] = 0.0;
    r[o + e] = e < n ? y[o + e] : 0.0;
    z[o + e] = 0.0;
    p[o + e] = 0.0;
    if (e < n) v1[0] += y[o + e] * y[o + e];
  }
  double s[1];
  cta_sum<1>(v1, s);
  if (threadIdx.x == 0) {
    st[4 * l + 1] = sqrt(s[0]);
    st[4 * l + 2] = s[0] > 0.0 ? 1.0 : 0.0;
    st[4 * l + 3] = 0.0;
    if (!(s[0] > 0.0)) live[l] = 0;
  }
}

// after z = M^-1 r: p = z, rz
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_init_b(const int *sub_cam_ptr, const int *voff, const double *r,
                                                    const double *z, double *p, double *st, const int *live) {
  int l = blockIdx.x;
  if (!live[l]) return;
  int n = 6 * (sub_cam_ptr[l + 1] - sub_cam_ptr[l]);
  int o = voff[l];
  double v1[1] = {0.0};
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    p[o + e] = z[o + e];
    v1[0] += r[o + e] * z[o + e];
  }
  double s[1];
  cta_sum<1>(v1, s);
  if (threadIdx.x == 0) st[4 * l] = s[0];
}

// z = G^T G r over the cameras of the live sub-blocks, in FP32: three passes,
// the neighbour sums with one warp per camera (lanes split its graph entries).
// Per camera g: vector offset nvo[g]; rh and y hold 6 floats per camera.
__global__ void k_fsai_p1(int M, const int *node_sys, const int *live, const int *nvo, FsaiView P, const double *r,
                          float *rh) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M || (live && !live[node_sys[g]])) return;
  const float *A = P.Li + 36 * (size_t)g;
  const double *rg = r + nvo[g];
  float rc[6];
  for (int b = 0; b < 6; b++) rc[b] = (float)rg[b];
  for (int a = 0; a < 6; a++) {
    float t = 0.f;
    for (int b = 0; b <= a; b++) t += A[6 * a + b] * rc[b];
    rh[6 * (size_t)g + a] = t;
  }
}

__global__ void k_fsai_p2(int M, const int *node_sys, const int *live, const int *nvo, FsaiView P, const double *r,
                          const float *rh, float *y) {
  int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= M || (live && !live[node_sys[v]])) return;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = P.ptr[v] + lane; e < P.ptr[v + 1]; e += 32) {
    int u = P.adj[e];
    if (u >= v) continue;
    const float *Fe = P.F + 36 * (size_t)e;
    float x[6];
    for (int b = 0; b < 6; b++) x[b] = rh[6 * (size_t)u + b];
    for (int a = 0; a < 6; a++) {
      float t = 0.f;
      for (int b = 0; b < 6; b++) t += Fe[6 * a + b] * x[b];
      acc[a] += t;
    }
  }
  for (int a = 0; a < 6; a++)
    for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_down_sync(0xffffffffu, acc[a], o);
  if (lane == 0) {
    const float *A = P.D + 36 * (size_t)v;
    const double *rv = r + nvo[v];
    for (int a = 0; a < 6; a++) {
      float t = 0.f;
      for (int b = 0; b <= a; b++) t += A[6 * a + b] * (float)rv[b];
      y[6 * (size_t)v + a] = t - acc[a];
    }
  }
}

__global__ void k_fsai_p3(int M, const int *node_sys, const int *live, const int *nvo, FsaiView P, const float *y,
                          double *z) {
  int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= M || (live && !live[node_sys[v]])) return;
  float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = P.ptr[v] + lane; e < P.ptr[v + 1]; e += 32) {
    int u = P.adj[e];
    if (u <= v) continue;
    const float *Fe = P.F + 36 * (size_t)P.mir[e];
    float x[6];
    for (int a = 0; a < 6; a++) x[a] = y[6 * (size_t)u + a];
    for (int b = 0; b < 6; b++) {
      float t = 0.f;
      for (int a = 0; a < 6; a++) t += Fe[6 * a + b] * x[a];
      w[b] += t;
    }
  }
  for (int b = 0; b < 6; b++)
    for (int o = 16; o > 0; o >>= 1) w[b] += __shfl_down_sync(0xffffffffu, w[b], o);
  if (lane == 0) {
    const float *A = P.D + 36 * (size_t)v, *B = P.Li + 36 * (size_t)v;
    const float *yv = y + 6 * (size_t)v;
    double *zv = z + nvo[v];
    for (int b = 0; b < 6; b++) {
      float t = 0.f;
      for (int a = b; a < 6; a++) t += A[6 * a + b] * yv[a] - B[6 * a + b] * w[a];
      zv[b] = (double)t;
    }
  }
}

rpba_status fsai_apply(Ctx *ctx, const FsaiApply &F, const int *live, const double *r, double *z, bool skip_first) {
  int M = F.M;
  if (M == 0) return RPBA_OK;
  cudaStream_t st = ctx ? ctx->stream : F.stream;
  auto launch = [&](const char *name, auto fn) -> rpba_status {
    if (ctx) {
      RPBA_KERNEL(ctx, name, fn());
      return RPBA_OK;
    }
    fn();
    return cudaGetLastError() == cudaSuccess ? RPBA_OK : RPBA_ERR_CUDA;
  };
  if (!skip_first)
    RPBA_TRY(launch("k_fsai_p1", [&] {
      k_fsai_p1<<<nblk(M, 128), 128, 0, st>>>(M, F.node_sys, live, F.nvo, F.P, r, F.rh);
    }));
  RPBA_TRY(launch("k_fsai_p2", [&] {
    k_fsai_p2<<<nblk(32LL * M, 256), 256, 0, st>>>(M, F.node_sys, live, F.nvo, F.P, r, F.rh, F.y);
  }));
  RPBA_TRY(launch("k_fsai_p3", [&] {
    k_fsai_p3<<<nblk(32LL * M, 256), 256, 0, st>>>(M, F.node_sys, live, F.nvo, F.P, F.y, z);
  }));
  return RPBA_OK;
}

// ---- the CG step, one CTA per sub-block ----
// block-Jacobi step: alpha = rz / p.Sp, x += alpha p, r -= alpha q, z = M^-1 r,
// beta = rz' / rz, p = z + beta p, convergence ||r|| <= tol ||y||
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_step(const int *sub_cam_ptr, const int *voff,
                                                          const double *Minv_sub, double tol, double *x, double *r,
                                                          double *z, double *p, const double *q, const double *pq,
                                                          double *st, int *live) {
  int l = blockIdx.x;
  if (!live[l]) return;
  double rz_old = st[4 * l], pql = pq[l];
  if (!(pql > 0.0)) {  // breakdown: keep the current iterate
    if (threadIdx.x == 0) live[l] = 0;
    return;
  }
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = CD * ncam, o = voff[l];
  double alpha = rz_old / pql;
  double v[2] = {0.0, 0.0};
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    x[o + e] += alpha * p[o + e];
    double re = r[o + e] - alpha * q[o + e];
    r[o + e] = re;
    v[0] += re * re;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncam; c += blockDim.x) {
    const double *Mi = Minv_sub + CD * CD * (size_t)(g0 + c);
    const double *rc = r + o + CD * c;
    double *zc = z + o + CD * c;
    for (int a = 0; a < CD; a++) {
      double t = 0.0;
      for (int b = 0; b < CD; b++) t += Mi[CD * a + b] * rc[b];
      zc[a] = t;
      v[1] += rc[a] * t;
    }
  }
  double tot[2];
  cta_sum<2>(v, tot);
  double beta = tot[1] / rz_old;
  for (int e = threadIdx.x; e < n; e += blockDim.x) p[o + e] = z[o + e] + beta * p[o + e];
  if (threadIdx.x == 0) {
    st[4 * l] = tot[1];
    double rel = sqrt(tot[0]) / st[4 * l + 1];
    st[4 * l + 2] = rel;
    st[4 * l + 3] += 1.0;
    if (rel <= tol) live[l] = 0;
  }
}

// learned form, first half: alpha, x, r, ||r||, then rh = L^-1 r for the
// sub-block's cameras (the first pass of the factor's application)
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_alpha(const int *sub_cam_ptr, const int *voff, double tol,
                                                           double *x, double *r, const double *p, const double *q,
                                                           const double *pq, double *st, int *live, const float *Li,
                                                           float *rh) {
  int l = blockIdx.x;
  if (!live[l]) return;
  double rz_old = st[4 * l], pql = pq[l];
  if (!(pql > 0.0)) {
    if (threadIdx.x == 0) live[l] = 0;
    return;
  }
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = 6 * ncam, o = voff[l];
  double alpha = rz_old / pql;
  double v[1] = {0.0};
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    x[o + e] += alpha * p[o + e];
    double re = r[o + e] - alpha * q[o + e];
    r[o + e] = re;
    v[0] += re * re;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncam; c += blockDim.x) {
    const float *A = Li + 36 * (size_t)(g0 + c);
    const double *rc = r + o + 6 * c;
    float rf[6];
    for (int b = 0; b < 6; b++) rf[b] = (float)rc[b];
    for (int a = 0; a < 6; a++) {
      float t = 0.f;
      for (int b = 0; b <= a; b++) t += A[6 * a + b] * rf[b];
      rh[6 * (size_t)(g0 + c) + a] = t;
    }
  }
  double tot[1];
  cta_sum<1>(v, tot);
  if (threadIdx.x == 0) {
    double rel = sqrt(tot[0]) / st[4 * l + 1];
    st[4 * l + 2] = rel;
    st[4 * l + 3] += 1.0;
    if (rel <= tol) live[l] = 0;
  }
}

// learned form, second half (after z = M^-1 r): beta = rz' / rz, p = z + beta p
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_beta(const int *sub_cam_ptr, const int *voff, const double *r,
                                                          const double *z, double *p, double *st, const int *live) {
  int l = blockIdx.x;
  if (!live[l]) return;
  int n = 6 * (sub_cam_ptr[l + 1] - sub_cam_ptr[l]);
  int o = voff[l];
  double v[1] = {0.0};
  for (int e = threadIdx.x; e < n; e += blockDim.x) v[0] += r[o + e] * z[o + e];
  double tot[1];
  cta_sum<1>(v, tot);
  double beta = tot[0] / st[4 * l];
  for (int e = threadIdx.x; e < n; e += blockDim.x) p[o + e] = z[o + e] + beta * p[o + e];
  if (threadIdx.x == 0) st[4 * l] = tot[0];
}

// dC = x
__global__ void k_pcg_out(const int *run, const int *fail, const int *voff, const int *npad, int L, const double *x,
                          double *dC) {
  int l = blockIdx.y;
  if (l >= L || !run[l] || fail[l]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npad[l]; e += gridDim.x * blockDim.x)
    dC[voff[l] + e] = x[voff[l] + e];  // padding of x is zero
}

// count[0] = unconverged sub-blocks, count[1] = the most CG iterations any ran
__global__ void k_pcg_live_count(int L, const int *live, const double *st, int *count) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  if (live[l]) atomicAdd(count, 1);
  atomicMax(count + 1, (int)st[4 * l + 3]);
}

// The phases of a PCG solve, with the preconditioner set up by the caller:
// the inverse blocks in ctx->pcg_Minv (block-Jacobi, one fused step kernel
// per iteration), or the learned factor when fsai is given (the step split
// around the grid-wide apply). The loop stops per sub-block at the relative
// residual pcg_tol or after pcg_max_iter; it reads the count of unconverged
// sub-blocks every 8 iterations, so it runs outside any captured graph.
rpba_status pcg_init(Ctx *ctx, const int *run_dev, int *fail_dev, const FsaiApply *fsai) {
  int L = ctx->L;
  cudaStream_t st = ctx->stream;
  if (!fsai && ff_pcg(ctx)) {
    RPBA_CUDA(cudaMemsetAsync(ctx->pcg_q, 0, ctx->ytot * sizeof(double), st));
    auto init_ff = ctx->cd == 8 ? k_pcg_init_ff<8> : k_pcg_init_ff<6>;
    RPBA_KERNEL(ctx, "k_pcg_init_ff", init_ff<<<L, PCG_THREADS, 0, st>>>(
                                       run_dev, fail_dev, ctx->sub_cam_ptr, ctx->ycam_off, ctx->npad, ctx->pcg_Minv32,
                                       ctx->y, ctx->pcg_fx, ctx->pcg_fr, ctx->pcg_fz, ctx->pcg_fp, ctx->pcg_st,
                                       ctx->pcg_live));
    if (ctx->pcg_tiles_total)
      RPBA_KERNEL(ctx, "k_pcg_split", k_pcg_split<<<ctx->pcg_tiles_total, 256, 0, st>>>(
                                          ctx->S, ctx->S_off, ctx->npad, ctx->pcg_live, ctx->pcg_tiles, L,
                                          ctx->pcg_Sff));
    return RPBA_OK;
  }
  if (fsai) {
    RPBA_KERNEL(ctx, "k_pcg_init_a", k_pcg_init_a<<<L, PCG_THREADS, 0, st>>>(run_dev, fail_dev, ctx->sub_cam_ptr, ctx->ycam_off,
                                                                    ctx->npad, ctx->y, ctx->pcg_x, ctx->pcg_r,
                                                                    ctx->pcg_z, ctx->pcg_p, ctx->pcg_st,
                                                                    ctx->pcg_live));
    RPBA_TRY(fsai_apply(ctx, *fsai, ctx->pcg_live, ctx->pcg_r, ctx->pcg_z));
    RPBA_KERNEL(ctx, "k_pcg_init_b", k_pcg_init_b<<<L, PCG_THREADS, 0, st>>>(ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_r,
                                                                    ctx->pcg_z, ctx->pcg_p, ctx->pcg_st,
                                                                    ctx->pcg_live));
  } else {
    auto init = ctx->cd == 8 ? k_pcg_init<8> : k_pcg_init<6>;
    RPBA_KERNEL(ctx, "k_pcg_init", init<<<L, PCG_THREADS, 0, st>>>(
                                       run_dev, fail_dev, ctx->sub_cam_ptr, ctx->ycam_off, ctx->npad, ctx->pcg_Minv,
                                       ctx->y, ctx->pcg_x, ctx->pcg_r, ctx->pcg_z, ctx->pcg_p, ctx->pcg_st,
                                       ctx->pcg_live));
  }
  return RPBA_OK;
}

rpba_status pcg_loop(Ctx *ctx, const FsaiApply *fsai, int *iters) {
  int L = ctx->L;
  if (iters) *iters = 0;
  cudaStream_t st = ctx->stream;
  int tiles = ctx->pcg_tiles_total;
  int maxit = ctx->opt.pcg_max_iter;
  // the first convergence read after as many iterations as the previous solve
  // took (launches for converged sub-blocks return at once), then every 8
  int next_check = std::min(maxit, std::max(8, ctx->pcg_pred));
  auto step_ff = ctx->cd == 8 ? k_pcg_step_ff<8> : k_pcg_step_ff<6>;
  auto step64 = ctx->cd == 8 ? k_pcg_step<8> : k_pcg_step<6>;
  for (int it = 0; it < maxit; it++) {
    if (!fsai && ff_pcg(ctx)) {  // q starts at zero (init) and the step zeroes what it consumed
      RPBA_KERNEL(ctx, "k_pcg_symv_ff", k_pcg_symv_ff<<<tiles, SYMV_THREADS, 0, st>>>(
                                         ctx->pcg_Sff, ctx->S_off, ctx->npad, ctx->ycam_off, ctx->pcg_live,
                                         ctx->pcg_tiles, L, ctx->pcg_fp, ctx->pcg_q));
      RPBA_KERNEL(ctx, "k_pcg_step_ff", step_ff<<<L, PCG_THREADS, ctx->pcg_ff_smem, st>>>(
                                         ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_Minv32, ctx->opt.pcg_tol,
                                         ctx->pcg_fx, ctx->pcg_fr, ctx->pcg_fp, ctx->pcg_q, ctx->pcg_st,
                                         ctx->pcg_live));
    } else {
      RPBA_CUDA(cudaMemsetAsync(ctx->pcg_q, 0, ctx->ytot * sizeof(double), st));
      RPBA_CUDA(cudaMemsetAsync(ctx->pcg_pq, 0, L * sizeof(double), st));
      RPBA_KERNEL(ctx, "k_pcg_symv", k_pcg_symv<<<tiles, 256, 0, st>>>(
                                         ctx->S, ctx->S_off, ctx->npad, ctx->ycam_off, ctx->pcg_live, ctx->pcg_tiles,
                                         L, ctx->pcg_p, ctx->pcg_q, ctx->pcg_pq));
      if (fsai) {
        RPBA_KERNEL(ctx, "k_pcg_alpha", k_pcg_alpha<<<L, PCG_THREADS, 0, st>>>(
                                            ctx->sub_cam_ptr, ctx->ycam_off, ctx->opt.pcg_tol, ctx->pcg_x,
                                            ctx->pcg_r, ctx->pcg_p, ctx->pcg_q, ctx->pcg_pq, ctx->pcg_st,
                                            ctx->pcg_live, fsai->P.Li, fsai->rh));
        RPBA_TRY(fsai_apply(ctx, *fsai, ctx->pcg_live, ctx->pcg_r, ctx->pcg_z, /*skip_first=*/true));
        RPBA_KERNEL(ctx, "k_pcg_beta", k_pcg_beta<<<L, PCG_THREADS, 0, st>>>(
                                           ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_r, ctx->pcg_z, ctx->pcg_p,
                                           ctx->pcg_st, ctx->pcg_live));
      } else {
        RPBA_KERNEL(ctx, "k_pcg_step", step64<<<L, PCG_THREADS, 0, st>>>(
                                           ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_Minv, ctx->opt.pcg_tol,
                                           ctx->pcg_x, ctx->pcg_r, ctx->pcg_z, ctx->pcg_p, ctx->pcg_q, ctx->pcg_pq,
                                           ctx->pcg_st, ctx->pcg_live));
      }
    }
    if (it + 1 == next_check || it == maxit - 1) {
      RPBA_CUDA(cudaMemsetAsync(ctx->counters + 8, 0, 2 * sizeof(int), st));
      RPBA_KERNEL(ctx, "k_pcg_live_count", k_pcg_live_count<<<nblk(L, 128), 128, 0, st>>>(
                                               L, ctx->pcg_live, ctx->pcg_st, ctx->counters + 8));
      RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter + 8, ctx->counters + 8, 2 * sizeof(int),
                                cudaMemcpyDeviceToHost, st));
      RPBA_CUDA(cudaStreamSynchronize(st));
      int ran = ctx->h_pinned_counter[9];  // iterations of the slowest sub-block so far
      if (iters) *iters = ran;
      if (ctx->h_pinned_counter[8] == 0) {
        ctx->pcg_pred = ran;
        break;
      }
      next_check = it + 1 + 8;
    }
  }
  return RPBA_OK;
}

rpba_status pcg_out(Ctx *ctx, const int *run_dev, const int *fail_dev) {
  int L = ctx->L;
  if (ff_pcg(ctx)) {
    RPBA_KERNEL(ctx, "k_pcg_out_ff", k_pcg_out_ff<<<dim3(8, L), 256, 0, ctx->stream>>>(
                                      run_dev, fail_dev, ctx->ycam_off, ctx->npad, L, ctx->pcg_fx, ctx->dC));
    return RPBA_OK;
  }
  RPBA_KERNEL(ctx, "k_pcg_out", k_pcg_out<<<dim3(8, L), 256, 0, ctx->stream>>>(run_dev, fail_dev, ctx->ycam_off,
                                                                              ctx->npad, L, ctx->pcg_x, ctx->dC));
  return RPBA_OK;
}

rpba_status pcg_iterate(Ctx *ctx, const int *run_dev, int *fail_dev, const FsaiApply *fsai) {
  RPBA_TRY(pcg_init(ctx, run_dev, fail_dev, fsai));
  RPBA_TRY(pcg_loop(ctx, fsai, nullptr));
  return pcg_out(ctx, run_dev, fail_dev);
}

// block-Jacobi: the inverse camera blocks (failure flags reset first)
rpba_status pcg_bj_setup(Ctx *ctx, const int *run_dev, int *fail_dev) {
  RPBA_CUDA(cudaMemsetAsync(fail_dev, 0, ctx->L * sizeof(int), ctx->stream));
  if (ctx->M)
    RPBA_KERNEL(ctx, "k_pcg_bj_setup", (ctx->cd == 8 ? k_pcg_bj_setup<8> : k_pcg_bj_setup<6>)<<<nblk(ctx->M, 128), 128, 0, ctx->stream>>>(
                                           ctx->M, ctx->cam_sub, ctx->cam_local, ctx->sub_cam_ptr, run_dev, ctx->S,
                                           ctx->S_off, ctx->npad, ctx->pcg_Minv, fail_dev,
                                           ff_pcg(ctx) ? ctx->pcg_Minv32 : nullptr));
  return RPBA_OK;
}

rpba_status launch_pcg_blockjacobi(Ctx *ctx, const int *run_dev, int *fail_dev) {
  RPBA_TRY(pcg_bj_setup(ctx, run_dev, fail_dev));
  return pcg_iterate(ctx, run_dev, fail_dev, nullptr);
}

}  // namespace rpba
