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
// FP32 form, block-Jacobi: mixed-precision refinement around FP32 CG. Once
// per solve the RCS is split into a hi plane (S rounded to FP32) and a lo
// plane (hi + lo = S to 2^-48 relative). A stage runs FP32 CG on
// S_hi d = r, with r the current residual rounded to FP32, until
// ||r_k|| <= 1e-4 ||r_0|| (k_pcg_symv32 reads 4 B per stored entry, one warp
// per tile with plain FMAs; k_pcg_step32 is the FP32 step); then
// X += d in float-float and the true residual R = y - S X is formed in
// float-float from both planes (k_pcg_symv_ff, TwoProduct and TwoSum per
// entry, ~1e-13 relative) by k_pcg_stage, which ends the solve at
// ||R|| <= pcg_tol ||y|| or starts the next stage. The entrywise rounding of
// S_hi is a relative perturbation of 2^-24, so a stage reduces the residual
// by about max(1e-4, 2^-24 cond) with cond the condition of the Jacobi-scaled
// RCS; at the benchmark sizes two stages reach 1e-8. The CG steps thus read
// half the bytes and run no float-float arithmetic, and the stopping test is
// on the float-float true residual, not on a recurrence.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>

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

// Per-sub-block words of the FP32 form's refinement (PCG_S32_WORDS floats
// each): rz, the stage's ||r_0|| and tolerance, the last relative true
// residual, the stage count, a bound on max |p|, the exponent of the
// fixed-point product and max |S_hi| (as float bits, for atomicMax)
#define PCG_S32 PCG_S32_WORDS
enum {
  S32_RZ = 0, S32_RN0 = 1, S32_TOL = 2, S32_PREV = 3, S32_STAGES = PCG_S32_STAGES, S32_PMAX = 5, S32_QEXP = 6,
  S32_SMAX = 7
};

// FP32 form: the lower tiles of the running sub-blocks as hi + lo floats, in
// two planes with the layout of S (hi: S rounded to 24 bits; hi + lo: S to
// 2^-48 relative), and max |S_hi| per sub-block (its word zeroed before). One
// warp per tile (lane c: column c, one 256-byte row load per step), the warps
// striding over the tile table.
__global__ void __launch_bounds__(256) k_pcg_split(const double *__restrict__ S, const long long *S_off,
                                                   const int *npad, const int *run, const int *fail,
                                                   const int2 *__restrict__ tile_map, int tiles, float *Shi,
                                                   float *Slo, float *s32) {
  int lane = threadIdx.x & 31;
  int nw = gridDim.x * (blockDim.x >> 5);
  for (int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); idx < tiles; idx += nw) {
    int2 tm = tile_map[idx];
    int l = tm.x, a = tm.y >> 16, b = tm.y & 0xffff;
    if (!run[l] || fail[l]) continue;  // the same for the whole warp
    int np = npad[l];
    size_t base = (size_t)S_off[l] + (size_t)(a * PT) * np + b * PT + lane;
    double v[PT];
#pragma unroll
    for (int r = 0; r < PT; r++) v[r] = __ldg(S + base + (size_t)r * np);
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < PT; r++) {
      float2 h = ff_split_bits(v[r]);
      Shi[base + (size_t)r * np] = h.x;
      Slo[base + (size_t)r * np] = h.y;
      mx = fmaxf(mx, fabsf(h.x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) atomicMax(reinterpret_cast<int *>(s32 + PCG_S32 * l + S32_SMAX), __float_as_int(mx));
  }
}

// Exponent s of the FP32 form's fixed-point product: every partial sum of
// S_hi p (and their total) is below np max|S_hi| max|p| < 2^61 2^-s, so the
// partials scaled by 2^s fit 64-bit integers, whose sums are exact and do not
// depend on the order of the atomics. Computed from the exponents alone.
__device__ inline int fixed_exp(int np, float smax, float pmax) {
  if (!(smax > 0.f) || !(pmax > 0.f) || isinf(smax) || isinf(pmax)) return 0;
  int e1, e2, e3;
  frexpf((float)np, &e1);
  frexpf(smax, &e2);
  frexpf(pmax, &e3);
  return 61 - (e1 + e2 + e3);
}

// FP32 form, refinement residual: q += S (X + dx) in float-float over the
// lower tiles of the active sub-blocks (X float-float, dx the FP32 solution of
// the stage just ended), summed over the tiles with FP64 atomics. One warp per
// tile, the warps striding over the tile table (as k_pcg_symv32): lane c reads
// column c's hi and lo words one row at a time, accumulates the transposed
// product in float-float and keeps the 32 row terms (hi, lo); a transposing
// butterfly of float-float additions leaves row r's sum in lane r.
#define SYMV_THREADS 256
__device__ __forceinline__ float2 warp_transpose_sum_ff(float (&th)[PT], float (&tl)[PT], int lane) {
#pragma unroll
  for (int o = PT / 2; o >= 1; o >>= 1) {
    bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      float sh = up ? th[i] : th[i + o], sl = up ? tl[i] : tl[i + o];
      float kh = up ? th[i + o] : th[i], kl = up ? tl[i + o] : tl[i];
      float2 r = ff_add(make_float2(kh, kl),
                        make_float2(__shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o)));
      th[i] = r.x;
      tl[i] = r.y;
    }
  }
  return make_float2(th[0], tl[0]);
}

__global__ void __launch_bounds__(SYMV_THREADS) k_pcg_symv_ff(const float *__restrict__ Shi,
                                                              const float *__restrict__ Slo, const long long *S_off,
                                                              const int *npad, const int *voff, const int *act,
                                                              const int2 *__restrict__ tile_map, int tiles,
                                                              const float2 *__restrict__ X,
                                                              const float *__restrict__ dx, double *q) {
  int lane = threadIdx.x & 31;
  int nw = gridDim.x * (SYMV_THREADS / 32);
  for (int idx = blockIdx.x * (SYMV_THREADS / 32) + (threadIdx.x >> 5); idx < tiles; idx += nw) {
    int2 tm = tile_map[idx];
    int l = tm.x, a = tm.y >> 16, b = tm.y & 0xffff;
    if (!act[l]) continue;  // the same for the whole warp
    int np = npad[l];
    size_t base = (size_t)S_off[l] + (size_t)(a * PT) * np + b * PT + lane;
    const float2 *Xl = X + voff[l];
    const float *dxl = dx + voff[l];
    float2 pI = ff_add(Xl[a * PT + lane], make_float2(dxl[a * PT + lane], 0.f));
    float2 pJ = ff_add(Xl[b * PT + lane], make_float2(dxl[b * PT + lane], 0.f));
    float th[PT], tl[PT];
#pragma unroll
    for (int r = 0; r < PT; r++) {
      th[r] = __ldg(Shi + base + (size_t)r * np);
      tl[r] = __ldg(Slo + base + (size_t)r * np);
    }
    float2 col = make_float2(0.f, 0.f);
    const bool diag = a == b;
#pragma unroll
    for (int r = 0; r < PT; r++) {
      float2 m = make_float2(th[r], tl[r]);
      if (diag && lane > r) m = make_float2(0.f, 0.f);  // row r, columns 0 .. r
      float2 pr = make_float2(__shfl_sync(0xffffffffu, pI.x, r), __shfl_sync(0xffffffffu, pI.y, r));
      if (!diag || lane < r) col = ff_add(col, ff_mul(m, pr));
      float2 t = ff_mul(m, pJ);
      th[r] = t.x;
      tl[r] = t.y;
    }
    float2 row = warp_transpose_sum_ff(th, tl, lane);
    double *ql = q + voff[l];
    if (!diag) {
      atomicAdd(ql + a * PT + lane, ff_to_double(row));
      atomicAdd(ql + b * PT + lane, ff_to_double(col));
    } else {
      atomicAdd(ql + a * PT + lane, ff_to_double(ff_add(row, col)));
    }
  }
}

// Sums over the warp's lanes of 32 values at once: on return lane i holds
// the sum over all lanes of t[i]. Five halving exchange steps (16 + 8 + 4 + 2
// + 1 shuffles): at the step of width o a lane keeps the half of its values
// whose index has bit o equal to its own lane bit o, sends the other half to
// lane ^ o and adds what it receives.
__device__ __forceinline__ float warp_transpose_sum(float (&t)[PT], int lane) {
#pragma unroll
  for (int o = PT / 2; o >= 1; o >>= 1) {
    bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; i++) {
      float send = up ? t[i] : t[i + o];
      float keep = up ? t[i + o] : t[i];
      t[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return t[0];
}

// FP32 form, inner CG product: q += S_hi p over the lower tiles of the live
// sub-blocks, one warp per tile and no shared memory. Lane c reads column c
// of the tile one row at a time (each load a 128-byte row of the warp), adds
// S_rc p_I[r] to the transposed product in a register and keeps the 32 row
// terms S_rc p_J[c]; warp_transpose_sum leaves row r's sum in lane r. On a
// diagonal tile only the entries on and below the diagonal are used. The two
// sums of a lane (formed in a fixed order) are added to q as 64-bit fixed-point
// integers (scale 2^s, fixed_exp), so q does not depend on the order of the
// atomics and two runs give the same CG iterates.
// one tile (one warp): tm = (sub-block, a << 16 | b)
__device__ __forceinline__ void symv32_tile(const float *__restrict__ Shi, const long long *S_off, const int *npad,
                                            const int *voff, const int *live, int2 tm,
                                            const float *__restrict__ s32, const float *__restrict__ p,
                                            unsigned long long *q, int lane) {
  int l = tm.x, a = tm.y >> 16, b = tm.y & 0xffff;
  if (!live[l]) return;
  int np = npad[l];
  int sc = (int)s32[PCG_S32 * l + S32_QEXP];
  const float *A = Shi + S_off[l] + (size_t)(a * PT) * np + b * PT + lane;
  const float *pl = p + voff[l];
  float pIc = pl[a * PT + lane], pJc = pl[b * PT + lane];
  float t[PT];
#pragma unroll
  for (int r = 0; r < PT; r++) t[r] = __ldg(A + (size_t)r * np);
  float col = 0.f;
  if (a != b) {
#pragma unroll
    for (int r = 0; r < PT; r++) {
      col = __fmaf_rn(t[r], __shfl_sync(0xffffffffu, pIc, r), col);
      t[r] = __fmul_rn(t[r], pJc);
    }
  } else {
#pragma unroll
    for (int r = 0; r < PT; r++) {
      float m = lane <= r ? t[r] : 0.f;  // row r, columns 0 .. r
      col = __fmaf_rn(lane < r ? m : 0.f, __shfl_sync(0xffffffffu, pIc, r), col);
      t[r] = __fmul_rn(m, pJc);
    }
  }
  float row = warp_transpose_sum(t, lane);
  unsigned long long *ql = q + voff[l];
  long long vr = __float2ll_rn(scalbnf(row, sc)), vc = __float2ll_rn(scalbnf(col, sc));
  if (a != b) {
    atomicAdd(ql + a * PT + lane, (unsigned long long)vr);
    atomicAdd(ql + b * PT + lane, (unsigned long long)vc);
  } else {
    atomicAdd(ql + a * PT + lane, (unsigned long long)(vr + vc));
  }
}

// The warps stride over the tiles (a grid of a few CTAs per SM), each tile's
// sub-block and position read from a table (tile_map) in one load.
#define SYMV32_WARPS 8
__global__ void __launch_bounds__(32 * SYMV32_WARPS) k_pcg_symv32(const float *__restrict__ Shi,
                                                                  const long long *S_off, const int *npad,
                                                                  const int *voff, const int *live,
                                                                  const int2 *__restrict__ tile_map, int tiles,
                                                                  const float *__restrict__ s32,
                                                                  const float *__restrict__ p,
                                                                  unsigned long long *q) {
  int lane = threadIdx.x & 31;
  int nw = gridDim.x * SYMV32_WARPS;
  for (int idx = blockIdx.x * SYMV32_WARPS + (threadIdx.x >> 5); idx < tiles; idx += nw)
    symv32_tile(Shi, S_off, npad, voff, live, tile_map[idx], s32, p, q, lane);
}

// four CTAs of eight warps per SM (152 SMs), or one warp per tile if fewer
static inline int symv32_grid(int tiles) { return std::max(1, std::min(nblk(tiles, SYMV32_WARPS), 4 * 152)); }

// q[e] (fixed point, scale 2^s) as a float
__device__ __forceinline__ float fixed_to_float(unsigned long long v, int sc) {
  return scalbnf(__ll2float_rn((long long)v), -sc);
}

// FP32 sums of NV values over the CTA; every thread gets the totals
template <int NV>
__device__ inline void f_cta_sum(float (&v)[NV], float (&out)[NV]) {
  __shared__ float sh[NV][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; k++) {
    float s = 0.f;
    for (int w = 0; w < nw; w++) s += sh[k][w];
    out[k] = s;
  }
  __syncthreads();
}


// FP32 sums of NV values and the maximum of one more over the CTA; every
// thread gets the results
template <int NV>
__device__ inline void f_cta_sum_max(float (&v)[NV], float m, float (&out)[NV], float &mout) {
  __shared__ float sh[NV + 1][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][wid] = x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) sh[NV][wid] = m;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; k++) {
    float t = 0.f;
    for (int w = 0; w < nw; w++) t += sh[k][w];
    out[k] = t;
  }
  float mm = 0.f;
  for (int w = 0; w < nw; w++) mm = fmaxf(mm, sh[NV][w]);
  mout = mm;
  __syncthreads();
}

// FP32 form: start of a refinement stage, one CTA per active sub-block.
// first: X = 0 and R = y (every running sub-block becomes active); otherwise
// X += x, the FP32 solution of the stage just ended, and R = y - q with
// q = S X from k_pcg_symv_ff (q is zeroed once read). The solve of the
// sub-block ends when ||R|| <= tol ||y||, when a stage has not halved ||R||,
// after max_stage stages, or at the CG step cap (final set, or the device
// loop's step count loop_cnt[0] at max_iter);
// otherwise the FP32 CG restarts on S_hi d = R rounded to FP32: x = 0,
// z = M^-1 r, p = z, stopping at ||r|| <= max(tol_in, 0.3 tol ||y|| / ||R||)
// ||R||. st[4l + 2] is the relative true residual ||R|| / ||y||.
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_stage(
    int first, int final_stage, const int *loop_cnt, int max_iter, const int *run, const int *fail,
    const int *sub_cam_ptr, const int *voff,
    const int *npad, const float *__restrict__ Minv32, const double *__restrict__ y, double *qd, float2 *X,
    float *x, float *r, float *z, float *p, unsigned long long *q, double *st, float *s32, int *act, int *live,
    double tol, double tol_in, int max_stage) {
  __shared__ int stop;
  int l = blockIdx.x;
  int stage;
  if (first) {
    int ok = run[l] && !fail[l];
    if (threadIdx.x == 0) {
      act[l] = ok;
      live[l] = 0;
      st[4 * l + 3] = 0.0;  // CG iterations of this solve
      st[4 * l + 2] = ok ? 1.0 : 0.0;
      s32[PCG_S32 * l + S32_STAGES] = 0.f;
    }
    if (!ok) return;
    stage = 0;
  } else {
    stage = act[l];
    if (!stage) return;
  }
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = CD * ncam, o = voff[l], np = npad[l];
  float rr = 0.f;             // ||R||^2: FP32 terms and per-thread sums, FP64 across the CTA
  double v[2] = {0.0, 0.0};  // ||R||^2, ||y||^2
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    float re = 0.f;
    if (e < n) {
      float2 yf = ff_split_bits(y[o + e]);
      float2 R = yf;
      if (first) {
        X[o + e] = make_float2(0.f, 0.f);
        v[1] += y[o + e] * y[o + e];
      } else {
        X[o + e] = ff_add(X[o + e], make_float2(x[o + e], 0.f));
        float2 qf = ff_split_bits(qd[o + e]);
        R = ff_add(yf, make_float2(-qf.x, -qf.y));
      }
      rr = __fmaf_rn(R.x, R.x, rr);
      re = R.x;
    } else if (first) {
      X[o + e] = make_float2(0.f, 0.f);
    }
    qd[o + e] = 0.0;
    r[o + e] = re;
    x[o + e] = 0.f;
    z[o + e] = 0.f;
    p[o + e] = 0.f;
    q[o + e] = 0ull;
  }
  v[0] = f2d(rr);
  double s[2];
  cta_sum<2>(v, s);  // its barriers also order the r writes before the reads below
  if (threadIdx.x == 0) {
    double ny = first ? sqrt(s[1]) : st[4 * l + 1];
    double nr = sqrt(s[0]);
    double rel = ny > 0.0 ? nr / ny : 0.0;
    if (first) st[4 * l + 1] = ny;
    st[4 * l + 2] = rel;
    float *w = s32 + PCG_S32 * l;
    bool fin = final_stage || (loop_cnt && loop_cnt[0] >= max_iter);
    bool done = !(ny > 0.0) || rel <= tol || fin || stage >= max_stage ||
                (!first && !(rel <= 0.5 * (double)w[S32_PREV]));
    if (done) {
      act[l] = 0;
      live[l] = 0;
    } else {
      act[l] = stage + 1;
      live[l] = 1;
      w[S32_RN0] = (float)nr;
      w[S32_TOL] = (float)fmax(tol_in, 0.3 * tol / rel);
      w[S32_PREV] = (float)rel;
      w[S32_STAGES] = (float)(stage + 1);
    }
    stop = done;
  }
  __syncthreads();
  if (stop) return;
  float rz = 0.f, zmax = 0.f;
  for (int c = threadIdx.x; c < ncam; c += blockDim.x) {
    const float *Mi = Minv32 + CD * CD * (size_t)(g0 + c);
    const float *rc = r + o + CD * c;
    float rl[CD];
#pragma unroll
    for (int b = 0; b < CD; b++) rl[b] = rc[b];
#pragma unroll
    for (int a = 0; a < CD; a++) {
      float t = 0.f;
#pragma unroll
      for (int b = 0; b < CD; b++) t = __fmaf_rn(Mi[CD * a + b], rl[b], t);
      z[o + CD * c + a] = t;
      p[o + CD * c + a] = t;
      rz = __fmaf_rn(rl[a], t, rz);
      zmax = fmaxf(zmax, fabsf(t));
    }
  }
  float v1[1] = {rz}, t1[1], pmax;
  f_cta_sum_max<1>(v1, zmax, t1, pmax);
  if (threadIdx.x == 0) {
    float *w = s32 + PCG_S32 * l;
    w[S32_RZ] = t1[0];
    w[S32_PMAX] = pmax;
    w[S32_QEXP] = (float)fixed_exp(np, w[S32_SMAX], pmax);
  }
}

// FP32 form, inner CG step of a refinement stage (one CTA per live
// sub-block): alpha = rz / p.q, x += alpha p, r -= alpha q, z = M^-1 r,
// beta = r.z / rz, p = z + beta p; the stage ends when ||r|| <= tol_s ||r_0||.
// FP32 throughout, block sums included (the stage needs ~1e-4 of its right-hand
// side; the refinement's float-float residual corrects the rest). Each thread
// loads all of its elements at once (up to PCGF_PER) so that each phase waits
// for one memory latency; r and z pass between the phases in shared memory;
// q is zeroed once read.
#define PCGF_PER 8
template <int CD>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_step32(const int *sub_cam_ptr, const int *voff,
                                                            const float *__restrict__ Minv32,
                                                            const int *npad, float *__restrict__ x,
                                                            float *__restrict__ r, float *__restrict__ p,
                                                            unsigned long long *__restrict__ q, double *st,
                                                            float *s32, int *live) {
  extern __shared__ float rzs[];  // r (n), then z (n)
  int l = blockIdx.x;
  if (!live[l]) return;
  int g0 = sub_cam_ptr[l], ncam = sub_cam_ptr[l + 1] - g0;
  int n = CD * ncam, o = voff[l];
  float *rs = rzs, *zs = rzs + n;
  float *w = s32 + PCG_S32 * l;
  float rz_old = w[S32_RZ], rn0 = w[S32_RN0], tol_s = w[S32_TOL], pmax_old = w[S32_PMAX];
  int sc = (int)w[S32_QEXP];
  constexpr int M4 = CD * CD / 4;
  float m[CD * CD];
  int c0 = threadIdx.x;
  if (c0 < ncam) {
    const float4 *Mi = reinterpret_cast<const float4 *>(Minv32 + CD * CD * (size_t)(g0 + c0));
#pragma unroll
    for (int k = 0; k < M4; k++) {
      float4 u = __ldg(Mi + k);
      m[4 * k] = u.x; m[4 * k + 1] = u.y; m[4 * k + 2] = u.z; m[4 * k + 3] = u.w;
    }
  }
  float pv[PCGF_PER], xv[PCGF_PER], rv[PCGF_PER], qv[PCGF_PER];
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) { pv[k] = p[o + e]; xv[k] = x[o + e]; rv[k] = r[o + e]; qv[k] = fixed_to_float(q[o + e], sc); }
  }
  float pq = 0.f;
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) {
      q[o + e] = 0ull;
      pq = __fmaf_rn(pv[k], qv[k], pq);
    }
  }
  float v1[1] = {pq}, t1[1];
  f_cta_sum<1>(v1, t1);
  if (!(t1[0] > 0.f)) {  // breakdown: the stage keeps its current iterate
    if (threadIdx.x == 0) live[l] = 0;
    return;
  }
  float alpha = rz_old / t1[0];
  float rr = 0.f;
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) {
      x[o + e] = __fmaf_rn(alpha, pv[k], xv[k]);
      float re = __fmaf_rn(-alpha, qv[k], rv[k]);
      r[o + e] = re;
      rs[e] = re;
      rr = __fmaf_rn(re, re, rr);
    }
  }
  __syncthreads();
  float rz = 0.f, zmax = 0.f;
  for (int c = threadIdx.x; c < ncam; c += PCG_THREADS) {
    if (c != c0) {  // more cameras than threads: load this block too
      const float4 *Mi = reinterpret_cast<const float4 *>(Minv32 + CD * CD * (size_t)(g0 + c));
#pragma unroll
      for (int k = 0; k < M4; k++) {
        float4 u = __ldg(Mi + k);
        m[4 * k] = u.x; m[4 * k + 1] = u.y; m[4 * k + 2] = u.z; m[4 * k + 3] = u.w;
      }
    }
    float rl[CD];
#pragma unroll
    for (int b2 = 0; b2 < CD; b2++) rl[b2] = rs[CD * c + b2];
#pragma unroll
    for (int a2 = 0; a2 < CD; a2++) {
      float t = 0.f;
#pragma unroll
      for (int b2 = 0; b2 < CD; b2++) t = __fmaf_rn(m[CD * a2 + b2], rl[b2], t);
      zs[CD * c + a2] = t;
      rz = __fmaf_rn(rl[a2], t, rz);
      zmax = fmaxf(zmax, fabsf(t));
    }
  }
  float v2[2] = {rr, rz}, t2[2], zm;
  f_cta_sum_max<2>(v2, zmax, t2, zm);  // its barrier also orders the z writes before the reads below
  float beta = t2[1] / rz_old;
  if (threadIdx.x == 0) {
    w[S32_RZ] = t2[1];
    // max |z + beta p| <= max |z| + |beta| max |p|: the next product's scale
    float pmax = zm + fabsf(beta) * pmax_old;
    w[S32_PMAX] = pmax;
    w[S32_QEXP] = (float)fixed_exp(npad[l], w[S32_SMAX], pmax);
    st[4 * l + 3] += 1.0;
    if (sqrtf(t2[0]) <= tol_s * rn0) live[l] = 0;
  }
#pragma unroll
  for (int k = 0; k < PCGF_PER; k++) {
    int e = threadIdx.x + k * PCG_THREADS;
    if (e < n) p[o + e] = __fmaf_rn(beta, pv[k], zs[e]);
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
    RPBA_CUDA(cudaMemsetAsync(ctx->pcg_s32, 0, (size_t)PCG_S32_WORDS * L * sizeof(float), st));
    if (ctx->pcg_tiles_total)
      RPBA_KERNEL(ctx, "k_pcg_split", k_pcg_split<<<symv32_grid(ctx->pcg_tiles_total), 256, 0, st>>>(
                                          ctx->S, ctx->S_off, ctx->npad, run_dev, fail_dev, ctx->pcg_tile_map,
                                          ctx->pcg_tiles_total, ctx->pcg_Shi, ctx->pcg_Slo, ctx->pcg_s32));
    auto stage = ctx->cd == 8 ? k_pcg_stage<8> : k_pcg_stage<6>;
    RPBA_KERNEL(ctx, "k_pcg_stage", stage<<<L, PCG_THREADS, 0, st>>>(
                                        1, 0, nullptr, 0, run_dev, fail_dev, ctx->sub_cam_ptr, ctx->ycam_off,
                                        ctx->npad,
                                        ctx->pcg_Minv32, ctx->y, ctx->pcg_q, ctx->pcg_fx, ctx->pcg_x32, ctx->pcg_r32,
                                        ctx->pcg_z32, ctx->pcg_p32, ctx->pcg_qi, ctx->pcg_st, ctx->pcg_s32,
                                        ctx->pcg_act, ctx->pcg_live, ctx->opt.pcg_tol, RPBA_PCG_INNER_TOL,
                                        RPBA_PCG_MAX_STAGES));
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

// count[0] = sub-blocks whose flag is set, count[1] = the most CG iterations
// any ran; read on the host (synchronising the stream)
static rpba_status pcg_read_count(Ctx *ctx, const int *flags, int *n_set, int *ran) {
  cudaStream_t st = ctx->stream;
  RPBA_CUDA(cudaMemsetAsync(ctx->counters + 8, 0, 2 * sizeof(int), st));
  RPBA_KERNEL(ctx, "k_pcg_live_count", k_pcg_live_count<<<nblk(ctx->L, 128), 128, 0, st>>>(
                                           ctx->L, flags, ctx->pcg_st, ctx->counters + 8));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter + 8, ctx->counters + 8, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                            st));
  RPBA_CUDA(cudaStreamSynchronize(st));
  *n_set = ctx->h_pinned_counter[8];
  *ran = ctx->h_pinned_counter[9];
  return RPBA_OK;
}

// FP32 form: the stages of the refinement after k_pcg_stage's start. Per
// stage, FP32 CG steps (k_pcg_symv32 + k_pcg_step32) until no sub-block is
// live, then the float-float residual (k_pcg_symv_ff + k_pcg_stage), which
// ends the solve of a sub-block or starts its next stage. The live count is
// read after as many steps as the same stage took in the previous solve,
// then every 4; the active count after every stage. pcg_max_iter caps the CG
// steps of all stages together.
static rpba_status pcg_loop_refined(Ctx *ctx, int *iters) {
  int L = ctx->L;
  cudaStream_t st = ctx->stream;
  int tiles = ctx->pcg_tiles_total;
  int maxit = ctx->opt.pcg_max_iter;
  auto step32 = ctx->cd == 8 ? k_pcg_step32<8> : k_pcg_step32<6>;
  auto stage_k = ctx->cd == 8 ? k_pcg_stage<8> : k_pcg_stage<6>;
  int it = 0, ran = 0;
  for (int stage = 0; stage < RPBA_PCG_MAX_STAGES; stage++) {
    int it0 = it;
    int next_check = std::min(maxit, it + std::max(2, ctx->pcg_pred_stage[stage]));
    for (; it < maxit; it++) {
      RPBA_KERNEL(ctx, "k_pcg_symv32", k_pcg_symv32<<<symv32_grid(tiles), 32 * SYMV32_WARPS, 0, st>>>(
                                           ctx->pcg_Shi, ctx->S_off, ctx->npad, ctx->ycam_off, ctx->pcg_live,
                                           ctx->pcg_tile_map, tiles, ctx->pcg_s32, ctx->pcg_p32, ctx->pcg_qi));
      RPBA_KERNEL(ctx, "k_pcg_step32", step32<<<L, PCG_THREADS, ctx->pcg_ff_smem, st>>>(
                                           ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_Minv32, ctx->npad,
                                           ctx->pcg_x32, ctx->pcg_r32, ctx->pcg_p32, ctx->pcg_qi, ctx->pcg_st,
                                           ctx->pcg_s32, ctx->pcg_live));
      if (it + 1 == next_check || it == maxit - 1) {
        int n_live;
        RPBA_TRY(pcg_read_count(ctx, ctx->pcg_live, &n_live, &ran));
        if (n_live == 0) {
          it++;
          break;
        }
        next_check = std::min(maxit, it + 1 + 4);
      }
    }
    ctx->pcg_pred_stage[stage] = it - it0;
    bool last = it >= maxit || stage + 1 == RPBA_PCG_MAX_STAGES;
    RPBA_KERNEL(ctx, "k_pcg_symv_ff", k_pcg_symv_ff<<<symv32_grid(tiles), SYMV_THREADS, 0, st>>>(
                                          ctx->pcg_Shi, ctx->pcg_Slo, ctx->S_off, ctx->npad, ctx->ycam_off,
                                          ctx->pcg_act, ctx->pcg_tile_map, tiles, ctx->pcg_fx, ctx->pcg_x32,
                                          ctx->pcg_q));
    RPBA_KERNEL(ctx, "k_pcg_stage", stage_k<<<L, PCG_THREADS, 0, st>>>(
                                        0, last ? 1 : 0, nullptr, 0, nullptr, nullptr, ctx->sub_cam_ptr, ctx->ycam_off,
                                        ctx->npad, ctx->pcg_Minv32, ctx->y, ctx->pcg_q, ctx->pcg_fx, ctx->pcg_x32,
                                        ctx->pcg_r32, ctx->pcg_z32, ctx->pcg_p32, ctx->pcg_qi, ctx->pcg_st,
                                        ctx->pcg_s32, ctx->pcg_act, ctx->pcg_live, ctx->opt.pcg_tol,
                                        RPBA_PCG_INNER_TOL, RPBA_PCG_MAX_STAGES));
    int n_act;
    RPBA_TRY(pcg_read_count(ctx, ctx->pcg_act, &n_act, &ran));
    if (n_act == 0) break;
  }
  if (iters) *iters = ran;
  return RPBA_OK;
}

// Condition of a while node of the device-driven loop: some sub-block's flag
// set and the loop's counter below its limit; inc first adds one to the
// counter (the body's last kernel counts the pass it ends). The counters
// bound both loops whatever the flags do: at most max_iter CG steps in all
// and RPBA_PCG_MAX_STAGES stages.
__global__ void __launch_bounds__(256) k_pcg_cond(cudaGraphConditionalHandle h, int L, const int *flags, int *cnt,
                                                  int inc, int limit) {
  int any = 0;
  for (int l = threadIdx.x; l < L; l += blockDim.x) any |= flags[l] != 0;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    int c = *cnt + inc;
    *cnt = c;
    cudaGraphSetConditional(h, (any && c < limit) ? 1u : 0u);
  }
}

static bool pcg_loop_kernel(const std::string &n) {
  return n == "k_pcg_symv32" || n == "k_pcg_step32" || n == "k_pcg_cond" || n == "k_pcg_symv_ff" ||
         n == "k_pcg_stage";
}

bool pcg_device_loop(const Ctx *ctx) {
  if (!ff_pcg(ctx) || ctx->pcg_no_device_loop || !ctx->pcg_body_stream[0] || !ctx->pcg_body_stream[1])
    return false;
  // conditional bodies take no event-record nodes: a loop kernel that is
  // being timed runs in the host-driven loop
  return !(ctx->prof_enabled && (ctx->prof_only.empty() || pcg_loop_kernel(ctx->prof_only)));
}

// a while node after the work captured so far on st, with its handle; the
// node's body graph is returned for capture
static rpba_status add_while(Ctx *ctx, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t *body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  RPBA_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) {
    ctx->err = "PCG loop: stream not capturing";
    return RPBA_ERR_CUDA;
  }
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};  // the other fields zero
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  RPBA_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  *body = p.conditional.phGraph_out[0];
  RPBA_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return RPBA_OK;
}

static rpba_status handle_for(Ctx *ctx, cudaStream_t st, cudaGraphConditionalHandle *h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  RPBA_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  RPBA_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, 0));
  return RPBA_OK;
}

// capture fn's launches on stream bs into body, always ending the capture
template <class F>
static rpba_status capture_body(Ctx *ctx, cudaStream_t bs, cudaGraph_t body, std::vector<const char *> *names, F fn) {
  RPBA_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  std::vector<const char *> *prev = ctx->capture_list;
  ctx->capture_list = names;
  rpba_status st = fn();
  ctx->capture_list = prev;
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(bs, &out);  // out is body, owned by its node
  if (st != RPBA_OK) return st;
  RPBA_CUDA(e);
  return RPBA_OK;
}

// FP32 form, the refinement loop inside the graph being captured on the
// context's stream: a while node over the stages whose body holds a while
// node over the CG steps, so a solve needs no host read. The step and stage
// counts go to pinned memory (counters PCG_LOOP_COUNTERS, +1) for the launch
// count and solver 4's switch, read after the step's synchronisation.
static rpba_status pcg_loop_device(Ctx *ctx) {
  int L = ctx->L;
  cudaStream_t st = ctx->stream, bo = ctx->pcg_body_stream[0], bi = ctx->pcg_body_stream[1];
  int tiles = ctx->pcg_tiles_total;
  int maxit = ctx->opt.pcg_max_iter;
  int *cnt = ctx->counters + PCG_LOOP_COUNTERS;  // [0] CG steps, [1] stages
  auto step32 = ctx->cd == 8 ? k_pcg_step32<8> : k_pcg_step32<6>;
  auto stage_k = ctx->cd == 8 ? k_pcg_stage<8> : k_pcg_stage<6>;
  GraphRec *g = ctx->capture;
  g->pcg_loop = true;
  RPBA_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st));
  cudaGraphConditionalHandle h_out, h_in;
  RPBA_TRY(handle_for(ctx, st, &h_out));
  RPBA_KERNEL(ctx, "k_pcg_cond", k_pcg_cond<<<1, 256, 0, st>>>(h_out, L, ctx->pcg_act, cnt + 1, 0,
                                                                  RPBA_PCG_MAX_STAGES));
  cudaGraph_t body_out, body_in;
  RPBA_TRY(add_while(ctx, st, h_out, &body_out));
  RPBA_TRY(capture_body(ctx, bo, body_out, &g->loop_outer, [&]() -> rpba_status {
    RPBA_TRY(handle_for(ctx, bo, &h_in));
    RPBA_KERNEL(ctx, "k_pcg_cond", k_pcg_cond<<<1, 256, 0, bo>>>(h_in, L, ctx->pcg_live, cnt, 0, maxit));
    RPBA_TRY(add_while(ctx, bo, h_in, &body_in));
    RPBA_TRY(capture_body(ctx, bi, body_in, &g->loop_inner, [&]() -> rpba_status {
      RPBA_KERNEL(ctx, "k_pcg_symv32", k_pcg_symv32<<<symv32_grid(tiles), 32 * SYMV32_WARPS, 0, bi>>>(
                                           ctx->pcg_Shi, ctx->S_off, ctx->npad, ctx->ycam_off, ctx->pcg_live,
                                           ctx->pcg_tile_map, tiles, ctx->pcg_s32, ctx->pcg_p32, ctx->pcg_qi));
      RPBA_KERNEL(ctx, "k_pcg_step32", step32<<<L, PCG_THREADS, ctx->pcg_ff_smem, bi>>>(
                                           ctx->sub_cam_ptr, ctx->ycam_off, ctx->pcg_Minv32, ctx->npad,
                                           ctx->pcg_x32, ctx->pcg_r32, ctx->pcg_p32, ctx->pcg_qi, ctx->pcg_st,
                                           ctx->pcg_s32, ctx->pcg_live));
      RPBA_KERNEL(ctx, "k_pcg_cond", k_pcg_cond<<<1, 256, 0, bi>>>(h_in, L, ctx->pcg_live, cnt, 1, maxit));
      return RPBA_OK;
    }));
    RPBA_KERNEL(ctx, "k_pcg_symv_ff", k_pcg_symv_ff<<<symv32_grid(tiles), SYMV_THREADS, 0, bo>>>(
                                          ctx->pcg_Shi, ctx->pcg_Slo, ctx->S_off, ctx->npad, ctx->ycam_off,
                                          ctx->pcg_act, ctx->pcg_tile_map, tiles, ctx->pcg_fx, ctx->pcg_x32,
                                          ctx->pcg_q));
    RPBA_KERNEL(ctx, "k_pcg_stage", stage_k<<<L, PCG_THREADS, 0, bo>>>(
                                        0, 0, cnt, maxit, nullptr, nullptr, ctx->sub_cam_ptr, ctx->ycam_off,
                                        ctx->npad, ctx->pcg_Minv32, ctx->y, ctx->pcg_q, ctx->pcg_fx, ctx->pcg_x32,
                                        ctx->pcg_r32, ctx->pcg_z32, ctx->pcg_p32, ctx->pcg_qi, ctx->pcg_st,
                                        ctx->pcg_s32, ctx->pcg_act, ctx->pcg_live, ctx->opt.pcg_tol,
                                        RPBA_PCG_INNER_TOL, RPBA_PCG_MAX_STAGES));
    RPBA_KERNEL(ctx, "k_pcg_cond", k_pcg_cond<<<1, 256, 0, bo>>>(h_out, L, ctx->pcg_act, cnt + 1, 1,
                                                                    RPBA_PCG_MAX_STAGES));
    return RPBA_OK;
  }));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter + PCG_LOOP_COUNTERS, cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                            st));
  return RPBA_OK;
}

rpba_status pcg_loop(Ctx *ctx, const FsaiApply *fsai, int *iters) {
  if (!fsai && ff_pcg(ctx)) {
    if (ctx->capture && pcg_device_loop(ctx)) {
      if (iters) *iters = 0;  // known after the replay (pinned counters)
      return pcg_loop_device(ctx);
    }
    return pcg_loop_refined(ctx, iters);
  }
  int L = ctx->L;
  if (iters) *iters = 0;
  cudaStream_t st = ctx->stream;
  int tiles = ctx->pcg_tiles_total;
  int maxit = ctx->opt.pcg_max_iter;
  // the first convergence read after as many iterations as the previous solve
  // took (launches for converged sub-blocks return at once), then every 8
  int next_check = std::min(maxit, std::max(8, ctx->pcg_pred));
  auto step64 = ctx->cd == 8 ? k_pcg_step<8> : k_pcg_step<6>;
  for (int it = 0; it < maxit; it++) {
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
    if (it + 1 == next_check || it == maxit - 1) {
      int n_live, ran;  // ran: iterations of the slowest sub-block so far
      RPBA_TRY(pcg_read_count(ctx, ctx->pcg_live, &n_live, &ran));
      if (iters) *iters = ran;
      if (n_live == 0) {
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
