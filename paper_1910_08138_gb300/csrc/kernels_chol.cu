// kernels_chol.cu -- solve of the reduced camera systems S_l dC_l = y_l of all
// running sub-blocks at once (Sec. 2: Cholesky factorisation of the RCS).
//
// Layout: each S_l is dense, row-major, padded to n_pad = 32 * tiles with the
// identity on the padding; only the lower triangle is read.
//
// Blocked right-looking Cholesky with 32 x 32 tiles, batched over sub-blocks
// of different sizes, templated on the arithmetic type T:
//   k_chol_first   tile (0,0): factor and invert (one warp)
//   step k:
//   k_chol_panel   one CTA per tile row i > k:  L_ik = A_ik Linv_kk^T
//   k_chol_update  one CTA per trailing tile (i, j), k < j <= i:
//                  A_ij -= L_ik L_jk^T; the CTA of tile (k+1, k+1) then
//                  factors and inverts it, so the next panel can start
// The inverted diagonal tiles Linv_kk turn the panel solve into a GEMM and
// the diagonal steps of the triangular solves into 32 x 32 matrix-vector
// products. k_trsv_cluster: forward and backward substitution, one thread
// block cluster per sub-block.
//
// Two solvers use these kernels:
//   FP64 direct: factor S in place (the all-FP64 form).
//   mixed: Jacobi-scaled S' = D S D (D = diag(S)^-1/2) is rounded to FP32 and
//   factored in FP32; the FP64 solution comes from iterative refinement
//   x += L^-T L^-1 (D y - D S D x) with the residual in FP64 (k_symv).
// A non-positive pivot marks the sub-block as failed (its LM step is rejected).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "rpba_internal.cuh"
#include "tc_sm100.cuh"

namespace rpba {

#define CT 32  // tile size
#define CLD (CT + 1)

struct CholView {
  const long long *off;  // per sub-block offset of its matrix (elements)
  const int *npad;       // padded size
  const int *linv_off;   // per sub-block offset of its inverted diagonal tiles (elements)
  const int *run;
  int *fail;
  const int *sched;      // per step k: L+1 prefix sums of panel tiles, then L+1 of update tiles
  int L;
};

// p -> (a, b), b <= a, p = a (a + 1) / 2 + b; FP32 estimate, exact integer fix-up
// (an FP64 sqrt here would occupy the slow FP64 pipe of every thread)
__device__ inline void tri_index(int p, int &a, int &b) {
  a = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= p) a++;
  while (a * (a + 1) / 2 > p) a--;
  b = p - a * (a + 1) / 2;
}

// CTA -> (sub-block, local index) through the prefix sums of step k
__device__ inline int sched_find(const int *base, int L, int idx, int *local) {
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  *local = idx - base[lo];
  return lo;
}

// ---------------------------------------------------------------------------
// one warp: factor the 32 x 32 tile held as rows in registers (lane = row),
// then invert the factor into smem Xs (row-major, CLD stride). Returns false on
// a non-positive pivot (uniform across the warp).
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool warp_potrf_inv(T (&x)[CT], T *Ls, T *Xs) {
  int lane = threadIdx.x & 31;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < CT; j++) {
    T piv = __shfl_sync(0xffffffffu, x[j], j);
    if (!(piv > T(0))) ok = false;
    T d = sqrt(piv);
    T lj = (lane == j) ? d : x[j] / d;  // L[lane][j] for lane >= j
    if (lane >= j) x[j] = lj;
#pragma unroll
    for (int c = j + 1; c < CT; c++) {
      T lcj = __shfl_sync(0xffffffffu, lj, c);  // L[c][j]
      if (lane >= c) x[c] -= lj * lcj;
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  if (!ok) return false;
  // L to smem (row lane), zeros above the diagonal
#pragma unroll
  for (int c = 0; c < CT; c++) Ls[lane * CLD + c] = (c <= lane) ? x[c] : T(0);
  __syncwarp();
  // inverse, column `lane`: forward substitution L xcol = e_lane
  T xc[CT];
#pragma unroll
  for (int r = 0; r < CT; r++) {
    T s = (r == lane) ? T(1) : T(0);
#pragma unroll
    for (int m = 0; m < r; m++) s -= Ls[r * CLD + m] * xc[m];
    xc[r] = (r >= lane) ? s / Ls[r * CLD + r] : T(0);
  }
#pragma unroll
  for (int r = 0; r < CT; r++) Xs[r * CLD + lane] = xc[r];
  __syncwarp();
  return true;
}

// store the factored tile (lower part) and its inverse
template <typename T>
__device__ void store_diag(T *A, int np, int k, const T *Ls, const T *Xs, T *Linv) {
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    int r = e / CT, c = e - r * CT;
    if (c <= r) A[(size_t)(k * CT + r) * np + k * CT + c] = Ls[r * CLD + c];
    Linv[e] = Xs[r * CLD + c];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_first(T *S, T *Linv, CholView cv) {
  int l = blockIdx.x;
  if (!cv.run[l] || cv.fail[l] || cv.npad[l] == 0) return;
  int np = cv.npad[l];
  T *A = S + cv.off[l];
  __shared__ T Ls[CT * CLD], Xs[CT * CLD];
  __shared__ int bad;
  if (threadIdx.x < 32) {
    T x[CT];
    int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < CT; c++) x[c] = A[(size_t)lane * np + c];
    bool ok = warp_potrf_inv<T>(x, Ls, Xs);
    if (lane == 0) bad = !ok;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) cv.fail[l] = 1;
    return;
  }
  store_diag<T>(A, np, 0, Ls, Xs, Linv + cv.linv_off[l]);
}

// 32 x 32 x 32 product on 256 threads, 2 x 2 outputs per thread:
// out[r][c] = sum_m P[r][m] Q[c][m]  (P, Q in smem, CLD stride)
template <typename T>
__device__ inline void tile_nt(const T *P, const T *Q, T (&acc)[2][2]) {
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int c = 0; c < 2; c++) acc[r][c] = T(0);
#pragma unroll 8
  for (int m = 0; m < CT; m++) {
    T a0 = P[ty * CLD + m], a1 = P[(ty + 16) * CLD + m];
    T b0 = Q[tx * CLD + m], b1 = Q[(tx + 16) * CLD + m];
    acc[0][0] = fma(a0, b0, acc[0][0]);
    acc[0][1] = fma(a0, b1, acc[0][1]);
    acc[1][0] = fma(a1, b0, acc[1][0]);
    acc[1][1] = fma(a1, b1, acc[1][1]);
  }
}

template <typename T>
__device__ inline void load_tile(T *dst, const T *A, int np, int ti, int tj) {
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    int r = e / CT, c = e - r * CT;
    dst[r * CLD + c] = A[(size_t)(ti * CT + r) * np + tj * CT + c];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_panel(T *S, const T *Linv, CholView cv, int k) {
  int loc;
  int l = sched_find(cv.sched + (size_t)k * 2 * (cv.L + 1), cv.L, blockIdx.x, &loc);
  if (!cv.run[l] || cv.fail[l]) return;
  int np = cv.npad[l];
  int nt = np / CT;
  int ti = k + 1 + loc;
  if (ti >= nt) return;
  T *A = S + cv.off[l];
  __shared__ T P[CT * CLD], Q[CT * CLD];
  load_tile<T>(P, A, np, ti, k);
  const T *Li = Linv + cv.linv_off[l] + (size_t)k * CT * CT;
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) Q[(e / CT) * CLD + e % CT] = Li[e];
  __syncthreads();
  T acc[2][2];
  tile_nt<T>(P, Q, acc);  // A_ik Linv_kk^T
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int c = 0; c < 2; c++) A[(size_t)(ti * CT + ty + 16 * r) * np + k * CT + tx + 16 * c] = acc[r][c];
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_chol_update(T *S, T *Linv, CholView cv, int k) {
  int loc;
  int l = sched_find(cv.sched + (size_t)k * 2 * (cv.L + 1) + (cv.L + 1), cv.L, blockIdx.x, &loc);
  if (!cv.run[l] || cv.fail[l]) return;
  int np = cv.npad[l];
  int nt = np / CT;
  int rem = nt - k - 1;
  if (rem <= 0) return;
  int a, b;
  tri_index(loc, a, b);
  if (a >= rem) return;
  int ti = k + 1 + a, tj = k + 1 + b;
  T *A = S + cv.off[l];
  __shared__ T P[CT * CLD], Q[CT * CLD], C[CT * CLD];
  __shared__ int bad;
  load_tile<T>(P, A, np, ti, k);
  load_tile<T>(Q, A, np, tj, k);
  __syncthreads();
  T acc[2][2];
  tile_nt<T>(P, Q, acc);
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  bool diag_next = (ti == k + 1) && (tj == k + 1);
  if (!diag_next) {
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
      for (int c = 0; c < 2; c++) A[(size_t)(ti * CT + ty + 16 * r) * np + tj * CT + tx + 16 * c] -= acc[r][c];
    return;
  }
  // tile (k+1, k+1) is complete: update, factor and invert it here
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int c = 0; c < 2; c++) {
      int rr = ty + 16 * r, cc = tx + 16 * c;
      C[rr * CLD + cc] = A[(size_t)(ti * CT + rr) * np + tj * CT + cc] - acc[r][c];
    }
  __syncthreads();
  if (threadIdx.x < 32) {
    T x[CT];
    int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < CT; c++) x[c] = C[lane * CLD + c];
    bool ok = warp_potrf_inv<T>(x, P, Q);  // P <- L, Q <- L^-1
    if (lane == 0) bad = !ok;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) cv.fail[l] = 1;
    return;
  }
  store_diag<T>(A, np, k + 1, P, Q, Linv + cv.linv_off[l] + (size_t)(k + 1) * CT * CT);
}

// ---------------------------------------------------------------------------
// FP32 factorisation with the updates on the tensor cores (chol_tc)
//
// Left-looking over block columns J of 32. A task (sub-block l, step J, row
// block i) gathers the 128 rows {diagonal rows 32J .. 32J+31} and {96 rows
// below, from 32J + 32 + 96 i} of every finished block column k < J and
// accumulates in tensor memory
//     U = sum_k P_k[rows] P_k[32J .. 32J+31]^T          (128 x 32, K = 32 J)
// with tcgen05.mma kind::tf32: each factor entry is held as three TF32 pieces
// h + m + l (h, m rounded to TF32, l the exact FP32 remainder) and the six
// products hh, hm, mh, hl, lh, mm are accumulated, which keeps the update at
// FP32 accuracy (the dropped products are below 2^-31 relative). Operands
// arrive by TMA (128-byte swizzle) in a two-stage ring; one thread issues the
// TMA loads and the MMAs, tcgen05.commit frees a stage. Then every task of the
// step factors the updated diagonal tile A_JJ - U[0:32] itself (one warp; the
// result is the same in every task) and solves its rows:
//     L_iJ = (A_iJ - U_i) L_JJ^-T,
// writing them to the row-major factor (read by the triangular solves, which
// take the diagonal steps from the inverted tiles, so A_JJ itself is only
// read here) and as TF32 pieces to block column J's panel (read by the later
// steps). The task of row block 0 stores L_JJ^-1. Every wait is bounded
// (tc::mbar_wait); on a timeout the task records it in err, marks the
// sub-block failed, waits (bounded) for its own MMAs and loads.
//
// Two launch forms: one launch per step (k_chol_tc), or one persistent
// cooperative launch (k_chol_tc_persistent) whose CTAs take the tasks of all
// steps of all sub-blocks from a queue ordered by step (within a step the
// larger sub-blocks first); a task waits (bounded) until every task of its
// sub-block's previous step has finished, so sub-blocks of uneven size
// advance independently instead of in lock step.
// ---------------------------------------------------------------------------
#define TC_ROWS 128                            // rows of one MMA (M)
#define TC_BELOW 96                            // rows below the diagonal tile per task
#define TC_PIECE_BYTES (TC_ROWS * CT * 4)      // one piece of one stage: 16 KB
#define TC_STAGE_BYTES (3 * TC_PIECE_BYTES)    // three pieces: 48 KB
#define TC_STAGES 2
#define TC_SMEM (TC_STAGES * TC_STAGE_BYTES + 1024)
#define TC_WAIT_NS 200000000ull                // 0.2 s: no wait of a healthy launch comes near it

struct TcView {
  float *S;                 // FP32 factor storage (row-major, the layout of S32)
  const long long *off;
  const int *npad;
  float *Linv;
  const int *linv_off;
  const int *run;
  int *fail;
  float *P0, *P1, *P2;      // panel pieces
  const long long *prow;
  const int *sched;         // per-step launch: this step's L+1 prefix sums of CTAs
  int L;
  int *err;
  // persistent launch: the task queue (l, J, i) and its head, the finished
  // tasks per (sub-block, step), the task count per (sub-block, step)
  const int4 *tasks;
  int n_tasks;
  int *head;
  int *done;
  const int *need;
  int T_max;
};

__device__ inline void tc_split3(float x, float &h, float &m, float &l) {
  h = tc::tf32_round(x);
  float r = x - h;  // exact
  m = tc::tf32_round(r);
  l = r - m;        // exact
}

// what a CTA keeps across the tasks it runs: its barriers, TMEM, and the
// count of stage fills and accumulations (the barriers' phase parities)
struct TcCta {
  uint64_t *full, *empty, *done;
  uint32_t tmem;
  uint8_t *base;
  uint32_t fills;  // stage fills so far (stage = fills % TC_STAGES)
  uint32_t dones;  // accumulations completed so far
};

struct TcShared {
  float Ls[CT * CLD], Xs[CT * CLD];
  int ok, bad;
};

// one task: the update of (l, J, loc), the diagonal factor, the rows' solve.
// Returns false when a bounded wait gave up (the sub-block is marked failed).
__device__ bool tc_task(const CUtensorMap *tm0, const CUtensorMap *tm1, const CUtensorMap *tm2, const TcView &v,
                        int l, int J, int loc, TcCta &c, TcShared &sh) {
  const int np = v.npad[l];
  const int d0 = 32 * J, r0 = d0 + 32 + TC_BELOW * loc;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float *A = v.S + v.off[l];
  float acc[32];
#pragma unroll
  for (int q = 0; q < 32; q++) acc[q] = 0.f;

  if (J > 0) {
    if (tid == 0) {
      bool ok = true;
      const long long prow = v.prow[l];
      const CUtensorMap *maps[3] = {tm0, tm1, tm2};
      const uint32_t f0 = c.fills;
      auto load = [&](int k) {
        uint32_t f = f0 + (uint32_t)k;
        int s = (int)(f % TC_STAGES);
        uint8_t *st = c.base + s * TC_STAGE_BYTES;
        tc::mbar_arrive_expect_tx(&c.full[s], TC_STAGE_BYTES);
        int y = (int)(prow + (long long)k * np);
        for (int p = 0; p < 3; p++) {
          uint8_t *pb = st + p * TC_PIECE_BYTES;
          tc::tma_load_2d(pb, maps[p], 0, y + d0, &c.full[s]);
          for (int b = 0; b < 3; b++) tc::tma_load_2d(pb + (1 + b) * 32 * 128, maps[p], 0, y + r0 + 32 * b, &c.full[s]);
        }
      };
      const uint32_t idesc = tc::idesc_tf32(TC_ROWS, CT);
      // products of the pieces (A piece, B piece): hh hm mh hl lh mm
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
      int issued = 0;
      for (int k = 0; k < J && k < TC_STAGES; k++) {
        // a stage is reused only after the MMAs that read it completed: the
        // previous task's accumulation finished before its epilogue
        load(k);
        issued++;
      }
      int k = 0;
      for (; k < J; k++) {
        uint32_t f = f0 + (uint32_t)k;
        int s = (int)(f % TC_STAGES);
        uint32_t ph = (f / TC_STAGES) & 1u;
        if (!tc::mbar_wait(&c.full[s], ph, TC_WAIT_NS)) { ok = false; break; }
        tc::tc_fence_after();
        uint32_t sa = tc::smem_u32(c.base + s * TC_STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {  // K = 8 TF32 (32 bytes) per MMA
          uint64_t d[3];
#pragma unroll
          for (int p = 0; p < 3; p++) d[p] = tc::desc_sw128_kmajor(sa + p * TC_PIECE_BYTES + kk * 32);
#pragma unroll
          for (int t = 0; t < 6; t++)  // B = the diagonal rows: the first 32 rows of its piece
            tc::mma_tf32(c.tmem, d[pa[t]], d[pb[t]], idesc, (k > 0 || kk > 0 || t > 0) ? 1u : 0u);
        }
        tc::mma_commit(&c.empty[s]);
        if (k + TC_STAGES < J) {
          if (!tc::mbar_wait(&c.empty[s], ph, TC_WAIT_NS)) { ok = false; k++; break; }
          load(k + TC_STAGES);
          issued++;
        }
      }
      // every MMA issued so far completes before this arrival
      tc::mma_commit(c.done);
      bool fin = tc::mbar_wait(c.done, c.dones & 1u, TC_WAIT_NS);
      if (!ok) {
        // loads still in flight land in this CTA's shared memory: wait for
        // them (bounded) before going on
        for (int q = k; q < issued; q++) {
          uint32_t f = f0 + (uint32_t)q;
          tc::mbar_wait(&c.full[f % TC_STAGES], (f / TC_STAGES) & 1u, TC_WAIT_NS);
        }
      }
      sh.ok = ok && fin;
    }
    c.fills += (uint32_t)J;
    c.dones += 1;
    __syncthreads();
    tc::tc_fence_after();
    if (sh.ok) tc::tmem_ld32(c.tmem + ((uint32_t)(32 * warp) << 16), acc);
    tc::tc_fence_before();
    __syncthreads();
    if (!sh.ok) {
      if (tid == 0) {
        atomicExch(v.err, 1);
        v.fail[l] = 1;
      }
      return false;
    }
  }

  // diagonal tile: A_JJ - U[0:32] (lower part), factored and inverted by warp 0
  if (warp == 0) {
    float x[CT];
#pragma unroll
    for (int q = 0; q < CT; q++) x[q] = (q <= lane) ? A[(size_t)(d0 + lane) * np + d0 + q] - acc[q] : 0.f;
    bool okp = warp_potrf_inv<float>(x, sh.Ls, sh.Xs);
    if (lane == 0) sh.bad = !okp;
  }
  __syncthreads();
  if (sh.bad) {
    if (tid == 0 && loc == 0) v.fail[l] = 1;
    return true;
  }
  if (warp == 0 && loc == 0) {
    float *Li = v.Linv + v.linv_off[l] + (size_t)J * CT * CT;
    for (int q = 0; q < CT; q++) Li[lane * CT + q] = sh.Xs[lane * CLD + q];
  }
  // rows below: L_iJ = (A_iJ - U_i) L_JJ^-T (L_JJ^-1 lower triangular)
  if (warp > 0) {
    int r = r0 + 32 * (warp - 1) + lane;
    if (r < np) {
      float crow[CT];
#pragma unroll
      for (int q = 0; q < CT; q++) crow[q] = A[(size_t)r * np + d0 + q] - acc[q];
      long long pr = (v.prow[l] + (long long)J * np + r) * CT;
#pragma unroll
      for (int q = 0; q < CT; q++) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e <= q; e++) s = fmaf(crow[e], sh.Xs[q * CLD + e], s);
        A[(size_t)r * np + d0 + q] = s;
        float h, m, lo;
        tc_split3(s, h, m, lo);
        v.P0[pr + q] = h;
        v.P1[pr + q] = m;
        v.P2[pr + q] = lo;
      }
    }
  }
  return true;
}

// barriers and TMEM of a CTA (128 threads)
__device__ inline void tc_cta_init(TcCta &c, uint64_t *full, uint64_t *empty, uint64_t *done, uint32_t *tmem_slot,
                                   uint8_t *raw, const CUtensorMap *tm0, const CUtensorMap *tm1,
                                   const CUtensorMap *tm2) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(tm0);
    tc::prefetch_tmap(tm1);
    tc::prefetch_tmap(tm2);
  }
  if ((tid >> 5) == 0) {
    tc::tmem_alloc(tmem_slot, 32);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  c.full = full;
  c.empty = empty;
  c.done = done;
  c.tmem = *tmem_slot;
  c.base = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  c.fills = 0;
  c.dones = 0;
}

__device__ inline void tc_cta_fini(TcCta &c) {
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(c.tmem, 32);
}

__global__ void __launch_bounds__(128) k_chol_tc(const __grid_constant__ CUtensorMap tm0,
                                                 const __grid_constant__ CUtensorMap tm1,
                                                 const __grid_constant__ CUtensorMap tm2, TcView v, int J) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ TcShared sh;
  int loc;
  int l = sched_find(v.sched, v.L, blockIdx.x, &loc);
  if (!v.run[l] || v.fail[l]) return;  // CTA-uniform
  if (32 * J >= v.npad[l]) return;
  if (J == 0) {  // no update: no barriers, no TMEM
    TcCta c{};
    tc_task(&tm0, &tm1, &tm2, v, l, J, loc, c, sh);
    return;
  }
  TcCta c;
  tc_cta_init(c, bar_full, bar_empty, &bar_done, &tmem_slot, tc_smem_raw, &tm0, &tm1, &tm2);
  tc_task(&tm0, &tm1, &tm2, v, l, J, loc, c, sh);
  tc_cta_fini(c);
}

// acquire load of a completion counter
__device__ inline int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(128) k_chol_tc_persistent(const __grid_constant__ CUtensorMap tm0,
                                                            const __grid_constant__ CUtensorMap tm1,
                                                            const __grid_constant__ CUtensorMap tm2, TcView v) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ TcShared sh;
  __shared__ int cur, go;
  TcCta c;
  tc_cta_init(c, bar_full, bar_empty, &bar_done, &tmem_slot, tc_smem_raw, &tm0, &tm1, &tm2);
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(v.head, 1);
    __syncthreads();
    const int t = cur;
    if (t >= v.n_tasks) break;
    const int4 task = v.tasks[t];
    const int l = task.x, J = task.y, loc = task.z;
    if (threadIdx.x == 0) {
      // every task of the previous step of this sub-block has finished: the
      // queue holds all of them before this one, and they run on CTAs that
      // are resident (cooperative launch), so the wait ends
      bool ok = true;
      if (J > 0) {
        const int *cnt = v.done + (size_t)l * v.T_max + (J - 1);
        const int want = v.need[(size_t)l * v.T_max + (J - 1)];
        if (ld_acquire(cnt) < want) {
          uint64_t t0 = tc::global_ns();
          while (ld_acquire(cnt) < want) {
            __nanosleep(200);
            if (tc::global_ns() - t0 > TC_WAIT_NS) { ok = false; break; }
          }
        }
        // the panels that task wrote with generic stores are read by TMA
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
      if (!ok) {
        atomicExch(v.err, 1);
        v.fail[l] = 1;
      }
      // after any error the remaining tasks are only counted, so that no
      // task waits on work that will not come
      go = ok && v.run[l] && !v.fail[l] && !*(volatile int *)v.err;
    }
    __syncthreads();
    if (go) tc_task(&tm0, &tm1, &tm2, v, l, J, loc, c, sh);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(v.done + (size_t)l * v.T_max + J, 1);
    }
  }
  tc_cta_fini(c);
}

// forward L z = r and backward L^T x = z (r in, x out, may alias), one thread
// block cluster of TS CTAs per sub-block. Tile rows are owned round-robin
// (tile t by CTA t % TS); each step the owner of tile k solves its 32 entries
// with the inverted diagonal tile and publishes them in its shared memory,
// one cluster barrier later every CTA reads them through distributed shared
// memory and updates the tiles it owns. The barrier is the hardware cluster
// barrier (no software wait). Two buffers alternate between steps.
#define TS 8
template <typename T>
__global__ void __cluster_dims__(TS, 1, 1) __launch_bounds__(256)
    k_trsv_cluster(const T *S, const T *Linv, CholView cv, const int *voff, T *r, T *x) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  int rank = (int)cluster.block_rank();
  int l = blockIdx.y;
  if (!cv.run[l] || cv.fail[l]) return;  // uniform over the cluster
  int np = cv.npad[l];
  int nt = np / CT;
  const T *A = S + cv.off[l];
  const T *LI = Linv + cv.linv_off[l];
  T *z = r + voff[l];
  T *xo = x + voff[l];
  __shared__ T buf[2][CT];
  __shared__ T loc[CT];
  int tid = threadIdx.x;
  int row = tid >> 3, part = tid & 7;  // 32 rows x 8 parts of 4 columns
  // forward; the L tiles a CTA needs after the barrier of step k are read
  // into registers before it, so their latency overlaps the barrier
  const int MAXT = 8;  // owned tiles prefetched per step (more are read late)
  for (int k = 0; k < nt; k++) {
    int owner = k % TS;
    int t0 = k + 1 + ((rank - (k + 1)) % TS + TS) % TS;
    T pre[MAXT][4];
#pragma unroll
    for (int m = 0; m < MAXT; m++) {
      int t = t0 + m * TS;
      if (t < nt) {
        const T *Lt = A + (size_t)(t * CT + row) * np + k * CT + part * 4;
#pragma unroll
        for (int c = 0; c < 4; c++) pre[m][c] = Lt[c];
      }
    }
    if (rank == owner) {
      const T *Li = LI + (size_t)k * CT * CT;
      T s = 0;
#pragma unroll
      for (int c = 0; c < 4; c++) s += Li[row * CT + part * 4 + c] * z[k * CT + part * 4 + c];
      for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
      if (part == 0) {
        buf[k & 1][row] = s;
        z[k * CT + row] = s;
      }
    }
    cluster.sync();
    const T *src = cluster.map_shared_rank(&buf[k & 1][0], owner);
    if (tid < CT) loc[tid] = src[tid];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MAXT; m++) {
      int t = t0 + m * TS;
      if (t < nt) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) s += pre[m][c] * loc[part * 4 + c];
        for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
        if (part == 0) z[t * CT + row] -= s;
      }
    }
    for (int t = t0 + MAXT * TS; t < nt; t += TS) {
      const T *Lt = A + (size_t)(t * CT + row) * np + k * CT + part * 4;
      T s = 0;
#pragma unroll
      for (int c = 0; c < 4; c++) s += Lt[c] * loc[part * 4 + c];
      for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
      if (part == 0) z[t * CT + row] -= s;
    }
    __syncthreads();
  }
  // backward
  for (int k = nt - 1; k >= 0; k--) {
    int owner = k % TS;
    int col = tid >> 3;
    T pre[MAXT][4];
#pragma unroll
    for (int m = 0; m < MAXT; m++) {
      int t = rank + m * TS;
      if (t < k) {
        const T *Lt = A + (size_t)(k * CT + part * 4) * np + t * CT + col;
#pragma unroll
        for (int rr = 0; rr < 4; rr++) pre[m][rr] = Lt[(size_t)rr * np];
      }
    }
    if (rank == owner) {
      const T *Li = LI + (size_t)k * CT * CT;
      T s = 0;
#pragma unroll
      for (int c = 0; c < 4; c++) s += Li[(part * 4 + c) * CT + row] * z[k * CT + part * 4 + c];
      for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
      if (part == 0) {
        buf[k & 1][row] = s;
        xo[k * CT + row] = s;
      }
    }
    cluster.sync();
    const T *src = cluster.map_shared_rank(&buf[k & 1][0], owner);
    if (tid < CT) loc[tid] = src[tid];
    __syncthreads();
    // z_j -= L_kj^T x_k for owned tiles j < k: column c of the tile, 8 parts of 4 rows
#pragma unroll
    for (int m = 0; m < MAXT; m++) {
      int t = rank + m * TS;
      if (t < k) {
        T s = 0;
#pragma unroll
        for (int rr = 0; rr < 4; rr++) s += pre[m][rr] * loc[part * 4 + rr];
        for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
        if (part == 0) z[t * CT + col] -= s;
      }
    }
    for (int t = rank + MAXT * TS; t < k; t += TS) {
      const T *Lt = A + (size_t)(k * CT + part * 4) * np + t * CT + col;
      T s = 0;
#pragma unroll
      for (int rr = 0; rr < 4; rr++) s += Lt[(size_t)rr * np] * loc[part * 4 + rr];
      for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, 8);
      if (part == 0) z[t * CT + col] -= s;
    }
    __syncthreads();
  }
  cluster.sync();  // keep every CTA's shared memory alive until all reads are done
}

template <typename T>
static rpba_status factor(Ctx *ctx, T *S, T *Linv, CholView cv, int T_max) {
  const char *n_first = sizeof(T) == 8 ? "k_chol_first_f64" : "k_chol_first_f32";
  const char *n_panel = sizeof(T) == 8 ? "k_chol_panel_f64" : "k_chol_panel_f32";
  const char *n_upd = sizeof(T) == 8 ? "k_chol_update_f64" : "k_chol_update_f32";
  RPBA_KERNEL(ctx, n_first, k_chol_first<T><<<ctx->L, 256, 0, ctx->stream>>>(S, Linv, cv));
  for (int k = 0; k + 1 < T_max; k++) {
    int np_k = ctx->h_sched[(size_t)k * 2 * (ctx->L + 1) + ctx->L];
    int nu_k = ctx->h_sched[(size_t)k * 2 * (ctx->L + 1) + 2 * ctx->L + 1];
    if (np_k == 0) break;
    RPBA_KERNEL(ctx, n_panel, k_chol_panel<T><<<np_k, 256, 0, ctx->stream>>>(S, Linv, cv, k));
    RPBA_KERNEL(ctx, n_upd, k_chol_update<T><<<nu_k, 256, 0, ctx->stream>>>(S, Linv, cv, k));
  }
  return RPBA_OK;
}

// ---------------------------------------------------------------------------
// mixed-precision solve: scaling, FP64 residual, refinement updates
// ---------------------------------------------------------------------------
// d = diag(S)^-1/2 (1 on the padding), rs = D y, x = 0
__global__ void k_mixed_scale(const double *S, const long long *off, const int *npad, const int *voff,
                              const int *run, const double *y, double *d, double *rs, double *x) {
  int l = blockIdx.y;
  if (!run[l]) return;
  int np = npad[l];
  const double *A = S + off[l];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np; e += gridDim.x * blockDim.x) {
    double s = A[(size_t)e * np + e];
    double de = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    int g = voff[l] + e;
    d[g] = de;
    rs[g] = de * y[g];
    x[g] = 0.0;
  }
}

// S32 = D S D rounded to FP32 (lower triangle); the products are formed in
// FP32 (the refinement corrects the factor's rounding)
__global__ void k_mixed_convert(const double *S, float *S32, const long long *off, const long long *off32,
                                const int *npad, const int *voff, const int *run, const double *d) {
  int l = blockIdx.y;
  if (!run[l]) return;
  int np = npad[l];
  const double *A = S + off[l];
  float *B = S32 + off32[l];
  const double *dl = d + voff[l];
  size_t tot = (size_t)np * np;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    size_t r = e / np, c = e - r * np;
    if (c > r) continue;
    B[e] = (float)A[e] * (float)dl[r] * (float)dl[c];
  }
}

// u = D x (FP64); t = S u with S symmetric from its lower triangle, one CTA per
// 32 x 32 lower tile: t_I += S_IJ u_J and, off the diagonal, t_J += S_IJ^T u_I
__global__ void __launch_bounds__(256) k_symv(const double *S, const long long *off, const int *npad,
                                              const int *voff, const int *run, const int *fail, const double *d,
                                              const double *x, double *t, int T_max) {
  int l = blockIdx.y;
  if (!run[l] || fail[l]) return;
  int np = npad[l];
  int nt = np / CT;
  int a, b;
  tri_index((int)blockIdx.x, a, b);
  if (a >= nt) return;
  const double *A = S + off[l];
  const double *dl = d + voff[l], *xl = x + voff[l];
  double *tl = t + voff[l];
  __shared__ double uI[CT], uJ[CT];
  __shared__ double blk[CT][CLD];
  int tid = threadIdx.x;
  if (tid < CT) {
    uI[tid] = dl[a * CT + tid] * xl[a * CT + tid];
    uJ[tid] = dl[b * CT + tid] * xl[b * CT + tid];
  }
  for (int e = tid; e < CT * CT; e += blockDim.x) {
    int r = e / CT, c = e - r * CT;
    double v = A[(size_t)(a * CT + r) * np + b * CT + c];
    if (a == b && c > r) v = A[(size_t)(a * CT + c) * np + b * CT + r];  // mirror the diagonal tile
    blk[r][c] = v;
  }
  __syncthreads();
  if (tid < CT) {
    double s = 0.0;
    for (int c = 0; c < CT; c++) s += blk[tid][c] * uJ[c];
    atomicAdd(tl + a * CT + tid, s);
  } else if (tid < 2 * CT && a != b) {
    int c = tid - CT;
    double s = 0.0;
    for (int r = 0; r < CT; r++) s += blk[r][c] * uI[r];
    atomicAdd(tl + b * CT + c, s);
  }
}

// r32 = (float)(rs - D t)   (residual of the scaled system), or rs on the first pass
__global__ void k_mixed_residual(const int *run, const int *fail, const int *voff, const int *npad, int L,
                                 const double *rs, const double *d, const double *t, float *r32, int first) {
  int l = blockIdx.y;
  if (l >= L || !run[l] || fail[l]) return;
  int np = npad[l];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np; e += gridDim.x * blockDim.x) {
    int g = voff[l] + e;
    r32[g] = (float)(first ? rs[g] : rs[g] - d[g] * t[g]);
  }
}

// x += z; on the last pass dC = D x
__global__ void k_mixed_update(const int *run, const int *fail, const int *voff, const int *npad, int L,
                               const float *z, double *x, const double *d, double *dC, int last) {
  int l = blockIdx.y;
  if (l >= L || !run[l] || fail[l]) return;
  int np = npad[l];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np; e += gridDim.x * blockDim.x) {
    int g = voff[l] + e;
    double v = x[g] + (double)z[g];
    x[g] = v;
    if (last) dC[g] = d[g] * v;
  }
}

// the panel layout, per-step schedule and TMA tensor maps of the
// tensor-core factorisation (once per context)
rpba_status tc_chol_setup(Ctx *ctx) {
  int L = ctx->L, steps = ctx->max_tiles;
  if (L == 0 || steps == 0) return RPBA_OK;
  std::vector<long long> prow(L);
  long long rows = 0;
  for (int l = 0; l < L; l++) {
    prow[l] = rows;
    rows += (long long)(ctx->h_npad[l] / CT) * ctx->h_npad[l];
  }
  if (rows + TC_ROWS >= (1LL << 31)) {
    ctx->err = "RCS too large for the tensor-core factorisation's 32-bit panel rows";
    return RPBA_ERR_INVALID_ARG;
  }
  std::vector<int> sched((size_t)steps * (L + 1), 0);
  ctx->h_tc_ctas.assign(steps, 0);
  for (int J = 0; J < steps; J++) {
    int *pb = &sched[(size_t)J * (L + 1)];
    for (int l = 0; l < L; l++) {
      int np = ctx->h_npad[l], below = np - CT * J - CT;
      int c = (CT * J < np) ? 1 + (below > 0 ? (below + TC_BELOW - 1) / TC_BELOW : 0) : 0;
      pb[l + 1] = pb[l] + c;
    }
    ctx->h_tc_ctas[J] = pb[L];
  }
  for (int p = 0; p < 3; p++) {
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_panel[p], (size_t)(rows + TC_ROWS) * CT * sizeof(float)));
    RPBA_CUDA(cudaMemsetAsync(ctx->tc_panel[p], 0, (size_t)(rows + TC_ROWS) * CT * sizeof(float), ctx->stream));
  }
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_prow, sizeof(long long) * L));
  RPBA_CUDA(cudaMemcpyAsync(ctx->tc_prow, prow.data(), sizeof(long long) * L, cudaMemcpyHostToDevice, ctx->stream));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_sched, sizeof(int) * sched.size()));
  RPBA_CUDA(cudaMemcpyAsync(ctx->tc_sched, sched.data(), sizeof(int) * sched.size(), cudaMemcpyHostToDevice,
                            ctx->stream));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_err, sizeof(int)));
  RPBA_CUDA(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->stream));
  // cuTensorMapEncodeTiled through the runtime (no link against the driver library)
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    ctx->err = "cuTensorMapEncodeTiled is not available";
    return RPBA_ERR_CUDA;
  }
  auto encode = (CUresult(*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill))fn;
  // 2-D: 32 floats (128 B) per row, all panel rows; boxes of 32 rows, 128-byte swizzle
  cuuint64_t dims[2] = {(cuuint64_t)CT, (cuuint64_t)(rows + TC_ROWS)};
  cuuint64_t strides[1] = {(cuuint64_t)CT * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)CT, 32};
  cuuint32_t estr[2] = {1, 1};
  for (int p = 0; p < 3; p++) {
    CUresult r = encode(&ctx->tc_map[p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ctx->tc_panel[p], dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      ctx->err = "cuTensorMapEncodeTiled failed for the factor panels";
      return RPBA_ERR_CUDA;
    }
  }
  RPBA_CUDA(cudaFuncSetAttribute(k_chol_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  RPBA_CUDA(cudaFuncSetAttribute(k_chol_tc_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  // the persistent form's queue: every (sub-block, step, row block) task,
  // ordered by step, within a step the larger sub-blocks first
  {
    std::vector<int4> tasks;
    std::vector<int> need((size_t)L * steps, 0);
    std::vector<int> order(L);
    for (int l = 0; l < L; l++) order[l] = l;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctx->h_npad[a] > ctx->h_npad[b]; });
    for (int J = 0; J < steps; J++)
      for (int l : order) {
        int np = ctx->h_npad[l], below = np - CT * J - CT;
        if (CT * J >= np) continue;
        int c = 1 + (below > 0 ? (below + TC_BELOW - 1) / TC_BELOW : 0);
        need[(size_t)l * steps + J] = c;
        for (int i = 0; i < c; i++) tasks.push_back(make_int4(l, J, i, 0));
      }
    ctx->tc_n_tasks = (int)tasks.size();
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_tasks, sizeof(int4) * std::max<size_t>(tasks.size(), 1)));
    RPBA_CUDA(cudaMemcpyAsync(ctx->tc_tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_need, sizeof(int) * need.size()));
    RPBA_CUDA(cudaMemcpyAsync(ctx->tc_need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
    // counters: the queue head, then the finished tasks per (sub-block, step)
    RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->tc_count, sizeof(int) * (1 + need.size())));
    int per_sm = 0, sms = 0, dev = 0;
    RPBA_CUDA(cudaGetDevice(&dev));
    RPBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RPBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_tc_persistent, 128, TC_SMEM));
    ctx->tc_grid = std::max(1, std::min(ctx->tc_n_tasks, std::max(per_sm, 1) * sms));
    RPBA_CUDA(cudaStreamSynchronize(ctx->stream));  // the host vectors go out of scope
  }
  ctx->tc_ready = true;
  return RPBA_OK;
}

// the FP32 factorisation of every running sub-block on the tensor cores
static rpba_status factor_tc(Ctx *ctx, float *S, float *Linv, const long long *off, const int *run, int *fail) {
  TcView tv{S, off, ctx->npad, Linv, ctx->linv_off, run, fail, ctx->tc_panel[0], ctx->tc_panel[1],
            ctx->tc_panel[2], ctx->tc_prow, nullptr, ctx->L, ctx->tc_err,
            ctx->tc_tasks, ctx->tc_n_tasks, ctx->tc_count, ctx->tc_count + 1, ctx->tc_need, ctx->max_tiles};
  if (ctx->opt.chol_tc == 2) {  // one persistent cooperative launch
    RPBA_CUDA(cudaMemsetAsync(ctx->tc_count, 0, sizeof(int) * (1 + (size_t)ctx->L * ctx->max_tiles), ctx->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctx->tc_grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = TC_SMEM;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RPBA_KERNEL(ctx, "k_chol_tc_persistent",
                RPBA_CUDA(cudaLaunchKernelEx(&cfg, k_chol_tc_persistent, ctx->tc_map[0], ctx->tc_map[1],
                                             ctx->tc_map[2], tv)));
    return RPBA_OK;
  }
  for (int J = 0; J < ctx->max_tiles; J++) {
    int n = ctx->h_tc_ctas[J];
    if (n == 0) break;
    tv.sched = ctx->tc_sched + (size_t)J * (ctx->L + 1);
    RPBA_KERNEL(ctx, "k_chol_tc", k_chol_tc<<<n, 128, TC_SMEM, ctx->stream>>>(ctx->tc_map[0], ctx->tc_map[1],
                                                                                ctx->tc_map[2], tv, J));
  }
  return RPBA_OK;
}

rpba_status launch_solve_rcs(Ctx *ctx, const int *run_dev, int *fail_dev) {
  if (ctx->opt.solver == 1) return launch_pcg_blockjacobi(ctx, run_dev, fail_dev);
  if (ctx->opt.solver == 3) return launch_pcg_learned(ctx, run_dev, fail_dev);
  RPBA_CUDA(cudaMemsetAsync(fail_dev, 0, ctx->L * sizeof(int), ctx->stream));
  int T_max = ctx->max_tiles;
  if (T_max == 0) return RPBA_OK;
  if (ctx->opt.solver != 2) {
    // FP64 direct: factor S in place, one forward/backward solve
    CholView cv{ctx->S_off, ctx->npad, ctx->linv_off, run_dev, fail_dev, ctx->sched, ctx->L};
    RPBA_TRY(factor<double>(ctx, ctx->S, ctx->Linv64, cv, T_max));
    RPBA_CUDA(cudaMemcpyAsync(ctx->dC, ctx->y, ctx->ytot * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    RPBA_KERNEL(ctx, "k_trsv_f64", k_trsv_cluster<double><<<dim3(TS, ctx->L), 256, 0, ctx->stream>>>(
                                     ctx->S, ctx->Linv64, cv, ctx->ycam_off, ctx->dC, ctx->dC));
    return RPBA_OK;
  }
  // mixed: FP32 factor of the scaled system, FP64 iterative refinement
  dim3 g(16, ctx->L);
  RPBA_KERNEL(ctx, "k_mixed_scale",
              k_mixed_scale<<<g, 256, 0, ctx->stream>>>(ctx->S, ctx->S_off, ctx->npad, ctx->ycam_off, run_dev, ctx->y,
                                                        ctx->ir_d, ctx->ir_rs, ctx->ir_x));
  RPBA_KERNEL(ctx, "k_mixed_convert",
              k_mixed_convert<<<dim3(64, ctx->L), 256, 0, ctx->stream>>>(ctx->S, ctx->S32, ctx->S_off, ctx->S32_off,
                                                                         ctx->npad, ctx->ycam_off, run_dev,
                                                                         ctx->ir_d));
  CholView cv{ctx->S32_off, ctx->npad, ctx->linv_off, run_dev, fail_dev, ctx->sched, ctx->L};
  if (ctx->opt.chol_tc && ctx->tc_ready)
    RPBA_TRY(factor_tc(ctx, ctx->S32, ctx->Linv32, ctx->S32_off, run_dev, fail_dev));
  else
    RPBA_TRY(factor<float>(ctx, ctx->S32, ctx->Linv32, cv, T_max));
  int passes = 1 + ctx->opt.ir_steps;
  for (int it = 0; it < passes; it++) {
    if (it > 0) {
      RPBA_CUDA(cudaMemsetAsync(ctx->ir_t, 0, ctx->ytot * sizeof(double), ctx->stream));
      dim3 gs((unsigned)((long long)T_max * (T_max + 1) / 2), ctx->L);
      RPBA_KERNEL(ctx, "k_symv", k_symv<<<gs, 256, 0, ctx->stream>>>(ctx->S, ctx->S_off, ctx->npad, ctx->ycam_off,
                                                                     run_dev, fail_dev, ctx->ir_d, ctx->ir_x,
                                                                     ctx->ir_t, T_max));
    }
    RPBA_KERNEL(ctx, "k_mixed_residual",
                k_mixed_residual<<<g, 256, 0, ctx->stream>>>(run_dev, fail_dev, ctx->ycam_off, ctx->npad, ctx->L,
                                                             ctx->ir_rs, ctx->ir_d, ctx->ir_t, ctx->ir_r32, it == 0));
    RPBA_KERNEL(ctx, "k_trsv_f32", k_trsv_cluster<float><<<dim3(TS, ctx->L), 256, 0, ctx->stream>>>(
                                     ctx->S32, ctx->Linv32, cv, ctx->ycam_off, ctx->ir_r32, ctx->ir_r32));
    RPBA_KERNEL(ctx, "k_mixed_update",
                k_mixed_update<<<g, 256, 0, ctx->stream>>>(run_dev, fail_dev, ctx->ycam_off, ctx->npad, ctx->L,
                                                           ctx->ir_r32, ctx->ir_x, ctx->ir_d, ctx->dC,
                                                           it == passes - 1));
  }
  return RPBA_OK;
}

}  // namespace rpba
