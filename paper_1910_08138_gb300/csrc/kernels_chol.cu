// kernels_chol.cu -- solve of the reduced camera systems S_l dC_l = y_l of all
// running sub-blocks at once (Sec. 2: direct Cholesky factorisation of the RCS).
//
// Each S_l is dense, row-major, padded to n_pad = 64 * tiles (identity on the
// padding). Right-looking blocked Cholesky with 64 x 64 tiles, lower factor
// in place, batched over sub-blocks of different sizes:
//   step k: k_potrf_panel  one CTA per tile row i >= k: factor A_kk in shared
//                          memory (every CTA redundantly), then L_ik = A_ik L_kk^-T
//           k_syrk_update  one CTA per trailing tile (i, j), k < j <= i:
//                          A_ij -= L_ik L_jk^T
// then k_trsv: one CTA per sub-block, forward and backward substitution.
// A non-positive pivot marks the sub-block as failed (its LM step is rejected).
#include <cuda_runtime.h>
#include <math.h>

#include "rpba_internal.cuh"

namespace rpba {

#define NB RPBA_TILE
#define LDS (NB + 1)

__global__ void __launch_bounds__(256) k_potrf_panel(double *S, const long long *S_off, const int *npad,
                                                     const int *run, int *fail, int k) {
  int l = blockIdx.y;
  if (!run[l] || fail[l]) return;
  int np = npad[l];
  int T = np / NB;
  int ti = k + blockIdx.x;
  if (ti >= T) return;
  extern __shared__ double sm[];
  double *D = sm, *B = sm + NB * LDS;
  __shared__ int bad;
  double *A = S + S_off[l];
  int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e - r * NB;
    D[r * LDS + c] = A[(size_t)(k * NB + r) * np + k * NB + c];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < NB; j++) {
    if (tid == 0) {
      double d = D[j * LDS + j];
      if (!(d > 0.0)) bad = 1;
      else D[j * LDS + j] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    double dj = D[j * LDS + j];
    for (int r = j + 1 + tid; r < NB; r += blockDim.x) D[r * LDS + j] /= dj;
    __syncthreads();
    int w = NB - 1 - j;
    for (int e = tid; e < w * w; e += blockDim.x) {
      int rr = j + 1 + e / w, cc = j + 1 + e % w;
      if (cc <= rr) D[rr * LDS + cc] -= D[rr * LDS + j] * D[cc * LDS + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) fail[l] = 1;
    return;
  }
  if (ti == k) {
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int r = e / NB, c = e - r * NB;
      if (c <= r) A[(size_t)(k * NB + r) * np + k * NB + c] = D[r * LDS + c];
    }
    return;
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e - r * NB;
    B[r * LDS + c] = A[(size_t)(ti * NB + r) * np + k * NB + c];
  }
  __syncthreads();
  // X L_kk^T = B, row by row (each row independent)
  if (tid < NB) {
    double *x = B + tid * LDS;
    for (int c = 0; c < NB; c++) {
      double s = x[c];
      for (int cp = 0; cp < c; cp++) s -= x[cp] * D[c * LDS + cp];
      x[c] = s / D[c * LDS + c];
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e - r * NB;
    A[(size_t)(ti * NB + r) * np + k * NB + c] = B[r * LDS + c];
  }
}

__global__ void __launch_bounds__(256) k_syrk_update(double *S, const long long *S_off, const int *npad,
                                                     const int *run, const int *fail, int k) {
  int l = blockIdx.y;
  if (!run[l] || fail[l]) return;
  int np = npad[l];
  int T = np / NB;
  int rem = T - k - 1;
  if (rem <= 0) return;
  long long p = blockIdx.x;
  int a = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((long long)(a + 1) * (a + 2) / 2 <= p) a++;
  while ((long long)a * (a + 1) / 2 > p) a--;
  int b = (int)(p - (long long)a * (a + 1) / 2);
  if (a >= rem) return;
  int ti = k + 1 + a, tj = k + 1 + b;
  extern __shared__ double sm[];
  double *Li = sm, *Lj = sm + NB * LDS;
  double *A = S + S_off[l];
  int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e - r * NB;
    Li[r * LDS + c] = A[(size_t)(ti * NB + r) * np + k * NB + c];
    Lj[r * LDS + c] = A[(size_t)(tj * NB + r) * np + k * NB + c];
  }
  __syncthreads();
  int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
#pragma unroll 4
  for (int kk = 0; kk < NB; kk++) {
    double av[4], bv[4];
#pragma unroll
    for (int r = 0; r < 4; r++) av[r] = Li[(ty + 16 * r) * LDS + kk];
#pragma unroll
    for (int c = 0; c < 4; c++) bv[c] = Lj[(tx + 16 * c) * LDS + kk];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      size_t off = (size_t)(ti * NB + ty + 16 * r) * np + tj * NB + tx + 16 * c;
      A[off] -= acc[r][c];
    }
}

// forward L z = y (z stored in y) and backward L^T x = z (x stored in dC)
__global__ void __launch_bounds__(256) k_trsv(const double *S, const long long *S_off, const int *npad,
                                              const int *ycam_off, const int *run, const int *fail, double *y,
                                              double *dC) {
  int l = blockIdx.x;
  if (!run[l] || fail[l]) return;
  int np = npad[l];
  int T = np / NB;
  const double *A = S + S_off[l];
  double *z = y + ycam_off[l];
  double *x = dC + ycam_off[l];
  __shared__ double xs[NB];
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int kt = 0; kt < T; kt++) {
    int base = kt * NB;
    if (warp == 0) {
      for (int r = 0; r < NB; r++) {
        const double *row = A + (size_t)(base + r) * np + base;
        double s = 0.0;
        for (int c = lane; c < r; c += 32) s += row[c] * xs[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) xs[r] = (z[base + r] - s) / row[r];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = tid; r < NB; r += blockDim.x) z[base + r] = xs[r];
    for (int i = base + NB + warp; i < np; i += nw) {
      const double *row = A + (size_t)i * np + base;
      double s = row[lane] * xs[lane] + row[lane + 32] * xs[lane + 32];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) z[i] -= s;
    }
    __syncthreads();
  }
  for (int e = tid; e < np; e += blockDim.x) x[e] = z[e];
  __syncthreads();
  for (int kt = T - 1; kt >= 0; kt--) {
    int base = kt * NB;
    if (warp == 0) {
      for (int r = NB - 1; r >= 0; r--) {
        double s = 0.0;
        for (int c = r + 1 + lane; c < NB; c += 32) s += A[(size_t)(base + c) * np + base + r] * xs[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) xs[r] = (x[base + r] - s) / A[(size_t)(base + r) * np + base + r];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = tid; r < NB; r += blockDim.x) x[base + r] = xs[r];
    for (int c = tid; c < base; c += blockDim.x) {
      double s = 0.0;
      for (int r = 0; r < NB; r++) s += A[(size_t)(base + r) * np + c] * xs[r];
      x[c] -= s;
    }
    __syncthreads();
  }
}

rpba_status launch_solve_rcs(Ctx *ctx, const int *run_dev, int *fail_dev) {
  RPBA_CUDA(cudaMemsetAsync(fail_dev, 0, ctx->L * sizeof(int), ctx->stream));
  size_t smem = 2 * NB * LDS * sizeof(double);
  static bool attr_done = false;
  if (!attr_done) {
    RPBA_CUDA(cudaFuncSetAttribute(k_potrf_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RPBA_CUDA(cudaFuncSetAttribute(k_syrk_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done = true;
  }
  int T = ctx->max_tiles;
  for (int k = 0; k < T; k++) {
    dim3 gp(T - k, ctx->L);
    RPBA_KERNEL(ctx, "k_potrf_panel", k_potrf_panel<<<gp, 256, smem, ctx->stream>>>(ctx->S, ctx->S_off, ctx->npad, run_dev, fail_dev, k));
    int rem = T - k - 1;
    if (rem > 0) {
      dim3 gu((unsigned)((long long)rem * (rem + 1) / 2), ctx->L);
      RPBA_KERNEL(ctx, "k_syrk_update", k_syrk_update<<<gu, 256, smem, ctx->stream>>>(ctx->S, ctx->S_off, ctx->npad, run_dev, fail_dev, k));
    }
  }
  RPBA_KERNEL(ctx, "k_trsv", k_trsv<<<ctx->L, 256, 0, ctx->stream>>>(ctx->S, ctx->S_off, ctx->npad, ctx->ycam_off, run_dev, fail_dev, ctx->y,
                                          ctx->dC));
  return RPBA_OK;
}

}  // namespace rpba
