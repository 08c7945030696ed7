// gnn.cu -- learned preconditioner of PCG on the reduced camera system
// (solver 3) and the kernels that train it.
//
// The paper solves the RCS by conjugate gradients with block-Jacobi
// preconditioning, the inverses of the 6x6 camera blocks S_ii (Sec. 5.5). Here
// a graph network over the cameras of a sub-block (an edge where two cameras
// share a point, i.e. S_ij != 0) predicts a correction of every camera block
// and a gain for every camera pair:
//
//   x_i   = [log S_ii[k,k] - system mean (6), S_ii[k,l] / sqrt(S_ii[k,k] S_ii[l,l]), k > l (15)]
//   e_ij  = ||S_ij||_F / sqrt(||S_ii||_F ||S_jj||_F)
//   h0    = relu(W0 x + b0)
//   h_t   = relu(A_t h_{t-1} + B_t sum_j e_ij h_{t-1,j} + c_t),  t = 1..3  (width 64)
//   C_i   = Wo h3_i + bo  (21 values of a lower-triangular 6x6)
//   q_ij  = ws.(h3_i + h3_j) + wp.(h3_i * h3_j) + we e_ij + bq  (i > j)
//   M_i   = I + 0.5 tanh(C_i),  L_i = chol(S_ii),  N_ij = tanh(q_ij) L_i^-1 S_ij L_j^-T
//   G     = M^-1 (I - N) L^-1  (block lower triangular),  P^-1 = G^T G
//
// P^-1 is SPD for any parameters and is block-Jacobi when both heads are
// zero. Training minimises Kaporin's condition number of G S G^T per unit of
// dimension, log(tr(G S G^T) / d) - log det(G S G^T) / d, with the trace
// estimated from Gaussian probes; block-Jacobi minimises it among
// block-diagonal preconditioners, so the gain comes from the coupling N.
//
// Precision: weight matrices are read as BF16 (FP32 master copy for Adam),
// activations and accumulation FP32, the per-camera 6x6 algebra (features,
// Cholesky, factor, loss) FP64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rpba_internal.cuh"

namespace rpba {

// ---------------------------------------------------------------------------
// parameter layout: one flat vector W0, b0, (A_t, B_t, c_t) t = 1..3, Wo, bo,
// ws, wp, we, bq
// ---------------------------------------------------------------------------
constexpr int GNF = RPBA_GNN_FEATURES, GH = RPBA_GNN_HIDDEN, GNL = RPBA_GNN_LAYERS;
constexpr int G_W0 = 0, G_b0 = G_W0 + GH * GNF, G_L1 = G_b0 + GH, G_LSZ = 2 * GH * GH + GH;
constexpr int G_Wo = G_L1 + GNL * G_LSZ, G_bo = G_Wo + GNF * GH, G_ws = G_bo + GNF, G_wp = G_ws + GH,
              G_we = G_wp + GH, G_bq = G_we + 1, G_NPARAM = G_bq + 1;
constexpr int G_EDGE_PARAMS = 2 * GH + 2;
__host__ __device__ constexpr int g_A(int t) { return G_L1 + (t - 1) * G_LSZ; }
__host__ __device__ constexpr int g_B(int t) { return g_A(t) + GH * GH; }
__host__ __device__ constexpr int g_c(int t) { return g_B(t) + GH * GH; }
constexpr double G_EPS = 0.5;

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// node v belongs to system node_sys[v]; the system's matrix is the lower
// triangle of S + off[s] (row-major, leading dimension ld[s]); its nodes are
// node0[s] .. node0[s+1]-1 and node v is camera v - node0[s] of it
struct GSys {
  const double *S;
  const long long *off;
  const int *ld, *node0, *node_sys, *run;
};

__device__ inline double gsym(const GSys &g, int s, int r, int c) {
  const double *A = g.S + g.off[s];
  long long ld = g.ld[s];
  return r >= c ? A[r * ld + c] : A[c * ld + r];
}

__host__ __device__ inline int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// ---------------------------------------------------------------------------
// graph inputs
// ---------------------------------------------------------------------------
// per node: raw features (log-diagonal not yet centred), ||S_ii||_F and the
// packed Cholesky factor of S_ii (ok = 0 when S_ii is not positive definite)
__global__ void k_gnn_features(int n, GSys g, float *x, double *Lc, double *nrm, int *ok) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int s = g.node_sys[v];
  if (g.run && !g.run[s]) return;
  int b = 6 * (v - g.node0[s]);
  double B[6][6], f2 = 0.0;
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) {
      B[r][c] = gsym(g, s, b + r, b + c);
      f2 += B[r][c] * B[r][c];
    }
  double Lm[6][6];
  bool good = true;
  for (int j = 0; j < 6; j++) {
    double d = B[j][j];
    for (int k = 0; k < j; k++) d -= Lm[j][k] * Lm[j][k];
    if (!(d > 0.0)) { good = false; d = 1.0; }
    Lm[j][j] = sqrt(d);
    for (int i = j + 1; i < 6; i++) {
      double t = B[i][j];
      for (int k = 0; k < j; k++) t -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = t / Lm[j][j];
    }
  }
  for (int r = 0; r < 6; r++)
    for (int c = 0; c <= r; c++) Lc[21 * (size_t)v + tri(r, c)] = Lm[r][c];
  float *xv = x + 21 * (size_t)v;
  if (good) {
    for (int k = 0; k < 6; k++) xv[k] = (float)log(B[k][k]);
    int o = 6;
    for (int r = 1; r < 6; r++)
      for (int c = 0; c < r; c++) xv[o++] = (float)(B[r][c] / sqrt(B[r][r] * B[c][c]));
  } else {
    for (int k = 0; k < 21; k++) xv[k] = 0.0f;
  }
  nrm[v] = good ? sqrt(f2) : 0.0;
  ok[v] = good ? 1 : 0;
}

// per system: x[:, 0:6] -= their mean over the system's nodes
__global__ void __launch_bounds__(256) k_gnn_center(int nsys, GSys g, float *x) {
  int s = blockIdx.x;
  if (s >= nsys || (g.run && !g.run[s])) return;
  int a = g.node0[s], b = g.node0[s + 1];
  __shared__ double sh[6][8];
  __shared__ double mean[6];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int v = a + threadIdx.x; v < b; v += blockDim.x)
    for (int k = 0; k < 6; k++) acc[k] += x[21 * (size_t)v + k];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 6; k++) {
    double t = acc[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += sh[threadIdx.x][w];
    mean[threadIdx.x] = b > a ? t / (b - a) : 0.0;
  }
  __syncthreads();
  for (int v = a + threadIdx.x; v < b; v += blockDim.x)
    for (int k = 0; k < 6; k++) x[21 * (size_t)v + k] = (float)((double)x[21 * (size_t)v + k] - mean[k]);
}

// per CSR entry a = (row v, column u): e = ||S_vu||_F / sqrt(||S_vv||_F ||S_uu||_F)
__global__ void k_gnn_edges(int nnz, GSys g, const int *row, const int *adj, const double *nrm, float *e) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nnz) return;
  int v = row[a], u = adj[a];
  int s = g.node_sys[v];
  if (g.run && !g.run[s]) return;
  int bv = 6 * (v - g.node0[s]), bu = 6 * (u - g.node0[s]);
  double f2 = 0.0;
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) {
      double t = gsym(g, s, bv + r, bu + c);
      f2 += t * t;
    }
  double d = nrm[v] * nrm[u];
  e[a] = d > 0.0 ? (float)sqrt(f2 / d) : 0.0f;
}

// nz[i * n + j] = 1 when the block (i, j), i != j, of the system has a non-zero entry
__global__ void k_gnn_block_nz(int n, const double *S, int ld, uint8_t *nz) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
  if (i <= j) return;
  bool any = false;
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) any |= S[(size_t)(6 * i + r) * ld + 6 * j + c] != 0.0;
  nz[(size_t)i * n + j] = any;
  nz[(size_t)j * n + i] = any;
}

__device__ inline void fwd_lower(const double *Lc, double *y) {  // y <- L^-1 y, L packed
  for (int r = 0; r < 6; r++) {
    double t = y[r];
    for (int c = 0; c < r; c++) t -= Lc[tri(r, c)] * y[c];
    y[r] = t / Lc[tri(r, r)];
  }
}
__device__ inline void bwd_lower_t(const double *Lc, double *y) {  // y <- L^-T y
  for (int r = 5; r >= 0; r--) {
    double t = y[r];
    for (int c = r + 1; c < 6; c++) t -= Lc[tri(c, r)] * y[c];
    y[r] = t / Lc[tri(r, r)];
  }
}

// ---------------------------------------------------------------------------
// network layers
// ---------------------------------------------------------------------------
// out[v][o] = act(sum_k W1(o,k) in1[v][k] + sum_k W2(o,k) in2[v][k] + bias[o])
// W(o,k) = W[o k_in + k]; with TRANS, W(o,k) = W[k nout + o] (backward data).
// One CTA: 16 nodes x up to 64 outputs, weights staged in shared memory.
#define GL_NODES 16
template <bool TRANS>
__global__ void __launch_bounds__(256)
    k_gnn_linear(int n, const float *in1, int k1, const __nv_bfloat16 *W1, const float *in2, int k2,
                 const __nv_bfloat16 *W2, const float *bias, int nout, int relu, int accumulate, float *out) {
  __shared__ float w1s[GH][GH + 1], w2s[GH][GH + 1];
  __shared__ float i1s[GL_NODES][GH + 1], i2s[GL_NODES][GH + 1];
  int tid = threadIdx.x;
  for (int e = tid; e < nout * k1; e += blockDim.x) {
    int o = e / k1, k = e - o * k1;
    w1s[o][k] = __bfloat162float(TRANS ? W1[(size_t)k * nout + o] : W1[(size_t)o * k1 + k]);
  }
  if (in2)
    for (int e = tid; e < nout * k2; e += blockDim.x) {
      int o = e / k2, k = e - o * k2;
      w2s[o][k] = __bfloat162float(TRANS ? W2[(size_t)k * nout + o] : W2[(size_t)o * k2 + k]);
    }
  int v0 = blockIdx.x * GL_NODES;
  for (int e = tid; e < GL_NODES * k1; e += blockDim.x) {
    int j = e / k1, k = e - j * k1;
    i1s[j][k] = v0 + j < n ? in1[(size_t)(v0 + j) * k1 + k] : 0.0f;
  }
  if (in2)
    for (int e = tid; e < GL_NODES * k2; e += blockDim.x) {
      int j = e / k2, k = e - j * k2;
      i2s[j][k] = v0 + j < n ? in2[(size_t)(v0 + j) * k2 + k] : 0.0f;
    }
  __syncthreads();
  int o = tid & 63, grp = tid >> 6;  // 4 groups of 4 nodes
  if (o >= nout) return;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < k1; k++) {
    float w = w1s[o][k];
#pragma unroll
    for (int j = 0; j < 4; j++) acc[j] += w * i1s[4 * grp + j][k];
  }
  if (in2)
    for (int k = 0; k < k2; k++) {
      float w = w2s[o][k];
#pragma unroll
      for (int j = 0; j < 4; j++) acc[j] += w * i2s[4 * grp + j][k];
    }
  float b = bias ? bias[o] : 0.0f;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    int v = v0 + 4 * grp + j;
    if (v >= n) continue;
    float r = acc[j] + b;
    if (relu) r = fmaxf(r, 0.0f);
    float *po = out + (size_t)v * nout + o;
    *po = accumulate ? *po + r : r;
  }
}

// out[v] (+)= sum_{u ~ v} e_vu in[u]   (one warp per node, 64 features)
__global__ void k_gnn_aggregate(int n, const int *ptr, const int *adj, const float *e, const float *in, float *out,
                                int accumulate) {
  int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (v >= n) return;
  float a0 = 0.f, a1 = 0.f;
  for (int a = ptr[v]; a < ptr[v + 1]; a++) {
    int u = adj[a];
    float w = e[a];
    a0 += w * in[(size_t)u * GH + lane];
    a1 += w * in[(size_t)u * GH + lane + 32];
  }
  float *o = out + (size_t)v * GH;
  if (accumulate) { o[lane] += a0; o[lane + 32] += a1; }
  else { o[lane] = a0; o[lane + 32] = a1; }
}

__global__ void k_gnn_relu_bwd(long long n, const float *dh, const float *h, float *dz) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dz[i] = h[i] > 0.0f ? dh[i] : 0.0f;
}

// partial weight gradients of one CTA's nodes: part[blk][o][k] = sum_v dz[v][o] in[v][k],
// k = nin is the bias column (in = 1)
#define WG_NODES 128
#define WG_PER_THREAD 17  // ceil(64 * 65 / 256)
__global__ void __launch_bounds__(256) k_gnn_wgrad(int n, const float *dz, int nout, const float *in, int nin,
                                                   float *part) {
  __shared__ float dzs[16][GH + 1], ins[16][GH + 2];
  int tid = threadIdx.x;
  int tot = nout * (nin + 1);
  float acc[WG_PER_THREAD];
#pragma unroll
  for (int q = 0; q < WG_PER_THREAD; q++) acc[q] = 0.f;
  int base = blockIdx.x * WG_NODES, end = min(base + WG_NODES, n);
  for (int c0 = base; c0 < end; c0 += 16) {
    for (int e = tid; e < 16 * nout; e += blockDim.x) {
      int j = e / nout, o = e - j * nout;
      dzs[j][o] = c0 + j < end ? dz[(size_t)(c0 + j) * nout + o] : 0.f;
    }
    for (int e = tid; e < 16 * (nin + 1); e += blockDim.x) {
      int j = e / (nin + 1), k = e - j * (nin + 1);
      ins[j][k] = c0 + j < end ? (k < nin ? in[(size_t)(c0 + j) * nin + k] : 1.0f) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < WG_PER_THREAD; q++) {
      int idx = tid + 256 * q;
      if (idx < tot) {
        int o = idx / (nin + 1), k = idx - o * (nin + 1);
        float s = 0.f;
        for (int j = 0; j < 16; j++) s += dzs[j][o] * ins[j][k];
        acc[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < WG_PER_THREAD; q++) {
    int idx = tid + 256 * q;
    if (idx < tot) part[(size_t)blockIdx.x * tot + idx] = acc[q];
  }
}

// sum of the partials over the CTAs in a fixed order -> gW (nout x nin), gb (nout)
__global__ void k_gnn_wgrad_reduce(int nparts, int nout, int nin, const float *part, float *gW, float *gb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int tot = nout * (nin + 1);
  if (idx >= tot) return;
  double s = 0.0;
  for (int b = 0; b < nparts; b++) s += part[(size_t)b * tot + idx];
  int o = idx / (nin + 1), k = idx - o * (nin + 1);
  if (k < nin) gW[(size_t)o * nin + k] = (float)s;
  else gb[o] = (float)s;
}

// ---------------------------------------------------------------------------
// preconditioner factor: normalised couplings, edge gains, M^-1 L^-1, F
// ---------------------------------------------------------------------------
// per CSR entry a = (row v, column u < v): shat[a] = L_v^-1 S_vu L_u^-T (row-major 36)
__global__ void k_gnn_shat(int nnz, GSys g, const int *row, const int *adj, const double *Lc, double *shat) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nnz) return;
  int v = row[a], u = adj[a];
  if (u >= v) return;
  int s = g.node_sys[v];
  if (g.run && !g.run[s]) return;
  int bv = 6 * (v - g.node0[s]), bu = 6 * (u - g.node0[s]);
  const double *Lv = Lc + 21 * (size_t)v, *Lu = Lc + 21 * (size_t)u;
  double X[6][6];
  for (int c = 0; c < 6; c++) {  // X = L_v^-1 S_vu, column by column
    double y[6];
    for (int r = 0; r < 6; r++) y[r] = gsym(g, s, bv + r, bu + c);
    fwd_lower(Lv, y);
    for (int r = 0; r < 6; r++) X[r][c] = y[r];
  }
  double *o = shat + 36 * (size_t)a;
  for (int r = 0; r < 6; r++) {  // row r of X L_u^-T = (L_u^-1 X[r,:]^T)^T
    double y[6];
    for (int c = 0; c < 6; c++) y[c] = X[r][c];
    fwd_lower(Lu, y);
    for (int c = 0; c < 6; c++) o[6 * r + c] = y[c];
  }
}

// per CSR entry a = (row v, column u < v): gamma = tanh(ws.(h_v + h_u) + wp.(h_v * h_u) + we e + bq)
__global__ void k_gnn_edge_gain(int nnz, GSys g, const int *row, const int *adj, const float *e, const float *h,
                                const float *w, double *gam) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nnz) return;
  int v = row[a], u = adj[a];
  if (u >= v) return;
  if (g.run && !g.run[g.node_sys[v]]) return;
  const float *hv = h + (size_t)v * GH, *hu = h + (size_t)u * GH, *ws = w + G_ws, *wp = w + G_wp;
  float q = w[G_we] * e[a] + w[G_bq];
  for (int k = 0; k < GH; k++) q += ws[k] * (hv[k] + hu[k]) + wp[k] * hv[k] * hu[k];
  gam[a] = tanh((double)q);
}

// M = I + 0.5 tanh(C) (lower triangular), th = tanh(C)
__device__ inline void head_M(const float *C, double M[6][6], double th[21]) {
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) M[r][c] = 0.0;
  for (int r = 0; r < 6; r++)
    for (int c = 0; c <= r; c++) {
      th[tri(r, c)] = tanh((double)C[tri(r, c)]);
      M[r][c] = (r == c ? 1.0 : 0.0) + G_EPS * th[tri(r, c)];
    }
}
__device__ inline void fwd_M(const double M[6][6], double *y) {  // y <- M^-1 y
  for (int r = 0; r < 6; r++) {
    double t = y[r];
    for (int c = 0; c < r; c++) t -= M[r][c] * y[c];
    y[r] = t / M[r][r];
  }
}
__device__ inline void bwd_Mt(const double M[6][6], double *y) {  // y <- M^-T y
  for (int r = 5; r >= 0; r--) {
    double t = y[r];
    for (int c = r + 1; c < 6; c++) t -= M[c][r] * y[c];
    y[r] = t / M[r][r];
  }
}

// per node: D = M^-1 L^-1 and Li = L^-1 (36 each, FP32). A node whose S_vv
// is not positive definite fails its system; a non-finite D falls back to
// block-Jacobi (D = Li).
__global__ void k_gnn_head_node(int n, GSys g, const float *C, const double *Lc, const int *ok, float *D, float *Li,
                                int *fail) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int s = g.node_sys[v];
  if (g.run && !g.run[s]) return;
  if (!ok[v]) {
    if (fail) atomicExch(fail + s, 1);
    return;
  }
  const double *L = Lc + 21 * (size_t)v;
  double M[6][6], th[21], Lv[6][6], Dv[6][6];
  head_M(C + 21 * (size_t)v, M, th);
  bool finite = true;
  for (int c = 0; c < 6; c++) {
    double y[6] = {0, 0, 0, 0, 0, 0};
    y[c] = 1.0;
    fwd_lower(L, y);
    for (int r = 0; r < 6; r++) Lv[r][c] = y[r];
    fwd_M(M, y);
    for (int r = 0; r < 6; r++) {
      Dv[r][c] = y[r];
      finite &= isfinite(y[r]);
    }
  }
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) {
      D[36 * (size_t)v + 6 * r + c] = (float)(finite ? Dv[r][c] : Lv[r][c]);
      Li[36 * (size_t)v + 6 * r + c] = (float)Lv[r][c];
    }
}

// per CSR entry a = (row v, column u < v): F = gamma M_v^-1 shat (FP32; a
// non-finite block is dropped, F = 0)
__global__ void k_gnn_head_F(int nnz, GSys g, const int *row, const int *adj, const float *C, const double *shat,
                             const double *gam, float *F) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nnz) return;
  int v = row[a];
  if (adj[a] >= v) return;
  if (g.run && !g.run[g.node_sys[v]]) return;
  double M[6][6], th[21], Fa[6][6];
  head_M(C + 21 * (size_t)v, M, th);
  const double *Sh = shat + 36 * (size_t)a;
  bool finite = true;
  for (int c = 0; c < 6; c++) {
    double y[6];
    for (int r = 0; r < 6; r++) y[r] = gam[a] * Sh[6 * r + c];
    fwd_M(M, y);
    for (int r = 0; r < 6; r++) {
      Fa[r][c] = y[r];
      finite &= isfinite(y[r]);
    }
  }
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) F[36 * (size_t)a + 6 * r + c] = finite ? (float)Fa[r][c] : 0.0f;
}

// ---------------------------------------------------------------------------
// training loss (Kaporin's number with a probe estimate of the trace) and its
// gradient. Per node and probe the vectors are stored at ((v np + p) 6 + k).
// ---------------------------------------------------------------------------
// t = M_v^-T z
__global__ void k_gnn_loss_t(int n, int np, const float *C, const double *z, double *T) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * np) return;
  int v = idx / np;
  double M[6][6], th[21], y[6];
  head_M(C + 21 * (size_t)v, M, th);
  for (int k = 0; k < 6; k++) y[k] = z[6 * (size_t)idx + k];
  bwd_Mt(M, y);
  for (int k = 0; k < 6; k++) T[6 * (size_t)idx + k] = y[k];
}

// s_j = t_j - sum_{i > j} N_ij^T t_i ; v_j = L_j^-T s_j
__global__ void k_gnn_loss_v(int n, int np, const int *ptr, const int *adj, const int *mir, const double *Lc,
                             const double *shat, const double *gam, const double *T, double *V) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * np) return;
  int j = idx / np, p = idx - j * np;
  double s[6];
  for (int k = 0; k < 6; k++) s[k] = T[6 * (size_t)idx + k];
  for (int a = ptr[j]; a < ptr[j + 1]; a++) {
    int i = adj[a];
    if (i <= j) continue;
    int e = mir[a];
    const double *Sh = shat + 36 * (size_t)e;
    const double *ti = T + 6 * ((size_t)i * np + p);
    double gm = gam[e];
    for (int c = 0; c < 6; c++) {
      double t = 0.0;
      for (int r = 0; r < 6; r++) t += Sh[6 * r + c] * ti[r];
      s[c] -= gm * t;
    }
  }
  bwd_lower_t(Lc + 21 * (size_t)j, s);
  for (int k = 0; k < 6; k++) V[6 * (size_t)idx + k] = s[k];
}

// U = S V per system (one thread per matrix row and probe)
__global__ void k_gnn_loss_symv(int n, int np, const int *node_sys, const int *node0, const long long *soff,
                                const int *sdim, const double *S, const double *V, double *U) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 6LL * n * np) return;
  int p = (int)(idx % np);
  int row = (int)(idx / np);  // global row 6 v + k
  int v = row / 6, k = row - 6 * v;
  int s = node_sys[v];
  int g0 = node0[s], d = sdim[s];
  int lr = 6 * (v - g0) + k;
  const double *A = S + soff[s];
  double t = 0.0;
  for (int c = 0; c < d; c++) {
    double a = lr >= c ? A[(size_t)lr * d + c] : A[(size_t)c * d + lr];
    int u = c / 6;
    t += a * V[6 * ((size_t)(g0 + u) * np + p) + (c - 6 * u)];
  }
  U[6 * ((size_t)v * np + p) + k] = t;
}

// per system: T_s = (1/np) sum v.u, loss_s = log(T_s / d) + (2/d) sum_v log det(M_v L_v)
__global__ void __launch_bounds__(256) k_gnn_loss_sys(int nsys, int np, const int *node0, const int *sdim,
                                                      const float *C, const double *Lc, const double *V,
                                                      const double *U, double *Ts, double *loss_s) {
  int s = blockIdx.x;
  if (s >= nsys) return;
  int a = node0[s], b = node0[s + 1];
  double acc[2] = {0.0, 0.0};
  for (int v = a + threadIdx.x; v < b; v += blockDim.x) {
    for (int p = 0; p < np; p++)
      for (int k = 0; k < 6; k++) acc[0] += V[6 * ((size_t)v * np + p) + k] * U[6 * ((size_t)v * np + p) + k];
    for (int k = 0; k < 6; k++)
      acc[1] += log(1.0 + G_EPS * tanh((double)C[21 * (size_t)v + tri(k, k)])) + log(Lc[21 * (size_t)v + tri(k, k)]);
  }
  __shared__ double sh[2][8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = 0; e < 2; e++) {
    double t = acc[e];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[e][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ld = 0.0;
    for (int w = 0; w < 8; w++) { tr += sh[0][w]; ld += sh[1][w]; }
    tr /= np;
    double d = sdim[s];
    Ts[s] = tr;
    loss_s[s] = log(tr / d) + 2.0 * ld / d;
  }
}

__global__ void k_gnn_loss_total(int nsys, const double *loss_s, double *out) {
  if (blockIdx.x || threadIdx.x) return;
  double t = 0.0;
  for (int s = 0; s < nsys; s++) t += loss_s[s];
  *out = nsys ? t / nsys : 0.0;
}

// sbar = L^-1 vbar, vbar = 2 u / (np T_s nsys)
__global__ void k_gnn_loss_sbar(int n, int np, int nsys, const int *node_sys, const double *Lc, const double *Ts,
                                const double *U, double *SB) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * np) return;
  int v = idx / np;
  double c = 2.0 / (np * Ts[node_sys[v]] * nsys);
  double y[6];
  for (int k = 0; k < 6; k++) y[k] = c * U[6 * (size_t)idx + k];
  fwd_lower(Lc + 21 * (size_t)v, y);
  for (int k = 0; k < 6; k++) SB[6 * (size_t)idx + k] = y[k];
}

// per node i: tbar = sbar_i - sum_{j<i} N_ij sbar_j, Mbar = -sum_p t (M^-1 tbar)^T
// + (2 / (d nsys)) diag(1 / M_kk), dC = Mbar * 0.5 (1 - th^2); per lower entry
// qbar = -(1 - gamma^2) sum_p t_i^T shat sbar_j
__global__ void k_gnn_loss_node_bwd(int n, int np, int nsys, const int *node_sys, const int *sdim, const int *ptr,
                                    const int *adj, const float *C, const double *shat, const double *gam,
                                    const double *T, const double *SB, float *dC, float *qbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double M[6][6], th[21], Mb[6][6];
  head_M(C + 21 * (size_t)i, M, th);
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) Mb[r][c] = 0.0;
  for (int a = ptr[i]; a < ptr[i + 1]; a++)
    if (adj[a] < i) qbar[a] = 0.0f;
  for (int p = 0; p < np; p++) {
    const double *ti = T + 6 * ((size_t)i * np + p);
    double tb[6];
    for (int k = 0; k < 6; k++) tb[k] = SB[6 * ((size_t)i * np + p) + k];
    for (int a = ptr[i]; a < ptr[i + 1]; a++) {
      int j = adj[a];
      if (j >= i) continue;
      const double *Sh = shat + 36 * (size_t)a;
      const double *sj = SB + 6 * ((size_t)j * np + p);
      double gsum = 0.0;
      for (int r = 0; r < 6; r++) {
        double t = 0.0;
        for (int c = 0; c < 6; c++) t += Sh[6 * r + c] * sj[c];
        tb[r] -= gam[a] * t;
        gsum += ti[r] * t;
      }
      qbar[a] -= (float)(gsum * (1.0 - gam[a] * gam[a]));
    }
    fwd_M(M, tb);  // M^-1 tbar
    for (int r = 0; r < 6; r++)
      for (int c = 0; c <= r; c++) Mb[r][c] -= ti[r] * tb[c];
  }
  double dd = 2.0 / ((double)sdim[node_sys[i]] * nsys);
  float *o = dC + 21 * (size_t)i;
  for (int r = 0; r < 6; r++)
    for (int c = 0; c <= r; c++) {
      double m = Mb[r][c] + (r == c ? dd / M[r][r] : 0.0);
      double t = th[tri(r, c)];
      o[tri(r, c)] = (float)(m * G_EPS * (1.0 - t * t));
    }
}

// edge head backward, one warp per node v: dh_v += sum over v's entries of
// qbar (ws + wp * h_u); per-node partial gradients of ws, wp, we, bq from the
// node's lower entries -> EP[v][130]
__global__ void k_gnn_edge_bwd(int n, const int *ptr, const int *adj, const int *mir, const float *e, const float *h,
                               const float *w, const float *qbar, float *dh, float *EP) {
  int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (v >= n) return;
  const float *hv = h + (size_t)v * GH;
  float d0 = 0.f, d1 = 0.f, s0 = 0.f, s1 = 0.f, p0 = 0.f, p1 = 0.f, se = 0.f, sb = 0.f;
  float ws0 = w[G_ws + lane], ws1 = w[G_ws + lane + 32], wp0 = w[G_wp + lane], wp1 = w[G_wp + lane + 32];
  for (int a = ptr[v]; a < ptr[v + 1]; a++) {
    int u = adj[a];
    bool low = u < v;
    float qb = qbar[low ? a : mir[a]];
    const float *hu = h + (size_t)u * GH;
    float hu0 = hu[lane], hu1 = hu[lane + 32];
    d0 += qb * (ws0 + wp0 * hu0);
    d1 += qb * (ws1 + wp1 * hu1);
    if (low) {
      s0 += qb * (hv[lane] + hu0);
      s1 += qb * (hv[lane + 32] + hu1);
      p0 += qb * hv[lane] * hu0;
      p1 += qb * hv[lane + 32] * hu1;
      se += qb * e[a];
      sb += qb;
    }
  }
  dh[(size_t)v * GH + lane] += d0;
  dh[(size_t)v * GH + lane + 32] += d1;
  float *o = EP + (size_t)v * G_EDGE_PARAMS;
  o[lane] = s0;
  o[lane + 32] = s1;
  o[GH + lane] = p0;
  o[GH + lane + 32] = p1;
  if (lane == 0) {
    o[2 * GH] = se;
    o[2 * GH + 1] = sb;
  }
}

// out[c] = sum_v in[v][c] in node order
__global__ void k_gnn_colsum(int n, int ncol, const float *in, float *out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double t = 0.0;
  for (int v = 0; v < n; v++) t += in[(size_t)v * ncol + c];
  out[c] = (float)t;
}

// z[i] ~ N(0, 1) from a counter: splitmix64 (Steele, Lea, Flood 2014) of
// (seed, step, i), its two 32-bit halves as uniforms, Box-Muller
__device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
__global__ void k_gnn_draw_probes(long long nz, uint64_t seed, uint64_t step, double *z) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nz) return;
  uint64_t r = splitmix64(splitmix64(seed ^ (step * 0xD1B54A32D192ED03ULL)) + (uint64_t)i);
  double u1 = ((double)(r >> 32) + 0.5) * (1.0 / 4294967296.0);
  double u2 = ((double)(r & 0xFFFFFFFFULL) + 0.5) * (1.0 / 4294967296.0);
  z[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__global__ void k_gnn_adam(int np, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                           float eps, float c1, float c2, __nv_bfloat16 *wb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float mi = b1 * m[i] + (1.f - b1) * g[i];
  float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_gnn_to_bf16(int np, const float *w, __nv_bfloat16 *wb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) wb[i] = __float2bfloat16_rn(w[i]);
}

// ---------------------------------------------------------------------------
// forward pass (host side)
// ---------------------------------------------------------------------------
// launches one kernel: counted and timed on a context, error-checked otherwise
struct KL {
  Ctx *ctx = nullptr;
  std::string *err = nullptr;
  template <class F>
  rpba_status operator()(const char *name, F f) {
    if (ctx) {
      RPBA_KERNEL(ctx, name, f());
      return RPBA_OK;
    }
    f();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      *err = std::string(name) + ": " + cudaGetErrorString(e);
      return RPBA_ERR_CUDA;
    }
    return RPBA_OK;
  }
};

struct GnnNet {
  const float *w = nullptr;            // FP32 parameters (biases and the edge head)
  const __nv_bfloat16 *wb = nullptr;   // BF16 copy (weight matrices)
};

struct GnnAct {  // graph and activations of n nodes
  int n = 0;
  const int *ptr = nullptr, *adj = nullptr;
  const float *e = nullptr, *x = nullptr;
  float *h[GNL + 1] = {}, *m[GNL] = {}, *C = nullptr;
};

static rpba_status gnn_forward(KL &kl, const GnnNet &net, const GnnAct &a, cudaStream_t st) {
  int n = a.n;
  if (n == 0) return RPBA_OK;
  int gl = nblk(n, GL_NODES);
  RPBA_TRY(kl("k_gnn_linear", [&] {
    k_gnn_linear<false><<<gl, 256, 0, st>>>(n, a.x, GNF, net.wb + G_W0, nullptr, 0, nullptr, net.w + G_b0, GH, 1, 0,
                                            a.h[0]);
  }));
  for (int t = 1; t <= GNL; t++) {
    RPBA_TRY(kl("k_gnn_aggregate", [&] {
      k_gnn_aggregate<<<nblk((long long)n * 32, 256), 256, 0, st>>>(n, a.ptr, a.adj, a.e, a.h[t - 1], a.m[t - 1], 0);
    }));
    RPBA_TRY(kl("k_gnn_linear", [&] {
      k_gnn_linear<false><<<gl, 256, 0, st>>>(n, a.h[t - 1], GH, net.wb + g_A(t), a.m[t - 1], GH, net.wb + g_B(t),
                                              net.w + g_c(t), GH, 1, 0, a.h[t]);
    }));
  }
  RPBA_TRY(kl("k_gnn_linear", [&] {
    k_gnn_linear<false><<<gl, 256, 0, st>>>(n, a.h[GNL], GH, net.wb + G_Wo, nullptr, 0, nullptr, net.w + G_bo, GNF, 0,
                                            0, a.C);
  }));
  return RPBA_OK;
}

// graph inputs, network and factor of the systems in g (every node of a
// running system): features, centring, edge weights, couplings, forward,
// gains, D / Li / F
struct GnnInputs {
  int n = 0, nsys = 0, nnz = 0;
  GSys g;
  const int *ptr = nullptr, *adj = nullptr, *row = nullptr;
  float *x = nullptr, *e = nullptr;
  double *Lc = nullptr, *nrm = nullptr, *shat = nullptr, *gam = nullptr;
  int *ok = nullptr;
};

static rpba_status gnn_inputs(KL &kl, const GnnInputs &in, cudaStream_t st) {
  int n = in.n;
  if (n == 0) return RPBA_OK;
  RPBA_TRY(kl("k_gnn_features", [&] {
    k_gnn_features<<<nblk(n, 128), 128, 0, st>>>(n, in.g, in.x, in.Lc, in.nrm, in.ok);
  }));
  RPBA_TRY(kl("k_gnn_center", [&] { k_gnn_center<<<in.nsys, 256, 0, st>>>(in.nsys, in.g, in.x); }));
  if (in.nnz == 0) return RPBA_OK;
  RPBA_TRY(kl("k_gnn_edges", [&] {
    k_gnn_edges<<<nblk(in.nnz, 128), 128, 0, st>>>(in.nnz, in.g, in.row, in.adj, in.nrm, in.e);
  }));
  RPBA_TRY(kl("k_gnn_shat", [&] {
    k_gnn_shat<<<nblk(in.nnz, 128), 128, 0, st>>>(in.nnz, in.g, in.row, in.adj, in.Lc, in.shat);
  }));
  return RPBA_OK;
}

}  // namespace rpba

using namespace rpba;

// ---------------------------------------------------------------------------
// solver 3 inside a context
// ---------------------------------------------------------------------------
namespace rpba {

// camera graph of every sub-block in sub-block order (CSR, sorted rows, and
// the position of every entry's reverse), from the cameras of every point
// instance; built at create for solver 3
void build_camera_graph(Ctx *ctx, const std::vector<int> &inst_obs_ptr, const std::vector<int> &obs_cam_sorted,
                        const std::vector<int> &inst_sub, const std::vector<int> &cam_local) {
  int L = ctx->L, M = ctx->M;
  std::vector<int> &ptr = ctx->h_nadj_ptr, &adj = ctx->h_nadj, &mir = ctx->h_nadj_mir;
  ptr.assign(M + 1, 0);
  adj.clear();
  std::vector<std::vector<int>> nb(M);
  int P = (int)inst_sub.size();
  for (int l = 0, q = 0; l < L; l++) {
    int n = ctx->h_sub_cam_ptr[l + 1] - ctx->h_sub_cam_ptr[l];
    std::vector<uint8_t> bit((size_t)n * n, 0);
    for (; q < P && inst_sub[q] == l; q++)
      for (int a = inst_obs_ptr[q]; a < inst_obs_ptr[q + 1]; a++)
        for (int b = inst_obs_ptr[q]; b < inst_obs_ptr[q + 1]; b++) {
          int la = cam_local[obs_cam_sorted[a]], lb = cam_local[obs_cam_sorted[b]];
          if (la != lb) bit[(size_t)la * n + lb] = 1;
        }
    int g0 = ctx->h_sub_cam_ptr[l];
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++)
        if (bit[(size_t)i * n + j]) nb[g0 + i].push_back(g0 + j);
  }
  for (int v = 0; v < M; v++) {
    ptr[v + 1] = ptr[v] + (int)nb[v].size();
    adj.insert(adj.end(), nb[v].begin(), nb[v].end());
  }
  mir.assign(adj.size(), 0);
  ctx->h_nadj_row.assign(adj.size(), 0);
  for (int v = 0; v < M; v++)
    for (int a = ptr[v]; a < ptr[v + 1]; a++) {
      ctx->h_nadj_row[a] = v;
      int u = adj[a];
      mir[a] = (int)(std::lower_bound(adj.begin() + ptr[u], adj.begin() + ptr[u + 1], v) - adj.begin());
    }
}

template <typename T>
static rpba_status ctx_upload(Ctx *ctx, T **p, const T *host, size_t n) {
  RPBA_TRY(ctx_alloc(ctx, (void **)p, std::max<size_t>(n, 1) * sizeof(T)));
  if (n) RPBA_CUDA(cudaMemcpyAsync(*p, host, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return RPBA_OK;
}

static rpba_status gnn_ctx_buffers(Ctx *ctx) {
  if (ctx->gnn_h) return RPBA_OK;
  int M = std::max(ctx->M, 1);
  size_t nnz = std::max<size_t>(ctx->h_nadj.size(), 1);
  std::vector<int> ns(ctx->M);
  for (int l = 0; l < ctx->L; l++)
    for (int g = ctx->h_sub_cam_ptr[l]; g < ctx->h_sub_cam_ptr[l + 1]; g++) ns[g] = l;
  RPBA_TRY(ctx_upload(ctx, &ctx->node_sys, ns.data(), ns.size()));
  RPBA_TRY(ctx_upload(ctx, &ctx->nadj_ptr, ctx->h_nadj_ptr.data(), ctx->h_nadj_ptr.size()));
  RPBA_TRY(ctx_upload(ctx, &ctx->nadj, ctx->h_nadj.data(), ctx->h_nadj.size()));
  RPBA_TRY(ctx_upload(ctx, &ctx->nadj_mir, ctx->h_nadj_mir.data(), ctx->h_nadj_mir.size()));
  RPBA_TRY(ctx_upload(ctx, &ctx->nadj_row, ctx->h_nadj_row.data(), ctx->h_nadj_row.size()));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_w, G_NPARAM * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, &ctx->gnn_wb, G_NPARAM * sizeof(__nv_bfloat16)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_x, (size_t)M * GNF * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_e, nnz * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_h, (size_t)M * GH * (2 * GNL + 1) * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_C, (size_t)M * GNF * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_L, (size_t)M * 21 * sizeof(double)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_nrm, (size_t)M * sizeof(double)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_shat, nnz * 36 * sizeof(double)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_gam, nnz * sizeof(double)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_ok, (size_t)M * sizeof(int)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->pcg_D32, (size_t)M * 36 * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->pcg_Li32, (size_t)M * 36 * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->pcg_F32, nnz * 36 * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_rh, (size_t)M * 6 * sizeof(float)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->gnn_y, (size_t)M * 6 * sizeof(float)));
  std::vector<int> nvo(ctx->M);
  std::vector<int> yoff(ctx->L);
  RPBA_CUDA(cudaMemcpyAsync(yoff.data(), ctx->ycam_off, ctx->L * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l < ctx->L; l++)
    for (int g = ctx->h_sub_cam_ptr[l]; g < ctx->h_sub_cam_ptr[l + 1]; g++)
      nvo[g] = yoff[l] + 6 * (g - ctx->h_sub_cam_ptr[l]);
  RPBA_TRY(ctx_upload(ctx, &ctx->node_voff, nvo.data(), nvo.size()));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->pcg_run2, (size_t)std::max(ctx->L, 1) * sizeof(int)));
  RPBA_TRY(ctx_alloc(ctx, (void **)&ctx->pcg_fail2, (size_t)std::max(ctx->L, 1) * sizeof(int)));
  return RPBA_OK;
}

__global__ void k_or_flags(int L, const int *a, int *b) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < L && a[l]) b[l] = 1;
}

// run2[l] = the sub-block ran, did not fail and did not reach the tolerance
__global__ void k_pcg_unconverged(int L, const int *run, const int *fail, const double *st, double tol, int *run2,
                                  int *count) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  int r = run[l] && !fail[l] && !(st[4 * l + 2] <= tol);
  run2[l] = r;
  if (r) atomicAdd(count, 1);
}

// learned preconditioner for this LM iteration: network inference on the
// current RCS and the factor G; fills F (failure flags reset first)
rpba_status learned_setup(Ctx *ctx, const int *run_dev, int *fail_dev, FsaiApply *F) {
  if (!ctx->gnn_ready) {
    ctx->err = "solver 3 needs the network weights (rpba_set_gnn_weights)";
    return RPBA_ERR_STATE;
  }
  cudaStream_t st = ctx->stream;
  int M = ctx->M, L = ctx->L;
  RPBA_CUDA(cudaMemsetAsync(fail_dev, 0, L * sizeof(int), st));
  KL kl{ctx, &ctx->err};
  GSys g{ctx->S, ctx->S_off, ctx->npad, ctx->sub_cam_ptr, ctx->node_sys, run_dev};
  FsaiView P{ctx->nadj_ptr, ctx->nadj, ctx->nadj_mir, ctx->pcg_D32, ctx->pcg_Li32, ctx->pcg_F32};
  if (M) {
    GnnInputs in;
    int nnz = (int)ctx->h_nadj.size();
    in.n = M;
    in.nsys = L;
    in.nnz = nnz;
    in.g = g;
    in.ptr = ctx->nadj_ptr;
    in.adj = ctx->nadj;
    in.row = ctx->nadj_row;
    in.x = ctx->gnn_x;
    in.e = ctx->gnn_e;
    in.Lc = ctx->gnn_L;
    in.nrm = ctx->gnn_nrm;
    in.shat = ctx->gnn_shat;
    in.gam = ctx->gnn_gam;
    in.ok = ctx->gnn_ok;
    RPBA_TRY(gnn_inputs(kl, in, st));
    GnnNet net{ctx->gnn_w, (const __nv_bfloat16 *)ctx->gnn_wb};
    GnnAct a;
    a.n = M;
    a.ptr = ctx->nadj_ptr;
    a.adj = ctx->nadj;
    a.e = ctx->gnn_e;
    a.x = ctx->gnn_x;
    for (int t = 0; t <= GNL; t++) a.h[t] = ctx->gnn_h + (size_t)t * M * GH;
    for (int t = 0; t < GNL; t++) a.m[t] = ctx->gnn_h + (size_t)(GNL + 1 + t) * M * GH;
    a.C = ctx->gnn_C;
    RPBA_TRY(gnn_forward(kl, net, a, st));
    if (nnz)
      RPBA_TRY(kl("k_gnn_edge_gain", [&] {
        k_gnn_edge_gain<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, ctx->nadj_row, ctx->nadj, ctx->gnn_e, a.h[GNL],
                                                        ctx->gnn_w, ctx->gnn_gam);
      }));
    RPBA_TRY(kl("k_gnn_head_node", [&] {
      k_gnn_head_node<<<nblk(M, 128), 128, 0, st>>>(M, g, ctx->gnn_C, ctx->gnn_L, ctx->gnn_ok, ctx->pcg_D32,
                                                    ctx->pcg_Li32, fail_dev);
    }));
    if (nnz)
      RPBA_TRY(kl("k_gnn_head_F", [&] {
        k_gnn_head_F<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, ctx->nadj_row, ctx->nadj, ctx->gnn_C, ctx->gnn_shat,
                                                     ctx->gnn_gam, ctx->pcg_F32);
      }));
  }
  F->M = M;
  F->node_sys = ctx->node_sys;
  F->nvo = ctx->node_voff;
  F->P = P;
  F->rh = ctx->gnn_rh;
  F->y = ctx->gnn_y;
  return RPBA_OK;
}

// fallback: a sub-block the learned preconditioner did not bring to pcg_tol is
// solved again with block-Jacobi PCG (reads a count on the host)
rpba_status learned_fallback(Ctx *ctx, const int *run_dev, int *fail_dev) {
  cudaStream_t st = ctx->stream;
  int L = ctx->L;
  KL kl{ctx, &ctx->err};
  RPBA_CUDA(cudaMemsetAsync(ctx->counters + 9, 0, sizeof(int), st));
  RPBA_TRY(kl("k_pcg_unconverged", [&] {
    k_pcg_unconverged<<<nblk(L, 128), 128, 0, st>>>(L, run_dev, fail_dev, ctx->pcg_st, ctx->opt.pcg_tol,
                                                    ctx->pcg_run2, ctx->counters + 9);
  }));
  RPBA_CUDA(cudaMemcpyAsync(ctx->h_pinned_counter + 9, ctx->counters + 9, sizeof(int), cudaMemcpyDeviceToHost, st));
  RPBA_CUDA(cudaStreamSynchronize(st));
  int nfb = ctx->h_pinned_counter[9];
  if (nfb > 0) {
    ctx->gnn_fallbacks += nfb;
    // the block-Jacobi pass resets the failure flags: keep those of this pass
    RPBA_CUDA(cudaMemcpyAsync(ctx->pcg_fail2, fail_dev, L * sizeof(int), cudaMemcpyDeviceToDevice, st));
    RPBA_TRY(launch_pcg_blockjacobi(ctx, ctx->pcg_run2, fail_dev));
    RPBA_TRY(kl("k_or_flags", [&] { k_or_flags<<<nblk(L, 128), 128, 0, st>>>(L, ctx->pcg_fail2, fail_dev); }));
  }
  return RPBA_OK;
}

rpba_status launch_pcg_learned(Ctx *ctx, const int *run_dev, int *fail_dev) {
  FsaiApply F;
  RPBA_TRY(learned_setup(ctx, run_dev, fail_dev, &F));
  RPBA_TRY(pcg_iterate(ctx, run_dev, fail_dev, &F));
  return learned_fallback(ctx, run_dev, fail_dev);
}

}  // namespace rpba

// ---------------------------------------------------------------------------
// trainer
// ---------------------------------------------------------------------------
struct rpba_gnn {
  int dev = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr;
  int t = 0;
  // dataset, host mirror: systems (dense S), graph, features, factors, probes
  int n = 0, nsys = 0, np = 0;
  std::vector<int> h_ptr{0}, h_adj, h_mir, h_row, h_node0{0}, h_node_sys, h_sdim;
  std::vector<long long> h_soff;
  std::vector<float> h_e, h_x;
  std::vector<double> h_L, h_shat, h_z, h_S;
  // device copies and work buffers (rebuilt when the dataset grows)
  bool dirty = true;
  std::vector<void *> dbufs;
  int *ptr = nullptr, *adj = nullptr, *mir = nullptr, *row = nullptr, *node0 = nullptr, *node_sys = nullptr,
      *sdim = nullptr;
  long long *soff = nullptr;
  float *e = nullptr, *x = nullptr;
  double *L = nullptr, *shat = nullptr, *z = nullptr, *S = nullptr;
  float *act = nullptr, *C = nullptr, *dC = nullptr, *dh = nullptr, *dz = nullptr, *tmp = nullptr, *part = nullptr,
        *qbar = nullptr, *EP = nullptr;
  double *gam = nullptr, *T = nullptr, *V = nullptr, *U = nullptr, *SB = nullptr, *Ts = nullptr, *loss_s = nullptr,
         *loss = nullptr;
  float *D = nullptr, *Li = nullptr, *F = nullptr;
};

namespace {

#define GNN_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      G->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return RPBA_ERR_CUDA;                                                   \
    }                                                                         \
  } while (0)

// splitmix64 (Steele, Lea, Flood 2014) and Box-Muller normals
struct Rng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    double u1 = uniform(), u2 = uniform();
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
};

rpba_status galloc(rpba_gnn *G, void **p, size_t bytes) {
  GNN_CUDA(cudaMalloc(p, std::max<size_t>(bytes, 16)));
  G->dbufs.push_back(*p);
  return RPBA_OK;
}

void free_dataset(rpba_gnn *G) {
  for (void *p : G->dbufs) cudaFree(p);
  G->dbufs.clear();
}

// one system whose dense matrix (lower triangle, leading dimension ld) is on
// the device: graph, features, factors and couplings derived on the device
// and appended to the host mirror with the matrix itself and the probes
rpba_status add_dense(rpba_gnn *G, const double *S, int ld, int ncam, int np, const double *zh, cudaStream_t st) {
  if (ncam <= 0) return RPBA_OK;
  int dim = 6 * ncam;
  std::vector<void *> tmp;
  rpba_status s = RPBA_OK;
  auto cleanup = [&]() {
    for (void *p : tmp) cudaFree(p);
    tmp.clear();
  };
  auto talloc = [&](void **p, size_t b) -> rpba_status {
    cudaError_t e_ = cudaMalloc(p, std::max<size_t>(b, 16));
    if (e_ != cudaSuccess) {
      G->err = std::string("cudaMalloc: ") + cudaGetErrorString(e_);
      return RPBA_ERR_CUDA;
    }
    tmp.push_back(*p);
    return RPBA_OK;
  };
  auto fail = [&](cudaError_t e_) -> rpba_status {
    G->err = cudaGetErrorString(e_);
    cleanup();
    return RPBA_ERR_CUDA;
  };
  uint8_t *nz;
  int *node_sys, *node0, *ld_d, *ok, *ptr_d, *adj_d;
  long long *off;
  float *x, *e;
  double *Lc, *nrm, *shat;
#define TA(p, b)                                           \
  if ((s = talloc((void **)&(p), (b))) != RPBA_OK) {      \
    cleanup();                                             \
    return s;                                              \
  }
  TA(nz, (size_t)ncam * ncam);
  TA(node_sys, ncam * sizeof(int));
  TA(node0, 2 * sizeof(int));
  TA(ld_d, sizeof(int));
  TA(off, sizeof(long long));
  TA(ok, ncam * sizeof(int));
  TA(x, (size_t)ncam * 21 * sizeof(float));
  TA(Lc, (size_t)ncam * 21 * sizeof(double));
  TA(nrm, ncam * sizeof(double));
  cudaError_t ce;
  int h0[2] = {0, ncam};
  long long o0 = 0;
  if ((ce = cudaMemsetAsync(nz, 0, (size_t)ncam * ncam, st)) != cudaSuccess) return fail(ce);
  if ((ce = cudaMemsetAsync(node_sys, 0, ncam * sizeof(int), st)) != cudaSuccess) return fail(ce);
  if ((ce = cudaMemcpyAsync(node0, h0, sizeof(h0), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(ce);
  if ((ce = cudaMemcpyAsync(ld_d, &ld, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(ce);
  if ((ce = cudaMemcpyAsync(off, &o0, sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(ce);
  k_gnn_block_nz<<<nblk((long long)ncam * ncam, 256), 256, 0, st>>>(ncam, S, ld, nz);
  std::vector<uint8_t> hnz((size_t)ncam * ncam);
  if ((ce = cudaMemcpyAsync(hnz.data(), nz, hnz.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(ce);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return fail(ce);
  std::vector<int> hp(ncam + 1, 0), ha;
  for (int i = 0; i < ncam; i++) {
    for (int j = 0; j < ncam; j++)
      if (hnz[(size_t)i * ncam + j]) ha.push_back(j);
    hp[i + 1] = (int)ha.size();
  }
  int nnz = (int)ha.size();
  std::vector<int> hr(nnz);
  for (int i = 0; i < ncam; i++)
    for (int a = hp[i]; a < hp[i + 1]; a++) hr[a] = i;
  int *row_d;
  TA(ptr_d, (ncam + 1) * sizeof(int));
  TA(adj_d, std::max(nnz, 1) * sizeof(int));
  TA(row_d, std::max(nnz, 1) * sizeof(int));
  TA(e, std::max(nnz, 1) * sizeof(float));
  TA(shat, (size_t)std::max(nnz, 1) * 36 * sizeof(double));
#undef TA
  if ((ce = cudaMemcpyAsync(ptr_d, hp.data(), hp.size() * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(ce);
  if (nnz && (ce = cudaMemcpyAsync(adj_d, ha.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(ce);
  if (nnz && (ce = cudaMemcpyAsync(row_d, hr.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(ce);
  GSys g{S, off, ld_d, node0, node_sys, nullptr};
  k_gnn_features<<<nblk(ncam, 128), 128, 0, st>>>(ncam, g, x, Lc, nrm, ok);
  k_gnn_center<<<1, 256, 0, st>>>(1, g, x);
  if (nnz) {
    k_gnn_edges<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, row_d, adj_d, nrm, e);
    k_gnn_shat<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, row_d, adj_d, Lc, shat);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return fail(ce);
  std::vector<int> hok(ncam);
  size_t n0 = G->h_x.size() / 21, e0 = G->h_e.size(), s0 = G->h_S.size();
  G->h_x.resize((n0 + ncam) * 21);
  G->h_L.resize((n0 + ncam) * 21);
  G->h_e.resize(e0 + nnz);
  G->h_shat.resize((e0 + nnz) * 36);
  G->h_S.resize(s0 + (size_t)dim * dim);
  if ((ce = cudaMemcpyAsync(hok.data(), ok, ncam * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(G->h_x.data() + n0 * 21, x, (size_t)ncam * 21 * sizeof(float), cudaMemcpyDeviceToHost,
                            st)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(G->h_L.data() + n0 * 21, Lc, (size_t)ncam * 21 * sizeof(double), cudaMemcpyDeviceToHost,
                            st)) != cudaSuccess ||
      (nnz && (ce = cudaMemcpyAsync(G->h_e.data() + e0, e, nnz * sizeof(float), cudaMemcpyDeviceToHost, st)) !=
                  cudaSuccess) ||
      (nnz && (ce = cudaMemcpyAsync(G->h_shat.data() + e0 * 36, shat, (size_t)nnz * 36 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
      (ce = cudaMemcpy2DAsync(G->h_S.data() + s0, dim * sizeof(double), S, (size_t)ld * sizeof(double),
                              dim * sizeof(double), dim, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
    G->h_x.resize(n0 * 21);
    G->h_L.resize(n0 * 21);
    G->h_e.resize(e0);
    G->h_shat.resize(e0 * 36);
    G->h_S.resize(s0);
    return fail(ce);
  }
  cleanup();
  for (int v = 0; v < ncam; v++)
    if (!hok[v]) {
      G->h_x.resize(n0 * 21);
      G->h_L.resize(n0 * 21);
      G->h_e.resize(e0);
      G->h_shat.resize(e0 * 36);
      G->h_S.resize(s0);
      G->err = "a diagonal camera block is not positive definite";
      return RPBA_ERR_NUMERIC;
    }
  int base = (int)n0;
  for (int i = 0; i < ncam; i++) {
    G->h_ptr.push_back(G->h_ptr.back() + (hp[i + 1] - hp[i]));
    G->h_node_sys.push_back(G->nsys);
  }
  for (int j : ha) G->h_adj.push_back(base + j);
  for (int r : hr) G->h_row.push_back(base + r);
  for (int i = 0; i < ncam; i++)
    for (int a = hp[i]; a < hp[i + 1]; a++) {
      int j = ha[a];
      int r = (int)(std::lower_bound(ha.begin() + hp[j], ha.begin() + hp[j + 1], i) - ha.begin());
      G->h_mir.push_back((int)e0 + r);
    }
  // probes in node-major layout ((v np + p) 6 + k)
  size_t z0 = G->h_z.size();
  G->h_z.resize(z0 + (size_t)np * dim);
  for (int v = 0; v < ncam; v++)
    for (int p = 0; p < np; p++)
      for (int k = 0; k < 6; k++) G->h_z[z0 + 6 * ((size_t)v * np + p) + k] = zh[(size_t)p * dim + 6 * v + k];
  G->h_soff.push_back((long long)s0);
  G->h_sdim.push_back(dim);
  G->n += ncam;
  G->nsys++;
  G->h_node0.push_back(G->n);
  G->dirty = true;
  return RPBA_OK;
}

template <typename T>
rpba_status put(rpba_gnn *G, T **p, const std::vector<T> &h) {
  RPBA_TRY(galloc(G, (void **)p, std::max<size_t>(h.size(), 1) * sizeof(T)));
  if (!h.empty()) GNN_CUDA(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, G->stream));
  return RPBA_OK;
}

rpba_status prepare(rpba_gnn *G) {
  if (!G->dirty) return RPBA_OK;
  free_dataset(G);
  int n = G->n, np = G->np;
  size_t nnz = std::max<size_t>(G->h_adj.size(), 1), nv = (size_t)n * np * 6;
  RPBA_TRY(put(G, &G->ptr, G->h_ptr));
  RPBA_TRY(put(G, &G->adj, G->h_adj));
  RPBA_TRY(put(G, &G->mir, G->h_mir));
  RPBA_TRY(put(G, &G->row, G->h_row));
  RPBA_TRY(put(G, &G->node0, G->h_node0));
  RPBA_TRY(put(G, &G->node_sys, G->h_node_sys));
  RPBA_TRY(put(G, &G->sdim, G->h_sdim));
  RPBA_TRY(put(G, &G->soff, G->h_soff));
  RPBA_TRY(put(G, &G->e, G->h_e));
  RPBA_TRY(put(G, &G->x, G->h_x));
  RPBA_TRY(put(G, &G->L, G->h_L));
  RPBA_TRY(put(G, &G->shat, G->h_shat));
  RPBA_TRY(put(G, &G->z, G->h_z));
  RPBA_TRY(put(G, &G->S, G->h_S));
  RPBA_TRY(galloc(G, (void **)&G->act, (size_t)n * GH * (2 * GNL + 1) * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->C, (size_t)n * 21 * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->dC, (size_t)n * 21 * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->dh, (size_t)n * GH * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->dz, (size_t)n * GH * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->tmp, (size_t)n * GH * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->part, (size_t)nblk(n, WG_NODES) * GH * (GH + 1) * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->qbar, nnz * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->EP, (size_t)n * G_EDGE_PARAMS * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->gam, nnz * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->T, nv * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->V, nv * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->U, nv * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->SB, nv * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->Ts, (size_t)G->nsys * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->loss_s, (size_t)G->nsys * sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->loss, sizeof(double)));
  RPBA_TRY(galloc(G, (void **)&G->D, (size_t)n * 36 * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->Li, (size_t)n * 36 * sizeof(float)));
  RPBA_TRY(galloc(G, (void **)&G->F, nnz * 36 * sizeof(float)));
  GNN_CUDA(cudaStreamSynchronize(G->stream));
  G->dirty = false;
  return RPBA_OK;
}

GnnAct dataset_act(rpba_gnn *G) {
  GnnAct a;
  int n = G->n;
  a.n = n;
  a.ptr = G->ptr;
  a.adj = G->adj;
  a.e = G->e;
  a.x = G->x;
  for (int t = 0; t <= GNL; t++) a.h[t] = G->act + (size_t)t * n * GH;
  for (int t = 0; t < GNL; t++) a.m[t] = G->act + (size_t)(GNL + 1 + t) * n * GH;
  a.C = G->C;
  return a;
}

GSys dataset_sys(rpba_gnn *G) { return GSys{G->S, G->soff, G->sdim, G->node0, G->node_sys, nullptr}; }

// network forward and edge gains on the dataset
rpba_status dataset_forward(rpba_gnn *G, KL &kl) {
  RPBA_TRY(prepare(G));
  if (G->n == 0) {
    G->err = "empty dataset";
    return RPBA_ERR_STATE;
  }
  cudaStream_t st = G->stream;
  GnnNet net{G->w, G->wb};
  GnnAct a = dataset_act(G);
  RPBA_TRY(gnn_forward(kl, net, a, st));
  GSys g = dataset_sys(G);
  int nnz = (int)G->h_adj.size();
  if (nnz == 0) return RPBA_OK;
  return kl("k_gnn_edge_gain", [&] {
    k_gnn_edge_gain<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, G->row, G->adj, G->e, a.h[GNL], G->w, G->gam);
  });
}

// loss and gradient (into G->g) at the current weights
rpba_status loss_grad(rpba_gnn *G) {
  KL kl{nullptr, &G->err};
  RPBA_TRY(dataset_forward(G, kl));
  int n = G->n, np = G->np, ns = G->nsys;
  cudaStream_t st = G->stream;
  GnnAct a = dataset_act(G);
  int nvp = n * np;
  RPBA_TRY(kl("k_gnn_loss_t", [&] { k_gnn_loss_t<<<nblk(nvp, 128), 128, 0, st>>>(n, np, G->C, G->z, G->T); }));
  RPBA_TRY(kl("k_gnn_loss_v", [&] {
    k_gnn_loss_v<<<nblk(nvp, 128), 128, 0, st>>>(n, np, G->ptr, G->adj, G->mir, G->L, G->shat, G->gam, G->T, G->V);
  }));
  RPBA_TRY(kl("k_gnn_loss_symv", [&] {
    k_gnn_loss_symv<<<nblk(6LL * nvp, 128), 128, 0, st>>>(n, np, G->node_sys, G->node0, G->soff, G->sdim, G->S,
                                                          G->V, G->U);
  }));
  RPBA_TRY(kl("k_gnn_loss_sys", [&] {
    k_gnn_loss_sys<<<ns, 256, 0, st>>>(ns, np, G->node0, G->sdim, G->C, G->L, G->V, G->U, G->Ts, G->loss_s);
  }));
  RPBA_TRY(kl("k_gnn_loss_total", [&] { k_gnn_loss_total<<<1, 32, 0, st>>>(ns, G->loss_s, G->loss); }));
  RPBA_TRY(kl("k_gnn_loss_sbar", [&] {
    k_gnn_loss_sbar<<<nblk(nvp, 128), 128, 0, st>>>(n, np, ns, G->node_sys, G->L, G->Ts, G->U, G->SB);
  }));
  RPBA_TRY(kl("k_gnn_loss_node_bwd", [&] {
    k_gnn_loss_node_bwd<<<nblk(n, 64), 64, 0, st>>>(n, np, ns, G->node_sys, G->sdim, G->ptr, G->adj, G->C, G->shat,
                                                    G->gam, G->T, G->SB, G->dC, G->qbar);
  }));
  int nw = nblk(n, WG_NODES);
  auto wgrad = [&](const float *dz, int nout, const float *in, int nin, int offW, int offb) -> rpba_status {
    RPBA_TRY(kl("k_gnn_wgrad", [&] { k_gnn_wgrad<<<nw, 256, 0, st>>>(n, dz, nout, in, nin, G->part); }));
    return kl("k_gnn_wgrad_reduce", [&] {
      k_gnn_wgrad_reduce<<<nblk(nout * (nin + 1), 256), 256, 0, st>>>(nw, nout, nin, G->part, G->g + offW,
                                                                    G->g + offb);
    });
  };
  int gl = nblk(n, GL_NODES);
  long long nh = (long long)n * GH;
  // output heads
  RPBA_TRY(wgrad(G->dC, GNF, a.h[GNL], GH, G_Wo, G_bo));
  RPBA_TRY(kl("k_gnn_linear", [&] {
    k_gnn_linear<true><<<gl, 256, 0, st>>>(n, G->dC, GNF, G->wb + G_Wo, nullptr, 0, nullptr, nullptr, GH, 0, 0, G->dh);
  }));
  RPBA_TRY(kl("k_gnn_edge_bwd", [&] {
    k_gnn_edge_bwd<<<nblk((long long)n * 32, 256), 256, 0, st>>>(n, G->ptr, G->adj, G->mir, G->e, a.h[GNL], G->w,
                                                                 G->qbar, G->dh, G->EP);
  }));
  RPBA_TRY(kl("k_gnn_colsum", [&] {
    k_gnn_colsum<<<nblk(G_EDGE_PARAMS, 64), 64, 0, st>>>(n, G_EDGE_PARAMS, G->EP, G->g + G_ws);
  }));
  for (int t = GNL; t >= 1; t--) {
    RPBA_TRY(kl("k_gnn_relu_bwd", [&] { k_gnn_relu_bwd<<<nblk(nh, 256), 256, 0, st>>>(nh, G->dh, a.h[t], G->dz); }));
    RPBA_TRY(wgrad(G->dz, GH, a.h[t - 1], GH, g_A(t), g_c(t)));
    RPBA_TRY(wgrad(G->dz, GH, a.m[t - 1], GH, g_B(t), g_c(t)));  // the same bias gradient, written twice
    // dm = B^T dz ; dh_prev = A^T dz + aggregate(dm)
    RPBA_TRY(kl("k_gnn_linear", [&] {
      k_gnn_linear<true><<<gl, 256, 0, st>>>(n, G->dz, GH, G->wb + g_B(t), nullptr, 0, nullptr, nullptr, GH, 0, 0,
                                             G->tmp);
    }));
    RPBA_TRY(kl("k_gnn_linear", [&] {
      k_gnn_linear<true><<<gl, 256, 0, st>>>(n, G->dz, GH, G->wb + g_A(t), nullptr, 0, nullptr, nullptr, GH, 0, 0,
                                             G->dh);
    }));
    RPBA_TRY(kl("k_gnn_aggregate", [&] {
      k_gnn_aggregate<<<nblk((long long)n * 32, 256), 256, 0, st>>>(n, a.ptr, a.adj, a.e, G->tmp, G->dh, 1);
    }));
  }
  RPBA_TRY(kl("k_gnn_relu_bwd", [&] { k_gnn_relu_bwd<<<nblk(nh, 256), 256, 0, st>>>(nh, G->dh, a.h[0], G->dz); }));
  RPBA_TRY(wgrad(G->dz, GH, a.x, GNF, G_W0, G_b0));
  return RPBA_OK;
}

}  // namespace

extern "C" int32_t rpba_gnn_param_count(void) { return G_NPARAM; }

extern "C" rpba_status rpba_gnn_create(uint64_t seed, rpba_gnn **out) {
  if (!out) return RPBA_ERR_INVALID_ARG;
  *out = nullptr;
  rpba_gnn *G = new (std::nothrow) rpba_gnn();
  if (!G) return RPBA_ERR_OOM;
  *out = G;
  GNN_CUDA(cudaGetDevice(&G->dev));
  GNN_CUDA(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
  GNN_CUDA(cudaMalloc((void **)&G->w, G_NPARAM * sizeof(float)));
  GNN_CUDA(cudaMalloc((void **)&G->g, G_NPARAM * sizeof(float)));
  GNN_CUDA(cudaMalloc((void **)&G->m, G_NPARAM * sizeof(float)));
  GNN_CUDA(cudaMalloc((void **)&G->v, G_NPARAM * sizeof(float)));
  GNN_CUDA(cudaMalloc((void **)&G->wb, G_NPARAM * sizeof(__nv_bfloat16)));
  // He-normal hidden layers; zero output and edge heads (block-Jacobi)
  std::vector<float> w(G_NPARAM, 0.0f);
  Rng r{seed};
  auto fill = [&](int off, int rows, int cols) {
    double sd = sqrt(2.0 / cols);
    for (int e = 0; e < rows * cols; e++) w[off + e] = (float)(sd * r.normal());
  };
  fill(G_W0, GH, GNF);
  for (int t = 1; t <= GNL; t++) {
    fill(g_A(t), GH, GH);
    fill(g_B(t), GH, GH);
  }
  return rpba_gnn_set_weights(G, w.data());
}

extern "C" void rpba_gnn_destroy(rpba_gnn *G) {
  if (!G) return;
  free_dataset(G);
  cudaFree(G->w);
  cudaFree(G->g);
  cudaFree(G->m);
  cudaFree(G->v);
  cudaFree(G->wb);
  if (G->stream) cudaStreamDestroy(G->stream);
  delete G;
}

extern "C" const char *rpba_gnn_last_error(const rpba_gnn *G) { return G ? G->err.c_str() : "null network"; }

extern "C" rpba_status rpba_gnn_set_weights(rpba_gnn *G, const float *w) {
  if (!G || !w) return RPBA_ERR_INVALID_ARG;
  GNN_CUDA(cudaMemcpyAsync(G->w, w, G_NPARAM * sizeof(float), cudaMemcpyHostToDevice, G->stream));
  GNN_CUDA(cudaMemsetAsync(G->m, 0, G_NPARAM * sizeof(float), G->stream));
  GNN_CUDA(cudaMemsetAsync(G->v, 0, G_NPARAM * sizeof(float), G->stream));
  k_gnn_to_bf16<<<nblk(G_NPARAM, 256), 256, 0, G->stream>>>(G_NPARAM, G->w, G->wb);
  GNN_CUDA(cudaGetLastError());
  GNN_CUDA(cudaStreamSynchronize(G->stream));
  G->t = 0;
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_get_weights(rpba_gnn *G, float *w) {
  if (!G || !w) return RPBA_ERR_INVALID_ARG;
  GNN_CUDA(cudaMemcpyAsync(w, G->w, G_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, G->stream));
  GNN_CUDA(cudaStreamSynchronize(G->stream));
  return RPBA_OK;
}

static rpba_status check_probes(rpba_gnn *G, int np) {
  if (np < 1) return RPBA_ERR_INVALID_ARG;
  if (G->np == 0) G->np = np;
  if (G->np != np) {
    G->err = "every system needs the same number of probes";
    return RPBA_ERR_INVALID_ARG;
  }
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_add_system(rpba_gnn *G, int32_t n_cams, const double *S, int32_t ld,
                                           int32_t n_probes, const double *z) {
  if (!G || n_cams < 0 || (n_cams && (!S || !z || ld < 6 * n_cams))) return RPBA_ERR_INVALID_ARG;
  RPBA_TRY(check_probes(G, n_probes));
  if (n_cams == 0) return RPBA_OK;
  double *Sd = nullptr;
  size_t bytes = (size_t)6 * n_cams * ld * sizeof(double);
  GNN_CUDA(cudaMalloc((void **)&Sd, bytes));
  cudaError_t ce = cudaMemcpyAsync(Sd, S, bytes, cudaMemcpyHostToDevice, G->stream);
  rpba_status s = ce == cudaSuccess ? add_dense(G, Sd, ld, n_cams, n_probes, z, G->stream) : RPBA_ERR_CUDA;
  if (ce != cudaSuccess) G->err = cudaGetErrorString(ce);
  cudaStreamSynchronize(G->stream);
  cudaFree(Sd);
  return s;
}

extern "C" rpba_status rpba_gnn_add_rcs(rpba_gnn *G, rpba_ctx *h, double lambda, int32_t n_probes, uint64_t seed) {
  if (!G || !h) return RPBA_ERR_INVALID_ARG;
  RPBA_TRY(check_probes(G, n_probes));
  Ctx *ctx = &h->c;
  RPBA_TRY(launch_fill_double(ctx, ctx->lm_lambda, ctx->L, lambda));
  RPBA_TRY(launch_fill_int(ctx, ctx->lm_run, ctx->L, 1));
  RPBA_TRY(launch_build_rcs(ctx, ctx->lm_lambda, ctx->lm_run));
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  Rng r{seed};
  for (int l = 0; l < ctx->L; l++) {
    int ncam = ctx->h_sub_cam_ptr[l + 1] - ctx->h_sub_cam_ptr[l];
    std::vector<double> z((size_t)n_probes * 6 * ncam);
    for (double &v : z) v = r.normal();
    RPBA_TRY(add_dense(G, ctx->S + ctx->h_S_off[l], ctx->h_npad[l], ncam, n_probes, z.data(), G->stream));
  }
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_dataset_size(rpba_gnn *G, int32_t *n_nodes, int32_t *n_edges, int32_t *n_systems) {
  if (!G) return RPBA_ERR_INVALID_ARG;
  if (n_nodes) *n_nodes = G->n;
  if (n_edges) *n_edges = (int32_t)G->h_adj.size();
  if (n_systems) *n_systems = G->nsys;
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_graph(rpba_gnn *G, float *x, int32_t *ptr, int32_t *adj, float *e) {
  if (!G) return RPBA_ERR_INVALID_ARG;
  if (x) memcpy(x, G->h_x.data(), G->h_x.size() * sizeof(float));
  if (ptr) memcpy(ptr, G->h_ptr.data(), G->h_ptr.size() * sizeof(int));
  if (adj) memcpy(adj, G->h_adj.data(), G->h_adj.size() * sizeof(int));
  if (e) memcpy(e, G->h_e.data(), G->h_e.size() * sizeof(float));
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_precondition(rpba_gnn *G, const double *r, double *z) {
  if (!G || !r || !z) return RPBA_ERR_INVALID_ARG;
  KL kl{nullptr, &G->err};
  RPBA_TRY(dataset_forward(G, kl));
  int n = G->n, ns = G->nsys;
  cudaStream_t st = G->stream;
  GSys g = dataset_sys(G);
  std::vector<int> ones(n, 1);
  int *okd = nullptr, *nvo = nullptr;
  double *rd = nullptr, *zd = nullptr;
  float *yd = nullptr;
  std::vector<int> hv(n);
  for (int v = 0; v < n; v++) hv[v] = 6 * v;
  GNN_CUDA(cudaMalloc((void **)&okd, n * sizeof(int)));
  GNN_CUDA(cudaMalloc((void **)&nvo, n * sizeof(int)));
  GNN_CUDA(cudaMalloc((void **)&rd, (size_t)n * 6 * sizeof(double)));
  GNN_CUDA(cudaMalloc((void **)&zd, (size_t)n * 6 * sizeof(double)));
  GNN_CUDA(cudaMalloc((void **)&yd, (size_t)n * 12 * sizeof(float)));
  cudaError_t ce = cudaMemcpyAsync(okd, ones.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(nvo, hv.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(rd, r, (size_t)n * 6 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) {
    int nnz = (int)G->h_adj.size();
    k_gnn_head_node<<<nblk(n, 128), 128, 0, st>>>(n, g, G->C, G->L, okd, G->D, G->Li, nullptr);
    if (nnz) k_gnn_head_F<<<nblk(nnz, 128), 128, 0, st>>>(nnz, g, G->row, G->adj, G->C, G->shat, G->gam, G->F);
    FsaiApply F;
    F.M = n;
    F.node_sys = G->node_sys;
    F.nvo = nvo;
    F.P = FsaiView{G->ptr, G->adj, G->mir, G->D, G->Li, G->F};
    F.rh = yd;
    F.y = yd + 6 * (size_t)n;
    F.stream = st;
    ce = cudaGetLastError();
    if (ce == cudaSuccess && fsai_apply(nullptr, F, nullptr, rd, zd) != RPBA_OK) ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(z, zd, (size_t)n * 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaFree(okd);
  cudaFree(nvo);
  cudaFree(rd);
  cudaFree(zd);
  cudaFree(yd);
  if (ce != cudaSuccess) {
    G->err = cudaGetErrorString(ce);
    return RPBA_ERR_CUDA;
  }
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_loss_grad(rpba_gnn *G, double *loss, float *grad) {
  if (!G) return RPBA_ERR_INVALID_ARG;
  RPBA_TRY(loss_grad(G));
  double l = 0.0;
  GNN_CUDA(cudaMemcpyAsync(&l, G->loss, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
  if (grad) GNN_CUDA(cudaMemcpyAsync(grad, G->g, G_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, G->stream));
  GNN_CUDA(cudaStreamSynchronize(G->stream));
  if (loss) *loss = l;
  return RPBA_OK;
}

extern "C" rpba_status rpba_gnn_train(rpba_gnn *G, int32_t steps, float lr, uint64_t probe_seed,
                                      double *loss_hist) {
  if (!G || steps < 0 || !(lr > 0.0f)) return RPBA_ERR_INVALID_ARG;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int s = 0; s < steps; s++) {
    if (probe_seed) {
      RPBA_TRY(prepare(G));
      long long nz = 6LL * G->n * G->np;
      k_gnn_draw_probes<<<nblk(nz, 256), 256, 0, G->stream>>>(nz, probe_seed, (uint64_t)G->t, G->z);
      GNN_CUDA(cudaGetLastError());
    }
    RPBA_TRY(loss_grad(G));
    if (loss_hist) {
      GNN_CUDA(cudaMemcpyAsync(loss_hist + s, G->loss, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
    }
    G->t++;
    float c1 = 1.0f - powf(b1, (float)G->t), c2 = 1.0f - powf(b2, (float)G->t);
    k_gnn_adam<<<nblk(G_NPARAM, 256), 256, 0, G->stream>>>(G_NPARAM, G->w, G->g, G->m, G->v, lr, b1, b2, eps, c1, c2,
                                                          G->wb);
    GNN_CUDA(cudaGetLastError());
  }
  GNN_CUDA(cudaStreamSynchronize(G->stream));
  return RPBA_OK;
}

extern "C" rpba_status rpba_set_gnn_weights(rpba_ctx *h, const float *w, int32_t n) {
  if (!h) return RPBA_ERR_INVALID_ARG;
  Ctx *ctx = &h->c;
  if (!w || n != G_NPARAM) {
    ctx->err = "rpba_set_gnn_weights: expected rpba_gnn_param_count() weights";
    return RPBA_ERR_INVALID_ARG;
  }
  if (ctx->opt.solver != 3) {
    ctx->err = "the network weights are used by solver 3 only";
    return RPBA_ERR_STATE;
  }
  RPBA_TRY(gnn_ctx_buffers(ctx));
  RPBA_CUDA(cudaMemcpyAsync(ctx->gnn_w, w, G_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  KL kl{ctx, &ctx->err};
  RPBA_TRY(kl("k_gnn_to_bf16", [&] {
    k_gnn_to_bf16<<<nblk(G_NPARAM, 256), 256, 0, ctx->stream>>>(G_NPARAM, ctx->gnn_w,
                                                               (__nv_bfloat16 *)ctx->gnn_wb);
  }));
  RPBA_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->gnn_ready = true;
  return RPBA_OK;
}
