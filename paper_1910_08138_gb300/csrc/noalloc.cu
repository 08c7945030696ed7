// noalloc.cu -- sigma_0 and RMS (Eq. sigma0) of a block held entirely in
// caller-owned device memory, computed without allocating any device memory.
//
// Some callers cannot allocate device memory per call: a pipeline that runs
// under a device-memory budget fixed at start-up, or a process whose device
// allocator belongs to another framework. This entry point serves them: its
// only scratch is the file-scope array below, of a fixed size stated in
// include/rpba.h (RPBA_NOALLOC_MAX_OBS / RPBA_NOALLOC_MAX_POINTS).
//
// The array is a device symbol. In host code its name is only a stand-in, so
// the host obtains its device address once per device, with that device
// current, through cudaGetSymbolAddress (first call on the device), and passes
// that address to the kernels. Every call shares the array and it keeps the
// previous call's contents; nothing in it needs to start at zero because each
// block overwrites its own slots before they are read. Calls whose work
// overlaps on the GPU (two streams, or two host threads) race on the array.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/rpba.h"

namespace {

constexpr int kThreads = 256;
constexpr int kObsBlocks = RPBA_NOALLOC_MAX_OBS / kThreads;
constexpr int kPtBlocks = RPBA_NOALLOC_MAX_POINTS / kThreads;
// layout: 4 doubles per observation block, 1 per point block, 5 final sums
constexpr int kSlots = 4 * kObsBlocks + kPtBlocks + 8;

static __device__ __align__(256) double g_scratch[kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_dev[kMaxDevices] = {nullptr};

__device__ inline void block_sum(double *v, int nv, double *out) {
  __shared__ double sh[8][kThreads / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = 0; e < nv; e++) {
    double x = v[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[e][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; w++) s += sh[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

// one thread per observation: [w v^T C^-1 v, 1, |v|^2 if w == 1, 1 if w == 1]
__global__ void __launch_bounds__(kThreads)
    k_na_obs(int K, const double *R, const double *t, const double *intr, const double *X, const uint8_t *active,
             const int32_t *obs_cam, const int32_t *obs_point, const double *obs_xy, const double *obs_winv,
             const double *obs_w, double *scratch) {
  int k = blockIdx.x * kThreads + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (k < K) {
    int j = obs_point[k];
    if (!active || active[j]) {
      int i = obs_cam[k];
      const double *Ri = R + 9 * (size_t)i, *ti = t + 3 * (size_t)i, *Xj = X + 3 * (size_t)j;
      double xc[3];
      for (int r = 0; r < 3; r++) xc[r] = Ri[3 * r] * Xj[0] + Ri[3 * r + 1] * Xj[1] + Ri[3 * r + 2] * Xj[2] + ti[r];
      double f = intr[3 * i];
      double r0 = f * xc[0] / xc[2] + intr[3 * i + 1] - obs_xy[2 * (size_t)k];
      double r1 = f * xc[1] / xc[2] + intr[3 * i + 2] - obs_xy[2 * (size_t)k + 1];
      double a = 1.0, b = 0.0, c = 1.0;
      if (obs_winv) { a = obs_winv[3 * (size_t)k]; b = obs_winv[3 * (size_t)k + 1]; c = obs_winv[3 * (size_t)k + 2]; }
      double w = obs_w ? obs_w[k] : 1.0;
      v[0] = w * (a * r0 * r0 + 2.0 * b * r0 * r1 + c * r1 * r1);
      v[1] = 1.0;
      if (w == 1.0) {
        v[2] = r0 * r0 + r1 * r1;
        v[3] = 1.0;
      }
    }
  }
  block_sum(v, 4, scratch + 4 * (size_t)blockIdx.x);
}

// one thread per point: active count
__global__ void __launch_bounds__(kThreads) k_na_points(int N, const uint8_t *active, double *scratch) {
  int j = blockIdx.x * kThreads + threadIdx.x;
  double v[1] = {(j < N && (!active || active[j])) ? 1.0 : 0.0};
  block_sum(v, 1, scratch + 4 * (size_t)kObsBlocks + blockIdx.x);
}

// one block: the partials of this call, in block order
__global__ void __launch_bounds__(kThreads) k_na_final(int n_obs_blocks, int n_pt_blocks, double *scratch) {
  double v[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < n_obs_blocks; b += kThreads)
    for (int e = 0; e < 4; e++) v[e] += scratch[4 * (size_t)b + e];
  for (int b = threadIdx.x; b < n_pt_blocks; b += kThreads) v[4] += scratch[4 * (size_t)kObsBlocks + b];
  block_sum(v, 5, scratch + 4 * (size_t)kObsBlocks + kPtBlocks);
}

// device address of the scratch array for the current device (set up once)
rpba_status scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RPBA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RPBA_ERR_CUDA;
    g_scratch_dev[dev] = (double *)p;
  }
  *out = g_scratch_dev[dev];
  return RPBA_OK;
}

}  // namespace

extern "C" rpba_status rpba_sigma0_noalloc(int32_t n_cams, int32_t n_points, int32_t n_obs, const double *R,
                                           const double *t, const double *intr, const double *X,
                                           const uint8_t *active, const int32_t *obs_cam, const int32_t *obs_point,
                                           const double *obs_xy, const double *obs_winv, const double *obs_w,
                                           void *cuda_stream, double *sums5, double *sigma0, double *rms) {
  if (n_cams < 0 || n_points < 0 || n_obs < 0) return RPBA_ERR_INVALID_ARG;
  if (n_obs > RPBA_NOALLOC_MAX_OBS || n_points > RPBA_NOALLOC_MAX_POINTS) return RPBA_ERR_INVALID_ARG;
  if ((n_cams && (!R || !t || !intr)) || (n_points && !X) || (n_obs && (!obs_cam || !obs_point || !obs_xy)))
    return RPBA_ERR_INVALID_ARG;
  // observations index cameras and points: a block with observations but no
  // cameras or no points has nothing valid for them to reference
  if (n_obs && (!n_cams || !n_points)) return RPBA_ERR_INVALID_ARG;
  double *scratch = nullptr;
  rpba_status st = scratch_for_current_device(&scratch);
  if (st != RPBA_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int nbo = (n_obs + kThreads - 1) / kThreads, nbp = (n_points + kThreads - 1) / kThreads;
  if (nbo) k_na_obs<<<nbo, kThreads, 0, s>>>(n_obs, R, t, intr, X, active, obs_cam, obs_point, obs_xy, obs_winv,
                                              obs_w, scratch);
  if (nbp) k_na_points<<<nbp, kThreads, 0, s>>>(n_points, active, scratch);
  k_na_final<<<1, kThreads, 0, s>>>(nbo, nbp, scratch);
  if (cudaGetLastError() != cudaSuccess) return RPBA_ERR_CUDA;
  double h[5];
  if (cudaMemcpyAsync(h, scratch + 4 * (size_t)kObsBlocks + kPtBlocks, sizeof(h), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RPBA_ERR_CUDA;
  if (sums5)
    for (int e = 0; e < 5; e++) sums5[e] = h[e];
  double red = 2.0 * h[1] - 6.0 * n_cams - 3.0 * h[4] + 7.0;
  if (red < 1.0) red = 1.0;
  if (sigma0) *sigma0 = sqrt(h[0] / red);
  if (rms) *rms = h[3] > 0 ? sqrt(h[2] / (2.0 * h[3])) : 0.0;
  return RPBA_OK;
}
