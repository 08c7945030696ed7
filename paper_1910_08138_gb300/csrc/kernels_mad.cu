// kernels_mad.cu -- per-camera robust scale (Sec. 5.3): 1.4826 times the
// median absolute deviation of the whitened residual components of every
// observation of the camera. One CTA per camera, the 2 K_i components in
// shared memory. FP32 form: the two medians by radix select (below). FP64
// form: the components are sorted (bitonic network, padded to a power of two
// >= 64; the stages with stride < 64 run in registers, one warp per 64-key
// chunk, with shuffles) and the median is read off. The absolute deviations need no second sort: those of
// the components below the median, read backwards, and those of the
// components from the median up are two ascending lists, and their median
// is found by a binary search over the two.
// The values are sorted as order-preserving integer keys: 64-bit for the
// FP64 form, 32-bit for the FP32 form, whose residuals are float-float
// evaluations rounded to FP32. On this GPU FP64 compares run on the slow FP64
// pipe, integer compares do not.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "rpba_internal.cuh"

namespace rpba {

// IEEE-754 double -> unsigned key with the same order (and back)
__device__ inline unsigned long long dkey(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ inline double dval(unsigned long long k) {
  unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)u);
}
__device__ inline unsigned fkey(float x) {
  unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline double dval(unsigned k) {
  unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return (double)__uint_as_float(u);
}
__device__ inline unsigned long long key_of(double x, unsigned long long) { return dkey(x); }
__device__ inline unsigned key_of(double x, unsigned) { return fkey((float)x); }

// compare-exchange of the bitonic network for the key held at position pos,
// partner at pos ^ stride (value y): keep the min at the lower position of an
// ascending pair, the max at its upper position (reversed when descending)
template <typename Key>
__device__ inline Key bitonic_keep(Key x, Key y, int pos, int stride, int size) {
  bool asc = (pos & size) == 0;
  bool lower = (pos & stride) == 0;
  bool take_min = (lower == asc);
  return take_min ? (x < y ? x : y) : (x < y ? y : x);
}

// the stages of one merge size with stride <= 32 on 64-key chunks, one warp
// per chunk, keys in registers (lane and lane + 32 of the chunk)
template <typename Key>
__device__ inline void bitonic_chunk_stages(Key *a, int n2, int size, int first_stride) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 64 * warp; c < n2; c += 64 * nw) {
    Key x0 = a[c + lane], x1 = a[c + 32 + lane];
    for (int stride = first_stride; stride > 0; stride >>= 1) {
      if (stride == 32) {  // the pair is (lane, lane + 32) of this thread
        bool asc = ((c + lane) & size) == 0;
        Key lo = x0 < x1 ? x0 : x1, hi = x0 < x1 ? x1 : x0;
        x0 = asc ? lo : hi;
        x1 = asc ? hi : lo;
      } else {
        Key y0 = __shfl_xor_sync(0xffffffffu, x0, stride);
        Key y1 = __shfl_xor_sync(0xffffffffu, x1, stride);
        x0 = bitonic_keep(x0, y0, c + lane, stride, size);
        x1 = bitonic_keep(x1, y1, c + 32 + lane, stride, size);
      }
    }
    a[c + lane] = x0;
    a[c + 32 + lane] = x1;
  }
}

// ascending bitonic sort of a[0..n2), n2 a power of two >= 64: the stages with
// stride >= 64 as shared-memory passes, the others in registers per 64-key chunk
template <typename Key>
__device__ static void bitonic_sort(Key *a, int n2) {
  for (int size = 2; size <= 64; size <<= 1) bitonic_chunk_stages(a, n2, size, size >> 1);
  __syncthreads();
  for (int size = 128; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride >= 64; stride >>= 1) {
      for (int idx = threadIdx.x; idx < (n2 >> 1); idx += blockDim.x) {
        int i = 2 * stride * (idx / stride) + (idx % stride);
        int j = i + stride;
        bool up = (i & size) == 0;
        Key x = a[i], y = a[j];
        if ((x > y) == up) {
          a[i] = y;
          a[j] = x;
        }
      }
      __syncthreads();
    }
    bitonic_chunk_stages(a, n2, size, 32);
    __syncthreads();
  }
}

template <typename Key>
__device__ static double sorted_median(const Key *a, int n) {
  return (n & 1) ? dval(a[n / 2]) : 0.5 * (dval(a[n / 2 - 1]) + dval(a[n / 2]));
}

// the deviation lists of the sorted values a[0..n) around med, split at s
// (a[s-1] < med <= a[s]): lower list j -> med - a[s-1-j] (j < s), upper list
// j -> a[s+j] - med (j < n - s); both ascending
template <typename Key>
struct DevLists {
  const Key *a;
  int n, s;
  double med;
  __device__ double lo(int j) const { return med - dval(a[s - 1 - j]); }
  __device__ double hi(int j) const { return dval(a[s + j]) - med; }
};

// k-th smallest (0-based) of the union of the two deviation lists
template <typename Key>
__device__ static double dev_select(const DevLists<Key> &D, int k) {
  int na = D.s, nb = D.n - D.s;
  int lo = max(0, k + 1 - nb), hi = min(k + 1, na);  // i values taken from the lower list
  while (lo < hi) {
    int i = (lo + hi) >> 1;  // candidate: i from the lower list, k + 1 - i from the upper
    int j = k + 1 - i;
    // too few from the lower list when its next element is below the upper list's last taken one
    if (i < na && j > 0 && D.lo(i) < D.hi(j - 1)) lo = i + 1;
    else hi = i;
  }
  int i = lo, j = k + 1 - lo;
  double x = i > 0 ? D.lo(i - 1) : -1.0, y = j > 0 ? D.hi(j - 1) : -1.0;
  return x > y ? x : y;
}

// ---- FP32 form: order statistics by radix select instead of a sort ----
// k-th smallest (0-based) of the 32-bit keys a[0..n): most significant digit
// first, 8 bits per pass. Each pass histograms the keys that share the digits
// found so far (lanes with the same bin add once, __match_any_sync), and warp 0
// finds the bin that holds rank k by a prefix sum over the 256 bins.
struct SelScratch {
  unsigned hist[256];
  int bin, rank;
  unsigned cnt, minv;
};

__device__ static unsigned radix_select(const unsigned *a, int n, int k, SelScratch &S) {
  unsigned prefix = 0, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) S.hist[b] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
      int e = base + threadIdx.x;
      unsigned x = e < n ? a[e] : 0u;
      bool in = e < n && (x & mask) == prefix;
      unsigned bin = in ? (x >> shift) & 255u : 256u;
      unsigned peers = __match_any_sync(__activemask(), bin);
      if (in && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&S.hist[bin], (unsigned)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      int lane = threadIdx.x;
      unsigned c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; q++) { c[q] = S.hist[8 * lane + q]; sum += c[q]; }
      unsigned incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      unsigned excl = incl - sum;
      if (excl <= (unsigned)k && (unsigned)k < incl) {
        unsigned acc = excl;
        int q = 0;
        while (acc + c[q] <= (unsigned)k) acc += c[q++];
        S.bin = 8 * lane + q;
        S.rank = k - (int)acc;
      }
    }
    __syncthreads();
    prefix |= (unsigned)S.bin << shift;
    mask |= 255u << shift;
    k = S.rank;
    __syncthreads();  // every thread has read S before the next pass clears it
  }
  return prefix;
}

// the k-th and (k+1)-th smallest keys (k + 1 < n)
__device__ static void radix_select_pair(const unsigned *a, int n, int k, SelScratch &S, unsigned &v0, unsigned &v1) {
  v0 = radix_select(a, n, k, S);
  if (threadIdx.x == 0) { S.cnt = 0; S.minv = 0xffffffffu; }
  __syncthreads();
  unsigned le = 0, mn = 0xffffffffu;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    unsigned x = a[e];
    if (x <= v0) le++;
    else mn = x < mn ? x : mn;
  }
  atomicAdd(&S.cnt, le);
  atomicMin(&S.minv, mn);
  __syncthreads();
  v1 = S.cnt >= (unsigned)(k + 2) ? v0 : S.minv;  // a tie with the k-th, or the next larger key
  __syncthreads();
}

__device__ inline float fval(unsigned k) {
  unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// median of the n keys as hi + lo (the mean of the middle pair for even n, exact)
__device__ static float2 radix_median(const unsigned *a, int n, SelScratch &S) {
  if (n & 1) return make_float2(fval(radix_select(a, n, n / 2, S)), 0.f);
  unsigned v0, v1;
  radix_select_pair(a, n, n / 2 - 1, S, v0, v1);
  float e;
  float h = ff_two_sum(fval(v0), fval(v1), e);
  return make_float2(0.5f * h, 0.5f * e);  // halving is exact
}

// inputs of the residuals: FP64 state (FP64 form) or the FP32 form's
// camera records, points as hi + lo and observations as hi + lo
struct MadIn {
  const double *R, *t, *intr, *X, *obs_xy, *whiten;
  const float *camff, *Xh, *Xl, *oxy, *oxylo, *whiten32;
  const double *k1;  // per-camera radial parameter (NULL without intrinsics)
  // FP32 form: the observation streams in camera-major order (the order of cam_obs)
  const int *cm_pt;
  const float *cm_xy, *cm_xylo, *cm_whiten32;
};

template <typename Key, bool K1>
__global__ void k_camera_mad(int M, MadIn in, const uint8_t *active, const int *cam_obs_ptr, const int *cam_obs,
                             const int *obs_pt, int has_winv, double *sigma, float *sigma32) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  Key *sh = reinterpret_cast<Key *>(sh_raw);
  __shared__ int count;
  int i = blockIdx.x;
  if (i >= M) return;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  int p0 = cam_obs_ptr[i], p1 = cam_obs_ptr[i + 1];
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    Key k0, k1;
    if constexpr (sizeof(Key) == 4) {  // keys straight from the FP32 components
      // the observation from the camera-major streams (coalesced); the active
      // flag is read beside the residual's gathers, not before them
      int j = in.cm_pt[p];
      const bool act = active[j] != 0;
      float r0, r1;
      ff_residual(in.camff + FF_CAM * (size_t)i, in.Xh + 3 * (size_t)j, in.Xl + 3 * (size_t)j, in.cm_xy[2 * (size_t)p],
                  in.cm_xylo[2 * (size_t)p], in.cm_xy[2 * (size_t)p + 1], in.cm_xylo[2 * (size_t)p + 1], r0, r1, K1);
      if (!act) continue;
      if (has_winv) {
        const float *F = in.cm_whiten32 + 3 * (size_t)p;
        float a = F[0] * r0 + F[1] * r1, b = F[2] * r1;
        r0 = a;
        r1 = b;
      }
      k0 = fkey(r0);
      k1 = fkey(r1);
    } else {
      int k = cam_obs[p];
      int j = obs_pt[k];
      if (!active[j]) continue;
      double pu, pv;
      proj64(in.R + 9 * i, in.t + 3 * i, in.intr[3 * i], in.k1 ? in.k1[i] : 0.0, in.intr[3 * i + 1],
             in.intr[3 * i + 2], in.X + 3 * j, pu, pv);
      double r0 = pu - in.obs_xy[2 * k];
      double r1 = pv - in.obs_xy[2 * k + 1];
      double e0 = r0, e1 = r1;
      if (has_winv) {  // upper Cholesky factor of C^-1, precomputed: (sqrt(w11), w12/sqrt(w11), sqrt(w22 - w12^2/w11))
        const double *F = in.whiten + 3 * k;
        e0 = F[0] * r0 + F[1] * r1;
        e1 = F[2] * r1;
      }
      k0 = key_of(e0, Key());
      k1 = key_of(e1, Key());
    }
    int slot = atomicAdd(&count, 2);
    sh[slot] = k0;
    sh[slot + 1] = k1;
  }
  __syncthreads();
  int n = count;
  if (n == 0) {
    if (threadIdx.x == 0) {
      sigma[i] = 0.0;
      if (sigma32) sigma32[i] = 0.f;
    }
    return;
  }
  if constexpr (sizeof(Key) == 4) {
    // FP32 form: median by radix select; the absolute deviations from it (in
    // float-float, then FP32) overwrite the keys, and their median is the MAD
    __shared__ SelScratch S;
    unsigned *ka = reinterpret_cast<unsigned *>(sh);
    float2 med = radix_median(ka, n, S);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      float d = fabsf(__fsub_rn(__fsub_rn(fval(ka[e]), med.x), med.y));
      ka[e] = __float_as_uint(d);  // non-negative floats order as their bit patterns
    }
    __syncthreads();
    double mad;
    if (n & 1) {
      mad = (double)__uint_as_float(radix_select(ka, n, n / 2, S));
    } else {
      unsigned v0, v1;
      radix_select_pair(ka, n, n / 2 - 1, S, v0, v1);
      mad = 0.5 * ((double)__uint_as_float(v0) + (double)__uint_as_float(v1));
    }
    if (threadIdx.x == 0) {
      sigma[i] = 1.4826 * mad;
      if (sigma32) sigma32[i] = (float)(1.4826 * mad);
    }
    return;
  }
  int n2 = 64;
  while (n2 < n) n2 <<= 1;
  for (int e = n + threadIdx.x; e < n2; e += blockDim.x) sh[e] = ~Key(0);  // sorts last
  __syncthreads();
  bitonic_sort(sh, n2);
  if (threadIdx.x == 0) {
    double med = sorted_median(sh, n);
    int a = 0, b = n;  // s = first index with a[s] >= med (compared as values: med need not be a key)
    while (a < b) {
      int c = (a + b) >> 1;
      if (dval(sh[c]) < med) a = c + 1; else b = c;
    }
    DevLists<Key> D{sh, n, a, med};
    double mad = (n & 1) ? dev_select(D, n / 2) : 0.5 * (dev_select(D, n / 2 - 1) + dev_select(D, n / 2));
    sigma[i] = 1.4826 * mad;
    if (sigma32) sigma32[i] = (float)(1.4826 * mad);
  }
}

rpba_status launch_camera_scale(Ctx *ctx) {
  if (ctx->M == 0) return RPBA_OK;
  bool f32 = ctx->opt.precision == 1;
  int n2 = 64;
  while (n2 < 2 * ctx->max_cam_obs) n2 <<= 1;
  // FP32 form: 32-bit keys, radix select (no padding); FP64 form: 64-bit keys
  // padded to a power of two for the bitonic sort
  size_t smem = f32 ? (size_t)std::max(2 * ctx->max_cam_obs, 1) * sizeof(unsigned)
                    : (size_t)n2 * sizeof(unsigned long long);
  if (smem > 200 * 1024) {
    ctx->err = "camera with too many observations for the shared-memory median";
    return RPBA_ERR_INVALID_ARG;
  }
  MadIn in{ctx->R, ctx->t, ctx->intr, ctx->X, ctx->obs_xy, ctx->obs_whiten,
           ctx->camff, ctx->X_hi, ctx->X_lo, ctx->obs_xy32, ctx->obs_xylo, ctx->obs_whiten32,
           ctx->cd == 8 ? ctx->k1 : nullptr, ctx->cm_pt, ctx->cm_xy32, ctx->cm_xylo, ctx->cm_whiten32};
  int threads = std::min(1024, std::max(32, n2 / 2));  // one thread per compare-exchange of a pass
  if (f32) {
    // two observations per thread, at most 512 threads: with the camera-major
    // streams the residual phase is no longer a chain of gathers, and the
    // selects' barriers are cheaper on smaller CTAs (more of them per SM)
    threads = std::min(512, std::max(64, 32 * ((ctx->max_cam_obs + 63) / 64)));
    auto kern = ctx->cd == 8 ? k_camera_mad<unsigned, true> : k_camera_mad<unsigned, false>;
    if (smem > 48 * 1024)
      RPBA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RPBA_KERNEL(ctx, "k_camera_mad_u32", kern<<<ctx->M, threads, smem, ctx->stream>>>(
                                         ctx->M, in, ctx->active, ctx->cam_obs_ptr, ctx->cam_obs, ctx->obs_pt,
                                         ctx->has_winv, ctx->cam_sigma, ctx->cam_sigma32));
  } else {
    auto kern = k_camera_mad<unsigned long long, false>;  // the FP64 path reads k1 from in.k1
    if (smem > 48 * 1024)
      RPBA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RPBA_KERNEL(ctx, "k_camera_mad_u64", kern<<<ctx->M, threads, smem, ctx->stream>>>(
                                         ctx->M, in, ctx->active, ctx->cam_obs_ptr, ctx->cam_obs, ctx->obs_pt,
                                         ctx->has_winv, ctx->cam_sigma, nullptr));
  }
  return RPBA_OK;
}

}  // namespace rpba
