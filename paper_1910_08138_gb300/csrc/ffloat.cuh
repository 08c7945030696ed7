// ffloat.cuh -- float-float arithmetic for the FP32 form's residuals.
//
// A value is carried as an unevaluated sum hi + lo of two floats (about 48
// significant bits). The building blocks are the classical error-free
// transformations: Knuth's TwoSum (a + b = s + e exactly, any a, b), Dekker's
// Fast2Sum (the same when |a| >= |b|) and the FMA form of Dekker's
// TwoProduct (a b = p + e exactly). A dot product of float-float operands
// follows the compensated scheme of Ogita, Rump and Oishi ("Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005, Algorithm Dot2), with the
// cross terms hi*lo folded into the compensation.
//
// The rounded intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) are used
// throughout: the compiler never contracts or reassociates them, which the
// transformations rely on.
#pragma once

#include <cuda_runtime.h>

namespace rpba {

__device__ __forceinline__ float ff_two_sum(float a, float b, float &e) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ float ff_fast_two_sum(float a, float b, float &e) {
  float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ float ff_two_prod(float a, float b, float &e) {
  float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

// sum_c (ah[c] + al[c]) (bh[c] + bl[c]) over three terms, as hi + lo
__device__ __forceinline__ float ff_dot3(const float *ah, const float *al, const float *bh, const float *bl,
                                         float &lo) {
  float pe;
  float s = ff_two_prod(ah[0], bh[0], pe);
  float c = __fmaf_rn(al[0], bh[0], __fmaf_rn(ah[0], bl[0], pe));
#pragma unroll
  for (int k = 1; k < 3; k++) {
    float p = ff_two_prod(ah[k], bh[k], pe);
    float se;
    s = ff_two_sum(s, p, se);
    c = __fadd_rn(c, __fadd_rn(se, __fmaf_rn(al[k], bh[k], __fmaf_rn(ah[k], bl[k], pe))));
  }
  return ff_fast_two_sum(s, c, lo);
}

// (ah + al) / (bh + bl) as hi + lo, bh != 0: the quotient of the leading
// parts, then one correction from the remainder (computed with an FMA)
__device__ __forceinline__ float ff_div(float ah, float al, float bh, float bl, float rb, float &lo) {
  float q = __fmul_rn(ah, rb);
  float rho = __fmaf_rn(-q, bh, ah);
  rho = __fmaf_rn(-q, bl, __fadd_rn(rho, al));
  lo = __fmul_rn(rho, rb);
  return q;
}

// (ah + al) + (bh + bl), renormalised
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float e;
  float s = ff_two_sum(a.x, b.x, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float2 o;
  o.x = ff_fast_two_sum(s, e, o.y);
  return o;
}

// (ah + al) (bh + bl), renormalised (the al*bl term is below the precision)
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  float e;
  float p = ff_two_prod(a.x, b.x, e);
  e = __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.y, e));
  float2 o;
  o.x = ff_fast_two_sum(p, e, o.y);
  return o;
}

// running sum s (hi + lo) += x (one float), without renormalising
__device__ __forceinline__ void ff_acc(float &sh, float &sl, float x) {
  float e;
  sh = ff_two_sum(sh, x, e);
  sl = __fadd_rn(sl, e);
}

__device__ __forceinline__ float2 ff_of(double x) {
  float2 o;
  o.x = (float)x;
  o.y = (float)(x - (double)o.x);
  return o;
}

// Format changes without the FP64 pipe. On this GPU one FP64 instruction,
// conversions included, holds the SM's FP64 unit for 16 cycles per warp, so
// kernels that only move values between the two formats become FP64-bound.
// These build the IEEE-754 bit patterns with integer operations instead.

// float -> double, exact (zero and subnormal floats give a signed zero)
__device__ __forceinline__ double f2d(float f) {
  unsigned b = __float_as_uint(f);
  unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return __longlong_as_double((long long)sign);
  unsigned long long ed = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 1023u - 127u);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// double -> hi + lo: hi the value truncated to 24 significant bits (exact),
// lo the remaining 29 bits rounded to float (2^-48 relative in all). Values
// whose hi or lo would leave the normal float range take the FP64 route.
__device__ __forceinline__ float2 ff_split_bits(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  int e = (int)((u >> 52) & 0x7ffull);
  if (e == 0) return make_float2(0.f, 0.f);
  if (e < 949 || e > 1150) return ff_of(x);  // |x| < 2^-74 or >= 2^128 (or inf / NaN)
  unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  unsigned long long m = u & 0xfffffffffffffull;
  float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
  float lo = __fmul_rn(__uint2float_rn((unsigned)(m & 0x1fffffffull)), scale);
  return make_float2(hi, sign ? -lo : lo);
}

// hi + lo -> double: one FP64 add
__device__ __forceinline__ double ff_to_double(float2 a) { return f2d(a.x) + f2d(a.y); }

// host-side or device-side split of a double into hi + lo
__host__ __device__ __forceinline__ void ff_split(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Camera record of the FP32 form, FF_CAM floats (128 bytes, read as float4):
//   [0, 9) R hi (row-major)   [9, 12) centre C = -R^T t hi   [12, 15) C lo
//   [15] f hi                 [16, 25) R lo                   [25] f lo
//   [26] k1 hi  [27] k1 lo    [28] zero                       [29, 32) t rounded to FP32
// (k1: the first radial parameter of per-camera intrinsics, 0 without.)
// The FP32 projection and Jacobians read floats [0, 16), [24, 28) for k1 and
// [28, 32); the float-float residual reads [0, 28).
#define FF_CAM 32

__host__ __device__ inline void ff_camera_record(const double *R, const double *t, double f, double k1, float *o) {
  for (int e = 0; e < 9; e++) ff_split(R[e], o[e], o[16 + e]);
  for (int c = 0; c < 3; c++) {
    double C = -(R[c] * t[0] + R[3 + c] * t[1] + R[6 + c] * t[2]);
    ff_split(C, o[9 + c], o[12 + c]);
  }
  ff_split(f, o[15], o[25]);
  ff_split(k1, o[26], o[27]);
  o[28] = 0.f;
  for (int e = 0; e < 3; e++) o[29 + e] = (float)t[e];
}

// floats [0, 4 n4) of a record into registers
template <int N4>
__device__ __forceinline__ void ff_load_record(const float *cf, float (&c)[4 * N4]) {
  const float4 *p = reinterpret_cast<const float4 *>(cf);
#pragma unroll
  for (int e = 0; e < N4; e++) {
    float4 a = __ldg(p + e);
    c[4 * e] = a.x; c[4 * e + 1] = a.y; c[4 * e + 2] = a.z; c[4 * e + 3] = a.w;
  }
}

// Reprojection residual (Eq. ta) of a point X = Xh + Xl in the camera of
// record c (floats [0, 28) of it, in registers) against an observation given relative to the principal point as
// (oxh + oxl, oyh + oyl): X_c = R (X - C) as float-float, the perspective
// division with one remainder correction, f times the quotient, and the
// subtraction of the observation, whose leading parts cancel exactly. The
// residual is returned in FP32 (it is small: its leading bits are exact).
// Returns z_c > 0; the residual is computed either way, as in FP64. With
// k1on (per-camera intrinsics) f is replaced by f (1 + k1 |q|^2), q the
// normalised coordinates, all in float-float.
__device__ __forceinline__ bool ff_residual_rec(const float (&c)[28], const float *Xh, const float *Xl, float oxh,
                                                float oxl, float oyh, float oyl, float &r0, float &r1,
                                                bool k1on = false) {
  float dh[3], dl[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float e;
    dh[k] = ff_two_sum(Xh[k], -c[9 + k], e);
    dl[k] = __fadd_rn(e, __fsub_rn(Xl[k], c[12 + k]));
  }
  float xl, yl, zl;
  float xh = ff_dot3(c + 0, c + 16, dh, dl, xl);
  float yh = ff_dot3(c + 3, c + 19, dh, dl, yl);
  float zh = ff_dot3(c + 6, c + 22, dh, dl, zl);
  float rz = __frcp_rn(zh);
  float qxl, qyl;
  float qx = ff_div(xh, xl, zh, zl, rz, qxl);
  float qy = ff_div(yh, yl, zh, zl, rz, qyl);
  float fh = c[15], fl = c[25];
  if (k1on) {
    // f (1 + k1 |q|^2) in float-float: |q|^2 from the quotients and their
    // remainders, then k1 |q|^2, 1 + that, and the product with f
    float e1, e2, e3, te, se, ge;
    float r2h = ff_two_prod(qx, qx, e1);
    e1 = __fmaf_rn(2.f * qx, qxl, e1);
    float r2b = ff_two_prod(qy, qy, e2);
    e2 = __fmaf_rn(2.f * qy, qyl, e2);
    r2h = ff_two_sum(r2h, r2b, e3);
    float r2l = __fadd_rn(__fadd_rn(e1, e2), e3);
    float kh = c[26], kl = c[27];
    float th = ff_two_prod(kh, r2h, te);
    te = __fmaf_rn(kl, r2h, __fmaf_rn(kh, r2l, te));
    float sh = ff_two_sum(1.f, th, se);
    float sl = __fadd_rn(se, te);
    float gh = ff_two_prod(fh, sh, ge);
    ge = __fmaf_rn(fl, sh, __fmaf_rn(fh, sl, ge));
    fh = ff_two_sum(gh, ge, fl);
  }
  float ue, ve;
  float uh = ff_two_prod(fh, qx, ue);
  ue = __fmaf_rn(fl, qx, __fmaf_rn(fh, qxl, ue));
  float vh = ff_two_prod(fh, qy, ve);
  ve = __fmaf_rn(fl, qy, __fmaf_rn(fh, qyl, ve));
  r0 = __fadd_rn(__fsub_rn(uh, oxh), __fsub_rn(ue, oxl));
  r1 = __fadd_rn(__fsub_rn(vh, oyh), __fsub_rn(ve, oyl));
  return zh > 0.f;
}

// the same with the record read from global memory
__device__ __forceinline__ bool ff_residual(const float *cf, const float *Xh, const float *Xl, float oxh, float oxl,
                                            float oyh, float oyl, float &r0, float &r1, bool k1on = false) {
  float c[28];
  ff_load_record<7>(cf, c);
  return ff_residual_rec(c, Xh, Xl, oxh, oxl, oyh, oyl, r0, r1, k1on);
}

// Camera records staged in shared memory: FF_CAM_S float4 per record (seven
// used), the odd stride spreading neighbouring records over the banks
#define FF_CAM_S 9
__device__ __forceinline__ void ff_load_record_s(const float4 *p, float (&c)[28]) {
#pragma unroll
  for (int e = 0; e < 7; e++) {
    float4 a = p[e];
    c[4 * e] = a.x; c[4 * e + 1] = a.y; c[4 * e + 2] = a.z; c[4 * e + 3] = a.w;
  }
}

}  // namespace rpba
