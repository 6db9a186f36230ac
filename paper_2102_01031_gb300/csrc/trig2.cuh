// trig2.cuh -- sines and cosines of FP32 link and plaquette angles two at a time,
// for the gauge passes: the polynomials of the scalar FP32 sine and cosine
// (common.cuh) in the packed two-lane form (one FFMA2 / FMUL2 for both lanes,
// each lane rounded as the scalar form), with one range check for many angles.
#pragma once

#include "common.cuh"

namespace clg {

constexpr float TRIG_PI4 = 0.78539816f;  // the polynomials' range, |x| <= pi/4

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sin_taylor2(float2 x2) {
  float2 p = __ffma2_rn(x2, f2(1.f / 362880.f), f2(-1.f / 5040.f));
  p = __ffma2_rn(x2, p, f2(1.f / 120.f));
  p = __ffma2_rn(x2, p, f2(-1.f / 6.f));
  return __ffma2_rn(x2, p, f2(1.f));
}
__device__ __forceinline__ float2 cos_taylor2(float2 x2) {
  float2 p = __ffma2_rn(x2, f2(-1.f / 3628800.f), f2(1.f / 40320.f));
  p = __ffma2_rn(x2, p, f2(-1.f / 720.f));
  p = __ffma2_rn(x2, p, f2(1.f / 24.f));
  p = __ffma2_rn(x2, p, f2(-0.5f));
  return __ffma2_rn(x2, p, f2(1.f));
}

// One angle, every product rounded on its own, so that an in-range angle gets
// the packed lanes' value wherever it is evaluated; beyond pi/4 the library.
__device__ __forceinline__ float sin_rn(float x) {
  if (fabsf(x) <= TRIG_PI4) return __fmul_rn(x, sin_taylor(__fmul_rn(x, x)));
  return sin_slow(x);
}
__device__ __forceinline__ void sincos_rn(float x, float& s, float& c) {
  if (fabsf(x) <= TRIG_PI4) {
    const float x2 = __fmul_rn(x, x);
    s = __fmul_rn(x, sin_taylor(x2));
    c = cos_taylor(x2);
  } else {
    sincos_slow(x, &s, &c);
  }
}

// Two angles.  Where either is beyond pi/4 each lane takes the one-angle path,
// so an angle gets the same value whichever angle it is paired with.
__device__ __forceinline__ void sincos2_t(float2 x, float2& s, float2& c) {
  if (fmaxf(fabsf(x.x), fabsf(x.y)) <= TRIG_PI4) {
    const float2 x2 = __fmul2_rn(x, x);
    s = __fmul2_rn(x, sin_taylor2(x2));
    c = cos_taylor2(x2);
  } else {
    sincos_rn(x.x, s.x, c.x);
    sincos_rn(x.y, s.y, c.y);
  }
}
__device__ __forceinline__ float2 sin2_t(float2 x) {
  if (fmaxf(fabsf(x.x), fabsf(x.y)) <= TRIG_PI4) return __fmul2_rn(x, sin_taylor2(__fmul2_rn(x, x)));
  return make_float2(sin_rn(x.x), sin_rn(x.y));
}

// Sines of the N angles x[]: one range check for all of them, then the
// polynomials two angles at a time in one block (independent chains the
// scheduler interleaves; an odd last angle fills both lanes of its pair).
// Where any angle is beyond pi/4 every angle takes the one-angle path.
template <int N>
__device__ __forceinline__ void sin_many(const float (&x)[N], float (&s)[N]) {
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) m = fmaxf(m, fabsf(x[k]));
  if (m <= TRIG_PI4) {
#pragma unroll
    for (int k = 0; k < N; k += 2) {
      const float2 v = make_float2(x[k], x[k + 1 < N ? k + 1 : k]);
      const float2 r = __fmul2_rn(v, sin_taylor2(__fmul2_rn(v, v)));
      s[k] = r.x;
      if (k + 1 < N) s[k + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = sin_rn(x[k]);
  }
}
template <int N>
__device__ __forceinline__ void sin_many(const double (&x)[N], double (&s)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) s[k] = sin_t(x[k]);
}
__device__ __forceinline__ double sin_rn(double x) { return sin_t(x); }
__device__ __forceinline__ void sincos_rn(double x, double& s, double& c) { sincos_t(x, s, c); }

}  // namespace clg
