// Shared device helpers of the radial-line 3D NUFFT library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace nufft {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 (x = real, y = imaginary)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc += a * b
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += s * b (s real)
__device__ __forceinline__ void rmac(float2& acc, float s, float2 b) {
  acc.x = fmaf(s, b.x, acc.x);
  acc.y = fmaf(s, b.y, acc.y);
}

// ---------------------------------------------------------------------------
// grid storage types: complex64, or a pair of bf16 / fp16 with a global scale
// ---------------------------------------------------------------------------
// Power-of-two scale for a reduced-precision grid from a bound on |Y|: the
// scaled grid stays below 2^14 (inside fp16's range, with headroom).
__device__ __forceinline__ float lp_scale_from_bound(float bound) {
  const float b = fmaxf(bound, 1e-30f);
  float e = floorf(__log2f(16384.f / b));
  e = fminf(fmaxf(e, -100.f), 100.f);
  return exp2f(e);
}

struct GridC64 {
  typedef float2 T;
  static constexpr bool kLowPrecision = false;
  static __device__ __forceinline__ float2 to_f2(T v) { return v; }
  static __device__ __forceinline__ float2 load(const T* p, size_t i, float) { return p[i]; }
  static __device__ __forceinline__ T pack(float2 v, float) { return v; }
};
struct GridBF16 {
  typedef __nv_bfloat162 T;
  static constexpr bool kLowPrecision = true;
  static __device__ __forceinline__ float2 to_f2(T v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ float2 load(const T* p, size_t i, float inv_scale) {
    float2 v = __bfloat1622float2(p[i]);
    return make_float2(v.x * inv_scale, v.y * inv_scale);
  }
  static __device__ __forceinline__ T pack(float2 v, float scale) {
    return __floats2bfloat162_rn(v.x * scale, v.y * scale);
  }
};
struct GridF16 {
  typedef __half2 T;
  static constexpr bool kLowPrecision = true;
  static __device__ __forceinline__ float2 to_f2(T v) { return __half22float2(v); }
  static __device__ __forceinline__ float2 load(const T* p, size_t i, float inv_scale) {
    float2 v = __half22float2(p[i]);
    return make_float2(v.x * inv_scale, v.y * inv_scale);
  }
  static __device__ __forceinline__ T pack(float2 v, float scale) {
    return __floats2half2_rn(v.x * scale, v.y * scale);
  }
};

// ---------------------------------------------------------------------------
// coordinate reduction: u = r * d (both given as unevaluated FP32 pairs
// hi + lo) split into floor(u) and f = u - floor(u) in [0, 1).
//
// The product r_hi * d_hi is formed exactly as p + e (FMA two-product); the
// cross terms r_hi d_lo + r_lo d_hi are added as a correction; floor is taken
// on p (p - floor(p) is exact below 2^23) and the correction moves f across
// an integer boundary when needed.  The result agrees with FP64 rounding of u
// to about 2^-24 in f, so FP64 units are not needed on the GPU.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_coord(float r_hi, float r_lo, float d_hi, float d_lo,
                                             int& fl_out, float& f_out) {
  float p = __fmul_rn(r_hi, d_hi);
  float e = __fmaf_rn(r_hi, d_hi, -p);
  float c = __fmaf_rn(r_hi, d_lo, __fmaf_rn(r_lo, d_hi, e));
  float fl = floorf(p);
  float fr = __fsub_rn(p, fl);
  float f = __fadd_rn(fr, c);
  if (f < 0.f) {
    f = __fadd_rn(f, 1.f);
    fl -= 1.f;
    if (f >= 1.f) f = 0.99999994f;
  } else if (f >= 1.f) {
    f = __fsub_rn(f, 1.f);
    fl += 1.f;
  }
  fl_out = (int)fl;
  f_out = f;
}

// Min-max coefficients of one axis from the table (L + 1 rows of J complex
// values at f_i = i / L), linearly interpolated in f.
template <int J>
__device__ __forceinline__ void table_coeffs(const float2* __restrict__ table, int L, float f, float2 (&c)[J]) {
  float fl = f * (float)L;
  int i = (int)fl;
  if (i > L - 1) i = L - 1;
  float t = fl - (float)i;
  const float2* r0 = table + (size_t)i * J;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float2 a = __ldg(r0 + j);
    float2 b = __ldg(r0 + J + j);
    c[j] = make_float2(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y));
  }
}

// Same as table_coeffs, reading rows i and i + 1 (2 J contiguous values) as J
// float4 loads (J even; rows are 16-byte aligned).
template <int J>
__device__ __forceinline__ void table_coeffs_v4(const float2* __restrict__ table, int L, float f, float2 (&c)[J]) {
  float fl = f * (float)L;
  int i = (int)fl;
  if (i > L - 1) i = L - 1;
  const float t = fl - (float)i;
  const float4* r = (const float4*)(table + (size_t)i * J);
  float4 v[J];
#pragma unroll
  for (int q = 0; q < J; ++q) v[q] = __ldg(r + q);
#pragma unroll
  for (int q = 0; q < J / 2; ++q) {
    const float4 a = v[q], b = v[q + J / 2];
    c[2 * q] = make_float2(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y));
    c[2 * q + 1] = make_float2(fmaf(t, b.z - a.z, a.z), fmaf(t, b.w - a.w, a.w));
  }
}

// device check word codes
enum : int { DEVCHK_TILE_RANGE = -6 };

}  // namespace nufft
