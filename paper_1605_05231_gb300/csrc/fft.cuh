// Shared-memory Stockham FFT (mixed radix 2/3/4/5/8) for W interleaved columns.
//
// Element i of column c lives at buf[i * pitch + c]; all NT threads of the
// CTA cooperate.  Each stage reads every butterfly input into registers,
// barriers, then writes the outputs (so the transform is in place in shared
// memory).  Stage s of radix R with span Ns: butterfly j reads x[j + r L/R],
// multiplies by w^(k r), k = j mod Ns, w = exp(-+2 pi i / (Ns R)), applies the
// R-point DFT and writes y[(j / Ns) Ns R + k + r Ns] (Stockham autosort).
// Twiddles come from a table tw[i] = exp(-2 pi i i / L) built in FP64 on the
// host.  Forward (INV = false) is exp(-i), inverse exp(+i), both unnormalised.
#pragma once

#include "common.cuh"

namespace nufft {

__host__ __device__ constexpr int c_ilog2(int x) { int r = 0; while (x > 1) { x >>= 1; ++r; } return r; }
__host__ __device__ constexpr int c_count3(int L) { int c = 0; while (L % 3 == 0) { L /= 3; ++c; } return c; }
__host__ __device__ constexpr int c_count5(int L) { int c = 0; while (L % 5 == 0) { L /= 5; ++c; } return c; }
__host__ __device__ constexpr int c_pow2part(int L) {
  while (L % 3 == 0) L /= 3;
  while (L % 5 == 0) L /= 5;
  return L;
}
// stages: the radix-5 ones first, then radix 3, then the power of two as one
// radix-2 or radix-4 stage (if its exponent is not a multiple of 3) and radix 8
__host__ __device__ constexpr int fft_num_stages(int L) {
  return c_count5(L) + c_count3(L) + (c_ilog2(c_pow2part(L)) + 2) / 3;
}
__host__ __device__ constexpr int fft_stage_radix(int L, int s) {
  return s < c_count5(L)                 ? 5
         : s < c_count5(L) + c_count3(L) ? 3
         : ((c_ilog2(c_pow2part(L)) % 3 != 0 && s == c_count5(L) + c_count3(L))
                ? (c_ilog2(c_pow2part(L)) % 3 == 1 ? 2 : 4)
                : 8);
}
__host__ __device__ constexpr int fft_span_before(int L, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= fft_stage_radix(L, i);
  return ns;
}

// R-point DFT in registers (forward exp(-i), inverse exp(+i))
template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2* v);

template <>
__device__ __forceinline__ void small_dft<2, false>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void small_dft<2, true>(float2* v) { small_dft<2, false>(v); }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <>
__device__ __forceinline__ void small_dft<4, false>(float2* v) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void small_dft<4, true>(float2* v) { dft4<true>(v[0], v[1], v[2], v[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  // even / odd split: E = DFT4(v0, v2, v4, v6), O = DFT4(v1, v3, v5, v7)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float h = 0.70710678118654752440f;  // 1 / sqrt(2)
  // w8^1 = (1 -+ i)/sqrt2, w8^2 = -+i, w8^3 = (-1 -+ i)/sqrt2
  float2 t1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
                  : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  float2 t2 = mul_mi<INV>(o2);
  float2 t3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y))
                  : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}
template <>
__device__ __forceinline__ void small_dft<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void small_dft<8, true>(float2* v) { dft8<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float s3 = 0.86602540378443864676f;  // sqrt(3) / 2
  float2 t = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
  // (-+ i sqrt3/2) d
  float2 r = INV ? make_float2(-s3 * d.y, s3 * d.x) : make_float2(s3 * d.y, -s3 * d.x);
  v[0] = cadd(v[0], t);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}
template <>
__device__ __forceinline__ void small_dft<3, false>(float2* v) { dft3<false>(v); }
template <>
__device__ __forceinline__ void small_dft<3, true>(float2* v) { dft3<true>(v); }

// 5-point DFT: with t1 = v1 + v4, t2 = v2 + v3, d1 = v1 - v4, d2 = v2 - v3,
// y0 = v0 + t1 + t2, y1,4 = v0 + c1 t1 + c2 t2 -+ i (s1 d1 + s2 d2),
// y2,3 = v0 + c2 t1 + c1 t2 -+ i (s2 d1 - s1 d2) (forward; the inverse swaps
// the signs of i), c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5)
template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
  const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  const float2 b1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
  const float2 b2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
  // -i b (forward) or +i b (inverse)
  const float2 m1 = mul_mi<INV>(b1), m2 = mul_mi<INV>(b2);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, m1);
  v[4] = csub(a1, m1);
  v[2] = cadd(a2, m2);
  v[3] = csub(a2, m2);
}
template <>
__device__ __forceinline__ void small_dft<5, false>(float2* v) { dft5<false>(v); }
template <>
__device__ __forceinline__ void small_dft<5, true>(float2* v) { dft5<true>(v); }

// v[r] *= w^r (w = tw[b], conjugated for the inverse), r = 1 .. R-1.  w and
// w^2 come from the table; the higher powers are products of two lower ones
// (w^3 = w w^2, w^4 = w^2 w^2, w^5 = w^2 w^3, w^6 = w^3 w^3, w^7 = w^3 w^4),
// at most two roundings deep, so a butterfly reads two table entries instead
// of R - 1 (the table reads share the L1 path with the shared-memory
// exchanges of the stage).
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles(float2* v, const float2* __restrict__ tw, int b) {
  float2 w[R];
  w[1] = __ldg(&tw[b]);
  if (INV) w[1].y = -w[1].y;
  if (R > 2) {
    w[2] = __ldg(&tw[2 * b]);
    if (INV) w[2].y = -w[2].y;
  }
#pragma unroll
  for (int r = 3; r < R; ++r) w[r] = cmul(w[r / 2], w[r - r / 2]);
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
}

template <int L, int R, int NS, int W, int NT, bool INV>
__device__ __forceinline__ void stockham_stage(float2* buf, int pitch, const float2* __restrict__ tw) {
  constexpr int NBF = W * (L / R);
  constexpr int PER = (NBF + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = threadIdx.x + p * NT;
    if (NBF % NT == 0 || b < NBF) {
      const int c = b % W, j = b / W;
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = buf[(j + r * (L / R)) * pitch + c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = threadIdx.x + p * NT;
    if (NBF % NT == 0 || b < NBF) {
      const int c = b % W, j = b / W;
      const int k = j % NS;
      if (NS > 1) apply_twiddles<R, INV>(v[p], tw, k * (L / (NS * R)));
      small_dft<R, INV>(v[p]);
      const int o = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(o + r * NS) * pitch + c] = v[p][r];
    }
  }
  __syncthreads();
}

template <int L, int W, int NT, bool INV, int S = 0, int SEND = fft_num_stages(L)>
__device__ __forceinline__ void smem_fft(float2* buf, int pitch, const float2* __restrict__ tw) {
  if constexpr (S < SEND) {
    constexpr int R = fft_stage_radix(L, S);
    constexpr int NS = fft_span_before(L, S);
    stockham_stage<L, R, NS, W, NT, INV>(buf, pitch, tw);
    smem_fft<L, W, NT, INV, S + 1, SEND>(buf, pitch, tw);
  }
}

// The same transform with the first stage fed from registers loaded straight
// from global memory and the last stage written straight to global memory:
// shared memory carries only the exchanges between stages (one write and one
// read per element and exchange, instead of an extra staging write and read
// at each end), and zero rows of a padded input are never touched.
// load(i, c) returns input row i of column c; store(i, c, v) writes output row
// i.  The first stage has span 1 (no twiddles); the last stage's butterfly j
// writes rows j + r L / R.
struct NoPostLoad {
  __device__ __forceinline__ void operator()(int, int) const {}
};

// Optional scaling of the butterflies' inputs (first stage, after the loads,
// before the first radix-R DFT of inputs j + r L/R) and of their outputs (last
// stage, after the last DFT, before the stores of outputs j + r L/R).
struct NoHook {
  template <int R>
  __device__ __forceinline__ void first(float2 (&)[R], int, int) const {}
  template <int R>
  __device__ __forceinline__ void last(float2 (&)[R], int, int) const {}
};

// post_load(i, c) runs once for every input row i and column c after the
// first barrier, when every first-stage load of the CTA has completed (it is
// called from the last stage, whose rows j + r NS cover each row once; a
// consumer that clears its input does it there, so that no load waits behind a
// store to a possibly aliasing address and no load address stays live).
template <int L, int W, int NT, bool INV, class Load, class Store, class PostLoad = NoPostLoad,
          class Hook = NoHook>
__device__ __forceinline__ void reg_fft(float2* buf, int pitch, const float2* __restrict__ tw, Load&& load,
                                        Store&& store, PostLoad&& post_load = PostLoad{}, Hook&& hook = Hook{}) {
  constexpr int S = fft_num_stages(L);
  static_assert(S >= 2, "reg_fft needs at least two stages");
  {
    constexpr int R = fft_stage_radix(L, 0);
    constexpr int NBF = W * (L / R);
    constexpr int PER = (NBF + NT - 1) / NT;
    // all of this thread's loads are issued before the first butterfly (more
    // bytes in flight per SM); two butterflies per thread at 512 threads
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int b = threadIdx.x + p * NT;
      if (NBF % NT == 0 || b < NBF) {
        const int c = b % W, j = b / W;
#pragma unroll
        for (int r = 0; r < R; ++r) v[p][r] = load(j + r * (L / R), c);
      }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int b = threadIdx.x + p * NT;
      if (NBF % NT == 0 || b < NBF) {
        const int c = b % W, j = b / W;
        hook.template first<R>(v[p], j, c);
        small_dft<R, INV>(v[p]);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(j * R + r) * pitch + c] = v[p][r];
      }
    }
    __syncthreads();
  }
  smem_fft<L, W, NT, INV, 1, S - 1>(buf, pitch, tw);
  {
    constexpr int R = fft_stage_radix(L, S - 1);
    constexpr int NS = L / R;
    constexpr int NBF = W * NS;
    constexpr int PER = (NBF + NT - 1) / NT;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int b = threadIdx.x + p * NT;
      if (NBF % NT == 0 || b < NBF) {
        const int c = b % W, j = b / W;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[(j + r * NS) * pitch + c];
        apply_twiddles<R, INV>(v, tw, j);
        small_dft<R, INV>(v);
        hook.template last<R>(v, j, c);
#pragma unroll
        for (int r = 0; r < R; ++r) store(j + r * NS, c, v[r]);
#pragma unroll
        for (int r = 0; r < R; ++r) post_load(j + r * NS, c);
      }
    }
  }
}

}  // namespace nufft
