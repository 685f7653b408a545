// Direct resampling of the polar Radon grid (Sec. 2.1, Eq. 2.15 with T2 = I):
// the radially sampled Radon data are uniform in (s, theta, phi) (Fig. 2.10),
// and a separable truncated-sinc interpolator takes them to arbitrary points:
//
//   x~(u) = sum_{k} sinc(u_s - k_s) sinc(u_theta - k_theta) sinc(u_phi - k_phi)
//                  x[k_phi mod n_phi, k_theta, k_s],
//
// with the J integers k0 .. k0 + J - 1, k0 = floor(u - J/2) + 1, on every axis;
// the azimuth is periodic, taps beyond the ends of the theta and s ranges add
// nothing.  The paper's runs use J = 3 ([3 3 3], Sec. 3.2).
//
// One thread per target.  The J sinc weights of an axis share one sine:
// sin(pi (u - k)) = (-1)^k sin(pi u), so an axis costs one sinpi and J
// divisions.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nufft {

constexpr int POLAR_NT = 256;


// weights and grid indices of one axis: periodic axes wrap the index; on the
// others a tap beyond [0, n) gets weight 0 and a safe index
template <int J>
__device__ __forceinline__ void sinc_axis(float u, int n, bool periodic, float (&w)[J], int (&k)[J]) {
  const int k0 = (int)floorf(u - 0.5f * (float)J) + 1;
  const float su = sinpif(u);
  constexpr float kInvPi = 0.318309886183790671537767526745f;
  // periodic axis: one modulo for the first tap, then wrap by subtraction
  // (one subtraction suffices when the period is at least J)
  int p0 = 0;
  if (periodic) {
    p0 = k0 % n;
    p0 += p0 < 0 ? n : 0;
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int kj = k0 + j;
    const float t = u - (float)kj;
    float wj = t == 0.f ? 1.f : __fdividef(((kj & 1) ? -su : su) * kInvPi, t);
    int idx = kj;
    if (periodic) {
      idx = p0 + j;
      if (n >= J) {
        idx -= idx >= n ? n : 0;
      } else {
        idx %= n;
      }
    } else {
      const bool inside = (unsigned)kj < (unsigned)n;
      wj = inside ? wj : 0.f;
      idx = inside ? kj : 0;
    }
    w[j] = wj;
    k[j] = idx;
  }
}

// One non-periodic axis with the J taps kept consecutive: they run from
// base = clamp(k0, 0, n - J) (n >= J), and a tap outside k0 .. k0 + J - 1 gets
// weight 0, so the same taps add the same terms as sinc_axis while the
// addresses of the J taps differ by constants.
template <int J>
__device__ __forceinline__ int sinc_axis_contig(float u, int n, float (&w)[J]) {
  const int k0 = (int)floorf(u - 0.5f * (float)J) + 1;
  const int base = min(max(k0, 0), n - J);
  const float su = sinpif(u);
  constexpr float kInvPi = 0.318309886183790671537767526745f;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int kj = base + j;
    const float t = u - (float)kj;
    const float wj = t == 0.f ? 1.f : __fdividef(((kj & 1) ? -su : su) * kInvPi, t);
    w[j] = (unsigned)(kj - k0) < (unsigned)J ? wj : 0.f;
  }
  return base;
}

// The periodic axis: the J taps wrapped into [0, n) (n >= J); the first by
// one add when k0 is within a period of the range, else by a modulo.
template <int J>
__device__ __forceinline__ void sinc_axis_periodic(float u, int n, float (&w)[J], int (&k)[J]) {
  const int k0 = (int)floorf(u - 0.5f * (float)J) + 1;
  const float su = sinpif(u);
  constexpr float kInvPi = 0.318309886183790671537767526745f;
  int p0 = k0;
  if ((unsigned)(k0 + n) < (unsigned)(2 * n)) {
    p0 += k0 < 0 ? n : 0;
  } else {
    p0 = k0 % n;
    p0 += p0 < 0 ? n : 0;
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int kj = k0 + j;
    const float t = u - (float)kj;
    w[j] = t == 0.f ? 1.f : __fdividef(((kj & 1) ? -su : su) * kInvPi, t);
    const int idx = p0 + j;
    k[j] = idx - (idx >= n ? n : 0);
  }
}

// CONTIG: every axis has at least J cells and the grid fewer than 2^31 cells,
// so taps are consecutive along s and theta and offsets fit in 32 bits.
template <int J, bool CONTIG>
__device__ __forceinline__ void polar_resample_targets(const float2* __restrict__ grid, int n_phi, int n_theta,
                                                       int n_s, const float* __restrict__ targets, long long n,
                                                       float2* __restrict__ out) {
  const long long stride = (long long)gridDim.x * POLAR_NT;
  for (long long i = (long long)blockIdx.x * POLAR_NT + threadIdx.x; i < n; i += stride) {
    const float us = targets[3 * i], ut = targets[3 * i + 1], up = targets[3 * i + 2];
    // coordinates must be finite and below 2^24 in magnitude (exact integers in float)
    const float lim = 16777216.f;
    if (!(fabsf(us) < lim && fabsf(ut) < lim && fabsf(up) < lim)) {
      out[i] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
      continue;
    }
    float ws[J], wt[J], wp[J];
    float2 acc = make_float2(0.f, 0.f);
    if constexpr (CONTIG) {
      int kp[J];
      const int bs = sinc_axis_contig<J>(us, n_s, ws);
      const int bt = sinc_axis_contig<J>(ut, n_theta, wt);
      sinc_axis_periodic<J>(up, n_phi, wp, kp);
      // all J^3 loads independent and in flight at once; the J of a row at
      // constant offsets from one address
#pragma unroll
      for (int a = 0; a < J; ++a) {
        float2 pacc = make_float2(0.f, 0.f);
        const int plane = (kp[a] * n_theta + bt) * n_s + bs;
#pragma unroll
        for (int b = 0; b < J; ++b) {
          const float2* row = grid + (plane + b * n_s);
          float2 racc = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < J; ++c) {
            const float2 v = __ldg(row + c);
            racc.x = fmaf(ws[c], v.x, racc.x);
            racc.y = fmaf(ws[c], v.y, racc.y);
          }
          pacc.x = fmaf(wt[b], racc.x, pacc.x);
          pacc.y = fmaf(wt[b], racc.y, pacc.y);
        }
        acc.x = fmaf(wp[a], pacc.x, acc.x);
        acc.y = fmaf(wp[a], pacc.y, acc.y);
      }
    } else {
      int ks[J], kt[J], kp[J];
      sinc_axis<J>(us, n_s, false, ws, ks);
      sinc_axis<J>(ut, n_theta, false, wt, kt);
      sinc_axis<J>(up, n_phi, true, wp, kp);
#pragma unroll
      for (int a = 0; a < J; ++a) {
        const float2* plane = grid + (size_t)kp[a] * n_theta * n_s;
        float2 pacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < J; ++b) {
          const float2* row = plane + (size_t)kt[b] * n_s;
          float2 racc = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < J; ++c) {
            const float2 v = __ldg(row + ks[c]);
            racc.x = fmaf(ws[c], v.x, racc.x);
            racc.y = fmaf(ws[c], v.y, racc.y);
          }
          pacc.x = fmaf(wt[b], racc.x, pacc.x);
          pacc.y = fmaf(wt[b], racc.y, pacc.y);
        }
        acc.x = fmaf(wp[a], pacc.x, acc.x);
        acc.y = fmaf(wp[a], pacc.y, acc.y);
      }
    }
    out[i] = acc;
  }
}

template <int J, bool CONTIG>
__global__ void __launch_bounds__(POLAR_NT) k_polar_resample(const float2* __restrict__ grid, int n_phi, int n_theta,
                                                            int n_s, const float* __restrict__ targets,
                                                            long long n, float2* __restrict__ out) {
  polar_resample_targets<J, CONTIG>(grid, n_phi, n_theta, n_s, targets, n, out);
}

// J <= 3 with consecutive taps fits in 32 registers: eight CTAs (64 warps) per
// SM to hide the latency of the tap loads.  (A minimum-blocks bound on the
// other instances made the compiler use registers up to its cap, so they keep
// the plain bound.)
template <int J>
__global__ void __launch_bounds__(POLAR_NT, 8) k_polar_resample_contig8(const float2* __restrict__ grid, int n_phi,
                                                                       int n_theta, int n_s,
                                                                       const float* __restrict__ targets, long long n,
                                                                       float2* __restrict__ out) {
  polar_resample_targets<J, true>(grid, n_phi, n_theta, n_s, targets, n, out);
}

// one target per thread: blocks start in target order, so the grid rows in
// use at any time stay within a few phi slices and are re-read from L2
static int polar_grid_cap() { return 1 << 30; }

template <int J>
static cudaError_t launch_polar_t(const float2* grid, int n_phi, int n_theta, int n_s, const float* targets,
                                  long long n, float2* out, cudaStream_t st) {
  const long long blocks = (n + POLAR_NT - 1) / POLAR_NT;
  const int cap = polar_grid_cap();
  const int nb = (int)(blocks < cap ? blocks : cap);
  const bool contig = n_s >= J && n_theta >= J && n_phi >= J && (long long)n_phi * n_theta * n_s < (1LL << 31);
  if constexpr (J <= 3) {
    if (contig) {
      k_polar_resample_contig8<J><<<nb, POLAR_NT, 0, st>>>(grid, n_phi, n_theta, n_s, targets, n, out);
      return cudaGetLastError();
    }
  } else {
    if (contig) {
      k_polar_resample<J, true><<<nb, POLAR_NT, 0, st>>>(grid, n_phi, n_theta, n_s, targets, n, out);
      return cudaGetLastError();
    }
  }
  k_polar_resample<J, false><<<nb, POLAR_NT, 0, st>>>(grid, n_phi, n_theta, n_s, targets, n, out);
  return cudaGetLastError();
}

cudaError_t launch_polar_resample(const float2* grid, int n_phi, int n_theta, int n_s, const float* targets,
                                  long long n, int J, float2* out, cudaStream_t st) {
  switch (J) {
    case 2: return launch_polar_t<2>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 3: return launch_polar_t<3>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 4: return launch_polar_t<4>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 5: return launch_polar_t<5>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 6: return launch_polar_t<6>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 7: return launch_polar_t<7>(grid, n_phi, n_theta, n_s, targets, n, out, st);
    case 8: return launch_polar_t<8>(grid, n_phi, n_theta, n_s, targets, n, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nufft

extern "C" int nufft3d_polar_resample(const void* grid_dev, int n_phi, int n_theta, int n_s,
                                      const float* targets_dev, long long n_targets, int J, void* out_dev,
                                      void* cuda_stream) {
  if (n_targets < 0 || n_phi < 1 || n_theta < 1 || n_s < 1 || J < 2 || J > 8) return NUFFT3D_ERR_ARG;
  if ((long long)n_phi * n_theta * n_s > (1LL << 40)) return NUFFT3D_ERR_ARG;
  if (n_targets == 0) return NUFFT3D_OK;
  if (!grid_dev || !targets_dev || !out_dev) return NUFFT3D_ERR_ARG;
  const cudaError_t e = nufft::launch_polar_resample((const float2*)grid_dev, n_phi, n_theta, n_s, targets_dev,
                                                     n_targets, J, (float2*)out_dev, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? NUFFT3D_OK : NUFFT3D_ERR_CUDA;
}
