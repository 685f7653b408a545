// NUFFT-based resampling of the polar Radon grid (Sec. 2.1.3, Eqs. 2.8-2.11):
//
//   x~ ~= T_sparse F P F^-1 x,
//
// x uniform on the polar grid x[phi][theta][s] (Fig. 2.10), x~ at arbitrary
// targets u = (u_s, u_theta, u_phi) in grid-index units.  Every axis is
// periodic, as the DFT makes it.  Per axis a with n_a points (even) and
// K_a = 2 n_a (the twofold oversampling the paper prefers):
//
//   F^-1  a[m] = (1/n) sum_k x[k] e^{+2 pi i m k / n}, m = -n/2 .. n/2 - 1;
//   P     the Kaiser-Bessel pre-window s(m) = Psi(0) / Psi((m + 1/2) / K),
//         symmetric about the middle of the index range;
//   F     the unnormalised K-point DFT (e^{-i}) of the zero-padded result;
//   T     the J-tap min-max interpolator at u' = 2 u (omega / gamma).
//
// F P F^-1 is a tensor product of per-axis maps n_a -> K_a, so it runs as
// three HBM-bound passes, one per axis (s, then theta, then phi), each
// reading its lines once, taking the n-point inverse DFT and the pre-window
// (with 1/n folded in) in shared memory, and writing K-point lines.  For
// power-of-two n the 2n-point DFT of the zero-padded spectrum g is taken as
// two n-point DFTs: its even outputs Y[2k] are the n-point DFT of g and its
// odd outputs Y[2k + 1] that of g[m] e^{-i pi m / n} (m the centred index),
// so no zero is stored or transformed; other n pad and take one 2n-point DFT.  The min-max coefficients factor as
// c_j(f) = e^{i gamma (f + J/2 - j)/2} rho_j(f) with rho_j real (the window is
// symmetric), so each pass also multiplies its output by the axis phase
// e^{-i pi k_c / K} (k_c the centred index), and the gather applies real
// weights rho_j (sign-flipped where a tap wraps across the centred range) and
// one phase e^{i pi (u'_s/K_s + u'_theta/K_theta + u'_phi/K_phi)} per target.
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "fft.cuh"
#include "host_math.h"
#include "internal.h"

namespace nufft {

constexpr int PN_NT = 256;     // threads of an axis-pass CTA
constexpr int PN_CHUNK = 8;    // loads a thread issues before its shared stores
constexpr int PG_NT = 256;     // threads of a gather CTA

// Power-of-two lengths take the 2n-point DFT of the padded spectrum as two
// n-point DFTs of 2W columns (no zeros stored or transformed); the others (the
// radix-5 lengths) keep one K-point DFT of W columns, which measured faster
// for the 360-point azimuths (3.05 against 3.62 ms at 720 x 512 x 1024).
// Lines per CTA: 16 (128-byte segments of the strided passes) while the
// buffer stays under 100 KB, else 8.
template <int N>
struct AxisShape {
  static constexpr int K = 2 * N;
  static constexpr bool SPLIT = (N & (N - 1)) == 0;
  static constexpr int W = (SPLIT ? N * 33 * 8 : K * 17 * 8) <= 100 * 1024 ? 16 : 8;
  static constexpr int P = SPLIT ? 2 * W + 1 : W + 1;  // odd pitch: conflict-free column and row accesses
  static constexpr size_t smem = (size_t)(SPLIT ? N : K) * P * sizeof(float2);
};

// One axis of F P F^-1 for W lines per CTA.
//   row kind (the contiguous s axis): in [lines][N] -> out [lines][K],
//     blockIdx.x over groups of W lines;
//   column kind: in [outer][N][S] -> out [outer][K][S], blockIdx.x over groups
//     of W consecutive columns, blockIdx.y = outer.
// The inverse DFT runs on columns 0 .. W-1 of the buffer.  Split form: g =
// s a / N goes to column c and g e^{-i pi m / N} to column W + c, and one
// forward N-point DFT of the 2W columns gives output row 2k (column c) and
// 2k + 1 (column W + c).  Padded form: g moves to row m mod K of a K-row
// buffer, the rest is zeroed, and one forward K-point DFT follows.
// sq[q] = s(m(q)) / N and sqr[q] = sq[q] e^{-i pi m(q) / N} for the inverse
// DFT's output index q (m = q, or q - N for q >= N/2); twN / twK the forward
// twiddles of N and K points; ph[k] the axis phase e^{-i pi k_c / K}.
template <int N>
__global__ void __launch_bounds__(PN_NT) k_axis_pass(const float2* __restrict__ in, float2* __restrict__ out,
                                                     int row_kind, long long n_lines, long long S,
                                                     const float* __restrict__ sq, const float2* __restrict__ twN,
                                                     const float2* __restrict__ sqr, const float2* __restrict__ twK,
                                                     const float2* __restrict__ ph) {
  using A = AxisShape<N>;
  constexpr int K = A::K, W = A::W, P = A::P, H = N / 2;
  extern __shared__ float2 buf[];
  const float2 zero = make_float2(0.f, 0.f);
  const long long g0 = (long long)blockIdx.x * W;  // first line (row kind) or column (column kind)
  const size_t in_base = row_kind ? 0 : (size_t)blockIdx.y * N * (size_t)S;
  const size_t out_base = row_kind ? 0 : (size_t)blockIdx.y * K * (size_t)S;
  // load: a thread's PN_CHUNK loads are in flight together
  for (int base = threadIdx.x; base < W * N; base += PN_CHUNK * PN_NT) {
    float2 t[PN_CHUNK];
#pragma unroll
    for (int u = 0; u < PN_CHUNK; ++u) {
      const int e = base + u * PN_NT;
      t[u] = zero;
      if (e < W * N) {
        if (row_kind) {
          const int c = e / N, i = e - c * N;
          if (g0 + c < n_lines) t[u] = __ldg(in + (size_t)(g0 + c) * N + i);
        } else {
          const int i = e / W, c = e - i * W;
          if (g0 + c < S) t[u] = __ldg(in + in_base + (size_t)i * S + (size_t)(g0 + c));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < PN_CHUNK; ++u) {
      const int e = base + u * PN_NT;
      if (e < W * N) {
        int c, i;
        if (row_kind) {
          c = e / N;
          i = e - c * N;
        } else {
          i = e / W;
          c = e - i * W;
        }
        buf[i * P + c] = t[u];
      }
    }
  }
  __syncthreads();
  // F^-1 (unnormalised; 1/N is in sq)
  smem_fft<N, W, PN_NT, true>(buf, P, twN);
  if constexpr (A::SPLIT) {
    // P, and the odd half's modulation
    for (int e = threadIdx.x; e < W * N; e += PN_NT) {
      const int i = e / W, c = e - i * W;
      const float2 a = buf[i * P + c];
      buf[i * P + c] = cscale(a, __ldg(sq + i));
      buf[i * P + W + c] = cmul(a, __ldg(sqr + i));
    }
    __syncthreads();
    // F: the even and odd outputs of the zero-padded K-point DFT
    smem_fft<N, 2 * W, PN_NT, false>(buf, P, twN);
  } else {
    // P and the zero padding: q < N/2 stays at row q, q >= N/2 (m = q - N)
    // moves to row q + N (= m mod K); the source and target rows are disjoint
    for (int e = threadIdx.x; e < W * H; e += PN_NT) {
      const int i = e / W, c = e - i * W;
      buf[i * P + c] = cscale(buf[i * P + c], __ldg(sq + i));
      buf[(i + H + N) * P + c] = cscale(buf[(i + H) * P + c], __ldg(sq + i + H));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * N; e += PN_NT) {
      const int i = e / W + H, c = e - (e / W) * W;
      buf[i * P + c] = zero;
    }
    __syncthreads();
    // F
    smem_fft<K, W, PN_NT, false>(buf, P, twK);
  }
  // store with the axis phase (split form: output row k from row k / 2 of
  // column c + (k odd) W)
  auto at = [&](int k, int c) -> float2 {
    if constexpr (A::SPLIT) return buf[(k >> 1) * P + c + ((k & 1) ? W : 0)];
    else return buf[k * P + c];
  };
  for (int e = threadIdx.x; e < W * K; e += PN_NT) {
    if (row_kind) {
      const int c = e / K, k = e - c * K;
      if (g0 + c < n_lines) out[(size_t)(g0 + c) * K + k] = cmul(at(k, c), __ldg(ph + k));
    } else {
      const int k = e / W, c = e - k * W;
      if (g0 + c < S) out[out_base + (size_t)k * S + (size_t)(g0 + c)] = cmul(at(k, c), __ldg(ph + k));
    }
  }
}

struct PolarNufftGeom {
  int K[3];          // oversampled lengths (phi, theta, s)
  float inv_n[3];    // 1 / n_a: the point phase pi u'_a / K_a = pi u_a / n_a
  RealPoly rp[3];    // rho_j(f) per axis, monomials in t = 2 f - 1
};

// Taps of one axis at u' = 2 u: first unwrapped tap k0 + 1 with k0 = floor(u')
// - J/2, offset f = u' - floor(u') (exact in FP32), and for tap j the storage
// index of (k0 + 1 + j) mod K with the sign (-1)^m of its wrap count m, where
// k_u = k_c + m K and k_c is the centred index in [-K/2, K/2).
__device__ __forceinline__ void wrap_first(int ku, int K, int& rr, int& m) {
  const int r = ku + (K >> 1);
  m = r >= 0 ? r / K : -((K - 1 - r) / K);
  rr = r - m * K;  // in [0, K)
}

template <int J>
__device__ __forceinline__ void rho_eval(const RealPoly& P, float f, float (&rho)[J]) {
  const float t = fmaf(2.f, f, -1.f);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float v = P.a[j][kPolyDeg];
#pragma unroll
    for (int q = kPolyDeg - 1; q >= 0; --q) v = fmaf(v, t, P.a[j][q]);
    rho[j] = v;
  }
}

// one axis with J signed weights and storage indices (the phi and theta axes)
template <int J>
__device__ __forceinline__ void axis_taps(float up, int K, const RealPoly& P, float (&w)[J], int (&idx)[J]) {
  const float fl = floorf(up);
  const float f = up - fl;
  float rho[J];
  rho_eval<J>(P, f, rho);
  int rr, m;
  wrap_first((int)fl - J / 2 + 1, K, rr, m);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    int r = rr + j;
    const bool wrapped = r >= K;
    r -= wrapped ? K : 0;
    const bool neg = ((m + (wrapped ? 1 : 0)) & 1) != 0;
    idx[j] = r >= (K >> 1) ? r - (K >> 1) : r + (K >> 1);
    w[j] = neg ? -rho[j] : rho[j];
  }
}

// the contiguous s axis, read as J/2 + 1 aligned pairs of cells: cell i of the
// window (i = 0 .. J + 1) is unwrapped cell c0 + i, c0 = k0 + 1 - e even,
// e = (k0 + 1) & 1, and carries tap i - e (weight 0 outside 0 .. J - 1);
// pidx[q] is the (even) storage index of the pair's first cell
template <int J>
__device__ __forceinline__ void s_axis_pairs(float up, int K, const RealPoly& P, float (&w)[J + 2],
                                             int (&pidx)[J / 2 + 1]) {
  const float fl = floorf(up);
  const float f = up - fl;
  float rho[J];
  rho_eval<J>(P, f, rho);
  const int k1 = (int)fl - J / 2 + 1;  // first tap, unwrapped
  const int e = k1 & 1;
  int rr, m;
  wrap_first(k1 - e, K, rr, m);
#pragma unroll
  for (int i = 0; i < J + 2; ++i) {
    int r = rr + i;
    const bool wrapped = r >= K;
    r -= wrapped ? K : 0;
    const bool neg = ((m + (wrapped ? 1 : 0)) & 1) != 0;
    // tap i - e: rho[i] when e = 0 (i < J), rho[i - 1] when e = 1 (1 <= i <= J)
    float v = 0.f;
    if (i < J) v = e ? 0.f : rho[i];
    if (i >= 1 && i <= J) v = e ? rho[i - 1] : v;
    w[i] = neg ? -v : v;
    if ((i & 1) == 0) pidx[i >> 1] = r >= (K >> 1) ? r - (K >> 1) : r + (K >> 1);
  }
}

// Loads of the spectrum carry an L2 evict-last policy: each of its rows is
// read again by the targets of the next two theta lines and, one phi slice
// later, by the next two phi slices, while the targets and outputs stream
// through once (evict-first loads and stores).
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ float4 ld_keep(const float4* p, unsigned long long pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

// T_sparse: one thread per target; Y holds the phased oversampled spectrum
// Y'[k_phi][k_theta][k_s] (K_phi x K_theta x K_s).
template <int J>
__global__ void __launch_bounds__(PG_NT) k_polar_nufft_gather(const float2* __restrict__ Y, const PolarNufftGeom g,
                                                              const float* __restrict__ targets, long long n,
                                                              float2* __restrict__ out) {
  const long long stride = (long long)gridDim.x * PG_NT;
  const int Kp = g.K[0], Kt = g.K[1], Ks = g.K[2];
  const unsigned long long keep = l2_evict_last_policy();
  for (long long i = (long long)blockIdx.x * PG_NT + threadIdx.x; i < n; i += stride) {
    const float us = __ldcs(targets + 3 * i), ut = __ldcs(targets + 3 * i + 1), up = __ldcs(targets + 3 * i + 2);
    // coordinates must be finite and below 2^22 in magnitude (2 u exact, its
    // integer part and fraction exact in FP32)
    const float lim = 4194304.f;
    if (!(fabsf(us) < lim && fabsf(ut) < lim && fabsf(up) < lim)) {
      __stcs(out + i, make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000)));
      continue;
    }
    float wp[J], wt[J], ws[J + 2];
    int ip[J], it[J], ps[J / 2 + 1];
    axis_taps<J>(2.f * up, Kp, g.rp[0], wp, ip);
    axis_taps<J>(2.f * ut, Kt, g.rp[1], wt, it);
    s_axis_pairs<J>(2.f * us, Ks, g.rp[2], ws, ps);
    // an even first tap leaves the window's last pair without taps
    const bool last_pair = ((__float2int_rd(2.f * us) - J / 2 + 1) & 1) != 0;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < J; ++a) {
#pragma unroll
      for (int b = 0; b < J; ++b) {
        const float4* row = reinterpret_cast<const float4*>(Y + ((size_t)ip[a] * Kt + it[b]) * (size_t)Ks);
        float2 r = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q <= J / 2; ++q) {
          const float4 v = (q < J / 2 || last_pair) ? ld_keep(row + (ps[q] >> 1), keep) : make_float4(0.f, 0.f, 0.f, 0.f);
          r.x = fmaf(ws[2 * q], v.x, r.x);
          r.y = fmaf(ws[2 * q], v.y, r.y);
          r.x = fmaf(ws[2 * q + 1], v.z, r.x);
          r.y = fmaf(ws[2 * q + 1], v.w, r.y);
        }
        const float wab = wp[a] * wt[b];
        acc.x = fmaf(wab, r.x, acc.x);
        acc.y = fmaf(wab, r.y, acc.y);
      }
    }
    // e^{i pi (u_s / n_s + u_theta / n_theta + u_phi / n_phi)}
    float sn, cs;
    sincospif(us * g.inv_n[2] + ut * g.inv_n[1] + up * g.inv_n[0], &sn, &cs);
    __stcs(out + i, make_float2(acc.x * cs - acc.y * sn, acc.x * sn + acc.y * cs));
  }
}

}  // namespace nufft

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
namespace {

using nufft::AxisShape;

#define POLAR_NUFFT_LENGTHS(X) X(10) X(12) X(16) X(20) X(24) X(32) X(40) X(64) X(90) X(128) X(180) X(256) X(360) X(384) X(512)

bool polar_length_supported(int n) {
  switch (n) {
#define CASE_N(V) case V:
    POLAR_NUFFT_LENGTHS(CASE_N)
#undef CASE_N
    return true;
    default:
      return false;
  }
}

template <int N>
cudaError_t launch_axis_t(const float2* in, float2* out, bool row_kind, long long n_lines, long long S, int outer,
                          const float* sq, const float2* twN, const float2* sqr, const float2* twK, const float2* ph,
                          cudaStream_t st) {
  using A = AxisShape<N>;
  auto f = nufft::k_axis_pass<N>;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A::smem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (row_kind) {
    grid = dim3((unsigned)((n_lines + A::W - 1) / A::W), 1, 1);
  } else {
    grid = dim3((unsigned)((S + A::W - 1) / A::W), (unsigned)outer, 1);
  }
  f<<<grid, nufft::PN_NT, A::smem, st>>>(in, out, row_kind ? 1 : 0, n_lines, S, sq, twN, sqr, twK, ph);
  return cudaGetLastError();
}

cudaError_t launch_axis(int N, const float2* in, float2* out, bool row_kind, long long n_lines, long long S,
                        int outer, const float* sq, const float2* twN, const float2* sqr, const float2* twK,
                        const float2* ph, cudaStream_t st) {
  switch (N) {
#define CASE_N(V) \
  case V:         \
    return launch_axis_t<V>(in, out, row_kind, n_lines, S, outer, sq, twN, sqr, twK, ph, st);
    POLAR_NUFFT_LENGTHS(CASE_N)
#undef CASE_N
  }
  return cudaErrorInvalidValue;
}

}  // namespace

struct nufft3d_polar_nufft_s {
  int n[3] = {0, 0, 0};  // (phi, theta, s)
  int K[3] = {0, 0, 0};
  int J = 6;
  int device = 0;
  double fit_err = 0.0;
  float2* Y = nullptr;      // K_phi x K_theta x K_s: the phased oversampled spectrum
  float2* B = nullptr;      // n_phi x K_theta x K_s: after the s and theta passes
  void* tables = nullptr;   // per axis: sq[n], twN[n], sqr[n], twK[K], ph[K]
  const float* sq[3];
  const float2 *twN[3], *sqr[3], *twK[3], *ph[3];
  nufft::PolarNufftGeom geom{};
};

namespace {

// Per-axis FP64 tables: the pre-window with 1/n folded in, on the inverse
// DFT's output index; the twiddles; the axis phase; and the real weights
// rho_j(f) = c_j(f) e^{-i gamma (f + J/2 - j)/2} of the min-max coefficients
// c(f) = T^-1 r(f) (the same construction as the projector's, on N = n, K = 2n),
// fitted as polynomials.  Returns the fit error relative to max |c|, or a
// negative value if rho is not real to rounding.
double axis_tables(int n, int J, std::vector<float>& sq, std::vector<float2>& twN, std::vector<float2>& sqr,
                   std::vector<float2>& twK, std::vector<float2>& ph, nufft::RealPoly& rp) {
  typedef std::complex<double> cd;
  const int K = 2 * n;
  const double alpha = 2.34 * J, gam = 2.0 * M_PI / K;
  const double psi0 = nufft::kb_ft(0.0, J, alpha);
  std::vector<double> s(n);  // centred m = i - n/2
  for (int i = 0; i < n; ++i) s[i] = psi0 / nufft::kb_ft(((double)(i - n / 2) + 0.5) / K, J, alpha);
  sq.resize(n);
  sqr.resize(n);
  for (int q = 0; q < n; ++q) {
    const int m = q < n / 2 ? q : q - n;
    const double v = s[m + n / 2] / n;
    sq[q] = (float)v;
    sqr[q] = make_float2((float)(v * std::cos(-M_PI * m / n)), (float)(v * std::sin(-M_PI * m / n)));
  }
  auto tw = [](int L, std::vector<float2>& out) {
    out.resize(L);
    for (int k = 0; k < L; ++k) {
      const double a = -2.0 * M_PI * k / L;
      out[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  };
  tw(n, twN);
  tw(K, twK);
  ph.resize(K);
  for (int k = 0; k < K; ++k) {
    const int kc = k < K / 2 ? k : k - K;
    ph[k] = make_float2((float)std::cos(-M_PI * kc / K), (float)std::sin(-M_PI * kc / K));
  }
  std::vector<cd> T((size_t)J * J);
  for (int a = 0; a < J; ++a)
    for (int b = 0; b < J; ++b) {
      cd acc = 0;
      for (int i = 0; i < n; ++i) acc += s[i] * s[i] * std::exp(cd(0, gam * (a - b) * (double)(i - n / 2)));
      T[(size_t)a * J + b] = acc;
    }
  if (!nufft::invert(T, J)) return -1.0;
  std::vector<cd> rv(J);
  auto coeffs_at = [&](double f, cd* c) {
    for (int j = 1; j <= J; ++j) {
      cd acc = 0;
      const double dist = f + 0.5 * J - j;
      for (int i = 0; i < n; ++i) acc += s[i] * std::exp(cd(0, -gam * dist * (double)(i - n / 2)));
      rv[j - 1] = acc;
    }
    for (int a = 0; a < J; ++a) {
      cd v = 0;
      for (int b = 0; b < J; ++b) v += T[(size_t)a * J + b] * rv[b];
      c[a] = v;
    }
  };
  double imax = 0.0, cmax = 0.0;
  std::vector<cd> c(J);
  for (int i = 0; i <= 256; ++i) {
    const double f = i / 256.0;
    coeffs_at(f, c.data());
    for (int a = 0; a < J; ++a) {
      const cd rho = c[a] * std::exp(cd(0, -0.5 * gam * (f + 0.5 * J - (a + 1))));
      imax = std::max(imax, std::fabs(rho.imag()));
      cmax = std::max(cmax, std::abs(c[a]));
    }
  }
  if (!(imax <= 1e-9 * cmax)) return -1.0;
  nufft::CoefPoly cp{};
  const double err = nufft::fit_coeff_polys(
      J,
      [&](double f, cd* out) {
        coeffs_at(f, out);
        for (int a = 0; a < J; ++a)
          out[a] = cd((out[a] * std::exp(cd(0, -0.5 * gam * (f + 0.5 * J - (a + 1))))).real(), 0.0);
      },
      cp);
  rp = nufft::RealPoly{};
  for (int a = 0; a < J; ++a)
    for (int q = 0; q <= nufft::kPolyDeg; ++q) rp.a[a][q] = cp.a[a][0][q];
  return err;
}

void free_polar(nufft3d_polar_nufft p) {
  if (!p) return;
  nufft::DeviceGuard g(p->device);
  if (p->Y) cudaFree(p->Y);
  if (p->B) cudaFree(p->B);
  if (p->tables) cudaFree(p->tables);
  delete p;
}

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

}  // namespace

extern "C" {

int nufft3d_polar_nufft_create(nufft3d_polar_nufft* out, int n_phi, int n_theta, int n_s, int J) {
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  if (n_phi < 1 || n_theta < 1 || n_s < 1) return NUFFT3D_ERR_ARG;
  if (J != 4 && J != 6 && J != 8) return NUFFT3D_ERR_UNSUPPORTED;
  if (!polar_length_supported(n_phi) || !polar_length_supported(n_theta) || !polar_length_supported(n_s))
    return NUFFT3D_ERR_UNSUPPORTED;
  nufft3d_polar_nufft p = new (std::nothrow) nufft3d_polar_nufft_s();
  if (!p) return NUFFT3D_ERR_NOMEM;
  p->n[0] = n_phi;
  p->n[1] = n_theta;
  p->n[2] = n_s;
  p->J = J;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return rc_of(e);
  }
  // host tables
  std::vector<float> sq[3];
  std::vector<float2> twN[3], sqr[3], twK[3], ph[3];
  for (int a = 0; a < 3; ++a) {
    p->K[a] = 2 * p->n[a];
    const double err = axis_tables(p->n[a], J, sq[a], twN[a], sqr[a], twK[a], ph[a], p->geom.rp[a]);
    if (!(err >= 0.0 && err <= 1e-7)) {
      delete p;
      return NUFFT3D_ERR_UNSUPPORTED;
    }
    p->fit_err = std::max(p->fit_err, err);
    p->geom.K[a] = p->K[a];
    p->geom.inv_n[a] = (float)(1.0 / p->n[a]);
  }
  // one device block for the tables: per axis sq (padded to 16 bytes), twN, sqr, twK, ph
  size_t bytes = 0;
  size_t off[3][5];
  for (int a = 0; a < 3; ++a) {
    off[a][0] = bytes;
    bytes += ((sizeof(float) * p->n[a] + 15) / 16) * 16;
    off[a][1] = bytes;
    bytes += sizeof(float2) * p->n[a];
    off[a][2] = bytes;
    bytes += sizeof(float2) * p->n[a];
    off[a][3] = bytes;
    bytes += sizeof(float2) * p->K[a];
    off[a][4] = bytes;
    bytes += sizeof(float2) * p->K[a];
  }
  std::vector<unsigned char> host(bytes, 0);
  for (int a = 0; a < 3; ++a) {
    std::memcpy(host.data() + off[a][0], sq[a].data(), sizeof(float) * p->n[a]);
    std::memcpy(host.data() + off[a][1], twN[a].data(), sizeof(float2) * p->n[a]);
    std::memcpy(host.data() + off[a][2], sqr[a].data(), sizeof(float2) * p->n[a]);
    std::memcpy(host.data() + off[a][3], twK[a].data(), sizeof(float2) * p->K[a]);
    std::memcpy(host.data() + off[a][4], ph[a].data(), sizeof(float2) * p->K[a]);
  }
  const size_t nY = (size_t)p->K[0] * p->K[1] * p->K[2];
  const size_t nB = (size_t)p->n[0] * p->K[1] * p->K[2];
  e = cudaMalloc(&p->tables, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(p->tables, host.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->Y, nY * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->B, nB * sizeof(float2));
  if (e != cudaSuccess) {
    free_polar(p);
    return rc_of(e);
  }
  const unsigned char* base = (const unsigned char*)p->tables;
  for (int a = 0; a < 3; ++a) {
    p->sq[a] = (const float*)(base + off[a][0]);
    p->twN[a] = (const float2*)(base + off[a][1]);
    p->sqr[a] = (const float2*)(base + off[a][2]);
    p->twK[a] = (const float2*)(base + off[a][3]);
    p->ph[a] = (const float2*)(base + off[a][4]);
  }
  *out = p;
  return NUFFT3D_OK;
}

int nufft3d_polar_nufft_destroy(nufft3d_polar_nufft p) {
  if (!p) return NUFFT3D_ERR_ARG;
  free_polar(p);
  return NUFFT3D_OK;
}

int nufft3d_polar_nufft_info(nufft3d_polar_nufft p, long long* workspace_bytes, double* fit_error) {
  if (!p) return NUFFT3D_ERR_ARG;
  if (workspace_bytes)
    *workspace_bytes = (long long)(((size_t)p->K[0] * p->K[1] * p->K[2] + (size_t)p->n[0] * p->K[1] * p->K[2]) *
                                   sizeof(float2));
  if (fit_error) *fit_error = p->fit_err;
  return NUFFT3D_OK;
}

int nufft3d_polar_nufft_prepare(nufft3d_polar_nufft p, const void* grid_dev, void* cuda_stream) {
  if (!p || !grid_dev) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard g(p->device);
  if (g.status != cudaSuccess) return rc_of(g.status);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int np = p->n[0], nt = p->n[1], ns = p->n[2];
  const int Kt = p->K[1], Ks = p->K[2];
  float2* A = p->Y;  // the s pass's output lives in Y until the phi pass overwrites it
  // s: x[phi][theta][s] -> A[phi][theta][k_s]
  cudaError_t e = launch_axis(ns, (const float2*)grid_dev, A, true, (long long)np * nt, 1, 1, p->sq[2], p->twN[2],
                              p->sqr[2], p->twK[2], p->ph[2], st);
  // theta: A[phi][theta][k_s] -> B[phi][k_theta][k_s]
  if (e == cudaSuccess)
    e = launch_axis(nt, A, p->B, false, 0, Ks, np, p->sq[1], p->twN[1], p->sqr[1], p->twK[1], p->ph[1], st);
  // phi: B[phi][k_theta][k_s] -> Y[k_phi][k_theta][k_s]
  if (e == cudaSuccess)
    e = launch_axis(np, p->B, p->Y, false, 0, (long long)Kt * Ks, 1, p->sq[0], p->twN[0], p->sqr[0], p->twK[0],
                    p->ph[0], st);
  return rc_of(e);
}

int nufft3d_polar_nufft_gather(nufft3d_polar_nufft p, const float* targets_dev, long long n_targets, void* out_dev,
                               void* cuda_stream) {
  if (!p || n_targets < 0) return NUFFT3D_ERR_ARG;
  if (n_targets == 0) return NUFFT3D_OK;
  if (!targets_dev || !out_dev) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard g(p->device);
  if (g.status != cudaSuccess) return rc_of(g.status);
  // one target per thread: blocks start in target order, so the spectrum rows
  // in use at any time stay within a few phi slices (L2 reuse)
  const long long blocks = (n_targets + nufft::PG_NT - 1) / nufft::PG_NT;
  const long long cap = 1LL << 30;
  const int grid = (int)(blocks < cap ? blocks : cap);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (p->J) {
    case 4:
      nufft::k_polar_nufft_gather<4><<<grid, nufft::PG_NT, 0, st>>>(p->Y, p->geom, targets_dev, n_targets,
                                                                   (float2*)out_dev);
      break;
    case 6:
      nufft::k_polar_nufft_gather<6><<<grid, nufft::PG_NT, 0, st>>>(p->Y, p->geom, targets_dev, n_targets,
                                                                   (float2*)out_dev);
      break;
    default:
      nufft::k_polar_nufft_gather<8><<<grid, nufft::PG_NT, 0, st>>>(p->Y, p->geom, targets_dev, n_targets,
                                                                   (float2*)out_dev);
      break;
  }
  return rc_of(cudaGetLastError());
}

int nufft3d_polar_nufft_resample(nufft3d_polar_nufft p, const void* grid_dev, const float* targets_dev,
                                 long long n_targets, void* out_dev, void* cuda_stream) {
  const int rc = nufft3d_polar_nufft_prepare(p, grid_dev, cuda_stream);
  if (rc != NUFFT3D_OK) return rc;
  return nufft3d_polar_nufft_gather(p, targets_dev, n_targets, out_dev, cuda_stream);
}

}  // extern "C"
