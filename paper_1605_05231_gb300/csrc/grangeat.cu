// Per-view reverse Grangeat step (Sec. 2.2.2, Fig. 2.15; the costs C3a-C3d of
// Sec. 2.4, Eqs. 2.21-2.24): for every cone-beam view v, from its umbrella
// subset y[v][l][t] (L lines at detector-plane angles alpha_l, M samples at
// offsets t - M/2) to its N x N detector image:
//
//   C3a  y' = w_post y                                    (caller's weights)
//   C3b  Y[l][q] = sum_t y'[l][t] e^{-2 pi i (q - M/2)(t - M/2) / M}
//   C3c  z = the 2D min-max NUFFT transpose of Y at omega_lq = 2 pi (q - M/2)/M
//        (cos alpha_l, sin alpha_l): spread with conj(c_y c_x) onto K x K
//        (K = 2N, J x J taps), unnormalised inverse 2D DFT, crop to the centred
//        N x N box, Kaiser-Bessel pre-window s(n_y) s(n_x)
//   C3d  out = w_pre z                                    (caller's weights)
//
// GB300 design.  Every view shares the sampling pattern, so the spread is one
// fixed sparse matrix S (K^2 x LM, J^2 nonzeros per column) applied to all
// views at once: the plan stores S by rows (cells) and the spread kernel is a
// gather over each cell's (point, weight) list with the views as the
// contiguous fastest axis, so there are no atomics and every spectrum value is
// read as part of a coalesced row of views.  The line DFTs write the spectra
// in that [point][view] layout through a shared-memory transpose, the first
// inverse FFT pass works on [k_y][k_x][view] columns, and the last pass crops,
// weights and writes each view's image rows contiguously.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "fft.cuh"
#include "host_math.h"
#include "internal.h"

namespace nufft {

constexpr int GV_W = 16;    // views per CTA of the line and FFT kernels (128-byte segments)
constexpr int GV_P = GV_W + 1;
constexpr int GV_NT = 256;
constexpr int GV_CHUNK = 8;  // loads a thread issues before its shared stores
constexpr int GS_WARPS = 8;  // warps per spread CTA
constexpr int GS_VPL = 4;    // views per lane per pass of the spread (64 registers, four CTAs per SM)

// acc + a b (complex)
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}

template <int L>
constexpr size_t gv_smem() {
  return (size_t)L * GV_P * sizeof(float2);
}

// C3a + C3b for one line l and GV_W views: the centred DFT as
// Y[q] = (-1)^{q + M/2} sum_t (-1)^t y'[t] e^{-2 pi i q t / M} (M even)
template <int M>
__global__ void __launch_bounds__(GV_NT) k_view_lines(const float2* __restrict__ y, const float* __restrict__ w_post,
                                                      int L, int Vc, float2* __restrict__ Yhat,
                                                      const float2* __restrict__ twM) {
  extern __shared__ float2 buf[];
  const int l = blockIdx.x;
  const int vb = blockIdx.y * GV_W;
  // a thread's GV_CHUNK loads are in flight together before its shared stores
  for (int base = threadIdx.x; base < GV_W * M; base += GV_CHUNK * GV_NT) {
    float2 yv[GV_CHUNK];
    float wv[GV_CHUNK];
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      const int c = e / M, t = e - c * M;
      yv[u] = make_float2(0.f, 0.f);
      wv[u] = 0.f;
      if (e < GV_W * M && vb + c < Vc) {
        const size_t i = ((size_t)(vb + c) * L + l) * M + t;
        yv[u] = __ldg(y + i);
        wv[u] = __ldg(w_post + i);
      }
    }
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      if (e < GV_W * M) {
        const int c = e / M, t = e - c * M;
        buf[t * GV_P + c] = cscale(yv[u], (t & 1) ? -wv[u] : wv[u]);
      }
    }
  }
  __syncthreads();
  smem_fft<M, GV_W, GV_NT, false>(buf, GV_P, twM);
  for (int e = threadIdx.x; e < GV_W * M; e += GV_NT) {
    const int q = e / GV_W, c = e - q * GV_W;
    const int v = vb + c;
    if (v < Vc) {
      const float sg = ((q + M / 2) & 1) ? -1.f : 1.f;
      Yhat[((size_t)l * M + q) * Vc + v] = cscale(buf[q * GV_P + c], sg);
    }
  }
}

// C3c's spread as a gather over the cells' rows of S: G[c][v] = sum_e w_e
// Yhat[col_e][v]; lanes over views.  A row is cut into work items of at most
// 32 entries (the cells near the origin, where all lines cross, hold up to
// L (J/2 + 1) J entries): a warp takes one item, reads its entries in one
// coalesced load and hands them out by shuffles, so the spectrum loads of
// consecutive entries are in flight together.  A cell of one item stores its
// sums; the items of a longer row add theirs to the zeroed grid atomically.
__global__ void __launch_bounds__(GS_WARPS * 32, 4) k_view_spread(const int4* __restrict__ items, int n_items,
                                                               const int* __restrict__ col,
                                                               const float2* __restrict__ wt,
                                                               const float2* __restrict__ Yhat, int Vc,
                                                               float2* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * GS_WARPS + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * GS_WARPS;
  for (int it = warp; it < n_items; it += n_warps) {
    const int4 item = __ldg(items + it);  // (cell, first entry, entries, shared row)
    const int c = item.x, n = item.z;
    int my_p = 0;
    float2 my_w = make_float2(0.f, 0.f);
    if (lane < n) {
      my_p = __ldg(col + item.y + lane);
      my_w = __ldg(wt + item.y + lane);
    }
    for (int v0 = 0; v0 < Vc; v0 += 32 * GS_VPL) {
      float2 acc[GS_VPL];
#pragma unroll
      for (int k = 0; k < GS_VPL; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const int p = __shfl_sync(0xffffffffu, my_p, j);
        const float2 w = make_float2(__shfl_sync(0xffffffffu, my_w.x, j), __shfl_sync(0xffffffffu, my_w.y, j));
        const float2* row = Yhat + (size_t)p * Vc;
#pragma unroll
        for (int k = 0; k < GS_VPL; ++k) {
          const int v = v0 + lane + 32 * k;
          if (v < Vc) acc[k] = cfma(w, __ldg(row + v), acc[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < GS_VPL; ++k) {
        const int v = v0 + lane + 32 * k;
        if (v < Vc) {
          float2* dst = G + (size_t)c * Vc + v;
          if (item.w) {
            atomicAdd(&dst->x, acc[k].x);
            atomicAdd(&dst->y, acc[k].y);
          } else {
            *dst = acc[k];
          }
        }
      }
    }
  }
}

// C3c's inverse DFT along k_y, cropped: G[k_y][S] -> H[r][S], r = 0 .. N-1 the
// centred row n_y = r - N/2 (k_y = n_y mod K); S = K Vc columns (k_x, v)
template <int K>
__global__ void __launch_bounds__(GV_NT) k_view_ifft_y(const float2* __restrict__ G, long long S, int N,
                                                       float2* __restrict__ H, const float2* __restrict__ twK) {
  extern __shared__ float2 buf[];
  const long long g0 = (long long)blockIdx.x * GV_W;
  for (int base = threadIdx.x; base < GV_W * K; base += GV_CHUNK * GV_NT) {
    float2 t[GV_CHUNK];
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      const int i = e / GV_W, c = e - i * GV_W;
      t[u] = (e < GV_W * K && g0 + c < S) ? __ldg(G + (size_t)i * S + (size_t)(g0 + c)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      if (e < GV_W * K) buf[(e / GV_W) * GV_P + (e % GV_W)] = t[u];
    }
  }
  __syncthreads();
  smem_fft<K, GV_W, GV_NT, true>(buf, GV_P, twK);
  for (int e = threadIdx.x; e < GV_W * N; e += GV_NT) {
    const int r = e / GV_W, c = e - r * GV_W;
    int k = r - N / 2;
    k += k < 0 ? K : 0;
    if (g0 + c < S) H[(size_t)r * S + (size_t)(g0 + c)] = buf[k * GV_P + c];
  }
}

// C3c's inverse DFT along k_x, cropped, pre-window, and C3d: H[r][k_x][v] ->
// out[v][r][x] = w_pre[v][r][x] s(r) s(x) (inverse DFT at n_x = x - N/2)
template <int K>
__global__ void __launch_bounds__(GV_NT) k_view_ifft_x(const float2* __restrict__ H, int Vc, int N,
                                                       const float* __restrict__ s, const float* __restrict__ w_pre,
                                                       float2* __restrict__ out, const float2* __restrict__ twK) {
  extern __shared__ float2 buf[];
  const int vb = blockIdx.x * GV_W;
  const int r = blockIdx.y;
  for (int base = threadIdx.x; base < GV_W * K; base += GV_CHUNK * GV_NT) {
    float2 t[GV_CHUNK];
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      const int i = e / GV_W, c = e - i * GV_W;
      t[u] = (e < GV_W * K && vb + c < Vc) ? __ldg(H + ((size_t)r * K + i) * Vc + vb + c) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < GV_CHUNK; ++u) {
      const int e = base + u * GV_NT;
      if (e < GV_W * K) buf[(e / GV_W) * GV_P + (e % GV_W)] = t[u];
    }
  }
  __syncthreads();
  smem_fft<K, GV_W, GV_NT, true>(buf, GV_P, twK);
  const float sr = __ldg(s + r);
  for (int e = threadIdx.x; e < GV_W * N; e += GV_NT) {
    const int c = e / N, x = e - c * N;
    const int v = vb + c;
    if (v < Vc) {
      int k = x - N / 2;
      k += k < 0 ? K : 0;
      const size_t o = ((size_t)v * N + r) * N + x;
      out[o] = cscale(buf[k * GV_P + c], sr * __ldg(s + x) * __ldg(w_pre + o));
    }
  }
}

}  // namespace nufft

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
namespace {

#define GRANGEAT_LINE_LENGTHS(X) X(16) X(32) X(64) X(128) X(256) X(512)
#define GRANGEAT_GRID_LENGTHS(X) X(32) X(64) X(128) X(256) X(512)

bool line_length_ok(int M) {
  switch (M) {
#define CASE_N(V) case V:
    GRANGEAT_LINE_LENGTHS(CASE_N)
#undef CASE_N
    return true;
    default:
      return false;
  }
}

bool grid_length_ok(int K) {
  switch (K) {
#define CASE_N(V) case V:
    GRANGEAT_GRID_LENGTHS(CASE_N)
#undef CASE_N
    return true;
    default:
      return false;
  }
}

template <class F>
cudaError_t set_smem_attr(F* f, size_t bytes) {
  return cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int M>
cudaError_t launch_lines_t(const float2* y, const float* w_post, int L, int Vc, float2* Yhat, const float2* twM,
                           cudaStream_t st) {
  auto f = nufft::k_view_lines<M>;
  cudaError_t e = set_smem_attr(f, nufft::gv_smem<M>());
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)L, (unsigned)((Vc + nufft::GV_W - 1) / nufft::GV_W));
  f<<<grid, nufft::GV_NT, nufft::gv_smem<M>(), st>>>(y, w_post, L, Vc, Yhat, twM);
  return cudaGetLastError();
}

cudaError_t launch_lines(int M, const float2* y, const float* w_post, int L, int Vc, float2* Yhat, const float2* twM,
                         cudaStream_t st) {
  switch (M) {
#define CASE_N(V) \
  case V:         \
    return launch_lines_t<V>(y, w_post, L, Vc, Yhat, twM, st);
    GRANGEAT_LINE_LENGTHS(CASE_N)
#undef CASE_N
  }
  return cudaErrorInvalidValue;
}

template <int K>
cudaError_t launch_ifft_t(const float2* G, float2* H, int N, int Vc, const float* s, const float* w_pre, float2* out,
                          const float2* twK, cudaStream_t st) {
  auto fy = nufft::k_view_ifft_y<K>;
  auto fx = nufft::k_view_ifft_x<K>;
  cudaError_t e = set_smem_attr(fy, nufft::gv_smem<K>());
  if (e == cudaSuccess) e = set_smem_attr(fx, nufft::gv_smem<K>());
  if (e != cudaSuccess) return e;
  const long long S = (long long)K * Vc;
  fy<<<(unsigned)((S + nufft::GV_W - 1) / nufft::GV_W), nufft::GV_NT, nufft::gv_smem<K>(), st>>>(G, S, N, H, twK);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((Vc + nufft::GV_W - 1) / nufft::GV_W), (unsigned)N);
  fx<<<grid, nufft::GV_NT, nufft::gv_smem<K>(), st>>>(H, Vc, N, s, w_pre, out, twK);
  return cudaGetLastError();
}

cudaError_t launch_ifft(int K, const float2* G, float2* H, int N, int Vc, const float* s, const float* w_pre,
                        float2* out, const float2* twK, cudaStream_t st) {
  switch (K) {
#define CASE_N(V) \
  case V:         \
    return launch_ifft_t<V>(G, H, N, Vc, s, w_pre, out, twK, st);
    GRANGEAT_GRID_LENGTHS(CASE_N)
#undef CASE_N
  }
  return cudaErrorInvalidValue;
}

int rc_from(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

}  // namespace

struct nufft3d_grangeat_s {
  int N = 0, K = 0, L = 0, M = 0, J = 0, Vmax = 0, device = 0;
  long long nnz = 0;
  double fit_err = 0.0;
  int4* items = nullptr;    // spread work items (cell, first entry, entries, shared row)
  int n_items = 0;
  bool any_shared = false;  // a row split into several items: the grid is zeroed first
  int* col = nullptr;       // [nnz] point index l M + q
  float2* wt = nullptr;     // [nnz] conj(c_y c_x)
  float2* Yhat = nullptr;   // [L M][Vmax]
  float2* G = nullptr;      // [K][K][Vmax]
  float2* H = nullptr;      // [N][K][Vmax]
  float* s = nullptr;       // [N]
  float2* twM = nullptr;    // [M]
  float2* twK = nullptr;    // [K]
};

namespace {

void free_grangeat(nufft3d_grangeat g) {
  if (!g) return;
  nufft::DeviceGuard dg(g->device);
  for (void* p : {(void*)g->items, (void*)g->col, (void*)g->wt, (void*)g->Yhat, (void*)g->G, (void*)g->H,
                  (void*)g->s, (void*)g->twM, (void*)g->twK})
    if (p) cudaFree(p);
  delete g;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

extern "C" {

int nufft3d_grangeat_create(nufft3d_grangeat* out, int N, int L, int M, int J, const double* angles, int max_views) {
  typedef std::complex<double> cd;
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  if (N < 2 || L < 1 || L > 65535 || M < 2 || J < 2 || J > 8 || max_views < 1 || !angles) return NUFFT3D_ERR_ARG;
  for (int l = 0; l < L; ++l)
    if (!std::isfinite(angles[l])) return NUFFT3D_ERR_ARG;
  const int K = 2 * N;
  if ((N & 1) || !grid_length_ok(K) || !line_length_ok(M)) return NUFFT3D_ERR_UNSUPPORTED;
  const long long P = (long long)L * M;
  const long long nnz = P * J * J;
  if (nnz >= (1LL << 31)) return NUFFT3D_ERR_UNSUPPORTED;
  nufft3d_grangeat g = new (std::nothrow) nufft3d_grangeat_s();
  if (!g) return NUFFT3D_ERR_NOMEM;
  g->N = N;
  g->K = K;
  g->L = L;
  g->M = M;
  g->J = J;
  g->Vmax = max_views;
  g->nnz = nnz;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    delete g;
    return rc_from(e);
  }
  // FP64 pre-window and min-max coefficients of one axis (N, K = 2N, J), the
  // same construction as the projector's: s(n) = Psi(0)/Psi((n + 1/2)/K),
  // c(f) = T^-1 r(f), fitted as polynomials in t = 2 f - 1
  const double alpha = 2.34 * J, gam = 2.0 * M_PI / K;
  const double psi0 = nufft::kb_ft(0.0, J, alpha);
  std::vector<double> sd(N);
  for (int i = 0; i < N; ++i) sd[i] = psi0 / nufft::kb_ft(((double)(i - N / 2) + 0.5) / K, J, alpha);
  std::vector<cd> T((size_t)J * J);
  for (int a = 0; a < J; ++a)
    for (int b = 0; b < J; ++b) {
      cd acc = 0;
      for (int i = 0; i < N; ++i) acc += sd[i] * sd[i] * std::exp(cd(0, gam * (a - b) * (double)(i - N / 2)));
      T[(size_t)a * J + b] = acc;
    }
  if (!nufft::invert(T, J)) {
    delete g;
    return NUFFT3D_ERR_UNSUPPORTED;
  }
  std::vector<cd> rv(J);
  auto coeffs_at = [&](double f, cd* c) {
    for (int j = 1; j <= J; ++j) {
      cd acc = 0;
      const double dist = f + 0.5 * J - j;
      for (int i = 0; i < N; ++i) acc += sd[i] * std::exp(cd(0, -gam * dist * (double)(i - N / 2)));
      rv[j - 1] = acc;
    }
    for (int a = 0; a < J; ++a) {
      cd v = 0;
      for (int b = 0; b < J; ++b) v += T[(size_t)a * J + b] * rv[b];
      c[a] = v;
    }
  };
  nufft::CoefPoly cp{};
  g->fit_err = nufft::fit_coeff_polys(J, coeffs_at, cp);
  if (!(g->fit_err <= 1e-7)) {
    delete g;
    return NUFFT3D_ERR_UNSUPPORTED;
  }
  auto eval = [&](double f, cd* c) {
    const double t = 2.0 * f - 1.0;
    for (int j = 0; j < J; ++j) {
      double re = cp.a[j][0][nufft::kPolyDeg], im = cp.a[j][1][nufft::kPolyDeg];
      for (int q = nufft::kPolyDeg - 1; q >= 0; --q) {
        re = re * t + cp.a[j][0][q];
        im = im * t + cp.a[j][1][q];
      }
      c[j] = cd(re, im);
    }
  };
  // the sparse matrix S by cells: point p = l M + q at u = K (q - M/2)/M
  // (cos alpha_l, sin alpha_l), taps k0 + 1 .. k0 + J, k0 = floor(u - J/2)
  std::vector<int> cell((size_t)nnz);
  std::vector<float2> w((size_t)nnz);
  std::vector<int> count((size_t)K * K + 1, 0);
  std::vector<cd> cx(J), cy(J);
  for (int l = 0; l < L; ++l) {
    const double ca = std::cos(angles[l]), sa = std::sin(angles[l]);
    for (int q = 0; q < M; ++q) {
      const double rho = (double)(q - M / 2) / M;  // cycles per detector pixel
      const double ux = ca * rho * K - 0.5 * J, uy = sa * rho * K - 0.5 * J;
      const double kx0 = std::floor(ux), ky0 = std::floor(uy);
      eval(ux - kx0, cx.data());
      eval(uy - ky0, cy.data());
      const long long p = (long long)l * M + q;
      for (int jy = 0; jy < J; ++jy) {
        long long iy = ((long long)ky0 + 1 + jy) % K;
        iy += iy < 0 ? K : 0;
        for (int jx = 0; jx < J; ++jx) {
          long long ix = ((long long)kx0 + 1 + jx) % K;
          ix += ix < 0 ? K : 0;
          const size_t e_ = (size_t)p * J * J + (size_t)jy * J + jx;
          cell[e_] = (int)(iy * K + ix);
          const cd wv = std::conj(cy[jy] * cx[jx]);
          w[e_] = make_float2((float)wv.real(), (float)wv.imag());
          ++count[(size_t)cell[e_] + 1];
        }
      }
    }
  }
  std::vector<int> row_ptr((size_t)K * K + 1, 0);
  for (size_t c = 0; c < (size_t)K * K; ++c) row_ptr[c + 1] = row_ptr[c] + count[c + 1];
  std::vector<int> fill(row_ptr.begin(), row_ptr.end() - 1);
  std::vector<int> col((size_t)nnz);
  std::vector<float2> wt((size_t)nnz);
  for (size_t e_ = 0; e_ < (size_t)nnz; ++e_) {
    const int d = fill[(size_t)cell[e_]]++;
    col[(size_t)d] = (int)(e_ / ((size_t)J * J));
    wt[(size_t)d] = w[e_];
  }
  std::vector<float> sf(N);
  for (int i = 0; i < N; ++i) sf[i] = (float)sd[i];
  auto tw = [](int Lt) {
    std::vector<float2> o(Lt);
    for (int k = 0; k < Lt; ++k) {
      const double a = -2.0 * M_PI * k / Lt;
      o[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return o;
  };
  // work items of at most 32 entries; every cell gets one (empty rows store zeros)
  std::vector<int4> items;
  for (int c = 0; c < K * K; ++c) {
    const int b0 = row_ptr[(size_t)c], b1 = row_ptr[(size_t)c + 1];
    const int shared = b1 - b0 > 32 ? 1 : 0;
    g->any_shared = g->any_shared || shared;
    int b = b0;
    do {
      const int n = std::min(32, b1 - b);
      items.push_back(make_int4(c, b, n, shared));
      b += n;
    } while (b < b1);
  }
  g->n_items = (int)items.size();
  e = upload(&g->items, items);
  if (e == cudaSuccess) e = upload(&g->col, col);
  if (e == cudaSuccess) e = upload(&g->wt, wt);
  if (e == cudaSuccess) e = upload(&g->s, sf);
  if (e == cudaSuccess) e = upload(&g->twM, tw(M));
  if (e == cudaSuccess) e = upload(&g->twK, tw(K));
  const size_t V = (size_t)max_views;
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->Yhat, (size_t)P * V * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->G, (size_t)K * K * V * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->H, (size_t)N * K * V * sizeof(float2));
  if (e != cudaSuccess) {
    free_grangeat(g);
    return rc_from(e);
  }
  *out = g;
  return NUFFT3D_OK;
}

int nufft3d_grangeat_info(nufft3d_grangeat g, long long* workspace_bytes, long long* nnz, double* fit_error) {
  if (!g) return NUFFT3D_ERR_ARG;
  const size_t V = (size_t)g->Vmax;
  if (workspace_bytes)
    *workspace_bytes = (long long)(((size_t)g->L * g->M + (size_t)g->K * g->K + (size_t)g->N * g->K) * V *
                                       sizeof(float2) +
                                   (size_t)g->nnz * (sizeof(int) + sizeof(float2)) +
                                   (size_t)g->n_items * sizeof(int4));
  if (nnz) *nnz = g->nnz;
  if (fit_error) *fit_error = g->fit_err;
  return NUFFT3D_OK;
}

int nufft3d_grangeat_run(nufft3d_grangeat g, const void* y_dev, const float* w_post_dev, const float* w_pre_dev,
                         int n_views, void* out_dev, void* cuda_stream) {
  if (!g || n_views < 0) return NUFFT3D_ERR_ARG;
  if (n_views == 0) return NUFFT3D_OK;
  if (!y_dev || !w_post_dev || !w_pre_dev || !out_dev) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard dg(g->device);
  if (dg.status != cudaSuccess) return rc_from(dg.status);
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e != cudaSuccess) return rc_from(e);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t LM = (size_t)g->L * g->M, NN = (size_t)g->N * g->N;
  const int n_cells = g->K * g->K;
  const int sp_blocks = std::min((g->n_items + nufft::GS_WARPS - 1) / nufft::GS_WARPS, sms * 16);
  for (int v0 = 0; v0 < n_views && e == cudaSuccess; v0 += g->Vmax) {
    const int Vc = std::min(g->Vmax, n_views - v0);
    e = launch_lines(g->M, (const float2*)y_dev + (size_t)v0 * LM, w_post_dev + (size_t)v0 * LM, g->L, Vc, g->Yhat,
                     g->twM, st);
    if (e != cudaSuccess) break;
    if (g->any_shared) e = cudaMemsetAsync(g->G, 0, (size_t)n_cells * Vc * sizeof(float2), st);
    if (e != cudaSuccess) break;
    nufft::k_view_spread<<<sp_blocks, nufft::GS_WARPS * 32, 0, st>>>(g->items, g->n_items, g->col, g->wt, g->Yhat,
                                                                     Vc, g->G);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    e = launch_ifft(g->K, g->G, g->H, g->N, Vc, g->s, w_pre_dev + (size_t)v0 * NN, (float2*)out_dev + (size_t)v0 * NN,
                    g->twK, st);
  }
  return rc_from(e);
}

int nufft3d_grangeat_destroy(nufft3d_grangeat g) {
  if (!g) return NUFFT3D_ERR_ARG;
  free_grangeat(g);
  return NUFFT3D_OK;
}

}  // extern "C"
