// FFT passes of the projector: the pruned 3D FFT (x, y, z passes) with the
// deapodisation and zero padding fused into the first pass (P and F of
// Eq. 2.11), the pruned inverse passes with cropping and deapodisation fused
// into the last (their transposes), and the centred per-line DFTs that turn
// Fourier samples on a radial line into plane integrals (Fourier Slice
// Theorem, Sec. 2.2.1).  All are HBM-bound: each pass reads and writes its
// array once; the butterflies run in shared memory.
#include "fft.cuh"
#include "internal.h"

namespace nufft {

constexpr int FFT_W = 16;    // columns (rows) per CTA: 16 complex64 = 128 B segments
constexpr int FFT_NT = 256;  // threads per CTA
constexpr int FFT_PITCH = FFT_W + 1;
// row passes (x) and line DFTs: 8 rows per CTA (pitch 9: the Stockham writes
// stay conflict-free), 37 KB of shared memory at L = 512, four CTAs per SM;
// a thread's loads of a CTA's rows are issued in one batch of ROW_CHUNK
constexpr int ROW_W = 8;
constexpr int ROW_PITCH = ROW_W + 1;
constexpr int ROW_MIN_CTAS = 4;
constexpr int ROW_CHUNK = 16;

__device__ __forceinline__ int centred_to_grid(int i, int half, int L) {
  int k = i - half;
  return k < 0 ? k + L : k;
}

// ----------------------------------------------------------------------------
// forward x pass: volume rows (z, y) -> deapodised, zero-padded, FFT along x.
// out[(z N + y) K + kx]
// ----------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(FFT_NT, ROW_MIN_CTAS) k_row_fwd(const void* __restrict__ vol, int cplx,
                                                    float2* __restrict__ out, const float* __restrict__ s,
                                                    int N, const float2* __restrict__ tw) {
  extern __shared__ float2 buf[];
  const int nrows = N * N;
  const int row0 = blockIdx.x * ROW_W;
  const int half = N / 2;
  // loads of a chunk are issued before its shared stores (batched in flight)
  for (int base = threadIdx.x; base < ROW_W * N; base += ROW_CHUNK * FFT_NT) {
    float2 t[ROW_CHUNK];
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      t[u] = make_float2(0.f, 0.f);
      if (idx < ROW_W * N) {
        const int c = idx / N, x = idx - c * N;
        const int r = row0 + c;
        if (r < nrows) {
          if (cplx) t[u] = ((const float2*)vol)[(size_t)r * N + x];
          else t[u] = make_float2(((const float*)vol)[(size_t)r * N + x], 0.f);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      if (idx < ROW_W * N) {
        const int c = idx / N, x = idx - c * N;
        const int r = row0 + c;
        const int z = r / N, y = r - z * N;
        const float sc = r < nrows ? __ldg(s + x) * __ldg(s + y) * __ldg(s + z) : 0.f;
        buf[centred_to_grid(x, half, K) * ROW_PITCH + c] = cscale(t[u], sc);
      }
    }
  }
  for (int idx = threadIdx.x; idx < ROW_W * (K - N); idx += FFT_NT) {
    const int c = idx % ROW_W, i = idx / ROW_W + (N - half);
    buf[i * ROW_PITCH + c] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  smem_fft<K, ROW_W, FFT_NT, false>(buf, ROW_PITCH, tw);
  for (int idx = threadIdx.x; idx < ROW_W * K; idx += FFT_NT) {
    const int c = idx / K, k = idx - c * K;
    const int r = row0 + c;
    if (r < nrows) out[(size_t)r * K + k] = buf[k * ROW_PITCH + c];
  }
}

// ----------------------------------------------------------------------------
// forward x pass of a real volume: two real rows per complex transform.  Rows
// a = row0 + 2c and b = a + 1 go in as Z = a + i b; with Z~[k] = conj(Z[-k]),
// the transforms are A = (Z + Z~) / 2 and B = (Z - Z~) / (2i), so one
// transform of 8 columns serves 16 rows.
// ----------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(FFT_NT, ROW_MIN_CTAS) k_row_fwd_real(const float* __restrict__ vol,
                                                         float2* __restrict__ out, const float* __restrict__ s,
                                                         int N, const float2* __restrict__ tw) {
  extern __shared__ float2 buf[];
  const int nrows = N * N;
  const int row0 = blockIdx.x * (2 * ROW_W);
  const int half = N / 2;
  for (int base = threadIdx.x; base < ROW_W * N; base += ROW_CHUNK * FFT_NT) {
    float2 t[ROW_CHUNK];
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      t[u] = make_float2(0.f, 0.f);
      if (idx < ROW_W * N) {
        const int c = idx / N, x = idx - c * N;
        const int ra = row0 + 2 * c;
        if (ra < nrows) t[u].x = vol[(size_t)ra * N + x];
        if (ra + 1 < nrows) t[u].y = vol[(size_t)(ra + 1) * N + x];
      }
    }
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      if (idx < ROW_W * N) {
        const int c = idx / N, x = idx - c * N;
        const int ra = row0 + 2 * c, rb = ra + 1;
        const int za = ra / N, ya = ra - za * N, zb = rb / N, yb = rb - zb * N;
        const float sx = __ldg(s + x);
        const float sa = ra < nrows ? sx * __ldg(s + ya) * __ldg(s + za) : 0.f;
        const float sb = rb < nrows ? sx * __ldg(s + yb) * __ldg(s + zb) : 0.f;
        buf[centred_to_grid(x, half, K) * ROW_PITCH + c] = make_float2(t[u].x * sa, t[u].y * sb);
      }
    }
  }
  for (int idx = threadIdx.x; idx < ROW_W * (K - N); idx += FFT_NT) {
    const int c = idx % ROW_W, i = idx / ROW_W + (N - half);
    buf[i * ROW_PITCH + c] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  smem_fft<K, ROW_W, FFT_NT, false>(buf, ROW_PITCH, tw);
  for (int idx = threadIdx.x; idx < ROW_W * K; idx += FFT_NT) {
    const int c = idx / K, k = idx - c * K;
    const int ra = row0 + 2 * c;
    const float2 z = buf[k * ROW_PITCH + c];
    const float2 zm = buf[(k == 0 ? 0 : K - k) * ROW_PITCH + c];
    if (ra < nrows) out[(size_t)ra * K + k] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    if (ra + 1 < nrows) out[(size_t)(ra + 1) * K + k] = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
  }
}

// ----------------------------------------------------------------------------
// column pass: for each outer index o and chunk of W contiguous columns
// (32 W threads; W = 16: 128-byte row segments, two CTAs per SM),
// transform along a strided axis.
//   PAD_IN : input has N entries (centred), zero-padded to L (forward passes)
//   CROP_OUT: only the N centred outputs are written (inverse passes)
// element (i, c) of the input at in[o in_outer + i in_stride + ch W + c]
// ----------------------------------------------------------------------------
// e^{-i pi r / R} for the radices of the transforms (compile-time r and R)
template <int R>
__device__ __forceinline__ float2 conj_unit_rot(int r) {
  constexpr float c8 = 0.92387953251128674f, s8 = 0.38268343236508977f, h = 0.70710678118654752f,
                  t = 0.86602540378443865f;
  if (R == 2) return r == 0 ? make_float2(1.f, 0.f) : make_float2(0.f, -1.f);
  if (R == 3) return r == 0 ? make_float2(1.f, 0.f) : r == 1 ? make_float2(0.5f, -t) : make_float2(-0.5f, -t);
  if (R == 4) {
    switch (r) {
      case 0: return make_float2(1.f, 0.f);
      case 1: return make_float2(h, -h);
      case 2: return make_float2(0.f, -1.f);
      default: return make_float2(-h, -h);
    }
  }
  switch (r) {  // R == 8
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c8, -s8);
    case 2: return make_float2(h, -h);
    case 3: return make_float2(s8, -c8);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-s8, -c8);
    case 6: return make_float2(-h, -h);
    default: return make_float2(-c8, -s8);
  }
}

// The phase hook of the real-weight z passes: rows j + r L/R of a butterfly
// carry e^{-i gamma k_c/2} = e^{-i gamma j/2} e^{-i pi r/R} (negated for k >= L/2,
// where k_c = k - L); applied, times the thread's column factor, to the
// outputs of the forward pass's last stage and (conjugated) to the inputs of
// the inverse pass's first stage.
template <int L, bool INV, bool PHASE>
struct PhaseHook {
  const float2* ph;
  float2 col;
  template <int R>
  __device__ __forceinline__ void apply(float2 (&v)[R], int j) const {
    const float2 f = cmul(__ldg(ph + j), col);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 t = cmul(f, conj_unit_rot<R>(r));
      if (j + r * (L / R) >= L / 2) t = make_float2(-t.x, -t.y);
      v[r] = INV ? cmulc(v[r], t) : cmul(v[r], t);
    }
  }
  template <int R>
  __device__ __forceinline__ void first(float2 (&v)[R], int j, int) const {
    if constexpr (PHASE && INV) apply<R>(v, j);
  }
  template <int R>
  __device__ __forceinline__ void last(float2 (&v)[R], int j, int) const {
    if constexpr (PHASE && !INV) apply<R>(v, j);
  }
};

template <int L, bool INV, bool PAD_IN, bool CROP_OUT, typename OutT, int W, bool PHASE = false>
__global__ void __launch_bounds__(32 * W, 32 / W) k_col(const float2* __restrict__ in, OutT* __restrict__ out,
                                                int N, int n_chunks, long long in_outer, long long in_stride,
                                                long long out_outer, long long out_stride,
                                                const float2* __restrict__ tw, const float* __restrict__ bound,
                                                ColPrune pr) {
  extern __shared__ float2 buf[];
  const float out_scale = bound ? lp_scale_from_bound(*bound) : 1.f;
  const int ch = blockIdx.x % n_chunks;
  const long long o = blockIdx.x / n_chunks;
  const float2* ib = in + o * in_outer + (long long)ch * W;
  OutT* ob = out + o * out_outer + (long long)ch * W;
  const int half = N / 2;
  // pruning to the ball of cells the interpolation touches: the column's grid
  // frequency kx = ch W + c, and for z passes ky = o (centred)
  const int hk = pr.K / 2;
  auto cen = [&](int k) -> int { return k < hk ? k : k - pr.K; };
  const int cy2 = pr.mode == 2 ? cen((int)o) * cen((int)o) : 0;
  int mcx2 = 0;  // smallest kx^2 over the CTA's columns
  if (pr.mode != 0) {
    // columns k_lo .. k_hi: centred kx = k below K/2 (smallest square at k_lo >= 0)
    // and k - K from K/2 on (smallest at k_hi)
    const int k_lo = ch * W, k_hi = ch * W + W - 1;
    mcx2 = 0x7fffffff;
    if (k_lo < hk) mcx2 = k_lo * k_lo;
    if (k_hi >= hk) {
      const int e = k_hi - pr.K;
      mcx2 = e * e < mcx2 ? e * e : mcx2;
    }
    // a z pass whose columns all lie outside the disk kx^2 + ky^2 <= r2 has nothing to do
    if (pr.mode == 2 && (long long)mcx2 + cy2 > pr.r2) return;
  }
  // exact test of cell (k, column c): inverse passes read only cells inside the
  // ball (the adjoint clears nothing outside it)
  auto live = [&](int k, int c) -> bool {
    if (pr.mode == 0) return true;
    const int cx = cen(ch * W + c), ck = cen(k);
    return (long long)cx * cx + cy2 + (long long)ck * ck <= pr.r2;
  };
  // row test shared by the CTA's columns: forward passes write whole 128-byte
  // rows whenever one of the 16 columns needs the row (no partial lines)
  auto row_live = [&](int k) -> bool {
    if (pr.mode == 0) return true;
    const int ck = cen(k);
    return (long long)mcx2 + cy2 + (long long)ck * ck <= pr.r2;
  };
  auto col_live = [&](int c) -> bool {
    if (pr.mode != 2) return true;
    const int cx = cen(ch * W + c);
    return (long long)cx * cx + cy2 <= pr.r2;
  };
  // z passes of the real-weight kernels: the cell (kz = k, ky = o, kx = ch W + c)
  // carries e^{-i gamma (kx + ky + kz)/2} (centred k).  A thread always serves
  // column c = threadIdx.x % W, so its (ky, kx) factor is fixed; the kz factor
  // of rows j + r L/R (a butterfly's rows in the first / last stage) is
  // e^{-i gamma j/2} e^{-i pi r/R}, negated for rows k >= L/2 (k_c = k - L), so
  // only e^{-i gamma j/2} is looked up, once per butterfly.
  float2 col_ph = make_float2(1.f, 0.f);
  if (PHASE) col_ph = cmul(__ldg(pr.phase + o), __ldg(pr.phase + ch * W + (int)(threadIdx.x % W)));
  const PhaseHook<L, INV, PHASE> hook{pr.phase, col_ph};
  // centred row i of an N-row input or output <-> grid row k of the L-point
  // transform: k = i - N/2 (mod L); rows N/2 <= k < L - N/2 are the padding
  auto load = [&](int k, int c) -> float2 {
    int i = k;
    if (PAD_IN) {
      if (k < half) i = k + half;
      else if (k >= L - half) i = k - (L - half);
      else return make_float2(0.f, 0.f);
      if (!col_live(c)) return make_float2(0.f, 0.f);
    } else if (INV && pr.consume) {
      // the adjoint grid is zero outside the ball: whole rows are read when a
      // column of the CTA needs them (and cleared after the loads, below)
      if (!row_live(k)) return make_float2(0.f, 0.f);
    } else if (INV && !live(k, c)) {
      return make_float2(0.f, 0.f);  // cells outside the touched ball are zero
    }
    return ib[(long long)i * in_stride + c];
  };
  auto store = [&](int k, int c, float2 v) {
    int i = k;
    if (CROP_OUT) {
      if (k < half) i = k + half;
      else if (k >= L - half) i = k - (L - half);
      else return;
    } else if (!INV && !row_live(k)) {
      return;  // no column of this CTA has the row in the touched region
    }
    if constexpr (sizeof(OutT) == sizeof(float2)) {
      ob[(long long)i * out_stride + c] = *(const OutT*)&v;
    } else if constexpr (std::is_same<OutT, __nv_bfloat162>::value) {
      // reduced-precision grid store (forward z pass only)
      ob[(long long)i * out_stride + c] = GridBF16::pack(v, out_scale);
    } else {
      ob[(long long)i * out_stride + c] = GridF16::pack(v, out_scale);
    }
  };
  // consume: every adjoint-grid row read is cleared for the next adjoint call
  auto clear_read = [&](int k, int c) {
    if (INV && !PAD_IN && pr.consume && row_live(k))
      const_cast<float2*>(ib)[(long long)k * in_stride + c] = make_float2(0.f, 0.f);
  };
  reg_fft<L, W, 32 * W, INV>(buf, W + 1, tw, load, store, clear_read, hook);
}

// ----------------------------------------------------------------------------
// inverse x pass: rows of K -> inverse FFT -> crop to N, deapodise, real part
// ----------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(FFT_NT, ROW_MIN_CTAS) k_row_adj(const float2* __restrict__ in, void* __restrict__ vol,
                                                    int cplx, const float* __restrict__ s, int N,
                                                    const float2* __restrict__ tw) {
  extern __shared__ float2 buf[];
  const int nrows = N * N;
  const int row0 = blockIdx.x * ROW_W;
  const int half = N / 2;
  for (int base = threadIdx.x; base < ROW_W * K; base += ROW_CHUNK * FFT_NT) {
    float2 t[ROW_CHUNK];
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      const int c = idx / K, k = idx - c * K;
      const int r = row0 + c;
      t[u] = (idx < ROW_W * K && r < nrows) ? in[(size_t)r * K + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      if (idx < ROW_W * K) {
        const int c = idx / K, k = idx - c * K;
        buf[k * ROW_PITCH + c] = t[u];
      }
    }
  }
  __syncthreads();
  smem_fft<K, ROW_W, FFT_NT, true>(buf, ROW_PITCH, tw);
  for (int idx = threadIdx.x; idx < ROW_W * N; idx += FFT_NT) {
    const int c = idx / N, x = idx - c * N;
    const int r = row0 + c;
    if (r < nrows) {
      const int z = r / N, y = r - z * N;
      const float sc = __ldg(s + x) * __ldg(s + y) * __ldg(s + z);
      const float2 v = cscale(buf[centred_to_grid(x, half, K) * ROW_PITCH + c], sc);
      if (cplx) ((float2*)vol)[(size_t)r * N + x] = v;
      else ((float*)vol)[(size_t)r * N + x] = v.x;
    }
  }
}

// ----------------------------------------------------------------------------
// inverse x pass to a real volume: two rows per complex transform.  Only the
// real part of each row's transform is kept, and Re IFFT(a) = IFFT(H a) with
// the Hermitian part (H a)[k] = (a[k] + conj a[-k]) / 2.  So rows a and b go in
// as Z = H a + i H b and come out as Re IFFT(a) + i Re IFFT(b).  A thread
// builds Z[j] and Z[-j] = conj(H a[j]) + i conj(H b[j]) from the four loads
// a[j], a[-j], b[j], b[-j]; 16 rows share one transform of 8 columns.
// ----------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(FFT_NT, ROW_MIN_CTAS) k_row_adj_real(const float2* __restrict__ in,
                                                         float* __restrict__ vol, const float* __restrict__ s,
                                                         int N, const float2* __restrict__ tw) {
  extern __shared__ float2 buf[];
  const int nrows = N * N;
  const int row0 = blockIdx.x * (2 * ROW_W);
  const int half = N / 2;
  constexpr int KH = K / 2 + 1;  // j = 0 .. K/2 pairs with K - j
  constexpr int U = ROW_CHUNK / 4;
  for (int base = threadIdx.x; base < ROW_W * KH; base += U * FFT_NT) {
    float2 a[U], am[U], b[U], bm[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * FFT_NT;
      a[u] = am[u] = b[u] = bm[u] = make_float2(0.f, 0.f);
      if (idx < ROW_W * KH) {
        const int c = idx / KH, j = idx - c * KH;
        const int jm = j == 0 ? 0 : K - j;
        const int ra = row0 + 2 * c;
        if (ra < nrows) {
          a[u] = in[(size_t)ra * K + j];
          am[u] = in[(size_t)ra * K + jm];
        }
        if (ra + 1 < nrows) {
          b[u] = in[(size_t)(ra + 1) * K + j];
          bm[u] = in[(size_t)(ra + 1) * K + jm];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * FFT_NT;
      if (idx < ROW_W * KH) {
        const int c = idx / KH, j = idx - c * KH;
        const int jm = j == 0 ? 0 : K - j;
        const float2 ha = make_float2(0.5f * (a[u].x + am[u].x), 0.5f * (a[u].y - am[u].y));
        const float2 hb = make_float2(0.5f * (b[u].x + bm[u].x), 0.5f * (b[u].y - bm[u].y));
        buf[j * ROW_PITCH + c] = make_float2(ha.x - hb.y, ha.y + hb.x);
        buf[jm * ROW_PITCH + c] = make_float2(ha.x + hb.y, hb.x - ha.y);
      }
    }
  }
  __syncthreads();
  smem_fft<K, ROW_W, FFT_NT, true>(buf, ROW_PITCH, tw);
  for (int idx = threadIdx.x; idx < ROW_W * N; idx += FFT_NT) {
    const int c = idx / N, x = idx - c * N;
    const int ra = row0 + 2 * c, rb = ra + 1;
    const float2 v = buf[centred_to_grid(x, half, K) * ROW_PITCH + c];
    const float sx = __ldg(s + x);
    if (ra < nrows) {
      const int z = ra / N, y = ra - z * N;
      vol[(size_t)ra * N + x] = v.x * (sx * __ldg(s + y) * __ldg(s + z));
    }
    if (rb < nrows) {
      const int z = rb / N, y = rb - z * N;
      vol[(size_t)rb * N + x] = v.y * (sx * __ldg(s + y) * __ldg(s + z));
    }
  }
}

// ----------------------------------------------------------------------------
// per-line centred DFTs.  FWD (projection): a[m] = lw[l] w[m] (-1)^m X[m];
// p[t] = (-1)^{M/2} (-1)^t / M * sum_m a[m] e^{+2 pi i m t / M}.
// ADJ: a[t] = (-1)^t y[t]; Y[m] = (-1)^{M/2} (-1)^m lw[l] conj(w[m]) / M * sum_t a[t] e^{-2 pi i m t / M}.
// w: radial weights (or null for 1), lw: real per-line weights (or null for 1).
// Rows are lines (l0 + c); in-place operation (in == out) is allowed.
// ----------------------------------------------------------------------------
template <int M, bool FWD>
__global__ void __launch_bounds__(FFT_NT, ROW_MIN_CTAS) k_line(const float2* in, float2* out, int D,
                                                 const float2* __restrict__ weight,
                                                 const float* __restrict__ line_weight,
                                                 const float2* __restrict__ tw) {
  extern __shared__ float2 buf[];
  const int l0 = blockIdx.x * ROW_W;
  for (int base = threadIdx.x; base < ROW_W * M; base += ROW_CHUNK * FFT_NT) {
    float2 t[ROW_CHUNK];
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      const int c = idx / M, m = idx - c * M;
      const int l = l0 + c;
      t[u] = (idx < ROW_W * M && l < D) ? in[(size_t)l * M + m] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < ROW_CHUNK; ++u) {
      const int idx = base + u * FFT_NT;
      if (idx < ROW_W * M) {
        const int c = idx / M, m = idx - c * M;
        float2 v = t[u];
        if (FWD && weight) v = cmul(v, __ldg(weight + m));
        if (m & 1) v = make_float2(-v.x, -v.y);
        buf[m * ROW_PITCH + c] = v;
      }
    }
  }
  __syncthreads();
  smem_fft<M, ROW_W, FFT_NT, FWD>(buf, ROW_PITCH, tw);
  const float sc = (((M / 2) & 1) ? -1.f : 1.f) / (float)M;
  if (!line_weight) {
    for (int idx = threadIdx.x; idx < ROW_W * M; idx += FFT_NT) {
      const int c = idx / M, t = idx - c * M;
      const int l = l0 + c;
      if (l < D) {
        float2 v = cscale(buf[t * ROW_PITCH + c], (t & 1) ? -sc : sc);
        if (!FWD && weight) v = cmulc(v, __ldg(weight + t));
        out[(size_t)l * M + t] = v;
      }
    }
  } else {
    // the per-line weight is a scalar: applied with the output scale (both directions)
    for (int idx = threadIdx.x; idx < ROW_W * M; idx += FFT_NT) {
      const int c = idx / M, t = idx - c * M;
      const int l = l0 + c;
      if (l < D) {
        const float s_l = sc * __ldg(line_weight + l);
        float2 v = cscale(buf[t * ROW_PITCH + c], (t & 1) ? -s_l : s_l);
        if (!FWD && weight) v = cmulc(v, __ldg(weight + t));
        out[(size_t)l * M + t] = v;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// bound on the oversampled grid's magnitude: |Y[k]| <= sum_n |s(n) x[n]|,
// used to pick the power-of-two scale of a reduced-precision grid
// ----------------------------------------------------------------------------
__global__ void k_abs_bound(const void* __restrict__ vol, int cplx, const float* __restrict__ s, int N,
                            float* __restrict__ bound) {
  const long long n3 = (long long)N * N * N;
  float acc = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % N);
    const int y = (int)((i / N) % N);
    const int z = (int)(i / ((long long)N * N));
    const float sc = __ldg(s + x) * __ldg(s + y) * __ldg(s + z);
    float a;
    if (cplx) {
      const float2 v = ((const float2*)vol)[i];
      a = sqrtf(v.x * v.x + v.y * v.y);
    } else {
      a = fabsf(((const float*)vol)[i]);
    }
    acc = fmaf(a, sc, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(bound, acc);
}

cudaError_t launch_abs_bound(const void* vol, int cplx, const float* s, int N, float* bound, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bound, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  k_abs_bound<<<152 * 4, 256, 0, st>>>(vol, cplx, s, N, bound);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
static size_t fft_smem(int L) { return (size_t)L * FFT_PITCH * sizeof(float2); }
static size_t row_smem(int L) { return (size_t)L * ROW_PITCH * sizeof(float2); }

template <typename F>
static cudaError_t set_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define NUFFT_FFT_SIZES(X) X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

bool fft_length_supported(int L) {
  switch (L) {
#define CASE_L(V) case V:
    NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
    return true;
    default:
      return false;
  }
}

template <int K>
static cudaError_t launch_row_fwd_t(const void* vol, int cplx, float2* out, const float* s, int N,
                                    const float2* tw, cudaStream_t st) {
  if (!cplx) {
    auto f = k_row_fwd_real<K>;
    cudaError_t e = set_smem(f, row_smem(K));
    if (e != cudaSuccess) return e;
    const int grid = (N * N + 2 * ROW_W - 1) / (2 * ROW_W);
    f<<<grid, FFT_NT, row_smem(K), st>>>((const float*)vol, out, s, N, tw);
    return cudaGetLastError();
  }
  auto f = k_row_fwd<K>;
  cudaError_t e = set_smem(f, row_smem(K));
  if (e != cudaSuccess) return e;
  const int grid = (N * N + ROW_W - 1) / ROW_W;
  f<<<grid, FFT_NT, row_smem(K), st>>>(vol, cplx, out, s, N, tw);
  return cudaGetLastError();
}

cudaError_t launch_row_fwd(int K, const void* vol, int cplx, float2* out, const float* s, int N,
                           const float2* tw, cudaStream_t st) {
  switch (K) {
#define CASE_L(V) case V: return launch_row_fwd_t<V>(vol, cplx, out, s, N, tw, st);
    NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
  }
  return cudaErrorInvalidValue;
}

template <int K>
static cudaError_t launch_row_adj_t(const float2* in, void* vol, int cplx, const float* s, int N,
                                    const float2* tw, cudaStream_t st) {
  if (!cplx) {
    auto f = k_row_adj_real<K>;
    cudaError_t e = set_smem(f, row_smem(K));
    if (e != cudaSuccess) return e;
    const int grid = (N * N + 2 * ROW_W - 1) / (2 * ROW_W);
    f<<<grid, FFT_NT, row_smem(K), st>>>(in, (float*)vol, s, N, tw);
    return cudaGetLastError();
  }
  auto f = k_row_adj<K>;
  cudaError_t e = set_smem(f, row_smem(K));
  if (e != cudaSuccess) return e;
  const int grid = (N * N + ROW_W - 1) / ROW_W;
  f<<<grid, FFT_NT, row_smem(K), st>>>(in, vol, cplx, s, N, tw);
  return cudaGetLastError();
}

cudaError_t launch_row_adj(int K, const float2* in, void* vol, int cplx, const float* s, int N,
                           const float2* tw, cudaStream_t st) {
  switch (K) {
#define CASE_L(V) case V: return launch_row_adj_t<V>(in, vol, cplx, s, N, tw, st);
    NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
  }
  return cudaErrorInvalidValue;
}

template <int L, bool INV, bool PAD_IN, bool CROP_OUT, typename OutT, int W, bool PHASE>
static cudaError_t launch_col_w(const float2* in, OutT* out, int N, int n_outer, int row_len,
                                long long in_outer, long long in_stride, long long out_outer,
                                long long out_stride, const float2* tw, const float* out_scale, ColPrune pr,
                                cudaStream_t st) {
  auto f = k_col<L, INV, PAD_IN, CROP_OUT, OutT, W, PHASE>;
  const size_t smem = (size_t)L * (W + 1) * sizeof(float2);
  cudaError_t e = set_smem(f, smem);
  if (e != cudaSuccess) return e;
  const int n_chunks = row_len / W;
  const long long grid = (long long)n_outer * n_chunks;
  f<<<(unsigned)grid, 32 * W, smem, st>>>(in, out, N, n_chunks, in_outer, in_stride, out_outer, out_stride, tw,
                                          out_scale, pr);
  return cudaGetLastError();
}

template <int L, bool INV, bool PAD_IN, bool CROP_OUT, typename OutT>
static cudaError_t launch_col_t(const float2* in, OutT* out, int N, int n_outer, int row_len,
                                long long in_outer, long long in_stride, long long out_outer,
                                long long out_stride, const float2* tw, const float* out_scale, ColPrune pr,
                                cudaStream_t st) {
  // 16 columns (128-byte row segments), 512 threads, two CTAs per SM: 32
  // columns with 1024 threads (one CTA per SM) measured 0.1 ms slower per z pass
  if (pr.phase)
    return launch_col_w<L, INV, PAD_IN, CROP_OUT, OutT, 16, true>(in, out, N, n_outer, row_len, in_outer, in_stride,
                                                                   out_outer, out_stride, tw, out_scale, pr, st);
  return launch_col_w<L, INV, PAD_IN, CROP_OUT, OutT, 16, false>(in, out, N, n_outer, row_len, in_outer, in_stride,
                                                                  out_outer, out_stride, tw, out_scale, pr, st);
}

cudaError_t launch_col_fwd(int L, const float2* in, float2* out, int N, int n_outer, int row_len,
                           long long in_outer, long long in_stride, long long out_outer, long long out_stride,
                           const float2* tw, cudaStream_t st, ColPrune pr) {
  switch (L) {
#define CASE_L(V) case V: return launch_col_t<V, false, true, false, float2>(in, out, N, n_outer, row_len, in_outer, in_stride, out_outer, out_stride, tw, nullptr, pr, st);
    NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_fwd_lp(int L, int dtype, const float2* in, void* out, int N, int n_outer, int row_len,
                              long long in_outer, long long in_stride, long long out_outer,
                              long long out_stride, const float2* tw, const float* scale, cudaStream_t st,
                              ColPrune pr) {
  if (dtype == 1) {
    switch (L) {
#define CASE_L(V) case V: return launch_col_t<V, false, true, false, __nv_bfloat162>(in, (__nv_bfloat162*)out, N, n_outer, row_len, in_outer, in_stride, out_outer, out_stride, tw, scale, pr, st);
      NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
    }
  } else {
    switch (L) {
#define CASE_L(V) case V: return launch_col_t<V, false, true, false, __half2>(in, (__half2*)out, N, n_outer, row_len, in_outer, in_stride, out_outer, out_stride, tw, scale, pr, st);
      NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_inv(int L, const float2* in, float2* out, int N, int n_outer, int row_len,
                           long long in_outer, long long in_stride, long long out_outer, long long out_stride,
                           const float2* tw, cudaStream_t st, ColPrune pr) {
  switch (L) {
#define CASE_L(V) case V: return launch_col_t<V, true, false, true, float2>(in, out, N, n_outer, row_len, in_outer, in_stride, out_outer, out_stride, tw, nullptr, pr, st);
    NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
  }
  return cudaErrorInvalidValue;
}

template <int M, bool FWD>
static cudaError_t launch_line_t(const float2* in, float2* out, int D, const float2* w, const float* lw,
                                 const float2* tw, cudaStream_t st) {
  auto f = k_line<M, FWD>;
  cudaError_t e = set_smem(f, row_smem(M));
  if (e != cudaSuccess) return e;
  const int grid = (D + ROW_W - 1) / ROW_W;
  f<<<grid, FFT_NT, row_smem(M), st>>>(in, out, D, w, lw, tw);
  return cudaGetLastError();
}

cudaError_t launch_line(int M, bool fwd, const float2* in, float2* out, int D, const float2* w,
                        const float2* tw, cudaStream_t st, const float* lw) {
  if (fwd) {
    switch (M) {
#define CASE_L(V) case V: return launch_line_t<V, true>(in, out, D, w, lw, tw, st);
      NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
    }
  } else {
    switch (M) {
#define CASE_L(V) case V: return launch_line_t<V, false>(in, out, D, w, lw, tw, st);
      NUFFT_FFT_SIZES(CASE_L)
#undef CASE_L
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace nufft
