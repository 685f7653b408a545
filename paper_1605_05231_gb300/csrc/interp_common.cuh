// Device helpers shared by the gather and spread translation units: point
// decoding, tile staging, the layouts and lane assignments of the
// warp-cooperative variants, and device-attribute queries.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace nufft {

// The first tap fl - J/2 + 1 wrapped into [0, K).  The plan admits |u| <= K/2
// (|omega| <= pi, |d| <= 1), so one conditional add or subtract of K wraps it;
// anything else takes the general modulo.
__device__ __forceinline__ int wrap_tap(int s, int K) {
  s += s < 0 ? K : 0;
  s -= s >= K ? K : 0;
  if ((unsigned)s >= (unsigned)K) s = ((s % K) + K) % K;
  return s;
}

// first tap (wrapped into [0, K)) and fractional offset of each axis
template <int J>
__device__ __forceinline__ void decode_point(const InterpGeom& g, uint32_t id, int (&w0)[3], float (&f)[3]) {
  const int l = (int)(id / (uint32_t)g.M);
  const int m = (int)(id - (uint32_t)l * (uint32_t)g.M);
  const float2 r = __ldg(g.rad + m);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 d = __ldg(g.dir + (size_t)l * 3 + a);
    int fl;
    reduce_coord(r.x, r.y, d.x, d.y, fl, f[a]);
    w0[a] = wrap_tap(fl - J / 2 + 1, g.K);
  }
}

// decode_point plus what the real-weight kernels need: per axis the mask of
// taps whose unwrapped index k lies outside [-K/2, K/2) (their grid cell holds
// the phase of k -/+ K, which differs by a sign), and the point's phase
// e^{i gamma (ux + uy + uz) / 2} = e^{i pi (ux + uy + uz) / K}.
template <int J, class Geom>
__device__ __forceinline__ void decode_point_real(const Geom& g, uint32_t id, int (&w0)[3], float (&f)[3],
                                                  int (&flip)[3], float2& phase) {
  const int l = (int)(id / (uint32_t)g.M);
  const int m = (int)(id - (uint32_t)l * (uint32_t)g.M);
  const float2 r = __ldg(g.rad + m);
  const int K = g.K, h = K / 2;
  int su = 0;
  float sf = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 d = __ldg(g.dir + (size_t)l * 3 + a);
    int fl;
    reduce_coord(r.x, r.y, d.x, d.y, fl, f[a]);
    const int kf = fl - J / 2 + 1;  // unwrapped first tap
    w0[a] = wrap_tap(kf, K);
    int mk = 0;
    if (kf < -h || kf + J - 1 >= h) {
#pragma unroll
      for (int j = 0; j < J; ++j) mk |= ((kf + j < -h) || (kf + j >= h)) ? (1 << j) : 0;
    }
    flip[a] = mk;
    su += fl;
    sf += f[a];
  }
  // e^{i pi (su + sf) / K}: su reduced modulo 2K into [-K, K) first
  su = su % (2 * K);
  su += su < -K ? 2 * K : 0;
  su -= su >= K ? 2 * K : 0;
  float sn, cs;
  sincospif(((float)su + sf) / (float)K, &sn, &cs);
  phase = make_float2(cs, sn);
}

// real weights rho_j(f) of one axis from their fitted polynomials (Horner in
// t = 2 f - 1), with the taps of `flip` negated
template <int J>
__device__ __forceinline__ void real_coeffs(const RealPoly& P, float f, int flip, float (&c)[J]) {
  const float t = fmaf(2.f, f, -1.f);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float v = P.a[j][kPolyDeg];
#pragma unroll
    for (int q = kPolyDeg - 1; q >= 0; --q) v = fmaf(v, t, P.a[j][q]);
    c[j] = (flip >> j) & 1 ? -v : v;
  }
}

static int g_num_sms = 0;
static inline int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return g_num_sms;
}

// Min-max coefficients of the J taps of one axis at fractional offset f from
// the fitted polynomials: Horner's rule in t = 2 f - 1, coefficients read from
// the kernel parameters (uniform over the warp).
template <int J>
__device__ __forceinline__ void poly_coeffs(const CoefPoly& P, float f, float2 (&c)[J]) {
  const float t = fmaf(2.f, f, -1.f);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float re = P.a[j][0][kPolyDeg], im = P.a[j][1][kPolyDeg];
#pragma unroll
    for (int q = kPolyDeg - 1; q >= 0; --q) {
      re = fmaf(re, t, P.a[j][0][q]);
      im = fmaf(im, t, P.a[j][1][q]);
    }
    c[j] = make_float2(re, im);
  }
}

// Coefficients of one axis: the table's linear interpolation (L > 0) or the
// exact coefficients' polynomials (L == 0); the branch is uniform per launch.
template <int J>
__device__ __forceinline__ void point_coeffs(const InterpGeom& g, float f, float2 (&c)[J]) {
  if (g.L == 0)
    poly_coeffs<J>(g.poly, f, c);
  else
    table_coeffs_v4<J>(g.table, g.L, f, c);
}

template <typename G>
__device__ __forceinline__ float lp_inv_scale(const InterpGeom& g) {
  if constexpr (G::kLowPrecision) return 1.f / lp_scale_from_bound(*g.lp_bound);
  return 1.f;
}

// ---------------------------------------------------------------------------
// staging of a padded tile, plain [iz][iy][ix] layout (pitch E)
// ---------------------------------------------------------------------------
template <typename G>
__device__ __forceinline__ void stage_tile_plain(const typename G::T* __restrict__ grid, float inv_scale, int K,
                                                 int E, int x0, int y0, int z0, float2* tile) {
  const int n = E * E * E;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int ix = idx % E;
    const int t = idx / E;
    const int iy = t % E, iz = t / E;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    tile[idx] = G::load(grid, ((size_t)gz * K + gy) * K + gx, inv_scale);
  }
}

// ---------------------------------------------------------------------------
// variant 1 (J = 6): persistent CTAs (one per SM, 16 warps), the coefficient
// table resident in shared memory, one warp per point.
//
// Phase 1: each lane decodes one point of a batch of 32 and writes its 18
// coefficients (x, y, z) to a per-warp buffer.  Phase 2: for each of the 32
// points, lane (jx, jy) = (lane % 6, lane / 6) serves the taps (jx, jy, 0..5);
// the four pairs (2..5, 5) left over are served by lanes 0..23 as
// (jx, jz) = (2 + lane % 4, lane / 4).  With the tile's row pitch = 6 and
// plane pitch = 4 (mod 16 float2), every tap load of a phase-2 instruction
// hits a distinct bank pair.  The gather then sums each lane's 32 partial
// values across the warp with a transpose-reduction (31 shuffles per
// component for 32 points).
// ---------------------------------------------------------------------------
constexpr int V1_WARPS = 16;
constexpr int V1_THREADS = V1_WARPS * 32;
constexpr int V1_CSTRIDE = 20;  // float2 slots per point: cx[6] cy[6] cz[6] value pad

struct V1Layout {
  int E, P, PP;
  int tile_f2, table_f2;
  size_t bytes;
};

__host__ __device__ inline V1Layout v1_layout(int T, int L) {
  V1Layout l;
  l.E = T + 5;
  l.P = l.E + ((6 - l.E % 16) + 16) % 16;
  const int pp = l.E * l.P;
  l.PP = pp + ((4 - pp % 16) + 16) % 16;
  l.tile_f2 = l.E * l.PP;
  l.table_f2 = (L + 1) * 6;
  l.bytes = ((size_t)l.table_f2 + l.tile_f2 + (size_t)V1_WARPS * 32 * V1_CSTRIDE) * sizeof(float2) +
            (size_t)V1_WARPS * 32 * sizeof(int4);
  return l;
}

// Phase 1 for one lane: decode, locate in the tile, write coefficients.
// Returns the tile offset of the first tap (or -1 when the lane has no point).
__device__ __forceinline__ int v1_phase1(const InterpGeom& g, const float2* table, int pi, int cnt, int start,
                                         int x0, int y0, int z0, int P, int PP, float2* cp, uint32_t& id,
                                         uint32_t& tw) {
  if (pi >= cnt) return -1;
  const uint2 ent = g.sorted[start + pi];
  id = ent.x;
  tw = ent.y;
  int w0[3];
  float f[3];
  decode_point<6>(g, id, w0, f);
  const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
  if ((unsigned)lx >= (unsigned)g.T || (unsigned)ly >= (unsigned)g.T || (unsigned)lz >= (unsigned)g.T) {
    atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
    return -1;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float fl = f[a] * (float)g.L;
    int i = (int)fl;
    if (i > g.L - 1) i = g.L - 1;
    const float t = fl - (float)i;
    const float4* r0 = (const float4*)(table + i * 6);
    const float4* r1 = (const float4*)(table + i * 6 + 6);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 a0 = r0[q], a1 = r1[q];
      cp[a * 6 + 2 * q] = make_float2(fmaf(t, a1.x - a0.x, a0.x), fmaf(t, a1.y - a0.y, a0.y));
      cp[a * 6 + 2 * q + 1] = make_float2(fmaf(t, a1.z - a0.z, a0.z), fmaf(t, a1.w - a0.w, a0.w));
    }
  }
  return (lz * PP + ly * P + lx);
}

template <typename G>
__device__ __forceinline__ void stage_tile_padded(const typename G::T* __restrict__ grid, float inv_scale, int K,
                                                  int E, int P, int PP, int x0, int y0, int z0, float2* tile) {
  const int n = E * E * E;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int ix = idx % E;
    const int t = idx / E;
    const int iy = t % E, iz = t / E;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    tile[iz * PP + iy * P + ix] = G::load(grid, ((size_t)gz * K + gy) * K + gx, inv_scale);
  }
}

// ---------------------------------------------------------------------------
// variant 2 (J = 6): every warp owns a private, unpadded E^3 tile (E = T + 5)
// and takes whole subproblems from a device work counter; the coefficient
// table is shared by the CTA in shared memory.  The gather works as in
// variant 1; the spread accumulates with plain read-modify-writes (no shared
// atomics: the warp is the only writer of its tile, and within one point its
// lanes touch distinct cells), then adds the tile to the grid with vector
// atomics.
//
// Lane assignment: lanes 0..31 serve 32 of the 36 (jx, jy) tap pairs for every
// jz; lanes 0..23 serve the remaining 4 pairs x 6 jz.  The assignment is chosen
// so that within each half-warp the offsets jx + E jy (+ E^2 jz) are distinct
// modulo 16 float2 (= 32 banks): every shared access is one wavefront per
// half-warp with the unpadded pitch.  Encoded as jx + 8 jy (+ 64 jz).
// ---------------------------------------------------------------------------
static __device__ const unsigned char kLaneMain13[32] = {0, 8, 16, 32, 9, 17, 25, 2, 10, 18, 26, 34, 3, 35, 12, 5, 24, 40, 33, 42, 11, 19, 27, 43, 20, 28, 36, 13, 21, 29, 37, 45};
static __device__ const unsigned short kLaneOvf13[24] = {1, 65, 129, 193, 257, 321, 41, 105, 4, 68, 132, 196, 260, 172, 236, 300, 169, 233, 297, 361, 324, 44, 108, 364};
static __device__ const unsigned char kLaneMain21[32] = {0, 8, 16, 32, 9, 17, 2, 10, 18, 26, 3, 11, 19, 12, 20, 21, 24, 40, 1, 25, 34, 42, 27, 35, 43, 28, 36, 44, 5, 13, 29, 45};
static __device__ const unsigned short kLaneOvf21[24] = {33, 97, 161, 225, 289, 41, 105, 169, 4, 68, 132, 196, 260, 324, 101, 165, 353, 233, 297, 361, 37, 229, 293, 357};

// Lane tables of the fixed-point spread (variant 5, E = 13): 4-byte cells, so
// an instruction is one wavefront when its 32 lanes hit 32 distinct banks.  The
// column offsets jx + 13 jy of the 36 (jx, jy) pairs reach 31 residues mod 32:
// lanes 0..30 take 31 columns with distinct residues for every jz (lane 31
// none, 255); lanes 0..29 take the remaining 30 taps, lanes 0..14 and 15..29
// each with distinct residues of jx + 13 jy + 169 jz (lanes 30, 31 none).
static __device__ const unsigned char kLaneMainI13[32] = {0, 1, 2, 3, 4, 5, 45, 24, 25, 26, 27, 28, 29, 8, 9, 10, 11, 12, 13, 32, 33, 34, 35, 36, 37, 16, 17, 18, 19, 20, 21, 255};
static __device__ const unsigned short kLaneOvfI13[32] = {236, 40, 41, 42, 43, 296, 297, 298, 299, 300, 104, 105, 106, 107, 360, 44, 108, 361, 362, 363, 364, 168, 169, 170, 171, 172, 232, 233, 234, 235, 65535, 65535};
// Lanes without a tap of their own (main: lane 31; extra: lanes 30, 31) add
// zero to a cell at an offset whose residue is free in their instruction, so
// the instruction runs without a predicate and keeps its wavefront count.
static __device__ const unsigned char kPadI13[3] = {19, 24, 25};  // main lane 31, extra lanes 30 and 31

// ---------------------------------------------------------------------------
// fixed-point tile accumulation (spreads 5, 6 and 7): rounding of a
// contribution to an integer number of units by an FMA with 1.5 * 2^23 (floats
// in [2^23, 2^24) are spaced by 1), and the lanes' taps on a 13^3 int32 tile
// ---------------------------------------------------------------------------
constexpr float kRoundMagic = 12582912.0f;            // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;           // its bits
constexpr int kTileEmpty = -1000;                     // tile exponent before the first point
constexpr unsigned kBoundLimitBits = (100u + 127u) << 23;  // 2^100: larger bounds (and NaN) poison the tile

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }  // -126 <= k <= 127

// a b + c d rounded to an integer, for |a b|, |c d|, |a b + c d| < 2^22
__device__ __forceinline__ int round_units(float a, float b, float c, float d) {
  return __float_as_int(fmaf(a, b, fmaf(c, d, kRoundMagic))) - kRoundMagicBits;
}

struct V5Lanes {
  int main_off, ovf_off;
  int mjx, mjy, ojx, ojy, ojz;
  bool has_main, has_ovf;
};

__device__ __forceinline__ V5Lanes v5_lanes(int lane) {
  constexpr int E = 13;
  const unsigned m = kLaneMainI13[lane], o = kLaneOvfI13[lane];
  V5Lanes r;
  r.has_main = m != 255u;
  r.has_ovf = o != 65535u;
  r.mjx = r.has_main ? (m & 7) : 0;
  r.mjy = r.has_main ? ((m >> 3) & 7) : 0;
  r.ojx = r.has_ovf ? (o & 7) : 0;
  r.ojy = r.has_ovf ? ((o >> 3) & 7) : 0;
  r.ojz = r.has_ovf ? ((o >> 6) & 7) : 0;
  r.main_off = r.mjx + E * r.mjy;
  r.ovf_off = r.ojx + E * r.ojy + E * E * r.ojz;
  return r;
}

// a b rounded to an integer, for |a b| < 2^22
__device__ __forceinline__ int round_unit1(float a, float b) {
  return __float_as_int(fmaf(a, b, kRoundMagic)) - kRoundMagicBits;
}

constexpr int V2_WARPS = 8;
constexpr int V2_CSTRIDE = 18;  // float2 per point: cx[6] cy[6] cz[6]

struct V2Layout {
  int E;
  size_t table_bytes, warp_bytes, bytes;
};

__host__ __device__ inline V2Layout v2_layout(int T, int L) {
  V2Layout l;
  l.E = T + 5;
  l.table_bytes = (size_t)(L + 1) * 6 * sizeof(float2);
  size_t w = (size_t)32 * V2_CSTRIDE * sizeof(float2)   // coefficients
             + 32 * sizeof(float2)                      // point values (spread)
             + (size_t)l.E * l.E * l.E * sizeof(float2) // tile
             + 32 * sizeof(int);                        // tile offsets
  l.warp_bytes = (w + 15) / 16 * 16;
  l.bytes = l.table_bytes + V2_WARPS * l.warp_bytes;
  return l;
}

struct V2Lanes {
  int main_off, ovf_off;
  int mjx, mjy, ojx, ojy, ojz;
};

__device__ __forceinline__ V2Lanes v2_lanes(int E, int lane) {
  const unsigned m = (E == 13) ? kLaneMain13[lane] : kLaneMain21[lane];
  const unsigned o = lane < 24 ? ((E == 13) ? kLaneOvf13[lane] : kLaneOvf21[lane]) : 0u;
  V2Lanes r;
  r.mjx = m & 7;
  r.mjy = (m >> 3) & 7;
  r.ojx = o & 7;
  r.ojy = (o >> 3) & 7;
  r.ojz = (o >> 6) & 7;
  r.main_off = r.mjx + E * r.mjy;
  r.ovf_off = r.ojx + E * r.ojy + E * E * r.ojz;
  return r;
}

// Phase 1 (one point per lane): decode, locate in the tile, interpolate the 18
// coefficients from the shared table and store them as nine float4.
__device__ __forceinline__ int v2_phase1(const InterpGeom& g, const float2* table, int pi, int cnt, int start,
                                         int x0, int y0, int z0, int E, float2* cp, uint32_t& id, uint32_t& tw) {
  if (pi >= cnt) return -1;
  const uint2 ent = g.sorted[start + pi];
  id = ent.x;
  tw = ent.y;
  int w0[3];
  float f[3];
  decode_point<6>(g, id, w0, f);
  const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
  if ((unsigned)lx >= (unsigned)g.T || (unsigned)ly >= (unsigned)g.T || (unsigned)lz >= (unsigned)g.T) {
    atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
    return -1;
  }
  float4* c4 = (float4*)cp;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float fl = f[a] * (float)g.L;
    int i = (int)fl;
    if (i > g.L - 1) i = g.L - 1;
    const float t = fl - (float)i;
    const float4* r0 = (const float4*)(table + i * 6);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 a0 = r0[q], a1 = r0[q + 3];
      c4[a * 3 + q] = make_float4(fmaf(t, a1.x - a0.x, a0.x), fmaf(t, a1.y - a0.y, a0.y),
                                  fmaf(t, a1.z - a0.z, a0.z), fmaf(t, a1.w - a0.w, a0.w));
    }
  }
  return (lz * E + ly) * E + lx;
}

static inline int max_optin_smem() {
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return maxsm;
}

static inline bool v1_fits(const InterpGeom& g) {
  if (g.J != 6 || g.L == 0) return false;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v1_layout(g.T, g.L).bytes <= (size_t)maxsm;
}

}  // namespace nufft
