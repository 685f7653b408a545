// Interpolation kernels: the separable J-tap min-max interpolator T of
// Eq. 2.11 (gather, grid -> points on radial lines) and its transpose T^H
// (spread, points -> grid, Eq. 2.13 read as the NUFFT transpose).
//
// Points are enumerated as id = l * M + m (line l, radial sample m) and sorted
// by the grid tile (edge T) that holds their first tap.  A subproblem is a run
// of at most S sorted points of one tile; its CTA stages the tile plus a halo
// of J - 1 cells per axis ((T + J - 1)^3 cells, periodic in K) in shared memory
// and serves every tap from there.  Writes of the gather go straight to
// lines[id]: within a tile the sorted order keeps consecutive samples of a
// line together, so the stores are mostly coalesced runs.
#include "common.cuh"
#include "internal.h"
#include "spread_taps.inc"

namespace nufft {

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
    int s = (fl - J / 2 + 1) % g.K;
    if (s < 0) s += g.K;
    w0[a] = s;
  }
}

static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return g_num_sms;
}

template <int J>
__global__ void k_bin_points(InterpGeom g, const uint32_t* __restrict__ ids, long long P, uint32_t* __restrict__ bins) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    int w0[3];
    float f[3];
    decode_point<J>(g, ids[p], w0, f);
    bins[p] = (uint32_t)(((w0[2] / g.T) * g.nT + w0[1] / g.T) * g.nT + w0[0] / g.T);
  }
}

template <int J>
static cudaError_t launch_bin_t(const InterpGeom& g, const uint32_t* ids, long long P, uint32_t* bins,
                                cudaStream_t st) {
  long long blocks = (P + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  k_bin_points<J><<<(unsigned)blocks, 256, 0, st>>>(g, ids, P, bins);
  return cudaGetLastError();
}

cudaError_t launch_bin_points(const InterpGeom& g, const uint32_t* ids, long long count, uint32_t* bins,
                              cudaStream_t st) {
  switch (g.J) {
    case 2: return launch_bin_t<2>(g, ids, count, bins, st);
    case 4: return launch_bin_t<4>(g, ids, count, bins, st);
    case 6: return launch_bin_t<6>(g, ids, count, bins, st);
    case 8: return launch_bin_t<8>(g, ids, count, bins, st);
  }
  return cudaErrorInvalidValue;
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
// variant 0: one thread per point
// ---------------------------------------------------------------------------
template <int J, typename G>
__global__ void __launch_bounds__(256) k_gather_v0(InterpGeom g, const typename G::T* __restrict__ grid,
                                                   float inv_scale, const int4* __restrict__ subs,
                                                   float2* __restrict__ out) {
  inv_scale = lp_inv_scale<G>(g);
  extern __shared__ float2 tile[];
  const int4 sp = subs[blockIdx.x];
  const int T = g.T, nT = g.nT, E = T + J - 1;
  const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
  const int x0 = bx * T, y0 = by * T, z0 = bz * T;
  stage_tile_plain<G>(grid, inv_scale, g.K, E, x0, y0, z0, tile);
  __syncthreads();
  for (int i = threadIdx.x; i < sp.z; i += blockDim.x) {
    const uint2 ent = g.sorted[sp.y + i];
    const uint32_t id = ent.x;
    int w0[3];
    float f[3];
    decode_point<J>(g, id, w0, f);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
      atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      continue;
    }
    float2 cx[J], cy[J], cz[J];
    table_coeffs<J>(g.table, g.L, f[0], cx);
    table_coeffs<J>(g.table, g.L, f[1], cy);
    table_coeffs<J>(g.table, g.L, f[2], cz);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int jz = 0; jz < J; ++jz) {
      float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
      for (int jy = 0; jy < J; ++jy) {
        const float2* tp = tile + ((lz + jz) * E + ly + jy) * E + lx;
        float2 row = make_float2(0.f, 0.f);
#pragma unroll
        for (int jx = 0; jx < J; ++jx) cmac(row, cx[jx], tp[jx]);
        cmac(zacc, cy[jy], row);
      }
      cmac(acc, cz[jz], zacc);
    }
    out[id] = acc;
    if (ent.y != kNoTwin) out[ent.y] = acc;
  }
}

template <int J>
__global__ void __launch_bounds__(256) k_spread_v0(InterpGeom g, const float2* __restrict__ in,
                                                   const int4* __restrict__ subs, float2* __restrict__ grid) {
  extern __shared__ float2 tile[];
  const int4 sp = subs[blockIdx.x];
  const int T = g.T, nT = g.nT, E = T + J - 1, K = g.K;
  const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
  const int x0 = bx * T, y0 = by * T, z0 = bz * T;
  const int n = E * E * E;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) tile[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = threadIdx.x; i < sp.z; i += blockDim.x) {
    const uint2 ent = g.sorted[sp.y + i];
    const uint32_t id = ent.x;
    int w0[3];
    float f[3];
    decode_point<J>(g, id, w0, f);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
      atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      continue;
    }
    float2 v = in[id];
    if (ent.y != kNoTwin) v = cadd(v, in[ent.y]);
    float2 cx[J], cy[J], cz[J];
    table_coeffs<J>(g.table, g.L, f[0], cx);
    table_coeffs<J>(g.table, g.L, f[1], cy);
    table_coeffs<J>(g.table, g.L, f[2], cz);
#pragma unroll
    for (int jz = 0; jz < J; ++jz) {
      const float2 vz = cmulc(v, cz[jz]);
#pragma unroll
      for (int jy = 0; jy < J; ++jy) {
        const float2 vyz = cmulc(vz, cy[jy]);
        float2* tp = tile + ((lz + jz) * E + ly + jy) * E + lx;
#pragma unroll
        for (int jx = 0; jx < J; ++jx) {
          const float2 w = cmulc(vyz, cx[jx]);
          atomicAdd(&tp[jx].x, w.x);
          atomicAdd(&tp[jx].y, w.y);
        }
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const float2 v = tile[idx];
    if (v.x == 0.f && v.y == 0.f) continue;
    const int ix = idx % E;
    const int t = idx / E;
    const int iy = t % E, iz = t / E;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    atomicAdd(&grid[((size_t)gz * K + gy) * K + gx], v);
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

template <typename G>
__global__ void __launch_bounds__(V1_THREADS, 1) k_gather_v1(InterpGeom g, const typename G::T* __restrict__ grid,
                                                             float inv_scale, const int4* __restrict__ subs,
                                                             int n_subs, float2* __restrict__ out) {
  inv_scale = lp_inv_scale<G>(g);
  extern __shared__ __align__(16) float2 smem[];
  const V1Layout lay = v1_layout(g.T, g.L);
  float2* table = smem;
  float2* tile = table + lay.table_f2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* coef = tile + lay.tile_f2 + warp * 32 * V1_CSTRIDE;
  int* meta = (int*)(tile + lay.tile_f2 + V1_WARPS * 32 * V1_CSTRIDE) + warp * 32;
  for (int i = threadIdx.x; i < lay.table_f2; i += V1_THREADS) table[i] = __ldg(g.table + i);
  const int E = lay.E, P = lay.P, PP = lay.PP, T = g.T, nT = g.nT;
  const int jx = lane % 6, jy = lane / 6;
  const int ox = 2 + (lane & 3), oz = lane >> 2;
  const int main_off = jy * P + jx;
  const int ovf_off = 5 * P + ox + oz * PP;
  for (int s = blockIdx.x; s < n_subs; s += gridDim.x) {
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    __syncthreads();
    stage_tile_padded<G>(grid, inv_scale, g.K, E, P, PP, x0, y0, z0, tile);
    __syncthreads();
    for (int b0 = warp * 32; b0 < sp.z; b0 += V1_THREADS) {
      uint32_t id = 0, tw = kNoTwin;
      const int off = v1_phase1(g, table, b0 + lane, sp.z, sp.y, x0, y0, z0, P, PP, coef + lane * V1_CSTRIDE, id, tw);
      meta[lane] = off;
      __syncwarp();
      float2 acc[32];
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        const int mo = meta[p];
        float2 r = make_float2(0.f, 0.f);
        if (mo >= 0) {
          const float2* cp = coef + p * V1_CSTRIDE;
          const float2 cxy = cmul(cp[jx], cp[6 + jy]);
          const float4 z01 = *(const float4*)(cp + 12);
          const float4 z23 = *(const float4*)(cp + 14);
          const float4 z45 = *(const float4*)(cp + 16);
          const float2* tp = tile + mo + main_off;
          float2 sa = make_float2(0.f, 0.f);
          cmac(sa, make_float2(z01.x, z01.y), tp[0]);
          cmac(sa, make_float2(z01.z, z01.w), tp[PP]);
          cmac(sa, make_float2(z23.x, z23.y), tp[2 * PP]);
          cmac(sa, make_float2(z23.z, z23.w), tp[3 * PP]);
          cmac(sa, make_float2(z45.x, z45.y), tp[4 * PP]);
          cmac(sa, make_float2(z45.z, z45.w), tp[5 * PP]);
          r = cmul(cxy, sa);
          if (lane < 24) {
            const float2 w = cmul(cmul(cp[ox], cp[11]), cp[12 + oz]);
            cmac(r, w, tile[mo + ovf_off]);
          }
        }
        acc[p] = r;
      }
      // transpose-reduction: afterwards acc[0] of lane p holds the sum for point p
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const bool upper = (lane & sh) != 0;
#pragma unroll
        for (int i = 0; i < sh; ++i) {
          const float2 send = upper ? acc[i] : acc[i + sh];
          const float2 keep = upper ? acc[i + sh] : acc[i];
          const float rx = __shfl_xor_sync(0xffffffffu, send.x, sh);
          const float ry = __shfl_xor_sync(0xffffffffu, send.y, sh);
          acc[i] = make_float2(keep.x + rx, keep.y + ry);
        }
      }
      if (off >= 0) {
        out[id] = acc[0];
        if (tw != kNoTwin) out[tw] = acc[0];
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(V1_THREADS, 1) k_spread_v1(InterpGeom g, const float2* __restrict__ in,
                                                             const int4* __restrict__ subs, int n_subs,
                                                             float2* __restrict__ grid) {
  extern __shared__ __align__(16) float2 smem[];
  const V1Layout lay = v1_layout(g.T, g.L);
  float2* table = smem;
  float2* tile = table + lay.table_f2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* coef = tile + lay.tile_f2 + warp * 32 * V1_CSTRIDE;
  int* meta = (int*)(tile + lay.tile_f2 + V1_WARPS * 32 * V1_CSTRIDE) + warp * 32;
  for (int i = threadIdx.x; i < lay.table_f2; i += V1_THREADS) table[i] = __ldg(g.table + i);
  for (int i = threadIdx.x; i < lay.tile_f2; i += V1_THREADS) tile[i] = make_float2(0.f, 0.f);
  const int E = lay.E, P = lay.P, PP = lay.PP, T = g.T, nT = g.nT, K = g.K;
  const int jx = lane % 6, jy = lane / 6;
  const int ox = 2 + (lane & 3), oz = lane >> 2;
  const int main_off = jy * P + jx;
  const int ovf_off = 5 * P + ox + oz * PP;
  for (int s = blockIdx.x; s < n_subs; s += gridDim.x) {
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    __syncthreads();  // the tile is zero again
    for (int b0 = warp * 32; b0 < sp.z; b0 += V1_THREADS) {
      uint32_t id = 0, tw = kNoTwin;
      float2* mycp = coef + lane * V1_CSTRIDE;
      const int off = v1_phase1(g, table, b0 + lane, sp.z, sp.y, x0, y0, z0, P, PP, mycp, id, tw);
      if (off >= 0) mycp[18] = tw != kNoTwin ? cadd(in[id], in[tw]) : in[id];
      meta[lane] = off;
      __syncwarp();
      for (int p = 0; p < 32; ++p) {
        const int mo = meta[p];
        if (mo < 0) continue;
        const float2* cp = coef + p * V1_CSTRIDE;
        const float2 v = cp[18];
        const float2 a = cmulc(v, cmul(cp[jx], cp[6 + jy]));  // v conj(cx cy)
        float2* tp = tile + mo + main_off;
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) {
          const float2 w = cmulc(a, cp[12 + jz]);
          atomicAdd(&tp[jz * PP].x, w.x);
          atomicAdd(&tp[jz * PP].y, w.y);
        }
        if (lane < 24) {
          const float2 w = cmulc(v, cmul(cmul(cp[ox], cp[11]), cp[12 + oz]));
          atomicAdd(&tile[mo + ovf_off].x, w.x);
          atomicAdd(&tile[mo + ovf_off].y, w.y);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    const int n = E * E * E;
    for (int idx = threadIdx.x; idx < n; idx += V1_THREADS) {
      const int ix = idx % E;
      const int t = idx / E;
      const int iy = t % E, iz = t / E;
      float2* cell = tile + iz * PP + iy * P + ix;
      const float2 v = *cell;
      if (v.x == 0.f && v.y == 0.f) continue;
      *cell = make_float2(0.f, 0.f);
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      atomicAdd(&grid[((size_t)gz * K + gy) * K + gx], v);
    }
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
__device__ const unsigned char kLaneMain13[32] = {0, 8, 16, 32, 9, 17, 25, 2, 10, 18, 26, 34, 3, 35, 12, 5, 24, 40, 33, 42, 11, 19, 27, 43, 20, 28, 36, 13, 21, 29, 37, 45};
__device__ const unsigned short kLaneOvf13[24] = {1, 65, 129, 193, 257, 321, 41, 105, 4, 68, 132, 196, 260, 172, 236, 300, 169, 233, 297, 361, 324, 44, 108, 364};
__device__ const unsigned char kLaneMain21[32] = {0, 8, 16, 32, 9, 17, 2, 10, 18, 26, 3, 11, 19, 12, 20, 21, 24, 40, 1, 25, 34, 42, 27, 35, 43, 28, 36, 44, 5, 13, 29, 45};
__device__ const unsigned short kLaneOvf21[24] = {33, 97, 161, 225, 289, 41, 105, 169, 4, 68, 132, 196, 260, 324, 101, 165, 353, 233, 297, 361, 37, 229, 293, 357};

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

template <typename G>
__global__ void __launch_bounds__(V2_WARPS * 32, 1) k_gather_v2(InterpGeom g, const typename G::T* __restrict__ grid,
                                                                float inv_scale, const int4* __restrict__ subs,
                                                                int n_subs, int* __restrict__ counter,
                                                                float2* __restrict__ out) {
  inv_scale = lp_inv_scale<G>(g);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const V2Layout lay = v2_layout(g.T, g.L);
  float2* table = (float2*)smem_raw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* coef = (float2*)(smem_raw + lay.table_bytes + warp * lay.warp_bytes);
  float2* tile = coef + 32 * V2_CSTRIDE + 32;
  const int E = lay.E, E3 = E * E * E, PP = E * E;
  int* meta = (int*)(tile + E3);
  for (int i = threadIdx.x; i < (g.L + 1) * 6; i += blockDim.x) table[i] = __ldg(g.table + i);
  __syncthreads();
  const V2Lanes ln = v2_lanes(E, lane);
  const int T = g.T, nT = g.nT, K = g.K;
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    for (int idx = lane; idx < E3; idx += 32) {
      const int ix = idx % E;
      const int t = idx / E;
      const int iy = t % E, iz = t / E;
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      tile[idx] = G::load(grid, ((size_t)gz * K + gy) * K + gx, inv_scale);
    }
    __syncwarp();
    for (int b0 = 0; b0 < sp.z; b0 += 32) {
      uint32_t id = 0, tw = kNoTwin;
      const int off = v2_phase1(g, table, b0 + lane, sp.z, sp.y, x0, y0, z0, E, coef + lane * V2_CSTRIDE, id, tw);
      meta[lane] = off;
      __syncwarp();
      float2 acc[32];
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        const int mo = meta[p];
        float2 r = make_float2(0.f, 0.f);
        if (mo >= 0) {
          const float2* cp = coef + p * V2_CSTRIDE;
          const float2 cxy = cmul(cp[ln.mjx], cp[6 + ln.mjy]);
          const float4 z01 = *(const float4*)(cp + 12);
          const float4 z23 = *(const float4*)(cp + 14);
          const float4 z45 = *(const float4*)(cp + 16);
          const float2* tp = tile + mo + ln.main_off;
          float2 sa = make_float2(0.f, 0.f);
          cmac(sa, make_float2(z01.x, z01.y), tp[0]);
          cmac(sa, make_float2(z01.z, z01.w), tp[PP]);
          cmac(sa, make_float2(z23.x, z23.y), tp[2 * PP]);
          cmac(sa, make_float2(z23.z, z23.w), tp[3 * PP]);
          cmac(sa, make_float2(z45.x, z45.y), tp[4 * PP]);
          cmac(sa, make_float2(z45.z, z45.w), tp[5 * PP]);
          r = cmul(cxy, sa);
          if (lane < 24) {
            const float2 w = cmul(cmul(cp[ln.ojx], cp[6 + ln.ojy]), cp[12 + ln.ojz]);
            cmac(r, w, tile[mo + ln.ovf_off]);
          }
        }
        acc[p] = r;
      }
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const bool upper = (lane & sh) != 0;
#pragma unroll
        for (int i = 0; i < sh; ++i) {
          const float2 send = upper ? acc[i] : acc[i + sh];
          const float2 keep = upper ? acc[i + sh] : acc[i];
          const float rx = __shfl_xor_sync(0xffffffffu, send.x, sh);
          const float ry = __shfl_xor_sync(0xffffffffu, send.y, sh);
          acc[i] = make_float2(keep.x + rx, keep.y + ry);
        }
      }
      if (off >= 0) {
        out[id] = acc[0];
        if (tw != kNoTwin) out[tw] = acc[0];
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(V2_WARPS * 32, 1) k_spread_v2(InterpGeom g, const float2* __restrict__ in,
                                                                const int4* __restrict__ subs, int n_subs,
                                                                int* __restrict__ counter,
                                                                float2* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const V2Layout lay = v2_layout(g.T, g.L);
  float2* table = (float2*)smem_raw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* coef = (float2*)(smem_raw + lay.table_bytes + warp * lay.warp_bytes);
  float2* vals = coef + 32 * V2_CSTRIDE;
  float2* tile = vals + 32;
  const int E = lay.E, E3 = E * E * E, PP = E * E;
  int* meta = (int*)(tile + E3);
  for (int i = threadIdx.x; i < (g.L + 1) * 6; i += blockDim.x) table[i] = __ldg(g.table + i);
  for (int i = lane; i < E3; i += 32) tile[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const V2Lanes ln = v2_lanes(E, lane);
  const int T = g.T, nT = g.nT, K = g.K;
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    for (int b0 = 0; b0 < sp.z; b0 += 32) {
      uint32_t id = 0, tw = kNoTwin;
      const int off = v2_phase1(g, table, b0 + lane, sp.z, sp.y, x0, y0, z0, E, coef + lane * V2_CSTRIDE, id, tw);
      vals[lane] = off >= 0 ? (tw != kNoTwin ? cadd(in[id], in[tw]) : in[id]) : make_float2(0.f, 0.f);
      meta[lane] = off;
      __syncwarp();
      for (int p = 0; p < 32; ++p) {
        const int mo = meta[p];
        if (mo < 0) continue;
        const float2* cp = coef + p * V2_CSTRIDE;
        const float2 v = vals[p];
        const float2 a = cmulc(v, cmul(cp[ln.mjx], cp[6 + ln.mjy]));  // v conj(cx cy)
        float2* tp = tile + mo + ln.main_off;
        float2 t[6];
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) t[jz] = tp[jz * PP];
        const float4 z4[3] = {*(const float4*)(cp + 12), *(const float4*)(cp + 14), *(const float4*)(cp + 16)};
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) {
          const float2 cz = (jz & 1) ? make_float2(z4[jz >> 1].z, z4[jz >> 1].w) : make_float2(z4[jz >> 1].x, z4[jz >> 1].y);
          // t += a conj(cz)
          t[jz].x = fmaf(a.x, cz.x, fmaf(a.y, cz.y, t[jz].x));
          t[jz].y = fmaf(a.y, cz.x, fmaf(-a.x, cz.y, t[jz].y));
        }
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) tp[jz * PP] = t[jz];
        if (lane < 24) {
          const float2 w = cmulc(v, cmul(cmul(cp[ln.ojx], cp[6 + ln.ojy]), cp[12 + ln.ojz]));
          float2* q = tile + mo + ln.ovf_off;
          float2 u = *q;
          u.x += w.x;
          u.y += w.y;
          *q = u;
        }
        __syncwarp();
      }
    }
    __syncwarp();
    for (int idx = lane; idx < E3; idx += 32) {
      const float2 v = tile[idx];
      if (v.x == 0.f && v.y == 0.f) continue;
      tile[idx] = make_float2(0.f, 0.f);
      const int ix = idx % E;
      const int t = idx / E;
      const int iy = t % E, iz = t / E;
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      atomicAdd(&grid[((size_t)gz * K + gy) * K + gx], v);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// spread variant 3 (J = 6, T = 8): variant 2 with more warps per SM and less
// shared-memory traffic per point.  The coefficient table is read through L1
// in phase 1 (freeing its 49 KB of shared memory for two more warps per SM),
// a point's tile offset and value travel as one float4, and the coefficients
// of the next point are loaded into registers while the current point's
// read-modify-writes drain.
// ---------------------------------------------------------------------------
constexpr int V3S_WARPS = 10;

__host__ __device__ inline size_t v3s_warp_bytes(int T) {
  const int E = T + 5;
  const size_t w = (size_t)32 * V2_CSTRIDE * sizeof(float2) + 32 * sizeof(float4) +
                   (size_t)E * E * E * sizeof(float2);
  return (w + 15) / 16 * 16;
}

__host__ __device__ inline size_t v3s_bytes(int T) { return V3S_WARPS * v3s_warp_bytes(T); }

struct V3SCoef {
  float2 cx, cy, ox, oy, oz;
  float4 z01, z23, z45;
  float4 mv;  // tile offset (int bits), value
};

__device__ __forceinline__ void v3s_load(const float2* coef, const float4* mvs, int p, const V2Lanes& ln,
                                         V3SCoef& c) {
  const float2* cp = coef + p * V2_CSTRIDE;
  c.mv = mvs[p];
  c.cx = cp[ln.mjx];
  c.cy = cp[6 + ln.mjy];
  c.z01 = *(const float4*)(cp + 12);
  c.z23 = *(const float4*)(cp + 14);
  c.z45 = *(const float4*)(cp + 16);
  c.ox = cp[ln.ojx];
  c.oy = cp[6 + ln.ojy];
  c.oz = cp[12 + ln.ojz];
}

// read-modify-write of one point's taps held by this lane
template <int PP>
__device__ __forceinline__ void v3s_apply(float2* tile, const V3SCoef& c, const V2Lanes& ln, int lane) {
  const int mo = __float_as_int(c.mv.x);
  if (mo < 0) return;
  const float2 v = make_float2(c.mv.y, c.mv.z);
  const float2 a = cmulc(v, cmul(c.cx, c.cy));  // v conj(cx cy)
  float2* tp = tile + mo + ln.main_off;
  float2 t[6];
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) t[jz] = tp[jz * PP];
  const float2 cz[6] = {make_float2(c.z01.x, c.z01.y), make_float2(c.z01.z, c.z01.w),
                        make_float2(c.z23.x, c.z23.y), make_float2(c.z23.z, c.z23.w),
                        make_float2(c.z45.x, c.z45.y), make_float2(c.z45.z, c.z45.w)};
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) {
    t[jz].x = fmaf(a.x, cz[jz].x, fmaf(a.y, cz[jz].y, t[jz].x));
    t[jz].y = fmaf(a.y, cz[jz].x, fmaf(-a.x, cz[jz].y, t[jz].y));
  }
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) tp[jz * PP] = t[jz];
  if (lane < 24) {
    const float2 w = cmulc(v, cmul(cmul(c.ox, c.oy), c.oz));
    float2* q = tile + mo + ln.ovf_off;
    float2 u = *q;
    u.x += w.x;
    u.y += w.y;
    *q = u;
  }
}

template <int T>
__global__ void __launch_bounds__(V3S_WARPS * 32, 1) k_spread_v3(InterpGeom g, const float2* __restrict__ in,
                                                                 const int4* __restrict__ subs, int n_subs,
                                                                 int* __restrict__ counter,
                                                                 float2* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E = T + 5, E2 = E * E, E3 = E2 * E, PP = E2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nT = g.nT, K = g.K;
  const size_t KK = (size_t)K * K;
  float2* coef = (float2*)(smem_raw + warp * v3s_warp_bytes(T));
  float4* mvs = (float4*)(coef + 32 * V2_CSTRIDE);
  float2* tile = (float2*)(mvs + 32);
  for (int i = lane; i < E3; i += 32) tile[i] = make_float2(0.f, 0.f);
  __syncwarp();
  const V2Lanes ln = v2_lanes(E, lane);
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    for (int b0 = 0; b0 < sp.z; b0 += 32) {
      // phase 1: one point per lane
      int off = -1;
      float2 val = make_float2(0.f, 0.f);
      const int pi = b0 + lane;
      if (pi < sp.z) {
        const uint2 ent = g.sorted[sp.y + pi];
        int w0[3];
        float f[3];
        decode_point<6>(g, ent.x, w0, f);
        const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
        if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
          off = (lz * E + ly) * E + lx;
          val = in[ent.x];
          if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
          float4* c4 = (float4*)(coef + lane * V2_CSTRIDE);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float2 c[6];
            table_coeffs_v4<6>(g.table, g.L, f[a], c);
#pragma unroll
            for (int q = 0; q < 3; ++q) c4[a * 3 + q] = make_float4(c[2 * q].x, c[2 * q].y, c[2 * q + 1].x, c[2 * q + 1].y);
          }
        } else {
          atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
        }
      }
      mvs[lane] = make_float4(__int_as_float(off), val.x, val.y, 0.f);
      __syncwarp();
      const int np = min(32, sp.z - b0);
      // two points per iteration: the second point's coefficients load while
      // the first point's read-modify-writes drain
      int p = 0;
      for (; p + 1 < np; p += 2) {
        V3SCoef c0, c1;
        v3s_load(coef, mvs, p, ln, c0);
        v3s_load(coef, mvs, p + 1, ln, c1);
        v3s_apply<PP>(tile, c0, ln, lane);
        __syncwarp();
        v3s_apply<PP>(tile, c1, ln, lane);
        __syncwarp();
      }
      if (p < np) {
        V3SCoef c0;
        v3s_load(coef, mvs, p, ln, c0);
        v3s_apply<PP>(tile, c0, ln, lane);
        __syncwarp();
      }
    }
    // add the tile to the grid: lanes walk (y, x) columns, each column along z
    for (int c = lane; c < E2; c += 32) {
      const int iy = c / E, ix = c - iy * E;
      int gx = x0 + ix, gy = y0 + iy;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      int gz = z0;
      float2* cell = tile + c;
#pragma unroll
      for (int iz = 0; iz < E; ++iz) {
        const float2 v = cell[iz * E2];
        if (v.x != 0.f || v.y != 0.f) {
          cell[iz * E2] = make_float2(0.f, 0.f);
          atomicAdd(&grid[((size_t)(gz >= K ? gz - K : gz)) * KK + (size_t)gy * K + gx], v);
        }
        ++gz;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// spread variant 4 (J = 6): one thread per point without atomics.  Each warp
// owns a private E^3 tile.  The points of a subproblem are bucketed by the
// residue of their first-tap offset modulo 32; in round r lane l spreads the
// r-th point of bucket l, so the 32 points of a round have pairwise distinct
// residues.  Taps are visited in groups of equal offset residue (the order in
// spread_taps.inc): inside one group no two lanes touch the same cell and the
// warp's accesses hit 32 distinct banks, so plain read-modify-writes are safe;
// a __syncwarp separates the groups.
// ---------------------------------------------------------------------------
constexpr int V4S_WARPS = 10;

__host__ __device__ inline size_t v4s_warp_bytes(int T, int S) {
  const int E = T + 5;
  const size_t w = (size_t)E * E * E * sizeof(float2) + (size_t)S * 2 * sizeof(int) + 96 * sizeof(int);
  return (w + 15) / 16 * 16;
}

__host__ __device__ inline size_t v4s_bytes(int T, int S) { return V4S_WARPS * v4s_warp_bytes(T, S); }

template <int E>
__global__ void __launch_bounds__(V4S_WARPS * 32, 1) k_spread_v4(InterpGeom g, const float2* __restrict__ in,
                                                                 const int4* __restrict__ subs, int n_subs, int S,
                                                                 int* __restrict__ counter,
                                                                 float2* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int T = E - 5;
  constexpr int E3 = E * E * E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nT = g.nT, K = g.K;
  unsigned char* wb = smem_raw + warp * v4s_warp_bytes(T, S);
  float2* tile = (float2*)wb;
  int* order = (int*)(tile + E3);
  int* p_off = order + S;
  int* ncls = p_off + S;   // [32] counts
  int* cur = ncls + 32;    // [32] cursors
  for (int i = lane; i < E3; i += 32) tile[i] = make_float2(0.f, 0.f);
  __syncwarp();
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    const int cnt = sp.z;
    ncls[lane] = 0;
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const uint2 ent = g.sorted[sp.y + i];
      int w0[3];
      float f[3];
      decode_point<6>(g, ent.x, w0, f);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      int off = -1;
      if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
        off = (lz * E + ly) * E + lx;
        atomicAdd(&ncls[off & 31], 1);
      } else {
        atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      }
      p_off[i] = off;
    }
    __syncwarp();
    const int my_n = ncls[lane];
    int incl = my_n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int my_start = incl - my_n;
    int rounds = my_n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(0xffffffffu, rounds, o));
    cur[lane] = my_start;
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const int off = p_off[i];
      if (off >= 0) order[atomicAdd(&cur[off & 31], 1)] = i;
    }
    __syncwarp();
    for (int r = 0; r < rounds; ++r) {
      const bool act = r < my_n;
      int off = 0;
      float2 cx[6], vyz[6][6];
      if (act) {
        const int i = order[my_start + r];
        const uint2 ent = g.sorted[sp.y + i];
        int w0[3];
        float f[3];
        decode_point<6>(g, ent.x, w0, f);
        off = p_off[i];
        float2 v = in[ent.x];
        if (ent.y != kNoTwin) v = cadd(v, in[ent.y]);
        float2 cy[6], cz[6];
        table_coeffs_v4<6>(g.table, g.L, f[0], cx);
        table_coeffs_v4<6>(g.table, g.L, f[1], cy);
        table_coeffs_v4<6>(g.table, g.L, f[2], cz);
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) {
          const float2 vz = cmulc(v, cz[jz]);
#pragma unroll
          for (int jy = 0; jy < 6; ++jy) vyz[jy][jz] = cmulc(vz, cy[jy]);
        }
      }
      float2* base = tile + off;
#define NUFFT_SPREAD_TAP(jx, jy, jz, end)                                               \
  if (act) {                                                                            \
    float2* q = base + ((jx) + E * (jy) + E * E * (jz));                                \
    float2 t = *q;                                                                      \
    t.x = fmaf(vyz[jy][jz].x, cx[jx].x, fmaf(vyz[jy][jz].y, cx[jx].y, t.x));            \
    t.y = fmaf(vyz[jy][jz].y, cx[jx].x, fmaf(-vyz[jy][jz].x, cx[jx].y, t.y));           \
    *q = t;                                                                             \
  }                                                                                     \
  if (end) __syncwarp();
      if constexpr (E == 13) {
        NUFFT_SPREAD_TAPS_E13(NUFFT_SPREAD_TAP)
      } else {
        NUFFT_SPREAD_TAPS_E21(NUFFT_SPREAD_TAP)
      }
#undef NUFFT_SPREAD_TAP
    }
    __syncwarp();
    for (int idx = lane; idx < E3; idx += 32) {
      const float2 v = tile[idx];
      if (v.x == 0.f && v.y == 0.f) continue;
      tile[idx] = make_float2(0.f, 0.f);
      const int ix = idx % E;
      const int t = idx / E;
      const int iy = t % E, iz = t / E;
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      atomicAdd(&grid[((size_t)gz * K + gy) * K + gx], v);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// variant 3 (gather, any J): one thread per point, with the points of a
// subproblem reordered so that the 16 lanes of every half-warp hold points
// whose first-tap offsets in the unpadded tile differ modulo 16 float2.  All
// lanes then add the same tap offset, so every tap load of the warp touches 16
// distinct bank pairs per half-warp (one wavefront), while the arithmetic
// stays at one thread per point (no cross-lane reduction, no shared
// coefficient buffers).
//
// Order: points are counted per residue class c = off mod 16; the point of
// rank r in class c goes to position sum_c' min(n_c', r) + #{c' < c : n_c' > r}
// (round robin over the classes that still have points).
// ---------------------------------------------------------------------------
constexpr int V3_THREADS = 256;

struct V3Layout {
  int E;
  size_t tile_bytes, bytes;
};

// elem: bytes per grid cell in shared memory (8 for complex64, 4 for bf16/fp16 pairs)
__host__ __device__ inline V3Layout v3_layout(int T, int J, int S, int elem) {
  V3Layout l;
  l.E = T + J - 1;
  l.tile_bytes = ((size_t)l.E * l.E * l.E * elem + 15) / 16 * 16;
  // per point: id, twin, tile offset, f[3] (6 words) + ordered index (1 word); class counts and cursors
  l.bytes = l.tile_bytes + (size_t)S * 7 * sizeof(int) + 64 * sizeof(int);
  return l;
}

template <int J, typename G>
__global__ void __launch_bounds__(V3_THREADS) k_gather_v3(InterpGeom g, const typename G::T* __restrict__ grid,
                                                          float inv_scale, const int4* __restrict__ subs, int S,
                                                          float2* __restrict__ out) {
  typedef typename G::T TT;
  // a warp access of 4-byte cells is conflict-free with 32 distinct residues,
  // of 8-byte cells with 16 distinct residues per half-warp
  constexpr int kRes = sizeof(TT) == 4 ? 32 : 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  inv_scale = lp_inv_scale<G>(g);
  const int T = g.T, nT = g.nT, K = g.K;
  const V3Layout lay = v3_layout(T, J, S, (int)sizeof(TT));
  const int E = lay.E, PP = E * E;
  TT* tile = (TT*)smem_raw;
  int* p_id = (int*)(smem_raw + lay.tile_bytes);
  int* p_tw = p_id + S;
  int* p_off = p_tw + S;
  float* p_f = (float*)(p_off + S);  // [3][S]
  int* order = (int*)(p_f + 3 * S);
  int* ncls = order + S;             // [kRes] counts, [kRes] cursors
  const int4 sp = subs[blockIdx.x];
  const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
  const int x0 = bx * T, y0 = by * T, z0 = bz * T;
  const int cnt = sp.z;
  if (threadIdx.x < 2 * kRes) ncls[threadIdx.x] = 0;
  {
    const int n = E * E * E;
    for (int idx = threadIdx.x; idx < n; idx += V3_THREADS) {
      const int ix = idx % E;
      const int t = idx / E;
      const int iy = t % E, iz = t / E;
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      tile[idx] = grid[((size_t)gz * K + gy) * K + gx];
    }
  }
  __syncthreads();
  // decode every point of the subproblem once
  for (int i = threadIdx.x; i < cnt; i += V3_THREADS) {
    const uint2 ent = g.sorted[sp.y + i];
    const uint32_t id = ent.x;
    int w0[3];
    float f[3];
    decode_point<J>(g, id, w0, f);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    int off = -1;
    if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
      off = (lz * E + ly) * E + lx;
    } else {
      atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
    }
    p_id[i] = (int)id;
    p_tw[i] = (int)ent.y;
    p_off[i] = off;
    p_f[i] = f[0];
    p_f[S + i] = f[1];
    p_f[2 * S + i] = f[2];
    atomicAdd(&ncls[off < 0 ? 0 : (off & (kRes - 1))], 1);
  }
  __syncthreads();
  // rank within the class, then the round-robin position
  for (int i = threadIdx.x; i < cnt; i += V3_THREADS) {
    const int c = p_off[i] < 0 ? 0 : (p_off[i] & (kRes - 1));
    const int r = atomicAdd(&ncls[kRes + c], 1);
    int pos = 0;
#pragma unroll
    for (int q = 0; q < kRes; ++q) {
      const int n = ncls[q];
      pos += n < r ? n : r;
      pos += (q < c && n > r) ? 1 : 0;
    }
    order[pos] = i;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < cnt; k += V3_THREADS) {
    const int i = order[k];
    const int off = p_off[i];
    if (off < 0) continue;
    float2 cx[J], cy[J], cz[J];
    table_coeffs_v4<J>(g.table, g.L, p_f[i], cx);
    table_coeffs_v4<J>(g.table, g.L, p_f[S + i], cy);
    table_coeffs_v4<J>(g.table, g.L, p_f[2 * S + i], cz);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int jz = 0; jz < J; ++jz) {
      float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
      for (int jy = 0; jy < J; ++jy) {
        const TT* tp = tile + off + jz * PP + jy * E;
        float2 row = make_float2(0.f, 0.f);
#pragma unroll
        for (int jx = 0; jx < J; ++jx) cmac(row, cx[jx], G::to_f2(tp[jx]));
        cmac(zacc, cy[jy], row);
      }
      cmac(acc, cz[jz], zacc);
    }
    const float2 res = cscale(acc, inv_scale);
    out[p_id[i]] = res;
    if ((uint32_t)p_tw[i] != kNoTwin) out[p_tw[i]] = res;
  }
}

// ---------------------------------------------------------------------------
// variant 4 (gather, any J): variant 3 with the coefficient table in shared
// memory.  One persistent CTA per SM holds the table once and runs
// V4_GROUPS independent groups of 256 threads; each group takes whole
// subproblems from a device work counter and synchronises on its own named
// barrier.  Table reads become shared-memory loads instead of L1 tag lookups.
// ---------------------------------------------------------------------------
constexpr int V4_GROUPS = 4;
constexpr int V4_GT = 256;  // threads per group

__host__ __device__ inline size_t v4_group_bytes(int T, int J, int S, int elem) {
  return (v3_layout(T, J, S, elem).bytes + 16 + 15) / 16 * 16;
}

__host__ __device__ inline size_t v4_bytes(int T, int J, int S, int L, int elem) {
  const size_t table = ((size_t)(L + 1) * J * sizeof(float2) + 15) / 16 * 16;
  return table + V4_GROUPS * v4_group_bytes(T, J, S, elem);
}

__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(V4_GT) : "memory");
}

template <int J>
__device__ __forceinline__ void smem_table_coeffs(const float2* table, int L, float f, float2 (&c)[J]) {
  float fl = f * (float)L;
  int i = (int)fl;
  if (i > L - 1) i = L - 1;
  const float t = fl - (float)i;
  const float4* r = (const float4*)(table + (size_t)i * J);
  float4 v[J];
#pragma unroll
  for (int q = 0; q < J; ++q) v[q] = r[q];
#pragma unroll
  for (int q = 0; q < J / 2; ++q) {
    const float4 a = v[q], b = v[q + J / 2];
    c[2 * q] = make_float2(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y));
    c[2 * q + 1] = make_float2(fmaf(t, b.z - a.z, a.z), fmaf(t, b.w - a.w, a.w));
  }
}

template <int J, typename G>
__global__ void __launch_bounds__(V4_GROUPS * V4_GT, 1) k_gather_v4(InterpGeom g, const typename G::T* __restrict__ grid,
                                                                   const int4* __restrict__ subs, int n_subs, int S,
                                                                   int* __restrict__ counter, float2* __restrict__ out) {
  typedef typename G::T TT;
  constexpr int kRes = sizeof(TT) == 4 ? 32 : 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const float inv_scale = lp_inv_scale<G>(g);
  const int T = g.T, nT = g.nT, K = g.K;
  const V3Layout lay = v3_layout(T, J, S, (int)sizeof(TT));
  const int E = lay.E, PP = E * E;
  float2* table = (float2*)smem_raw;
  const size_t table_bytes = ((size_t)(g.L + 1) * J * sizeof(float2) + 15) / 16 * 16;
  for (int i = threadIdx.x; i < (g.L + 1) * J; i += blockDim.x) table[i] = __ldg(g.table + i);
  __syncthreads();
  const int grp = threadIdx.x / V4_GT, tid = threadIdx.x % V4_GT;
  unsigned char* gb = smem_raw + table_bytes + grp * v4_group_bytes(T, J, S, (int)sizeof(TT));
  TT* tile = (TT*)gb;
  int* p_id = (int*)(gb + lay.tile_bytes);
  int* p_tw = p_id + S;
  int* p_off = p_tw + S;
  float* p_f = (float*)(p_off + S);
  int* order = (int*)(p_f + 3 * S);
  int* ncls = order + S;
  int* work = ncls + 64;
  for (;;) {
    if (tid == 0) *work = atomicAdd(counter, 1);
    if (tid < 2 * kRes) ncls[tid] = 0;
    group_sync(grp);
    const int s = *work;
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    const int cnt = sp.z;
    {
      const int n = E * E * E;
      for (int idx = tid; idx < n; idx += V4_GT) {
        const int ix = idx % E;
        const int t = idx / E;
        const int iy = t % E, iz = t / E;
        int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
        gx -= gx >= K ? K : 0;
        gy -= gy >= K ? K : 0;
        gz -= gz >= K ? K : 0;
        tile[idx] = grid[((size_t)gz * K + gy) * K + gx];
      }
    }
    for (int i = tid; i < cnt; i += V4_GT) {
      const uint2 ent = g.sorted[sp.y + i];
      const uint32_t id = ent.x;
      int w0[3];
      float f[3];
      decode_point<J>(g, id, w0, f);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      int off = -1;
      if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
        off = (lz * E + ly) * E + lx;
      } else {
        atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      }
      p_id[i] = (int)id;
      p_tw[i] = (int)ent.y;
      p_off[i] = off;
      p_f[i] = f[0];
      p_f[S + i] = f[1];
      p_f[2 * S + i] = f[2];
      atomicAdd(&ncls[off < 0 ? 0 : (off & (kRes - 1))], 1);
    }
    group_sync(grp);
    for (int i = tid; i < cnt; i += V4_GT) {
      const int c = p_off[i] < 0 ? 0 : (p_off[i] & (kRes - 1));
      const int r = atomicAdd(&ncls[kRes + c], 1);
      int pos = 0;
#pragma unroll
      for (int q = 0; q < kRes; ++q) {
        const int n = ncls[q];
        pos += n < r ? n : r;
        pos += (q < c && n > r) ? 1 : 0;
      }
      order[pos] = i;
    }
    group_sync(grp);
    for (int k = tid; k < cnt; k += V4_GT) {
      const int i = order[k];
      const int off = p_off[i];
      if (off < 0) continue;
      float2 cx[J], cy[J], cz[J];
      smem_table_coeffs<J>(table, g.L, p_f[i], cx);
      smem_table_coeffs<J>(table, g.L, p_f[S + i], cy);
      smem_table_coeffs<J>(table, g.L, p_f[2 * S + i], cz);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int jz = 0; jz < J; ++jz) {
        float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int jy = 0; jy < J; ++jy) {
          const TT* tp = tile + off + jz * PP + jy * E;
          float2 row = make_float2(0.f, 0.f);
#pragma unroll
          for (int jx = 0; jx < J; ++jx) cmac(row, cx[jx], G::to_f2(tp[jx]));
          cmac(zacc, cy[jy], row);
        }
        cmac(acc, cz[jz], zacc);
      }
      const float2 res = cscale(acc, inv_scale);
      out[p_id[i]] = res;
      if ((uint32_t)p_tw[i] != kNoTwin) out[p_tw[i]] = res;
    }
    group_sync(grp);
  }
}

template <int J, typename G>
static cudaError_t launch_gather_v4_t(const InterpGeom& g, const void* grid, const int4* subs, int n_subs, int S,
                                      float2* out, cudaStream_t st) {
  auto f = k_gather_v4<J, G>;
  const size_t smem = v4_bytes(g.T, J, S, g.L, (int)sizeof(typename G::T));
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  e = cudaMemsetAsync(g.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  f<<<num_sms(), V4_GROUPS * V4_GT, smem, st>>>(g, (const typename G::T*)grid, subs, n_subs, S, g.counter, out);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v4_j(const InterpGeom& g, int dtype, const void* grid, const int4* subs, int n_subs,
                                      int S, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v4_t<J, GridC64>(g, grid, subs, n_subs, S, out, st);
    case 1: return launch_gather_v4_t<J, GridBF16>(g, grid, subs, n_subs, S, out, st);
    case 2: return launch_gather_v4_t<J, GridF16>(g, grid, subs, n_subs, S, out, st);
  }
  return cudaErrorInvalidValue;
}

template <int J, typename G>
static cudaError_t launch_gather_v3_t(const InterpGeom& g, const void* grid, float inv_scale, const int4* subs,
                                      int n_subs, int S, float2* out, cudaStream_t st) {
  auto f = k_gather_v3<J, G>;
  const size_t smem = v3_layout(g.T, J, S, (int)sizeof(typename G::T)).bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  f<<<n_subs, V3_THREADS, smem, st>>>(g, (const typename G::T*)grid, inv_scale, subs, S, out);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v3_j(const InterpGeom& g, int dtype, const void* grid, float inv_scale,
                                      const int4* subs, int n_subs, int S, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v3_t<J, GridC64>(g, grid, inv_scale, subs, n_subs, S, out, st);
    case 1: return launch_gather_v3_t<J, GridBF16>(g, grid, inv_scale, subs, n_subs, S, out, st);
    case 2: return launch_gather_v3_t<J, GridF16>(g, grid, inv_scale, subs, n_subs, S, out, st);
  }
  return cudaErrorInvalidValue;
}


static int max_optin_smem() {
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return maxsm;
}

bool v4s_supported(int T, int J, int S) {
  return J == 6 && T == 8 && v4s_bytes(T, S) <= (size_t)max_optin_smem();
}

bool v3s_supported(int T, int J) {
  return J == 6 && T == 8 && v3s_bytes(T) <= (size_t)max_optin_smem();
}

bool v4_supported(int T, int J, int S, int L) {
  return v4_bytes(T, J, S, L, 8) <= (size_t)max_optin_smem();
}

bool v3_supported(int T, int J, int S) {
  return v3_layout(T, J, S, 8).bytes <= (size_t)max_optin_smem();
}

bool v2_supported(int T, int J, int L) {
  return J == 6 && (T == 8 || T == 16) && v2_layout(T, L).bytes <= (size_t)max_optin_smem();
}

static bool v1_fits(const InterpGeom& g) {
  if (g.J != 6) return false;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v1_layout(g.T, g.L).bytes <= (size_t)maxsm;
}

template <typename G>
static cudaError_t launch_gather_v1_t(const InterpGeom& g, const void* grid, float inv_scale, const int4* subs,
                                      int n_subs, float2* out, cudaStream_t st) {
  auto f = k_gather_v1<G>;
  const size_t smem = v1_layout(g.T, g.L).bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  const int grid_x = n_subs < num_sms() ? n_subs : num_sms();
  f<<<grid_x, V1_THREADS, smem, st>>>(g, (const typename G::T*)grid, inv_scale, subs, n_subs, out);
  return cudaGetLastError();
}

static cudaError_t launch_spread_v1(const InterpGeom& g, const float2* in, const int4* subs, int n_subs,
                                    float2* grid, cudaStream_t st) {
  auto f = k_spread_v1;
  const size_t smem = v1_layout(g.T, g.L).bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  const int grid_x = n_subs < num_sms() ? n_subs : num_sms();
  f<<<grid_x, V1_THREADS, smem, st>>>(g, in, subs, n_subs, grid);
  return cudaGetLastError();
}

size_t interp_smem_bytes(int T, int J) {
  const size_t E = (size_t)T + J - 1;
  return E * E * E * sizeof(float2);
}

template <int J, typename G>
static cudaError_t launch_gather_v0_t(const InterpGeom& g, const void* grid, float inv_scale, const int4* subs,
                                      int n_subs, float2* out, cudaStream_t st) {
  auto f = k_gather_v0<J, G>;
  const size_t smem = interp_smem_bytes(g.T, J);
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  f<<<n_subs, 256, smem, st>>>(g, (const typename G::T*)grid, inv_scale, subs, out);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v0_j(const InterpGeom& g, int dtype, const void* grid, float inv_scale,
                                      const int4* subs, int n_subs, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v0_t<J, GridC64>(g, grid, inv_scale, subs, n_subs, out, st);
    case 1: return launch_gather_v0_t<J, GridBF16>(g, grid, inv_scale, subs, n_subs, out, st);
    case 2: return launch_gather_v0_t<J, GridF16>(g, grid, inv_scale, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

template <typename G>
static cudaError_t launch_gather_v2_t(const InterpGeom& g, const void* grid, float inv_scale, const int4* subs,
                                      int n_subs, int* counter, float2* out, cudaStream_t st) {
  auto f = k_gather_v2<G>;
  const size_t smem = v2_layout(g.T, g.L).bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  f<<<num_sms(), V2_WARPS * 32, smem, st>>>(g, (const typename G::T*)grid, inv_scale, subs, n_subs, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const InterpGeom& g, int variant, int grid_dtype, const void* grid, float inv_scale,
                          const int4* subs, int n_subs, float2* out, cudaStream_t st) {
  if (variant == 4) {
    switch (g.J) {
      case 2: return launch_gather_v4_j<2>(g, grid_dtype, grid, subs, n_subs, g.S, out, st);
      case 4: return launch_gather_v4_j<4>(g, grid_dtype, grid, subs, n_subs, g.S, out, st);
      case 6: return launch_gather_v4_j<6>(g, grid_dtype, grid, subs, n_subs, g.S, out, st);
      case 8: return launch_gather_v4_j<8>(g, grid_dtype, grid, subs, n_subs, g.S, out, st);
    }
    return cudaErrorInvalidValue;
  }
  if (variant == 3) {
    switch (g.J) {
      case 2: return launch_gather_v3_j<2>(g, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 4: return launch_gather_v3_j<4>(g, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 6: return launch_gather_v3_j<6>(g, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 8: return launch_gather_v3_j<8>(g, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
    }
    return cudaErrorInvalidValue;
  }
  if (variant == 2 && v2_supported(g.T, g.J, g.L)) {
    switch (grid_dtype) {
      case 0: return launch_gather_v2_t<GridC64>(g, grid, inv_scale, subs, n_subs, g.counter, out, st);
      case 1: return launch_gather_v2_t<GridBF16>(g, grid, inv_scale, subs, n_subs, g.counter, out, st);
      case 2: return launch_gather_v2_t<GridF16>(g, grid, inv_scale, subs, n_subs, g.counter, out, st);
    }
    return cudaErrorInvalidValue;
  }
  if (variant == 1 && v1_fits(g)) {
    switch (grid_dtype) {
      case 0: return launch_gather_v1_t<GridC64>(g, grid, inv_scale, subs, n_subs, out, st);
      case 1: return launch_gather_v1_t<GridBF16>(g, grid, inv_scale, subs, n_subs, out, st);
      case 2: return launch_gather_v1_t<GridF16>(g, grid, inv_scale, subs, n_subs, out, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (g.J) {
    case 2: return launch_gather_v0_j<2>(g, grid_dtype, grid, inv_scale, subs, n_subs, out, st);
    case 4: return launch_gather_v0_j<4>(g, grid_dtype, grid, inv_scale, subs, n_subs, out, st);
    case 6: return launch_gather_v0_j<6>(g, grid_dtype, grid, inv_scale, subs, n_subs, out, st);
    case 8: return launch_gather_v0_j<8>(g, grid_dtype, grid, inv_scale, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

template <int J>
static cudaError_t launch_spread_v0_t(const InterpGeom& g, const float2* in, const int4* subs, int n_subs,
                                      float2* grid, cudaStream_t st) {
  auto f = k_spread_v0<J>;
  const size_t smem = interp_smem_bytes(g.T, J);
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  f<<<n_subs, 256, smem, st>>>(g, in, subs, grid);
  return cudaGetLastError();
}

cudaError_t launch_spread(const InterpGeom& g, int variant, const float2* in, const int4* subs, int n_subs,
                          float2* grid, cudaStream_t st) {
  if (variant == 4 && v4s_supported(g.T, g.J, g.S)) {
    auto f = k_spread_v4<13>;
    const size_t smem = v4s_bytes(g.T, g.S);
    cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_subs == 0) return cudaSuccess;
    e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    f<<<num_sms(), V4S_WARPS * 32, smem, st>>>(g, in, subs, n_subs, g.S, g.counter + 1, grid);
    return cudaGetLastError();
  }
  if (variant == 3 && v3s_supported(g.T, g.J)) {
    auto f = k_spread_v3<8>;
    const size_t smem = v3s_bytes(g.T);
    cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_subs == 0) return cudaSuccess;
    e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    f<<<num_sms(), V3S_WARPS * 32, smem, st>>>(g, in, subs, n_subs, g.counter + 1, grid);
    return cudaGetLastError();
  }
  if (variant == 2 && v2_supported(g.T, g.J, g.L)) {
    auto f = k_spread_v2;
    const size_t smem = v2_layout(g.T, g.L).bytes;
    cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_subs == 0) return cudaSuccess;
    e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    f<<<num_sms(), V2_WARPS * 32, smem, st>>>(g, in, subs, n_subs, g.counter + 1, grid);
    return cudaGetLastError();
  }
  if (variant == 1 && v1_fits(g)) return launch_spread_v1(g, in, subs, n_subs, grid, st);
  switch (g.J) {
    case 2: return launch_spread_v0_t<2>(g, in, subs, n_subs, grid, st);
    case 4: return launch_spread_v0_t<4>(g, in, subs, n_subs, grid, st);
    case 6: return launch_spread_v0_t<6>(g, in, subs, n_subs, grid, st);
    case 8: return launch_spread_v0_t<8>(g, in, subs, n_subs, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nufft
