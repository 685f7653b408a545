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

template <int J>
__global__ void k_bin_points(InterpGeom g, long long P, uint32_t* __restrict__ bins) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    int w0[3];
    float f[3];
    decode_point<J>(g, (uint32_t)p, w0, f);
    bins[p] = (uint32_t)(((w0[2] / g.T) * g.nT + w0[1] / g.T) * g.nT + w0[0] / g.T);
  }
}

template <int J>
static cudaError_t launch_bin_t(const InterpGeom& g, uint32_t* bins, cudaStream_t st) {
  const long long P = (long long)g.D * g.M;
  long long blocks = (P + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_bin_points<J><<<(unsigned)blocks, 256, 0, st>>>(g, P, bins);
  return cudaGetLastError();
}

cudaError_t launch_bin_points(const InterpGeom& g, uint32_t* bins, cudaStream_t st) {
  switch (g.J) {
    case 2: return launch_bin_t<2>(g, bins, st);
    case 4: return launch_bin_t<4>(g, bins, st);
    case 6: return launch_bin_t<6>(g, bins, st);
    case 8: return launch_bin_t<8>(g, bins, st);
  }
  return cudaErrorInvalidValue;
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
  extern __shared__ float2 tile[];
  const int4 sp = subs[blockIdx.x];
  const int T = g.T, nT = g.nT, E = T + J - 1;
  const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
  const int x0 = bx * T, y0 = by * T, z0 = bz * T;
  stage_tile_plain<G>(grid, inv_scale, g.K, E, x0, y0, z0, tile);
  __syncthreads();
  for (int i = threadIdx.x; i < sp.z; i += blockDim.x) {
    const uint32_t id = g.sorted[sp.y + i];
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
    const uint32_t id = g.sorted[sp.y + i];
    int w0[3];
    float f[3];
    decode_point<J>(g, id, w0, f);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
      atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      continue;
    }
    const float2 v = in[id];
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

cudaError_t launch_gather(const InterpGeom& g, int variant, int grid_dtype, const void* grid, float inv_scale,
                          const int4* subs, int n_subs, float2* out, cudaStream_t st) {
  (void)variant;
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
  (void)variant;
  switch (g.J) {
    case 2: return launch_spread_v0_t<2>(g, in, subs, n_subs, grid, st);
    case 4: return launch_spread_v0_t<4>(g, in, subs, n_subs, grid, st);
    case 6: return launch_spread_v0_t<6>(g, in, subs, n_subs, grid, st);
    case 8: return launch_spread_v0_t<8>(g, in, subs, n_subs, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nufft
