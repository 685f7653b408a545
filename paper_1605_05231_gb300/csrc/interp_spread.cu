// Spread kernels (points -> grid, the transpose of the gather) and the
// point binning used at plan time.  Shared helpers are in interp_common.cuh.
#include "interp_common.cuh"
#include "spread_taps.inc"

namespace nufft {

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

// ---------------------------------------------------------------------------
// variant 0: one thread per point
// ---------------------------------------------------------------------------
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
    point_coeffs<J>(g, f[0], cx);
    point_coeffs<J>(g, f[1], cy);
    point_coeffs<J>(g, f[2], cz);
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
// phase 1 folds the point's value into its z coefficients (v conj(cz)) so that
// phase 2 reads only the tile offset besides the coefficients, and the
// coefficients of the next point are loaded into registers while the current
// point's read-modify-writes drain.
// ---------------------------------------------------------------------------
constexpr int V3S_WARPS = 10;

__host__ __device__ inline size_t v3s_warp_bytes(int T) {
  const int E = T + 5;
  const size_t w = (size_t)32 * V2_CSTRIDE * sizeof(float2) + 32 * sizeof(int) +
                   (size_t)E * E * E * sizeof(float2);
  return (w + 15) / 16 * 16;
}

__host__ __device__ inline size_t v3s_bytes(int T) { return V3S_WARPS * v3s_warp_bytes(T); }

struct V3SCoef {
  float2 cx, cy, ox, oy;
  float4 z01, z23, z45;  // v conj(cz[0..5])
  int mo;                // tile offset, or -1
};

__device__ __forceinline__ void v3s_load(const float2* coef, const int* mos, int p, const V2Lanes& ln,
                                         V3SCoef& c) {
  const float2* cp = coef + p * V2_CSTRIDE;
  c.mo = mos[p];
  c.cx = cp[ln.mjx];
  c.cy = cp[6 + ln.mjy];
  c.z01 = *(const float4*)(cp + 12);
  c.z23 = *(const float4*)(cp + 14);
  c.z45 = *(const float4*)(cp + 16);
  c.ox = cp[ln.ojx];
  c.oy = cp[6 + ln.ojy];
}

// read-modify-write of one point's taps held by this lane
template <int PP>
__device__ __forceinline__ void v3s_apply(float2* tile, const V3SCoef& c, const V2Lanes& ln, int lane) {
  if (c.mo < 0) return;
  // contribution conj(cx cy) (v conj(cz)) = v conj(cx cy cz)
  const float2 p = cmul(c.cx, c.cy);
  float2* tp = tile + c.mo + ln.main_off;
  float2 t[6];
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) t[jz] = tp[jz * PP];
  const float2 zv[6] = {make_float2(c.z01.x, c.z01.y), make_float2(c.z01.z, c.z01.w),
                        make_float2(c.z23.x, c.z23.y), make_float2(c.z23.z, c.z23.w),
                        make_float2(c.z45.x, c.z45.y), make_float2(c.z45.z, c.z45.w)};
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) {
    t[jz].x = fmaf(p.x, zv[jz].x, fmaf(p.y, zv[jz].y, t[jz].x));
    t[jz].y = fmaf(p.x, zv[jz].y, fmaf(-p.y, zv[jz].x, t[jz].y));
  }
#pragma unroll
  for (int jz = 0; jz < 6; ++jz) tp[jz * PP] = t[jz];
  if (lane < 24) {
    // the lane's overflow tap takes v conj(cz) of its own jz (a register select)
    float2 z = zv[0];
#pragma unroll
    for (int jz = 1; jz < 6; ++jz) z = ln.ojz == jz ? zv[jz] : z;
    const float2 q = cmul(c.ox, c.oy);
    float2* r = tile + c.mo + ln.ovf_off;
    float2 u = *r;
    u.x = fmaf(q.x, z.x, fmaf(q.y, z.y, u.x));
    u.y = fmaf(q.x, z.y, fmaf(-q.y, z.x, u.y));
    *r = u;
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
  int* mos = (int*)(coef + 32 * V2_CSTRIDE);
  float2* tile = (float2*)(mos + 32);
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
            point_coeffs<6>(g, f[a], c);
            if (a == 2) {
#pragma unroll
              for (int q = 0; q < 6; ++q) c[q] = cmulc(val, c[q]);  // v conj(cz)
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) c4[a * 3 + q] = make_float4(c[2 * q].x, c[2 * q].y, c[2 * q + 1].x, c[2 * q + 1].y);
          }
        } else {
          atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
        }
      }
      mos[lane] = off;
      __syncwarp();
      const int np = min(32, sp.z - b0);
      // two points per iteration: the second point's coefficients load while
      // the first point's read-modify-writes drain
      int p = 0;
      for (; p + 1 < np; p += 2) {
        V3SCoef c0, c1;
        v3s_load(coef, mos, p, ln, c0);
        v3s_load(coef, mos, p + 1, ln, c1);
        v3s_apply<PP>(tile, c0, ln, lane);
        __syncwarp();
        v3s_apply<PP>(tile, c1, ln, lane);
        __syncwarp();
      }
      if (p < np) {
        V3SCoef c0;
        v3s_load(coef, mos, p, ln, c0);
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
// spread variant 5 (J = 6, T = 8): variant 3 with the warp's tile accumulated
// in 32-bit fixed point.  A shared-memory integer add is a native reduction of
// one wavefront per 32 lanes, where a floating-point cell update is a 64-bit
// load plus a 64-bit store; the tile is kept as separate real and imaginary
// int32 planes.
//
// Scale: while a subproblem is spread, its tile carries an exponent e with
// 2^e >= |v| max|cx| max|cy| max|cz| for every point added so far, and counts
// contributions in units of 2^e / B, B = 2^min(22, 30 - ceil(log2 S)) (1 - 2^-10).
// Every contribution is then below 2^22 units, and no cell of a subproblem of
// at most S points (one contribution per point and cell) reaches 2^30.  When a
// batch of 32 points raises e, the tile is rescaled by a rounding right shift.
// Rounding: adding 1.5 * 2^23 puts x in [2^23, 2^24), where floats are spaced
// by 1, so the FMA that adds the constant rounds x to the nearest integer,
// which is read back from the float's bits.
// ---------------------------------------------------------------------------
constexpr int V5S_WARPS = 10;
// two int32 planes take the bytes of one float2 tile
__host__ __device__ inline size_t v5s_bytes(int T) { return V5S_WARPS * v3s_warp_bytes(T); }

// divide every cell by 2^d, rounding half up
__device__ __forceinline__ void v5s_rescale(int* tre, int* tim, int n, int d, int lane) {
  __syncwarp();
  if (d >= 31) {
    for (int i = lane; i < n; i += 32) {
      tre[i] = 0;
      tim[i] = 0;
    }
  } else {
    const int h = 1 << (d - 1);
    for (int i = lane; i < n; i += 32) {
      const int a = tre[i], b = tim[i];
      if (a) tre[i] = (a + h) >> d;
      if (b) tim[i] = (b + h) >> d;
    }
  }
  __syncwarp();
}

template <int T>
__global__ void __launch_bounds__(V5S_WARPS * 32, 1) k_spread_v5(InterpGeom g, const float2* __restrict__ in,
                                                                 const int4* __restrict__ subs, int n_subs,
                                                                 int* __restrict__ counter,
                                                                 float2* __restrict__ grid, float budget,
                                                                 float inv_budget) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E = T + 5, E2 = E * E, E3 = E2 * E;
  static_assert(E == 13, "lane tables are for E = 13");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nT = g.nT, K = g.K;
  const size_t KK = (size_t)K * K;
  float2* coef = (float2*)(smem_raw + warp * v3s_warp_bytes(T));
  int* mos = (int*)(coef + 32 * V2_CSTRIDE);
  int* tre = mos + 32;
  int* tim = tre + E3;
  for (int i = lane; i < E3; i += 32) {
    tre[i] = 0;
    tim[i] = 0;
  }
  __syncwarp();
  const V5Lanes ln = v5_lanes(lane);
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= n_subs) break;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    int e_tile = kTileEmpty;
    float scale = 0.f;
    bool poison = false;
    for (int b0 = 0; b0 < sp.z; b0 += 32) {
      // phase 1: one point per lane; the bound |v| max|cx| max|cy| max|cz|
      int off = -1;
      float bound = 0.f;
      const int pi = b0 + lane;
      if (pi < sp.z) {
        const uint2 ent = g.sorted[sp.y + pi];
        int w0[3];
        float f[3];
        decode_point<6>(g, ent.x, w0, f);
        const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
        if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
          off = (lz * E + ly) * E + lx;
          float2 val = in[ent.x];
          if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
          float4* c4 = (float4*)(coef + lane * V2_CSTRIDE);
          float m2 = 1.f;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float2 c[6];
            point_coeffs<6>(g, f[a], c);
            float mx = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) mx = fmaxf(mx, fmaf(c[q].x, c[q].x, c[q].y * c[q].y));
            m2 *= mx;
            if (a == 2) {
#pragma unroll
              for (int q = 0; q < 6; ++q) c[q] = cmulc(val, c[q]);  // v conj(cz)
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) c4[a * 3 + q] = make_float4(c[2 * q].x, c[2 * q].y, c[2 * q + 1].x, c[2 * q + 1].y);
          }
          bound = hypotf(val.x, val.y) * sqrtf(m2);
        } else {
          atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
        }
      }
      mos[lane] = off;
      // bounds are >= 0 (or NaN), so their bits order like the values
      const unsigned bb = __reduce_max_sync(0xffffffffu, __float_as_uint(bound));
      __syncwarp();
      if (bb > kBoundLimitBits) {
        poison = true;
      } else if (bb != 0u) {
        const int e = max((int)(bb >> 23) - 127 + ((bb & 0x7FFFFFu) ? 1 : 0), -100);
        if (e > e_tile) {
          if (e_tile != kTileEmpty) v5s_rescale(tre, tim, E3, e - e_tile, lane);
          e_tile = e;
          scale = budget * pow2f(-e);
        }
      }
      if (!poison && bb != 0u) {
        // phase 2: one point at a time for the whole warp
        const int np = min(32, sp.z - b0);
#pragma unroll 2
        for (int p = 0; p < np; ++p) {
          const int mo = mos[p];
          if (mo < 0) continue;
          const float2* cp = coef + p * V2_CSTRIDE;
          const float2 cx = cp[ln.mjx], cy = cp[6 + ln.mjy];
          const float4 z01 = *(const float4*)(cp + 12), z23 = *(const float4*)(cp + 14),
                       z45 = *(const float4*)(cp + 16);
          const float2 ox = cp[ln.ojx], oy = cp[6 + ln.ojy];
          const float2 zv[6] = {make_float2(z01.x, z01.y), make_float2(z01.z, z01.w),
                                make_float2(z23.x, z23.y), make_float2(z23.z, z23.w),
                                make_float2(z45.x, z45.y), make_float2(z45.z, z45.w)};
          // contribution conj(cx cy) (v conj(cz)), in units
          if (ln.has_main) {
            const float2 pm = cmul(cscale(cx, scale), cy);
            int* re = tre + mo + ln.main_off;
            int* im = tim + mo + ln.main_off;
#pragma unroll
            for (int jz = 0; jz < 6; ++jz) {
              atomicAdd(re + jz * E2, round_units(pm.x, zv[jz].x, pm.y, zv[jz].y));
              atomicAdd(im + jz * E2, round_units(pm.x, zv[jz].y, -pm.y, zv[jz].x));
            }
          }
          if (ln.has_ovf) {
            float2 z = zv[0];
#pragma unroll
            for (int jz = 1; jz < 6; ++jz) z = ln.ojz == jz ? zv[jz] : z;
            const float2 q = cmul(cscale(ox, scale), oy);
            atomicAdd(tre + mo + ln.ovf_off, round_units(q.x, z.x, q.y, z.y));
            atomicAdd(tim + mo + ln.ovf_off, round_units(q.x, z.y, -q.y, z.x));
          }
        }
      }
      __syncwarp();
    }
    // add the tile to the grid: lanes walk (y, x) columns, each column along z
    const float inv = e_tile == kTileEmpty ? 0.f : inv_budget * pow2f(e_tile);
    const float qnan = __int_as_float(0x7fc00000);
    for (int c = lane; c < E2; c += 32) {
      const int iy = c / E, ix = c - iy * E;
      int gx = x0 + ix, gy = y0 + iy;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      int gz = z0;
#pragma unroll
      for (int iz = 0; iz < E; ++iz) {
        const int idx = c + iz * E2;
        const int a = tre[idx], b = tim[idx];
        if ((a | b) != 0 || poison) {
          tre[idx] = 0;
          tim[idx] = 0;
          const float2 v = poison ? make_float2(qnan, qnan) : make_float2((float)a * inv, (float)b * inv);
          atomicAdd(&grid[((size_t)(gz >= K ? gz - K : gz)) * KK + (size_t)gy * K + gx], v);
        }
        ++gz;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// spread variant 6 (J = 6, T = 8, at most 256 points per subproblem): the
// fixed-point arithmetic of variant 5 with one tile per CTA.  Integer adds make
// the tile safe to share, so six warps spread one subproblem together and an
// SM holds four CTAs (24 warps) where the warp-private tiles allowed ten.
//  phase 1: thread per point (decode, coefficients, v folded into the z row,
//           the bound |v| max|cx| max|cy| max|cz|), then the CTA's largest
//           bound fixes the subproblem's exponent: no rescaling;
//  phase 2: warp w spreads points w, w + 6, ...; lanes without a tap of their
//           own add zero at a free bank, so no instruction is predicated;
//  flush:   all 192 threads add the tile to the grid and clear it, while the
//           next subproblem's phase 1 starts in the warps that are done.
// ---------------------------------------------------------------------------
constexpr int V6S_WARPS = 6, V6S_THREADS = V6S_WARPS * 32, V6S_MAX_PTS = 256;

struct V6SLayout {
  static constexpr int E = 13, E3 = E * E * E;
  static constexpr size_t coef = 0;                                                  // [256][18] float2
  static constexpr size_t mos = coef + (size_t)V6S_MAX_PTS * V2_CSTRIDE * sizeof(float2);  // [256] int
  static constexpr size_t tre = mos + V6S_MAX_PTS * sizeof(int);                      // [E3] int
  static constexpr size_t tim = tre + E3 * sizeof(int);                               // [E3] int
  static constexpr size_t wmax = tim + E3 * sizeof(int);                              // [6] unsigned
  static constexpr size_t nxt = wmax + V6S_WARPS * sizeof(unsigned);                  // [2] int
  static constexpr size_t bytes = (nxt + 2 * sizeof(int) + 15) / 16 * 16;
};

__global__ void __launch_bounds__(V6S_THREADS, 3) k_spread_v6(InterpGeom g, const float2* __restrict__ in,
                                                             const int4* __restrict__ subs, int n_subs,
                                                             int* __restrict__ counter,
                                                             float2* __restrict__ grid, float budget,
                                                             float inv_budget) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Lay = V6SLayout;
  constexpr int T = 8, E = Lay::E, E2 = E * E, E3 = Lay::E3;
  float2* coef = (float2*)(smem_raw + Lay::coef);
  int* mos = (int*)(smem_raw + Lay::mos);
  int* tre = (int*)(smem_raw + Lay::tre);
  int* tim = (int*)(smem_raw + Lay::tim);
  unsigned* wmax = (unsigned*)(smem_raw + Lay::wmax);
  int* nxt = (int*)(smem_raw + Lay::nxt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nT = g.nT, K = g.K;
  const size_t KK = (size_t)K * K;
  for (int i = tid; i < E3; i += V6S_THREADS) {
    tre[i] = 0;
    tim[i] = 0;
  }
  // lane taps: a (jx, jy) column for every jz, and one extra tap
  const V5Lanes ln = v5_lanes(lane);
  const int main_off = ln.has_main ? ln.main_off : kPadI13[0];
  const int ovf_off = ln.has_ovf ? ln.ovf_off : kPadI13[lane == 30 ? 1 : 2];
  const int ozo = 12 + ln.ojz;
  if (tid == 0) nxt[0] = atomicAdd(counter, 1);
  __syncthreads();
  int s = nxt[0], parity = 0;
  while (s < n_subs) {
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    // phase 1; bounds are >= 0 (or NaN), so their bits order like the values
    // (and a NaN wins, as it must)
    unsigned bound = 0u;
    for (int i = tid; i < sp.z; i += V6S_THREADS) {
      const uint2 ent = g.sorted[sp.y + i];
      int w0[3];
      float f[3];
      decode_point<6>(g, ent.x, w0, f);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      float4* c4 = (float4*)(coef + i * V2_CSTRIDE);
      int off = 0;
      if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
        off = (lz * E + ly) * E + lx;
        float2 val = in[ent.x];
        if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
        float m2 = 1.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float2 c[6];
          point_coeffs<6>(g, f[a], c);
          float mx = 0.f;
#pragma unroll
          for (int q = 0; q < 6; ++q) mx = fmaxf(mx, fmaf(c[q].x, c[q].x, c[q].y * c[q].y));
          m2 *= mx;
          if (a == 2) {
#pragma unroll
            for (int q = 0; q < 6; ++q) c[q] = cmulc(val, c[q]);  // v conj(cz)
          }
#pragma unroll
          for (int q = 0; q < 3; ++q) c4[a * 3 + q] = make_float4(c[2 * q].x, c[2 * q].y, c[2 * q + 1].x, c[2 * q + 1].y);
        }
        bound = max(bound, __float_as_uint(hypotf(val.x, val.y) * sqrtf(m2)));
      } else {
        // outside its tile (flagged): the point adds zero
        atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
#pragma unroll
        for (int q = 0; q < 9; ++q) c4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      mos[i] = off;
    }
    const unsigned wb = __reduce_max_sync(0xffffffffu, bound);
    if (lane == 0) wmax[warp] = wb;
    if (tid == 0) nxt[parity ^ 1] = atomicAdd(counter, 1);
    __syncthreads();
    unsigned bb = wmax[0];
#pragma unroll
    for (int w = 1; w < V6S_WARPS; ++w) bb = max(bb, wmax[w]);
    const bool poison = bb > kBoundLimitBits;
    int e_tile = kTileEmpty;
    if (!poison && bb != 0u) {
      e_tile = max((int)(bb >> 23) - 127 + ((bb & 0x7FFFFFu) ? 1 : 0), -100);
      const float sc = budget * pow2f(-e_tile);
      const float sm = ln.has_main ? sc : 0.f, so = ln.has_ovf ? sc : 0.f;
      // phase 2: contribution conj(cx cy) (v conj(cz)), in units
      for (int p = warp; p < sp.z; p += V6S_WARPS) {
        const int mo = mos[p];
        const float2* cp = coef + p * V2_CSTRIDE;
        const float2 cx = cp[ln.mjx], cy = cp[6 + ln.mjy];
        const float4 z01 = *(const float4*)(cp + 12), z23 = *(const float4*)(cp + 14),
                     z45 = *(const float4*)(cp + 16);
        const float2 ox = cp[ln.ojx], oy = cp[6 + ln.ojy], zo = cp[ozo];
        const float2 zv[6] = {make_float2(z01.x, z01.y), make_float2(z01.z, z01.w),
                              make_float2(z23.x, z23.y), make_float2(z23.z, z23.w),
                              make_float2(z45.x, z45.y), make_float2(z45.z, z45.w)};
        const float2 pm = cmul(cscale(cx, sm), cy);
        int* re = tre + mo + main_off;
        int* im = tim + mo + main_off;
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) {
          atomicAdd(re + jz * E2, round_units(pm.x, zv[jz].x, pm.y, zv[jz].y));
          atomicAdd(im + jz * E2, round_units(pm.x, zv[jz].y, -pm.y, zv[jz].x));
        }
        const float2 q = cmul(cscale(ox, so), oy);
        atomicAdd(tre + mo + ovf_off, round_units(q.x, zo.x, q.y, zo.y));
        atomicAdd(tim + mo + ovf_off, round_units(q.x, zo.y, -q.y, zo.x));
      }
    }
    __syncthreads();
    const int s_next = nxt[parity ^ 1];
    // flush: threads walk (y, x) columns, each column along z
    const float inv = e_tile == kTileEmpty ? 0.f : inv_budget * pow2f(e_tile);
    const float qnan = __int_as_float(0x7fc00000);
    for (int c = tid; c < E2; c += V6S_THREADS) {
      const int iy = c / E, ix = c - iy * E;
      int gx = x0 + ix, gy = y0 + iy;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      float2* col = grid + (size_t)gy * K + gx;
      int gz = z0;
#pragma unroll
      for (int iz = 0; iz < E; ++iz) {
        const int idx = c + iz * E2;
        const int a = tre[idx], b = tim[idx];
        if ((a | b) != 0 || poison) {
          tre[idx] = 0;
          tim[idx] = 0;
          const float2 v = poison ? make_float2(qnan, qnan) : make_float2((float)a * inv, (float)b * inv);
          atomicAdd(col + (size_t)(gz >= K ? gz - K : gz) * KK, v);
        }
        ++gz;
      }
    }
    parity ^= 1;
    s = s_next;
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
        point_coeffs<6>(g, f[0], cx);
        point_coeffs<6>(g, f[1], cy);
        point_coeffs<6>(g, f[2], cz);
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

bool v4s_supported(int T, int J, int S) {
  return J == 6 && T == 8 && v4s_bytes(T, S) <= (size_t)max_optin_smem();
}

bool v5s_supported(int T, int J, int S) {
  return J == 6 && T == 8 && S >= 1 && S <= 512 && v5s_bytes(T) <= (size_t)max_optin_smem();
}

bool v6s_supported(int T, int J, int S) {
  return J == 6 && T == 8 && S >= 1 && S <= V6S_MAX_PTS && V6SLayout::bytes <= (size_t)max_optin_smem();
}

bool v3s_supported(int T, int J) {
  return J == 6 && T == 8 && v3s_bytes(T) <= (size_t)max_optin_smem();
}

bool v2_supported(int T, int J, int L) {
  return L > 0 && J == 6 && (T == 8 || T == 16) && v2_layout(T, L).bytes <= (size_t)max_optin_smem();
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
  if (variant == 7) return launch_spread_real(g, in, subs, n_subs, grid, st);
  if (variant == 8) return launch_spread_sched(g, in, subs, n_subs, grid, st);
  if (variant == 6 && v6s_supported(g.T, g.J, g.S)) {
    auto f = k_spread_v6;
    const size_t smem = V6SLayout::bytes;
    cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_subs == 0) return cudaSuccess;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V6S_THREADS, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const float budget = ldexpf(1.f - 1.f / 1024.f, 22);  // at most 256 points per subproblem
    e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    f<<<num_sms() * per_sm, V6S_THREADS, smem, st>>>(g, in, subs, n_subs, g.counter + 1, grid, budget, 1.f / budget);
    return cudaGetLastError();
  }
  if (variant == 5 && v5s_supported(g.T, g.J, g.S)) {
    auto f = k_spread_v5<8>;
    const size_t smem = v5s_bytes(g.T);
    cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_subs == 0) return cudaSuccess;
    int lg = 0;
    while ((1 << lg) < g.S) ++lg;
    const int bits = lg > 8 ? 30 - lg : 22;
    const float budget = ldexpf(1.f - 1.f / 1024.f, bits);
    e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    f<<<num_sms(), V5S_WARPS * 32, smem, st>>>(g, in, subs, n_subs, g.counter + 1, grid, budget, 1.f / budget);
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
