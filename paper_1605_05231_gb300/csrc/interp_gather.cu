// Gather kernels (grid -> points): the separable J-tap min-max interpolator T of
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
// This file holds the gather variants; interp_spread.cu the spread variants.
#include "interp_common.cuh"

namespace nufft {

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
    point_coeffs<J>(g, f[0], cx);
    point_coeffs<J>(g, f[1], cy);
    point_coeffs<J>(g, f[2], cz);
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
  int copy2;  // cell offset of the second tile copy (0: one copy)
  size_t tile_bytes, bytes;
};

// elem: bytes per grid cell in shared memory (8 for complex64, 4 for bf16/fp16
// pairs).  With two copies the second starts at a cell offset congruent to
// half the residue range (kRes / 2, kRes = 128 / elem), so that a point read
// from it falls in the partner residue class.
__host__ __device__ inline V3Layout v3_layout(int T, int J, int S, int elem, bool two = false) {
  V3Layout l;
  l.E = T + J - 1;
  const int e3 = l.E * l.E * l.E;
  const int kres = 128 / elem;
  l.copy2 = two ? e3 + ((kres / 2 - e3 % kres) + kres) % kres : 0;
  const int cells = two ? l.copy2 + e3 : e3;
  l.tile_bytes = ((size_t)cells * elem + 15) / 16 * 16;
  // per point: id, twin, tile offset, f[3] (6 words) + ordered index (1 word); class counts and cursors
  l.bytes = l.tile_bytes + (size_t)S * 7 * sizeof(int) + 64 * sizeof(int);
  return l;
}

// TWO = false: one tile copy, points in round-robin order over their residue
// classes.  TWO = true (variants 6 and 7): two copies of the tile; the points
// of classes c and c + kRes/2 form one pool and are dealt alternately to the
// two classes (a point dealt to its partner class reads the second copy), so
// the classes of each pair hold equally many points and fewer half-warps
// repeat a class.
template <int J, int T, int NT, typename G, bool TWO = false>
__global__ void __launch_bounds__(NT, J <= 6 ? 1024 / NT : 1) k_gather_v3(InterpGeom g, const typename G::T* __restrict__ grid,
                                                  float inv_scale, const int4* __restrict__ subs, int S,
                                                  float2* __restrict__ out) {
  typedef typename G::T TT;
  // a warp access of 4-byte cells is conflict-free with 32 distinct residues,
  // of 8-byte cells with 16 distinct residues per half-warp
  constexpr int kRes = sizeof(TT) == 4 ? 32 : 16;
  constexpr int kHalf = kRes / 2;
  constexpr int E = T + J - 1, E2 = E * E, PP = E2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  inv_scale = lp_inv_scale<G>(g);
  const int nT = g.nT, K = g.K;
  const V3Layout lay = v3_layout(T, J, S, (int)sizeof(TT), TWO);
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
  // stage the tile: threads walk (z, y) rows; a row's x run is contiguous in the grid
  for (int r = threadIdx.x; r < E2 * E; r += NT) {
    const int row = r / E, ix = r - row * E;
    const int iz = row / E, iy = row - iz * E;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    const TT v = grid[((size_t)gz * K + gy) * K + gx];
    tile[r] = v;
    if (TWO) tile[lay.copy2 + r] = v;
  }
  __syncthreads();
  // decode every point of the subproblem once
  for (int i = threadIdx.x; i < cnt; i += NT) {
    const uint2 ent = g.sorted[sp.y + i];
    int w0[3];
    float f[3];
    decode_point<J>(g, ent.x, w0, f);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    int off = -1;
    if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
      off = (lz * E + ly) * E + lx;
    } else {
      atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
    }
    p_id[i] = (int)ent.x;
    p_tw[i] = (int)ent.y;
    p_off[i] = off;
    p_f[i] = f[0];
    p_f[S + i] = f[1];
    p_f[2 * S + i] = f[2];
    const int c = off < 0 ? 0 : (off & (kRes - 1));
    atomicAdd(&ncls[TWO ? (c & (kHalf - 1)) : c], 1);
  }
  __syncthreads();
  if (TWO) {
    // class sizes after dealing each pool alternately: ceil to c, floor to c + kHalf
    int pool = 0;
    if (threadIdx.x < kHalf) pool = ncls[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < kHalf) {
      ncls[threadIdx.x] = (pool + 1) >> 1;
      ncls[threadIdx.x + kHalf] = pool >> 1;
    }
    __syncthreads();
  }
  // rank within the class, then the round-robin position
  for (int i = threadIdx.x; i < cnt; i += NT) {
    int off = p_off[i];
    const int c0 = off < 0 ? 0 : (off & (kRes - 1));
    int c = c0, r;
    if (TWO) {
      const int pc = c0 & (kHalf - 1);
      const int q = atomicAdd(&ncls[kRes + pc], 1);
      c = pc + ((q & 1) ? kHalf : 0);
      r = q >> 1;
      if (c != c0 && off >= 0) p_off[i] = off + lay.copy2;  // read from the second copy
    } else {
      r = atomicAdd(&ncls[kRes + c], 1);
    }
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
  for (int k = threadIdx.x; k < cnt; k += NT) {
    const int i = order[k];
    const int off = p_off[i];
    if (off < 0) continue;
    float2 cx[J], cy[J], cz[J];
    point_coeffs<J>(g, p_f[i], cx);
    point_coeffs<J>(g, p_f[S + i], cy);
    point_coeffs<J>(g, p_f[2 * S + i], cz);
    float2 acc = make_float2(0.f, 0.f);
    const TT* base = tile + off;
#pragma unroll
    for (int jz = 0; jz < J; ++jz) {
      float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
      for (int jy = 0; jy < J; ++jy) {
        const TT* tp = base + jz * PP + jy * E;
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

template <int J, int T, int NT, typename G, bool TWO = false>
static cudaError_t launch_gather_v3_tt(const InterpGeom& g, const void* grid, float inv_scale, const int4* subs,
                                       int n_subs, int S, float2* out, cudaStream_t st) {
  auto f = k_gather_v3<J, T, NT, G, TWO>;
  const size_t smem = v3_layout(T, J, S, (int)sizeof(typename G::T), TWO).bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  f<<<n_subs, NT, smem, st>>>(g, (const typename G::T*)grid, inv_scale, subs, S, out);
  return cudaGetLastError();
}

template <int J, typename G>
static cudaError_t launch_gather_v3_t(const InterpGeom& g, int nt, const void* grid, float inv_scale,
                                      const int4* subs, int n_subs, int S, float2* out, cudaStream_t st) {
  if (nt == 128) {
    if (g.T == 8) return launch_gather_v3_tt<J, 8, 128, G>(g, grid, inv_scale, subs, n_subs, S, out, st);
  } else {
    switch (g.T) {
      case 4: return launch_gather_v3_tt<J, 4, 256, G>(g, grid, inv_scale, subs, n_subs, S, out, st);
      case 8: return launch_gather_v3_tt<J, 8, 256, G>(g, grid, inv_scale, subs, n_subs, S, out, st);
      case 16: return launch_gather_v3_tt<J, 16, 256, G>(g, grid, inv_scale, subs, n_subs, S, out, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <int J>
static cudaError_t launch_gather_v3_j(const InterpGeom& g, int nt, int dtype, const void* grid, float inv_scale,
                                      const int4* subs, int n_subs, int S, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v3_t<J, GridC64>(g, nt, grid, inv_scale, subs, n_subs, S, out, st);
    case 1: return launch_gather_v3_t<J, GridBF16>(g, nt, grid, inv_scale, subs, n_subs, S, out, st);
    case 2: return launch_gather_v3_t<J, GridF16>(g, nt, grid, inv_scale, subs, n_subs, S, out, st);
  }
  return cudaErrorInvalidValue;
}


bool v4_supported(int T, int J, int S, int L) {
  return L > 0 && v4_bytes(T, J, S, L, 8) <= (size_t)max_optin_smem();
}

bool v3_supported(int T, int J, int S) {
  return v3_layout(T, J, S, 8).bytes <= (size_t)max_optin_smem();
}

bool v3_two_copy_supported(int T, int J, int S) {
  return T == 8 && J == 6 && v3_layout(T, J, S, 8, true).bytes <= (size_t)max_optin_smem();
}

// variants 6 (256 threads) and 7 (128 threads): two tile copies, J = 6, T = 8
template <typename G>
static cudaError_t launch_gather_v3_two(const InterpGeom& g, int nt, const void* grid, float inv_scale,
                                        const int4* subs, int n_subs, int S, float2* out, cudaStream_t st) {
  if (nt == 128) return launch_gather_v3_tt<6, 8, 128, G, true>(g, grid, inv_scale, subs, n_subs, S, out, st);
  return launch_gather_v3_tt<6, 8, 256, G, true>(g, grid, inv_scale, subs, n_subs, S, out, st);
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
  if (variant == 8) return launch_gather_tma(g, grid_dtype, grid, subs, n_subs, out, st);
  if (variant == 9) return launch_gather_real(g, grid_dtype, grid, subs, n_subs, out, st);
  if (variant == 10) return launch_gather_sched(g, grid_dtype, grid, subs, n_subs, out, st);
  if (variant == 11) return launch_gather_sched_pipelined(g, grid_dtype, grid, subs, n_subs, out, st);
  if ((variant == 6 || variant == 7) && g.J == 6 && g.T == 8) {
    const int nt = variant == 7 ? 128 : 256;
    switch (grid_dtype) {
      case 0: return launch_gather_v3_two<GridC64>(g, nt, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 1: return launch_gather_v3_two<GridBF16>(g, nt, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 2: return launch_gather_v3_two<GridF16>(g, nt, grid, inv_scale, subs, n_subs, g.S, out, st);
    }
    return cudaErrorInvalidValue;
  }
  if (variant == 3 || variant == 5) {
    const int nt = variant == 5 ? 128 : 256;
    switch (g.J) {
      case 2: return launch_gather_v3_j<2>(g, nt, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 4: return launch_gather_v3_j<4>(g, nt, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 6: return launch_gather_v3_j<6>(g, nt, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
      case 8: return launch_gather_v3_j<8>(g, nt, grid_dtype, grid, inv_scale, subs, n_subs, g.S, out, st);
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

}  // namespace nufft
