// Interpolation kernels with real weights (gather variant 9, spread variant 7).
//
// With the pre-window symmetric about the middle of the index range the
// min-max coefficients of Eq. 2.11's interpolator factor exactly as
//   c_j(f) = e^{i gamma (u - k) / 2} rho_j(f),  rho_j real,  k = k0 + j,
// so the forward interpolation of one point is
//   X^(u) = e^{i gamma (ux + uy + uz)/2}
//           sum_k rho(fx) rho(fy) rho(fz) e^{-i gamma (kx + ky + kz)/2} Y[k mod K].
// The grid phase e^{-i gamma (kx + ky + kz)/2} is applied by the forward z pass
// (the grid then holds Y~), and its conjugate by the inverse z pass for the
// spread, which accumulates e^{-i gamma (ux + uy + uz)/2} v rho rho rho.  A tap
// whose unwrapped index lies outside [-K/2, K/2) reads a cell whose centred
// index differs by K, hence a phase of opposite sign: its weight is negated.
// Per tap this is a real weight times a complex value (2 FMAs) instead of a
// complex product (4), and the coefficient evaluation is real.
//
// Gather 9: the one-thread-per-point gather of variant 5 (128-thread CTAs,
// points in round-robin order over the residue classes of their tile offset).
// Spread 7: the fixed-point spread of variant 6 (one 13^3 int32 tile per CTA
// of six warps, lane tables, exponent per subproblem).
#include "interp_common.cuh"

namespace nufft {

// the plan of work item w of a group (the group's prefix table of work items)
__device__ __forceinline__ int group_item_of(const GroupParams& gp, int w) {
  int it = 0;
  while (it + 1 < gp.n_items && w >= gp.work_begin[it + 1]) ++it;
  return it;
}

// ---------------------------------------------------------------------------
// gather 9
// ---------------------------------------------------------------------------
constexpr int V9_NT = 128;

// per point: id, twin, tile offset, f[3], flip masks, phase (2), ordered index
__host__ __device__ inline size_t v9_bytes(int T, int J, int S, int elem) {
  const int E = T + J - 1;
  const size_t tile = ((size_t)E * E * E * elem + 15) / 16 * 16;
  return tile + (size_t)S * 10 * sizeof(int) + 64 * sizeof(int);
}

template <int J, typename G>
__global__ void __launch_bounds__(V9_NT, J <= 6 ? 8 : 1) k_gather_v9(InterpGeom g, const typename G::T* __restrict__ grid,
                                                                 const int4* __restrict__ subs, int S,
                                                                 float2* __restrict__ out) {
  typedef typename G::T TT;
  constexpr int T = 8, NT = V9_NT;
  constexpr int kRes = sizeof(TT) == 4 ? 32 : 16;
  constexpr int E = T + J - 1, E2 = E * E, PP = E2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const float inv_scale = lp_inv_scale<G>(g);
  const int nT = g.nT, K = g.K;
  const size_t tile_bytes = ((size_t)E * E * E * sizeof(TT) + 15) / 16 * 16;
  TT* tile = (TT*)smem_raw;
  int* p_id = (int*)(smem_raw + tile_bytes);
  int* p_tw = p_id + S;
  int* p_off = p_tw + S;
  float* p_f = (float*)(p_off + S);  // [3][S]
  int* p_flip = (int*)(p_f + 3 * S);
  float2* p_ph = (float2*)(p_flip + S);  // 8-byte aligned: S is even
  int* order = (int*)(p_ph + S);
  int* ncls = order + S;  // [kRes] counts, [kRes] cursors
  const int4 sp = subs[blockIdx.x];
  const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
  const int x0 = bx * T, y0 = by * T, z0 = bz * T;
  const int cnt = sp.z;
  if (threadIdx.x < 2 * kRes) ncls[threadIdx.x] = 0;
  for (int r = threadIdx.x; r < E2 * E; r += NT) {
    const int row = r / E, ix = r - row * E;
    const int iz = row / E, iy = row - iz * E;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    tile[r] = grid[((size_t)gz * K + gy) * K + gx];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += NT) {
    const uint2 ent = g.sorted[sp.y + i];
    int w0[3], fm[3];
    float f[3];
    float2 ph;
    decode_point_real<J>(g, ent.x, w0, f, fm, ph);
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
    p_flip[i] = fm[0] | (fm[1] << 8) | (fm[2] << 16);
    p_ph[i] = ph;
    atomicAdd(&ncls[off < 0 ? 0 : (off & (kRes - 1))], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += NT) {
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
  for (int k = threadIdx.x; k < cnt; k += NT) {
    const int i = order[k];
    const int off = p_off[i];
    if (off < 0) continue;
    const int fm = p_flip[i];
    float rx[J], ry[J], rz[J];
    real_coeffs<J>(g.rpoly, p_f[i], fm & 0xff, rx);
    real_coeffs<J>(g.rpoly, p_f[S + i], (fm >> 8) & 0xff, ry);
    real_coeffs<J>(g.rpoly, p_f[2 * S + i], fm >> 16, rz);
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
        for (int jx = 0; jx < J; ++jx) rmac(row, rx[jx], G::to_f2(tp[jx]));
        rmac(zacc, ry[jy], row);
      }
      rmac(acc, rz[jz], zacc);
    }
    const float2 res = cmul(cscale(acc, inv_scale), p_ph[i]);
    out[p_id[i]] = res;
    if ((uint32_t)p_tw[i] != kNoTwin) out[p_tw[i]] = res;
  }
}

template <int J, typename G>
static cudaError_t launch_gather_v9_t(const InterpGeom& g, const void* grid, const int4* subs, int n_subs,
                                      float2* out, cudaStream_t st) {
  auto f = k_gather_v9<J, G>;
  const size_t smem = v9_bytes(8, J, g.S, (int)sizeof(typename G::T));
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  f<<<n_subs, V9_NT, smem, st>>>(g, (const typename G::T*)grid, subs, g.S, out);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v9_j(const InterpGeom& g, int dtype, const void* grid, const int4* subs, int n_subs,
                                      float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v9_t<J, GridC64>(g, grid, subs, n_subs, out, st);
    case 1: return launch_gather_v9_t<J, GridBF16>(g, grid, subs, n_subs, out, st);
    case 2: return launch_gather_v9_t<J, GridF16>(g, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

bool v9_supported(int T, int J, int S) {
  return T == 8 && (J == 2 || J == 4 || J == 6 || J == 8) && S >= 2 && S % 2 == 0 &&
         v9_bytes(T, J, S, 8) <= (size_t)max_optin_smem();
}

cudaError_t launch_gather_real(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                               float2* out, cudaStream_t st) {
  if (!v9_supported(g.T, g.J, g.S)) return cudaErrorInvalidValue;
  switch (g.J) {
    case 2: return launch_gather_v9_j<2>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 4: return launch_gather_v9_j<4>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 6: return launch_gather_v9_j<6>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 8: return launch_gather_v9_j<8>(g, grid_dtype, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// spread 7
//  phase 1: thread per point: decode, real weights rho_x, rho_y, rho_z and
//           v' = e^{-i gamma (ux+uy+uz)/2} v into the point's row, the bound
//           |v| max|rx| max|ry| max|rz|;
//           the CTA's largest bound fixes the subproblem's exponent;
//  phase 2: warp w spreads points w, w + 6, ...: lane taps as in spread 6, each
//           contribution rho_z (w_xy v') with w_xy = rho_x rho_y real, rounded
//           to units by one FMA per plane;
//  flush:   all 192 threads add the tile to the grid and clear it.
// ---------------------------------------------------------------------------
constexpr int V7S_WARPS = 6, V7S_THREADS = V7S_WARPS * 32, V7S_MAX_PTS = 256;
constexpr int V7S_CSTRIDE = 24;  // floats per point: rx[6] ry[6] rz[6] v' (re, im), 4 unused (16-byte rows)

struct V7SLayout {
  static constexpr int E = 13, E3 = E * E * E;
  static constexpr size_t coef = 0;                                                     // [256][24] float
  static constexpr size_t mos = coef + (size_t)V7S_MAX_PTS * V7S_CSTRIDE * sizeof(float);  // [256] int
  static constexpr size_t tre = mos + V7S_MAX_PTS * sizeof(int);                         // [E3] int
  static constexpr size_t tim = tre + E3 * sizeof(int);                                  // [E3] int
  static constexpr size_t wmax = tim + E3 * sizeof(int);                                 // [6] unsigned
  static constexpr size_t nxt = wmax + V7S_WARPS * sizeof(unsigned);                     // [2] int
  static constexpr size_t bytes = (nxt + 2 * sizeof(int) + 15) / 16 * 16;
};

// Where a spread CTA finds its subproblem: one plan, or a group of plans (as
// for the scheduled gather).
struct SpreadWork {
  PointGeom pg;
  const uint2* sorted;
  int* err;
  int4 sp;
  const float2* in;
  float2* grid;
};

struct GroupSpreadSrc {
  GroupParams gp;
  const GroupItem* items;
  __device__ __forceinline__ const RealPoly& rpoly() const { return gp.rpoly; }
  __device__ __forceinline__ void at(int w, SpreadWork& k) const {
    const int it = group_item_of(gp, w);
    const GroupItem& I = items[it];
    k.pg = I.pg;
    k.sorted = I.sorted;
    k.err = I.err;
    k.sp = I.subs[w - gp.work_begin[it]];
    k.in = I.adj_in;
    k.grid = I.adj_grid;
  }
};

struct PlanSpreadSrc {
  InterpGeom g;
  const int4* subs;
  const float2* in;
  float2* grid;
  __device__ __forceinline__ const RealPoly& rpoly() const { return g.rpoly; }
  __device__ __forceinline__ void at(int w, SpreadWork& k) const {
    k.pg = PointGeom{g.K, g.M, g.dir, g.rad};
    k.sorted = g.sorted;
    k.err = g.err;
    k.sp = subs[w];
    k.in = in;
    k.grid = grid;
  }
};

template <class Src>
__global__ void __launch_bounds__(V7S_THREADS, 5) k_spread_v7(const Src src, int n_subs, int nT,
                                                             int* __restrict__ counter, float budget,
                                                             float inv_budget) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Lay = V7SLayout;
  constexpr int T = 8, E = Lay::E, E2 = E * E, E3 = Lay::E3;
  float* coef = (float*)(smem_raw + Lay::coef);
  int* mos = (int*)(smem_raw + Lay::mos);
  int* tre = (int*)(smem_raw + Lay::tre);
  int* tim = (int*)(smem_raw + Lay::tim);
  unsigned* wmax = (unsigned*)(smem_raw + Lay::wmax);
  int* nxt = (int*)(smem_raw + Lay::nxt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < E3; i += V7S_THREADS) {
    tre[i] = 0;
    tim[i] = 0;
  }
  const V5Lanes ln = v5_lanes(lane);
  const int main_off = ln.has_main ? ln.main_off : kPadI13[0];
  const int ovf_off = ln.has_ovf ? ln.ovf_off : kPadI13[lane == 30 ? 1 : 2];
  if (tid == 0) nxt[0] = atomicAdd(counter, 1);
  __syncthreads();
  int s = nxt[0], parity = 0;
  while (s < n_subs) {
    SpreadWork wk;
    src.at(s, wk);
    const int K = wk.pg.K;
    const size_t KK = (size_t)K * K;
    const float2* __restrict__ in = wk.in;
    float2* __restrict__ grid = wk.grid;
    const int4 sp = wk.sp;
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    unsigned bound = 0u;
    for (int i = tid; i < sp.z; i += V7S_THREADS) {
      const uint2 ent = wk.sorted[sp.y + i];
      int w0[3], fm[3];
      float f[3];
      float2 ph;
      decode_point_real<6>(wk.pg, ent.x, w0, f, fm, ph);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      float4* c4 = (float4*)(coef + i * V7S_CSTRIDE);
      int off = 0;
      if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
        off = (lz * E + ly) * E + lx;
        float2 val = in[ent.x];
        if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
        const float2 vp = cmulc(val, ph);  // e^{-i gamma sum u / 2} v
        float rx[6], ry[6], rz[6];
        real_coeffs<6>(src.rpoly(), f[0], fm[0], rx);
        real_coeffs<6>(src.rpoly(), f[1], fm[1], ry);
        real_coeffs<6>(src.rpoly(), f[2], fm[2], rz);
        float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          mx = fmaxf(mx, fabsf(rx[q]));
          my = fmaxf(my, fabsf(ry[q]));
          mz = fmaxf(mz, fabsf(rz[q]));
        }
        c4[0] = make_float4(rx[0], rx[1], rx[2], rx[3]);
        c4[1] = make_float4(rx[4], rx[5], ry[0], ry[1]);
        c4[2] = make_float4(ry[2], ry[3], ry[4], ry[5]);
        c4[3] = make_float4(rz[0], rz[1], rz[2], rz[3]);
        c4[4] = make_float4(rz[4], rz[5], vp.x, vp.y);
        bound = max(bound, __float_as_uint(hypotf(val.x, val.y) * (mx * my * mz)));
      } else {
        atomicExch(wk.err, (int)DEVCHK_TILE_RANGE);
#pragma unroll
        for (int q = 0; q < 6; ++q) c4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      mos[i] = off;
    }
    const unsigned wb = __reduce_max_sync(0xffffffffu, bound);
    if (lane == 0) wmax[warp] = wb;
    if (tid == 0) nxt[parity ^ 1] = atomicAdd(counter, 1);
    __syncthreads();
    unsigned bb = wmax[0];
#pragma unroll
    for (int w = 1; w < V7S_WARPS; ++w) bb = max(bb, wmax[w]);
    const bool poison = bb > kBoundLimitBits;
    int e_tile = kTileEmpty;
    if (!poison && bb != 0u) {
      e_tile = max((int)(bb >> 23) - 127 + ((bb & 0x7FFFFFu) ? 1 : 0), -100);
      const float sc = budget * pow2f(-e_tile);
      const float sm = ln.has_main ? sc : 0.f, so = ln.has_ovf ? sc : 0.f;
      for (int p = warp; p < sp.z; p += V7S_WARPS) {
        const int mo = mos[p];
        const float* cp = coef + p * V7S_CSTRIDE;
        // the lane's column weight rho_x rho_y times v' (complex), then the
        // six real rho_z of the z row: 24 bytes of broadcast row per point
        const float wxy = cp[ln.mjx] * cp[6 + ln.mjy] * sm;
        const float4 za = *(const float4*)(cp + 12), zb = *(const float4*)(cp + 16);
        const float rzv[6] = {za.x, za.y, za.z, za.w, zb.x, zb.y};
        const float wre = wxy * zb.z, wim = wxy * zb.w;
        const float wo = cp[ln.ojx] * cp[6 + ln.ojy] * cp[12 + ln.ojz] * so;
        int* re = tre + mo + main_off;
        int* im = tim + mo + main_off;
#pragma unroll
        for (int jz = 0; jz < 6; ++jz) {
          atomicAdd(re + jz * E2, round_unit1(rzv[jz], wre));
          atomicAdd(im + jz * E2, round_unit1(rzv[jz], wim));
        }
        atomicAdd(tre + mo + ovf_off, round_unit1(wo, zb.z));
        atomicAdd(tim + mo + ovf_off, round_unit1(wo, zb.w));
      }
    }
    __syncthreads();
    const int s_next = nxt[parity ^ 1];
    // flush: the tile added to the grid (the inverse z pass applies the grid phase)
    const float inv = e_tile == kTileEmpty ? 0.f : inv_budget * pow2f(e_tile);
    const float qnan = __int_as_float(0x7fc00000);
    for (int c = tid; c < E2; c += V7S_THREADS) {
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

bool v7s_supported(int T, int J, int S) {
  return J == 6 && T == 8 && S >= 1 && S <= V7S_MAX_PTS && V7SLayout::bytes <= (size_t)max_optin_smem();
}

cudaError_t launch_spread_real(const InterpGeom& g, const float2* in, const int4* subs, int n_subs, float2* grid,
                               cudaStream_t st) {
  if (!v7s_supported(g.T, g.J, g.S)) return cudaErrorInvalidValue;
  auto f = k_spread_v7<PlanSpreadSrc>;
  const size_t smem = V7SLayout::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V7S_THREADS, smem);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const float budget = ldexpf(1.f - 1.f / 1024.f, 22);  // at most 256 points per subproblem
  e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const PlanSpreadSrc src{g, subs, in, grid};
  f<<<num_sms() * per_sm, V7S_THREADS, smem, st>>>(src, n_subs, g.nT, g.counter + 1, budget, 1.f / budget);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gather 10: the real-weight gather with the plan's conflict schedule.  One
// CTA per subproblem stages the tile with the subproblem's plane pitch; then
// thread k serves slot k of the schedule (a point of the subproblem, or
// nothing): decode, weights and taps in registers, no reordering at run time.
// The 16 slots of a half-warp hold points whose base offsets are distinct
// modulo 16 cells or equal, so every tap read is one wavefront per half-warp.
// ---------------------------------------------------------------------------
constexpr int V10_NT = 128;

template <int J>
__host__ __device__ inline size_t v10_bytes(int elem) {
  constexpr int E = 8 + J - 1;
  return ((size_t)E * (E * E + kGatherPitchCodes - 1) * elem + 15) / 16 * 16;
}

// Where a scheduled-gather CTA finds its subproblem: one plan (work item w is
// subproblem w), or a group of plans sharing N, K and J (work items numbered
// across the plans; the plan of item w is found in the group's prefix table).
struct GatherWork {
  PointGeom pg;
  const uint2* sorted;
  int* err;
  int4 sp, sc;
  const int* box;
  int box_i;
  const uint16_t* gslots;
  const void* grid;
  float2* out;
};

struct PlanGatherSrc {
  InterpGeom g;
  const int4* subs;
  const void* grid;
  float2* out;
  __device__ __forceinline__ const RealPoly& rpoly() const { return g.rpoly; }
  __device__ __forceinline__ void at(int w, GatherWork& k) const {
    k.pg = PointGeom{g.K, g.M, g.dir, g.rad};
    k.sorted = g.sorted;
    k.err = g.err;
    k.sp = subs[w];
    k.sc = g.sched[w];
    k.box = g.box;
    k.box_i = w;
    k.gslots = g.gslots;
    k.grid = grid;
    k.out = out;
  }
};

struct GroupGatherSrc {
  GroupParams gp;
  const GroupItem* items;
  __device__ __forceinline__ const RealPoly& rpoly() const { return gp.rpoly; }
  __device__ __forceinline__ void at(int w, GatherWork& k) const {
    const int it = group_item_of(gp, w);
    const GroupItem& I = items[it];
    const int l = w - gp.work_begin[it];
    k.pg = I.pg;
    k.sorted = I.sorted;
    k.err = I.err;
    k.sp = I.subs[l];
    k.sc = I.sched[l];
    k.box = I.box;
    k.box_i = l;
    k.gslots = I.gslots;
    k.grid = I.grid;
    k.out = I.lines;
  }
};

template <int J, typename G, class Src>
__global__ void __launch_bounds__(V10_NT, 9) k_gather_v10(const Src src, int nT, float inv_scale_in,
                                                          const float* __restrict__ lp_bound) {
  typedef typename G::T TT;
  constexpr int T = 8, NT = V10_NT, E = T + J - 1, E2 = E * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TT* tile = (TT*)smem_raw;
  float inv_scale = inv_scale_in;
  if constexpr (G::kLowPrecision) inv_scale = 1.f / lp_scale_from_bound(*lp_bound);
  GatherWork wk;
  src.at(blockIdx.x, wk);
  const int K = wk.pg.K;
  const TT* __restrict__ grid = (const TT*)wk.grid;
  const int4 sp = wk.sp, sc = wk.sc;
  const int PP = E2 + (sc.y >> 16), nslots = sc.y & 0xffff;
  const int x0 = (sp.x % nT) * T, y0 = ((sp.x / nT) % nT) * T, z0 = (sp.x / (nT * nT)) * T;
  // only the cells the subproblem's taps can reach are staged (the plan's box;
  // the quotients below are exact: (r + 1/2) / e is at least 1/(2e) from an integer)
  const TileBox bx = unpack_box(wk.box, wk.box_i, E);
  const float inv_ex = 1.f / (float)bx.ex, inv_ey = 1.f / (float)bx.ey;
  for (int r = threadIdx.x; r < bx.ex * bx.ey * bx.ez; r += NT) {
    const int row = (int)(((float)r + 0.5f) * inv_ex), ix = bx.ox + r - row * bx.ex;
    const int rz = (int)(((float)row + 0.5f) * inv_ey), iy = bx.oy + row - rz * bx.ey, iz = bx.oz + rz;
    int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
    gx -= gx >= K ? K : 0;
    gy -= gy >= K ? K : 0;
    gz -= gz >= K ? K : 0;
    tile[iz * PP + iy * E + ix] = grid[((size_t)gz * K + gy) * K + gx];
  }
  __syncthreads();
  const uint16_t* slots = wk.gslots + sc.x;
  float2* __restrict__ out = wk.out;
  for (int k = threadIdx.x; k < nslots; k += NT) {
    const int li = slots[k];
    if (li == 0xffff) continue;
    const uint2 ent = wk.sorted[sp.y + li];
    int w0[3], fm[3];
    float f[3];
    float2 ph;
    decode_point_real<J>(wk.pg, ent.x, w0, f, fm, ph);
    const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
    if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
      atomicExch(wk.err, (int)DEVCHK_TILE_RANGE);
      continue;
    }
    float rx[J], ry[J], rz[J];
    real_coeffs<J>(src.rpoly(), f[0], fm[0], rx);
    real_coeffs<J>(src.rpoly(), f[1], fm[1], ry);
    real_coeffs<J>(src.rpoly(), f[2], fm[2], rz);
    float2 acc = make_float2(0.f, 0.f);
    const TT* base = tile + (lz * PP + ly * E + lx);
#pragma unroll
    for (int jz = 0; jz < J; ++jz) {
      const TT* pz = base + jz * PP;
      float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
      for (int jy = 0; jy < J; ++jy) {
        const TT* tp = pz + jy * E;
        float2 row = make_float2(0.f, 0.f);
#pragma unroll
        for (int jx = 0; jx < J; ++jx) rmac(row, rx[jx], G::to_f2(tp[jx]));
        rmac(zacc, ry[jy], row);
      }
      rmac(acc, rz[jz], zacc);
    }
    const float2 res = cmul(cscale(acc, inv_scale), ph);
    out[ent.x] = res;
    if (ent.y != kNoTwin) out[ent.y] = res;
  }
}

template <int J, typename G>
static cudaError_t launch_gather_v10_t(const InterpGeom& g, const void* grid, const int4* subs, int n_subs,
                                       float2* out, cudaStream_t st) {
  auto f = k_gather_v10<J, G, PlanGatherSrc>;
  const size_t smem = v10_bytes<J>((int)sizeof(typename G::T));
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  const PlanGatherSrc src{g, subs, grid, out};
  f<<<n_subs, V10_NT, smem, st>>>(src, g.nT, 1.f, g.lp_bound);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v10_j(const InterpGeom& g, int dtype, const void* grid, const int4* subs,
                                       int n_subs, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v10_t<J, GridC64>(g, grid, subs, n_subs, out, st);
    case 1: return launch_gather_v10_t<J, GridBF16>(g, grid, subs, n_subs, out, st);
    case 2: return launch_gather_v10_t<J, GridF16>(g, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// gather 11: gather 10 made persistent, with the next subproblem's tile
// copied into a second shared-memory buffer by asynchronous copies
// (cp.async, one cell per copy, at the subproblem's own plane pitch) while the
// current subproblem is interpolated, so the staging latency is hidden.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_cell(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <int J>
__host__ __device__ inline size_t v11_tile_bytes(int elem) {
  constexpr int E = 8 + J - 1;
  return ((size_t)E * (E * E + kGatherPitchCodes - 1) * elem + 127) / 128 * 128;
}

template <int J, typename G>
__global__ void __launch_bounds__(V10_NT, 5) k_gather_v11(InterpGeom g, const typename G::T* __restrict__ grid,
                                                          const int4* __restrict__ subs, int n_subs,
                                                          float2* __restrict__ out) {
  typedef typename G::T TT;
  constexpr int T = 8, NT = V10_NT, E = T + J - 1, E2 = E * E;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const size_t tb = v11_tile_bytes<J>((int)sizeof(TT));
  const float inv_scale = lp_inv_scale<G>(g);
  const int nT = g.nT, K = g.K;
  // copy subproblem s's tile into buffer b
  auto stage = [&](int s, int b) {
    const int4 sp = subs[s];
    const int PP = E2 + (g.sched[s].y >> 16);
    const int x0 = (sp.x % nT) * T, y0 = ((sp.x / nT) % nT) * T, z0 = (sp.x / (nT * nT)) * T;
    TT* tile = (TT*)(smem_raw + b * tb);
    for (int r = threadIdx.x; r < E2 * E; r += NT) {
      const int row = r / E, ix = r - row * E;
      const int iz = row / E, iy = row - iz * E;
      int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      gz -= gz >= K ? K : 0;
      cp_async_cell(tile + iz * PP + iy * E + ix, grid + ((size_t)gz * K + gy) * K + gx, (int)sizeof(TT));
    }
  };
  int b = 0;
  if ((int)blockIdx.x < n_subs) stage(blockIdx.x, 0);
  cp_async_commit();
  for (int s = blockIdx.x; s < n_subs; s += gridDim.x, b ^= 1) {
    const int nxt = s + gridDim.x;
    if (nxt < n_subs) stage(nxt, b ^ 1);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of tile s have landed
    __syncthreads();   // and everyone's
    const int4 sp = subs[s];
    const int4 sc = g.sched[s];
    const int PP = E2 + (sc.y >> 16), nslots = sc.y & 0xffff;
    const int x0 = (sp.x % nT) * T, y0 = ((sp.x / nT) % nT) * T, z0 = (sp.x / (nT * nT)) * T;
    const TT* tile = (const TT*)(smem_raw + b * tb);
    const uint16_t* slots = g.gslots + sc.x;
    for (int k = threadIdx.x; k < nslots; k += NT) {
      const int li = slots[k];
      if (li == 0xffff) continue;
      const uint2 ent = g.sorted[sp.y + li];
      int w0[3], fm[3];
      float f[3];
      float2 ph;
      decode_point_real<J>(g, ent.x, w0, f, fm, ph);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
        atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
        continue;
      }
      float rx[J], ry[J], rz[J];
      real_coeffs<J>(g.rpoly, f[0], fm[0], rx);
      real_coeffs<J>(g.rpoly, f[1], fm[1], ry);
      real_coeffs<J>(g.rpoly, f[2], fm[2], rz);
      float2 acc = make_float2(0.f, 0.f);
      const TT* base = tile + (lz * PP + ly * E + lx);
#pragma unroll
      for (int jz = 0; jz < J; ++jz) {
        const TT* pz = base + jz * PP;
        float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int jy = 0; jy < J; ++jy) {
          const TT* tp = pz + jy * E;
          float2 row = make_float2(0.f, 0.f);
#pragma unroll
          for (int jx = 0; jx < J; ++jx) rmac(row, rx[jx], G::to_f2(tp[jx]));
          rmac(zacc, ry[jy], row);
        }
        rmac(acc, rz[jz], zacc);
      }
      const float2 res = cmul(cscale(acc, inv_scale), ph);
      out[ent.x] = res;
      if (ent.y != kNoTwin) out[ent.y] = res;
    }
    __syncthreads();  // buffer b is refilled two subproblems on
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int J, typename G>
static cudaError_t launch_gather_v11_t(const InterpGeom& g, const void* grid, const int4* subs, int n_subs,
                                       float2* out, cudaStream_t st) {
  auto f = k_gather_v11<J, G>;
  const size_t smem = 2 * v11_tile_bytes<J>((int)sizeof(typename G::T));
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V10_NT, smem);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const long long want = (long long)num_sms() * per_sm;
  const int n_cta = (int)(want < n_subs ? want : n_subs);
  f<<<n_cta, V10_NT, smem, st>>>(g, (const typename G::T*)grid, subs, n_subs, out);
  return cudaGetLastError();
}

template <int J>
static cudaError_t launch_gather_v11_j(const InterpGeom& g, int dtype, const void* grid, const int4* subs,
                                       int n_subs, float2* out, cudaStream_t st) {
  switch (dtype) {
    case 0: return launch_gather_v11_t<J, GridC64>(g, grid, subs, n_subs, out, st);
    case 1: return launch_gather_v11_t<J, GridBF16>(g, grid, subs, n_subs, out, st);
    case 2: return launch_gather_v11_t<J, GridF16>(g, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gather_sched_pipelined(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs,
                                          int n_subs, float2* out, cudaStream_t st) {
  if (!g.sched || !v10_supported(g.T, g.J, g.S)) return cudaErrorInvalidValue;
  switch (g.J) {
    case 2: return launch_gather_v11_j<2>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 4: return launch_gather_v11_j<4>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 6: return launch_gather_v11_j<6>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 8: return launch_gather_v11_j<8>(g, grid_dtype, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

bool v10_supported(int T, int J, int S) {
  return T == 8 && (J == 2 || J == 4 || J == 6 || J == 8) && S >= 1 && S <= 256;
}

cudaError_t launch_gather_sched(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                                float2* out, cudaStream_t st) {
  if (!g.sched || !v10_supported(g.T, g.J, g.S)) return cudaErrorInvalidValue;
  switch (g.J) {
    case 2: return launch_gather_v10_j<2>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 4: return launch_gather_v10_j<4>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 6: return launch_gather_v10_j<6>(g, grid_dtype, grid, subs, n_subs, out, st);
    case 8: return launch_gather_v10_j<8>(g, grid_dtype, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// spread 8: the real-weight fixed-point spread, thread per point, with the
// plan's conflict schedule.  Persistent CTAs of 128 threads take subproblems
// (at most 256 points) from a work counter:
//  phase 1: the CTA's exponent from the largest |v| B_p over its points, B_p
//           = max|rho_x| max|rho_y| max|rho_z| of point p, kept by the plan
//           (k_point_bounds, the kernels' own arithmetic);
//  phase 2: thread k serves slot k of the schedule: it decodes its point,
//           evaluates the real weights and folds e^{-i gamma (ux+uy+uz)/2} v
//           into the z row in registers, then adds its J^3 taps, two int32
//           reductions each.  The 32 slots of a warp hold points with base
//           offsets distinct modulo 32 cells (the tile's plane pitch is the
//           subproblem's), so every reduction instruction is one wavefront,
//           and nothing is broadcast through shared memory;
//           a subproblem of points at the origin (all alike) sums their
//           values first and spreads the one point, thread per tap;
//  flush:   the tile added to the grid; the inverse z pass applies the grid
//           phase e^{+i gamma (kx+ky+kz)/2}.
// With only the tile in shared memory, several CTAs share an SM, so one
// waiting at a barrier leaves the SM to the others.
// ---------------------------------------------------------------------------
constexpr int V8S_THREADS = 128, V8S_WARPS = V8S_THREADS / 32, V8S_MAX_PTS = 256;

template <int J>
struct V8SLayout {
  static constexpr int E = 8 + J - 1;
  static constexpr int PPMAX = E * E + kSpreadPitchCodes - 1, CELLS = E * PPMAX;
  static constexpr size_t tre = 0;
  static constexpr size_t tim = tre + (size_t)CELLS * sizeof(int);
  static constexpr size_t red = tim + (size_t)CELLS * sizeof(int);  // [warps] x 3 words
  static constexpr size_t nxt = red + (size_t)V8S_WARPS * 3 * sizeof(float);
  static constexpr size_t bytes = (nxt + 2 * sizeof(int) + 15) / 16 * 16;
};

// B_p = max|rho_x| max|rho_y| max|rho_z| of every evaluated point, in the
// order of the sorted point list (plan time).
template <int J>
__global__ void k_point_bounds(InterpGeom g, long long P, float* __restrict__ cb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int w0[3], fm[3];
  float f[3];
  float2 ph;
  decode_point_real<J>(g, g.sorted[i].x, w0, f, fm, ph);
  float m = 1.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float r[J];
    real_coeffs<J>(g.rpoly, f[a], fm[a], r);
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < J; ++q) mx = fmaxf(mx, fabsf(r[q]));
    m *= mx;
  }
  cb[i] = m;
}

cudaError_t launch_point_bounds(const InterpGeom& g, long long P, float* cb, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((P + 255) / 256);
  switch (g.J) {
    case 2: k_point_bounds<2><<<blocks, 256, 0, st>>>(g, P, cb); break;
    case 4: k_point_bounds<4><<<blocks, 256, 0, st>>>(g, P, cb); break;
    case 6: k_point_bounds<6><<<blocks, 256, 0, st>>>(g, P, cb); break;
    case 8: k_point_bounds<8><<<blocks, 256, 0, st>>>(g, P, cb); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int J>
__global__ void __launch_bounds__(V8S_THREADS, 8) k_spread_v8(InterpGeom g, const float2* __restrict__ in,
                                                             const int4* __restrict__ subs, int n_subs,
                                                             int* __restrict__ counter, float2* __restrict__ grid,
                                                             float budget, float inv_budget) {
  using Lay = V8SLayout<J>;
  constexpr int T = 8, E = Lay::E, E2 = E * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* tre = (int*)(smem_raw + Lay::tre);
  int* tim = (int*)(smem_raw + Lay::tim);
  float* red = (float*)(smem_raw + Lay::red);  // [warps][3]: bound (max or sum), sum of v' (uniform)
  int* nxt = (int*)(smem_raw + Lay::nxt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nT = g.nT, K = g.K;
  const size_t KK = (size_t)K * K;
  for (int i = tid; i < Lay::CELLS; i += V8S_THREADS) {
    tre[i] = 0;
    tim[i] = 0;
  }
  if (tid == 0) nxt[0] = atomicAdd(counter, 1);
  __syncthreads();
  int s = nxt[0], parity = 0;
  while (s < n_subs) {
    const int4 sp = subs[s];
    const int4 sc = g.sched[s];
    const bool uniform = (sp.w & 1) != 0;
    const int PP = E2 + (sc.w >> 16), nslots = sc.w & 0xffff;
    const int x0 = (sp.x % nT) * T, y0 = ((sp.x / nT) % nT) * T, z0 = (sp.x / (nT * nT)) * T;
    // phase 1: the exponent (bounds are >= 0 or NaN: their bits order like the
    // values, and a NaN wins); points at the origin are summed, so their bound
    // is the sum, and their values are summed here too
    float bmax = 0.f, bsum = 0.f;
    float2 vsum = make_float2(0.f, 0.f);
    for (int i = tid; i < sp.z; i += V8S_THREADS) {
      const uint2 ent = g.sorted[sp.y + i];
      float2 val = in[ent.x];
      if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
      const float b = hypotf(val.x, val.y) * g.cbound[sp.y + i];
      bmax = __uint_as_float(max(__float_as_uint(bmax), __float_as_uint(b)));
      bsum += b;
      vsum = cadd(vsum, val);  // points at the origin: phase 1, e^{0} = 1
    }
    {
      const unsigned wb = __reduce_max_sync(0xffffffffu, __float_as_uint(bmax));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
        vsum.x += __shfl_xor_sync(0xffffffffu, vsum.x, o);
        vsum.y += __shfl_xor_sync(0xffffffffu, vsum.y, o);
      }
      if (lane == 0) {
        red[warp * 3] = uniform ? bsum : __uint_as_float(wb);
        red[warp * 3 + 1] = vsum.x;
        red[warp * 3 + 2] = vsum.y;
      }
    }
    if (tid == 0) nxt[parity ^ 1] = atomicAdd(counter, 1);
    __syncthreads();
    unsigned bb = 0u;
    float2 vtot = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < V8S_WARPS; ++w) {
      if (uniform) bb = __float_as_uint(__uint_as_float(bb) + red[w * 3]);
      else bb = max(bb, __float_as_uint(red[w * 3]));
      vtot.x += red[w * 3 + 1];
      vtot.y += red[w * 3 + 2];
    }
    const bool poison = bb > kBoundLimitBits;
    int e_tile = kTileEmpty;
    if (!poison && bb != 0u) {
      e_tile = max((int)(bb >> 23) - 127 + ((bb & 0x7FFFFFu) ? 1 : 0), -100);
      const float scl = budget * pow2f(-e_tile);
      if (!uniform) {
        const uint16_t* slots = g.sslots + sc.z;
        for (int k = tid; k < nslots; k += V8S_THREADS) {
          const int li = slots[k];
          if (li == 0xffff) continue;
          const uint2 ent = g.sorted[sp.y + li];
          int w0[3], fm[3];
          float f[3];
          float2 ph;
          decode_point_real<J>(g, ent.x, w0, f, fm, ph);
          const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
          if ((unsigned)lx >= (unsigned)T || (unsigned)ly >= (unsigned)T || (unsigned)lz >= (unsigned)T) {
            atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
            continue;
          }
          float2 val = in[ent.x];
          if (ent.y != kNoTwin) val = cadd(val, in[ent.y]);
          const float2 vp = cmulc(val, ph);  // e^{-i gamma sum u / 2} v
          float rx[J], ry[J], rz[J];
          real_coeffs<J>(g.rpoly, f[0], fm[0], rx);
          real_coeffs<J>(g.rpoly, f[1], fm[1], ry);
          real_coeffs<J>(g.rpoly, f[2], fm[2], rz);
          float z[2 * J];
#pragma unroll
          for (int q = 0; q < J; ++q) {
            z[2 * q] = vp.x * rz[q];
            z[2 * q + 1] = vp.y * rz[q];
            ry[q] *= scl;
          }
          const int mo = lz * PP + ly * E + lx;
          int* re = tre + mo;
          int* im = tim + mo;
#pragma unroll
          for (int jy = 0; jy < J; ++jy) {
#pragma unroll
            for (int jx = 0; jx < J; ++jx) {
              const float w = rx[jx] * ry[jy];
              int* pr = re + jy * E + jx;
              int* pi = im + jy * E + jx;
#pragma unroll
              for (int jz = 0; jz < J; ++jz) {
                atomicAdd(pr + jz * PP, round_unit1(w, z[2 * jz]));
                atomicAdd(pi + jz * PP, round_unit1(w, z[2 * jz + 1]));
              }
            }
          }
        }
      } else if (sp.z > 0) {
        // points at the origin: u = 0 for every one (weights alike, no phase);
        // the summed value is spread once, thread per tap
        const uint2 ent = g.sorted[sp.y];
        int w0[3], fm[3];
        float f[3];
        float2 ph;
        decode_point_real<J>(g, ent.x, w0, f, fm, ph);
        const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
        if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
          const float2 vp = cmulc(vtot, ph);
          float rx[J], ry[J], rz[J];
          real_coeffs<J>(g.rpoly, f[0], fm[0], rx);
          real_coeffs<J>(g.rpoly, f[1], fm[1], ry);
          real_coeffs<J>(g.rpoly, f[2], fm[2], rz);
          const int mo = lz * PP + ly * E + lx;
          for (int t = tid; t < J * J * J; t += V8S_THREADS) {
            const int jx = t % J, jy = (t / J) % J, jz = t / (J * J);
            float wx = 0.f, wy = 0.f, wz = 0.f;
#pragma unroll
            for (int q = 0; q < J; ++q) {
              wx = q == jx ? rx[q] : wx;
              wy = q == jy ? ry[q] : wy;
              wz = q == jz ? rz[q] : wz;
            }
            const float w = wx * wy * scl;
            const int o = mo + jz * PP + jy * E + jx;
            atomicAdd(tre + o, round_unit1(w, vp.x * wz));
            atomicAdd(tim + o, round_unit1(w, vp.y * wz));
          }
        } else if (tid == 0) {
          atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
        }
      }
    }
    __syncthreads();
    const int s_next = nxt[parity ^ 1];
    // flush: the tile added to the grid (the inverse z pass applies the grid phase)
    const float inv = e_tile == kTileEmpty ? 0.f : inv_budget * pow2f(e_tile);
    const float qnan = __int_as_float(0x7fc00000);
    // only the plan's box of the tile can hold values
    const TileBox bx = unpack_box(g.box, s, E);
    const float inv_ex = 1.f / (float)bx.ex;
    for (int cc = tid; cc < bx.ex * bx.ey; cc += V8S_THREADS) {
      const int r = (int)(((float)cc + 0.5f) * inv_ex);
      const int ix = bx.ox + cc - r * bx.ex, iy = bx.oy + r, c = iy * E + ix;
      int gx = x0 + ix, gy = y0 + iy;
      gx -= gx >= K ? K : 0;
      gy -= gy >= K ? K : 0;
      float2* col = grid + (size_t)gy * K + gx;
      int gz = z0 + bx.oz;
#pragma unroll
      for (int t = 0; t < E; ++t) {
        if (t >= bx.ez) break;
        const int idx = c + (bx.oz + t) * PP;
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

bool v8s_supported(int T, int J, int S) {
  if (T != 8 || S < 1 || S > V8S_MAX_PTS) return false;
  size_t b = 0;
  switch (J) {
    case 2: b = V8SLayout<2>::bytes; break;
    case 4: b = V8SLayout<4>::bytes; break;
    case 6: b = V8SLayout<6>::bytes; break;
    case 8: b = V8SLayout<8>::bytes; break;
    default: return false;
  }
  return b <= (size_t)max_optin_smem();
}

template <int J>
static cudaError_t launch_spread_v8_j(const InterpGeom& g, const float2* in, const int4* subs, int n_subs,
                                      float2* grid, cudaStream_t st) {
  auto f = k_spread_v8<J>;
  const size_t smem = V8SLayout<J>::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V8S_THREADS, smem);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const float budget = ldexpf(1.f - 1.f / 1024.f, 22);  // at most 256 points per subproblem
  e = cudaMemsetAsync(g.counter + 1, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  f<<<num_sms() * per_sm, V8S_THREADS, smem, st>>>(g, in, subs, n_subs, g.counter + 1, grid, budget, 1.f / budget);
  return cudaGetLastError();
}

cudaError_t launch_spread_sched(const InterpGeom& g, const float2* in, const int4* subs, int n_subs, float2* grid,
                                cudaStream_t st) {
  if (!g.sched || !g.cbound || !v8s_supported(g.T, g.J, g.S)) return cudaErrorInvalidValue;
  switch (g.J) {
    case 2: return launch_spread_v8_j<2>(g, in, subs, n_subs, grid, st);
    case 4: return launch_spread_v8_j<4>(g, in, subs, n_subs, grid, st);
    case 6: return launch_spread_v8_j<6>(g, in, subs, n_subs, grid, st);
    case 8: return launch_spread_v8_j<8>(g, in, subs, n_subs, grid, st);
  }
  return cudaErrorInvalidValue;
}
// ---------------------------------------------------------------------------
// a group of plans (one batch launch each for the gather and the spread)
// ---------------------------------------------------------------------------
cudaError_t launch_group_gather(const GroupParams& gp, const GroupItem* items, cudaStream_t st) {
  auto f = k_gather_v10<6, GridC64, GroupGatherSrc>;
  const size_t smem = v10_bytes<6>(8);
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int total = gp.work_begin[gp.n_items];
  if (total == 0) return cudaSuccess;
  const GroupGatherSrc src{gp, items};
  f<<<total, V10_NT, smem, st>>>(src, gp.nT, 1.f, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_group_spread(const GroupParams& gp, const GroupItem* items, int* counter, cudaStream_t st) {
  auto f = k_spread_v7<GroupSpreadSrc>;
  const size_t smem = V7SLayout::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int total = gp.work_begin[gp.n_items];
  if (total == 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V7S_THREADS, smem);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const float budget = ldexpf(1.f - 1.f / 1024.f, 22);  // at most 256 points per subproblem
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const GroupSpreadSrc src{gp, items};
  f<<<num_sms() * per_sm, V7S_THREADS, smem, st>>>(src, total, gp.nT, counter, budget, 1.f / budget);
  return cudaGetLastError();
}

}  // namespace nufft
