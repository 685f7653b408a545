// Gather variant 8 (J = 6, T = 8): the one-thread-per-point gather of variant
// 5 made persistent, with the grid tile of the next subproblem brought into
// shared memory by a TMA tensor copy (cp.async.bulk.tensor, completion counted
// on an mbarrier) while the current subproblem is decoded, ordered and
// interpolated.  Two tile buffers alternate, so the tile loads no longer stall
// the warps on global-memory latency.
//
// The copied box is 14 x 13 x 13 cells for complex64 cells (16 x 13 x 13 for
// 4-byte bf16 / fp16 cells): a box row must be a whole number of 16-byte units,
// so the row pitch in shared memory is 14 (16) cells and the last cells of a row
// are copied but never read.  Every tile origin x0 = 8 bx starts on a 16-byte
// boundary.  A tile that wraps around the periodic grid edge (x0 + 13 > K on
// some axis) cannot be one box; the threads load it instead.
//
// Every wait on an mbarrier is bounded: a copy that does not complete within
// the limit sets NUFFT3D_ERR_TIMEOUT in the device check word; the CTA then
// waits (bounded again, with the full limit) for both of its copies that may
// still be in flight, and returns.  The limit of the first wait on each copy is
// a launch parameter so that tests can make it run out.
#include <cudaTypedefs.h>

#include "interp_common.cuh"

namespace nufft {

constexpr int V8_NT = 128;
constexpr int V8_T = 8, V8_J = 6, V8_E = V8_T + V8_J - 1;  // 13
constexpr int kTmaWaitLimit = 1 << 22;                     // try_wait polls before giving up

template <int ELEM>
struct V8Geo {
  static constexpr int EX = ELEM == 8 ? 14 : 16;                  // row pitch (box x extent) in cells
  static constexpr int TILE_BYTES = EX * V8_E * V8_E * ELEM;      // bytes one box copy delivers
  static constexpr int TILE_STRIDE = (TILE_BYTES + 127) / 128 * 128;
  static constexpr int KRES = 128 / ELEM;                         // residue classes of a conflict-free access
};

// dynamic shared memory: 128 B of slack to align the tiles, two tiles, two
// mbarriers and two flags (32 B), the point arrays (7 words per point) and two
// sets of class counters and cursors
__host__ __device__ inline size_t v8_bytes(int S, int elem) {
  const int ex = elem == 8 ? 14 : 16;
  const size_t tile = ((size_t)ex * V8_E * V8_E * elem + 127) / 128 * 128;
  const int kres = 128 / elem;
  return 128 + 2 * tile + 32 + (size_t)S * 7 * sizeof(int) + (size_t)4 * kres * sizeof(int);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit = kTmaWaitLimit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <typename G>
__global__ void __launch_bounds__(V8_NT, 5) k_gather_v8(InterpGeom g, const __grid_constant__ CUtensorMap tmap,
                                                        const typename G::T* __restrict__ grid,
                                                        const int4* __restrict__ subs, int n_subs, int S,
                                                        float2* __restrict__ out, int first_wait_limit) {
  typedef typename G::T TT;
  typedef V8Geo<(int)sizeof(TT)> Geo;
  constexpr int J = V8_J, T = V8_T, E = V8_E, EX = Geo::EX, PP = E * EX, kRes = Geo::KRES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned long long* bars = (unsigned long long*)(base + 2 * Geo::TILE_STRIDE);
  int* manual = (int*)(bars + 2);  // [2] tile loaded by the threads (wraps the grid edge)
  int* p_id = manual + 4;
  int* p_tw = p_id + S;
  int* p_off = p_tw + S;
  float* p_f = (float*)(p_off + S);  // [3][S]
  int* order = (int*)(p_f + 3 * S);
  int* ncls = order + S;  // [2 stages][kRes counts, kRes cursors]
  const float inv_scale = lp_inv_scale<G>(g);
  const int nT = g.nT, K = g.K, tid = threadIdx.x;
  const uint32_t bar0 = smem_u32(&bars[0]);  // stage st uses bar0 + 8 st
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 4 * kRes) ncls[tid] = 0;
  __syncthreads();

  // thread 0: start the copy of subproblem s's tile into buffer st
  auto issue = [&](int s, int st) {
    const int4 sp = subs[s];
    const int x0 = (sp.x % nT) * T, y0 = ((sp.x / nT) % nT) * T, z0 = (sp.x / (nT * nT)) * T;
    const bool wrap = x0 + E > K || y0 + E > K || z0 + E > K;
    manual[st] = wrap ? 1 : 0;
    if (!wrap) {
      // order the generic-proxy reads of the previous use of this buffer before the copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar0 + 8 * st, (uint32_t)Geo::TILE_BYTES);
      tma_load_3d(smem_u32(base + st * Geo::TILE_STRIDE), &tmap, x0, y0, z0, bar0 + 8 * st);
    }
  };

  uint32_t parity = 0;  // bit st: parity of the next completion of bars[st]
  int st = 0;
  if (tid == 0 && (int)blockIdx.x < n_subs) issue(blockIdx.x, 0);
  for (int s = blockIdx.x; s < n_subs; s += gridDim.x, st ^= 1) {
    const int nxt = s + gridDim.x;
    if (tid == 0 && nxt < n_subs) issue(nxt, st ^ 1);
    int* cls = ncls + st * 2 * kRes;
    const int4 sp = subs[s];
    const int bx = sp.x % nT, by = (sp.x / nT) % nT, bz = sp.x / (nT * nT);
    const int x0 = bx * T, y0 = by * T, z0 = bz * T;
    const int cnt = sp.z;
    // decode every point once
    for (int i = tid; i < cnt; i += V8_NT) {
      const uint2 ent = g.sorted[sp.y + i];
      int w0[3];
      float f[3];
      decode_point<J>(g, ent.x, w0, f);
      const int lx = w0[0] - x0, ly = w0[1] - y0, lz = w0[2] - z0;
      int off = -1;
      if ((unsigned)lx < (unsigned)T && (unsigned)ly < (unsigned)T && (unsigned)lz < (unsigned)T) {
        off = (lz * E + ly) * EX + lx;
      } else {
        atomicExch(g.err, (int)DEVCHK_TILE_RANGE);
      }
      p_id[i] = (int)ent.x;
      p_tw[i] = (int)ent.y;
      p_off[i] = off;
      p_f[i] = f[0];
      p_f[S + i] = f[1];
      p_f[2 * S + i] = f[2];
      atomicAdd(&cls[off < 0 ? 0 : (off & (kRes - 1))], 1);
    }
    __syncthreads();
    // rank within the residue class, then the round-robin position
    for (int i = tid; i < cnt; i += V8_NT) {
      const int c = p_off[i] < 0 ? 0 : (p_off[i] & (kRes - 1));
      const int r = atomicAdd(&cls[kRes + c], 1);
      int pos = 0;
#pragma unroll
      for (int q = 0; q < kRes; ++q) {
        const int n = cls[q];
        pos += n < r ? n : r;
        pos += (q < c && n > r) ? 1 : 0;
      }
      order[pos] = i;
    }
    __syncthreads();
    TT* tile = (TT*)(base + st * Geo::TILE_STRIDE);
    if (manual[st]) {
      for (int r = tid; r < E * E * E; r += V8_NT) {
        const int row = r / E, ix = r - row * E;
        const int iz = row / E, iy = row - iz * E;
        int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
        gx -= gx >= K ? K : 0;
        gy -= gy >= K ? K : 0;
        gz -= gz >= K ? K : 0;
        tile[(iz * E + iy) * EX + ix] = grid[((size_t)gz * K + gy) * K + gx];
      }
      __syncthreads();
    } else {
      const uint32_t ph = (parity >> st) & 1u;
      const bool ok = mbar_wait_bounded(bar0 + 8 * st, ph, first_wait_limit);
      parity ^= 1u << st;
      if (!__syncthreads_and(ok)) {
        // give up on this CTA, but not while a copy into its shared memory is
        // in flight: wait (with the full limit) for the copy into this buffer
        // and for the next one, if it was started
        if (tid == 0) atomicExch(g.err, (int)NUFFT3D_ERR_TIMEOUT);
        mbar_wait_bounded(bar0 + 8 * st, ph);
        if (nxt < n_subs && !manual[st ^ 1]) mbar_wait_bounded(bar0 + 8 * (st ^ 1), (parity >> (st ^ 1)) & 1u);
        return;
      }
    }
    // the next iteration's counters (their last reader finished before the barrier above)
    if (tid < 2 * kRes) ncls[(st ^ 1) * 2 * kRes + tid] = 0;
    for (int k = tid; k < cnt; k += V8_NT) {
      const int i = order[k];
      const int off = p_off[i];
      if (off < 0) continue;
      float2 cx[J], cy[J], cz[J];
      point_coeffs<J>(g, p_f[i], cx);
      point_coeffs<J>(g, p_f[S + i], cy);
      point_coeffs<J>(g, p_f[2 * S + i], cz);
      float2 acc = make_float2(0.f, 0.f);
      const TT* tb = tile + off;
#pragma unroll
      for (int jz = 0; jz < J; ++jz) {
        float2 zacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int jy = 0; jy < J; ++jy) {
          const TT* tp = tb + jz * PP + jy * EX;
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
    __syncthreads();
  }
}

bool v8_supported(int T, int J, int S, int elem) {
  return T == V8_T && J == V8_J && S >= 1 && v8_bytes(S, elem) <= (size_t)max_optin_smem();
}

// Tensor map of a K^3 grid of elem-byte cells (x fastest) with the 3D box the
// variant-8 gather copies.  Host only; false if the driver entry point is
// unavailable or the encoding is refused.
bool make_grid_tmap(CUtensorMap* map, const void* grid, int K, int elem) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode || !grid || (elem != 4 && elem != 8) || K < 16 || K % 16 != 0) return false;
  if (((uintptr_t)grid & 15u) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)K, (cuuint64_t)K};
  const cuuint64_t strides[2] = {(cuuint64_t)K * elem, (cuuint64_t)K * K * elem};
  const cuuint32_t box[3] = {(cuuint32_t)(elem == 8 ? V8Geo<8>::EX : V8Geo<4>::EX), (cuuint32_t)V8_E,
                             (cuuint32_t)V8_E};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                            const_cast<void*>(grid), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename G>
static cudaError_t launch_gather_v8_t(const InterpGeom& g, const CUtensorMap* tmap, const void* grid,
                                      const int4* subs, int n_subs, float2* out, cudaStream_t st) {
  auto f = k_gather_v8<G>;
  const size_t smem = v8_bytes(g.S, (int)sizeof(typename G::T));
  cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n_subs == 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, V8_NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long want = (long long)num_sms() * per_sm;
  const int n_cta = (int)(want < n_subs ? want : n_subs);
  const int first_limit = g.first_wait_polls >= 0 ? g.first_wait_polls : kTmaWaitLimit;
  f<<<n_cta, V8_NT, smem, st>>>(g, *tmap, (const typename G::T*)grid, subs, n_subs, g.S, out, first_limit);
  return cudaGetLastError();
}

cudaError_t launch_gather_tma(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                              float2* out, cudaStream_t st) {
  if (!g.tmap || g.T != V8_T || g.J != V8_J) return cudaErrorInvalidValue;
  switch (grid_dtype) {
    case 0: return launch_gather_v8_t<GridC64>(g, g.tmap, grid, subs, n_subs, out, st);
    case 1: return launch_gather_v8_t<GridBF16>(g, g.tmap, grid, subs, n_subs, out, st);
    case 2: return launch_gather_v8_t<GridF16>(g, g.tmap, grid, subs, n_subs, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nufft
