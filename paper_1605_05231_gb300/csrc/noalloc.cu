// Allocation-free adjoint: the same computation as nufft3d_adjoint, with every
// scratch buffer (line-DFT output, K^3 grid, the two inverse-FFT intermediates
// and the spread's work counter) carved from one file-scope device array
// instead of the plan's workspace.
//
// Some callers cannot allocate device memory at the point where they need the
// adjoint: code that runs while a stream is being captured into a CUDA graph
// in global capture mode, host frameworks whose device memory belongs to their
// own pool allocator, or real-time loops that must not enter the driver's
// allocator.  For them this entry point calls no cudaMalloc or cudaFree and no
// allocating library routine.  The array costs every GPU that loads the
// library kNoAllocScratchBytes of device memory until the process exits.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr size_t kAlignF2 = 32;                           // 256-byte alignment in float2 units
constexpr int kMaxDevices = 64;

__device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float2)];

std::mutex g_mu;
float2* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t round_up(size_t v) { return (v + kAlignF2 - 1) / kAlignF2 * kAlignF2; }

// Device address of the scratch array on the current device (looked up once
// per device; the symbol's name in host code is not a device address).
cudaError_t scratch_address(int dev, float2** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (float2*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

}  // namespace

extern "C" int nufft3d_adjoint_noalloc(nufft3d_plan pl, const void* lines_dev, void* vol_dev, void* cuda_stream) {
  if (!pl || !lines_dev || !vol_dev) return NUFFT3D_ERR_ARG;
  const int N = pl->N, K = pl->K;
  const long long KK = (long long)K * K;
  const size_t n_lines = pl->do_line_fft ? round_up((size_t)pl->P) : 0;
  const size_t n_grid = round_up((size_t)K * KK);
  const size_t n_b = round_up((size_t)N * KK);
  const size_t n_a = round_up((size_t)N * N * K);
  const size_t n_cnt = kAlignF2;
  if ((n_lines + n_grid + n_b + n_a + n_cnt) * sizeof(float2) > kNoAllocScratchBytes) return NUFFT3D_ERR_UNSUPPORTED;
  // the plan's device is current until return; the caller's device is restored then
  nufft::DeviceGuard guard(pl->device);
  if (guard.status != cudaSuccess) return status_of(guard.status);
  const int dev = pl->device;
  float2* base = nullptr;
  cudaError_t e = scratch_address(dev, &base);
  if (e != cudaSuccess) return status_of(e);
  float2* lines_tmp = base;
  float2* grid = lines_tmp + n_lines;
  float2* bufB = grid + n_grid;
  float2* bufA = bufB + n_b;
  int* counter = (int*)(bufA + n_a);
  cudaStream_t st = (cudaStream_t)cuda_stream;

  nufft::InterpGeom g;
  g.K = K;
  g.J = pl->J;
  g.L = pl->L;
  g.T = pl->T;
  g.nT = pl->nT;
  g.M = pl->M;
  g.D = pl->D;
  g.dir = pl->d_dir;
  g.rad = pl->d_rad;
  g.table = pl->d_table;
  g.sorted = pl->d_sorted;
  g.err = pl->d_err;
  g.counter = counter;
  g.S = pl->pts_per_sub;
  g.lp_bound = pl->d_lp_bound;
  g.poly = pl->poly;
  g.rpoly = pl->rpoly;
  g.phase = pl->d_phase;
  g.sched = pl->sched_ok ? pl->d_sched : nullptr;
  g.gslots = pl->d_gslots;
  g.sslots = pl->d_sslots;
  g.cbound = pl->d_cbound;
  g.box = pl->sched_ok ? pl->d_box : nullptr;

  const float2* src = (const float2*)lines_dev;
  if (pl->do_line_fft) {
    e = nufft::launch_line(pl->M, false, src, lines_tmp, pl->D, pl->d_weight, pl->d_twM, st, pl->d_line_weight);
    if (e != cudaSuccess) return status_of(e);
    src = lines_tmp;
  }
  // the array keeps the previous call's contents: the grid and the counters start at zero
  e = cudaMemsetAsync(grid, 0, (size_t)K * KK * sizeof(float2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = nufft::launch_spread(g, pl->spread_variant, src, pl->d_sub, pl->n_sub, grid, st);
  nufft::ColPrune pz{};
  if (nufft::spread_real(pl->spread_variant)) pz.phase = pl->d_phase;  // the real-weight spread's grid phase
  if (e == cudaSuccess) e = nufft::launch_col_inv(K, grid, bufB, N, K, K, K, KK, K, KK, pl->d_twK, st, pz);
  if (e == cudaSuccess) e = nufft::launch_col_inv(K, bufB, bufA, N, N, K, KK, K, (long long)N * K, K, pl->d_twK, st);
  if (e == cudaSuccess) e = nufft::launch_row_adj(K, bufA, vol_dev, pl->complex_volume, pl->d_s, N, pl->d_twK, st);
  return status_of(e);
}
