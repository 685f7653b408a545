// Internal declarations shared by the translation units of libnufft3d.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <vector>

#include "../../include/nufft3d.h"

namespace nufft {

constexpr uint32_t kNoTwin = 0xffffffffu;

// Makes `dev` the current device for the lifetime of the guard and then
// restores the device that was current before (every C-ABI call that takes a
// plan or a batch runs on its device and leaves the caller's choice alone).
struct DeviceGuard {
  int prev = -1;
  cudaError_t status = cudaSuccess;
  explicit DeviceGuard(int dev) {
    status = cudaGetDevice(&prev);
    if (status == cudaSuccess && prev != dev) status = cudaSetDevice(dev);
    if (status != cudaSuccess || prev == dev) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Exact min-max coefficients without a table: each c_j(f), f in [0, 1], is
// replaced by its degree-kPolyDeg Chebyshev interpolant (fitted in FP64 at plan
// time), stored as monomials in t = 2 f - 1 and evaluated per point by Horner's
// rule.  The coefficients travel in the kernel parameters, so every lane reads
// them through the constant bank.
constexpr int kPolyDeg = 8;
constexpr int kPolyMaxJ = 8;
struct CoefPoly {
  float a[kPolyMaxJ][2][kPolyDeg + 1];  // [tap][re, im][power of t]
};
// With the pre-window symmetric about the middle of the index range, the
// min-max coefficients factor as c_j(f) = e^{i gamma (f + J/2 - j)/2} rho_j(f)
// with rho_j real; the real-weight kernels evaluate rho_j from these fits and
// carry the phases on the point (e^{i gamma (ux + uy + uz)/2}) and on the grid
// cell (e^{-i gamma (kx + ky + kz)/2}, applied by the z passes).
struct RealPoly {
  float a[kPolyMaxJ][kPolyDeg + 1];  // [tap][power of t]
};

// point-to-tile binning and the interpolation kernels' view of a plan
struct InterpGeom {
  int K, J, L, T, nT, M, D;
  const float2* dir;     // [D][3] (hi, lo) direction components
  const float2* rad;     // [M] (hi, lo) radius in grid units
  const float2* table;   // [(L + 1) * J] min-max coefficients
  const uint2* sorted;   // (point id, coincident twin id or kNoTwin), sorted by tile
  int* err;              // device check word
  int* counter;          // two work counters (gather, spread) for the persistent variants
  int S;                 // most points in one subproblem
  const float* lp_bound; // bound on |Y| for a reduced-precision grid (else null)
  CoefPoly poly;         // coefficient polynomials (used when L == 0)
  RealPoly rpoly;        // real weights rho_j (real-weight variants, L == 0)
  const float2* phase = nullptr;  // K entries e^{-i gamma k_c / 2} (real-weight variants)
  const CUtensorMap* tmap = nullptr;  // host copy of the grid's tensor map (gather variant 8), or null
  int first_wait_polls = -1;          // polls of the first wait on each TMA copy (< 0: the default limit)
  const int4* sched = nullptr;        // per-subproblem conflict schedules (gather 10, spread 8), or null
  const uint16_t* gslots = nullptr;
  const uint16_t* sslots = nullptr;
  const float* cbound = nullptr;      // per sorted point max|rho_x| max|rho_y| max|rho_z| (spread 8), or null
  const int* box = nullptr;           // per subproblem, the tile cells its taps can reach (TileBox), or null
};

// What decoding a point needs: the grid edge, the samples per line and the
// lines' directions and radii (InterpGeom has the same members).
struct PointGeom {
  int K, M;
  const float2* dir;
  const float2* rad;
};

// One item of a group of plans that share N, K and J (and so the coefficient
// polynomials, the phase table and the tiling), as the grouped interpolation
// kernels of a batch see it.
struct GroupItem {
  PointGeom pg;
  const uint2* sorted;
  const int4* subs;
  int n_subs;
  int sub_begin;          // first global work item of this plan
  const int4* sched;
  const uint16_t* gslots;
  const int* box;
  int* err;
  const float2* grid;     // forward grid (gather)
  float2* lines;          // forward output (gather)
  const float2* adj_in;   // adjoint line-DFT output (spread)
  float2* adj_grid;       // adjoint grid (spread)
};

// The part of a subproblem's E^3 tile its taps can reach, from the plan:
// origin and extent per axis (the whole tile without a plan box).
struct TileBox {
  int ox, ex, oy, ey, oz, ez;
};
__host__ __device__ inline TileBox unpack_box(const int* box, int s, int E) {
  TileBox b{0, E, 0, E, 0, E};
  if (box) {
    const int c = box[s];
    b.ox = c & 15;
    b.ex = (c >> 4) & 31;
    b.oy = (c >> 9) & 15;
    b.ey = (c >> 13) & 31;
    b.oz = (c >> 18) & 15;
    b.ez = (c >> 22) & 31;
  }
  return b;
}

// Pruning of the column FFT passes to the cells the interpolation touches:
// the ball |k| <= R in centred grid frequencies (R = K/2 + (J/2) sqrt 3 + 1
// covers every tap of every point with |u| <= K/2).  mode 1: y passes (rows
// ky, column kx; test kx^2 + ky^2 <= r2); mode 2: z passes (rows kz, columns
// (kx, ky = outer index); columns outside the disk skipped, rows tested with
// the ball).  Forward passes skip whole-row stores no column needs, inverse
// passes skip the loads of cells outside the ball (which are not cleared).
struct ColPrune {
  int mode = 0;
  int K = 0;
  long long r2 = 0;
  int consume = 0;  // inverse z pass: zero every grid row it reads (the adjoint grid is left clear)
  // z passes only: per-cell phase e^{-i gamma (kx + ky + kz)/2} (centred k) of the
  // real-weight interpolation kernels, from the K-entry table phase[k] =
  // e^{-i gamma k_c / 2}: the forward pass multiplies its output by it, the
  // inverse pass its input by the conjugate.  Null: no phase.
  const float2* phase = nullptr;
};

bool fft_length_supported(int L);
cudaError_t launch_row_fwd(int K, const void* vol, int cplx, float2* out, const float* s, int N,
                           const float2* tw, cudaStream_t st);
cudaError_t launch_row_adj(int K, const float2* in, void* vol, int cplx, const float* s, int N,
                           const float2* tw, cudaStream_t st);
cudaError_t launch_col_fwd(int L, const float2* in, float2* out, int N, int n_outer, int row_len,
                           long long in_outer, long long in_stride, long long out_outer, long long out_stride,
                           const float2* tw, cudaStream_t st, ColPrune pr = ColPrune{});
cudaError_t launch_col_fwd_lp(int L, int dtype, const float2* in, void* out, int N, int n_outer, int row_len,
                              long long in_outer, long long in_stride, long long out_outer,
                              long long out_stride, const float2* tw, const float* bound, cudaStream_t st,
                              ColPrune pr = ColPrune{});
cudaError_t launch_abs_bound(const void* vol, int cplx, const float* s, int N, float* bound, cudaStream_t st);
cudaError_t launch_col_inv(int L, const float2* in, float2* out, int N, int n_outer, int row_len,
                           long long in_outer, long long in_stride, long long out_outer, long long out_stride,
                           const float2* tw, cudaStream_t st, ColPrune pr = ColPrune{});
cudaError_t launch_line(int M, bool fwd, const float2* in, float2* out, int D, const float2* w,
                        const float2* tw, cudaStream_t st, const float* lw = nullptr);

cudaError_t launch_bin_points(const InterpGeom& g, const uint32_t* ids, long long count, uint32_t* bins,
                              cudaStream_t st);
// subs: int4 (bin, start, count, 0); variant 0 = thread per point, 1 = warp per point
cudaError_t launch_gather(const InterpGeom& g, int variant, int grid_dtype, const void* grid, float inv_scale,
                          const int4* subs, int n_subs, float2* out, cudaStream_t st);
cudaError_t launch_spread(const InterpGeom& g, int variant, const float2* in, const int4* subs, int n_subs,
                          float2* grid, cudaStream_t st);
size_t interp_smem_bytes(int T, int J);
bool v2_supported(int T, int J, int L);
// enqueue a plan's forward / adjoint on a stream (no argument checks; used by batches)
int plan_forward_enqueue(nufft3d_plan pl, const void* vol, void* lines, cudaStream_t st);
int plan_adjoint_enqueue(nufft3d_plan pl, const void* lines, void* vol, cudaStream_t st);
// parts of a call (bit 0: before the interpolation, 1: the interpolation, 2: after it)
int plan_forward_parts(nufft3d_plan pl, const void* vol, void* lines, cudaStream_t st, int parts);
int plan_adjoint_parts(nufft3d_plan pl, const void* lines, void* vol, cudaStream_t st, int parts);
// one launch over a group of plans sharing N, K and J (the scheduled gather,
// variant 10, and the real-weight spread, variant 7; complex64 grids)
constexpr int kMaxGroupItems = 32;
struct GroupParams {
  RealPoly rpoly;
  int K, nT, n_items;
  int work_begin[kMaxGroupItems + 1];  // first work item of every plan, then the total
};
cudaError_t launch_group_gather(const GroupParams& gp, const GroupItem* items, cudaStream_t st);
cudaError_t launch_group_spread(const GroupParams& gp, const GroupItem* items, int* counter, cudaStream_t st);
bool v3_supported(int T, int J, int S);
bool v3_two_copy_supported(int T, int J, int S);
bool v8_supported(int T, int J, int S, int elem);
bool make_grid_tmap(CUtensorMap* map, const void* grid, int K, int elem);
cudaError_t launch_gather_tma(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                              float2* out, cudaStream_t st);
bool v4_supported(int T, int J, int S, int L);
bool v3s_supported(int T, int J);
bool v4s_supported(int T, int J, int S);
bool v5s_supported(int T, int J, int S);
bool v6s_supported(int T, int J, int S);
bool v9_supported(int T, int J, int S);
bool v7s_supported(int T, int J, int S);
cudaError_t launch_gather_real(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                               float2* out, cudaStream_t st);
cudaError_t launch_spread_real(const InterpGeom& g, const float2* in, const int4* subs, int n_subs, float2* grid,
                               cudaStream_t st);
// the variants with real weights and phases (they need the phased grid)
inline bool gather_real(int variant) { return variant == 9 || variant == 10 || variant == 11; }
inline bool spread_real(int variant) { return variant == 7 || variant == 8; }
bool v10_supported(int T, int J, int S);
bool v8s_supported(int T, int J, int S);
cudaError_t launch_gather_sched(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs, int n_subs,
                                float2* out, cudaStream_t st);
cudaError_t launch_gather_sched_pipelined(const InterpGeom& g, int grid_dtype, const void* grid, const int4* subs,
                                          int n_subs, float2* out, cudaStream_t st);
cudaError_t launch_spread_sched(const InterpGeom& g, const float2* in, const int4* subs, int n_subs, float2* grid,
                                cudaStream_t st);
cudaError_t launch_point_bounds(const InterpGeom& g, long long P, float* cb, cudaStream_t st);
// plane pitches of the scheduled kernels' tiles: E^2 + code, code < 16 (gather) or < 32 (spread)
constexpr int kGatherPitchCodes = 16, kSpreadPitchCodes = 32;

}  // namespace nufft

constexpr int FWD_STAGES = 5;  // x pass, y pass, z pass, gather, line DFT
constexpr int ADJ_STAGES = 6;  // line DFT, grid clear, spread, z pass, y pass, x pass

struct nufft3d_plan_s {
  // resolved parameters
  int N, K, J, L, D, M;  // L = 0: exact coefficients from the fitted polynomials
  long long P;
  nufft::CoefPoly poly{};
  nufft::RealPoly rpoly{};
  bool real_ok = false;         // the real-weight variants may run (exact coefficients, phase table built)
  float2* d_phase = nullptr;    // K entries e^{-i gamma k_c / 2}
  CUtensorMap tmap_grid{};  // tensor map of the grid the gather reads (d_grid or d_grid_lp)
  bool tmap_ok = false;
  double poly_err = 0.0;  // max |fit - exact| / max |c| of the polynomials (0 with a table)
  long long ball_r2 = 0;  // squared radius of the ball of grid cells the interpolation touches
  int complex_volume, do_line_fft, grid_dtype;
  int T, nT;  // tile edge and tiles per axis
  int gather_variant, spread_variant, pts_per_sub;
  float* d_lp_bound = nullptr;  // device bound on |Y| (reduced-precision grid)
  int device;
  // device arrays (owned)
  float2* d_dir = nullptr;
  float2* d_rad = nullptr;
  float2* d_weight = nullptr;  // null when w = 1
  float* d_line_weight = nullptr;  // D real per-line weights, null when 1
  float* d_s = nullptr;
  float2* d_table = nullptr;
  float2* d_twK = nullptr;
  float2* d_twM = nullptr;
  uint2* d_sorted = nullptr;      // (id, twin) per evaluated point, sorted by tile
  uint32_t* d_unique = nullptr;   // ids of the evaluated points (plan time only)
  std::vector<uint32_t> h_unique; // same, host copy
  std::vector<uint32_t> h_twin;   // twin of each evaluated point (kNoTwin if none)
  long long P_eval = 0;           // number of evaluated points
  int n_pairs = 0;                // antipodal line pairs merged
  int4* d_sub = nullptr;
  int n_sub = 0;
  float2* d_grid = nullptr;   // K^3 (forward grid; also the adjoint grid with a reduced-precision forward grid)
  float2* d_grid_adj = nullptr;  // K^3 adjoint grid with a complex64 forward grid (kept clear between calls)
  bool adj_dirty = false;        // the adjoint grid may hold values (a call stopped before the z pass)
  void* d_grid_lp = nullptr;  // K^3 reduced precision (grid_dtype != 0)
  float2* d_bufA = nullptr;   // N * N * K
  float2* d_bufB = nullptr;   // N * K * K
  float2* d_lines = nullptr;  // D * M (adjoint line DFT output)
  int* d_err = nullptr;
  int* d_counter = nullptr;  // [2]
  // optional per-stage CUDA-event timing (ring of event sets, one per call)
  int timing_slots = 0, fwd_calls = 0, adj_calls = 0;
  std::vector<cudaEvent_t> ev_fwd, ev_adj;  // slots * (FWD_STAGES + 1), slots * (ADJ_STAGES + 1)
  // host copy of the per-bin offsets (for re-tuning the subproblem split)
  std::vector<long long> bin_offsets;
  std::vector<int> bin_dc;          // per bin: its leading points at the origin (radius 0)
  std::vector<uint2> h_sorted;      // host copy of d_sorted
  std::vector<int4> h_sub;          // host copy of d_sub
  std::vector<float2> h_dir, h_rad; // host copies of d_dir, d_rad
  // conflict schedules of the thread-per-point real-weight kernels (gather 10,
  // spread 8), one int4 per subproblem: (gather slot start, gather slots |
  // plane-pitch code << 16, spread slot start, spread slots | code << 16); the
  // slots hold the subproblem-local point index or 0xffff (an idle lane)
  int4* d_sched = nullptr;
  uint16_t* d_gslots = nullptr;
  uint16_t* d_sslots = nullptr;
  float* d_cbound = nullptr;  // per sorted point: max|rho_x| max|rho_y| max|rho_z|
  int* d_box = nullptr;       // per subproblem: packed TileBox
  bool sched_ok = false;
  cudaStream_t last_stream = nullptr;
  int first_wait_polls = -1;  // testing hook of nufft3d_plan_set_wait_limit (< 0: default)
};
