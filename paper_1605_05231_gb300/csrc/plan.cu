// Host side of libnufft3d: parameter validation, FP64 plan precompute (the
// Kaiser-Bessel deapodisation factors of Eq. 2.11, the min-max interpolation
// table, FFT twiddles, direction and radius splits), the point sort by grid
// tile, workspace management and the orchestration of the forward and adjoint
// passes.  Every entry point of include/nufft3d.h is defined here.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_math.h"
#include "internal.h"

using nufft::InterpGeom;
typedef std::complex<double> cd;
using nufft::fit_coeff_polys;
using nufft::invert;
using nufft::kb_ft;

namespace {

struct Resolved {
  int N, K, J, L, D, M, grid_dtype, cplx, line_fft, keep_dup, exact;
  long long P;
  int T, nT;
};

constexpr int kMaxEdge = 512;

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int resolve(const nufft3d_params* p, Resolved& r) {
  if (!p) return NUFFT3D_ERR_ARG;
  r.N = p->n;
  r.K = p->k ? p->k : 2 * p->n;
  r.J = p->j ? p->j : 6;
  r.L = p->table_oversamp ? p->table_oversamp : 1024;
  r.M = p->m ? p->m : 2 * p->n;
  r.D = p->n_dirs;
  r.grid_dtype = p->grid_dtype;
  r.cplx = p->complex_volume ? 1 : 0;
  r.line_fft = p->do_line_fft ? 1 : 0;
  r.keep_dup = p->keep_duplicates ? 1 : 0;
  r.exact = p->exact_coeffs;
  if (r.exact < 0 || r.exact > 1) return NUFFT3D_ERR_ARG;
  if (r.N < 8 || r.N > kMaxEdge || (r.N & 1)) return NUFFT3D_ERR_ARG;
  if (r.K < r.N || r.K > kMaxEdge) return NUFFT3D_ERR_ARG;
  if (r.J < 2 || r.J > 8) return NUFFT3D_ERR_ARG;
  if (r.J & 1) return NUFFT3D_ERR_UNSUPPORTED;
  if (!is_pow2(r.L) || r.L < 2 || r.L > 65536) return NUFFT3D_ERR_ARG;
  if (r.exact) r.L = 0;  // no table: the kernels evaluate the fitted polynomials
  if (r.M < 2 || (r.M & 1) || r.M > 1 << 20) return NUFFT3D_ERR_ARG;
  if (r.D < 1) return NUFFT3D_ERR_ARG;
  if (!p->dirs) return NUFFT3D_ERR_ARG;
  if (r.grid_dtype < 0 || r.grid_dtype > 2) return NUFFT3D_ERR_ARG;
  r.P = (long long)r.D * r.M;
  if (r.P >= (1ll << 32)) return NUFFT3D_ERR_ARG;
  if (r.K % 16 != 0 || !nufft::fft_length_supported(r.K)) return NUFFT3D_ERR_UNSUPPORTED;
  if (r.line_fft && !nufft::fft_length_supported(r.M)) return NUFFT3D_ERR_UNSUPPORTED;
  for (int i = 0; i < 3 * r.D; ++i)
    if (!std::isfinite(p->dirs[i])) return NUFFT3D_ERR_ARG;
  for (int l = 0; l < r.D; ++l) {
    const double* d = p->dirs + 3 * l;
    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > 1.0 + 1e-6) return NUFFT3D_ERR_ARG;
  }
  if (p->omega) {
    for (int m = 0; m < r.M; ++m)
      if (!std::isfinite(p->omega[m]) || std::fabs(p->omega[m]) > M_PI * (1 + 1e-12)) return NUFFT3D_ERR_ARG;
  }
  if (p->weight) {
    for (int m = 0; m < 2 * r.M; ++m)
      if (!std::isfinite(p->weight[m])) return NUFFT3D_ERR_ARG;
  }
  if (p->line_weight) {
    for (int l = 0; l < r.D; ++l)
      if (!std::isfinite(p->line_weight[l])) return NUFFT3D_ERR_ARG;
  }
  r.T = r.J == 6 ? 8 : 16;
  while (r.T > 4 && (r.K % r.T != 0 || r.T + r.J - 1 > r.K)) r.T /= 2;
  r.nT = r.K / r.T;
  return NUFFT3D_OK;
}

struct HostTables {
  std::vector<float> s;         // N
  std::vector<float2> table;    // (L + 1) * J
  std::vector<float2> twK, twM;
  std::vector<float2> dir;      // D * 3 (hi, lo)
  std::vector<float2> rad;      // M (hi, lo)
  std::vector<float2> weight;   // M or empty
  std::vector<float> line_weight;  // D or empty
  nufft::CoefPoly poly{};       // exact-coefficient mode (L = 0)
  double poly_err = 0.0;
  nufft::RealPoly rpoly{};      // real weights rho_j (L = 0)
  bool real_ok = false;
  std::vector<float2> phase;    // K entries e^{-i gamma k_c / 2}
};

float2 split(double v) {
  const float hi = (float)v;
  const float lo = (float)(v - (double)hi);
  return make_float2(hi, lo);
}

int build_tables(const nufft3d_params* p, const Resolved& r, HostTables& h) {
  const int N = r.N, K = r.K, J = r.J, L = r.L;
  const double alpha = 2.34 * J;
  const double gam = 2.0 * M_PI / K;
  // scaling factors s(n) = Psi(0) / Psi((n + 1/2) / K), n = -N/2 .. N/2 - 1
  // (Eq. 2.11, P): the Kaiser-Bessel pre-window centred on the middle -1/2 of
  // the (even) index range, so it is symmetric over the volume
  std::vector<double> s(N);
  const double psi0 = kb_ft(0.0, J, alpha);
  for (int i = 0; i < N; ++i) {
    const int n = i - N / 2;
    s[i] = psi0 / kb_ft(((double)n + 0.5) / K, J, alpha);
  }
  h.s.resize(N);
  for (int i = 0; i < N; ++i) h.s[i] = (float)s[i];
  // min-max interpolator: T_{jj'} = sum_n s(n)^2 e^{i gam (j - j') n}
  std::vector<cd> T(J * J);
  for (int a = 0; a < J; ++a)
    for (int b = 0; b < J; ++b) {
      cd acc = 0;
      for (int i = 0; i < N; ++i) {
        const double n = i - N / 2;
        acc += s[i] * s[i] * std::exp(cd(0, gam * (a - b) * n));
      }
      T[a * J + b] = acc;
    }
  if (!invert(T, J)) return NUFFT3D_ERR_ARG;
  // c(f) = T^{-1} r(f), r_j(f) = sum_n s(n) e^{-i gam (f + J/2 - j) n}, j = 1..J
  std::vector<cd> rv(J);
  auto coeffs_at = [&](double f, cd* c) {
    for (int j = 1; j <= J; ++j) {
      cd acc = 0;
      const double dist = f + 0.5 * J - j;
      for (int i = 0; i < N; ++i) {
        const double n = i - N / 2;
        acc += s[i] * std::exp(cd(0, -gam * dist * n));
      }
      rv[j - 1] = acc;
    }
    for (int a = 0; a < J; ++a) {
      cd v = 0;
      for (int b = 0; b < J; ++b) v += T[a * J + b] * rv[b];
      c[a] = v;
    }
  };
  std::vector<cd> c(J);
  if (L > 0) {
    // table: c(f_i) at f_i = i / L, i = 0..L
    h.table.resize((size_t)(L + 1) * J);
    for (int t = 0; t <= L; ++t) {
      coeffs_at((double)t / L, c.data());
      for (int a = 0; a < J; ++a) h.table[(size_t)t * J + a] = make_float2((float)c[a].real(), (float)c[a].imag());
    }
  } else {
    h.poly_err = fit_coeff_polys(J, coeffs_at, h.poly);
    if (!(h.poly_err <= 1e-7)) return NUFFT3D_ERR_UNSUPPORTED;
    // real weights rho_j(f) = c_j(f) e^{-i gam (f + J/2 - j)/2}: real because the
    // pre-window is symmetric about -1/2; kept only if the imaginary part
    // vanishes to rounding and the real fit is as close as the complex one
    double imax = 0.0, cmax = 0.0;
    for (int i = 0; i <= 256; ++i) {
      const double f = i / 256.0;
      coeffs_at(f, c.data());
      for (int a = 0; a < J; ++a) {
        const cd rho = c[a] * std::exp(cd(0, -0.5 * gam * (f + 0.5 * J - (a + 1))));
        imax = std::max(imax, std::fabs(rho.imag()));
        cmax = std::max(cmax, std::abs(c[a]));
      }
    }
    nufft::CoefPoly rp{};
    const double rerr = fit_coeff_polys(
        J,
        [&](double f, cd* out) {
          coeffs_at(f, out);
          for (int a = 0; a < J; ++a) out[a] = cd((out[a] * std::exp(cd(0, -0.5 * gam * (f + 0.5 * J - (a + 1))))).real(), 0.0);
        },
        rp);
    h.real_ok = imax <= 1e-9 * cmax && rerr <= 1e-7;
    for (int a = 0; a < J; ++a)
      for (int q = 0; q <= nufft::kPolyDeg; ++q) h.rpoly.a[a][q] = rp.a[a][0][q];
    h.phase.resize(K);
    for (int k = 0; k < K; ++k) {
      const int kc = k < K / 2 ? k : k - K;
      h.phase[k] = make_float2((float)std::cos(-0.5 * gam * kc), (float)std::sin(-0.5 * gam * kc));
    }
  }
  auto twiddles = [](int Lt, std::vector<float2>& out) {
    out.resize(Lt);
    for (int k = 0; k < Lt; ++k) {
      const double a = -2.0 * M_PI * k / Lt;
      out[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  };
  twiddles(K, h.twK);
  if (r.line_fft) twiddles(r.M, h.twM);
  h.dir.resize((size_t)r.D * 3);
  for (size_t i = 0; i < (size_t)r.D * 3; ++i) h.dir[i] = split(p->dirs[i]);
  h.rad.resize(r.M);
  for (int m = 0; m < r.M; ++m) {
    const double rad = p->omega ? p->omega[m] * K / (2.0 * M_PI) : (double)(m - r.M / 2) * K / r.M;
    h.rad[m] = split(rad);
  }
  if (p->line_weight) h.line_weight.assign(p->line_weight, p->line_weight + r.D);
  if (p->weight) {
    h.weight.resize(r.M);
    for (int m = 0; m < r.M; ++m) h.weight[m] = make_float2(p->weight[2 * m], p->weight[2 * m + 1]);
  }
  return NUFFT3D_OK;
}

// Coincident samples.  If line l2 runs opposite to line l (d_l2 = -d_l within
// 1e-13 per component) and the radii are symmetric (r[M - m] = -r[m]), sample
// (l2, M - m) is the same Fourier point as (l, m) for m >= 1.  Such pairs are
// interpolated once: l2 keeps only its sample m = 0 (whose partner radius is
// not sampled), and (l, m) carries (l2, M - m) as its twin.  The direction of
// l2 is snapped to the exact negation of d_l so both decode bit-identically.
void pair_lines(const nufft3d_params* p, const Resolved& r, HostTables& h, std::vector<uint32_t>& ids,
                std::vector<uint32_t>& twin, int& n_pairs) {
  const int D = r.D, M = r.M;
  ids.clear();
  twin.clear();
  n_pairs = 0;
  std::vector<int> partner(D, -1), role(D, 0);  // role 1: keeps all samples, 2: keeps m = 0 only
  bool symmetric = !r.keep_dup && (M % 2 == 0);
  if (symmetric) {
    std::vector<double> rad(M);
    for (int m = 0; m < M; ++m)
      rad[m] = p->omega ? p->omega[m] * r.K / (2.0 * M_PI) : (double)(m - M / 2) * r.K / M;
    for (int m = 1; m < M && symmetric; ++m) symmetric = rad[M - m] == -rad[m];
  }
  if (symmetric) {
    struct KeyHash {
      size_t operator()(const std::array<long long, 3>& k) const {
        return (size_t)(k[0] * 73856093ll ^ k[1] * 19349663ll ^ k[2] * 83492791ll);
      }
    };
    auto key = [](const double* d, double sgn) {
      return std::array<long long, 3>{std::llround(sgn * d[0] * 1e9), std::llround(sgn * d[1] * 1e9),
                                      std::llround(sgn * d[2] * 1e9)};
    };
    std::unordered_map<std::array<long long, 3>, std::vector<int>, KeyHash> by_dir;
    for (int l = 0; l < D; ++l) by_dir[key(p->dirs + 3 * l, 1.0)].push_back(l);
    for (int l = 0; l < D; ++l) {
      if (role[l]) continue;
      auto it = by_dir.find(key(p->dirs + 3 * l, -1.0));
      if (it == by_dir.end()) continue;
      for (int l2 : it->second) {
        if (l2 <= l || role[l2]) continue;
        const double* a = p->dirs + 3 * l;
        const double* b = p->dirs + 3 * l2;
        if (std::fabs(a[0] + b[0]) <= 1e-13 && std::fabs(a[1] + b[1]) <= 1e-13 && std::fabs(a[2] + b[2]) <= 1e-13) {
          role[l] = 1;
          role[l2] = 2;
          partner[l] = l2;
          for (int c = 0; c < 3; ++c) h.dir[(size_t)l2 * 3 + c] = split(-a[c]);
          ++n_pairs;
          break;
        }
      }
    }
  }
  for (int l = 0; l < D; ++l) {
    const uint32_t base = (uint32_t)l * (uint32_t)M;
    if (role[l] == 2) {
      ids.push_back(base);
      twin.push_back(nufft::kNoTwin);
      continue;
    }
    for (int m = 0; m < M; ++m) {
      ids.push_back(base + (uint32_t)m);
      twin.push_back(role[l] == 1 && m >= 1 ? (uint32_t)partner[l] * (uint32_t)M + (uint32_t)(M - m) : nufft::kNoTwin);
    }
  }
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  if (e == cudaErrorMemoryAllocation) return NUFFT3D_ERR_NOMEM;
  return NUFFT3D_ERR_CUDA;
}

#define CK(expr)                              \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc((void**)p, count * sizeof(T));
}

template <typename T>
cudaError_t upload(T** p, const std::vector<T>& v, cudaStream_t st) {
  cudaError_t e = dalloc(p, v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

void free_plan(nufft3d_plan pl) {
  if (!pl) return;
  void* ptrs[] = {pl->d_dir, pl->d_rad, pl->d_weight, pl->d_line_weight, pl->d_s, pl->d_table, pl->d_twK, pl->d_twM,
                  pl->d_sorted, pl->d_sub, pl->d_grid, pl->d_grid_adj, pl->d_grid_lp, pl->d_bufA, pl->d_bufB,
                  pl->d_lines, pl->d_err, pl->d_counter, pl->d_lp_bound, pl->d_phase};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (void* q : {(void*)pl->d_sched, (void*)pl->d_gslots, (void*)pl->d_sslots, (void*)pl->d_cbound, (void*)pl->d_box})
    if (q) cudaFree(q);
  for (cudaEvent_t e : pl->ev_fwd) cudaEventDestroy(e);
  for (cudaEvent_t e : pl->ev_adj) cudaEventDestroy(e);
  delete pl;
}

InterpGeom geom(const nufft3d_plan pl) {
  InterpGeom g;
  g.K = pl->K;
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
  g.counter = pl->d_counter;
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
  g.tmap = pl->tmap_ok ? &pl->tmap_grid : nullptr;
  g.first_wait_polls = pl->first_wait_polls;
  return g;
}

// ---------------------------------------------------------------------------
// Conflict schedules of the thread-per-point real-weight kernels (gather 10,
// spread 8).  The points are fixed at plan time, so the plan decides, per
// subproblem, the plane pitch of the shared-memory tile and which points run
// side by side in a half-warp (gather: 16 lanes, 8-byte cells) or a warp
// (spread: 32 lanes, 4-byte cells):
//  * gather: lanes of a half-warp read the same tap of their points, one
//    wavefront if the base offsets are distinct modulo 16 (cells) or equal
//    (broadcast).  A group takes at most one distinct offset per residue class
//    (all its points at that offset); the pitch minimises the lower bound
//    max(ceil(n / 16), most distinct offsets in a class) on the groups.
//  * spread: lanes of a warp add to the same tap of their points, one
//    wavefront if the offsets are distinct modulo 32 (equal offsets collide),
//    so a group holds at most one point per class: G = max(ceil(n / 32), the
//    largest class) groups, classes dealt cyclically; the pitch minimises G.
// The local first tap is recomputed here in FP64; should it differ from the
// device's by a rounding near an integer, only the quality of the schedule
// suffers, never the result (the kernels compute every offset themselves).
// ---------------------------------------------------------------------------
namespace {

struct SchedOut {
  std::vector<int4> sched;
  std::vector<uint16_t> g, s;
  std::vector<int> box;
};

// The cells a subproblem's taps can reach: per axis [min first tap, max first
// tap + J - 1] of its points, widened by one cell on each side (the first taps
// here are FP64 floors and may differ by one from the device's near an
// integer), clipped to the E^3 tile.  Packed as (origin 4 bits, extent 5 bits)
// per axis, x in the low bits.
int pack_box(const std::vector<int>& lx, const std::vector<int>& ly, const std::vector<int>& lz, int n, int J, int E) {
  int code = 0;
  const std::vector<int>* ax[3] = {&lx, &ly, &lz};
  for (int a = 0; a < 3; ++a) {
    int mn = E, mx = -1;
    for (int i = 0; i < n; ++i) {
      mn = std::min(mn, (*ax[a])[i]);
      mx = std::max(mx, (*ax[a])[i]);
    }
    int o = 0, e = E;
    if (n > 0) {
      o = std::max(0, mn - 1);
      e = std::min(E, mx + J + 1) - o;
    }
    code |= (o | (e << 4)) << (9 * a);
  }
  return code;
}

void schedule_range(const nufft3d_plan pl, size_t s0, size_t s1, SchedOut& out) {
  const int T = pl->T, J = pl->J, K = pl->K, E = T + J - 1, nT = pl->nT;
  const uint32_t M = (uint32_t)pl->M;
  std::vector<int> lx, ly, lz, off, order;
  std::vector<int> cls_n(32), cls_first(32), cls_cur(32);
  // one stamp per candidate marks the offsets seen (offsets < E * (E^2 + 32))
  std::vector<unsigned> stamp((size_t)E * (E * E + nufft::kSpreadPitchCodes), 0u);
  unsigned stamp_id = 0;
  for (size_t si = s0; si < s1; ++si) {
    const int4 sp = pl->h_sub[si];
    const int n = sp.z;
    const int ox = (sp.x % nT) * T, oy = ((sp.x / nT) % nT) * T, oz = (sp.x / (nT * nT)) * T;
    lx.resize(n);
    ly.resize(n);
    lz.resize(n);
    for (int i = 0; i < n; ++i) {
      const uint32_t id = pl->h_sorted[(size_t)sp.y + i].x;
      const uint32_t l = id / M, m = id - l * M;
      const double r = (double)pl->h_rad[m].x + (double)pl->h_rad[m].y;
      int* dst[3] = {&lx[i], &ly[i], &lz[i]};
      const int org[3] = {ox, oy, oz};
      for (int a = 0; a < 3; ++a) {
        const double d = (double)pl->h_dir[(size_t)l * 3 + a].x + (double)pl->h_dir[(size_t)l * 3 + a].y;
        long long f = (long long)std::floor(r * d) - J / 2 + 1;
        f %= K;
        if (f < 0) f += K;
        long long loc = f - org[a];
        if (loc < 0) loc += K;
        *dst[a] = (int)std::min<long long>(std::max<long long>(loc, 0), T - 1);
      }
    }
    out.box.push_back(pack_box(lx, ly, lz, n, J, E));
    int4 sc = make_int4((int)out.g.size(), 0, (int)out.s.size(), 0);
    off.resize(n);
    order.resize(n);
    // gather: pitch by the lower bound, then greedy groups
    {
      int best = 0, best_lb = 1 << 30;
      for (int code = 0; code < nufft::kGatherPitchCodes; ++code) {
        const int PP = E * E + code;
        ++stamp_id;
        std::fill(cls_n.begin(), cls_n.begin() + 16, 0);
        for (int i = 0; i < n; ++i) {
          const int o = lx[i] + E * ly[i] + PP * lz[i];
          if (stamp[o] != stamp_id) {  // a distinct offset of its class
            stamp[o] = stamp_id;
            cls_n[o & 15]++;
          }
        }
        int lb = (n + 15) / 16;
        for (int c = 0; c < 16; ++c) lb = std::max(lb, cls_n[c]);
        if (lb < best_lb) {
          best_lb = lb;
          best = code;
        }
      }
      const int PP = E * E + best;
      for (int i = 0; i < n; ++i) off[i] = lx[i] + E * ly[i] + PP * lz[i];
      for (int i = 0; i < n; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int ca = off[a] & 15, cb = off[b] & 15;
        return ca != cb ? ca < cb : off[a] < off[b];
      });
      // per class: [first, first + n) in `order`, cursor
      std::fill(cls_n.begin(), cls_n.begin() + 16, 0);
      for (int k = 0; k < n; ++k) cls_n[off[order[k]] & 15]++;
      int acc = 0;
      for (int c = 0; c < 16; ++c) {
        cls_first[c] = acc;
        cls_cur[c] = acc;
        acc += cls_n[c];
      }
      int left = n, slots = 0;
      std::vector<int> cls_idx(16);
      while (left > 0) {
        // classes by remaining points, largest first
        for (int c = 0; c < 16; ++c) cls_idx[c] = c;
        std::sort(cls_idx.begin(), cls_idx.end(), [&](int a, int b) {
          const int ra = cls_first[a] + cls_n[a] - cls_cur[a], rb = cls_first[b] + cls_n[b] - cls_cur[b];
          return ra != rb ? ra > rb : a < b;
        });
        int room = 16;
        for (int q = 0; q < 16 && room > 0; ++q) {
          const int c = cls_idx[q];
          const int end = cls_first[c] + cls_n[c];
          if (cls_cur[c] >= end) continue;
          const int o = off[order[cls_cur[c]]];
          while (room > 0 && cls_cur[c] < end && off[order[cls_cur[c]]] == o) {
            out.g.push_back((uint16_t)order[cls_cur[c]++]);
            --room;
            --left;
          }
        }
        for (; room > 0; --room) out.g.push_back(0xffff);
        slots += 16;
      }
      sc.y = slots | (best << 16);
    }
    // spread (not for the points at the origin, which the kernel sums first)
    if (!(sp.w & 1)) {
      int best = 0, best_g = 1 << 30;
      for (int code = 0; code < nufft::kSpreadPitchCodes; ++code) {
        const int PP = E * E + code;
        std::fill(cls_n.begin(), cls_n.end(), 0);
        for (int i = 0; i < n; ++i) cls_n[(lx[i] + E * ly[i] + PP * lz[i]) & 31]++;
        int G = (n + 31) / 32;
        for (int c = 0; c < 32; ++c) G = std::max(G, cls_n[c]);
        if (G < best_g) {
          best_g = G;
          best = code;
        }
      }
      const int PP = E * E + best, G = best_g;
      for (int i = 0; i < n; ++i) off[i] = (lx[i] + E * ly[i] + PP * lz[i]) & 31;
      for (int i = 0; i < n; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return off[a] < off[b]; });
      std::fill(cls_n.begin(), cls_n.end(), 0);
      for (int i = 0; i < n; ++i) cls_n[off[i]]++;
      // classes largest first, dealt cyclically over the G groups
      std::vector<int> cidx(32);
      for (int c = 0; c < 32; ++c) cidx[c] = c;
      std::stable_sort(cidx.begin(), cidx.end(), [&](int a, int b) { return cls_n[a] > cls_n[b]; });
      int acc = 0;
      for (int c = 0; c < 32; ++c) {
        cls_first[c] = acc;
        acc += cls_n[c];
      }
      std::vector<int> fill((size_t)G, 0);
      const size_t base = out.s.size();
      out.s.resize(base + (size_t)G * 32, 0xffff);
      int cur = 0;
      for (int q = 0; q < 32; ++q) {
        const int c = cidx[q];
        for (int k = 0; k < cls_n[c]; ++k) {
          out.s[base + (size_t)cur * 32 + fill[cur]] = (uint16_t)order[cls_first[c] + k];
          fill[cur]++;
          cur = cur + 1 == G ? 0 : cur + 1;
        }
      }
      sc.w = (G * 32) | (best << 16);
    }
    out.sched.push_back(sc);
  }
}

}  // namespace

int build_schedules(nufft3d_plan pl, cudaStream_t st) {
  for (void** q : {(void**)&pl->d_sched, (void**)&pl->d_gslots, (void**)&pl->d_sslots, (void**)&pl->d_cbound,
                   (void**)&pl->d_box})
    if (*q) {
      cudaFree(*q);
      *q = nullptr;
    }
  pl->sched_ok = false;
  if (!pl->real_ok || pl->T != 8 || pl->pts_per_sub > 256 || pl->h_sub.empty()) return NUFFT3D_OK;
  const size_t ns = pl->h_sub.size();
  unsigned nth = std::thread::hardware_concurrency();
  nth = std::max(1u, std::min(nth, 32u));
  if (ns < 4096) nth = 1;
  std::vector<SchedOut> parts(nth);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t) {
    const size_t a = ns * t / nth, b = ns * (t + 1) / nth;
    if (nth == 1) schedule_range(pl, a, b, parts[t]);
    else th.emplace_back([&, a, b, t] { schedule_range(pl, a, b, parts[t]); });
  }
  for (auto& x : th) x.join();
  std::vector<int4> sched;
  std::vector<uint16_t> gs, ss;
  std::vector<int> box;
  sched.reserve(ns);
  box.reserve(ns);
  for (auto& pt : parts) {
    const int gb = (int)gs.size(), sb = (int)ss.size();
    for (int4 v : pt.sched) sched.push_back(make_int4(v.x + gb, v.y, v.z + sb, v.w));
    gs.insert(gs.end(), pt.g.begin(), pt.g.end());
    ss.insert(ss.end(), pt.s.begin(), pt.s.end());
    box.insert(box.end(), pt.box.begin(), pt.box.end());
  }
  if (gs.size() > 0x7fffffffull || ss.size() > 0x7fffffffull) return NUFFT3D_OK;  // no schedule: variants 10 / 8 refuse
  if (ss.empty()) ss.push_back(0xffff);
  CK(upload(&pl->d_sched, sched, st));
  CK(upload(&pl->d_gslots, gs, st));
  CK(upload(&pl->d_sslots, ss, st));
  CK(upload(&pl->d_box, box, st));
  // the per-point bounds of the scheduled spread, with the kernels' arithmetic
  CK(dalloc(&pl->d_cbound, (size_t)pl->P_eval));
  CK(nufft::launch_point_bounds(geom(pl), pl->P_eval, pl->d_cbound, st));
  CK(cudaStreamSynchronize(st));
  pl->sched_ok = true;
  return NUFFT3D_OK;
}

int build_subproblems(nufft3d_plan pl, int S, cudaStream_t st) {
  // subproblems of tiles holding more than S points (the dense centre of the
  // radial pattern) come first, so the persistent kernels finish balanced;
  // the rest follow in tile order (neighbouring tiles share halo cells in L2)
  // the points at the origin of a bin (all alike) form subproblems of their
  // own, flagged in .w bit 0
  std::vector<int4> heavy, light;
  const size_t nb = pl->bin_offsets.size() - 1;
  for (size_t b = 0; b < nb; ++b) {
    const long long a = pl->bin_offsets[b], e = pl->bin_offsets[b + 1];
    const long long mid = a + (b < pl->bin_dc.size() ? pl->bin_dc[b] : 0);
    std::vector<int4>& dst = (e - a > S) ? heavy : light;
    for (long long s0 = a; s0 < mid; s0 += S)
      dst.push_back(make_int4((int)b, (int)s0, (int)std::min<long long>(S, mid - s0), 1));
    for (long long s0 = mid; s0 < e; s0 += S)
      dst.push_back(make_int4((int)b, (int)s0, (int)std::min<long long>(S, e - s0), 0));
  }
  std::vector<int4> subs(heavy);
  subs.insert(subs.end(), light.begin(), light.end());
  if (pl->d_sub) {
    cudaFree(pl->d_sub);
    pl->d_sub = nullptr;
  }
  pl->n_sub = (int)subs.size();
  CK(upload(&pl->d_sub, subs, st));
  CK(cudaStreamSynchronize(st));
  pl->h_sub.swap(subs);
  pl->pts_per_sub = S;
  return build_schedules(pl, st);
}

int sort_points(nufft3d_plan pl, cudaStream_t st) {
  const long long P = pl->P_eval;
  uint32_t* d_bins = nullptr;
  CK(dalloc(&d_bins, (size_t)P));
  uint32_t* d_ids = nullptr;
  cudaError_t e = upload(&d_ids, pl->h_unique, st);
  InterpGeom g = geom(pl);
  if (e == cudaSuccess) e = nufft::launch_bin_points(g, d_ids, P, d_bins, st);
  std::vector<uint32_t> bins;
  if (e == cudaSuccess) {
    try {
      bins.resize((size_t)P);
    } catch (...) {
      cudaFree(d_bins);
      cudaFree(d_ids);
      return NUFFT3D_ERR_NOMEM;
    }
    e = cudaMemcpyAsync(bins.data(), d_bins, (size_t)P * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d_bins);
  if (d_ids) cudaFree(d_ids);
  if (e != cudaSuccess) return cuda_status(e);
  // stable counting sort by bin
  const size_t nb = (size_t)pl->nT * pl->nT * pl->nT;
  std::vector<long long> off(nb + 1, 0);
  for (long long i = 0; i < P; ++i) {
    if (bins[i] >= nb) return NUFFT3D_ERR_DEVICE_CHECK;
    off[bins[i] + 1]++;
  }
  for (size_t b = 0; b < nb; ++b) off[b + 1] += off[b];
  std::vector<uint2> sorted((size_t)P);
  {
    std::vector<long long> pos(off.begin(), off.end() - 1);
    for (long long i = 0; i < P; ++i) sorted[pos[bins[i]]++] = make_uint2(pl->h_unique[i], pl->h_twin[i]);
  }
  // within a bin, the points at the origin (radius 0: identical coordinates on
  // every line) come first; the subproblems keep them apart from the others
  pl->bin_dc.assign(nb, 0);
  for (size_t b = 0; b < nb; ++b) {
    auto at_origin = [&](const uint2& v) {
      const float2 r = pl->h_rad[v.x % (uint32_t)pl->M];
      return r.x == 0.f && r.y == 0.f;
    };
    auto it = std::stable_partition(sorted.begin() + off[b], sorted.begin() + off[b + 1], at_origin);
    pl->bin_dc[b] = (int)(it - (sorted.begin() + off[b]));
  }
  pl->bin_offsets.swap(off);
  CK(upload(&pl->d_sorted, sorted, st));
  CK(cudaStreamSynchronize(st));
  pl->h_sorted.swap(sorted);
  return NUFFT3D_OK;
}

int plan_create_impl(nufft3d_plan* out, const nufft3d_params* p, cudaStream_t st) {
  Resolved r;
  int rc = resolve(p, r);
  if (rc != NUFFT3D_OK) return rc;
  HostTables h;
  rc = build_tables(p, r, h);
  if (rc != NUFFT3D_OK) return rc;
  std::vector<uint32_t> ids, twin;
  int n_pairs = 0;
  pair_lines(p, r, h, ids, twin, n_pairs);
  nufft3d_plan pl = new (std::nothrow) nufft3d_plan_s();
  if (!pl) return NUFFT3D_ERR_NOMEM;
  *out = pl;  // freed by the caller on failure
  pl->N = r.N;
  pl->K = r.K;
  pl->J = r.J;
  pl->L = r.L;
  pl->poly = h.poly;
  pl->rpoly = h.rpoly;
  pl->real_ok = r.L == 0 && h.real_ok;
  {
    // every tap of a point with |u| <= K/2 lies within (J/2) sqrt 3 of it; one
    // more cell covers a rounding of the tap base
    const double R = 0.5 * r.K + 0.5 * r.J * std::sqrt(3.0) + 1.0;
    pl->ball_r2 = (long long)std::ceil(R * R);
  }
  pl->poly_err = h.poly_err;
  pl->D = r.D;
  pl->M = r.M;
  pl->P = r.P;
  pl->complex_volume = r.cplx;
  pl->do_line_fft = r.line_fft;
  pl->grid_dtype = r.grid_dtype;
  pl->T = r.T;
  pl->nT = r.nT;
  pl->h_unique.swap(ids);
  pl->h_twin.swap(twin);
  pl->h_dir = h.dir;
  pl->h_rad = h.rad;
  pl->P_eval = (long long)pl->h_unique.size();
  pl->n_pairs = n_pairs;
  // defaults measured at 256^3: with the table, 256-thread gather CTAs, 512
  // points per subproblem and the warp-private FP32 spread; with exact
  // coefficients (no table traffic), 128-thread gather CTAs, 256 points per
  // subproblem and the CTA-shared fixed-point spread
  const int S0 = r.L == 0 && r.T == 8 ? 256 : 512;
  pl->gather_variant = nufft::v3_supported(r.T, r.J, S0) ? (r.L == 0 && r.T == 8 ? 5 : 3) : 0;
  pl->spread_variant = r.L == 0 && nufft::v6s_supported(r.T, r.J, S0) ? 6
                       : nufft::v3s_supported(r.T, r.J)             ? 3
                       : (nufft::v2_supported(r.T, r.J, r.L) ? 2 : 0);
  CK(cudaGetDevice(&pl->device));
  CK(upload(&pl->d_s, h.s, st));
  CK(upload(&pl->d_table, h.table, st));
  CK(upload(&pl->d_twK, h.twK, st));
  CK(upload(&pl->d_twM, h.twM, st));
  CK(upload(&pl->d_dir, h.dir, st));
  CK(upload(&pl->d_rad, h.rad, st));
  CK(upload(&pl->d_weight, h.weight, st));
  CK(upload(&pl->d_line_weight, h.line_weight, st));
  CK(upload(&pl->d_phase, h.phase, st));
  CK(dalloc(&pl->d_err, 1));
  CK(dalloc(&pl->d_counter, 2));
  CK(cudaMemsetAsync(pl->d_err, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  rc = sort_points(pl, st);
  if (rc != NUFFT3D_OK) return rc;
  rc = build_subproblems(pl, S0, st);
  if (rc != NUFFT3D_OK) return rc;
  // with exact coefficients the real-weight kernels are the defaults: the
  // scheduled gather (10) and the warp-cooperative fixed-point spread (7)
  if (pl->real_ok && pl->sched_ok && nufft::v10_supported(r.T, r.J, S0)) pl->gather_variant = 10;
  if (pl->real_ok && nufft::v7s_supported(r.T, r.J, S0)) pl->spread_variant = 7;
  const size_t K3 = (size_t)r.K * r.K * r.K;
  CK(dalloc(&pl->d_grid, K3));
  if (r.grid_dtype == NUFFT3D_GRID_C64) {
    CK(dalloc(&pl->d_grid_adj, K3));
    CK(cudaMemsetAsync(pl->d_grid_adj, 0, K3 * sizeof(float2), st));
  } else {
    CK(cudaMemsetAsync(pl->d_grid, 0, K3 * sizeof(float2), st));  // the adjoint grid
  }
  pl->adj_dirty = false;
  if (r.grid_dtype != NUFFT3D_GRID_C64) {
    CK(cudaMalloc(&pl->d_grid_lp, K3 * 4));
    CK(dalloc(&pl->d_lp_bound, 1));
  }
  // tensor map of the grid the gather reads (TMA tile copies of gather variant 8)
  pl->tmap_ok = nufft::make_grid_tmap(&pl->tmap_grid, r.grid_dtype == NUFFT3D_GRID_C64 ? (const void*)pl->d_grid
                                                                                       : pl->d_grid_lp,
                                      r.K, r.grid_dtype == NUFFT3D_GRID_C64 ? 8 : 4);
  CK(dalloc(&pl->d_bufA, (size_t)r.N * r.N * r.K));
  CK(dalloc(&pl->d_bufB, (size_t)r.N * r.K * r.K));
  if (r.line_fft) CK(dalloc(&pl->d_lines, (size_t)r.P));
  CK(cudaStreamSynchronize(st));
  pl->last_stream = st;
  return NUFFT3D_OK;
}

// the plan's device, current until the end of the calling scope; the caller's
// current device is restored on return
#define PLAN_DEVICE(pl)                                 \
  nufft::DeviceGuard dev_guard_((pl)->device);          \
  if (dev_guard_.status != cudaSuccess) return NUFFT3D_ERR_CUDA

// records the event closing stage `stage` of the current timed call (stage -1 opens it)
struct StageClock {
  cudaEvent_t* ev = nullptr;
  cudaStream_t st;
  StageClock(std::vector<cudaEvent_t>& v, int slots, int& calls, int nst, cudaStream_t s) : st(s) {
    if (calls < slots) ev = v.data() + (size_t)calls++ * (nst + 1);
  }
  cudaError_t mark(int stage) { return ev ? cudaEventRecord(ev[stage + 1], st) : cudaSuccess; }
};

nufft::ColPrune prune(const nufft3d_plan pl, int mode) {
  nufft::ColPrune p;
  p.mode = mode;
  p.K = pl->K;
  p.r2 = pl->ball_r2;
  return p;
}

// The stages of a call, in three parts (bit 0: before the interpolation, bit 1:
// the interpolation, bit 2: after it); a batch runs the interpolation of a
// group of plans as one launch and the other parts per plan.  Only a whole
// call is timed.
constexpr int kAllParts = 7;

int forward_impl(nufft3d_plan pl, const void* vol, void* lines, cudaStream_t st, int parts = kAllParts) {
  const int N = pl->N, K = pl->K;
  const long long KK = (long long)K * K;
  int no_slots = 0, no_calls = 0;
  StageClock clk(pl->ev_fwd, parts == kAllParts ? pl->timing_slots : no_slots,
                 parts == kAllParts ? pl->fwd_calls : no_calls, FWD_STAGES, st);
  CK(clk.mark(-1));
  if (parts & 1) {
  if (pl->grid_dtype != NUFFT3D_GRID_C64)
    CK(nufft::launch_abs_bound(vol, pl->complex_volume, pl->d_s, N, pl->d_lp_bound, st));
  CK(nufft::launch_row_fwd(K, vol, pl->complex_volume, pl->d_bufA, pl->d_s, N, pl->d_twK, st));
  CK(clk.mark(0));
  CK(nufft::launch_col_fwd(K, pl->d_bufA, pl->d_bufB, N, N, K, (long long)N * K, K, KK, K, pl->d_twK, st));
  CK(clk.mark(1));
  nufft::ColPrune pzf = prune(pl, 2);
  if (nufft::gather_real(pl->gather_variant)) pzf.phase = pl->d_phase;
  if (pl->grid_dtype == NUFFT3D_GRID_C64) {
    CK(nufft::launch_col_fwd(K, pl->d_bufB, pl->d_grid, N, K, K, K, KK, K, KK, pl->d_twK, st, pzf));
  } else {
    CK(nufft::launch_col_fwd_lp(K, pl->grid_dtype, pl->d_bufB, pl->d_grid_lp, N, K, K, K, KK, K, KK, pl->d_twK,
                                pl->d_lp_bound, st, pzf));
  }
  CK(clk.mark(2));
  }
  if (parts & 2) {
    const void* grid = pl->grid_dtype == NUFFT3D_GRID_C64 ? (const void*)pl->d_grid : pl->d_grid_lp;
    InterpGeom g = geom(pl);
    CK(nufft::launch_gather(g, pl->gather_variant, pl->grid_dtype, grid, 1.f, pl->d_sub, pl->n_sub,
                            (float2*)lines, st));
  }
  CK(clk.mark(3));
  if ((parts & 4) && pl->do_line_fft)
    CK(nufft::launch_line(pl->M, true, (const float2*)lines, (float2*)lines, pl->D, pl->d_weight, pl->d_twM, st,
                          pl->d_line_weight));
  CK(clk.mark(4));
  return NUFFT3D_OK;
}

int adjoint_impl(nufft3d_plan pl, const void* lines, void* vol, cudaStream_t st, int parts = kAllParts) {
  const int N = pl->N, K = pl->K;
  const long long KK = (long long)K * K;
  const float2* src = (const float2*)lines;
  int no_slots = 0, no_calls = 0;
  StageClock clk(pl->ev_adj, parts == kAllParts ? pl->timing_slots : no_slots,
                 parts == kAllParts ? pl->adj_calls : no_calls, ADJ_STAGES, st);
  CK(clk.mark(-1));
  if (pl->do_line_fft) {
    if (parts & 1)
      CK(nufft::launch_line(pl->M, false, src, pl->d_lines, pl->D, pl->d_weight, pl->d_twM, st,
                            pl->d_line_weight));
    src = pl->d_lines;
  }
  CK(clk.mark(0));
  // the adjoint grid is clear between calls: the inverse z pass zeroes every
  // cell it reads, and nothing outside the touched ball is ever written.  A
  // call that stopped between the spread and that pass left it dirty.
  float2* ag = pl->d_grid_adj ? pl->d_grid_adj : pl->d_grid;
  if ((parts & 1) && pl->adj_dirty) CK(cudaMemsetAsync(ag, 0, (size_t)K * KK * sizeof(float2), st));
  CK(clk.mark(1));
  if (parts & 2) {
    InterpGeom g = geom(pl);
    pl->adj_dirty = true;
    CK(nufft::launch_spread(g, pl->spread_variant, src, pl->d_sub, pl->n_sub, ag, st));
  }
  CK(clk.mark(2));
  if (!(parts & 4)) return NUFFT3D_OK;
  nufft::ColPrune pz = prune(pl, 2);
  pz.consume = 1;
  if (nufft::spread_real(pl->spread_variant)) pz.phase = pl->d_phase;
  CK(nufft::launch_col_inv(K, ag, pl->d_bufB, N, K, K, K, KK, K, KK, pl->d_twK, st, pz));
  pl->adj_dirty = false;
  CK(clk.mark(3));
  CK(nufft::launch_col_inv(K, pl->d_bufB, pl->d_bufA, N, N, K, KK, K, (long long)N * K, K, pl->d_twK, st,
                           prune(pl, 1)));
  CK(clk.mark(4));
  CK(nufft::launch_row_adj(K, pl->d_bufA, vol, pl->complex_volume, pl->d_s, N, pl->d_twK, st));
  CK(clk.mark(5));
  return NUFFT3D_OK;
}

}  // namespace

namespace nufft {
int plan_forward_enqueue(nufft3d_plan pl, const void* vol, void* lines, cudaStream_t st) {
  pl->last_stream = st;
  return forward_impl(pl, vol, lines, st);
}
int plan_forward_parts(nufft3d_plan pl, const void* vol, void* lines, cudaStream_t st, int parts) {
  pl->last_stream = st;
  return forward_impl(pl, vol, lines, st, parts);
}
int plan_adjoint_parts(nufft3d_plan pl, const void* lines, void* vol, cudaStream_t st, int parts) {
  pl->last_stream = st;
  return adjoint_impl(pl, lines, vol, st, parts);
}
int plan_adjoint_enqueue(nufft3d_plan pl, const void* lines, void* vol, cudaStream_t st) {
  pl->last_stream = st;
  return adjoint_impl(pl, lines, vol, st);
}
}  // namespace nufft

extern "C" {

int nufft3d_plan_create(nufft3d_plan* out, const nufft3d_params* p, void* cuda_stream) {
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  nufft3d_plan pl = nullptr;
  int rc;
  try {
    rc = plan_create_impl(&pl, p, (cudaStream_t)cuda_stream);
  } catch (const std::bad_alloc&) {
    rc = NUFFT3D_ERR_NOMEM;
  } catch (...) {
    rc = NUFFT3D_ERR_CUDA;
  }
  if (rc != NUFFT3D_OK) {
    if (pl) {
      cudaStreamSynchronize((cudaStream_t)cuda_stream);
      free_plan(pl);
    }
    return rc;
  }
  *out = pl;
  return NUFFT3D_OK;
}

int nufft3d_forward(nufft3d_plan plan, const void* vol_dev, void* lines_dev, void* cuda_stream) {
  if (!plan || !vol_dev || !lines_dev) return NUFFT3D_ERR_ARG;
  PLAN_DEVICE(plan);
  plan->last_stream = (cudaStream_t)cuda_stream;
  return forward_impl(plan, vol_dev, lines_dev, (cudaStream_t)cuda_stream);
}

int nufft3d_adjoint(nufft3d_plan plan, const void* lines_dev, void* vol_dev, void* cuda_stream) {
  if (!plan || !vol_dev || !lines_dev) return NUFFT3D_ERR_ARG;
  PLAN_DEVICE(plan);
  plan->last_stream = (cudaStream_t)cuda_stream;
  return adjoint_impl(plan, lines_dev, vol_dev, (cudaStream_t)cuda_stream);
}

int nufft3d_fourier_slice_weights(int n_az, int n_pol, double cone_half_angle, int m, float* radial_weight,
                                  float* line_weight) {
  if (n_az < 1 || n_pol < 1 || m < 2 || (m & 1) || !radial_weight || !line_weight) return NUFFT3D_ERR_ARG;
  if (!std::isfinite(cone_half_angle) || cone_half_angle < 0.0 || cone_half_angle >= 0.5 * M_PI)
    return NUFFT3D_ERR_ARG;
  const double dth = (M_PI - 2.0 * cone_half_angle) / n_pol, dph = 2.0 * M_PI / n_az;
  double sum = 0.0;
  for (int a = 0; a < n_az; ++a)
    for (int p = 0; p < n_pol; ++p) {
      const double th = cone_half_angle + dth * (p + 0.5);
      const double w = 0.5 * std::sin(th) * dth * dph;
      line_weight[(size_t)a * n_pol + p] = (float)w;
      sum += w;
    }
  const double mm = (double)m * m;
  for (int i = 0; i < m; ++i) {
    const double q = i - m / 2;
    const double w = q != 0.0 ? q * q / mm : M_PI / (6.0 * mm * sum);
    radial_weight[2 * i] = (float)w;
    radial_weight[2 * i + 1] = 0.f;
  }
  return NUFFT3D_OK;
}

int nufft3d_workspace_bytes(const nufft3d_params* p, size_t* bytes) {
  if (!bytes) return NUFFT3D_ERR_ARG;
  Resolved r;
  const int rc = resolve(p, r);
  if (rc != NUFFT3D_OK) return rc;
  const size_t K3 = (size_t)r.K * r.K * r.K;
  size_t b = 0;
  b += K3 * sizeof(float2);
  if (r.grid_dtype != NUFFT3D_GRID_C64) b += K3 * 4 + sizeof(float);
  else b += K3 * sizeof(float2);  // separate adjoint grid
  b += (size_t)r.N * r.N * r.K * sizeof(float2);
  b += (size_t)r.N * r.K * r.K * sizeof(float2);
  if (r.line_fft) b += (size_t)r.P * sizeof(float2);
  b += (size_t)r.P * sizeof(uint2);                                      // point sort (upper bound)
  b += r.L ? (size_t)(r.L + 1) * r.J * sizeof(float2) : 0;               // table
  b += (size_t)r.D * 3 * sizeof(float2) + (size_t)r.M * 2 * sizeof(float2) + r.N * sizeof(float);
  b += (size_t)(r.K + r.M) * sizeof(float2);
  *bytes = b;
  return NUFFT3D_OK;
}

int nufft3d_plan_sync_status(nufft3d_plan plan, int* device_status) {
  if (!plan || !device_status) return NUFFT3D_ERR_ARG;
  PLAN_DEVICE(plan);
  int v = 0;
  CK(cudaStreamSynchronize(plan->last_stream));
  CK(cudaMemcpy(&v, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(plan->d_err, 0, sizeof(int)));
  *device_status = v;
  return NUFFT3D_OK;
}

int nufft3d_plan_destroy(nufft3d_plan plan) {
  if (!plan) return NUFFT3D_OK;
  nufft::DeviceGuard guard(plan->device);
  cudaDeviceSynchronize();
  free_plan(plan);
  return NUFFT3D_OK;
}

const char* nufft3d_error_string(int status) {
  switch (status) {
    case NUFFT3D_OK: return "success";
    case NUFFT3D_ERR_ARG: return "invalid argument";
    case NUFFT3D_ERR_NOMEM: return "out of memory";
    case NUFFT3D_ERR_CUDA: return "CUDA runtime error";
    case NUFFT3D_ERR_UNSUPPORTED: return "unsupported parameters";
    case NUFFT3D_ERR_TIMEOUT: return "bounded device wait timed out";
    case NUFFT3D_ERR_DEVICE_CHECK: return "device-side consistency check failed";
  }
  return "unknown status";
}

int nufft3d_plan_info(nufft3d_plan plan, int* out) {
  if (!plan || !out) return NUFFT3D_ERR_ARG;
  int nonempty = 0;
  long long maxc = 0;
  for (size_t b = 0; b + 1 < plan->bin_offsets.size(); ++b) {
    const long long c = plan->bin_offsets[b + 1] - plan->bin_offsets[b];
    nonempty += c > 0;
    maxc = std::max(maxc, c);
  }
  out[0] = plan->T;
  out[1] = plan->nT;
  out[2] = plan->n_sub;
  out[3] = plan->gather_variant;
  out[4] = plan->spread_variant;
  out[5] = plan->pts_per_sub;
  out[6] = nonempty;
  out[7] = (int)std::min<long long>(maxc, 0x7fffffff);
  out[8] = (int)std::min<long long>(plan->P_eval, 0x7fffffff);
  out[9] = plan->n_pairs;
  out[10] = plan->L == 0 ? 1 : 0;
  out[11] = (int)std::min(std::ceil(plan->poly_err * 1e12), 2147483647.0);
  return NUFFT3D_OK;
}

int nufft3d_plan_tune(nufft3d_plan plan, int gather_variant, int spread_variant, int points_per_subproblem,
                      int tile_edge, void* cuda_stream) {
  if (!plan) return NUFFT3D_ERR_ARG;
  if (gather_variant < -1 || gather_variant > 11 || spread_variant < -1 || spread_variant > 8) return NUFFT3D_ERR_ARG;
  if (points_per_subproblem < 0 || tile_edge < 0) return NUFFT3D_ERR_ARG;
  if (tile_edge > 0 && (tile_edge != 4 && tile_edge != 8 && tile_edge != 16)) return NUFFT3D_ERR_ARG;
  if (tile_edge > 0 && (plan->K % tile_edge != 0 || tile_edge + plan->J - 1 > plan->K)) return NUFFT3D_ERR_UNSUPPORTED;
  const int T = tile_edge > 0 ? tile_edge : plan->T;
  const int gv = gather_variant >= 0 ? gather_variant : plan->gather_variant;
  const int sv = spread_variant >= 0 ? spread_variant : plan->spread_variant;
  if ((gv == 2 || sv == 2) && !nufft::v2_supported(T, plan->J, plan->L)) return NUFFT3D_ERR_UNSUPPORTED;
  if ((gv == 1 || sv == 1) && (plan->J != 6 || plan->L == 0)) return NUFFT3D_ERR_UNSUPPORTED;
  const int S_new = points_per_subproblem > 0 ? points_per_subproblem : plan->pts_per_sub;
  if ((gv == 3 || gv == 5) && !nufft::v3_supported(T, plan->J, S_new)) return NUFFT3D_ERR_UNSUPPORTED;
  if (gv == 5 && T != 8) return NUFFT3D_ERR_UNSUPPORTED;
  if ((gv == 6 || gv == 7) && !nufft::v3_two_copy_supported(T, plan->J, S_new)) return NUFFT3D_ERR_UNSUPPORTED;
  if (gv == 8 && (!plan->tmap_ok ||
                  !nufft::v8_supported(T, plan->J, S_new, plan->grid_dtype == NUFFT3D_GRID_C64 ? 8 : 4)))
    return NUFFT3D_ERR_UNSUPPORTED;
  if (gv == 4 && !nufft::v4_supported(T, plan->J, S_new, plan->L)) return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 3 && !nufft::v3s_supported(T, plan->J)) return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 4 && !nufft::v4s_supported(T, plan->J, S_new)) return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 5 && !nufft::v5s_supported(T, plan->J, S_new)) return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 6 && !nufft::v6s_supported(T, plan->J, S_new)) return NUFFT3D_ERR_UNSUPPORTED;
  if (gv == 9 && (!plan->real_ok || !nufft::v9_supported(T, plan->J, S_new))) return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 7 && (!plan->real_ok || !nufft::v7s_supported(T, plan->J, S_new))) return NUFFT3D_ERR_UNSUPPORTED;
  // the scheduled variants: real weights, T = 8, at most 256 points per subproblem
  if ((gv == 10 || gv == 11) && (!plan->real_ok || !nufft::v10_supported(T, plan->J, S_new)))
    return NUFFT3D_ERR_UNSUPPORTED;
  if (sv == 8 && (!plan->real_ok || !nufft::v8s_supported(T, plan->J, S_new))) return NUFFT3D_ERR_UNSUPPORTED;
  PLAN_DEVICE(plan);
  int rc = NUFFT3D_OK;
  CK(cudaStreamSynchronize(plan->last_stream));
  plan->gather_variant = gv;
  plan->spread_variant = sv;
  const int S = points_per_subproblem > 0 ? points_per_subproblem : plan->pts_per_sub;
  if (T != plan->T) {
    plan->T = T;
    plan->nT = plan->K / T;
    if (plan->d_sorted) {
      cudaFree(plan->d_sorted);
      plan->d_sorted = nullptr;
    }
    rc = sort_points(plan, (cudaStream_t)cuda_stream);
    if (rc != NUFFT3D_OK) return rc;
    rc = build_subproblems(plan, S, (cudaStream_t)cuda_stream);
  } else if (S != plan->pts_per_sub) {
    rc = build_subproblems(plan, S, (cudaStream_t)cuda_stream);
  }
  if (rc == NUFFT3D_OK && (gv == 10 || gv == 11 || sv == 8) && !plan->sched_ok) {
    // no schedule could be built for this split: keep runnable variants
    if (gv == 10 || gv == 11) plan->gather_variant = nufft::v9_supported(plan->T, plan->J, plan->pts_per_sub) ? 9 : 0;
    if (sv == 8) plan->spread_variant = 0;
    return NUFFT3D_ERR_UNSUPPORTED;
  }
  return rc;
}

int nufft3d_plan_set_wait_limit(nufft3d_plan plan, int first_wait_polls) {
  if (!plan) return NUFFT3D_ERR_ARG;
  plan->first_wait_polls = first_wait_polls < 0 ? -1 : first_wait_polls;
  return NUFFT3D_OK;
}

int nufft3d_plan_set_timing(nufft3d_plan plan, int max_calls) {
  if (!plan || max_calls < 0) return NUFFT3D_ERR_ARG;
  PLAN_DEVICE(plan);
  CK(cudaStreamSynchronize(plan->last_stream));
  for (cudaEvent_t e : plan->ev_fwd) cudaEventDestroy(e);
  for (cudaEvent_t e : plan->ev_adj) cudaEventDestroy(e);
  plan->ev_fwd.clear();
  plan->ev_adj.clear();
  plan->timing_slots = 0;
  plan->fwd_calls = plan->adj_calls = 0;
  const size_t nf = (size_t)max_calls * (FWD_STAGES + 1), na = (size_t)max_calls * (ADJ_STAGES + 1);
  for (size_t i = 0; i < nf + na; ++i) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    (i < nf ? plan->ev_fwd : plan->ev_adj).push_back(e);
  }
  plan->timing_slots = max_calls;
  return NUFFT3D_OK;
}

int nufft3d_plan_stage_times(nufft3d_plan plan, float* fwd_ms, float* adj_ms, int* calls) {
  if (!plan || !fwd_ms || !adj_ms || !calls) return NUFFT3D_ERR_ARG;
  PLAN_DEVICE(plan);
  CK(cudaStreamSynchronize(plan->last_stream));
  for (int s = 0; s < FWD_STAGES; ++s) fwd_ms[s] = 0.f;
  for (int s = 0; s < ADJ_STAGES; ++s) adj_ms[s] = 0.f;
  for (int c = 0; c < plan->fwd_calls; ++c)
    for (int s = 0; s < FWD_STAGES; ++s) {
      float ms = 0.f;
      cudaEvent_t* e = plan->ev_fwd.data() + (size_t)c * (FWD_STAGES + 1);
      CK(cudaEventSynchronize(e[s + 1]));
      CK(cudaEventElapsedTime(&ms, e[s], e[s + 1]));
      fwd_ms[s] += ms;
    }
  for (int c = 0; c < plan->adj_calls; ++c)
    for (int s = 0; s < ADJ_STAGES; ++s) {
      float ms = 0.f;
      cudaEvent_t* e = plan->ev_adj.data() + (size_t)c * (ADJ_STAGES + 1);
      CK(cudaEventSynchronize(e[s + 1]));
      CK(cudaEventElapsedTime(&ms, e[s], e[s + 1]));
      adj_ms[s] += ms;
    }
  calls[0] = plan->fwd_calls;
  calls[1] = plan->adj_calls;
  plan->fwd_calls = plan->adj_calls = 0;
  return NUFFT3D_OK;
}

}  // extern "C"
