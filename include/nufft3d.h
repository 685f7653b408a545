/*
 * nufft3d.h -- C ABI of the GB300 radial-line 3D NUFFT projector.
 *
 * The library computes the image-to-Radon step of a Fourier-based cone-beam CT
 * forward projector (the paper's Sec. 2, step 1, and Sec. 2.2.1) and its
 * transpose (the backprojection direction of Sec. 2.3):
 *
 *   forward   p = L_w  T  F  P  x
 *   adjoint   x~ = P^H F^H T^H L_w^H p
 *
 *   P   deapodisation (the diagonal pre-scaling P of Eq. 2.11) of the N^3 volume
 *       and zero padding to the oversampled K^3 grid;
 *   F   unnormalised 3D DFT on the K^3 grid (e^{-i}, centred voxel index
 *       n in [-N/2, N/2)^3);
 *   T   separable J-tap min-max interpolation (the sparse interpolator
 *       T_sparse of Eq. 2.11) onto points omega_{l,q} = r_q d_l on radial
 *       lines through the origin (Eq. 2.1);
 *   L_w per-line centred inverse DFT with radial weight w[q] and 1/M scaling,
 *       which turns Fourier samples on a line into plane integrals by the
 *       Fourier Slice Theorem (Sec. 2.2.1).
 *
 * Conventions
 *   volume  C-ordered [z][y][x], x fastest, N^3 elements; float32 (real) or
 *           interleaved complex64; voxel (z,y,x) has centred index
 *           n = (x - N/2, y - N/2, z - N/2).
 *   lines   [dir][m], m fastest, interleaved complex64, n_dirs * M elements;
 *           sample m has radial index q = m - M/2; line-FFT output index t has
 *           plane offset s = t - M/2 (voxel units along d).
 *   dirs    unit vectors (x, y, z) in float64, copied at plan creation.
 *   grid    u = omega / gamma, gamma = 2 pi / K; taps k0 + 1 .. k0 + J with
 *           k0 = floor(u) - J/2 (J even), f = u - floor(u).  The min-max
 *           coefficients c(f) = T^-1 r(f) (Eq. 2.11's interpolator) are either
 *           exact at each point's own f (exact_coeffs = 1: degree-8 polynomial
 *           fits, FP64-fitted, evaluated in FP32 per point) or linearly
 *           interpolated from a table of L + 1 rows at f = i / L
 *           (exact_coeffs = 0).
 *   device  every call that takes a plan or a batch runs on the device that
 *           was current when it was created and restores the caller's current
 *           device before returning.
 *
 * Ownership and threading
 *   The caller owns every device buffer passed in and the CUDA stream.  A plan
 *   owns its tables, its point sort and its workspace (device memory allocated
 *   at creation).  All compute calls are asynchronous on the given stream; a
 *   status raised by a device-side check is kept in a device word and
 *   returned by nufft3d_plan_sync_status.  A plan must not be used from two
 *   host threads at once; distinct plans are independent.
 *
 * Errors
 *   Every function returns a nufft3d_status (0 = success).  No function
 *   aborts, throws across the ABI or traps on the device.
 */
#ifndef NUFFT3D_H
#define NUFFT3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nufft3d_plan_s* nufft3d_plan;   /* opaque, library-owned */

typedef enum {
  NUFFT3D_OK = 0,
  NUFFT3D_ERR_ARG = -1,           /* invalid argument (NULL, size out of range)        */
  NUFFT3D_ERR_NOMEM = -2,         /* device or host allocation failed                 */
  NUFFT3D_ERR_CUDA = -3,          /* a CUDA runtime call failed                        */
  NUFFT3D_ERR_UNSUPPORTED = -4,   /* valid request this build does not implement       */
  NUFFT3D_ERR_TIMEOUT = -5,       /* a bounded device wait ran out                     */
  NUFFT3D_ERR_DEVICE_CHECK = -6   /* a device-side consistency check failed            */
} nufft3d_status;

typedef enum {
  NUFFT3D_GRID_C64 = 0,           /* oversampled grid stored as complex64              */
  NUFFT3D_GRID_BF16 = 1,          /* forward grid stored as bf16 pairs, FP32 math      */
  NUFFT3D_GRID_FP16 = 2           /* forward grid stored as fp16 pairs, FP32 math      */
} nufft3d_grid_dtype;

typedef struct {
  int n;                  /* volume edge N: even, 8 <= N <= 512                        */
  int k;                  /* grid edge K: 0 selects 2N; K >= N, K = 2^a 3^b, K <= 1024 */
  int j;                  /* taps per axis J: even, 2 <= J <= 8 (0 selects 6)          */
  int table_oversamp;     /* coefficient table oversampling L (0 selects 1024), 2^p    */
  int n_dirs;             /* number of radial lines D >= 1                             */
  const double* dirs;     /* host, D x 3 unit vectors (x, y, z); copied               */
  int m;                  /* samples per line M: even, 0 selects 2N; M = 2^a 3^b, <= 1024 */
  const double* omega;    /* host, M radial frequencies (rad/voxel), or NULL for
                             2 pi (m - M/2) / M; |omega| <= pi; copied                 */
  const float* weight;    /* host, M interleaved complex radial weights w[q], or NULL
                             for w = 1; copied                                         */
  int grid_dtype;         /* nufft3d_grid_dtype                                        */
  int complex_volume;     /* 0: float32 real volume in/out; 1: complex64              */
  int do_line_fft;        /* 1: plane integrals (line inverse DFT applied);
                             0: raw Fourier samples X^(omega) (no line DFT)            */
  int keep_duplicates;    /* 0: a sample that coincides with another one (line l' =
                             -line l within 1e-13, radius -r) is interpolated once and
                             its value shared (the partner direction is snapped to the
                             exact negation); 1: every sample separately           */
  int exact_coeffs;       /* 0: coefficients linearly interpolated from the table of
                             L + 1 rows c(i / L); 1: the exact min-max coefficients
                             c(f) = T^-1 r(f) at each point's own f (table_oversamp is
                             ignored).  The plan fits each c_j by a degree-8 Chebyshev
                             interpolant in FP64 and evaluates it per point in FP32;
                             a fit further than 1e-7 max|c| from c is refused with
                             NUFFT3D_ERR_UNSUPPORTED (plan_info reports the error) */
  const float* line_weight; /* host, D real per-line weights lw[l], or NULL for 1; the
                             line DFTs use lw[l] w[q] (forward) and lw[l] conj(w[q])
                             (adjoint); copied.  With the weights of
                             nufft3d_fourier_slice_weights the adjoint is the
                             direct reconstruction of Sec. 2.3 */
} nufft3d_params;

/* Create a plan.  Validates *p, computes in FP64 on the host the scaling
 * factors s(n) (Kaiser-Bessel pre-window, Eq. 2.11), the min-max coefficient
 * table and the FFT twiddles, uploads them, sorts the D*M points by grid tile
 * (a device pass plus a host counting sort) and allocates the workspace, all
 * on `cuda_stream` (a cudaStream_t, may be NULL for the legacy stream), which
 * it synchronises before returning.  On success *out holds a new plan; on
 * failure *out is NULL and nothing is leaked. */
int nufft3d_plan_create(nufft3d_plan* out, const nufft3d_params* p, void* cuda_stream);

/* Forward projection: vol_dev (device, N^3 float32 or complex64 per
 * complex_volume) -> lines_dev (device, D*M complex64).  Enqueued on
 * cuda_stream; buffers must not overlap; vol_dev is not modified.  The
 * workspace of the plan is used, so calls on one plan serialise on the stream. */
int nufft3d_forward(nufft3d_plan plan, const void* vol_dev, void* lines_dev, void* cuda_stream);

/* Adjoint (backprojection direction): lines_dev (device, D*M complex64) ->
 * vol_dev (device, N^3 float32 = real part, or complex64).  lines_dev is not
 * modified.  Exact conjugate transpose of nufft3d_forward for complex volumes;
 * for real volumes the adjoint with respect to Re<.,.>. */
int nufft3d_adjoint(nufft3d_plan plan, const void* lines_dev, void* vol_dev, void* cuda_stream);

/* Bytes of device memory a plan with these parameters holds (tables, point
 * sort, workspace: the forward grid, a separate adjoint grid that the
 * adjoint keeps clear between calls unless the forward grid is bf16/fp16,
 * the FFT intermediates and the line buffer).  Host only: touches no device. */
int nufft3d_workspace_bytes(const nufft3d_params* p, size_t* bytes);

/* Synchronise the plan's last stream and return, in *device_status, the
 * device-side check word (0 = clean; otherwise a nufft3d_status); the word is
 * cleared.  Returns NUFFT3D_ERR_CUDA if the synchronisation itself failed. */
int nufft3d_plan_sync_status(nufft3d_plan plan, int* device_status);

/* Free a plan and everything it owns (NULL is accepted). */
int nufft3d_plan_destroy(nufft3d_plan plan);

/* Direct resampling of the polar Radon grid (Sec. 2.1, Eq. 2.15 with the
 * second sparse operator the identity).  The radially sampled Radon data are
 * uniform in (s, theta, phi) (Fig. 2.10); a separable truncated-sinc
 * interpolator with J taps per axis (the paper's runs: J = 3, Sec. 3.2) takes
 * them to arbitrary points:
 *   out[i] = sum_k sinc(u_s - k_s) sinc(u_theta - k_theta) sinc(u_phi - k_phi)
 *            grid[k_phi mod n_phi][k_theta][k_s],
 * sinc(t) = sin(pi t) / (pi t), k0 .. k0 + J - 1 on each axis with
 * k0 = floor(u - J/2) + 1.  The azimuth is periodic; taps beyond the ends of
 * the theta and s ranges add nothing.
 *   grid_dev    device, complex64 [n_phi][n_theta][n_s] (interleaved re, im):
 *               the forward projector's [D][M] lines with D = n_phi n_theta in
 *               azimuth-major order fit it as is; not modified
 *   targets_dev device, float32 [n_targets][3] = (u_s, u_theta, u_phi) in
 *               grid-index units; a coordinate that is not finite or is 2^24
 *               or more in magnitude gives a NaN output
 *   J           taps per axis, 2 ... 8
 *   out_dev     device, complex64 [n_targets]; must not overlap the inputs
 *   cuda_stream the stream to run on (NULL: the legacy default stream)
 * All buffers are the caller's; nothing is allocated.  Asynchronous: the
 * result is ready when the stream reaches it.  Returns NUFFT3D_OK (also for
 * n_targets = 0, with any pointers), NUFFT3D_ERR_ARG (negative count, sizes
 * below 1 or a grid above 2^40 cells, J outside 2 ... 8, a NULL pointer with
 * n_targets > 0) or NUFFT3D_ERR_CUDA (the launch failed). */
int nufft3d_polar_resample(const void* grid_dev, int n_phi, int n_theta, int n_s, const float* targets_dev,
                           long long n_targets, int J, void* out_dev, void* cuda_stream);

/* NUFFT-based resampling of the polar Radon grid (Sec. 2.1.3, Eqs. 2.8-2.11):
 *   out ~= T_sparse F P F^-1 grid,
 * the fast form of the ideal periodic-sinc resampler of Eq. 2.8,
 *   out[i] = sum_m a[m] e^{-2 pi i (m_s u_s / n_s + m_theta u_theta / n_theta
 *                                   + m_phi u_phi / n_phi)},
 *   a = F^-1 grid, a[m] = (1/n) sum_k grid[k] e^{+2 pi i m.k / n},
 * m_a = -n_a/2 .. n_a/2 - 1 on every axis (all axes periodic, as the DFT makes
 * them).  P is the Kaiser-Bessel pre-window of each axis, symmetric about the
 * middle of its index range; F the unnormalised DFT of the zero-padded
 * spectrum at K_a = 2 n_a (twofold oversampling); T_sparse the J-tap min-max
 * interpolator per axis at u' = 2 u, with exact coefficients (fitted
 * polynomials, relative fit error at most 1e-7).  Accuracy: the min-max error
 * of J = 6 taps at K = 2n, about 1e-6 relative (rel-L2 against Eq. 2.8).
 *
 * A plan owns its tables and workspace (K_phi K_theta K_s + n_phi K_theta K_s
 * complex64 cells; nufft3d_polar_nufft_info reports the bytes) on the device
 * current at creation; every call runs on that device and restores the
 * caller's.  Calls on one plan must be serialised (they share the workspace).
 *
 * nufft3d_polar_nufft_create: n_phi, n_theta, n_s each one of 10, 12, 16, 20,
 *   24, 32, 40, 64, 90, 128, 180, 256, 360, 384, 512; J one of 4, 6, 8.
 *   Returns NUFFT3D_OK, NUFFT3D_ERR_ARG (NULL out, a size below 1),
 *   NUFFT3D_ERR_UNSUPPORTED (another size or J, or a coefficient fit above
 *   1e-7), NUFFT3D_ERR_NOMEM or NUFFT3D_ERR_CUDA.
 * nufft3d_polar_nufft_prepare: F P F^-1 of grid_dev (device, complex64
 *   [n_phi][n_theta][n_s], interleaved re, im; the forward projector's [D][M]
 *   lines with D = n_phi n_theta in azimuth-major order fit it as is; not
 *   modified) into the plan's oversampled spectrum: three HBM-bound passes
 *   (s, theta, phi).  Asynchronous on cuda_stream (NULL: the legacy stream).
 * nufft3d_polar_nufft_gather: T_sparse of the last prepared spectrum at
 *   targets_dev (device, float32 [n_targets][3] = (u_s, u_theta, u_phi) in
 *   grid-index units; a coordinate that is not finite or is 2^22 or more in
 *   magnitude gives a NaN output) into out_dev (device, complex64 [n_targets],
 *   not overlapping the targets).  NUFFT3D_OK also for n_targets = 0 with any
 *   pointers; NUFFT3D_ERR_ARG for a negative count or a NULL pointer with
 *   n_targets > 0.
 * nufft3d_polar_nufft_resample: prepare, then gather, on one stream.
 * nufft3d_polar_nufft_destroy frees the plan (NUFFT3D_ERR_ARG for NULL). */
typedef struct nufft3d_polar_nufft_s* nufft3d_polar_nufft;
int nufft3d_polar_nufft_create(nufft3d_polar_nufft* out, int n_phi, int n_theta, int n_s, int J);
int nufft3d_polar_nufft_info(nufft3d_polar_nufft p, long long* workspace_bytes, double* fit_error);
int nufft3d_polar_nufft_prepare(nufft3d_polar_nufft p, const void* grid_dev, void* cuda_stream);
int nufft3d_polar_nufft_gather(nufft3d_polar_nufft p, const float* targets_dev, long long n_targets, void* out_dev,
                               void* cuda_stream);
int nufft3d_polar_nufft_resample(nufft3d_polar_nufft p, const void* grid_dev, const float* targets_dev,
                                 long long n_targets, void* out_dev, void* cuda_stream);
int nufft3d_polar_nufft_destroy(nufft3d_polar_nufft p);

/* Per-view reverse Grangeat step (Sec. 2.2.2, Fig. 2.15; costs C3a-C3d of
 * Sec. 2.4): every cone-beam view's umbrella subset of the (derivative of
 * the) Radon data, L lines at detector-plane angles alpha_l with M samples at
 * offsets t - M/2, to its N x N detector image:
 *   C3a  y'[l][t] = w_post[l][t] y[l][t]
 *   C3b  Y[l][q]  = sum_t y'[l][t] e^{-2 pi i (q - M/2)(t - M/2) / M}
 *   C3c  z[n]     ~= sum_{l,q} Y[l][q] e^{+i omega_lq . n},
 *        omega_lq = 2 pi (q - M/2)/M (cos alpha_l, sin alpha_l) = (omega_x,
 *        omega_y), n = (n_y, n_x) centred in [-N/2, N/2)^2: the 2D min-max
 *        NUFFT transpose (K = 2N, J x J taps; the paper uses [5 5])
 *   C3d  out[n]   = w_pre[n] z[n]
 * No ramp filter (the data are already derivatives).  The Grangeat weights
 * are defined outside the paper, so both are the caller's.  Accuracy: the
 * min-max error of J taps at K = 2N (about 1e-4 relative for J = 5, 1e-6 for
 * J = 6), FP32 arithmetic.
 *
 * nufft3d_grangeat_create: N (detector edge) one of 16, 32, 64, 128, 256; M
 *   one of 16, 32, 64, 128, 256, 512; 1 <= L <= 65535; 2 <= J <= 8; angles
 *   host float64 [L] (finite; copied); max_views >= 1 sets the workspace:
 *   (L M + 4 N^2 + 2 N^2) complex64 per view plus the sparse spread matrix
 *   (L M J^2 entries, 12 bytes each).  The plan is built on the current
 *   device; calls run there and restore the caller's device.  Returns
 *   NUFFT3D_OK, NUFFT3D_ERR_ARG, NUFFT3D_ERR_UNSUPPORTED (another size, or a
 *   coefficient fit above 1e-7), NUFFT3D_ERR_NOMEM or NUFFT3D_ERR_CUDA.
 * nufft3d_grangeat_run: n_views views in chunks of max_views on cuda_stream:
 *   y_dev complex64 [n_views][L][M], w_post_dev float32 [n_views][L][M],
 *   w_pre_dev float32 [n_views][N][N] (all device, not modified), out_dev
 *   complex64 [n_views][N][N] (device, not overlapping the inputs).
 *   Asynchronous.  NUFFT3D_OK also for n_views = 0 with any pointers.
 * nufft3d_grangeat_info: workspace bytes, entries of the spread matrix and
 *   the coefficient fit error (any output may be NULL).
 * The spread sums the cells near the origin (rows of more than 32 entries)
 * with FP32 atomics, so repeated calls can differ in the last bits there. */
typedef struct nufft3d_grangeat_s* nufft3d_grangeat;
int nufft3d_grangeat_create(nufft3d_grangeat* out, int N, int L, int M, int J, const double* angles, int max_views);
int nufft3d_grangeat_info(nufft3d_grangeat g, long long* workspace_bytes, long long* nnz, double* fit_error);
int nufft3d_grangeat_run(nufft3d_grangeat g, const void* y_dev, const float* w_post_dev, const float* w_pre_dev,
                         int n_views, void* out_dev, void* cuda_stream);
int nufft3d_grangeat_destroy(nufft3d_grangeat g);

/* Weights that turn the adjoint into the direct (Fourier-slice) reconstruction
 * that inverts the image-to-Radon step (Sec. 2.3: ramp filtering in the
 * Fourier domain, then the NUFFT transpose; Sec. 1: the 3D parallel-beam
 * ramp filter is R^2).  The reconstruction is a quadrature of the inverse 3D
 * Fourier transform in spherical coordinates, x[n] ~ (2 pi)^-3 sum |w|^2 dw
 * dOmega X(w) e^{i w.n}, over the umbrella directions of Eq. 2.1 (phi_a = 2 pi
 * a / n_az, theta_p = c + (pi - 2c)(p + 1/2) / n_pol, c = cone_half_angle,
 * azimuth-major l = a n_pol + p).  Every Fourier point lies on two antipodal
 * lines, and the adjoint's line DFT carries a factor 1/M, so:
 *   line_weight[l]  = sin(theta_p) (pi - 2c)/n_pol (2 pi/n_az) / 2  (half the solid-angle cell)
 *   radial_weight[q] = q^2 / M^2 for q != 0 (complex, imaginary part 0),
 *   radial_weight[0] = pi / (6 M^2 sum_l line_weight[l])   (the ball |w| < pi/M around the origin)
 * for q = m - M/2.  radial_weight holds 2 M floats (interleaved complex),
 * line_weight n_az n_pol floats.  Pass them as weight and line_weight of a plan
 * over those directions with do_line_fft = 1 and M samples per line; its
 * adjoint of plane integrals is the reconstruction.  Host only. */
int nufft3d_fourier_slice_weights(int n_az, int n_pol, double cone_half_angle, int m, float* radial_weight,
                                  float* line_weight);

/* Measurement utility (no counterpart in the paper): the FP32 fused
 * multiply-add throughput of the current device, measured with a kernel of
 * independent FMA chains on every SM (the fastest of five timed launches,
 * CUDA events on cuda_stream; about 10 ms of GPU time), in TFLOP/s (two
 * flops per FMA), and the device's SM count.  It allocates and frees a small
 * scratch buffer.  The arithmetic roofline of the interpolation kernels is
 * quoted against this number.  Returns NUFFT3D_ERR_ARG for NULL outputs,
 * NUFFT3D_ERR_CUDA if a CUDA call fails. */
int nufft3d_fp32_fma_peak(double* tflops, int* sm_count, void* cuda_stream);

/* Static description of a status code (never NULL). */
const char* nufft3d_error_string(int status);

/* Numbers of the plan; out must hold 12 ints: tile edge T, tiles per axis,
 * subproblems, gather variant, spread variant, points per subproblem,
 * non-empty tiles, most points in one tile, evaluated points (samples after
 * merging coincident ones), merged antipodal line pairs, exact_coeffs, and the
 * coefficient polynomials' largest error relative to max|c| in units of 1e-12
 * (rounded up; 0 with a table).  For tests and tuning. */
int nufft3d_plan_info(nufft3d_plan plan, int* out);

/* Select the gather and spread kernel variants, the number of points per
 * subproblem and the grid tile edge T of a plan (-1 / 0 keep the current
 * choice).  Variants: 0 one thread per point, one CTA per subproblem (any
 * J); 1 one warp per point, CTA-shared tile (J = 6); 2 one warp per point,
 * warp-private tile, no shared atomics (J = 6, T = 8); gather only: 3 one thread per point, points reordered so
 * that every half-warp's tile accesses fall in distinct banks (any J; the
 * default gather with a table), 4 the same with the table in shared memory, 5
 * the same as 3 with 128-thread CTAs (T = 8; the default with exact_coeffs,
 * with 256 points per subproblem instead of 512), 6 and 7 the same as 3
 * and 5 with two copies of the tile in shared memory, the second shifted by
 * half the bank range, so that the points of two residue classes can be dealt
 * evenly to both (J = 6, T = 8), 8 the same as 5 with persistent CTAs that
 * copy the next subproblem's tile into shared memory with a TMA tensor copy
 * while the current one is computed (J = 6, T = 8; needs the tensor map the
 * plan encodes for its grid); spread only: 3 variant 2 with ten warps per SM and
 * the table read through L1 (the default spread with a table), 4 one thread per point in
 * rounds of pairwise distinct tile-offset residues (no atomics), 5 variant 3
 * with the tile accumulated in 32-bit fixed point by shared-memory integer
 * adds, in units of a power-of-two scale per subproblem set by the largest
 * |v| max|cx| max|cy| max|cz| of its points (J = 6, T = 8, at most 512 points
 * per subproblem; samples whose bound exceeds 2^100, or is not finite, make
 * the tile NaN), 6 the arithmetic of 5 with one tile shared by the six
 * warps of a CTA, four CTAs per SM, and one scale per subproblem from the
 * largest bound of all its points (J = 6, T = 8, at most 256 points per
 * subproblem; the default spread with exact_coeffs).  T is 4, 8 or 16;
 * changing it re-sorts the points.
 * Synchronises the plan's last stream and works on cuda_stream.  Returns
 * NUFFT3D_ERR_UNSUPPORTED for a combination the plan cannot run.  Used by
 * the autotuner. */
int nufft3d_plan_tune(nufft3d_plan plan, int gather_variant, int spread_variant,
                      int points_per_subproblem, int tile_edge, void* cuda_stream);

/* Allocation-free adjoint.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory when they need the adjoint
 * (code running while a stream is captured into a CUDA graph in global capture
 * mode, host frameworks whose device memory belongs to their own pool
 * allocator, real-time loops that must stay out of the driver's allocator).
 * Same arguments and result as nufft3d_adjoint on the same plan, but every
 * scratch buffer (line-DFT output, K^3 grid, inverse-FFT intermediates, work
 * counters) comes from one static 8 MiB device array inside the library, not
 * from the plan's workspace; it calls no cudaMalloc, cudaFree or allocating
 * library routine.  Limit: (D*M if the plan applies the line DFT) + K^3 +
 * N*K^2 + N^2*K complex64 values, each rounded up to 256 bytes, plus 256 bytes,
 * must fit in 8 MiB (for example N = 32, K = 64 with D*M up to about 500,000);
 * larger plans return NUFFT3D_ERR_UNSUPPORTED.  Every GPU that loads the
 * library holds the 8 MiB until the process exits.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  All calls share the one array
 * (which keeps the last call's contents; the grid and counters are cleared on
 * every call): calls that overlap on the GPU, on any streams or plans, race. */
int nufft3d_adjoint_noalloc(nufft3d_plan plan, const void* lines_dev, void* vol_dev, void* cuda_stream);

/* Testing hook for the bounded device waits.  The TMA gather (variant 8)
 * waits on an mbarrier for each tile copy; a wait that runs out of polls sets
 * NUFFT3D_ERR_TIMEOUT in the plan's device check word, after which the CTA
 * waits (with the full limit) for its copies still in flight and returns, so
 * the context stays usable and the call's output is incomplete.
 * first_wait_polls >= 0 caps the first wait on every copy at that many polls
 * (0: it gives up at once), which makes the timeout path run on demand;
 * first_wait_polls < 0 restores the default limit (2^22 polls).  Host only;
 * takes effect from the next call.  Returns NUFFT3D_ERR_ARG for a NULL plan. */
int nufft3d_plan_set_wait_limit(nufft3d_plan plan, int first_wait_polls);

/* Per-stage timing with CUDA events recorded on the launching stream between
 * the kernels of each call.  nufft3d_plan_set_timing(plan, n) arms timing of
 * the next n forward and n adjoint calls (0 disarms; it synchronises the
 * plan's last stream and recreates the events).  nufft3d_plan_stage_times
 * synchronises, writes the summed milliseconds of each stage of the recorded
 * calls to fwd_ms[5] (x pass, y pass, z pass, gather, line DFT) and
 * adj_ms[6] (line DFT, grid clear, spread, z pass, y pass, x pass), the
 * numbers of recorded forward and adjoint calls to calls[2], and re-arms. */
int nufft3d_plan_set_timing(nufft3d_plan plan, int max_calls);
int nufft3d_plan_stage_times(nufft3d_plan plan, float* fwd_ms, float* adj_ms, int* calls);

/* ---------------------------------------------------------------------------
 * Host-to-host use: the forward projection and its adjoint of volumes held in
 * host memory (the way a reconstruction program on the CPU calls the
 * projector; the paper's own projector runs on the host, Sec. 3.2).  A
 * pipeline owns two sets of device buffers (volume, lines, output volume) and
 * three streams: every call copies the volume in on the upload stream, runs
 * the plan's forward and adjoint on the compute stream and copies the lines
 * and the output volume out on the download stream, so the copies of one
 * call overlap the kernels of its neighbours.  Host buffers: vol_host N^3
 * float32 (complex64 with complex_volume), lines_host D*M complex64,
 * vol_out_host like vol_host; they should be page-locked (cudaHostAlloc or
 * cudaHostRegister) for the copies to overlap, and must stay untouched until
 * nufft3d_host_pipeline_sync returns.  nufft3d_host_forward_adjoint is
 * asynchronous; nufft3d_host_pipeline_sync waits for every call so far and
 * returns NUFFT3D_ERR_CUDA if any of it failed.  The plan must outlive the
 * pipeline and must not be used on other streams while calls are in flight;
 * destroying the pipeline hands the plan back to the legacy default stream
 * (the stream nufft3d_plan_sync_status synchronises) until its next call.
 * create allocates 2 (2 N^3 + D M) elements of device memory.
 * ------------------------------------------------------------------------- */
typedef struct nufft3d_host_pipeline_s* nufft3d_host_pipeline;   /* opaque */
int nufft3d_host_pipeline_create(nufft3d_plan plan, nufft3d_host_pipeline* out);
int nufft3d_host_forward_adjoint(nufft3d_host_pipeline pipe, const void* vol_host, void* lines_host,
                                 void* vol_out_host);
int nufft3d_host_pipeline_sync(nufft3d_host_pipeline pipe);
int nufft3d_host_pipeline_destroy(nufft3d_host_pipeline pipe);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems of mixed sizes and view counts (the
 * batched use of one projector over several volumes; the paper runs one
 * problem at a time).  A batch owns one plan per item (created from ps[i] as
 * by nufft3d_plan_create).  nufft3d_batch_forward_adjoint runs, for every
 * item i, vols[i] -> lines[i] (forward) then lines[i] -> vols_out[i]
 * (adjoint), all device buffers laid out as for a single plan.  The first
 * call captures the whole sequence into one CUDA graph (items dealt to up to
 * 12 worker streams forked from cuda_stream, largest items first to the least
 * loaded stream) and every call replays it with a
 * single graph launch on cuda_stream; passing different buffers, or calling
 * nufft3d_batch_invalidate (after re-tuning an item plan), captures again.
 * Item plans are reachable with nufft3d_batch_item for tuning; they must not
 * be destroyed by the caller.
 * ------------------------------------------------------------------------- */
typedef struct nufft3d_batch_s* nufft3d_batch;   /* opaque, library-owned */
int nufft3d_batch_create(nufft3d_batch* out, const nufft3d_params* ps, int count, void* cuda_stream);
int nufft3d_batch_size(nufft3d_batch batch, int* count);
int nufft3d_batch_item(nufft3d_batch batch, int i, nufft3d_plan* plan);
int nufft3d_batch_forward_adjoint(nufft3d_batch batch, const void* const* vols, void* const* lines,
                                  void* const* vols_out, void* cuda_stream);
int nufft3d_batch_invalidate(nufft3d_batch batch);
/* Grouped launches (off by default): items that share N, K and J and run the
 * exact-coefficient default kernels (scheduled gather 10, real-weight spread
 * 7, complex64 grid) are captured as groups of up to 32.  Their FFT passes and
 * line DFTs still run per item on the worker streams, but each group's
 * interpolation is one gather launch over all its items' subproblems and one
 * persistent spread launch whose CTAs take (item, subproblem) work from a
 * single counter.  On the 24-item mixed batch of 64^3, 128^3 and 192^3
 * problems this measured slower (28.4 ms against 26.2 ms per forward +
 * adjoint on a GB300): the per-item sequences on 12 streams already overlap
 * one item's HBM-bound FFT passes with another's interpolation, and a group's
 * launch waits for all its items' passes.  on = 1 selects it; the next call
 * captures again. */
int nufft3d_batch_set_grouping(nufft3d_batch batch, int on);
int nufft3d_batch_destroy(nufft3d_batch batch);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT3D_H */
