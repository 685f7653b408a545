"""Parity of the exact-coefficient mode (exact_coeffs = 1) with the oracle's
exact per-point min-max coefficients (OraclePlan with L = 0: c(f) = T^-1 r(f)
solved in FP64 at every point's own offset f).

The CUDA path replaces the table by degree-8 Chebyshev fits of each c_j made
at plan time; their error (reported by plan_info) must stay below 1e-7 of
max|c|, which is below FP32 rounding of the coefficients, so the bar is the
same rel-L2 <= 1e-5 as for the table mode.  Every variant that can run
without a table is checked; those that stage the table in shared memory
must refuse the mode.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5
# fp16 grid storage meets the 1e-4 bar; bf16 (unit roundoff 2^-8) misses it by
# storage rounding, so its bound pins the measured level instead
LP_BOUND = {"bf16": 1e-3, "fp16": 1e-4}


def _plan(binding, n, dirs, m=0, k=0, j=6, **kw):
    return binding.Plan(n, dirs, m=m, k=k, j=j, exact_coeffs=True, **kw)


def _oplan(n, dirs, m=0, k=0, j=6, **kw):
    return O.OraclePlan(n, k or 2 * n, j, 0, dirs, m or 2 * n, **kw)


def _fwd_adj(plan, x, y):
    import torch

    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy() if x is not None else None
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy() if y is not None else None
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return p, a


def test_tiny_workload_exact_coefficients(cuda_lib):
    """32^3 ellipsoids, K = 64, 64 x 32 umbrella lines, M = 64."""
    w = I.workload("tiny32")
    dirs = w.directions()
    x = w.volume(np.float32)
    y = I.random_lines(dirs.shape[0], w.m, 3).astype(np.complex64)
    plan = _plan(cuda_lib, w.n, dirs, w.m, w.k, w.j)
    info = plan.info()
    assert info["exact_coeffs"] == 1
    assert 0.0 < info["coeff_fit_error"] < 1e-7, info["coeff_fit_error"]
    # the exact-mode defaults: scheduled real-weight gather, real-weight fixed-point spread
    assert info["gather_variant"] == 10 and info["spread_variant"] == 7 and info["points_per_subproblem"] == 256
    p, a = _fwd_adj(plan, x, y)
    op = _oplan(w.n, dirs, w.m, w.k, w.j)
    ef = O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op))
    ea = O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op))
    print(f"exact coefficients, tiny workload: forward {ef:.2e}, adjoint {ea:.2e}")
    assert ef < TOL and ea < TOL
    # the table plan differs from the exact one by the table's interpolation error only
    tplan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, table_oversamp=1024)
    pt, _ = _fwd_adj(tplan, x, None)
    assert O.rel_l2(pt, p) < 1e-5


@pytest.mark.parametrize("n,k,m,ndir,j", [
    (16, 32, 32, 37, 6),      # ragged line count
    (24, 48, 48, 50, 6),      # radix-3 grid and lines
    (32, 48, 64, 40, 6),      # K = 1.5 N
    (32, 96, 64, 40, 6),      # K = 3 N
    (16, 32, 32, 33, 4),      # J = 4
    (16, 32, 32, 33, 8),      # J = 8
    (20, 64, 48, 17, 2),      # J = 2, M != K
    (64, 128, 128, 300, 6),   # several tiles per axis
])
def test_shapes_and_taps(cuda_lib, n, k, m, ndir, j):
    dirs = I.random_directions(ndir, n + ndir)
    x = I.random_volume(n, 1).astype(np.float32)
    y = I.random_lines(ndir, m, 2).astype(np.complex64)
    plan = _plan(cuda_lib, n, dirs, m, k, j)
    assert plan.info()["coeff_fit_error"] < 1e-7
    p, a = _fwd_adj(plan, x, y)
    op = _oplan(n, dirs, m, k, j)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


@pytest.mark.parametrize("gv,sv,pps,tile", [(0, 0, 1024, 8), (3, 3, 512, 8), (3, 3, 37, 8), (5, 4, 512, 8),
                                            (3, 4, 300, 8), (0, 3, 77, 8), (3, 0, 1024, 16), (5, 3, 2048, 8),
                                            (6, 3, 512, 8), (7, 3, 256, 8), (7, 4, 100, 8), (8, 3, 256, 8),
                                            (8, 3, 5, 8), (5, 5, 256, 8), (8, 5, 100, 8),
                                            (5, 6, 256, 8), (8, 6, 100, 8), (3, 6, 7, 8)])
def test_variants_without_table(cuda_lib, gv, sv, pps, tile):
    n = 32
    dirs = I.umbrella_directions(35, 20)
    x = I.random_volume(n, 12).astype(np.float32)
    y = I.random_lines(dirs.shape[0], 2 * n, 13).astype(np.complex64)
    plan = _plan(cuda_lib, n, dirs)
    plan.tune(gv, sv, pps, tile)
    p, a = _fwd_adj(plan, x, y)
    op = _oplan(n, dirs)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


@pytest.mark.parametrize("gv,sv", [(1, 3), (2, 3), (4, 3), (3, 1), (3, 2)])
def test_table_staging_variants_refuse_exact_mode(cuda_lib, gv, sv):
    plan = _plan(cuda_lib, 32, I.random_directions(10, 1))
    with pytest.raises(cuda_lib.NufftError) as ei:
        plan.tune(gv, sv, 512, 8)
    assert ei.value.status == -4


def test_complex_volume_weights_raw_samples_exact(cuda_lib):
    n, ndir = 16, 45
    dirs = I.random_directions(ndir, 5)
    rng = np.random.default_rng(9)
    w = (rng.normal(size=2 * n) + 1j * rng.normal(size=2 * n)).astype(np.complex64)
    x = I.random_volume(n, 3, complex_values=True).astype(np.complex64)
    y = I.random_lines(ndir, 2 * n, 4).astype(np.complex64)
    p, a = _fwd_adj(_plan(cuda_lib, n, dirs, weight=w, complex_volume=True), x, y)
    op = _oplan(n, dirs, weight=w.astype(np.complex128), complex_volume=True)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.complex128), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL
    p, a = _fwd_adj(_plan(cuda_lib, n, dirs, complex_volume=True, do_line_fft=False), x, y)
    op = _oplan(n, dirs, complex_volume=True, do_line_fft=False)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.complex128), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_reduced_precision_grid_exact(cuda_lib, dtype):
    w = I.workload("tiny32")
    dirs = w.directions()
    x = w.volume(np.float32)
    y = I.random_lines(dirs.shape[0], w.m, 3).astype(np.complex64)
    p, a = _fwd_adj(_plan(cuda_lib, w.n, dirs, w.m, w.k, grid_dtype=dtype), x, y)
    op = _oplan(w.n, dirs, w.m, w.k)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op)) < LP_BOUND[dtype]
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_exact_mode_against_direct_nudft(cuda_lib):
    """Against the direct NUDFT the remaining error is the min-max
    interpolation error itself, the same for both coefficient modes."""
    n = 16
    dirs = I.random_directions(24, 40)
    x = I.random_volume(n, 5).astype(np.float32)
    p, _ = _fwd_adj(_plan(cuda_lib, n, dirs), x, None)
    op = _oplan(n, dirs)
    ex = O.forward_exact(x.astype(np.float64), op)
    assert O.rel_l2(p, ex) < 3e-5
