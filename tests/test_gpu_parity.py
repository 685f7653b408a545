"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (the method's floating-point contract): relative L2 error at most 1e-5
against the table-coefficient oracle on the same seeded inputs, for both the
forward projection and its adjoint; the adjoint also passes the dot-product
test to 1e-6.  Sizes span several shared-memory tiles, ragged line counts,
radix-3 grid sizes, non-default taps, weights and radial frequencies.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _run(binding, n, dirs, m=0, k=0, j=6, L=1024, x=None, y=None, gather_variant=-1, **kw):
    import torch

    plan = binding.Plan(n, dirs, m=m, k=k, j=j, table_oversamp=L, **kw)
    if gather_variant >= 0:
        try:
            plan.tune(gather_variant, -1, 512 if gather_variant == 4 else 0)
        except binding.NufftError as e:
            if e.status == -4:
                pytest.skip(f"gather variant {gather_variant} does not fit this plan")
            raise
    out = {}
    if x is not None:
        out["fwd"] = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    if y is not None:
        out["adj"] = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    plan.close()
    return out


def _oplan(n, dirs, m=0, k=0, j=6, L=1024, **kw):
    return O.OraclePlan(n, k or 2 * n, j, L, dirs, m or 2 * n, **kw)


def test_tiny_workload_forward_adjoint(cuda_lib):
    """32^3 ellipsoids, K = 64, 64 x 32 umbrella lines, M = 64 (131k points)."""
    w = I.workload("tiny32")
    dirs = w.directions()
    x = w.volume(np.float32)
    y = I.random_lines(dirs.shape[0], w.m, 3).astype(np.complex64)
    r = _run(cuda_lib, w.n, dirs, w.m, w.k, w.j, w.table_oversamp, x=x, y=y)
    op = _oplan(w.n, dirs, w.m, w.k, w.j, w.table_oversamp)
    ef = O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.float64), op))
    ea = O.rel_l2(r["adj"], O.nufft_adjoint(y.astype(np.complex128), op))
    assert ef < TOL, ef
    assert ea < TOL, ea
    # against the exact transform the NUFFT approximation error dominates
    lines = np.arange(0, dirs.shape[0], 31)
    ex = O.forward_exact(x.astype(np.float64), op, lines=lines)
    assert O.rel_l2(r["fwd"][lines], ex) < 3e-5


@pytest.mark.parametrize("gv", [-1, 3, 4, 5])
@pytest.mark.parametrize("n,k,m,ndir,j,L", [
    (16, 32, 32, 37, 6, 1024),     # ragged line count (not a multiple of 16)
    (24, 48, 48, 50, 6, 1024),     # radix-3 grid and line lengths
    (32, 96, 64, 40, 6, 512),      # K = 3N, table L = 512
    (16, 32, 32, 33, 4, 1024),     # J = 4
    (16, 32, 32, 33, 8, 256),      # J = 8
    (20, 64, 48, 17, 2, 2048),     # J = 2, M != K
    (64, 128, 128, 300, 6, 1024),  # several 16^3 tiles per axis
])
def test_shapes_taps_tables(cuda_lib, n, k, m, ndir, j, L, gv):
    dirs = I.random_directions(ndir, n + ndir)
    x = I.random_volume(n, 1).astype(np.float32)
    y = I.random_lines(ndir, m, 2).astype(np.complex64)
    r = _run(cuda_lib, n, dirs, m, k, j, L, x=x, y=y, gather_variant=gv)
    op = _oplan(n, dirs, m, k, j, L)
    assert O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(r["adj"], O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_complex_volume_weights_and_raw_samples(cuda_lib):
    n, ndir = 16, 45
    dirs = I.random_directions(ndir, 5)
    rng = np.random.default_rng(9)
    w = (rng.normal(size=2 * n) + 1j * rng.normal(size=2 * n)).astype(np.complex64)
    x = I.random_volume(n, 3, complex_values=True).astype(np.complex64)
    y = I.random_lines(ndir, 2 * n, 4).astype(np.complex64)
    r = _run(cuda_lib, n, dirs, x=x, y=y, weight=w, complex_volume=True)
    op = _oplan(n, dirs, weight=w.astype(np.complex128), complex_volume=True)
    assert O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.complex128), op)) < TOL
    assert O.rel_l2(r["adj"], O.nufft_adjoint(y.astype(np.complex128), op)) < TOL
    r = _run(cuda_lib, n, dirs, x=x, y=y, complex_volume=True, do_line_fft=False)
    op = _oplan(n, dirs, complex_volume=True, do_line_fft=False)
    assert O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.complex128), op)) < TOL
    assert O.rel_l2(r["adj"], O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_custom_radial_frequencies(cuda_lib):
    n, ndir, m = 16, 20, 30
    dirs = I.random_directions(ndir, 6)
    omega = np.sort(np.random.default_rng(1).uniform(-np.pi, np.pi, m))
    x = I.random_volume(n, 4).astype(np.float32)
    y = I.random_lines(ndir, m, 5).astype(np.complex64)
    r = _run(cuda_lib, n, dirs, m=m, x=x, y=y, omega=omega, do_line_fft=False)
    op = _oplan(n, dirs, m=m, omega=omega, do_line_fft=False)
    assert O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(r["adj"], O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_axis_aligned_lines_give_slice_sums(cuda_lib):
    """Fourier-slice exactness: lines along the axes return plain slice sums."""
    n = 32
    x = I.random_volume(n, 8).astype(np.float32)
    r = _run(cuda_lib, n, I.axis_directions(), x=x)
    sums = [x.sum(axis=(0, 1)), x.sum(axis=(0, 2)), x.sum(axis=(1, 2))]
    for a in range(3):
        expect = np.zeros(2 * n)
        expect[n // 2: n // 2 + n] = sums[a]
        assert np.max(np.abs(r["fwd"][a] - expect)) < 3e-5 * np.abs(expect).max()


def test_adjoint_dot_product_gpu(cuda_lib):
    import torch

    n, ndir = 32, 500
    dirs = I.random_directions(ndir, 77)
    plan = cuda_lib.Plan(n, dirs, complex_volume=True)
    x = torch.from_numpy(I.random_volume(n, 1, complex_values=True).astype(np.complex64)).cuda()
    y = torch.from_numpy(I.random_lines(ndir, 2 * n, 2).astype(np.complex64)).cuda()
    Ax = plan.forward(x)
    Ahy = plan.adjoint(y)
    lhs = torch.vdot(y.flatten().to(torch.complex128), Ax.flatten().to(torch.complex128))
    rhs = torch.vdot(Ahy.flatten().to(torch.complex128), x.flatten().to(torch.complex128))
    denom = torch.linalg.norm(Ax.to(torch.complex128)) * torch.linalg.norm(y.to(torch.complex128))
    assert abs(complex(lhs - rhs)) / float(denom) < 1e-6


def test_degenerate_single_line_and_dc_only(cuda_lib):
    """One line, and a line of two samples (q = -1, 0)."""
    n = 8
    x = I.random_volume(n, 2).astype(np.float32)
    dirs = np.array([[0.0, 0.6, 0.8]])
    r = _run(cuda_lib, n, dirs, m=16, x=x, y=I.random_lines(1, 16, 3).astype(np.complex64))
    op = _oplan(n, dirs, m=16)
    assert O.rel_l2(r["fwd"], O.nufft_forward(x.astype(np.float64), op)) < TOL
    r = _run(cuda_lib, n, dirs, m=2, x=x, do_line_fft=False)
    op = _oplan(n, dirs, m=2, do_line_fft=False)
    X = O.nufft_forward(x.astype(np.float64), op)
    assert O.rel_l2(r["fwd"], X) < TOL
    assert abs(r["fwd"][0, 1] - x.sum()) < 1e-4 * np.abs(x).sum()


def test_mid_workload_sampled_lines(cuda_lib):
    """128^3, K = 256, 180 x 128 lines, M = 256 (5.9M points): forward on a
    sample of lines and the full adjoint on a sub-plan, against the oracle."""
    import torch

    w = I.workload("mid128")
    dirs = w.directions()
    x = w.volume(np.float32)
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp)
    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    op = _oplan(w.n, dirs, w.m, w.k, w.j, w.table_oversamp)
    lines = np.random.default_rng(0).choice(dirs.shape[0], 64, replace=False)
    ref = O.nufft_forward(x.astype(np.float64), op, lines=lines)
    assert O.rel_l2(p[lines], ref) < TOL
    # adjoint: a sub-plan of 96 lines (the oracle spreads every point)
    sub = dirs[lines[:48]]
    y = I.random_lines(sub.shape[0], w.m, 11).astype(np.complex64)
    r = _run(cuda_lib, w.n, sub, w.m, w.k, w.j, w.table_oversamp, y=y)
    ref = O.nufft_adjoint(y.astype(np.complex128), _oplan(w.n, sub, w.m, w.k, w.j, w.table_oversamp))
    assert O.rel_l2(r["adj"], ref) < TOL


@pytest.mark.parametrize("gv,sv,pps,tile", [(0, 0, 1024, 8), (0, 0, 700, 16), (1, 1, 1024, 16), (1, 1, 300, 8),
                                            (2, 2, 1024, 8), (2, 2, 64, 8), (2, 2, 5000, 8), (3, 2, 1024, 8),
                                            (3, 0, 2048, 16), (3, 2, 37, 8), (4, 2, 512, 8), (4, 2, 400, 8), (3, 3, 1024, 8), (4, 3, 512, 8), (0, 3, 77, 8), (3, 4, 512, 8), (3, 4, 33, 8), (3, 4, 560, 8), (5, 3, 512, 8), (5, 0, 300, 8), (6, 3, 512, 8), (7, 3, 256, 8), (7, 0, 37, 8), (6, 2, 2048, 8), (8, 3, 256, 8), (8, 0, 37, 8),
                                            (8, 2, 1024, 8), (3, 5, 256, 8), (4, 5, 512, 8), (0, 5, 37, 8),
                                            (5, 5, 1, 8), (3, 5, 300, 8), (3, 6, 256, 8), (5, 6, 37, 8),
                                            (0, 6, 1, 8), (4, 6, 200, 8), (8, 6, 256, 8),
                                            (4, 0, 300, 8)])
def test_kernel_variants_and_subproblem_split(cuda_lib, gv, sv, pps, tile):
    """Every gather/spread variant, tile edge and subproblem size gives the same operator."""
    import torch

    n, ndir = 32, 700
    dirs = I.umbrella_directions(35, 20)
    x = I.random_volume(n, 12).astype(np.float32)
    y = I.random_lines(ndir, 2 * n, 13).astype(np.complex64)
    plan = cuda_lib.Plan(n, dirs)
    plan.tune(gv, sv, pps, tile)
    info = plan.info()
    assert info["gather_variant"] == gv and info["spread_variant"] == sv
    assert info["points_per_subproblem"] == pps and info["tile"] == tile
    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    op = _oplan(n, dirs)
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_unsupported_tuning_is_refused(cuda_lib):
    """Variant 2 needs a warp-private tile that fits shared memory (T = 8)."""
    n = 32
    plan = cuda_lib.Plan(n, I.random_directions(10, 1))
    with pytest.raises(cuda_lib.NufftError) as ei:
        plan.tune(2, 2, 1024, 16)
    assert ei.value.status == -4
    with pytest.raises(cuda_lib.NufftError):
        plan.tune(9, 0, 0, 0)
    # the fixed-point spread bounds its cells for at most 512 points per subproblem
    with pytest.raises(cuda_lib.NufftError) as ei:
        plan.tune(-1, 5, 1024, 8)
    assert ei.value.status == -4
    with pytest.raises(cuda_lib.NufftError) as ei:
        plan.tune(-1, 6, 300, 8)
    assert ei.value.status == -4
    with pytest.raises(cuda_lib.NufftError):
        plan.tune(-1, 7, 0, 0)
    assert plan.info()["gather_variant"] == 3 and plan.info()["tile"] == 8
    plan.tune(-1, 5, 512, 8)
    with pytest.raises(cuda_lib.NufftError) as ei:
        plan.tune(-1, -1, 513, 8)
    assert ei.value.status == -4
    assert plan.info()["spread_variant"] == 5 and plan.info()["points_per_subproblem"] == 512


@pytest.mark.parametrize("sv", [3, 5, 6])
@pytest.mark.parametrize("scale", [1e-25, 1.0, 1e15])
def test_spread_dynamic_range_and_growing_batches(cuda_lib, sv, scale):
    """Line magnitudes that grow by 2^(1/16) per line, 40 binary orders over
    the 640 lines, make later batches of a subproblem larger than the first
    (the fixed-point spread rescales its tile as they arrive); three overall
    scales."""
    import torch

    n = 32
    dirs = I.umbrella_directions(40, 16)
    y = I.random_lines(dirs.shape[0], 2 * n, 17) * (2.0 ** (np.arange(dirs.shape[0]) / 16.0))[:, None] * scale
    y = y.astype(np.complex64)
    plan = cuda_lib.Plan(n, dirs)
    plan.tune(-1, sv, 256, 8)
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.nufft_adjoint(y.astype(np.complex128), _oplan(n, dirs))
    err = O.rel_l2(a, ref)
    print(f"spread {sv}, scale {scale:g}: adjoint rel-L2 {err:.2e}")
    assert err < TOL


@pytest.mark.parametrize("sv", [3, 5, 6])
def test_nan_sample_gives_nan_adjoint(cuda_lib, sv):
    """A NaN sample reaches every output of the adjoint (the line transform
    and the 3D FFT mix it into everything) in both spread arithmetics."""
    import torch

    n = 16
    dirs = I.umbrella_directions(16, 8)
    y = I.random_lines(dirs.shape[0], 2 * n, 19).astype(np.complex64)
    y[5, 3] = np.nan
    plan = cuda_lib.Plan(n, dirs)
    plan.tune(-1, sv, 256, 8)
    a = plan.adjoint(torch.from_numpy(y).cuda())
    assert plan.sync_status() == 0
    assert bool(torch.isnan(a).all())
    # the plan stays usable: a finite input afterwards gives the oracle's result
    y[5, 3] = 0
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), _oplan(n, dirs))) < TOL


def test_variant1_dense_center_and_repeat_calls(cuda_lib):
    """Many lines through the centre (dense tiles, split subproblems), repeated
    calls on one plan give identical forward results."""
    import torch

    n = 32
    dirs = I.umbrella_directions(90, 64)
    x = torch.from_numpy(I.random_volume(n, 14).astype(np.float32)).cuda()
    plan = cuda_lib.Plan(n, dirs)
    assert plan.info()["spread_variant"] == 3  # the default for J = 6
    plan.tune(-1, -1, 2048)
    p1 = plan.forward(x).clone()
    p2 = plan.forward(x)
    assert torch.equal(p1, p2)
    op = _oplan(n, dirs)
    lines = np.arange(0, dirs.shape[0], 41)
    ref = O.nufft_forward(x.cpu().numpy().astype(np.float64), op, lines=lines)
    assert O.rel_l2(p1.cpu().numpy()[lines], ref) < TOL
    y = torch.from_numpy(I.random_lines(dirs.shape[0], 2 * n, 15).astype(np.complex64)).cuda()
    a1 = plan.adjoint(y).cpu().numpy()
    sub = np.arange(0, dirs.shape[0], 7)
    ysub = y.cpu().numpy()[sub]
    r = _run(cuda_lib, n, dirs[sub], y=ysub)
    ref = O.nufft_adjoint(ysub.astype(np.complex128), _oplan(n, dirs[sub]))
    assert O.rel_l2(r["adj"], ref) < TOL
    assert np.isfinite(a1).all()


def test_coincident_samples_merged_and_equal(cuda_lib):
    """Antipodal umbrella lines share their samples: (l', -q) is (l, q).  The
    merged plan evaluates each such point once and must equal the plan that
    evaluates every sample separately, and the oracle."""
    import torch

    n = 32
    dirs = I.umbrella_directions(40, 16)   # azimuth count even: every line has its antipode
    D, M = dirs.shape[0], 2 * n
    x = torch.from_numpy(I.random_volume(n, 41).astype(np.float32)).cuda()
    y = torch.from_numpy(I.random_lines(D, M, 42).astype(np.complex64)).cuda()
    merged = cuda_lib.Plan(n, dirs)
    full = cuda_lib.Plan(n, dirs, keep_duplicates=True)
    im, iff = merged.info(), full.info()
    assert im["merged_line_pairs"] == D // 2 and iff["merged_line_pairs"] == 0
    assert im["evaluated_points"] == (D // 2) * M + D // 2 and iff["evaluated_points"] == D * M
    pm, pf = merged.forward(x), full.forward(x)
    am, af = merged.adjoint(y), full.adjoint(y)
    assert float(torch.linalg.norm(pm - pf) / torch.linalg.norm(pf)) < 1e-6
    assert float(torch.linalg.norm(am - af) / torch.linalg.norm(af)) < 1e-6
    op = _oplan(n, dirs)
    assert O.rel_l2(am.cpu().numpy(), O.nufft_adjoint(y.cpu().numpy().astype(np.complex128), op)) < TOL
    rnd = cuda_lib.Plan(n, I.random_directions(50, 3))
    assert rnd.info()["merged_line_pairs"] == 0
    # custom radii without symmetry: nothing merged
    om = np.linspace(-3.0, 3.1, M)
    asym = cuda_lib.Plan(n, dirs, m=M, omega=om, do_line_fft=False)
    assert asym.info()["merged_line_pairs"] == 0


def test_host_pipeline_matches_device_path(cuda_lib):
    """Overlapped host<->device pipeline gives the device path's results."""
    import torch

    n = 32
    dirs = I.umbrella_directions(20, 10)
    plan = cuda_lib.Plan(n, dirs)
    pipe = cuda_lib.HostPipeline(plan)
    vols = [torch.from_numpy(I.random_volume(n, 60 + i).astype(np.float32)).pin_memory() for i in range(3)]
    lines = [torch.empty((plan.n_dirs, plan.m), dtype=torch.complex64).pin_memory() for _ in range(3)]
    outs = [torch.empty_like(v).pin_memory() for v in vols]
    for v, l, o in zip(vols, lines, outs):
        pipe.run(v, l, o)
    pipe.synchronize()
    for v, l, o in zip(vols, lines, outs):
        ref_l = plan.forward(v.cuda())
        ref_o = plan.adjoint(ref_l)
        assert torch.allclose(l, ref_l.cpu(), rtol=0, atol=1e-5 * float(ref_l.abs().max()))
        assert torch.allclose(o, ref_o.cpu(), rtol=0, atol=1e-5 * float(ref_o.abs().max()))
    pipe2 = cuda_lib.HostPipeline(plan)
    pipe2.run(vols[0], lines[0], outs[0])
    pipe2.synchronize()
    pipe2.close()
    pipe.close()
    # the plan no longer refers to the pipelines' streams
    assert plan.sync_status() == 0
    plan.close()


def test_fp32_fma_peak_is_plausible(cuda_lib):
    """The measured FP32 FMA throughput lies between half and 1.05x of the
    nominal SMs x 128 lanes x 2 flops x the device's maximum clock."""
    import torch

    tflops, sms = cuda_lib.fp32_fma_peak()
    props = torch.cuda.get_device_properties(0)
    assert sms == props.multi_processor_count
    lib = cuda_lib.load_library()
    assert lib.nufft3d_fp32_fma_peak(None, None, None) == -1
    nominal_at_2_1ghz = sms * 128 * 2 * 2.1e9 / 1e12
    print(f"FP32 FMA peak {tflops:.1f} TFLOP/s on {sms} SMs")
    assert 0.5 * nominal_at_2_1ghz < tflops < 1.05 * nominal_at_2_1ghz


@pytest.mark.parametrize("grid_dtype", ["c64", "bf16"])
def test_adjoint_grid_left_clear_between_calls(cuda_lib, grid_dtype):
    """The inverse z pass clears the adjoint grid as it reads it, so repeated
    adjoints, with forward calls in between, must keep agreeing with the
    oracle (a leftover value would add to the next call)."""
    import torch

    n, ndir = 32, 300
    dirs = I.random_directions(ndir, 91)
    x = torch.from_numpy(I.random_volume(n, 92).astype(np.float32)).cuda()
    ys = [I.random_lines(ndir, 2 * n, 93 + i).astype(np.complex64) for i in range(3)]
    plan = cuda_lib.Plan(n, dirs, grid_dtype=grid_dtype)
    op = _oplan(n, dirs)
    for rep in range(2):
        for y in ys:
            a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
            plan.forward(x)
            assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL, rep
    assert plan.sync_status() == 0
