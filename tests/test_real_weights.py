"""The real-weight interpolation kernels (gather 9, spread 7) against the FP64 oracle.

They use the factoring c_j(f) = e^{i gamma (f + J/2 - j)/2} rho_j(f), rho_j real,
of the min-max coefficients (exact for a pre-window symmetric about the middle
of the index range): the grid carries the phase e^{-i gamma (kx + ky + kz)/2}
(applied by the z passes), every point its own phase, and taps whose unwrapped
index leaves [-K/2, K/2) a sign.  The oracle knows none of this: it applies the
complex coefficients c = T^-1 r to the plain grid.  Points with taps across the
+-K/2 faces come from the q = -M/2 samples of lines near the axes.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _plan(binding, n, dirs, m=0, k=0, j=6, **kw):
    return binding.Plan(n, dirs, m=m, k=k, j=j, exact_coeffs=True, **kw)


def _oplan(n, dirs, m=0, k=0, j=6, **kw):
    return O.OraclePlan(n, k or 2 * n, j, 0, dirs, m or 2 * n, **kw)


def _run(plan, x, y):
    import torch

    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return p, a


def _face_dirs(n_rand, seed):
    """Axis directions, directions a little off the axes, and random ones: the
    q = -M/2 samples of the first put taps on both sides of the -K/2 face."""
    rng = np.random.default_rng(seed)
    near = np.eye(3)[rng.integers(0, 3, 12)] + rng.normal(scale=0.02, size=(12, 3))
    near /= np.linalg.norm(near, axis=1, keepdims=True)
    return np.concatenate([I.axis_directions(), -I.axis_directions(), near, I.random_directions(n_rand, seed)])


@pytest.mark.parametrize("gv,sv", [(9, 7), (9, 6), (5, 7), (9, 3), (8, 7), (9, 0), (10, 8), (10, 7), (9, 8), (5, 8),
                                   (10, 3), (11, 7), (11, 8)])
def test_real_variants_umbrella(cuda_lib, gv, sv):
    n = 32
    dirs = I.umbrella_directions(35, 20)
    x = I.random_volume(n, 12).astype(np.float32)
    y = I.random_lines(dirs.shape[0], 2 * n, 13).astype(np.complex64)
    plan = _plan(cuda_lib, n, dirs)
    plan.tune(gv, sv, 256, 8)
    info = plan.info()
    assert (info["gather_variant"], info["spread_variant"]) == (gv, sv)
    p, a = _run(plan, x, y)
    op = _oplan(n, dirs)
    ef = O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op))
    ea = O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op))
    print(f"gather {gv} spread {sv}: forward {ef:.2e}, adjoint {ea:.2e}")
    assert ef < TOL and ea < TOL


@pytest.mark.parametrize("n,k,m,j,pps", [
    (16, 32, 32, 6, 256),     # K = 2N
    (24, 48, 48, 6, 100),     # radix 3
    (32, 48, 64, 6, 256),     # K = 1.5 N: faces closer to the ball
    (32, 96, 64, 6, 37 + 1),  # K = 3 N, small subproblems
    (16, 32, 32, 4, 256),     # J = 4 (gather 9, spread 0)
    (16, 32, 32, 8, 128),     # J = 8
    (20, 64, 48, 2, 256),     # J = 2, M != K
])
@pytest.mark.parametrize("sched", [0, 1, 2], ids=["rank", "sched", "pipelined"])
def test_real_variants_faces_shapes_and_taps(cuda_lib, n, k, m, j, pps, sched):
    """gather 9 / spread 7 (or 0), the scheduled gather 10 / spread 8 and the
    pipelined scheduled gather 11 (any J)."""
    dirs = _face_dirs(40, n + k)
    x = I.random_volume(n, 1).astype(np.float32)
    y = I.random_lines(dirs.shape[0], m, 2).astype(np.complex64)
    plan = _plan(cuda_lib, n, dirs, m, k, j)
    gv, sv = ((9, 7 if j == 6 else 0), (10, 8), (11, 8))[sched]
    plan.tune(gv, sv, pps, 8)
    p, a = _run(plan, x, y)
    op = _oplan(n, dirs, m, k, j)
    ef = O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op))
    ea = O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op))
    assert ef < TOL and ea < TOL, (ef, ea)
    # the face samples themselves (q = -M/2 of the first 18 lines), element by element
    import torch

    pr = O.nufft_forward(x.astype(np.float64), op, return_samples=True)
    plan_raw = _plan(cuda_lib, n, dirs, m, k, j, do_line_fft=False)
    plan_raw.tune(gv, sv, pps, 8)
    raw = plan_raw.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.max(np.abs(raw[:18, 0] - pr[:18, 0])) < TOL * np.max(np.abs(pr)), "face samples"


def test_real_variants_complex_volume_weights_raw_samples(cuda_lib):
    n, ndir = 16, 45
    dirs = _face_dirs(ndir, 5)
    rng = np.random.default_rng(9)
    w = (rng.normal(size=2 * n) + 1j * rng.normal(size=2 * n)).astype(np.complex64)
    x = I.random_volume(n, 3, complex_values=True).astype(np.complex64)
    y = I.random_lines(dirs.shape[0], 2 * n, 4).astype(np.complex64)
    for kw, (gv, sv) in ((dict(weight=w), (9, 7)), (dict(do_line_fft=False), (9, 7)), (dict(weight=w), (10, 8)),
                         (dict(do_line_fft=False), (10, 8))):
        plan = _plan(cuda_lib, n, dirs, complex_volume=True, **kw)
        plan.tune(gv, sv, 256, 8)
        p, a = _run(plan, x, y)
        okw = dict(kw)
        if "weight" in okw:
            okw["weight"] = w.astype(np.complex128)
        op = _oplan(n, dirs, complex_volume=True, **okw)
        assert O.rel_l2(p, O.nufft_forward(x.astype(np.complex128), op)) < TOL
        assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


@pytest.mark.parametrize("dtype,bound", [("bf16", 1e-3), ("fp16", 1e-4)])
@pytest.mark.parametrize("gv,sv", [(9, 7), (10, 8), (11, 7)])
def test_real_gather_reduced_precision_grid(cuda_lib, dtype, bound, gv, sv):
    """The phase is applied before the grid is rounded to bf16 / fp16."""
    w = I.workload("tiny32")
    dirs = w.directions()
    x = w.volume(np.float32)
    y = I.random_lines(dirs.shape[0], w.m, 3).astype(np.complex64)
    plan = _plan(cuda_lib, w.n, dirs, w.m, w.k, grid_dtype=dtype)
    plan.tune(gv, sv, 256, 8)
    p, a = _run(plan, x, y)
    op = _oplan(w.n, dirs, w.m, w.k)
    ef = O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op))
    print(f"gather 9 with a {dtype} grid: forward rel-L2 {ef:.2e}")
    assert ef < bound
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


def test_real_variants_refused_with_a_table(cuda_lib):
    plan = cuda_lib.Plan(32, I.random_directions(10, 1))
    for gv, sv in ((9, -1), (-1, 7), (10, -1), (-1, 8), (11, -1)):
        with pytest.raises(cuda_lib.NufftError) as ei:
            plan.tune(gv, sv, 256, 8)
        assert ei.value.status == -4


def test_switching_between_real_and_complex_variants(cuda_lib):
    """The grid phase follows the variant of every call."""
    import torch

    n = 32
    dirs = I.umbrella_directions(30, 16)
    x = torch.from_numpy(I.random_volume(n, 5).astype(np.float32)).cuda()
    y = torch.from_numpy(I.random_lines(dirs.shape[0], 2 * n, 6).astype(np.complex64)).cuda()
    plan = _plan(cuda_lib, n, dirs)
    res = []
    for gv, sv in ((5, 6), (9, 7), (5, 6), (10, 8), (9, 7), (10, 8)):
        plan.tune(gv, sv, 256, 8)
        res.append((plan.forward(x).clone(), plan.adjoint(y).clone()))
    assert plan.sync_status() == 0
    for p, a in res[1:]:
        assert float(torch.linalg.norm(p - res[0][0]) / torch.linalg.norm(res[0][0])) < 1e-5
        assert float(torch.linalg.norm(a - res[0][1]) / torch.linalg.norm(res[0][1])) < 1e-5


def test_scheduled_variants_refuse_large_subproblems(cuda_lib):
    """The schedules exist for subproblems of at most 256 points."""
    plan = _plan(cuda_lib, 32, I.umbrella_directions(20, 10))
    for gv, sv in ((10, -1), (-1, 8), (11, -1)):
        with pytest.raises(cuda_lib.NufftError) as ei:
            plan.tune(gv, sv, 512, 8)
        assert ei.value.status == -4


def test_scheduled_variants_mid_workload_sampled(cuda_lib):
    """128^3 (K = 256, 180 x 128 lines of 256 samples): the scheduled pair on a
    sample of lines forward, and the adjoint of a 48-line support element by
    element, against the oracle; the dense centre (many subproblems per tile,
    the 23,040 points at the origin) is exercised."""
    import torch

    w = I.workload("mid128")
    dirs = w.directions()
    x = w.volume(np.float32)
    plan = _plan(cuda_lib, w.n, dirs, w.m, w.k)
    plan.tune(10, 8, 256, 8)
    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    sel = np.sort(np.random.default_rng(5).choice(dirs.shape[0], 48, replace=False))
    op = _oplan(w.n, dirs, w.m, w.k)
    assert O.rel_l2(p[sel], O.nufft_forward(x.astype(np.float64), op, lines=sel)) < TOL
    ys = I.random_lines(sel.size, w.m, 6).astype(np.complex64)
    y = np.zeros((dirs.shape[0], w.m), dtype=np.complex64)
    y[sel] = ys
    # the lines through the origin carry their q = 0 samples into the subproblems of points at the origin
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.nufft_adjoint(ys.astype(np.complex128), _oplan(w.n, dirs[sel], w.m, w.k))
    err = O.rel_l2(a, ref)
    print(f"128^3 scheduled spread, 48-line support: adjoint rel-L2 {err:.2e}")
    assert err < TOL
