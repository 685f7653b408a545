"""The allocation-free adjoint entry point (nufft3d_adjoint_noalloc).

It serves callers that cannot allocate device memory when they run the
adjoint (for example while a stream is captured into a CUDA graph in global
mode, or inside a host framework that owns all device memory through its own
pool): its scratch lives in a static device array of the library.  Checked
through the C ABI against nufft3d_adjoint on the same plan, on two calls in a
row (the static array keeps the previous call's contents, so the second call
shows that everything that must start at zero is cleared).  This file is
collected last so a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _noalloc(lib, plan, lines, out):
    import torch

    return lib.nufft3d_adjoint_noalloc(plan._handle, ctypes.c_void_p(lines.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("exact", [False, True], ids=["table", "exact"])
def test_noalloc_adjoint_matches_adjoint_twice(cuda_lib, exact):
    """Both coefficient modes: the table with its default spread (FP32 tiles)
    and the exact coefficients with theirs (real weights, fixed-point tiles
    shared by a CTA, the grid phase applied as the tile is added to the grid)."""
    import torch

    lib = cuda_lib.load_library()
    w = I.workload("tiny32")
    dirs = w.directions()
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp, exact_coeffs=exact)
    assert plan.info()["spread_variant"] == (7 if exact else 3)
    for seed in (21, 22):
        y = torch.from_numpy(I.random_lines(dirs.shape[0], w.m, seed).astype(np.complex64)).cuda()
        ref = plan.adjoint(y).clone()
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(lib, plan, y, out) == 0
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err < TOL, err
    # and against the FP64 oracle for the last call
    op = O.OraclePlan(w.n, w.k, w.j, 0 if exact else w.table_oversamp, dirs, w.m)
    assert O.rel_l2(out.cpu().numpy(), O.nufft_adjoint(y.cpu().numpy().astype(np.complex128), op)) < TOL
    plan.close()


def test_noalloc_adjoint_rejects_plans_beyond_its_scratch(cuda_lib):
    import torch

    lib = cuda_lib.load_library()
    plan = cuda_lib.Plan(64, I.random_directions(8, 3))  # K^3 alone is 16 MiB > 8 MiB
    y = torch.zeros((8, 128), dtype=torch.complex64, device="cuda")
    out = torch.zeros((64, 64, 64), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, plan, y, out) == -4
    plan.close()
