"""The bounded device waits report a timeout instead of hanging.

The TMA gather (variant 8) waits on an mbarrier for every tile copy.  A wait
that runs out of polls sets NUFFT3D_ERR_TIMEOUT (-5) in the plan's device check
word; the CTA then waits, with the full limit, for its copies still in flight
and returns, so the context stays usable.  The testing hook
nufft3d_plan_set_wait_limit caps the first wait on every copy; with a cap of 0
polls every such wait gives up at once, which makes the timeout path run
without any fault or hang: the copies themselves complete normally.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TIMEOUT = -5


def test_tma_gather_wait_timeout_is_reported_and_recoverable(cuda_lib):
    import torch

    w = I.workload("tiny32")
    dirs = w.directions()
    x = torch.from_numpy(w.volume(np.float32)).cuda()
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, exact_coeffs=True)
    plan.tune(8, -1, 256, 8)
    assert plan.info()["gather_variant"] == 8
    ref = plan.forward(x).clone()
    assert plan.sync_status() == 0
    plan.set_wait_limit(0)
    plan.forward(x)
    assert plan.sync_status() == TIMEOUT
    # the word was cleared by the read; the default limit gives the full result again
    plan.set_wait_limit(-1)
    p = plan.forward(x)
    assert plan.sync_status() == 0
    assert float(torch.linalg.norm(p - ref) / torch.linalg.norm(ref)) == 0.0
    op = O.OraclePlan(w.n, w.k, w.j, 0, dirs, w.m)
    assert O.rel_l2(p.cpu().numpy(), O.nufft_forward(x.cpu().numpy().astype(np.float64), op)) < 1e-5
    plan.close()


def test_wait_limit_hook_rejects_null_plan(cuda_lib):
    lib = cuda_lib.load_library()
    assert lib.nufft3d_plan_set_wait_limit(None, 0) == -1
