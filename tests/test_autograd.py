"""Differentiation through the projector: torch.autograd with the hand-written
adjoint kernel as backward.

For L(x) = 1/2 ||A x - b||^2 with real x the gradient is Re(A^H (A x - b)).
L is quadratic, so a central difference (L(x + e v) - L(x - e v)) / (2 e)
equals <grad L, v> up to rounding for any step e: the 64 random probes are
checked to 1e-3 relative (FP32 projector, loss accumulated in FP64).  The
probes are seeded random smooth fields (white noise low-passed by a Gaussian
of 4 voxels): a white-noise direction in 256^3 dimensions has a directional
derivative near ||grad|| / 4096, below the FP32 rounding of L itself.
Gradient descent with step 1 / ||A||^2 (power iteration) must decrease the
loss monotonically, and its first iterate must match the FP64 oracle's.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _loss(y, b):
    import torch

    d = (y - b).to(torch.complex128)
    return 0.5 * float(torch.sum(d.real ** 2 + d.imag ** 2))


def test_backward_is_adjoint_kernel_and_matches_oracle(cuda_lib):
    import torch

    w = I.workload("tiny32")
    dirs = w.directions()
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k)
    x0 = w.volume(np.float32)
    b = torch.from_numpy(I.random_lines(dirs.shape[0], w.m, 5).astype(np.complex64)).cuda()
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    y = cuda_lib.project(x, plan)
    loss = 0.5 * (y - b).abs().pow(2).sum()
    loss.backward()
    r = (y.detach() - b).contiguous()
    ref = plan.adjoint(r)
    assert torch.allclose(x.grad, ref, rtol=0, atol=1e-6 * float(ref.abs().max()))
    op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
    ro = O.nufft_forward(x0.astype(np.float64), op) - b.cpu().numpy().astype(np.complex128)
    g_oracle = O.nufft_adjoint(ro, op)
    assert O.rel_l2(x.grad.cpu().numpy(), g_oracle) < TOL


def test_complex_volume_backward(cuda_lib):
    import torch

    n = 16
    dirs = I.random_directions(40, 3)
    plan = cuda_lib.Plan(n, dirs, complex_volume=True)
    x = torch.from_numpy(I.random_volume(n, 4, complex_values=True).astype(np.complex64)).cuda()
    x.requires_grad_(True)
    b = torch.from_numpy(I.random_lines(40, 2 * n, 6).astype(np.complex64)).cuda()
    y = cuda_lib.project(x, plan)
    (0.5 * (y - b).abs().pow(2).sum()).backward()
    ref = plan.adjoint((y.detach() - b).contiguous())
    assert torch.allclose(x.grad, ref, rtol=0, atol=1e-6 * float(ref.abs().max()))


@pytest.fixture(scope="module")
def full_problem(cuda_lib):
    """256^3 ellipsoid phantom + N(0, 0.01^2) noise, K = 512, 360 x 256 lines, M = 512."""
    import torch

    w = I.workload("full256")
    plan = cuda_lib.Plan(w.n, w.directions(), m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp)
    x_true = torch.from_numpy(w.volume(np.float32)).cuda()
    b = plan.forward(x_true).clone()
    yield plan, x_true, b
    plan.close()


def test_finite_differences_64_probes_full_size(cuda_lib, full_problem):
    import torch

    plan, x_true, b = full_problem
    g = torch.Generator(device="cuda").manual_seed(0)
    x = (0.5 * x_true + 0.05 * torch.randn(x_true.shape, generator=g, device="cuda")).contiguous()
    xg = x.clone().requires_grad_(True)
    y = cuda_lib.project(xg, plan)
    (0.5 * (y - b).abs().pow(2).sum()).backward()
    grad = xg.grad.to(torch.float64)
    r_norm = float(torch.linalg.norm((y.detach() - b).to(torch.complex128)))
    n = x.shape[0]
    k = torch.fft.fftfreq(n, device="cuda")
    kk = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    lowpass = torch.exp(-0.5 * (2 * np.pi * 4.0) ** 2 * kk)
    worst = 0.0
    for _ in range(64):
        v = torch.randn(x.shape, generator=g, device="cuda")
        v = torch.fft.ifftn(torch.fft.fftn(v) * lowpass).real.float()
        v /= torch.linalg.norm(v)
        av = float(torch.linalg.norm(plan.forward(v.contiguous()).to(torch.complex128)))
        eps = r_norm / av
        lp = _loss(plan.forward((x + eps * v).contiguous()), b)
        lm = _loss(plan.forward((x - eps * v).contiguous()), b)
        fd = (lp - lm) / (2 * eps)
        an = float(torch.sum(grad * v.to(torch.float64)))
        rel = abs(fd - an) / max(abs(an), 1e-12 * float(torch.linalg.norm(grad)))
        worst = max(worst, rel)
    print(f"finite differences, 64 smooth random probes: worst relative mismatch {worst:.2e}")
    assert worst < 1e-3, worst


def test_gradient_descent_10_steps_full_size(cuda_lib, full_problem):
    import torch

    plan, x_true, b = full_problem
    # ||A||^2 by 10 power iterations on A^H A
    g = torch.Generator(device="cuda").manual_seed(1)
    v = torch.randn(x_true.shape, generator=g, device="cuda")
    v /= torch.linalg.norm(v)
    lam = 0.0
    for _ in range(10):
        w = plan.adjoint(plan.forward(v))
        lam = float(torch.linalg.norm(w))
        v = (w / lam).contiguous()
    tau = 1.0 / lam
    x = torch.zeros_like(x_true)
    losses = [_loss(plan.forward(x), b)]
    for _ in range(10):
        x.requires_grad_(True)
        y = cuda_lib.project(x, plan)
        (0.5 * (y - b).abs().pow(2).sum()).backward()
        with torch.no_grad():
            x = (x - tau * x.grad).contiguous()
        losses.append(_loss(plan.forward(x), b))
    assert all(l1 < l0 for l0, l1 in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0]


def test_gradient_descent_first_iterate_matches_oracle(cuda_lib):
    import torch

    w = I.workload("tiny32")
    dirs = w.directions()
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k)
    b = torch.from_numpy(I.random_lines(dirs.shape[0], w.m, 8).astype(np.complex64)).cuda()
    tau = 1e-3
    x = torch.zeros((w.n,) * 3, device="cuda", requires_grad=True)
    y = cuda_lib.project(x, plan)
    (0.5 * (y - b).abs().pow(2).sum()).backward()
    x1 = (x.detach() - tau * x.grad).cpu().numpy()
    op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
    bo = b.cpu().numpy().astype(np.complex128)
    x1_oracle = -tau * O.nufft_adjoint(-bo, op)
    assert O.rel_l2(x1, x1_oracle) < TOL
