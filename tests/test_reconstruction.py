"""Direct (Fourier-slice) reconstruction: the adjoint with ramp and
solid-angle weights inverts the image-to-Radon step (Sec. 2.3: Fourier-domain
ramp filtering, R^2 in 3D per Sec. 1, then the NUFFT transpose).

CPU pins, on the oracle:
- a Gaussian blob, whose spectrum is negligible beyond |w| = pi, is
  reconstructed from its own plane integrals over a full umbrella sphere to
  within the quadrature error, and that error falls with N;
- the 15-degree missing cone of a circular trajectory raises the error;
- planted mistakes in the weights (a factor 2, a |q| instead of q^2 ramp) fail;
- the library's closed-form weights match the oracle's independently derived
  quadrature (exact solid-angle cells, rho^2 d rho).

GPU: the weighted forward and adjoint, and the whole reconstruction, match
the oracle with the same weights at rel-L2 <= 1e-5.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

TOL = 1e-5


def _oracle_weights(n_az, n_pol, cone, M):
    """Quadrature of x[n] = (2 pi)^-3 int X(w) e^{i w.n} d^3w over the umbrella
    directions, d^3w = rho^2 d rho d Omega: exact solid angle of each
    (phi, theta) cell, halved (each Fourier point lies on two antipodal lines);
    rho = 2 pi q / M with d rho = 2 pi / M, the q = 0 sample standing for the
    ball rho < pi / M; times M to undo the 1/M of the adjoint's line DFT."""
    edges = cone + (np.pi - 2 * cone) * np.arange(n_pol + 1) / n_pol
    cell = (2 * np.pi / n_az) * (np.cos(edges[:-1]) - np.cos(edges[1:]))
    lw = np.tile(cell / 2, n_az)
    q = np.arange(M) - M // 2
    rho, drho = 2 * np.pi * q / M, 2 * np.pi / M
    rad = rho ** 2 * drho
    rad = np.where(q == 0, (4 * np.pi / 3) * (drho / 2) ** 3 / lw.sum(), rad)
    return rad * M / (2 * np.pi) ** 3, lw


def _blob(N, sigma=2.5, c=(1.3, -0.7, 2.1)):
    n = np.arange(N) - N // 2
    z, y, x = np.meshgrid(n, n, n, indexing="ij")
    return np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * sigma ** 2))


def _oracle_recon(N, n_az, n_pol, cone_deg, vol, rad=None, lw=None):
    M = K = 2 * N
    dirs = I.umbrella_directions(n_az, n_pol, cone_deg)
    if rad is None:
        rad, lw = _oracle_weights(n_az, n_pol, np.deg2rad(cone_deg), M)
    p = O.nufft_forward(vol, O.OraclePlan(N, K, 6, 1024, dirs, M))
    return O.nufft_adjoint(p, O.OraclePlan(N, K, 6, 1024, dirs, M, weight=rad, line_weight=lw))


def test_oracle_reconstructs_blob_and_converges():
    e16 = O.rel_l2(_oracle_recon(16, 64, 32, 0.0, _blob(16)), _blob(16))
    e32 = O.rel_l2(_oracle_recon(32, 64, 32, 0.0, _blob(32)), _blob(32))
    print(f"blob reconstruction error: N=16 {e16:.2e}, N=32 {e32:.2e}")
    assert e16 < 0.04 and e32 < 0.015 and e32 < e16


def test_missing_cone_raises_error():
    full = O.rel_l2(_oracle_recon(32, 64, 32, 0.0, _blob(32)), _blob(32))
    cone = O.rel_l2(_oracle_recon(32, 64, 32, 15.0, _blob(32)), _blob(32))
    assert cone > 3 * full and cone < 0.3


@pytest.mark.parametrize("mistake", ["factor2", "ramp_q"])
def test_planted_weight_mistakes_fail(mistake):
    N, M = 32, 64
    rad, lw = _oracle_weights(64, 32, 0.0, M)
    if mistake == "factor2":
        rad = 2 * rad
    else:
        q = np.arange(M) - M // 2
        rad = np.where(q != 0, np.abs(q) / M, rad)
    err = O.rel_l2(_oracle_recon(N, 64, 32, 0.0, _blob(N), rad, lw), _blob(N))
    assert err > 0.5


@pytest.mark.parametrize("n_az,n_pol,cone_deg,M", [(64, 32, 15.0, 64), (360, 256, 15.0, 512), (8, 4, 0.0, 16)])
def test_library_weights_match_oracle_quadrature(n_az, n_pol, cone_deg, M):
    from paper_1605_05231_gb300 import binding

    rad, lw = binding.fourier_slice_weights(n_az, n_pol, np.deg2rad(cone_deg), M)
    orad, olw = _oracle_weights(n_az, n_pol, np.deg2rad(cone_deg), M)
    q = np.arange(M) - M // 2
    assert np.all(rad.imag == 0)
    assert np.array_equal(rad.real[q != 0], (q[q != 0] ** 2 / M ** 2).astype(np.float32))
    # midpoint sin(theta) d theta against the exact cell areas: relative error
    # below d theta^2 / 12 (the sphere's area between the cones is 4 pi cos c,
    # halved for the antipodal pairs)
    dth = (np.pi - 2 * np.deg2rad(cone_deg)) / n_pol
    assert np.max(np.abs(lw - olw) / olw) < dth ** 2 / 12 + 1e-6
    assert abs(lw.sum() / (2 * np.pi * np.cos(np.deg2rad(cone_deg))) - 1) < dth ** 2 / 12 + 1e-6
    assert np.allclose(rad.real[q != 0], orad[q != 0], rtol=1e-6, atol=0)
    # the q = 0 weight divides by the sum of the line weights: same bound
    assert abs(rad.real[q == 0][0] / orad[q == 0][0] - 1) < dth ** 2 / 12 + 1e-6


def test_library_weights_reject_bad_arguments():
    from paper_1605_05231_gb300 import binding

    for args in [(0, 4, 0.0, 16), (4, 4, 0.0, 15), (4, 4, 2.0, 16), (4, 4, -0.1, 16)]:
        with pytest.raises(binding.NufftError):
            binding.fourier_slice_weights(*args)


# ---------------------------------------------------------------------------
# GPU parity
# ---------------------------------------------------------------------------
@pytest.mark.gpu
@pytest.mark.parametrize("exact", [False, True])
def test_weighted_forward_adjoint_match_oracle(cuda_lib, exact):
    import torch

    w = I.workload("tiny32")
    dirs = w.directions()
    rad, lw = cuda_lib.fourier_slice_weights(w.n_az, w.n_pol, np.deg2rad(15.0), w.m)
    plan = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, weight=rad, line_weight=lw, exact_coeffs=exact)
    x = w.volume(np.float32)
    y = I.random_lines(dirs.shape[0], w.m, 41).astype(np.complex64)
    p = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    a = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    op = O.OraclePlan(w.n, w.k, w.j, 0 if exact else 1024, dirs, w.m, weight=rad.astype(np.complex128),
                      line_weight=lw.astype(np.float64))
    assert O.rel_l2(p, O.nufft_forward(x.astype(np.float64), op)) < TOL
    assert O.rel_l2(a, O.nufft_adjoint(y.astype(np.complex128), op)) < TOL


@pytest.mark.gpu
def test_direct_reconstruction_matches_oracle(cuda_lib):
    """Plane integrals of the 32^3 ellipsoid phantom over the 64 x 32
    umbrella lines, then the weighted adjoint: the GPU reconstruction equals
    the oracle's, and both are the phantom up to the missing cone."""
    import torch

    w = I.workload("tiny32")
    dirs = w.directions()
    rad, lw = cuda_lib.fourier_slice_weights(w.n_az, w.n_pol, np.deg2rad(15.0), w.m)
    proj = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, exact_coeffs=True)
    back = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, weight=rad, line_weight=lw, exact_coeffs=True)
    x = w.volume(np.float32)
    xr = back.adjoint(proj.forward(torch.from_numpy(x).cuda())).cpu().numpy()
    assert back.sync_status() == 0 and proj.sync_status() == 0
    op = O.OraclePlan(w.n, w.k, w.j, 0, dirs, w.m)
    opw = O.OraclePlan(w.n, w.k, w.j, 0, dirs, w.m, weight=rad.astype(np.complex128),
                       line_weight=lw.astype(np.float64))
    xo = O.nufft_adjoint(O.nufft_forward(x.astype(np.float64), op), opw)
    err = O.rel_l2(xr, xo)
    print(f"direct reconstruction: GPU vs oracle {err:.2e}; vs phantom {O.rel_l2(xr, x):.3f}")
    assert err < TOL
    assert O.rel_l2(xr, x) < 0.3


@pytest.mark.gpu
def test_direct_reconstruction_128(cuda_lib):
    """The 128^3 workload (180 x 128 lines, M = 256): reconstruction error
    against the phantom, reported beside the oracle's at the smaller size."""
    import torch

    w = I.workload("mid128")
    dirs = w.directions()
    rad, lw = cuda_lib.fourier_slice_weights(w.n_az, w.n_pol, np.deg2rad(15.0), w.m)
    proj = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, exact_coeffs=True)
    back = cuda_lib.Plan(w.n, dirs, m=w.m, k=w.k, weight=rad, line_weight=lw, exact_coeffs=True)
    x = torch.from_numpy(w.volume(np.float32)).cuda()
    xr = back.adjoint(proj.forward(x))
    assert back.sync_status() == 0
    err = float(torch.linalg.norm(xr - x) / torch.linalg.norm(x))
    print(f"128^3 direct reconstruction error vs phantom: {err:.3f}")
    assert err < 0.3
