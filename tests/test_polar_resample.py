"""Direct resampling of the polar Radon grid with truncated sincs (Sec. 2.1,
Eq. 2.15 with T2 = I; the paper's runs use [3 3 3] taps, Sec. 3.2).

CPU pins of the oracle (oracle/polar_resample.py):
- at integer targets the operator reproduces the grid samples exactly
  (sinc(0) = 1, sinc(k) = 0), also at the phi wrap and next to the theta / s
  ends;
- it equals an explicit dense matrix T1 built cell by cell, for in-range and
  out-of-range targets;
- it is shift invariant and periodic in phi (checked against np.roll);
- 1D interpolation of a sampled Gaussian converges to the Gaussian as J grows;
- a planted off-by-one tap start fails the integer-target pin.

GPU: the CUDA resampler against the oracle at rel-L2 <= 1e-5, including
ragged target counts, wrap and edge targets, J = 2..8, and a sampled check on
the 360 x 256 x 512 grid of the 256^3 workload.
"""
import numpy as np
import pytest

from oracle import polar_resample as R
from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

TOL = 1e-5


def _grid(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _targets(n, shape, seed, margin=1.5):
    rng = np.random.default_rng(seed)
    n_phi, n_theta, n_s = shape
    return np.stack([rng.uniform(-margin, n_s - 1 + margin, n), rng.uniform(-margin, n_theta - 1 + margin, n),
                     rng.uniform(-2 * n_phi, 3 * n_phi, n)], axis=1)


@pytest.mark.parametrize("J", [2, 3, 4, 6])
def test_integer_targets_reproduce_samples(J):
    shape = (11, 7, 13)
    x = _grid(shape, 1)
    rng = np.random.default_rng(2)
    k = np.stack([rng.integers(0, shape[2], 200), rng.integers(0, shape[1], 200), rng.integers(-30, 30, 200)], axis=1)
    got = R.polar_sinc_resample(x, k.astype(np.float64), J)
    want = x[np.mod(k[:, 2], shape[0]), k[:, 1], k[:, 0]]
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("J", [2, 3, 5, 6])
def test_matches_explicit_sparse_matrix(J):
    shape = (7, 5, 9)
    x = _grid(shape, 3)
    t = _targets(300, shape, 4)
    assert np.max(np.abs(R.polar_sinc_resample(x, t, J) - R.sparse_matrix_resample(x, t, J))) < 1e-12


@pytest.mark.parametrize("J", [3, 4])
def test_phi_shift_invariance_and_period(J):
    shape = (10, 6, 12)
    x = _grid(shape, 5)
    t = _targets(400, shape, 6, margin=0.0)
    r = 3
    shifted = t.copy()
    shifted[:, 2] += r
    a = R.polar_sinc_resample(x, shifted, J)
    b = R.polar_sinc_resample(np.roll(x, -r, axis=0), t, J)
    assert np.max(np.abs(a - b)) < 1e-12
    period = t.copy()
    period[:, 2] += shape[0] * 2
    assert np.max(np.abs(R.polar_sinc_resample(x, period, J) - R.polar_sinc_resample(x, t, J))) < 1e-9


def test_sampled_gaussian_converges_with_taps():
    """A Gaussian of sigma = 2.5 samples is band-limited to far below FP64
    rounding at the Nyquist frequency, so the full sinc series reproduces it;
    the truncated series misses the samples beyond J/2, whose sinc weights fall
    off only like 1/(pi t).  Near the centre the error falls fast with J."""
    n_s, sigma, c = 64, 2.5, 31.3
    g = np.exp(-0.5 * ((np.arange(n_s) - c) / sigma) ** 2)
    x = np.broadcast_to(g, (3, 2, n_s)).astype(np.complex128)
    us = np.linspace(29.5, 33.0, 41)
    t = np.stack([us, np.ones_like(us), np.ones_like(us)], axis=1)   # integer theta, phi: weight 1
    exact = np.exp(-0.5 * ((us - c) / sigma) ** 2)
    errs = [np.max(np.abs(R.polar_sinc_resample(x, t, J) - exact)) for J in (3, 4, 8, 16, 24)]
    print("max error, J = 3 4 8 16 24:", ["%.1e" % e for e in errs])
    assert errs[1] > errs[2] > errs[3] > errs[4]
    assert errs[0] < 0.12 and errs[4] < 2e-4


def test_planted_off_by_one_tap_start_is_caught(monkeypatch):
    """A tap window shifted by one still contains an integer target (so the
    integer pin alone cannot see it), but it changes every fractional target:
    the dense-matrix pin catches it."""
    shape = (9, 6, 10)
    x = _grid(shape, 7)
    t = _targets(200, shape, 8)
    want = R.sparse_matrix_resample(x, t, 4)
    monkeypatch.setattr(R, "tap_start", lambda u, J: np.floor(np.asarray(u) - J / 2.0).astype(np.int64))
    got = R.polar_sinc_resample(x, t, 4)
    assert np.max(np.abs(got - want)) > 0.1


def test_library_rejects_bad_arguments():
    from paper_1605_05231_gb300 import binding

    lib = binding.load_library()
    import ctypes

    f = lib.nufft3d_polar_resample
    nul = ctypes.c_void_p(0)
    # null pointers with a nonzero count, bad J and bad grid sizes fail before any device work
    assert f(nul, 4, 4, 4, nul, 10, 3, nul, nul) == -1
    assert f(nul, 4, 4, 4, nul, 0, 3, nul, nul) == 0
    assert f(ctypes.c_void_p(16), 4, 4, 4, ctypes.c_void_p(16), 1, 1, ctypes.c_void_p(16), nul) == -1
    assert f(ctypes.c_void_p(16), 4, 4, 4, ctypes.c_void_p(16), 1, 9, ctypes.c_void_p(16), nul) == -1
    assert f(ctypes.c_void_p(16), 0, 4, 4, ctypes.c_void_p(16), 1, 3, ctypes.c_void_p(16), nul) == -1


# ---------------------------------------------------------------------------
# GPU parity
# ---------------------------------------------------------------------------
def _gpu(cuda_lib, x, t, J):
    import torch

    xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t.astype(np.float32))).cuda()
    out = cuda_lib.polar_resample(xd, td, J)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("J", [2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("n", [1, 37, 1000, 4099])
def test_gpu_matches_oracle(cuda_lib, J, n):
    shape = (12, 9, 40)
    x = _grid(shape, 10 + J)
    t = _targets(n, shape, 20 + n).astype(np.float32)
    got = _gpu(cuda_lib, x, t, J)
    want = R.polar_sinc_resample(x.astype(np.complex64), t.astype(np.float64), J)
    assert O.rel_l2(got, want) < TOL


@pytest.mark.gpu
@pytest.mark.parametrize("J", [3, 6])
@pytest.mark.parametrize("shape", [(2, 9, 40), (12, 2, 40), (12, 9, 2), (1, 1, 1), (5, 4, 3)])
def test_gpu_axes_shorter_than_the_taps(cuda_lib, J, shape):
    """An axis with fewer cells than taps: the library keeps per-tap indices
    there (taps wrap several times on the periodic azimuth, or fall off both
    ends of theta / s), instead of the consecutive taps it uses when every
    axis holds at least J cells."""
    x = _grid(shape, 50 + J)
    t = _targets(1000, shape, 60 + J).astype(np.float32)
    got = _gpu(cuda_lib, x, t, J)
    want = R.polar_sinc_resample(x.astype(np.complex64), t.astype(np.float64), J)
    assert O.rel_l2(got, want) < TOL


@pytest.mark.gpu
def test_gpu_edges_wrap_and_integers(cuda_lib):
    shape = (16, 8, 32)
    x = _grid(shape, 30)
    t = np.array([[0.0, 0.0, 0.0], [31.0, 7.0, 15.0], [-0.4, 3.2, -0.5], [31.6, 7.9, 15.7], [10.5, 3.5, 47.25],
                  [5.0, 2.0, -17.0], [-3.0, -3.0, 2.0], [40.0, 12.0, 3.0], [15.5, 4.0, 1e4 + 0.25]], dtype=np.float32)
    for J in (3, 6):
        got = _gpu(cuda_lib, x, t, J)
        want = R.polar_sinc_resample(x.astype(np.complex64), t.astype(np.float64), J)
        assert np.max(np.abs(got - want)) < 1e-5 * np.max(np.abs(x))
    # nothing to do
    import torch

    out = cuda_lib.polar_resample(torch.from_numpy(x.astype(np.complex64)).cuda(),
                                  torch.zeros((0, 3), dtype=torch.float32, device="cuda"), 3)
    assert out.shape == (0,)


@pytest.mark.gpu
def test_gpu_full_size_polar_grid_sampled(cuda_lib):
    """The 360 x 256 x 512 polar grid of the 256^3 workload's plane integrals,
    resampled at 47,185,920 targets shifted off the grid by (0.37, 0.21, 0.43)
    cells, in the launch configuration bench.py times; 4096 sampled targets
    against the oracle."""
    import torch

    w = I.workload("full256")
    shape = (w.n_az, w.n_pol, w.m)
    x = _grid(shape, 40).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    td = I.shifted_polar_targets(shape, (0.37, 0.21, 0.43), device="cuda")
    out = cuda_lib.polar_resample(xd, td, 3)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(41).choice(td.shape[0], 4096, replace=False))
    t = td[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    want = R.polar_sinc_resample(x, t, 3)
    assert O.rel_l2(out[torch.from_numpy(idx).cuda()].cpu().numpy(), want) < TOL
