"""NUFFT-based resampling of the polar Radon grid (Sec. 2.1.3, Eqs. 2.8-2.11).

CPU pins of the oracle (oracle/polar_nufft_resample.py):
- the ideal resampler (Eq. 2.8) reproduces the grid at integer targets;
- its frequency-sum form equals the spatial periodic-sinc form, and the
  periodic sinc equals Eq. 2.7's closed form (a phasor times sin/sin);
- it interpolates band-limited trigonometric polynomials exactly (distinct
  frequencies per axis on a non-cubic grid, the unpaired Nyquist term
  included, so a swapped axis, a sign or a dropped shift fails);
- it is periodic on every axis;
- the fast form (Eq. 2.11) stays within the per-target min-max error bound of
  the exact form, and that bound is small (J = 6, K = 2n);
- planted mistakes (the pre-window of the wrong axis, no oversampling of the
  target coordinate, an unshifted inverse DFT) fail these pins.
"""
import numpy as np
import pytest

from oracle import polar_nufft_resample as R

SHAPE = (10, 12, 16)   # (n_phi, n_theta, n_s), every factor 2, 3, 5


def _grid(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _targets(n, shape, seed):
    rng = np.random.default_rng(seed)
    n_phi, n_theta, n_s = shape
    return np.stack([rng.uniform(-2, n_s + 2, n), rng.uniform(-2, n_theta + 2, n),
                     rng.uniform(-2, n_phi + 2, n)], axis=1)


def _integer_targets(shape, stride=1):
    n_phi, n_theta, n_s = shape
    g = np.stack(np.meshgrid(np.arange(n_s), np.arange(n_theta), np.arange(n_phi), indexing="ij"), -1)
    return g.reshape(-1, 3)[::stride].astype(np.float64)


def _at(x, t):
    k = t.astype(np.int64)
    return x[k[:, 2], k[:, 1], k[:, 0]]


def test_exact_reproduces_grid_samples():
    x = _grid(SHAPE, 1)
    t = _integer_targets(SHAPE)
    np.testing.assert_allclose(R.exact_resample(x, t), _at(x, t), rtol=0, atol=1e-12)


def test_frequency_form_equals_periodic_sinc_form():
    x = _grid(SHAPE, 2)
    t = _targets(40, SHAPE, 3)
    np.testing.assert_allclose(R.exact_resample(x, t), R.kernel_resample(x, t), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [9, 10, 16])
def test_periodic_sinc_closed_form(n):
    # Eq. 2.7: the sum of n unit phasors over a band of n frequencies is a
    # phasor times sin(pi t) / sin(pi t / n); the centred band -n/2 .. n/2-1
    # (n even) or -(n-1)/2 .. (n-1)/2 (n odd) puts the phasor at e^{i pi t/n}
    # for even n and removes it for odd n
    t = np.linspace(-2.7, 3.3, 37) + 1e-3
    phase = np.exp(1j * np.pi * t / n) if n % 2 == 0 else 1.0
    closed = phase * np.sin(np.pi * t) / (n * np.sin(np.pi * t / n))
    np.testing.assert_allclose(R.periodic_sinc(t, n), closed, rtol=0, atol=1e-13)
    # integer arguments: 1 at multiples of n, 0 elsewhere
    k = np.arange(-n, 2 * n)
    np.testing.assert_allclose(R.periodic_sinc(k.astype(float), n), (k % n == 0).astype(float), atol=1e-13)


@pytest.mark.parametrize("m", [(1, -2, 3), (-5, 4, -7), (0, -6, -8), (-5, -6, 5)])
def test_exact_interpolates_trigonometric_polynomials(m):
    # x[k] = prod_a e^{-2 pi i m_a k_a / n_a} has x~(u) = prod_a e^{-2 pi i m_a u_a / n_a}
    # for m_a in the centred band (m = -n/2 is the unpaired Nyquist term)
    n_phi, n_theta, n_s = SHAPE
    mp, mt, ms = m
    kp, kt, ks = np.meshgrid(np.arange(n_phi), np.arange(n_theta), np.arange(n_s), indexing="ij")
    x = np.exp(-2j * np.pi * (mp * kp / n_phi + mt * kt / n_theta + ms * ks / n_s))
    t = _targets(60, SHAPE, 4)
    want = np.exp(-2j * np.pi * (mp * t[:, 2] / n_phi + mt * t[:, 1] / n_theta + ms * t[:, 0] / n_s))
    np.testing.assert_allclose(R.exact_resample(x, t), want, rtol=0, atol=1e-11)


def test_exact_periodic_on_every_axis():
    x = _grid(SHAPE, 5)
    t = _targets(30, SHAPE, 6)
    base = R.exact_resample(x, t)
    n_phi, n_theta, n_s = SHAPE
    for col, n in ((0, n_s), (1, n_theta), (2, n_phi)):
        sh = t.copy()
        sh[:, col] += n * np.array([1, -2, 3] * 10)[: t.shape[0]]
        np.testing.assert_allclose(R.exact_resample(x, sh), base, rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", [SHAPE, (8, 6, 20), (18, 10, 12)])
def test_fast_within_minmax_bound(shape):
    x = _grid(shape, 7)
    t = np.concatenate([_targets(200, shape, 8), _integer_targets(shape, stride=7)])
    fast = R.nufft_resample(x, t)
    exact = R.exact_resample(x, t)
    bound = R.minmax_error_bound(x, t)
    err = np.abs(fast - exact)
    assert np.all(err <= bound * (1 + 1e-6) + 1e-13)
    # J = 6 with twofold oversampling: E(u) is a few 1e-6 of ||b3||_2 =
    # sqrt(n_phi n_theta n_s), the norm of the exact exponentials ...
    assert bound.max() < 1e-5 * np.linalg.norm(R.inverse_dft_centred(x)) * np.sqrt(np.prod(shape))
    # ... and in practice about 1e-6 relative
    assert np.linalg.norm(err) / np.linalg.norm(exact) < 1e-5


def test_fast_reproduces_grid_within_bound():
    x = _grid(SHAPE, 9)
    t = _integer_targets(SHAPE, stride=3)
    err = np.abs(R.nufft_resample(x, t) - _at(x, t))
    assert np.all(err <= R.minmax_error_bound(x, t) * (1 + 1e-6) + 1e-13)


def test_fast_error_shrinks_with_taps():
    x = _grid(SHAPE, 10)
    t = _targets(100, SHAPE, 11)
    exact = R.exact_resample(x, t)
    errs = [np.linalg.norm(R.nufft_resample(x, t, J=J) - exact) for J in (2, 4, 6)]
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


# ---- planted mistakes: each must fail a pin above ---------------------------

def test_planted_wrong_axis_prewindow_fails(monkeypatch):
    shape = (8, 6, 20)
    x = _grid(shape, 12)
    t = _targets(80, shape, 13)
    exact = R.exact_resample(x, t)
    real_axis = R.AxisNufft

    class Swapped(real_axis):
        # the pre-window of a 20-point axis used on every axis of length 8
        def __init__(self, n, os, J):
            super().__init__(n, os, J)
            if n == 8:
                self.s = real_axis(20, os, J).s[6:14]

    monkeypatch.setattr(R, "AxisNufft", Swapped)
    err = np.abs(R.nufft_resample(x, t) - exact)
    monkeypatch.setattr(R, "AxisNufft", real_axis)
    assert np.any(err > R.minmax_error_bound(x, t) * 1.5 + 1e-12)


def test_planted_unscaled_target_fails():
    x = _grid(SHAPE, 14)
    t = _targets(50, SHAPE, 15)
    # interpolating at u instead of os u on the oversampled grid
    wrong = R.nufft_resample(x, t / 2.0)
    assert np.max(np.abs(wrong - R.exact_resample(x, t))) > 1e-2


def test_planted_unshifted_inverse_dft_fails(monkeypatch):
    x = _grid(SHAPE, 16)
    t = _targets(30, SHAPE, 17)
    monkeypatch.setattr(R, "inverse_dft_centred", lambda v: np.fft.ifftn(np.asarray(v, dtype=np.complex128)))
    out = R.exact_resample(x, t)
    monkeypatch.undo()
    assert np.max(np.abs(out - R.kernel_resample(x, t))) > 1e-2


# ---- the library: argument checks without a GPU -----------------------------

def test_library_refuses_unsupported_sizes():
    import ctypes

    from paper_1605_05231_gb300 import binding

    lib = binding.load_library()
    h = ctypes.c_void_p()
    # sizes outside the supported set and odd J are refused before any device call
    assert lib.nufft3d_polar_nufft_create(ctypes.byref(h), 11, 12, 16, 6) == -4
    assert lib.nufft3d_polar_nufft_create(ctypes.byref(h), 10, 12, 1024, 6) == -4
    assert lib.nufft3d_polar_nufft_create(ctypes.byref(h), 10, 12, 16, 5) == -4
    assert lib.nufft3d_polar_nufft_create(ctypes.byref(h), 0, 12, 16, 6) == -1
    assert lib.nufft3d_polar_nufft_create(None, 10, 12, 16, 6) == -1
    assert lib.nufft3d_polar_nufft_destroy(None) == -1


# ---- GPU parity -------------------------------------------------------------
# The CUDA path computes in FP32 with the coefficients fitted to 1e-7; the
# oracle follows the same steps in FP64 with exact coefficients, on the same
# FP32 targets.  FP32 rounding through three n-point and three 2n-point FFTs
# and the J^3 sum gives a few 1e-7 relative; the bar is 1e-5 rel-L2 and, per
# element, 1e-5 of the output's RMS plus the oracle's own min-max bound where
# the exact form is the reference.

RTOL = 1e-5


def _gpu_resample(cuda_lib, x, t, J=6, plan=None):
    import torch

    p = plan or cuda_lib.PolarNufft(*x.shape, J=J)
    xd = torch.from_numpy(np.ascontiguousarray(x).astype(np.complex64)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t).astype(np.float32)).cuda()
    out = p.resample(xd, td)
    torch.cuda.synchronize()
    if plan is None:
        p.close()
    return out.cpu().numpy().astype(np.complex128)


def _check(got, want):
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < RTOL, rel
    rms = np.sqrt(np.mean(np.abs(want) ** 2))
    assert np.max(np.abs(got - want)) < 10 * RTOL * rms


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(10, 12, 16), (20, 24, 32), (40, 12, 10), (90, 64, 128)])
@pytest.mark.parametrize("J", [4, 6, 8])
def test_gpu_matches_oracle(cuda_lib, shape, J):
    x = _grid(shape, 21)
    t = _targets(3001, shape, 22).astype(np.float32).astype(np.float64)
    got = _gpu_resample(cuda_lib, x, t, J)
    _check(got, R.nufft_resample(x, t, J=J))


@pytest.mark.gpu
def test_gpu_against_exact_form_within_bound(cuda_lib):
    shape = (20, 24, 32)
    x = _grid(shape, 23)
    t = _targets(2000, shape, 24).astype(np.float32).astype(np.float64)
    got = _gpu_resample(cuda_lib, x, t)
    exact = R.exact_resample(x, t)
    bound = R.minmax_error_bound(x, t)
    rms = np.sqrt(np.mean(np.abs(exact) ** 2))
    assert np.all(np.abs(got - exact) <= bound + 2e-6 * rms)


@pytest.mark.gpu
def test_gpu_wrap_integer_and_far_targets(cuda_lib):
    shape = (10, 12, 16)
    x = _grid(shape, 25)
    n_phi, n_theta, n_s = shape
    ints = _integer_targets(shape)
    # every axis periodic: targets one to three periods away, negative ones,
    # and targets on the wrap boundary of the oversampled grid (u = n/2, n)
    far = ints + np.array([3 * n_s, -2 * n_theta, 5 * n_phi], dtype=np.float64)
    edge = np.array([[n_s / 2, n_theta / 2, n_phi / 2], [n_s, n_theta, n_phi], [-0.25, -0.5, -0.75],
                     [n_s - 0.5, n_theta - 1e-3, n_phi - 0.5], [0.0, 0.0, 0.0]], dtype=np.float64)
    t = np.concatenate([ints, far, edge]).astype(np.float32).astype(np.float64)
    got = _gpu_resample(cuda_lib, x, t)
    _check(got, R.nufft_resample(x, t))
    # grid reproduction at the integer targets, within the min-max error
    rms = np.sqrt(np.mean(np.abs(x) ** 2))
    assert np.max(np.abs(got[:len(ints)] - _at(x, ints))) < 1e-4 * rms


@pytest.mark.gpu
def test_gpu_ragged_counts_nan_and_gather_reuse(cuda_lib):
    import torch

    shape = (20, 24, 32)
    x = _grid(shape, 27)
    p = cuda_lib.PolarNufft(*shape)
    assert p.info()["fit_error"] < 1e-7
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    p.prepare(xd)
    for n in (0, 1, 255, 257, 4099):
        t = _targets(n, shape, 30 + n).astype(np.float32)
        out = p.gather(torch.from_numpy(t).cuda().reshape(n, 3))
        torch.cuda.synchronize()
        if n:
            _check(out.cpu().numpy().astype(np.complex128), R.nufft_resample(x, t.astype(np.float64)))
    bad = torch.tensor([[np.nan, 1.0, 1.0], [1.0, np.inf, 1.0], [1.0, 1.0, 2.0 ** 23], [1.0, 2.0, 3.0]],
                       dtype=torch.float32, device="cuda")
    out = p.gather(bad).cpu().numpy()
    assert np.all(np.isnan(out[:3].real)) and np.isfinite(out[3].real)
    p.close()


@pytest.mark.gpu
def test_gpu_full_size_trigonometric_polynomial(cuda_lib):
    """The 360 x 256 x 512 polar grid of the 256^3 workload holding a band-
    limited trigonometric polynomial, resampled onto the grid shifted by
    (0.37, 0.21, 0.43) cells: Eq. 2.8's exact value is the polynomial itself at
    every one of the 47 M targets; the fast form stays within J = 6's min-max
    error."""
    import torch

    from paper_1605_05231_gb300 import inputs as I

    shape = (360, 256, 512)
    m = (-31, 17, -180)
    dev = torch.device("cuda")
    kp = torch.arange(shape[0], device=dev, dtype=torch.float64)
    kt = torch.arange(shape[1], device=dev, dtype=torch.float64)
    ks = torch.arange(shape[2], device=dev, dtype=torch.float64)
    ph = (m[0] * kp / shape[0])[:, None, None] + (m[1] * kt / shape[1])[None, :, None] + \
        (m[2] * ks / shape[2])[None, None, :]
    x = torch.exp(-2j * np.pi * ph).to(torch.complex64)
    del ph
    t = I.shifted_polar_targets(shape, (0.37, 0.21, 0.43), device=dev)
    p = cuda_lib.PolarNufft(*shape)
    out = p.resample(x, t)
    td = t.double()
    want = torch.exp(-2j * np.pi * (m[0] * td[:, 2] / shape[0] + m[1] * td[:, 1] / shape[1] +
                                    m[2] * td[:, 0] / shape[2]))
    err = (out.to(torch.complex128) - want).abs()
    # per axis the min-max error of one frequency stays below 4.2e-6 at these
    # m (J = 6, K = 2n); three axes and FP32 rounding stay below 2e-5
    assert float(err.max()) < 2e-5
    p.close()


@pytest.mark.gpu
def test_gpu_full_size_sampled_against_exact(cuda_lib):
    """Seeded normal data on the full 360 x 256 x 512 grid: 48 sampled targets
    of the shifted grid against Eq. 2.8 evaluated directly in FP64."""
    import torch

    from paper_1605_05231_gb300 import inputs as I

    shape = (360, 256, 512)
    x = _grid(shape, 31)
    t = I.shifted_polar_targets(shape, (0.37, 0.21, 0.43))
    idx = np.random.default_rng(32).choice(t.shape[0], 48, replace=False)
    p = cuda_lib.PolarNufft(*shape)
    out = p.resample(torch.from_numpy(x.astype(np.complex64)).cuda(), torch.from_numpy(t).cuda())
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    p.close()
    want = R.exact_resample(x, t[idx].astype(np.float64), chunk=8)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < RTOL, rel
