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
