"""FP64 CPU oracle for the NUFFT-based resampling of the polar Radon grid
(the paper's first resampling method, Sec. 2.1.3, Eqs. 2.8-2.11).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it is used by ``tests/`` and the CPU legs of ``bench.py``
and nowhere else.  It shares no code with the CUDA library.

What it computes.  The radially sampled Radon data x are uniform on the polar
grid x[phi][theta][s] (Fig. 2.10).  Eq. 2.8 resamples them at nonuniform points
u = (u_s, u_theta, u_phi) (grid-index units) with the ideal interpolator T,
whose rows are shifted periodic sincs; Eq. 2.9 writes T = T F F^-1 and
Eq. 2.10 reads T F I as a NUFFT with a rectangular pre-window; Eq. 2.11 swaps
that for a smooth pre-window P and truncates the interpolator:

    x~ ~= T_sparse F P F^-1 x.

Definitions used here (per axis a with n_a grid points, centred frequency
index m in [-n_a/2, n_a/2), F the forward DFT with e^{-i} as in Eq. 2.3):

  * exact (Eq. 2.8):   x~(u) = sum_m a[m] e^{-2 pi i m.u / n},
                       a = F^-1 x, a[m] = (1/n) sum_k x[k] e^{+2 pi i m.k / n};
    equivalently x~(u) = sum_k x[k] prod_a D_{n_a}(u_a - k_a) with the
    periodic sinc D_n(t) = (1/n) sum_m e^{-2 pi i m t / n} (Eq. 2.7's kernel);
  * fast (Eq. 2.11):   the type-2 NUFFT of a at omega_a = 2 pi u_a / n_a, in the
    steps of Eq. 2.11: P multiplies a[m] by the Kaiser-Bessel pre-window of
    the axis (the projector's scaling factors with N = n_a, symmetric about
    the middle of the index range), F is the unnormalised K_a-point DFT of the
    zero-padded result (K_a = os n_a), and T_sparse is the J-tap min-max
    interpolator of the axis at u'_a = omega_a / gamma_a = os u_a, with taps
    k0 + 1 .. k0 + J, k0 = floor(u') - J/2 and exact per-point coefficients
    c = T^-1 r (the projector oracle's definitions, per axis).

Every axis is periodic, as the DFT makes it (the theta and s ranges wrap); the
unpaired frequency m = -n/2 makes the interpolant complex for real x.

Parity status: pinned by tests/test_polar_nufft_resample.py (exact reproduction
at grid points, exact interpolation of band-limited trigonometric
polynomials, periodicity, the per-point min-max error bound of the fast
method against the exact one, and planted mistakes).
"""
from __future__ import annotations

import numpy as np

from . import nufft3d_oracle as O


def inverse_dft_centred(x: np.ndarray) -> np.ndarray:
    """a = F^-1 x on centred frequencies: a[m] = (1/n) sum_k x[k] e^{+2 pi i m.k/n},
    returned with index m + n//2 (m = -n/2 .. n/2 - 1) on every axis."""
    return np.fft.fftshift(np.fft.ifftn(np.asarray(x, dtype=np.complex128)))


def exact_resample(x: np.ndarray, targets: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Eq. 2.8 with the ideal interpolator: x~(u) = sum_m a[m] e^{-2 pi i m.u/n},
    evaluated directly (separable sums over the three axes).  targets[P, 3] =
    (u_s, u_theta, u_phi); x[n_phi, n_theta, n_s]."""
    a = inverse_dft_centred(x)
    n_phi, n_theta, n_s = a.shape
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    mp = np.arange(n_phi) - n_phi // 2
    mt = np.arange(n_theta) - n_theta // 2
    ms = np.arange(n_s) - n_s // 2
    out = np.empty(t.shape[0], dtype=np.complex128)
    for b in range(0, t.shape[0], chunk):
        e = min(t.shape[0], b + chunk)
        Es = np.exp(-2j * np.pi * np.outer(t[b:e, 0], ms) / n_s)
        Et = np.exp(-2j * np.pi * np.outer(t[b:e, 1], mt) / n_theta)
        Ep = np.exp(-2j * np.pi * np.outer(t[b:e, 2], mp) / n_phi)
        out[b:e] = np.einsum("pa,pb,pc,abc->p", Ep, Et, Es, a, optimize=True)
    return out


def periodic_sinc(t: np.ndarray, n: int) -> np.ndarray:
    """D_n(t) = (1/n) sum_{m=-n/2}^{n/2-1} e^{-2 pi i m t / n}, summed term by term."""
    t = np.asarray(t, dtype=np.float64)
    m = np.arange(n) - n // 2
    return np.exp(-2j * np.pi * t[..., None] * m / n).sum(axis=-1) / n


def kernel_resample(x: np.ndarray, targets: np.ndarray) -> np.ndarray:
    """Eq. 2.8 written as T x with T's rows the products of periodic sincs
    D(u_a - k_a): the second, independent form of the exact definition (small
    grids only)."""
    x = np.asarray(x, dtype=np.complex128)
    n_phi, n_theta, n_s = x.shape
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.complex128)
    for i, (us, ut, up) in enumerate(t):
        ws = periodic_sinc(us - np.arange(n_s), n_s)
        wt = periodic_sinc(ut - np.arange(n_theta), n_theta)
        wp = periodic_sinc(up - np.arange(n_phi), n_phi)
        out[i] = np.einsum("a,b,c,abc->", wp, wt, ws, x)
    return out


class AxisNufft:
    """One axis of the fast method: N = n grid points, K = os n, J taps, its
    pre-window s(m) on centred m and its min-max interpolator with exact
    per-point coefficients c(f) = T^-1 r(f)."""

    def __init__(self, n: int, os: int, J: int):
        self.N, self.K, self.J = n, os * n, J
        self.s = O.scaling_factors(n, self.K, J)
        self.T = O.minmax_T(n, self.K, J, self.s)

    def coeffs(self, f) -> np.ndarray:
        return O.minmax_coeffs_exact(f, self.N, self.K, self.J, self.s, self.T)


def nufft_resample(x: np.ndarray, targets: np.ndarray, J: int = 6, os: int = 2,
                   chunk: int = 4096) -> np.ndarray:
    """Eq. 2.11, x~ ~= T_sparse F P F^-1 x, in the paper's order (the module
    docstring gives every step's definition).  x[n_phi, n_theta, n_s],
    targets[P, 3] = (u_s, u_theta, u_phi); returns complex128[P]."""
    x = np.asarray(x, dtype=np.complex128)
    n_phi, n_theta, n_s = x.shape
    axes = [AxisNufft(n_phi, os, J), AxisNufft(n_theta, os, J), AxisNufft(n_s, os, J)]
    # F^-1
    a = inverse_dft_centred(x)
    # P: the pre-window of every axis on centred m
    g = a * axes[0].s[:, None, None] * axes[1].s[None, :, None] * axes[2].s[None, None, :]
    # F: zero padding to K (centred m stored at m mod K), unnormalised K-point DFT (e^{-i})
    G = np.zeros((axes[0].K, axes[1].K, axes[2].K), dtype=np.complex128)
    idx = [(np.arange(ax.N) - ax.N // 2) % ax.K for ax in axes]
    G[np.ix_(idx[0], idx[1], idx[2])] = g
    Y = O.grid_fft(G)
    # T_sparse: min-max interpolation at u' = omega / gamma = os u
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.complex128)
    jj = np.arange(1, J + 1)
    for b in range(0, t.shape[0], chunk):
        e = min(t.shape[0], b + chunk)
        taps = []
        for ax, col in ((axes[0], 2), (axes[1], 1), (axes[2], 0)):
            k0, f = O.tap_base(os * t[b:e, col], J)
            taps.append(((k0[:, None] + jj[None, :]) % ax.K, ax.coeffs(f)))
        (ip, cp), (it, ct), (is_, cs) = taps
        V = Y[ip[:, :, None, None], it[:, None, :, None], is_[:, None, None, :]]
        out[b:e] = np.einsum("pa,pb,pc,pabc->p", cp, ct, cs, V)
    return out


def minmax_error_bound(x: np.ndarray, targets: np.ndarray, J: int = 6, os: int = 2) -> np.ndarray:
    """Per-target bound |x~_fast(u) - x~_exact(u)| <= ||a||_2 E(u), a = F^-1 x
    (Cauchy-Schwarz): E(u) = || b3 - a3 ||_2 with b3 the exact exponentials
    e^{-i omega.m} over the centred band and a3 the separable pre-windowed
    interpolator, each a product over the three axes of its 1D factor."""
    a = inverse_dft_centred(x)
    n_phi, n_theta, n_s = np.asarray(x).shape
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    parts = []
    for n, col in ((n_phi, 2), (n_theta, 1), (n_s, 0)):
        _, f = O.tap_base(os * t[:, col], J)
        parts.append(O.minmax_error_1d(f, AxisNufft(n, os, J)))
    bb = np.prod([p[0] for p in parts], axis=0)
    aa = np.prod([p[1] for p in parts], axis=0)
    ab = np.prod([p[2] for p in parts], axis=0)
    return np.linalg.norm(a) * np.sqrt(np.maximum(bb + aa - 2.0 * ab.real, 0.0))
