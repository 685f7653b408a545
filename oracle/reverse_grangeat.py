"""FP64 CPU oracle for the per-view reverse Grangeat step (Sec. 2.2.2,
Fig. 2.15; its costs C3a-C3d in Sec. 2.4, Eqs. 2.21-2.24).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it is used by ``tests/`` and the CPU legs of ``bench.py``
and nowhere else.  It shares no code with the CUDA library.

What it computes.  Each cone-beam view v owns one umbrella subset of the
(derivative of the) Radon data: L lines through the detector plane, line l at
angle alpha_l, M samples per line at offsets s = t - M/2 (t = 0 .. M-1).  The
reverse Grangeat step turns the subset into the view's N x N detector image:

  C3a  de-post-weighting:  y'[l][t] = w_post[l][t] y[l][t];
  C3b  radial FFTs:        Y[l][q] = sum_t y'[l][t] e^{-2 pi i (q - M/2)(t - M/2) / M},
                           the line's spectrum at radial frequency
                           rho = (q - M/2) / M cycles per detector pixel
                           (Fourier slice theorem in the detector plane);
  C3c  2D NUFFT transpose with [J J] neighbours (J = 5 in the paper):
                           z[n] = sum_{l,q} Y[l][q] e^{+i omega_lq . n},
                           omega_lq = 2 pi rho (cos alpha_l, sin alpha_l)
                           = (omega_x, omega_y), n = (n_y, n_x) centred in
                           [-N/2, N/2)^2, omega . n = omega_x n_x + omega_y n_y;
                           fast form: the adjoint of the min-max type-2 NUFFT
                           (K = 2N, Kaiser-Bessel pre-window, taps k0 + 1 ..
                           k0 + J with k0 = floor(u - J/2), u = omega / gamma),
                           i.e. spread with conj(c), unnormalised inverse K^2
                           DFT, crop, pre-window;
  C3d  de-pre-weighting:   out[n] = w_pre[n] z[n].

No ramp filter: the data are already the first derivative of the Radon
transform (Sec. 2.2.2).  The Grangeat pre- and post-weights are defined in a
report the paper cites but does not include, so both are inputs here.

Parity status: pinned by tests/test_reverse_grangeat.py (the radial DFT of a
delta and the 2D Fourier slice theorem on axis-aligned lines, the fast 2D
adjoint against the exact adjoint NUDFT within its per-pixel min-max bound,
the adjoint identity with a direct type-2 sum, and planted mistakes).
"""
from __future__ import annotations

import numpy as np

from . import nufft3d_oracle as O


def line_spectra(y: np.ndarray, w_post: np.ndarray) -> np.ndarray:
    """C3a and C3b: Y[..., l, q] = sum_t w_post y e^{-2 pi i (q - M/2)(t - M/2)/M},
    as a dense DFT matrix product."""
    M = y.shape[-1]
    c = np.arange(M) - M // 2
    E = np.exp(-2j * np.pi * np.outer(c, c) / M)          # [q][t]
    return (np.asarray(y, dtype=np.complex128) * w_post) @ E.T


def polar_u(angles: np.ndarray, M: int, K: int) -> np.ndarray:
    """Grid coordinates u = omega / gamma of the (l, q) samples, (L*M, 2) as
    (u_x, u_y), l-major."""
    rho = (np.arange(M) - M // 2) / M
    a = np.asarray(angles, dtype=np.float64)
    ux = np.outer(np.cos(a), rho) * K
    uy = np.outer(np.sin(a), rho) * K
    return np.stack([ux.ravel(), uy.ravel()], axis=1)


def adjoint_nudft_2d(Y: np.ndarray, angles: np.ndarray, N: int) -> np.ndarray:
    """C3c's exact form: z[n_y, n_x] = sum_p Y_p e^{+i (omega_x n_x + omega_y n_y)}."""
    L, M = Y.shape
    rho = (np.arange(M) - M // 2) / M
    a = np.asarray(angles, dtype=np.float64)
    wx = (2 * np.pi * np.outer(np.cos(a), rho)).ravel()
    wy = (2 * np.pi * np.outer(np.sin(a), rho)).ravel()
    n = np.arange(N) - N // 2
    Ex = np.exp(1j * np.outer(wx, n))                      # [p][n_x]
    Ey = np.exp(1j * np.outer(wy, n))                      # [p][n_y]
    return (Ey * Y.ravel()[:, None]).T @ Ex


class Nufft2D:
    """The 2D min-max NUFFT of one view size: N, K = 2N, J taps, exact
    per-point coefficients (the projector oracle's 1D definitions per axis)."""

    def __init__(self, N: int, J: int = 5, K: int = 0):
        self.N, self.J = N, J
        self.K = K or 2 * N
        self.s = O.scaling_factors(N, self.K, J)
        self.T = O.minmax_T(N, self.K, J, self.s)

    def coeffs(self, f) -> np.ndarray:
        return O.minmax_coeffs_exact(f, self.N, self.K, self.J, self.s, self.T)

    def spread(self, Yp: np.ndarray, u: np.ndarray) -> np.ndarray:
        """G[k_y][k_x] += conj(c_y c_x) Y_p over the J x J taps of every point."""
        K, J = self.K, self.J
        G = np.zeros(K * K, dtype=np.complex128)
        j = np.arange(1, J + 1)
        k0, f = O.tap_base(u, J)
        cx, cy = self.coeffs(f[:, 0]), self.coeffs(f[:, 1])
        ix = (k0[:, 0:1] + j[None, :]) % K
        iy = (k0[:, 1:2] + j[None, :]) % K
        flat = iy[:, :, None] * K + ix[:, None, :]
        w = np.conj(cy[:, :, None] * cx[:, None, :])
        np.add.at(G, flat.ravel(), (w * Yp[:, None, None]).ravel())
        return G.reshape(K, K)

    def adjoint(self, Yp: np.ndarray, u: np.ndarray) -> np.ndarray:
        """Spread, unnormalised inverse K^2 DFT, crop to the centred N^2 box,
        pre-window s(n_y) s(n_x)."""
        G = self.spread(Yp, u)
        z = np.fft.ifft2(G) * G.size
        idx = (np.arange(self.N) - self.N // 2) % self.K
        return z[np.ix_(idx, idx)] * self.s[:, None] * self.s[None, :]

    def forward(self, x: np.ndarray, u: np.ndarray) -> np.ndarray:
        """The type-2 NUFFT whose transpose adjoint() is (for the adjoint identity)."""
        K, J, N = self.K, self.J, self.N
        g = np.zeros((K, K), dtype=np.complex128)
        idx = (np.arange(N) - N // 2) % K
        g[np.ix_(idx, idx)] = x * self.s[:, None] * self.s[None, :]
        Yg = np.fft.fft2(g)
        j = np.arange(1, J + 1)
        k0, f = O.tap_base(u, J)
        cx, cy = self.coeffs(f[:, 0]), self.coeffs(f[:, 1])
        ix = (k0[:, 0:1] + j[None, :]) % K
        iy = (k0[:, 1:2] + j[None, :]) % K
        V = Yg[iy[:, :, None], ix[:, None, :]]
        return np.einsum("pa,pb,pab->p", cy, cx, V)

    def error_bound(self, u: np.ndarray) -> np.ndarray:
        """Per point, || a_p - b_p ||_2 over the N^2 box, with b_p[n] =
        e^{-i omega_p . n} and a_p the pre-windowed min-max interpolant
        (the 2D form of the projector oracle's bound)."""
        _, f = O.tap_base(u, self.J)
        parts = [O.minmax_error_1d(f[:, a], self) for a in range(2)]
        bb = parts[0][0] * parts[1][0]
        aa = parts[0][1] * parts[1][1]
        ab = parts[0][2] * parts[1][2]
        return np.sqrt(np.maximum(bb + aa - 2.0 * ab.real, 0.0))


def reverse_grangeat(y: np.ndarray, w_post: np.ndarray, w_pre: np.ndarray, angles: np.ndarray, N: int,
                     J: int = 5, exact: bool = False) -> np.ndarray:
    """All views: y, w_post [V][L][M], w_pre [V][N][N], angles [L] -> [V][N][N]
    complex, in the order C3a, C3b, C3c, C3d.  exact=True takes C3c's direct
    sum instead of the NUFFT."""
    y = np.asarray(y)
    V, L, M = y.shape
    nu = None if exact else Nufft2D(N, J)
    u = polar_u(angles, M, 2 * N)
    out = np.empty((V, N, N), dtype=np.complex128)
    for v in range(V):
        Y = line_spectra(y[v], w_post[v])
        z = adjoint_nudft_2d(Y, angles, N) if exact else nu.adjoint(Y.ravel(), u)
        out[v] = w_pre[v] * z
    return out


def pixel_error_bound(Y: np.ndarray, angles: np.ndarray, N: int, J: int = 5) -> float:
    """Bound on max_n |z_fast[n] - z_exact[n]| for one view's spectra Y[L][M]:
    z_fast - z_exact = sum_p Y_p conj(a_p - b_p), so every pixel is within
    sum_p |Y_p| max_n |a_p[n] - b_p[n]| <= sum_p |Y_p| E_p, E_p the l2 error
    of point p over the N^2 box (Nufft2D.error_bound)."""
    nu = Nufft2D(N, J)
    u = polar_u(angles, Y.shape[-1], 2 * N)
    return float(np.sum(np.abs(Y.ravel()) * nu.error_bound(u)))
