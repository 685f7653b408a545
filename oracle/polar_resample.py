"""FP64 CPU oracle for the direct (truncated-sinc) resampling of the polar
Radon grid, Sec. 2.1, Eqs. 2.12-2.15.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it is used by ``tests/`` and the CPU legs of ``bench.py``
and nowhere else.  It shares no code with the CUDA library.

What it computes.  The radially sampled Radon data are uniform on a polar grid
(Sec. 2.1, the paragraph before Eq. 2.8, and Fig. 2.10): index u_s along each
line (the plane offset), u_theta over the polar angles and u_phi over the
azimuths.  Eq. 2.15 resamples such a uniform signal at nonuniform points with
two truncated-sinc operators, x~ = T1 T2^T x, where T2 is the identity for data
that need no reordering; so x~ = T1 x with

    x~(u) = sum_{k in taps(u)} sinc(u_s - k_s) sinc(u_theta - k_theta)
                                sinc(u_phi - k_phi) x[k_phi, k_theta, k_s],
    sinc(t) = sin(pi t) / (pi t),  sinc(0) = 1,

each axis keeping the J integers nearest the target: the truncation after
Eq. 2.13 keeps the sinc's central lobe and its closest side lobes.  The
paper's runs use J = 3 ([3 3 3], Sec. 3.2).

Readings where the paper is silent:
  * taps k0 .. k0 + J - 1 with k0 = floor(u - J/2) + 1 on every axis;
  * the azimuth is periodic: k_phi is taken modulo n_phi;
  * the polar angle and the line offset are not: taps outside [0, n_theta) or
    [0, n_s) add nothing (the Radon data of a compact object vanish beyond the
    lines' ends; the polar range stops at the trajectory's missing cone);
  * grid layout x[phi][theta][s] (azimuth-major, the order of the forward
    projector's lines), targets as (u_s, u_theta, u_phi) in grid-index units.

Parity status: pinned by tests/test_polar_resample.py (exact reproduction at
integer targets, an explicit dense sparse-matrix build, shift invariance and
periodicity in phi against np.roll, convergence of a sampled Gaussian).
"""
from __future__ import annotations

import numpy as np


def tap_start(u: np.ndarray, J: int) -> np.ndarray:
    """First tap index k0 = floor(u - J/2) + 1 (the J nearest integers)."""
    return np.floor(np.asarray(u, dtype=np.float64) - J / 2.0).astype(np.int64) + 1


def polar_sinc_resample(x: np.ndarray, targets: np.ndarray, J: int, chunk: int = 65536) -> np.ndarray:
    """Eq. 2.15 with T2 = I: x[n_phi, n_theta, n_s] sampled at targets[P, 3] =
    (u_s, u_theta, u_phi); returns complex128[P]."""
    x = np.asarray(x, dtype=np.complex128)
    n_phi, n_theta, n_s = x.shape
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(t.shape[0], dtype=np.complex128)
    j = np.arange(J)
    for a in range(0, t.shape[0], chunk):
        b = min(t.shape[0], a + chunk)
        us, ut, up = t[a:b, 0], t[a:b, 1], t[a:b, 2]
        ks = tap_start(us, J)[:, None] + j          # (P, J)
        kt = tap_start(ut, J)[:, None] + j
        kp = tap_start(up, J)[:, None] + j
        ws = np.sinc(us[:, None] - ks)               # np.sinc(t) = sin(pi t)/(pi t)
        wt = np.sinc(ut[:, None] - kt)
        wp = np.sinc(up[:, None] - kp)
        ws = np.where((ks >= 0) & (ks < n_s), ws, 0.0)
        wt = np.where((kt >= 0) & (kt < n_theta), wt, 0.0)
        kpm = np.mod(kp, n_phi)
        kss = np.clip(ks, 0, n_s - 1)
        ktc = np.clip(kt, 0, n_theta - 1)
        vals = x[kpm[:, :, None, None], ktc[:, None, :, None], kss[:, None, None, :]]  # (P, J, J, J)
        w = wp[:, :, None, None] * wt[:, None, :, None] * ws[:, None, None, :]
        out[a:b] = np.sum(w * vals, axis=(1, 2, 3))
    return out


def sparse_matrix_resample(x: np.ndarray, targets: np.ndarray, J: int) -> np.ndarray:
    """The same operator built as an explicit dense matrix T1 (one row per
    target, one column per grid cell, entries sinc products where every axis
    distance is inside the tap window, phi distances taken on the circle) and
    applied as T1 @ vec(x).  For small grids only: it is the independent
    formulation the tap-based function is pinned against."""
    x = np.asarray(x, dtype=np.complex128)
    n_phi, n_theta, n_s = x.shape
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    T = np.zeros((t.shape[0], x.size), dtype=np.float64)
    cs = np.arange(n_s)
    ct = np.arange(n_theta)
    cp = np.arange(n_phi)
    for r, (us, ut, up) in enumerate(t):
        def axis_w(u, cells, period=None):
            k0 = int(np.floor(u - J / 2.0)) + 1
            w = np.zeros(len(cells))
            for k in range(k0, k0 + J):
                if period is None:
                    if 0 <= k < len(cells):
                        w[k] += np.sinc(u - k)
                else:
                    w[k % period] += np.sinc(u - k)
            return w
        ws = axis_w(us, cs)
        wt = axis_w(ut, ct)
        wp = axis_w(up, cp, period=n_phi)
        T[r] = np.einsum('p,t,s->pts', wp, wt, ws).ravel()
    return T @ x.ravel()
