"""FP64 CPU oracle for the radial-line 3D NUFFT projector and its adjoint.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it is used by ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference leg of ``bench.py`` and nowhere else.  It shares
no code with the CUDA library; both sides only consume the same seeded inputs.

What it computes (the image-to-Radon step of the forward projector, Sec. 2 step 1
and Sec. 2.2.1, and its transpose, Sec. 2.3):

  forward  p = L_w  T  F  P  x          (Eq. 2.11 structure T_sparse F P, then
                                           a radial 1D inverse DFT per line:
                                           Fourier Slice Theorem, Sec. 2.2.1)
  adjoint  x~ = P^H F^H T^H L_w^H p

  P  : diagonal deapodisation ("pre-scaling", Eq. 2.11) of the N^3 volume and
       zero padding to the K^3 oversampled grid;
  F  : unnormalised K^3 DFT, e^{-i}, centred voxel index n in [-N/2, N/2)^3;
  T  : separable J-tap min-max interpolation (Fessler-Sutton min-max NUFFT, the
       interpolator the paper uses through its toolbox) from the grid to the
       nonuniform points omega_{l,q} = r_q d_l lying on radial lines (Eq. 2.1);
  L_w: per-line centred inverse DFT with weight w[q] and 1/M scaling, giving
       plane integrals (Fourier Slice Theorem, Sec. 2.2.1).

Exact reference (O-exact): X(omega) = sum_n x[n] e^{-i omega.n} (the 3D analogue
of Eq. 2.3) evaluated directly, then L_w.  With w = 1 this is the periodic-sinc
(Dirichlet) plane sum of Eqs. 2.6-2.7: p[s] = sum_n x[n] D_M(d.n - s).

Readings of points the paper leaves open:
  * scaling s(n) = Psi(0) / Psi((n - n_c)/K), Psi the Fourier transform of the
    Kaiser-Bessel window of width J and shape alpha = 2.34 J, centred on the
    middle n_c of the index range (n_c = -1/2 for even N, 0 for odd N), so the
    pre-window is symmetric over the volume (the paper names a Kaiser-Bessel /
    raised-cosine pre-window, Sec. 2.1.3 and Eq. 2.11, without formula);
  * taps k0 + j, j = 1..J, k0 = floor(u - J/2), f = u - J/2 - k0 in [0, 1),
    u = omega / gamma, gamma = 2 pi / K;
  * min-max coefficients c(f) = T^{-1} r(f), T_{jj'} = sum_n s(n)^2 e^{i gamma (j-j') n},
    r_j(f) = sum_n s(n) e^{-i gamma (f + J/2 - j) n};
  * table variant: c tabulated at f_i = i / L, i = 0..L, linear interpolation;
  * radial samples q = m - M/2, m = 0..M-1, radius r_q = q K / M grid units
    (omega = 2 pi q / M rad/voxel), output index s = t - M/2.

Every function is plain NumPy in complex128 with no blocking or reordering
beyond the definitions above (chunking over points only bounds memory).
Parity status: every function here is pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

try:  # library FFT (pinned against a brute DFT in the tests)
    import scipy.fft as _sfft

    def _fftn(a):
        return _sfft.fftn(a, workers=-1)

    def _ifftn_unnorm(a):
        return _sfft.ifftn(a, workers=-1, norm="forward")
except Exception:  # pragma: no cover
    def _fftn(a):
        return np.fft.fftn(a)

    def _ifftn_unnorm(a):
        return np.fft.ifftn(a) * a.size


# -----------------------------------------------------------------------------
# scaling factors (the diagonal P of Eq. 2.11)
# -----------------------------------------------------------------------------
def kb_alpha(J: int) -> float:
    """Kaiser-Bessel shape parameter alpha = 2.34 J (K/N = 2 choice)."""
    return 2.34 * J


def kb_window_ft(nu, J: int, alpha: Optional[float] = None):
    """Fourier transform of the Kaiser-Bessel window
    psi(t) = I0(alpha sqrt(1 - (2t/J)^2)) on |t| <= J/2, at frequency nu
    (cycles per grid sample): J sinh(z) / z, z = sqrt(alpha^2 - (pi J nu)^2)
    (sin(|z|)/|z| when the radicand is negative)."""
    if alpha is None:
        alpha = kb_alpha(J)
    nu = np.asarray(nu, dtype=np.float64)
    z2 = alpha ** 2 - (np.pi * J * nu) ** 2
    out = np.empty_like(z2)
    pos = z2 > 0
    z = np.sqrt(np.abs(z2))
    with np.errstate(invalid="ignore", divide="ignore"):
        out[pos] = np.sinh(z[pos]) / z[pos]
        out[~pos] = np.where(z[~pos] > 0, np.sin(z[~pos]) / np.where(z[~pos] > 0, z[~pos], 1.0), 1.0)
    return J * out


def index_centre(N: int) -> float:
    """Middle of the centred index range -N//2 .. N - N//2 - 1: -1/2 for even N,
    0 for odd N."""
    return 0.5 * ((-(N // 2)) + (N - N // 2 - 1))


def scaling_factors(N: int, K: int, J: int) -> np.ndarray:
    """s(n) = Psi(0) / Psi((n - n_c) / K) for the centred index n = -N/2 .. N/2-1,
    n_c the middle of that range: the Kaiser-Bessel pre-window symmetric over
    the volume (s(n) = s(2 n_c - n))."""
    n = np.arange(-(N // 2), N - N // 2, dtype=np.float64)
    return kb_window_ft(0.0, J) / kb_window_ft((n - index_centre(N)) / K, J)


# -----------------------------------------------------------------------------
# min-max interpolator
# -----------------------------------------------------------------------------
def centred_index(N: int) -> np.ndarray:
    return np.arange(-(N // 2), N - N // 2, dtype=np.float64)


def minmax_T(N: int, K: int, J: int, s: np.ndarray) -> np.ndarray:
    """T_{jj'} = sum_n s(n)^2 exp(i gamma (j - j') n), j, j' = 1..J (J x J)."""
    n = centred_index(N)
    gam = 2.0 * np.pi / K
    j = np.arange(1, J + 1, dtype=np.float64)
    diff = j[:, None] - j[None, :]
    return np.sum((s ** 2)[None, None, :] * np.exp(1j * gam * diff[:, :, None] * n[None, None, :]), axis=2)


def minmax_r(f, N: int, K: int, J: int, s: np.ndarray) -> np.ndarray:
    """r_j(f) = sum_n s(n) exp(-i gamma (f + J/2 - j) n) for each f: shape (len(f), J)."""
    f = np.atleast_1d(np.asarray(f, dtype=np.float64))
    n = centred_index(N)
    gam = 2.0 * np.pi / K
    j = np.arange(1, J + 1, dtype=np.float64)
    dist = f[:, None] + J / 2.0 - j[None, :]  # (P, J)
    return np.exp(-1j * gam * dist[:, :, None] * n[None, None, :]) @ s


def minmax_coeffs_exact(f, N: int, K: int, J: int, s: np.ndarray,
                        T: Optional[np.ndarray] = None) -> np.ndarray:
    """Min-max coefficients c(f) = T^{-1} r(f) at each fractional offset f, (P, J)."""
    if T is None:
        T = minmax_T(N, K, J, s)
    r = minmax_r(f, N, K, J, s)
    return np.linalg.solve(T, r.T).T


def minmax_table(N: int, K: int, J: int, L: int, s: np.ndarray) -> np.ndarray:
    """c_j(f_i) at f_i = i / L, i = 0..L (inclusive): complex128 (L + 1, J)."""
    f = np.arange(L + 1, dtype=np.float64) / L
    return minmax_coeffs_exact(f, N, K, J, s)


def coeffs_from_table(table: np.ndarray, f) -> np.ndarray:
    """Linear interpolation of the table rows at f in [0, 1): (P, J)."""
    L = table.shape[0] - 1
    f = np.asarray(f, dtype=np.float64)
    fl = f * L
    i = np.minimum(np.floor(fl).astype(np.int64), L - 1)
    t = (fl - i)[:, None]
    return (1.0 - t) * table[i] + t * table[i + 1]


# -----------------------------------------------------------------------------
# plan: every derived quantity in FP64
# -----------------------------------------------------------------------------
@dataclasses.dataclass
class OraclePlan:
    N: int
    K: int
    J: int
    L: int            # table oversampling; 0 selects exact per-point coefficients
    dirs: np.ndarray  # (D, 3) unit vectors (x, y, z)
    M: int
    omega: Optional[np.ndarray] = None   # (M,) rad/voxel; None -> 2 pi (m - M/2) / M
    weight: Optional[np.ndarray] = None  # (M,) complex; None -> 1
    complex_volume: bool = False
    do_line_fft: bool = True
    line_weight: Optional[np.ndarray] = None  # (D,) real per-line weights; None -> 1

    def __post_init__(self):
        self.dirs = np.asarray(self.dirs, dtype=np.float64).reshape(-1, 3)
        self.s = scaling_factors(self.N, self.K, self.J)
        self.T = minmax_T(self.N, self.K, self.J, self.s)
        self.table = (minmax_table(self.N, self.K, self.J, self.L, self.s)
                      if self.L > 0 else None)
        w = np.ones(self.M, dtype=np.complex128) if self.weight is None else \
            np.asarray(self.weight, dtype=np.complex128)
        self.w = w
        self.lw = (np.ones(self.dirs.shape[0]) if self.line_weight is None else
                   np.asarray(self.line_weight, dtype=np.float64).reshape(-1))

    def line_weights(self, lines=None) -> np.ndarray:
        return self.lw if lines is None else self.lw[np.asarray(lines)]

    @property
    def D(self) -> int:
        return self.dirs.shape[0]

    def radii(self) -> np.ndarray:
        """Radial coordinate of each sample in grid units: u = radius * d."""
        if self.omega is None:
            q = np.arange(self.M, dtype=np.float64) - self.M // 2
            return q * (self.K / self.M)
        return np.asarray(self.omega, dtype=np.float64) * self.K / (2.0 * np.pi)

    def omegas(self) -> np.ndarray:
        """Radial frequency (rad/voxel) of each sample along a line."""
        if self.omega is None:
            q = np.arange(self.M, dtype=np.float64) - self.M // 2
            return 2.0 * np.pi * q / self.M
        return np.asarray(self.omega, dtype=np.float64)

    def point_u(self, lines=None) -> np.ndarray:
        """Grid coordinates u = omega / gamma of the points, (n_lines, M, 3) (x, y, z)."""
        d = self.dirs if lines is None else self.dirs[np.asarray(lines)]
        return self.radii()[None, :, None] * d[:, None, :]

    def coeffs(self, f) -> np.ndarray:
        if self.table is None:
            return minmax_coeffs_exact(f, self.N, self.K, self.J, self.s, self.T)
        return coeffs_from_table(self.table, f)


def tap_base(u: np.ndarray, J: int):
    """k0 = floor(u - J/2) and f = u - J/2 - k0 (taps k0 + 1 .. k0 + J)."""
    v = u - J / 2.0
    k0 = np.floor(v)
    return k0.astype(np.int64), v - k0


# -----------------------------------------------------------------------------
# the steps
# -----------------------------------------------------------------------------
def deapodize_pad(x: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """g[n mod K] = s(nx) s(ny) s(nz) x[n] on the K^3 grid, zero elsewhere."""
    N, K, s = plan.N, plan.K, plan.s
    g = np.zeros((K, K, K), dtype=np.complex128)
    idx = np.arange(-(N // 2), N - N // 2) % K
    scaled = x.astype(np.complex128) * s[:, None, None] * s[None, :, None] * s[None, None, :]
    g[np.ix_(idx, idx, idx)] = scaled
    return g


def grid_fft(g: np.ndarray) -> np.ndarray:
    """Y[k] = sum_n g[n] exp(-i 2 pi k.n / K), unnormalised."""
    return _fftn(g)


def grid_ifft_unnormalised(G: np.ndarray) -> np.ndarray:
    """z[n] = sum_k G[k] exp(+i 2 pi k.n / K) (the adjoint of grid_fft)."""
    return _ifftn_unnorm(G)


def crop_deapodize(z: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """x~[n] = s(n) z[n mod K] on the N^3 box (adjoint of deapodize_pad)."""
    N, K, s = plan.N, plan.K, plan.s
    idx = np.arange(-(N // 2), N - N // 2) % K
    out = z[np.ix_(idx, idx, idx)] * s[:, None, None] * s[None, :, None] * s[None, None, :]
    return out if plan.complex_volume else out.real


def _chunks(P: int, size: int):
    for a in range(0, P, size):
        yield a, min(P, a + size)


def interp_gather(Y: np.ndarray, u: np.ndarray, plan: OraclePlan, chunk: int = 4096) -> np.ndarray:
    """X^(omega_p) = sum_{jz,jy,jx} c_jz(fz) c_jy(fy) c_jx(fx) Y[(k0 + j) mod K].

    u: (P, 3) grid coordinates (x, y, z).  Y is indexed [kz][ky][kx]."""
    K, J = plan.K, plan.J
    P = u.shape[0]
    out = np.empty(P, dtype=np.complex128)
    j = np.arange(1, J + 1)
    for a, b in _chunks(P, chunk):
        k0, f = tap_base(u[a:b], J)
        cx, cy, cz = plan.coeffs(f[:, 0]), plan.coeffs(f[:, 1]), plan.coeffs(f[:, 2])
        ix = (k0[:, 0:1] + j[None, :]) % K
        iy = (k0[:, 1:2] + j[None, :]) % K
        iz = (k0[:, 2:3] + j[None, :]) % K
        V = Y[iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :]]
        out[a:b] = np.einsum("pz,py,px,pzyx->p", cz, cy, cx, V)
    return out


def interp_spread(Yhat: np.ndarray, u: np.ndarray, plan: OraclePlan, chunk: int = 4096) -> np.ndarray:
    """Adjoint of interp_gather: G[(k0 + j) mod K] += conj(c c c) Yhat_p."""
    K, J = plan.K, plan.J
    G = np.zeros(K * K * K, dtype=np.complex128)
    P = u.shape[0]
    j = np.arange(1, J + 1)
    for a, b in _chunks(P, chunk):
        k0, f = tap_base(u[a:b], J)
        cx, cy, cz = plan.coeffs(f[:, 0]), plan.coeffs(f[:, 1]), plan.coeffs(f[:, 2])
        ix = (k0[:, 0:1] + j[None, :]) % K
        iy = (k0[:, 1:2] + j[None, :]) % K
        iz = (k0[:, 2:3] + j[None, :]) % K
        flat = (iz[:, :, None, None] * K + iy[:, None, :, None]) * K + ix[:, None, None, :]
        w = np.conj(cz[:, :, None, None] * cy[:, None, :, None] * cx[:, None, None, :])
        np.add.at(G, flat.ravel(), (w * Yhat[a:b, None, None, None]).ravel())
    return G.reshape(K, K, K)


def line_exponent(M: int) -> np.ndarray:
    """E[q, s] = exp(2 pi i q s / M) for the centred q, s = -M/2 .. M/2-1."""
    q = np.arange(M, dtype=np.float64) - M // 2
    return np.exp(2j * np.pi * np.outer(q, q) / M)


def radial_idft(Xhat: np.ndarray, plan: OraclePlan, lines=None) -> np.ndarray:
    """p[l][s] = (1/M) lw[l] sum_q w[q] X^[l][q] exp(+2 pi i q s / M)  (Fourier
    Slice Theorem, Sec. 2.2.1; Eqs. 2.2-2.7 in the radial coordinate)."""
    M = plan.M
    lw = plan.line_weights(lines)[:, None]
    return ((Xhat * plan.w[None, :] * lw) @ line_exponent(M)) / M


def radial_idft_adjoint(y: np.ndarray, plan: OraclePlan, lines=None) -> np.ndarray:
    """Y^[l][q] = (1/M) lw[l] conj(w[q]) sum_s y[l][s] exp(-2 pi i q s / M)."""
    M = plan.M
    lw = plan.line_weights(lines)[:, None]
    return (y @ np.conj(line_exponent(M)).T) * np.conj(plan.w)[None, :] * lw / M


# -----------------------------------------------------------------------------
# the operators
# -----------------------------------------------------------------------------
def nufft_forward(x: np.ndarray, plan: OraclePlan, lines=None, return_samples: bool = False):
    """Forward projector step 1: volume -> line data (D, M) (or the selected lines).

    With plan.do_line_fft False the raw Fourier samples X^ are returned."""
    Y = grid_fft(deapodize_pad(x, plan))
    u = plan.point_u(lines)
    nl = u.shape[0]
    Xhat = interp_gather(Y, u.reshape(-1, 3), plan).reshape(nl, plan.M)
    if return_samples or not plan.do_line_fft:
        return Xhat
    return radial_idft(Xhat, plan, lines)


def nufft_adjoint(y: np.ndarray, plan: OraclePlan, lines=None) -> np.ndarray:
    """Adjoint of nufft_forward: line data (D, M) (or the selected lines) -> volume."""
    Yhat = radial_idft_adjoint(y, plan, lines) if plan.do_line_fft else y
    u = plan.point_u(lines)
    G = interp_spread(Yhat.reshape(-1), u.reshape(-1, 3), plan)
    return crop_deapodize(grid_ifft_unnormalised(G), plan)


# -----------------------------------------------------------------------------
# exact references
# -----------------------------------------------------------------------------
def nudft_type2(x: np.ndarray, omega_pts: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """X(omega) = sum_n x[n] exp(-i omega . n) at each point (P, 3) (x, y, z),
    n centred; computed as a separable contraction (Eq. 2.3 in 3D)."""
    N = x.shape[0]
    n = centred_index(N)
    xc = x.astype(np.complex128)
    P = omega_pts.shape[0]
    out = np.empty(P, dtype=np.complex128)
    for a, b in _chunks(P, chunk):
        om = omega_pts[a:b]
        Ex = np.exp(-1j * om[:, 0:1] * n[None, :])  # (p, nx)
        Ey = np.exp(-1j * om[:, 1:2] * n[None, :])
        Ez = np.exp(-1j * om[:, 2:3] * n[None, :])
        t1 = xc.reshape(N * N, N) @ Ex.T            # (nz*ny, p)
        t1 = t1.reshape(N, N, -1)                   # (nz, ny, p)
        t2 = np.einsum("zyp,py->zp", t1, Ey)
        out[a:b] = np.einsum("zp,pz->p", t2, Ez)
    return out


def forward_exact(x: np.ndarray, plan: OraclePlan, lines=None, return_samples: bool = False):
    """O-exact: exact Fourier samples on the radial lines, then the radial IDFT."""
    d = plan.dirs if lines is None else plan.dirs[np.asarray(lines)]
    om = plan.omegas()[None, :, None] * d[:, None, :]
    X = nudft_type2(x, om.reshape(-1, 3)).reshape(d.shape[0], plan.M)
    if return_samples:
        return X
    return radial_idft(X, plan, lines)


def dirichlet_kernel(t: np.ndarray, M: int) -> np.ndarray:
    """D_M(t) = (1/M) sum_{q=-M/2}^{M/2-1} exp(-2 pi i q t / M) in closed form:
    (1/M) exp(i pi t / M) sin(pi t) / sin(pi t / M) (Eqs. 2.6-2.7), equal to 1 at
    t = 0 mod M."""
    t = np.asarray(t, dtype=np.float64)
    den = np.sin(np.pi * t / M)
    near = np.abs(den) < 1e-12
    safe = np.where(near, 1.0, den)
    val = np.exp(1j * np.pi * t / M) * np.sin(np.pi * t) / (M * safe)
    # at t = k M (k integer) the limit is 1
    return np.where(near, 1.0 + 0j, val)


def dirichlet_plane_sums(x: np.ndarray, dirs: np.ndarray, M: int) -> np.ndarray:
    """p[l][s] = sum_n x[n] D_M(d_l . n - s), s = -M/2..M/2-1 (brute force)."""
    N = x.shape[0]
    n = centred_index(N)
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    xv = x.reshape(-1).astype(np.complex128)
    s = np.arange(M, dtype=np.float64) - M // 2
    out = np.empty((dirs.shape[0], M), dtype=np.complex128)
    for l, d in enumerate(np.asarray(dirs, dtype=np.float64)):
        proj = (d[0] * nx + d[1] * ny + d[2] * nz).reshape(-1)
        Dk = dirichlet_kernel(proj[None, :] - s[:, None], M)  # (M, N^3)
        out[l] = Dk @ xv
    return out


# -----------------------------------------------------------------------------
# closed forms for phantoms (pins of the physical scaling)
# -----------------------------------------------------------------------------
def ellipsoid_ft(ell, k: np.ndarray) -> np.ndarray:
    """Continuous FT F(k) = int f(r) exp(-2 pi i k . r) dr of one constant-density
    ellipsoid, k in cycles per field of view, (P, 3)."""
    a = np.asarray(ell.axes, dtype=np.float64)
    R = np.asarray(ell.rot, dtype=np.float64)
    kb = (k @ R) * a[None, :]                 # diag(a) R^T k
    kap = np.linalg.norm(kb, axis=1)
    tk = 2.0 * np.pi * kap
    with np.errstate(invalid="ignore", divide="ignore"):
        ball = (np.sin(tk) - tk * np.cos(tk)) / (2.0 * np.pi ** 2 * kap ** 3)
    ball = np.where(kap < 1e-8, 4.0 * np.pi / 3.0, ball)
    phase = np.exp(-2j * np.pi * (k @ np.asarray(ell.center, dtype=np.float64)))
    return ell.density * np.prod(a) * ball * phase


def ellipsoid_plane_integral(ell, d: np.ndarray, t: np.ndarray) -> np.ndarray:
    """P(t) = integral of the ellipsoid density over the plane d . r = t (FOV units)."""
    a = np.asarray(ell.axes, dtype=np.float64)
    R = np.asarray(ell.rot, dtype=np.float64)
    sig = np.linalg.norm((d @ R) * a)
    tt = (t - d @ np.asarray(ell.center, dtype=np.float64)) / sig
    return np.where(np.abs(tt) <= 1.0, ell.density * np.pi * np.prod(a) / sig * (1.0 - tt ** 2), 0.0)


def gaussian_ft(omega: np.ndarray, center_vox, sigma: float, amplitude: float = 1.0) -> np.ndarray:
    """Continuous FT of amplitude exp(-|r - c|^2 / (2 sigma^2)) (voxel units) at
    omega rad/voxel: A (2 pi sigma^2)^{3/2} exp(-sigma^2 |omega|^2 / 2) exp(-i omega.c)."""
    c = np.asarray(center_vox, dtype=np.float64)
    w2 = np.sum(omega ** 2, axis=1)
    return amplitude * (2 * np.pi * sigma ** 2) ** 1.5 * np.exp(-0.5 * sigma ** 2 * w2) * \
        np.exp(-1j * (omega @ c))


def gaussian_plane_integral(d: np.ndarray, s: np.ndarray, center_vox, sigma: float,
                            amplitude: float = 1.0) -> np.ndarray:
    """Plane integral over d . r = s (voxel units): A 2 pi sigma^2 exp(-(s - d.c)^2 / (2 sigma^2))."""
    c = np.asarray(center_vox, dtype=np.float64)
    return amplitude * 2 * np.pi * sigma ** 2 * np.exp(-0.5 * (s - d @ c) ** 2 / sigma ** 2)


# -----------------------------------------------------------------------------
# per-point worst-case error bound of the interpolator
# -----------------------------------------------------------------------------
def minmax_error_1d(f, plan: OraclePlan, coeffs: Optional[np.ndarray] = None):
    """For one axis: b_n = exp(-i gamma u n), a_n = s(n) sum_j c_j exp(-i gamma (k0 + j) n).
    Returns (|b|^2, |a|^2, <a, b>) per f, with u = k0 + J/2 + f, taking k0 = 0
    (the quantities depend only on f)."""
    N, K, J, s = plan.N, plan.K, plan.J, plan.s
    f = np.atleast_1d(np.asarray(f, dtype=np.float64))
    c = plan.coeffs(f) if coeffs is None else coeffs
    n = centred_index(N)
    gam = 2.0 * np.pi / K
    u = J / 2.0 + f
    b = np.exp(-1j * gam * u[:, None] * n[None, :])                       # (P, N)
    j = np.arange(1, J + 1, dtype=np.float64)
    A = s[None, :, None] * np.exp(-1j * gam * j[None, None, :] * n[None, :, None])  # (1, N, J)
    a = np.einsum("pnj,pj->pn", np.broadcast_to(A, (f.size, N, J)), c)
    bb = np.sum(np.abs(b) ** 2, axis=1)
    aa = np.sum(np.abs(a) ** 2, axis=1)
    ab = np.sum(np.conj(a) * b, axis=1)
    return bb, aa, ab


def minmax_error_bound(u: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """E(omega) = || b3 - a3 ||_2 for the separable 3D interpolator at each point
    (P, 3): |X^ - X| <= ||x||_2 E(omega) (Cauchy-Schwarz)."""
    _, f = tap_base(u, plan.J)
    parts = [minmax_error_1d(f[:, a], plan) for a in range(3)]
    bb = np.prod([p[0] for p in parts], axis=0)
    aa = np.prod([p[1] for p in parts], axis=0)
    ab = np.prod([p[2] for p in parts], axis=0)
    e2 = bb + aa - 2.0 * ab.real
    return np.sqrt(np.maximum(e2, 0.0))


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
