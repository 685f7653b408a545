"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test fixes one part of the oracle against a brute-force definition, a
closed form, a quadrature, a library least-squares solve or an invariant, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  The paper prints no numeric values for
this step, so no golden value below comes from it; golden fixtures under
tests/golden/ are closed-form values written by tests/golden/make_golden.py.
"""
import json
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _plan(N, K=None, J=6, L=1024, dirs=None, M=None, **kw):
    K = K or 2 * N
    M = M or 2 * N
    if dirs is None:
        dirs = I.random_directions(24, 11)
    return O.OraclePlan(N, K, J, L, dirs, M, **kw)


# --------------------------------------------------------------------------
# P8: the library FFT against a brute DFT
# --------------------------------------------------------------------------
def test_fft_matches_brute_dft():
    K = 8
    rng = np.random.default_rng(0)
    g = rng.normal(size=(K, K, K)) + 1j * rng.normal(size=(K, K, K))
    k = np.arange(K)
    F = np.exp(-2j * np.pi * np.outer(k, k) / K)
    brute = np.einsum("az,by,cx,zyx->abc", F, F, F, g)
    assert np.allclose(O.grid_fft(g), brute, rtol=0, atol=1e-11)
    Finv = np.conj(F)
    brute_inv = np.einsum("az,by,cx,zyx->abc", Finv, Finv, Finv, g)
    assert np.allclose(O.grid_ifft_unnormalised(g), brute_inv, rtol=0, atol=1e-11)


# --------------------------------------------------------------------------
# scaling factors: Kaiser-Bessel Fourier transform against quadrature
# --------------------------------------------------------------------------
@pytest.mark.parametrize("J", [4, 6, 8])
def test_kb_fourier_transform_matches_quadrature(J):
    alpha = O.kb_alpha(J)
    for nu in [0.0, 0.05, 0.13, 0.25, 0.4]:
        f = lambda t: special.i0(alpha * np.sqrt(max(0.0, 1 - (2 * t / J) ** 2))) * np.cos(2 * np.pi * nu * t)
        val, _ = integrate.quad(f, -J / 2, J / 2, limit=200, epsabs=1e-12, epsrel=1e-12)
        assert O.kb_window_ft(nu, J) == pytest.approx(val, rel=1e-9)


def test_scaling_factors_shape_and_symmetry():
    """The pre-window is centred on the middle of the index range: n = -8..7
    mirrored about -1/2, smallest at the two central indices, where it equals
    Psi(0) / Psi(1/(2K)) computed by quadrature of the window itself."""
    N, K, J = 16, 32, 6
    s = O.scaling_factors(N, K, J)
    assert s.shape == (16,)
    assert np.allclose(s, s[::-1], rtol=1e-15)   # s(n) = s(-1 - n)
    assert s[7] == s[8] == s.min()               # n = -1 and n = 0
    alpha = O.kb_alpha(J)
    psi = lambda nu: integrate.quad(
        lambda t: special.i0(alpha * np.sqrt(max(0.0, 1 - (2 * t / J) ** 2))) * np.cos(2 * np.pi * nu * t),
        -J / 2, J / 2, limit=200, epsabs=1e-12, epsrel=1e-12)[0]
    assert s[8] == pytest.approx(psi(0.0) / psi(0.5 / K), rel=1e-9)
    assert s[0] == pytest.approx(psi(0.0) / psi(7.5 / K), rel=1e-9)   # n = -8
    assert np.all(s >= 1.0)
    # odd N: the range -7..7 is centred on 0
    so = O.scaling_factors(15, 32, 6)
    assert np.allclose(so, so[::-1], rtol=1e-15) and so[7] == pytest.approx(1.0)


@pytest.mark.parametrize("N,K,J", [(16, 32, 6), (32, 64, 6), (64, 128, 8), (16, 24, 4)])
def test_minmax_coeffs_are_a_phase_times_real_weights(N, K, J):
    """With the pre-window symmetric about the middle n_c = -1/2 of an even
    index range, T = D T~ D^H and r(f) = e^{i gamma (f + J/2 - j)/2} r~(f) with T~,
    r~ real, so c_j(f) = e^{i gamma (f + J/2 - j)/2} rho_j(f) with rho real: the
    identity the GPU's real-weight kernels rest on.  A pre-window centred on
    n = 0 instead breaks it (the imaginary part is then of order 1e-3)."""
    s = O.scaling_factors(N, K, J)
    gam = 2 * np.pi / K
    f = np.random.default_rng(3).uniform(0, 1, 200)
    c = O.minmax_coeffs_exact(f, N, K, J, s)
    j = np.arange(1, J + 1)
    rho = c * np.exp(-1j * gam * (f[:, None] + J / 2 - j[None, :]) / 2)
    assert np.max(np.abs(rho.imag)) < 1e-10 * np.max(np.abs(c))   # rounding of the J x J solve
    n = O.centred_index(N)
    s0 = O.kb_window_ft(0.0, J) / O.kb_window_ft(n / K, J)   # centred on n = 0
    c0 = O.minmax_coeffs_exact(f, N, K, J, s0)
    rho0 = c0 * np.exp(-1j * gam * (f[:, None] + J / 2 - j[None, :]) / 2)
    assert np.max(np.abs(rho0.imag)) > 1e-5 * np.max(np.abs(c0))


# --------------------------------------------------------------------------
# min-max coefficients: normal equations vs a least-squares solve of the
# explicit worst-case error ||b - A c|| (the definition of the interpolator)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,K,J", [(16, 32, 6), (32, 64, 6), (12, 24, 5), (16, 40, 4)])
def test_minmax_coeffs_are_least_squares_solution(N, K, J):
    s = O.scaling_factors(N, K, J)
    n = O.centred_index(N)
    gam = 2 * np.pi / K
    f = np.array([0.0, 0.1234, 0.5, 0.77, 0.999])
    c = O.minmax_coeffs_exact(f, N, K, J, s)
    for i, fi in enumerate(f):
        k0 = 3  # arbitrary: the coefficients do not depend on k0
        u = k0 + J / 2 + fi
        A = s[:, None] * np.exp(-1j * gam * (k0 + np.arange(1, J + 1))[None, :] * n[:, None])
        b = np.exp(-1j * gam * u * n)
        c_ls = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.allclose(c[i], c_ls, atol=1e-9 * max(1, np.abs(c_ls).max()))


def test_table_interpolation_gap_small():
    """P9: table (L = 1024) vs exact coefficients (reported, bounded)."""
    N, K, J, L = 32, 64, 6, 1024
    s = O.scaling_factors(N, K, J)
    tab = O.minmax_table(N, K, J, L, s)
    f = np.random.default_rng(1).uniform(0, 1, 500)
    ce = O.minmax_coeffs_exact(f, N, K, J, s)
    ct = O.coeffs_from_table(tab, f)
    assert np.max(np.abs(ce - ct)) < 5e-6
    # the table endpoints are the exact coefficients
    assert np.allclose(tab[0], O.minmax_coeffs_exact([0.0], N, K, J, s)[0])
    assert np.allclose(tab[-1], O.minmax_coeffs_exact([1.0], N, K, J, s)[0])


def test_tap_base_convention():
    k0, f = O.tap_base(np.array([0.0, 2.5, -0.25, 7.0 - 1e-12]), 6)
    assert list(k0) == [-3, -1, -4, 3]
    assert np.allclose(f, [0.0, 0.5, 0.75, 1.0 - 1e-12])
    k0, f = O.tap_base(np.array([0.0, 1.2]), 5)  # odd J: floor(u - 2.5)
    assert list(k0) == [-3, -2] and np.allclose(f, [0.5, 0.7])


# --------------------------------------------------------------------------
# P7: J = N interpolates exactly; per-point worst-case bound holds
# --------------------------------------------------------------------------
def test_minmax_exact_when_taps_cover_support():
    N, K = 8, 16
    dirs = I.random_directions(30, 2)
    pl = O.OraclePlan(N, K, N, 0, dirs, 2 * N)
    x = I.random_volume(N, 3)
    Xn = O.nufft_forward(x, pl, return_samples=True)
    Xe = O.forward_exact(x, pl, return_samples=True)
    assert O.rel_l2(Xn, Xe) < 1e-10


@pytest.mark.parametrize("L", [0, 1024])
def test_interpolation_error_within_minmax_bound(L):
    """P1 + P7: NUFFT vs brute NUDFT, every point inside ||x|| E(omega)."""
    N = 16
    dirs = I.random_directions(40, 5)
    pl = _plan(N, L=L, dirs=dirs)
    x = I.random_volume(N, 7, complex_values=True)
    Xn = O.nufft_forward(x, pl, return_samples=True).reshape(-1)
    Xe = O.forward_exact(x, pl, return_samples=True).reshape(-1)
    E = O.minmax_error_bound(pl.point_u().reshape(-1, 3), pl)
    bound = np.linalg.norm(x) * E
    assert np.all(np.abs(Xn - Xe) <= bound * (1 + 1e-9) + 1e-12)
    assert O.rel_l2(Xn, Xe) < 3e-5


def test_nufft_vs_nudft_tiny_workload():
    """P1 on the 32^3 ellipsoid workload (a subset of its lines)."""
    w = I.workload("tiny32")
    dirs = w.directions()
    pl = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
    x = w.volume(np.float64)
    lines = np.arange(0, dirs.shape[0], 17)
    Xn = O.nufft_forward(x, pl, lines=lines, return_samples=True)
    Xe = O.forward_exact(x, pl, lines=lines, return_samples=True)
    err = O.rel_l2(Xn, Xe)
    assert err < 2e-5, err


def test_mutation_off_by_one_tap_breaks_bound(monkeypatch):
    """A planted off-by-one in the oracle's tap base must fail the bound check."""
    N = 16
    pl = _plan(N, L=0, dirs=I.random_directions(12, 9))
    x = I.random_volume(N, 8)
    Xe = O.forward_exact(x, pl, return_samples=True).reshape(-1)
    E = O.minmax_error_bound(pl.point_u().reshape(-1, 3), pl)
    orig = O.tap_base

    def shifted(u, J):
        k0, f = orig(u, J)
        return k0 + 1, f

    monkeypatch.setattr(O, "tap_base", shifted)
    Xn = O.nufft_forward(x, pl, return_samples=True).reshape(-1)
    assert np.any(np.abs(Xn - Xe) > np.linalg.norm(x) * E * 10)


def test_mutation_reversed_taps_break_nudft_agreement():
    """A planted reversal of the tap order in the oracle's table must be caught."""
    N = 16
    pl = _plan(N, L=1024, dirs=I.random_directions(12, 9))
    pl.table = pl.table[:, ::-1].copy()
    x = I.random_volume(N, 8)
    Xn = O.nufft_forward(x, pl, return_samples=True)
    Xe = O.forward_exact(x, pl, return_samples=True)
    assert O.rel_l2(Xn, Xe) > 1e-2


# --------------------------------------------------------------------------
# P2: radial IDFT of exact samples == brute Dirichlet plane sums (Eqs. 2.6-2.7)
# --------------------------------------------------------------------------
def test_radial_idft_equals_dirichlet_plane_sums():
    N = 12
    M = 2 * N
    dirs = I.random_directions(10, 21)
    x = I.random_volume(N, 22)
    pl = O.OraclePlan(N, 2 * N, 6, 0, dirs, M)
    p_exact = O.forward_exact(x, pl)
    p_brute = O.dirichlet_plane_sums(x, dirs, M)
    assert np.max(np.abs(p_exact - p_brute)) < 1e-10 * np.abs(p_brute).max()


def test_dirichlet_kernel_closed_form_matches_sum():
    M = 16
    t = np.array([0.0, 0.3, 1.0, 2.7, -5.5, 16.0, 32.0, 7.999])
    q = np.arange(M) - M // 2
    direct = np.exp(-2j * np.pi * np.outer(t, q) / M).sum(axis=1) / M
    assert np.allclose(O.dirichlet_kernel(t, M), direct, atol=1e-12)


# --------------------------------------------------------------------------
# P3: Fourier-slice exactness for axis-aligned lines
# --------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["exact", "nufft"])
def test_axis_aligned_lines_give_slice_sums(which):
    N = 16
    M = 2 * N
    x = I.random_volume(N, 31)
    dirs = I.axis_directions()
    pl = O.OraclePlan(N, 2 * N, 6, 1024, dirs, M)
    p = O.forward_exact(x, pl) if which == "exact" else O.nufft_forward(x, pl)
    sums = [x.sum(axis=(0, 1)), x.sum(axis=(0, 2)), x.sum(axis=(1, 2))]  # over (z,y), (z,x), (y,x)
    tol = 1e-11 if which == "exact" else 3e-5
    for a in range(3):
        expect = np.zeros(M, dtype=np.complex128)
        expect[M // 2 - N // 2: M // 2 + N // 2] = sums[a]
        assert np.max(np.abs(p[a] - expect)) < tol * np.abs(expect).max(), a


# --------------------------------------------------------------------------
# P4: closed forms (Gaussian: tight; ellipsoids: loose)
# --------------------------------------------------------------------------
def test_gaussian_blob_fourier_samples_and_plane_integrals():
    N, sig = 48, 2.5
    c = (1.3, -0.7, 0.4)
    x = I.gaussian_blob_volume(N, c, sig)
    dirs = I.random_directions(6, 41)
    M = 2 * N
    pl = O.OraclePlan(N, 2 * N, 6, 0, dirs, M)
    om = pl.omegas()[None, :, None] * dirs[:, None, :]
    X = O.nudft_type2(x, om.reshape(-1, 3))
    Xc = O.gaussian_ft(om.reshape(-1, 3), c, sig)
    assert np.max(np.abs(X - Xc)) < 1e-10 * np.abs(Xc).max()
    p = O.radial_idft(X.reshape(dirs.shape[0], M), pl)
    s = np.arange(M) - M // 2
    for l in range(dirs.shape[0]):
        pc = O.gaussian_plane_integral(dirs[l], s, c, sig)
        assert np.max(np.abs(p[l] - pc)) < 1e-10 * pc.max()


def test_gaussian_blob_through_nufft_matches_plane_integral():
    N, sig = 32, 2.0
    c = (0.5, 0.25, -1.0)
    x = I.gaussian_blob_volume(N, c, sig)
    dirs = I.random_directions(8, 42)
    pl = O.OraclePlan(N, 2 * N, 6, 1024, dirs, 2 * N)
    p = O.nufft_forward(x, pl)
    s = np.arange(2 * N) - N
    pc = np.stack([O.gaussian_plane_integral(d, s, c, sig) for d in dirs])
    assert O.rel_l2(p, pc) < 1e-5


def test_ellipsoid_closed_forms_loose():
    """Voxelisation error is O(1/N): sanity agreement only.  The ellipsoids lie
    wholly inside the field of view (the closed forms do not truncate)."""
    N = 48
    ells = I.random_ellipsoids(4, 5, center_range=0.15, axes_range=(0.1, 0.3))
    x = I.ellipsoid_volume(N, ells, dtype=np.float64)
    dirs = I.random_directions(5, 6)
    M = 2 * N
    pl = O.OraclePlan(N, 2 * N, 6, 0, dirs, M)
    om = pl.omegas()[None, :, None] * dirs[:, None, :]
    X = O.nudft_type2(x, om.reshape(-1, 3))
    k = om.reshape(-1, 3) * N / (2 * np.pi)  # cycles per field of view
    Xc = (N ** 3) * sum(O.ellipsoid_ft(e, k) for e in ells)
    lowf = np.linalg.norm(om.reshape(-1, 3), axis=1) < np.pi / 4
    assert O.rel_l2(X[lowf], Xc[lowf]) < 0.05
    p = O.radial_idft(X.reshape(dirs.shape[0], M), pl).real
    s = np.arange(M) - M // 2
    pc = np.stack([(N ** 2) * sum(O.ellipsoid_plane_integral(e, d, s / N) for e in ells) for d in dirs])
    assert O.rel_l2(p, pc) < 0.05


# --------------------------------------------------------------------------
# P5: adjoint dot-product test
# --------------------------------------------------------------------------
@pytest.mark.parametrize("complex_volume", [False, True])
@pytest.mark.parametrize("L", [0, 1024])
def test_adjoint_dot_product(complex_volume, L):
    N = 12
    dirs = I.random_directions(15, 51)
    rng = np.random.default_rng(52)
    w = rng.normal(size=2 * N) + 1j * rng.normal(size=2 * N)
    pl = O.OraclePlan(N, 2 * N, 6, L, dirs, 2 * N, weight=w, complex_volume=complex_volume)
    x = I.random_volume(N, 53, complex_values=complex_volume)
    y = I.random_lines(dirs.shape[0], 2 * N, 54)
    Ax = O.nufft_forward(x, pl)
    Ahy = O.nufft_adjoint(y, pl)
    lhs = np.vdot(y, Ax)                       # <Ax, y> = y^H A x
    rhs = np.vdot(Ahy, x) if complex_volume else np.vdot(Ahy, x).real
    if not complex_volume:
        lhs = lhs.real                          # real-volume adjoint: Re <., .>
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < 1e-13


def test_radial_idft_adjoint_dot_product():
    pl = _plan(8, L=0, dirs=I.random_directions(5, 3), weight=np.arange(16) + 0.5j)
    a = I.random_lines(5, 16, 1)
    b = I.random_lines(5, 16, 2)
    assert np.vdot(b, O.radial_idft(a, pl)) == pytest.approx(np.vdot(O.radial_idft_adjoint(b, pl), a), rel=1e-13)


# --------------------------------------------------------------------------
# P6: invariants
# --------------------------------------------------------------------------
def test_hermitian_symmetry_dc_linearity_shift():
    N = 16
    M = 2 * N
    dirs = I.random_directions(10, 61)
    pl = O.OraclePlan(N, 2 * N, 6, 1024, dirs, M)
    x = I.random_volume(N, 62)
    X = O.forward_exact(x, pl, return_samples=True)
    Xn = O.nufft_forward(x, pl, return_samples=True)
    # Hermitian symmetry: X(-omega) = conj X(omega), q -> -q, q != -M/2
    q = np.arange(1, M // 2)
    assert np.allclose(X[:, M // 2 - q], np.conj(X[:, M // 2 + q]), atol=1e-10)
    assert np.max(np.abs(Xn[:, M // 2 - q] - np.conj(Xn[:, M // 2 + q]))) < 1e-4 * np.abs(Xn).max()
    # DC: q = 0 column equals sum x
    assert np.allclose(X[:, M // 2], x.sum(), atol=1e-9)
    assert np.allclose(Xn[:, M // 2], x.sum(), rtol=0, atol=1e-5 * np.linalg.norm(x))
    # linearity
    x2 = I.random_volume(N, 63)
    a, b = 0.7, -1.9
    lhs = O.nufft_forward(a * x + b * x2, pl)
    rhs = a * O.nufft_forward(x, pl) + b * O.nufft_forward(x2, pl)
    assert np.allclose(lhs, rhs, atol=1e-10 * np.abs(rhs).max())
    # integer shift of a compactly supported volume: X_shift = e^{-i omega.delta} X
    xs = np.zeros_like(x)
    inner = x[4:12, 4:12, 4:12]
    xc = np.zeros_like(x)
    xc[4:12, 4:12, 4:12] = inner
    delta = (2, -1, 3)  # (dx, dy, dz) voxels
    xs[4 + delta[2]:12 + delta[2], 4 + delta[1]:12 + delta[1], 4 + delta[0]:12 + delta[0]] = inner
    om = pl.omegas()[None, :, None] * dirs[:, None, :]
    ph = np.exp(-1j * (om @ np.array(delta, dtype=np.float64)))
    Xc = O.forward_exact(xc, pl, return_samples=True)
    Xs = O.forward_exact(xs, pl, return_samples=True)
    assert np.allclose(Xs, ph * Xc, atol=1e-9)
    Xcn = O.nufft_forward(xc, pl, return_samples=True)
    Xsn = O.nufft_forward(xs, pl, return_samples=True)
    assert O.rel_l2(Xsn, ph * Xcn) < 3e-5


# --------------------------------------------------------------------------
# golden fixtures: closed-form values stored with their citation
# --------------------------------------------------------------------------
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_gaussian_plane_integrals():
    with open(os.path.join(GOLDEN, "gaussian_plane_integrals.json")) as fh:
        g = json.load(fh)
    x = I.gaussian_blob_volume(g["n"], g["center_vox"], g["sigma_vox"])
    dirs = np.array(g["dirs"], dtype=np.float64)
    pl = O.OraclePlan(g["n"], 2 * g["n"], 6, 1024, dirs, g["m"])
    p = O.nufft_forward(x, pl).real
    expect = np.array(g["plane_integrals"])
    assert O.rel_l2(p, expect) < 1e-5
