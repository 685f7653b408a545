"""Per-view reverse Grangeat step (Sec. 2.2.2, Fig. 2.15; C3a-C3d of Sec. 2.4).

CPU pins of the oracle (oracle/reverse_grangeat.py):
- the radial DFT of a delta is the closed-form phasor, and the post-weights
  scale the samples before it;
- the 2D Fourier slice theorem: the radial DFT of the column sums (alpha = 0)
  and row sums (alpha = pi/2) of an image equals its 2D DFT along the line;
- the exact adjoint NUDFT equals the transpose of the 2D DFT computed by
  np.fft.fft2 at on-grid frequencies;
- the fast 2D NUFFT forward / adjoint satisfy the adjoint identity, and the
  fast forward stays within the min-max bound of the exact type-2 sum;
- the fast adjoint stays within the per-pixel bound of the exact adjoint,
  for the whole C3a-C3d chain over several views;
- planted mistakes (sine and cosine swapped, the DFT sign flipped) fail.
"""
import numpy as np
import pytest

from oracle import reverse_grangeat as G


def _angles(L):
    return np.pi * (np.arange(L) + 0.5) / L


def test_radial_dft_of_a_delta_and_post_weights():
    M = 24
    L = 3
    y = np.zeros((L, M))
    w = np.full((L, M), 2.5)
    t0 = [0, 7, 23]
    for l, t in enumerate(t0):
        y[l, t] = 1.0
    Y = G.line_spectra(y, w)
    q = np.arange(M) - M // 2
    for l, t in enumerate(t0):
        want = 2.5 * np.exp(-2j * np.pi * q * (t - M // 2) / M)
        np.testing.assert_allclose(Y[l], want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,M", [(8, 16), (12, 12), (10, 32)])
def test_fourier_slice_theorem_axis_aligned(N, M):
    rng = np.random.default_rng(1)
    f = rng.normal(size=(N, N))
    n = np.arange(N) - N // 2
    # offsets s = t - M/2 cover the centred box: t = n + M/2
    R = np.zeros((2, M))
    R[0, n + M // 2] = f.sum(axis=0)   # alpha = 0: lines x = s, column sums
    R[1, n + M // 2] = f.sum(axis=1)   # alpha = pi/2: lines y = s, row sums
    Y = G.line_spectra(R, np.ones_like(R))
    rho = (np.arange(M) - M // 2) / M
    # the 2D DFT (e^{-i}) of f on the two lines
    Fx = np.exp(-2j * np.pi * np.outer(rho, n)) @ f.sum(axis=0)
    Fy = np.exp(-2j * np.pi * np.outer(rho, n)) @ f.sum(axis=1)
    np.testing.assert_allclose(Y[0], Fx, rtol=0, atol=1e-10)
    np.testing.assert_allclose(Y[1], Fy, rtol=0, atol=1e-10)
    # and the full 2D DFT through the library routine, at on-grid rho = k/N
    F = np.fft.fft2(np.fft.ifftshift(f))         # index k <-> frequency k/N
    if M % N == 0:
        k = (np.arange(M) - M // 2) * N // M
        on = ((np.arange(M) - M // 2) * N) % M == 0
        np.testing.assert_allclose(Y[0][on], F[0, k[on] % N], rtol=0, atol=1e-10)
        np.testing.assert_allclose(Y[1][on], F[k[on] % N, 0], rtol=0, atol=1e-10)


def test_exact_adjoint_is_transpose_of_fft2():
    # angles 0 and pi/2 with M = N put every sample on the N-point DFT grid
    N = 8
    M = N
    ang = np.array([0.0, np.pi / 2])
    rng = np.random.default_rng(2)
    Y = rng.normal(size=(2, M)) + 1j * rng.normal(size=(2, M))
    x = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    z = G.adjoint_nudft_2d(Y, ang, N)
    F = np.fft.fft2(np.fft.ifftshift(x))
    k = np.arange(M) - M // 2
    Ax = np.concatenate([F[0, k % N], F[k % N, 0]])   # (A x)_p = sum_n x[n] e^{-i omega_p . n}
    np.testing.assert_allclose(np.vdot(Y.ravel(), Ax), np.vdot(z, x), rtol=1e-12)


@pytest.mark.parametrize("N,J", [(12, 5), (16, 5), (16, 4)])
def test_fast_forward_adjoint_identity_and_bound(N, J):
    rng = np.random.default_rng(3)
    L, M = 7, 2 * N
    nu = G.Nufft2D(N, J)
    u = G.polar_u(_angles(L), M, 2 * N)
    x = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    Yp = rng.normal(size=L * M) + 1j * rng.normal(size=L * M)
    fx = nu.forward(x, u)
    np.testing.assert_allclose(np.vdot(Yp, fx), np.vdot(nu.adjoint(Yp, u), x), rtol=1e-12)
    # the fast forward against the exact type-2 sum, within ||x|| E_p
    n = np.arange(N) - N // 2
    w = 2 * np.pi * u / (2 * N)
    exact = np.einsum("pa,pb,ab->p", np.exp(-1j * np.outer(w[:, 1], n)), np.exp(-1j * np.outer(w[:, 0], n)), x)
    assert np.all(np.abs(fx - exact) <= np.linalg.norm(x) * nu.error_bound(u) * (1 + 1e-6) + 1e-12)


def test_chain_fast_within_pixel_bound():
    rng = np.random.default_rng(4)
    N, L, M, V = 16, 10, 32, 3
    ang = _angles(L)
    y = rng.normal(size=(V, L, M))
    wpost = rng.uniform(0.5, 1.5, (V, L, M))
    wpre = rng.uniform(0.5, 1.5, (V, N, N))
    fast = G.reverse_grangeat(y, wpost, wpre, ang, N)
    exact = G.reverse_grangeat(y, wpost, wpre, ang, N, exact=True)
    for v in range(V):
        Y = G.line_spectra(y[v], wpost[v])
        bound = G.pixel_error_bound(Y, ang, N) * wpre[v].max()
        assert np.max(np.abs(fast[v] - exact[v])) <= bound
    # J = 5 with twofold oversampling: about 1e-4 relative at most
    assert np.linalg.norm(fast - exact) / np.linalg.norm(exact) < 3e-4


def test_planted_swapped_axes_fails(monkeypatch):
    rng = np.random.default_rng(5)
    N, L, M = 12, 9, 24
    ang = _angles(L) * 0.7 + 0.1
    y = rng.normal(size=(1, L, M))
    ones = np.ones((1, L, M))
    wpre = np.ones((1, N, N))
    exact = G.reverse_grangeat(y, ones, wpre, ang, N, exact=True)
    real_u = G.polar_u
    monkeypatch.setattr(G, "polar_u", lambda a, M, K: real_u(a, M, K)[:, ::-1].copy())
    fast = G.reverse_grangeat(y, ones, wpre, ang, N)
    monkeypatch.undo()
    assert np.linalg.norm(fast - exact) / np.linalg.norm(exact) > 1e-2


def test_planted_dft_sign_fails(monkeypatch):
    N, M = 8, 16
    rng = np.random.default_rng(6)
    f = rng.normal(size=(N, N))
    n = np.arange(N) - N // 2
    R = np.zeros((1, M))
    R[0, n + M // 2] = f.sum(axis=0)
    real = G.line_spectra
    monkeypatch.setattr(G, "line_spectra", lambda y, w: np.conj(real(np.conj(y), w)))
    Y = G.line_spectra(R + 0j, np.ones_like(R))
    monkeypatch.undo()
    rho = (np.arange(M) - M // 2) / M
    Fx = np.exp(-2j * np.pi * np.outer(rho, n)) @ f.sum(axis=0)
    assert np.max(np.abs(Y[0] - Fx)) > 1e-3


# ---- the library --------------------------------------------------------------

def test_library_refuses_bad_plans():
    import ctypes

    from paper_1605_05231_gb300 import binding

    lib = binding.load_library()
    h = ctypes.c_void_p()
    a = (ctypes.c_double * 4)(0.1, 0.2, 0.3, 0.4)
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 24, 4, 32, 5, a, 8) == -4     # N not supported
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 16, 4, 48, 5, a, 8) == -4     # M not supported
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 16, 4, 32, 9, a, 8) == -1     # J
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 16, 4, 32, 5, None, 8) == -1  # angles
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 16, 4, 32, 5, a, 0) == -1     # views
    nan = (ctypes.c_double * 1)(float("nan"))
    assert lib.nufft3d_grangeat_create(ctypes.byref(h), 16, 1, 32, 5, nan, 8) == -1
    assert lib.nufft3d_grangeat_destroy(None) == -1


# ---- GPU parity against the oracle ---------------------------------------------
# FP32 with coefficients fitted to 1e-7 against the oracle's FP64 steps with
# exact coefficients: rel-L2 <= 1e-5 per view.

def _gpu_run(cuda_lib, N, ang, M, J, y, wpost, wpre, max_views=64):
    import torch

    g = cuda_lib.ReverseGrangeat(N, ang, M, J=J, max_views=max_views)
    out = g.run(torch.from_numpy(y.astype(np.complex64)).cuda(), torch.from_numpy(wpost.astype(np.float32)).cuda(),
                torch.from_numpy(wpre.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    info = g.info()
    g.close()
    return out.cpu().numpy().astype(np.complex128), info


@pytest.mark.gpu
@pytest.mark.parametrize("N,L,M,J,V,chunk", [(16, 10, 32, 5, 3, 64), (32, 24, 64, 5, 19, 8), (16, 7, 16, 4, 5, 2),
                                             (64, 40, 128, 6, 17, 16), (32, 64, 64, 5, 33, 33)])
def test_gpu_matches_oracle(cuda_lib, N, L, M, J, V, chunk):
    rng = np.random.default_rng(N + L + V)
    ang = np.sort(rng.uniform(0, np.pi, L))
    y = rng.normal(size=(V, L, M)) + 1j * rng.normal(size=(V, L, M))
    wpost = rng.uniform(0.5, 1.5, (V, L, M))
    wpre = rng.uniform(0.5, 1.5, (V, N, N))
    got, info = _gpu_run(cuda_lib, N, ang, M, J, y, wpost, wpre, max_views=chunk)
    assert info["nnz"] == L * M * J * J and info["fit_error"] < 1e-7
    want = G.reverse_grangeat(y.astype(np.complex64).astype(np.complex128), wpost.astype(np.float32).astype(np.float64),
                              wpre.astype(np.float32).astype(np.float64), ang, N, J=J)
    for v in range(V):
        rel = np.linalg.norm(got[v] - want[v]) / np.linalg.norm(want[v])
        assert rel < 1e-5, (v, rel)


@pytest.mark.gpu
def test_gpu_full_size_views_sampled(cuda_lib):
    """The configuration bench.py times: 256 views of 128 x 128, L = M = 256,
    [5 5] taps, all views in one chunk (max_views = 256); two of the views
    (views are independent) against the oracle at rel-L2 <= 1e-5."""
    N, V, L, M, J = 128, 256, 256, 256, 5
    ang = np.pi * (np.arange(L) + 0.5) / L
    rng = np.random.default_rng(70)
    y = (rng.normal(size=(V, L, M)) + 1j * rng.normal(size=(V, L, M))).astype(np.complex64)
    wpost = rng.uniform(0.5, 1.5, (V, L, M)).astype(np.float32)
    wpre = rng.uniform(0.5, 1.5, (V, N, N)).astype(np.float32)
    got, info = _gpu_run(cuda_lib, N, ang, M, J, y, wpost, wpre, max_views=V)
    assert info["nnz"] == L * M * J * J
    sel = [0, 137]
    want = G.reverse_grangeat(y[sel].astype(np.complex128), wpost[sel].astype(np.float64),
                              wpre[sel].astype(np.float64), ang, N, J=J)
    for i, v in enumerate(sel):
        rel = np.linalg.norm(got[v] - want[i]) / np.linalg.norm(want[i])
        assert rel < 1e-5, (v, rel)


@pytest.mark.gpu
def test_gpu_axis_aligned_fourier_slice(cuda_lib):
    """Column and row sums of a detector image as the two lines of a view:
    the GPU chain equals the oracle's, whose C3b is pinned to the 2D DFT."""
    N, M = 32, 64
    rng = np.random.default_rng(40)
    f = rng.normal(size=(2, N, N))
    n = np.arange(N) - N // 2
    y = np.zeros((2, 2, M), dtype=np.complex128)
    for v in range(2):
        y[v, 0, n + M // 2] = f[v].sum(axis=0)
        y[v, 1, n + M // 2] = f[v].sum(axis=1)
    ang = np.array([0.0, np.pi / 2])
    ones_l = np.ones((2, 2, M))
    ones_n = np.ones((2, N, N))
    got, _ = _gpu_run(cuda_lib, N, ang, M, 6, y, ones_l, ones_n)
    want = G.reverse_grangeat(y, ones_l, ones_n, ang, N, J=6)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5


@pytest.mark.gpu
def test_gpu_zero_views_and_argument_checks(cuda_lib):
    import torch

    g = cuda_lib.ReverseGrangeat(16, np.linspace(0, 3, 5), 32, J=5, max_views=4)
    z = torch.zeros((0, 5, 32), dtype=torch.complex64, device="cuda")
    out = g.run(z, torch.zeros((0, 5, 32), device="cuda"), torch.zeros((0, 16, 16), device="cuda"))
    assert out.shape == (0, 16, 16)
    with pytest.raises(ValueError):
        g.run(torch.zeros((1, 5, 31), dtype=torch.complex64, device="cuda"), torch.zeros((1, 5, 31), device="cuda"),
              torch.zeros((1, 16, 16), device="cuda"))
    g.close()
