"""The x passes of a real volume transform two rows at once (fft_passes.cu,
k_row_fwd_real and k_row_adj_real).  These CPU checks pin the identities they
rest on against NumPy's FFT, with the exact component expressions the kernels
evaluate:
  forward: Z = FFT(a + i b);  FFT(a) = (Z[k] + conj Z[-k]) / 2,
           FFT(b) = (Z[k] - conj Z[-k]) / 2i;
  inverse: Re IFFT(a) = IFFT(H a) with (H a)[k] = (a[k] + conj a[-k]) / 2, so
           IFFT(H a + i H b) = Re IFFT(a) + i Re IFFT(b)."""
import numpy as np
import pytest


@pytest.mark.parametrize("K", [16, 48, 512])
def test_forward_two_real_rows(K):
    rng = np.random.default_rng(K)
    a, b = rng.normal(size=K), rng.normal(size=K)
    Z = np.fft.fft(a + 1j * b)
    Zm = Z[(-np.arange(K)) % K]
    # the kernel's components: A = (0.5 (z.x + zm.x), 0.5 (z.y - zm.y)), B = (0.5 (z.y + zm.y), 0.5 (zm.x - z.x))
    A = 0.5 * (Z.real + Zm.real) + 1j * 0.5 * (Z.imag - Zm.imag)
    B = 0.5 * (Z.imag + Zm.imag) + 1j * 0.5 * (Zm.real - Z.real)
    assert np.allclose(A, np.fft.fft(a), atol=1e-10)
    assert np.allclose(B, np.fft.fft(b), atol=1e-10)


@pytest.mark.parametrize("K", [16, 48, 512])
def test_inverse_two_rows_real_parts(K):
    rng = np.random.default_rng(K + 1)
    a = rng.normal(size=K) + 1j * rng.normal(size=K)
    b = rng.normal(size=K) + 1j * rng.normal(size=K)
    j = np.arange(K)
    am, bm = a[(-j) % K], b[(-j) % K]
    ha = 0.5 * (a.real + am.real) + 1j * 0.5 * (a.imag - am.imag)
    hb = 0.5 * (b.real + bm.real) + 1j * 0.5 * (b.imag - bm.imag)
    # the kernel writes Z[j] = (ha.x - hb.y, ha.y + hb.x) and Z[-j] = (ha.x + hb.y, hb.x - ha.y)
    Z = np.empty(K, complex)
    Z[j] = (ha.real - hb.imag) + 1j * (ha.imag + hb.real)
    Zneg = (ha.real + hb.imag) + 1j * (hb.real - ha.imag)
    assert np.allclose(Z[(-j) % K], Zneg, atol=1e-12)      # the two writes agree
    out = np.fft.ifft(Z)
    assert np.allclose(out.real, np.fft.ifft(a).real, atol=1e-12)
    assert np.allclose(out.imag, np.fft.ifft(b).real, atol=1e-12)
