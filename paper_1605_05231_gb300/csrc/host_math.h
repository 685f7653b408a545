// Host-side FP64 helpers shared by the plans: the Kaiser-Bessel window's
// Fourier transform (the pre-window P of Eq. 2.11), a small complex matrix
// inverse (the min-max system T of the interpolator) and the Chebyshev fit of
// the min-max coefficients c_j(f) that the exact-coefficient kernels evaluate.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace nufft {

// Fourier transform of the Kaiser-Bessel window of width J, shape alpha,
// at nu cycles per grid sample: J sinh(z) / z, z = sqrt(alpha^2 - (pi J nu)^2).
inline double kb_ft(double nu, int J, double alpha) {
  const double z2 = alpha * alpha - (M_PI * J * nu) * (M_PI * J * nu);
  if (z2 > 0) {
    const double z = std::sqrt(z2);
    return J * std::sinh(z) / z;
  }
  const double z = std::sqrt(-z2);
  return z > 0 ? J * std::sin(z) / z : (double)J;
}

// in-place inverse of a complex n x n matrix (Gauss-Jordan, partial pivoting)
inline bool invert(std::vector<std::complex<double>>& a, int n) {
  std::vector<std::complex<double>> inv(n * n, std::complex<double>(0, 0));
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::abs(a[r * n + c]) > std::abs(a[piv * n + c])) piv = r;
    if (std::abs(a[piv * n + c]) == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    const std::complex<double> d = a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] /= d;
      inv[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const std::complex<double> f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// Degree-kPolyDeg Chebyshev interpolant of each c_j on f in [0, 1] (nodes
// t_i = cos(pi (i + 1/2) / (D + 1)), f = (t + 1) / 2), converted to monomials in
// t and rounded to FP32.  The FP32 coefficients are then checked against the
// exact c on 1025 evenly spaced f; the largest error relative to max |c| is
// kept for plan_info, and a fit above 1e-7 is refused.
template <class F>
double fit_coeff_polys(int J, F&& coeffs_at, nufft::CoefPoly& out) {
  constexpr int D = nufft::kPolyDeg, n = D + 1;
  std::vector<std::complex<double>> cv((size_t)n * J);
  for (int i = 0; i < n; ++i) {
    const double t = std::cos(M_PI * (i + 0.5) / n);
    coeffs_at(0.5 * (t + 1.0), cv.data() + (size_t)i * J);
  }
  // Chebyshev coefficients b_k = (2 - [k = 0]) / n sum_i c(t_i) T_k(t_i)
  std::vector<std::complex<double>> b((size_t)n * J, std::complex<double>(0, 0));
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < n; ++i) {
      const double tk = std::cos(M_PI * k * (i + 0.5) / n);
      for (int j = 0; j < J; ++j) b[(size_t)k * J + j] += cv[(size_t)i * J + j] * tk;
    }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < J; ++j) b[(size_t)k * J + j] *= (k == 0 ? 1.0 : 2.0) / n;
  // monomial coefficients of T_k: T_0 = 1, T_1 = t, T_k = 2 t T_{k-1} - T_{k-2}
  std::vector<double> Tm((size_t)n * n, 0.0);
  Tm[0] = 1.0;
  if (n > 1) Tm[(size_t)n + 1] = 1.0;
  for (int k = 2; k < n; ++k)
    for (int q = 0; q < n; ++q)
      Tm[(size_t)k * n + q] = (q > 0 ? 2.0 * Tm[(size_t)(k - 1) * n + q - 1] : 0.0) - Tm[(size_t)(k - 2) * n + q];
  out = nufft::CoefPoly{};
  for (int j = 0; j < J; ++j)
    for (int q = 0; q < n; ++q) {
      std::complex<double> m = 0;
      for (int k = q; k < n; ++k) m += b[(size_t)k * J + j] * Tm[(size_t)k * n + q];
      out.a[j][0][q] = (float)m.real();
      out.a[j][1][q] = (float)m.imag();
    }
  double err = 0.0, cmax = 0.0;
  std::vector<std::complex<double>> ce(J);
  for (int i = 0; i <= 1024; ++i) {
    const double f = i / 1024.0, t = 2.0 * f - 1.0;
    coeffs_at(f, ce.data());
    for (int j = 0; j < J; ++j) {
      double re = out.a[j][0][D], im = out.a[j][1][D];
      for (int q = D - 1; q >= 0; --q) {
        re = re * t + out.a[j][0][q];
        im = im * t + out.a[j][1][q];
      }
      err = std::max(err, std::abs(std::complex<double>(re, im) - ce[j]));
      cmax = std::max(cmax, std::abs(ce[j]));
    }
  }
  return err / cmax;
}

}  // namespace nufft
