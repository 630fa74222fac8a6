// Host-side Daubechies filters for the SARA dictionary (App. B): the low-pass filter of the
// orthonormal Daubechies wavelet with N vanishing moments by spectral factorisation of
// |m0(w)|^2 = cos^(2N)(w/2) P_N(sin^2(w/2)), P_N(y) = sum_{k<N} C(N-1+k, k) y^k: the roots of
// z^(N-1) P_N((2 - z - 1/z) / 4) by Durand-Kerner iteration with a Newton polish, the N - 1 roots
// inside the unit circle (minimum phase) times (1 + z)^N, normalised to sum sqrt(2); coefficients
// are listed from the highest power of z down.  Header-only so that a host test can compile it.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace pnp {
namespace daub {

using cd = std::complex<double>;

inline std::vector<double> polymul(const std::vector<double>& a, const std::vector<double>& b) {
  std::vector<double> r(a.size() + b.size() - 1, 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
  return r;
}

inline cd polyval(const std::vector<double>& c, cd z) {  // highest power first
  cd v = 0.0;
  for (double a : c) v = v * z + a;
  return v;
}

// low-pass filter of the orthonormal Daubechies wavelet with N vanishing moments (length 2N)
inline std::vector<double> daubechies(int N) {
  if (N == 1) return {1.0 / std::sqrt(2.0), 1.0 / std::sqrt(2.0)};
  const std::vector<double> yz = {-0.25, 0.5, -0.25};  // y z with y = (2 - z - 1/z) / 4
  std::vector<double> Q(2 * N - 1, 0.0);
  for (int k = 0; k < N; ++k) {
    std::vector<double> term = {1.0};
    for (int i = 0; i < k; ++i) term = polymul(term, yz);
    term.resize(term.size() + (N - 1 - k), 0.0);  // times z^(N-1-k)
    double binom = 1.0;                          // C(N-1+k, k)
    for (int i = 1; i <= k; ++i) binom = binom * (N - 1 + i) / i;
    const size_t off = Q.size() - term.size();
    for (size_t i = 0; i < term.size(); ++i) Q[off + i] += binom * term[i];
  }
  const int d = (int)Q.size() - 1;
  std::vector<double> a(Q);
  for (double& v : a) v /= Q[0];
  std::vector<cd> r(d);
  for (int i = 0; i < d; ++i) r[i] = std::pow(cd(0.4, 0.9), i);
  for (int it = 0; it < 2000; ++it) {  // Durand-Kerner
    double step = 0.0;
    for (int i = 0; i < d; ++i) {
      cd den = 1.0;
      for (int j = 0; j < d; ++j)
        if (j != i) den *= r[i] - r[j];
      const cd dz = polyval(a, r[i]) / den;
      r[i] -= dz;
      step = std::max(step, std::abs(dz));
    }
    if (step < 1e-15) break;
  }
  std::vector<double> da(d);  // derivative, for the Newton polish
  for (int i = 0; i < d; ++i) da[i] = a[i] * (d - i);
  for (int it = 0; it < 3; ++it)
    for (cd& z : r) z -= polyval(a, z) / polyval(da, z);
  std::vector<cd> L = {1.0};
  for (const cd& z : r)
    if (std::abs(z) < 1.0) {
      std::vector<cd> nl(L.size() + 1, 0.0);
      for (size_t i = 0; i < L.size(); ++i) {
        nl[i] += L[i];
        nl[i + 1] -= L[i] * z;
      }
      L.swap(nl);
    }
  std::vector<double> h(L.size());
  for (size_t i = 0; i < L.size(); ++i) h[i] = L[i].real();
  for (int i = 0; i < N; ++i) h = polymul(h, {1.0, 1.0});
  double s = 0.0;
  for (double v : h) s += v;
  for (double& v : h) v *= std::sqrt(2.0) / s;
  return h;
}

}  // namespace daub
}  // namespace pnp
