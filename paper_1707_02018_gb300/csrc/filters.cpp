// Filter-bank derivation for the device path (host C++, float64).
//
// Sec. I-B / I-C of the paper name the wavelets (Haar, Daubechies, CDF 9/7)
// but print no taps.  The taps are derived here from the Daubechies halfband
// polynomial P_p(y) = sum_{k<p} C(p-1+k, k) y^k, y = sin^2(w/2):
//  * Daubechies (orthogonal, p vanishing moments): all roots of P_p via the
//    Weierstrass (Durand-Kerner) iteration; each root y gives the z-root of
//    z^2 - (2 - 4y) z + 1 inside the unit circle (minimum phase); the scaling
//    filter is (1 + w)^p prod (1 - z_i w), w = z^-1, scaled to sum sqrt(2).
//  * CDF 9/7 (biorthogonal): P_4 = 1 + 4y + 10y^2 + 20y^3; its real root
//    (Newton's method) goes to the 7-tap synthesis lowpass, the complex pair
//    (the deflated quadratic) to the 9-tap analysis lowpass; both also carry
//    cos^4(w/2).  Placed at taps 1..9 / 1..7 of a length-10 array, which gives
//    perfect reconstruction with delay L' = 9.
// Highpass by modulation: rec_hi[k] = (-1)^k dec_lo[k],
// dec_hi[k] = (-1)^(k+1) rec_lo[k].  Orthogonal: dec_lo = reversed rec_lo.
#include <cmath>
#include <complex>
#include <vector>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

using cd = std::complex<double>;

double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Roots of sum_k c[k] y^k (c ascending, c.back() != 0) by Durand-Kerner.
std::vector<cd> poly_roots(const std::vector<double>& c) {
  const int deg = static_cast<int>(c.size()) - 1;
  std::vector<cd> z(deg);
  const cd seed(0.4, 0.9);
  for (int i = 0; i < deg; ++i) z[i] = std::pow(seed, i);
  auto eval = [&](cd y) {
    cd acc = 0.0;
    for (int k = deg; k >= 0; --k) acc = acc * y + c[k];
    return acc / c[deg];
  };
  for (int it = 0; it < 500; ++it) {
    double moved = 0.0;
    for (int i = 0; i < deg; ++i) {
      cd den = 1.0;
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (z[i] - z[j]);
      cd step = eval(z[i]) / den;
      z[i] -= step;
      moved = std::max(moved, std::abs(step));
    }
    if (moved < 1e-16) break;
  }
  // polish each root with Newton steps on the full polynomial
  for (auto& y : z) {
    for (int it = 0; it < 5; ++it) {
      cd p = 0.0, dp = 0.0;
      for (int k = deg; k >= 0; --k) {
        dp = dp * y + p;
        p = p * y + c[k];
      }
      if (std::abs(dp) == 0.0) break;
      y -= p / dp;
    }
  }
  return z;
}

cd inside_root(cd y) {
  cd b = 2.0 - 4.0 * y;
  cd d = std::sqrt(b * b - 4.0);
  cd z1 = 0.5 * (b + d), z2 = 0.5 * (b - d);
  return std::abs(z1) < std::abs(z2) ? z1 : z2;
}

std::vector<cd> pmul(const std::vector<cd>& a, const std::vector<cd>& b) {
  std::vector<cd> r(a.size() + b.size() - 1, 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
  return r;
}

std::vector<double> halfband(int p) {
  std::vector<double> c(p);
  for (int k = 0; k < p; ++k) c[k] = binom(p - 1 + k, k);
  return c;
}

std::vector<double> daubechies(int p) {
  std::vector<cd> h{1.0};
  for (int i = 0; i < p; ++i) h = pmul(h, {1.0, 1.0});
  if (p > 1) {
    for (cd y : poly_roots(halfband(p))) h = pmul(h, {1.0, -inside_root(y)});
  }
  std::vector<double> out(h.size());
  double sum = 0.0;
  for (size_t i = 0; i < h.size(); ++i) sum += (out[i] = h[i].real());
  for (double& v : out) v *= std::sqrt(2.0) / sum;
  return out;
}

// symmetric Laurent factor (1 - y/root), y = (2 - z - 1/z)/4, as 3 taps
std::vector<cd> y_factor(cd root) { return {0.25 / root, 1.0 - 0.5 / root, 0.25 / root}; }

void cdf97(std::vector<double>* ana9, std::vector<double>* syn7) {
  // real root of 20y^3 + 10y^2 + 4y + 1 by Newton from y = -0.3
  double y = -0.3;
  for (int it = 0; it < 100; ++it) {
    double f = ((20.0 * y + 10.0) * y + 4.0) * y + 1.0;
    double df = (60.0 * y + 20.0) * y + 4.0;
    double step = f / df;
    y -= step;
    if (std::fabs(step) < 1e-17) break;
  }
  // deflate: 20y^3+10y^2+4y+1 = (y - yr)(a y^2 + b y + c)
  const double a = 20.0, b = 10.0 + a * y, c = 4.0 + b * y;
  cd disc = std::sqrt(cd(b * b - 4.0 * a * c));
  cd yc = (-b + disc) / (2.0 * a);
  std::vector<cd> cos2{0.25, 0.5, 0.25};
  std::vector<cd> c4 = pmul(cos2, cos2);
  std::vector<cd> s7 = pmul(c4, y_factor(cd(y)));
  std::vector<cd> a9 = pmul(c4, pmul(y_factor(yc), y_factor(std::conj(yc))));
  auto finish = [](const std::vector<cd>& v, std::vector<double>* out) {
    out->resize(v.size());
    double sum = 0.0;
    for (size_t i = 0; i < v.size(); ++i) sum += ((*out)[i] = v[i].real());
    for (double& t : *out) t *= std::sqrt(2.0) / sum;
  };
  finish(a9, ana9);
  finish(s7, syn7);
}

}  // namespace

bool make_filter_bank(int wavelet, FilterBank* fb) {
  *fb = FilterBank();
  std::vector<double> dec_lo, rec_lo;
  switch (wavelet) {
    case ADJWT_HAAR:
    case ADJWT_DB2:
    case ADJWT_DB4: {
      const int p = wavelet == ADJWT_HAAR ? 1 : (wavelet == ADJWT_DB2 ? 2 : 4);
      rec_lo = daubechies(p);
      dec_lo.assign(rec_lo.rbegin(), rec_lo.rend());
      fb->L = 2 * p;
      break;
    }
    case ADJWT_CDF97: {
      std::vector<double> a9, s7;
      cdf97(&a9, &s7);
      fb->L = 10;
      dec_lo.assign(10, 0.0);
      rec_lo.assign(10, 0.0);
      for (int i = 0; i < 9; ++i) dec_lo[1 + i] = a9[i];
      for (int i = 0; i < 7; ++i) rec_lo[1 + i] = s7[i];
      break;
    }
    default:
      return false;
  }
  for (int k = 0; k < fb->L; ++k) {
    const double sgn = (k % 2 == 0) ? 1.0 : -1.0;
    fb->dec_lo[k] = dec_lo[k];
    fb->rec_lo[k] = rec_lo[k];
    fb->rec_hi[k] = sgn * dec_lo[k];
    fb->dec_hi[k] = -sgn * rec_lo[k];
  }
  return true;
}

}  // namespace adjwt
