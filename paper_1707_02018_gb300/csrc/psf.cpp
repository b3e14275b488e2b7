// Gaussian point-spread taps and their derivative with respect to the width,
// for building R and dR/dsigma (differentiation of the deblurring problem of
// Sec. 1, Eq. 1 through its blur).
//
// taps[i] = e_i / S with e_i = exp(-d_i^2 / (2 sigma^2)), d_i = i - (k-1)/2,
// S = sum_j e_j (a normalised sampled Gaussian).  Differentiating,
// de_i/dsigma = e_i d_i^2 / sigma^3, so
//   dtaps[i] = taps[i] (d_i^2 - sum_j taps[j] d_j^2) / sigma^3.
// A separable PSF g (x) g has d(g (x) g)/dsigma = g' (x) g + g (x) g', so
// dR/dsigma u = R[g', g] u + R[g, g'] u: two blur passes with these taps.
#include <cmath>

#include "adjwt_internal.h"

using namespace adjwt;

extern "C" int adjwt_gaussian_taps(int k, double sigma, double* taps, double* dtaps_dsigma) {
  if (k < 1 || k % 2 == 0) return fail(ADJWT_ERR_SHAPE, "adjwt_gaussian_taps: k must be odd and >= 1");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_gaussian_taps: sigma must be > 0");
  if (!taps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_gaussian_taps: taps is NULL");
  const double c = 0.5 * (k - 1);
  double sum = 0.0;
  for (int i = 0; i < k; ++i) {
    const double d = i - c;
    taps[i] = std::exp(-d * d / (2.0 * sigma * sigma));
    sum += taps[i];
  }
  double m2 = 0.0;  // sum_j taps[j] d_j^2 after normalisation
  for (int i = 0; i < k; ++i) {
    taps[i] /= sum;
    const double d = i - c;
    m2 += taps[i] * d * d;
  }
  if (dtaps_dsigma) {
    const double s3 = sigma * sigma * sigma;
    for (int i = 0; i < k; ++i) {
      const double d = i - c;
      dtaps_dsigma[i] = taps[i] * (d * d - m2) / s3;
    }
  }
  return ADJWT_OK;
}
