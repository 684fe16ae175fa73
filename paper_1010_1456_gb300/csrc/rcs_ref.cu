// Host-side RCS post-processing: the quadrature of the direction sphere, the
// error measure of eq. (1), and the Mie-series RCS of a PEC sphere that the
// paper's sphere results are measured against (Section 2.2, Table 2).
//
// Direction quadrature: Gauss-Legendre nodes in mu = cos(theta) (weights
// w_i, sum 2), uniform midpoint nodes in phi (weight 2 pi / n_phi); the
// weight of direction (i, j) is w_i 2 pi / n_phi, so the weights integrate
// over the full solid angle (sum 4 pi).  Legendre nodes by Newton's method
// on P_n from the three-term recurrence.
//
// Eq. (1): err = sqrt( sum_d w_d (s_d - r_d)^2 / sum_d w_d r_d^2 ).
//
// Mie series (PEC sphere of radius a, x = k a, time convention exp(+j w t),
// |S|^2 is convention-free):
//   a_n = psi_n'(x) / xi_n'(x),  b_n = psi_n(x) / xi_n(x),
//   psi_n = x j_n(x), xi_n = x (j_n + i y_n), f_n' = f_{n-1} - n f_n / x,
//   S2(t) = sum_n (2n+1) / (n (n+1)) (a_n tau_n(cos t) + b_n pi_n(cos t)),
// summed to n_max = ceil(x + 4 x^(1/3) + 10).  psi_n comes from Miller's
// downward recurrence (stable for n > x), normalised by psi_0 = sin x or
// psi_1 = sin x / x - cos x, whichever is larger; x y_n from the upward
// recurrence (stable).  For an x-polarised wave travelling along -z,
// sigma_thth(theta, phi) = (lambda^2 / pi) |S2(pi - theta)|^2 cos^2(phi)
// (the +z result rotated by pi about the x axis).
#include <cmath>
#include <complex>
#include <vector>

#include "common.h"
#include "geom.h"

namespace aim {

int rcs_grid(int n_theta, int n_phi, double* theta, double* phi, double* weight) {
  std::vector<double> mu(n_theta), wmu(n_theta);
  const int n = n_theta;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int l = 2; l <= n; ++l) {
        const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);  // P_n'
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute P_n' at the converged node for the weight
    double p0 = 1.0, p1 = z;
    for (int l = 2; l <= n; ++l) {
      const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    const double w = 2.0 / ((1.0 - z * z) * dp * dp);
    mu[i] = -z;  // ascending order, as numpy's leggauss
    mu[n - 1 - i] = z;
    wmu[i] = wmu[n - 1 - i] = w;
  }
  if (n % 2 == 1) mu[n / 2] = 0.0;
  const double dphi = 2.0 * kPi / n_phi;
  for (int i = 0; i < n_theta; ++i)
    for (int j = 0; j < n_phi; ++j) {
      const size_t d = (size_t)i * n_phi + j;
      theta[d] = std::acos(mu[i]);
      phi[d] = (j + 0.5) * dphi;
      weight[d] = wmu[i] * dphi;
    }
  return AIM_OK;
}

int err_thth(int nrhs, int ndir, const double* sig, const double* ref, const double* w, double* err) {
  for (int b = 0; b < nrhs; ++b) {
    double num = 0.0, den = 0.0;
    for (int d = 0; d < ndir; ++d) {
      const double s = sig[(size_t)b * ndir + d], r = ref[(size_t)b * ndir + d];
      num += w[d] * (s - r) * (s - r);
      den += w[d] * r * r;
    }
    if (!(den > 0.0)) {
      set_error("aim_err_thth: the reference pattern is zero");
      return AIM_EINVAL;
    }
    err[b] = std::sqrt(num / den);
  }
  return AIM_OK;
}

int mie_sigma_thth(double radius, double k, int ndir, const double* theta, const double* phi, double* sigma) {
  using C = std::complex<double>;
  const double x = k * radius;
  const int nmax = (int)std::ceil(x + 4.0 * std::cbrt(x) + 10.0);
  // psi_n, n = 0..nmax, by downward recurrence from well above nmax
  const int nstart = nmax + 16 + (int)std::sqrt(40.0 * (nmax + 1));
  std::vector<double> psi(nstart + 2, 0.0);
  psi[nstart + 1] = 0.0;
  psi[nstart] = 1e-250;
  for (int n = nstart; n >= 1; --n) {
    psi[n - 1] = (2.0 * n + 1.0) / x * psi[n] - psi[n + 1];
    if (std::fabs(psi[n - 1]) > 1e250) {  // rescale to stay in range
      for (int m = n - 1; m <= nstart + 1; ++m) psi[m] *= 1e-250;
    }
  }
  const double s0 = std::sin(x), s1 = std::sin(x) / x - std::cos(x);
  const double scale = std::fabs(s0) > std::fabs(s1) ? s0 / psi[0] : s1 / psi[1];
  for (int n = 0; n <= nmax; ++n) psi[n] *= scale;
  // eta_n = x y_n, upward: eta_{-1} = sin x, eta_0 = -cos x
  std::vector<double> eta(nmax + 1);
  double em1 = std::sin(x);
  eta[0] = -std::cos(x);
  for (int n = 1; n <= nmax; ++n) {
    const double prev = n >= 2 ? eta[n - 2] : em1;
    eta[n] = (2.0 * n - 1.0) / x * eta[n - 1] - prev;
  }
  std::vector<C> an(nmax + 1), bn(nmax + 1);
  for (int n = 1; n <= nmax; ++n) {
    const C xi(psi[n], eta[n]), xim1(psi[n - 1], eta[n - 1]);
    const double dpsi = psi[n - 1] - n * psi[n] / x;
    const C dxi = xim1 - (double)n * xi / x;
    an[n] = dpsi / dxi;
    bn[n] = psi[n] / xi;
  }
  const double lam = 2.0 * kPi / k;
  for (int d = 0; d < ndir; ++d) {
    const double mu = std::cos(kPi - theta[d]);
    double pim1 = 0.0, pin = 1.0;  // pi_0, pi_1
    C S2(0.0, 0.0);
    for (int n = 1; n <= nmax; ++n) {
      if (n >= 2) {
        const double p = ((2.0 * n - 1.0) * mu * pin - n * pim1) / (n - 1.0);
        pim1 = pin;
        pin = p;
      }
      const double tau = n * mu * pin - (n + 1.0) * pim1;
      S2 += (2.0 * n + 1.0) / (n * (n + 1.0)) * (an[n] * tau + bn[n] * pin);
    }
    const double cp = std::cos(phi[d]);
    sigma[d] = (lam * lam / kPi) * std::norm(S2) * cp * cp;
  }
  return AIM_OK;
}

}  // namespace aim
