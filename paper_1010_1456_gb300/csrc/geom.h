// FP64 geometry and integration helpers for the EFIE/AIM setup.
//
// Everything here is plain FP64 arithmetic usable on the host (setup threads)
// and on the device.  Rules and formulas:
//  * triangle rule: collapsed (Duffy) product of n-point Gauss-Legendre rules
//    on the triangle's stored vertex order, r = r0 + s (r1-r0) + t(1-s)(r2-r0),
//    weight 2 w_s w_t (1-s) (weights sum to 1; integral = area * sum);
//  * Gauss-Legendre nodes by Newton iteration on the three-term recurrence of
//    the Legendre polynomials;
//  * closed-form integrals of 1/R and (rho'-rho)/R over a planar triangle
//    (divergence theorem over the edges; the "R + l" factors are evaluated
//    as R0^2/(R - l) when l < 0 to avoid cancellation);
//  * EFIE triangle-pair block with singularity extraction for triangles that
//    share a vertex (paper Section 2.2 EFIE; the rule choice is this
//    library's, the paper gives none).
#pragma once

#include <cmath>

#include "common.h"

namespace aim {

struct V3 {
  double x, y, z;
};
AIM_HD inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
AIM_HD inline V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
AIM_HD inline V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
AIM_HD inline V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
AIM_HD inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
AIM_HD inline V3 cross(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
AIM_HD inline double norm(V3 a) { return sqrt(dot(a, a)); }

constexpr double kPi = 3.14159265358979323846;
constexpr double kEta0 = 376.730313668;
constexpr int kMaxRule = 12;  // max points per direction

// n-point Gauss-Legendre rule on [0, 1].
inline void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    // i-th root of P_n, largest first, from the classical initial guess
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? z : p1;
    double pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (z * pn - pnm1) / (z * z - 1.0);
    double wz = 2.0 / ((1.0 - z * z) * dp * dp);
    // map [-1, 1] -> [0, 1]; roots come largest first, so 0.5 (1 - z) ascends
    x[i] = 0.5 * (1.0 - z);
    w[i] = 0.5 * wz;
  }
}

// Collapsed triangle rule with n x n points, i-major (s outer, t inner).
struct TriRule {
  int q = 0;
  double xi1[kMaxRule * kMaxRule];
  double xi2[kMaxRule * kMaxRule];
  double w[kMaxRule * kMaxRule];
};
inline TriRule make_tri_rule(int n) {
  TriRule r;
  double s[kMaxRule], ws[kMaxRule];
  gauss_legendre01(n, s, ws);
  r.q = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int p = i * n + j;
      r.xi1[p] = s[i];
      r.xi2[p] = s[j] * (1.0 - s[i]);
      r.w[p] = 2.0 * ws[i] * ws[j] * (1.0 - s[i]);
    }
  return r;
}

AIM_HD inline V3 tri_point(V3 r0, V3 r1, V3 r2, double a, double b) {
  return r0 + a * (r1 - r0) + b * (r2 - r0);
}

// int_T 1/R dS' (I0) and int_T (rho' - rho)/R dS' (I1) for observer r.
AIM_HD inline void potential_integrals(V3 r, V3 v0, V3 v1, V3 v2, double* I0, V3* I1, V3* rho_out) {
  V3 nrm = cross(v1 - v0, v2 - v0);
  V3 nh = (1.0 / norm(nrm)) * nrm;
  double d = dot(r - v0, nh);
  V3 rho = r - d * nh;
  double ad = fabs(d);
  double i0 = 0.0;
  V3 i1 = v3(0, 0, 0);
  V3 va[3] = {v0, v1, v2};
  for (int e = 0; e < 3; ++e) {
    V3 a = va[e], b = va[(e + 1) % 3];
    V3 ed = b - a;
    double elen = norm(ed);
    V3 lh = (1.0 / elen) * ed;
    V3 u = cross(lh, nh);
    double lp = dot(b - rho, lh);
    double lm = dot(a - rho, lh);
    double t = dot(a - rho, u);
    double R02 = t * t + d * d;
    double Rp = sqrt(R02 + lp * lp);
    double Rm = sqrt(R02 + lm * lm);
    double lin = 0.5 * (lp * Rp - lm * Rm);
    if (R02 > 1e-30 * elen * elen) {
      double num = (lp >= 0.0) ? (Rp + lp) : (R02 / (Rp - lp));
      double den = (lm >= 0.0) ? (Rm + lm) : (R02 / (Rm - lm));
      double f2 = log(num / den);
      double at = atan(t * lp / (R02 + ad * Rp)) - atan(t * lm / (R02 + ad * Rm));
      i0 += t * f2 - ad * at;
      i1 = i1 + (0.5 * R02 * f2 + lin) * u;
    } else {
      i1 = i1 + lin * u;
    }
  }
  *I0 = i0;
  *I1 = i1;
  *rho_out = rho;
}

struct Cd {
  double re, im;
};
AIM_HD inline Cd cd(double a, double b) { return Cd{a, b}; }
AIM_HD inline Cd operator+(Cd a, Cd b) { return Cd{a.re + b.re, a.im + b.im}; }
AIM_HD inline Cd operator*(double s, Cd a) { return Cd{s * a.re, s * a.im}; }

// G(R) = exp(-jkR)/(4 pi R) (regular) or its smooth part [exp(-jkR)-1]/(4 pi R)
// written as -(jk/4pi) sinc(kR/2) exp(-jkR/2).
AIM_HD inline Cd green_full(double k, double R) {
  double s = 1.0 / (4.0 * kPi * R);
  double sn, cs;
  sincos(k * R, &sn, &cs);
  return Cd{cs * s, -sn * s};
}
AIM_HD inline Cd green_smooth(double k, double R) {
  double x = 0.5 * k * R;
  double sn, cs;
  sincos(x, &sn, &cs);
  double sc = (x == 0.0) ? 1.0 : sn / x;
  double c = -k / (4.0 * kPi) * sc;  // multiplies j * exp(-jx)
  // j * exp(-jx) = j (cos x - j sin x) = sin x + j cos x
  return Cd{c * sn, c * cs};
}

// EFIE triangle-pair block T[a][b] (a: slot on test triangle P, b: slot on
// source triangle Q):
//   T_ab = sum_i W_i [ (r_i - P_a).V_b(r_i) / (4 A_P A_Q) - S0(r_i) / (k^2 A_P A_Q) ]
//   S0(r) = int_Q G dS',  V_b(r) = int_Q (r' - Q_b) G dS' = V(r) - Q_b S0(r),  V(r) = int_Q r' G dS'
// so that Z_mn += j k eta s_m s_n l_m l_n T[a(m)][b(n)].  The source sum
// accumulates S0 and V only (four complex values per source point); the nine
// V_b follow per test point.
AIM_HD inline void pair_block(const V3 P[3], const V3 Q[3], double AP, double AQ, bool singular, double k,
                              const TriRule& test, const TriRule& src, Cd T[3][3]) {
  Cd acc[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) acc[a][b] = cd(0, 0);
  Cd s0acc = cd(0, 0);
  for (int i = 0; i < test.q; ++i) {
    V3 ri = tri_point(P[0], P[1], P[2], test.xi1[i], test.xi2[i]);
    double Wi = AP * test.w[i];
    Cd S0 = cd(0, 0);
    Cd V[3] = {cd(0, 0), cd(0, 0), cd(0, 0)};
    for (int q = 0; q < src.q; ++q) {
      V3 rq = tri_point(Q[0], Q[1], Q[2], src.xi1[q], src.xi2[q]);
      double R = norm(ri - rq);
      Cd g = singular ? green_smooth(k, R) : green_full(k, R);
      g = (AQ * src.w[q]) * g;
      S0 = S0 + g;
      V[0] = V[0] + rq.x * g;
      V[1] = V[1] + rq.y * g;
      V[2] = V[2] + rq.z * g;
    }
    Cd Vb[3][3];  // [b][xyz]
    for (int b = 0; b < 3; ++b) {
      Vb[b][0] = V[0] + (-Q[b].x) * S0;
      Vb[b][1] = V[1] + (-Q[b].y) * S0;
      Vb[b][2] = V[2] + (-Q[b].z) * S0;
    }
    if (singular) {
      double I0;
      V3 I1, rho;
      potential_integrals(ri, Q[0], Q[1], Q[2], &I0, &I1, &rho);
      const double f = 1.0 / (4.0 * kPi);
      S0.re += f * I0;
      for (int b = 0; b < 3; ++b) {
        V3 add = I1 + I0 * (rho - Q[b]);
        Vb[b][0].re += f * add.x;
        Vb[b][1].re += f * add.y;
        Vb[b][2].re += f * add.z;
      }
    }
    for (int a = 0; a < 3; ++a) {
      V3 ra = ri - P[a];
      for (int b = 0; b < 3; ++b) {
        Cd dt = ra.x * Vb[b][0] + ra.y * Vb[b][1] + ra.z * Vb[b][2];
        acc[a][b] = acc[a][b] + Wi * dt;
      }
    }
    s0acc = s0acc + Wi * S0;
  }
  double f1 = 1.0 / (4.0 * AP * AQ);
  double f2 = 1.0 / (k * k * AP * AQ);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) T[a][b] = cd(f1 * acc[a][b].re - f2 * s0acc.re, f1 * acc[a][b].im - f2 * s0acc.im);
}

// Derivative of the 1-D Lagrange basis on nodes 0..M at t.
AIM_HD inline double lagrange_d(int M, int i, double t) {
  double sum = 0.0;
  for (int q = 0; q <= M; ++q) {
    if (q == i) continue;
    double v = 1.0 / (double)(i - q);
    for (int p = 0; p <= M; ++p)
      if (p != i && p != q) v *= (t - p) / (double)(i - p);
    sum += v;
  }
  return sum;
}

// 1-D Lagrange basis on nodes 0..M evaluated at t.
AIM_HD inline double lagrange(int M, int i, double t) {
  double v = 1.0;
  for (int p = 0; p <= M; ++p)
    if (p != i) v *= (t - p) / (double)(i - p);
  return v;
}

}  // namespace aim
