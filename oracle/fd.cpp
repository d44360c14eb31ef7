// Finite-difference operators of Sec. III B and the MP5 reconstruction of
// Sec. III C.  Stencils are evaluated with differences against the centre
// value (or antisymmetric differences) first, so that constant data give an
// exactly zero derivative in floating point.
#include "oracle.hpp"

// Centred 4th-order first derivative D_x:
// (U_{i-2} - 8 U_{i-1} + 8 U_{i+1} - U_{i+2}) / (12 dx).
real fd_d1(const double* u, long s, real inv12dx) {
  real a = u[s], b = u[-s], c = u[2 * s], d = u[-2 * s];
  return (8.0 * (a - b) - (c - d)) * inv12dx;
}

// Compact 4th-order second derivative D_xx:
// (-U_{i-2} + 16 U_{i-1} - 30 U_i + 16 U_{i+1} - U_{i+2}) / (12 dx^2).
real fd_d2(const double* u, long s, real inv12dx2) {
  real c = u[0];
  real p1 = real(u[s]) - c, m1 = real(u[-s]) - c, p2 = real(u[2 * s]) - c, m2 = real(u[-2 * s]) - c;
  return (16.0 * (p1 + m1) - (p2 + m2)) * inv12dx2;
}

// Mixed second derivative D_{s1 s2} = D_{s2}(D_{s1} U): the centred first
// derivative along s1 evaluated at the four off-centre points of the centred
// first derivative along s2.  inv144dx2 = 1 / (144 dx^2).
real fd_d11(const double* u, long s1, long s2, real inv144dx2) {
  real a[5];
  for (int m = -2; m <= 2; ++m) {
    if (m == 0) continue;
    const double* v = u + m * s2;
    a[m + 2] = 8.0 * (real(v[s1]) - real(v[-s1])) - (real(v[2 * s1]) - real(v[-2 * s1]));
  }
  return (8.0 * (a[3] - a[1]) - (a[4] - a[0])) * inv144dx2;
}

// One-sided 4th-order advection derivative chosen by the sign of the shift
// component:  beta > 0: (U_{i+3} - 6 U_{i+2} + 18 U_{i+1} - 10 U_i - 3 U_{i-1}) / (12 dx)
//             beta < 0: (-U_{i-3} + 6 U_{i-2} - 18 U_{i-1} + 10 U_i + 3 U_{i+1}) / (12 dx)
// (beta = 0 takes the second form; the product with beta vanishes anyway).
real fd_up(const double* u, long s, real beta, real inv12dx) {
  real c = u[0];
  if (beta > 0.0) {
    real p3 = real(u[3 * s]) - c, p2 = real(u[2 * s]) - c, p1 = real(u[s]) - c, m1 = real(u[-s]) - c;
    return (p3 - 6.0 * p2 + 18.0 * p1 - 3.0 * m1) * inv12dx;
  }
  real m3 = real(u[-3 * s]) - c, m2 = real(u[-2 * s]) - c, m1 = real(u[-s]) - c, p1 = real(u[s]) - c;
  return -(m3 - 6.0 * m2 + 18.0 * m1 - 3.0 * p1) * inv12dx;
}

// Kreiss-Oliger dissipation along one axis, coef = sigma / (64 dx):
// coef (U_{i-3} - 6 U_{i-2} + 15 U_{i-1} - 20 U_i + 15 U_{i+1} - 6 U_{i+2} + U_{i+3}).
real fd_ko(const double* u, long s, real coef) {
  real c = u[0];
  real s3 = (real(u[-3 * s]) - c) + (real(u[3 * s]) - c);
  real s2 = (real(u[-2 * s]) - c) + (real(u[2 * s]) - c);
  real s1 = (real(u[-s]) - c) + (real(u[s]) - c);
  return (s3 - 6.0 * s2 + 15.0 * s1) * coef;
}

// Minmod(a, b) = (sgn a + sgn b)/2 min(|a|, |b|), sgn(0) = 0.
real minmod2(real a, real b) {
  if (a > 0.0 && b > 0.0) return fmin(a, b);
  if (a < 0.0 && b < 0.0) return fmax(a, b);
  return 0.0;
}

// Four-argument minmod: sgn(a) min(|a|,|b|,|c|,|d|) when all signs agree, else 0.
real minmod4(real a, real b, real c, real d) {
  if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return fmin(fmin(a, b), fmin(c, d));
  if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return fmax(fmax(a, b), fmax(c, d));
  return 0.0;
}

// MP5 reconstruction (Suresh & Huynh) of the value at the interface between
// the points holding c and d, from the five values a..e = F_{i-2}..F_{i+2};
// alpha = 4.  Eqs. MP5_unal, MP5_bounds, MP5_bounds2 and MP5_dm4.
real mp5(real a, real b, real c, real d, real e) {
  const double alpha = 4.0;
  real f_ip = (2.0 * a - 13.0 * b + 47.0 * c + 27.0 * d - 3.0 * e) / 60.0;
  real dlt_p = d - c;  // Delta_{i+1/2}
  real dlt_m = c - b;  // Delta_{i-1/2}
  real f_mp = c + minmod2(dlt_p, alpha * dlt_m);
  if ((f_ip - c) * (f_ip - f_mp) < 0.0) return f_ip;
  real d_m = (c - b) - (b - a);  // d_{i-1}
  real d_0 = dlt_p - dlt_m;      // d_i
  real d_p = (e - d) - (d - c);  // d_{i+1}
  real dm4_p = minmod4(4.0 * d_0 - d_p, 4.0 * d_p - d_0, d_0, d_p);
  real dm4_m = minmod4(4.0 * d_0 - d_m, 4.0 * d_m - d_0, d_0, d_m);
  real f_ul = c + alpha * dlt_m;
  real f_md = 0.5 * (c + d) - 0.5 * dm4_p;
  real f_lc = c + 0.5 * dlt_m + (4.0 / 3.0) * dm4_m;
  real f_min = fmax(fmin(fmin(c, d), f_md), fmin(fmin(c, f_ul), f_lc));
  real f_max = fmin(fmax(fmax(c, d), f_md), fmax(fmax(c, f_ul), f_lc));
  // Median(f_min, f_ip, f_max) = f_min + Minmod(f_ip - f_min, f_max - f_min).
  return f_min + minmod2(f_ip - f_min, f_max - f_min);
}
