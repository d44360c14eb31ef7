// Device-side building blocks of the GRMHD substep kernels (sm_103a, FP64):
// the fourth-order centred, compact second and mixed differences, the
// one-sided advection stencils and Kreiss-Oliger dissipation of Sec. III B,
// and small symmetric-matrix helpers.
//
// GB300 executes FP64 at a small fraction of its other pipes, so the kernels
// count FP64 instructions, not bytes: stencils are written with the fewest
// FP64 operations that still give exactly zero on constant data, divisions
// are replaced by products with shared reciprocals where the algebra allows,
// and min/max/select logic is used only where the method prescribes it.
#pragma once
#include <cstdint>
#include "../../include/grmhd.h"

#define DI __device__ __forceinline__

namespace gk {

// Evolved fields.
enum : int {
  GT = 0, AT = 6, CHI = 12, KH = 13, TH = 14, GH = 15, ALP = 18, BET = 19,
  DD = 22, DYE = 23, TAU = 24, SS = 25, BB = 28, PHI = 31, NF = 32, NST = 22
};
// Primitives.
enum : int { RHO = 0, EPS, PRS, VX, VY, VZ, WW, YE, TT, CS2, NP };
// Initial-data fields.
enum : int { IG = 0, IK = 6, IALP = 12, IBET = 13, IRHO = 16, IEPS = 17, IV = 18, IB = 21, IYE = 24, IT = 25 };

constexpr int S6(int i, int j) {
  return (i == j) ? (i == 0 ? 0 : (i == 1 ? 3 : 5)) : ((i + j) == 1 ? 1 : ((i + j) == 2 ? 2 : 4));
}

// Patch geometry on the device.
struct Geo {
  int n0, n1, n2, px;
  long long sy, sz, sf;  // strides (x stride 1)
  double dx;
  double i12, i12s, i144, ihdx;  // 1/(12 dx), 1/(12 dx^2), 1/(144 dx^2), 1/(2 dx)
};

DI long long at(const Geo& G, int i, int j, int k) {
  return (long long)(k + 3) * G.sz + (long long)(j + 3) * G.sy + (i + 3);
}

// Symmetric 3x3 determinant and inverse (adjugate / det).
DI double det3(const double g[6]) {
  return g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2]);
}
DI void inv3(const double g[6], double idet, double u[6]) {
  u[0] = (g[3] * g[5] - g[4] * g[4]) * idet;
  u[1] = (g[2] * g[4] - g[1] * g[5]) * idet;
  u[2] = (g[1] * g[4] - g[2] * g[3]) * idet;
  u[3] = (g[0] * g[5] - g[2] * g[2]) * idet;
  u[4] = (g[1] * g[2] - g[0] * g[4]) * idet;
  u[5] = (g[0] * g[3] - g[1] * g[1]) * idet;
}
// sum_ij a^ij b_ij for symmetric a, b.
DI double tr6(const double a[6], const double b[6]) {
  return a[0] * b[0] + a[3] * b[3] + a[5] * b[5] + 2.0 * (a[1] * b[1] + a[2] * b[2] + a[4] * b[4]);
}
DI void lower3(const double g[6], const double v[3], double o[3]) {
  o[0] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  o[1] = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  o[2] = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
}

DI double ld(const double* p) { return __ldg(p); }

// ---- 4th-order finite differences (scaled later by the caller) ------------
// d1:  8 (u1 - u-1) - (u2 - u-2)              [x 1/(12 dx)]
DI double fd1(const double* u, long long s) {
  return fma(8.0, ld(u + s) - ld(u - s), -(ld(u + 2 * s) - ld(u - 2 * s)));
}
// d2:  16 ((u1 - u0) + (u-1 - u0)) - ((u2 - u0) + (u-2 - u0))     [x 1/(12 dx^2)]
// Differences against the centre are exact for nearby values (Sterbenz), so
// the stencil keeps full relative accuracy on small variations of O(1) fields.
DI double fd2(const double* u, long long s, double c) {
  double a = (ld(u + s) - c) + (ld(u - s) - c);
  double b = (ld(u + 2 * s) - c) + (ld(u - 2 * s) - c);
  return fma(16.0, a, -b);
}
// mixed: d1 along s2 of d1 along s1      [x 1/(144 dx^2)]
DI double fd11(const double* u, long long s1, long long s2) {
  double p1 = fd1(u + s2, s1), m1 = fd1(u - s2, s1), p2 = fd1(u + 2 * s2, s1), m2 = fd1(u - 2 * s2, s1);
  return fma(8.0, p1 - m1, -(p2 - m2));
}
// One-sided advection derivative (upwind for beta^k d_k):             [x 1/(12 dx)]
//   b > 0:   (u3 - u0) - 6 (u2 - u0) + 18 (u1 - u0) - 3 (u-1 - u0)
//   b <= 0: -[(u-3 - u0) - 6 (u-2 - u0) + 18 (u-1 - u0) - 3 (u1 - u0)]
DI double fdup(const double* u, long long s, double c) {
  double t3 = ld(u + 3 * s) - c, t2 = ld(u + 2 * s) - c, t1 = ld(u + s) - c, tm = ld(u - s) - c;
  return fma(-3.0, tm, fma(18.0, t1, fma(-6.0, t2, t3)));
}
// KO 7-point stencil:  ((u-3 - u0) + (u3 - u0)) - 6 ((u-2 - u0) + (u2 - u0)) + 15 ((u-1 - u0) + (u1 - u0))
//                                                                       [x sigma/(64 dx)]
DI double fdko(const double* u, long long s, double c) {
  double a3 = (ld(u + 3 * s) - c) + (ld(u - 3 * s) - c);
  double a2 = (ld(u + 2 * s) - c) + (ld(u - 2 * s) - c);
  double a1 = (ld(u + s) - c) + (ld(u - s) - c);
  return fma(15.0, a1, fma(-6.0, a2, a3));
}

// ---- comparisons on the integer pipe ----------------------------------------
// FP64 min / max / compare issue on the same narrow pipe as DFMA on GB300
// (measured: fmin 1.3, compare+select 1.6, DFMA 1.6 lanes/clk/SM), while a
// 64-bit integer compare runs ~5x wider.  okey() maps doubles to int64 with
// the same order (-0 sorts just below +0), so min/max/sign tests move off the
// FP64 pipe and return the same values for every non-NaN input.
DI long long okey(double x) {
  long long k = __double_as_longlong(x);
  return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}
DI bool ipos(double x) { return __double_as_longlong(x) > 0; }  // x > 0
DI bool ineg(double x) { return okey(x) < -1; }                 // x < 0 (okey(-0) = -1)
DI double imin(double a, double b) { return okey(a) <= okey(b) ? a : b; }
DI double imax(double a, double b) { return okey(a) >= okey(b) ? a : b; }

// ---- MP5 (Suresh & Huynh) with alpha = 4 ------------------------------------
// Minmod(a, b) = (sgn a + sgn b)/2 min(|a|, |b|).
DI double mm2(double a, double b) {
  return (ipos(a) && ipos(b)) ? imin(a, b) : ((ineg(a) && ineg(b)) ? imax(a, b) : 0.0);
}
DI double mm4(double a, double b, double c, double d) {
  if (ipos(a) && ipos(b) && ipos(c) && ipos(d)) return imin(imin(a, b), imin(c, d));
  if (ineg(a) && ineg(b) && ineg(c) && ineg(d)) return imax(imax(a, b), imax(c, d));
  return 0.0;
}
// Order of x against y as the sign of the rounded difference x - y (which
// has the sign of the exact one, and is zero exactly when x == y, +0 == -0),
// taken on the integer pipe: -1, 0 or +1.
DI int iorder(double x, double y) {
  const long long kx = __double_as_longlong(x), ky = __double_as_longlong(y);
  if (kx == ky || ((kx | ky) << 1) == 0) return 0;
  return okey(x) > okey(y) ? 1 : -1;
}

// Interface value between c and d from a..e (= F_{i-2} .. F_{i+2}).
// The 5th-order value is formed from differences to c,
//   f = c + (2 (a - c) - 13 (b - c) + 27 (d - c) - 3 (e - c)) / 60,
// which is exact on constant data.  When f == c the limited value is f
// itself (f_min <= c <= f_max always), so that case returns at once.
DI double mp5(double a, double b, double c, double d, double e) {
  const double al = 4.0;
  double dp = d - c, dm = c - b;
  double t = fma(-3.0, e - c, fma(27.0, dp, fma(2.0, a - c, 13.0 * dm)));
  double f = fma(t, 1.0 / 60.0, c);
  // (f - c)(f - f_MP) < 0 as a test of the two differences' signs, taken by
  // integer comparisons (no FP64 subtraction, product or compare).
  const int s1 = iorder(f, c);
  if (s1 == 0) return f;
  double fmp = c + mm2(dp, al * dm);
  if (s1 * iorder(f, fmp) < 0) return f;
  double d_m = dm - (b - a), d_0 = dp - dm, d_p = (e - d) - dp;
  double m4p = mm4(fma(4.0, d_0, -d_p), fma(4.0, d_p, -d_0), d_0, d_p);
  double m4m = mm4(fma(4.0, d_0, -d_m), fma(4.0, d_m, -d_0), d_0, d_m);
  double ful = fma(al, dm, c);
  double fmd = fma(-0.5, m4p, 0.5 * (c + d));
  double flc = fma(4.0 / 3.0, m4m, fma(0.5, dm, c));
  double fmn = imax(imin(imin(c, d), fmd), imin(imin(c, ful), flc));
  double fmx = imin(imax(imax(c, d), fmd), imax(imax(c, ful), flc));
  return fmn + mm2(f - fmn, fmx - fmn);
}

}  // namespace gk
