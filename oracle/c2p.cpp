// Conservative-to-primitive recovery, following the paper's appendix
// "Conversion from conserved to primitive fields" (Kastaun et al.'s scheme
// extended to tabulated EOSs) step by step, with the error policy listed at
// the end of that appendix.  Definitions of the conserved variables:
// Sec. II B (eq. def_con2prim).
#include "oracle.hpp"
#include <cfloat>
#include <cmath>

// Undensitized (D, DYe, tau, S_i, B^i) from primitives; eq. def_con2prim
// with h = rho (1 + eps) + p.
void prim2con_point(const real prim[NP], const real B[3], const real gdd[6], real cons[9]) {
  real v[3] = {prim[P_VX], prim[P_VY], prim[P_VZ]};
  real vd[3], Bd[3];
  for (int i = 0; i < 3; ++i) {
    vd[i] = gdd[sym(i, 0)] * v[0] + gdd[sym(i, 1)] * v[1] + gdd[sym(i, 2)] * v[2];
    Bd[i] = gdd[sym(i, 0)] * B[0] + gdd[sym(i, 1)] * B[1] + gdd[sym(i, 2)] * B[2];
  }
  real v2 = v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2];
  real W = 1.0 / sqrt(1.0 - v2);
  real rho = prim[P_RHO], eps = prim[P_EPS], p = prim[P_P];
  real h = rho * (1.0 + eps) + p;
  real B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  real Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
  real D = rho * W;
  cons[0] = D;
  cons[1] = D * prim[P_YE];
  cons[2] = h * W * W - p + B2 - 0.5 * (Bv * Bv + B2 / (W * W)) - D;
  for (int i = 0; i < 3; ++i) cons[3 + i] = (h * W * W + B2) * vd[i] - Bv * Bd[i];
  for (int i = 0; i < 3; ++i) cons[6 + i] = B[i];
}

namespace {

// Quantities fixed during the iterations (step 1 of the appendix).
struct fixed_q {
  real D, Ye, q, r2, rB, B2, B2rp2, v02, h0;
};

// Master-function evaluation and the intermediate values it produces.
struct master_eval {
  real f, chi, rbar2, qbar, v2, W, rho, rho_raw, eps, eps_raw, p, T, cs2;
};

// chi(mu) and rbar^2(mu), eqs. (chi) and (r_bar_sqr).
inline void chi_rbar(const fixed_q& F, real mu, real* chi, real* rbar2) {
  real c = 1.0 / (1.0 + mu * F.B2);
  *chi = c;
  *rbar2 = F.r2 * c * c + mu * c * (1.0 + c) * F.rB * F.rB;
}

// Auxiliary function f_a(mu) = mu sqrt(h0^2 + rbar^2(mu)) - 1  (step 2).
inline real f_aux(const fixed_q& F, real mu) {
  real chi, rbar2;
  chi_rbar(F, mu, &chi, &rbar2);
  return mu * sqrt(F.h0 * F.h0 + rbar2) - 1.0;
}

// Master function f(mu) of step 3 with the EOS validity clamps.
master_eval f_master(const oracle_params* P, const oracle_eos_table* E, const fixed_q& F, real mu) {
  master_eval m;
  chi_rbar(F, mu, &m.chi, &m.rbar2);
  m.qbar = F.q - 0.5 * F.B2 - 0.5 * mu * mu * m.chi * m.chi * F.B2rp2;
  real v2 = mu * mu * m.rbar2;
  m.v2 = fmin(v2, F.v02);
  m.W = 1.0 / sqrt(1.0 - m.v2);
  m.rho_raw = F.D / m.W;
  m.rho = fmax(fmin(P->rho_max, m.rho_raw), P->rho_min);
  m.eps_raw = m.W * (m.qbar - mu * m.rbar2) + m.v2 * m.W * m.W / (1.0 + m.W);
  real emin = eos_eps_min(P, E, m.rho, F.Ye), emax = eos_eps_max(P, E, m.rho, F.Ye);
  m.eps = fmax(fmin(emax, m.eps_raw), emin);
  eos_state s = eos_from_eps(P, E, m.rho, m.eps, F.Ye);
  m.p = s.p;
  m.T = s.T;
  m.cs2 = s.cs2;
  real a = m.p / (m.rho * (1.0 + m.eps));
  real nuA = (1.0 + a) * (1.0 + m.eps) / m.W;
  real nuB = (1.0 + a) * (1.0 + m.qbar - mu * m.rbar2);
  real nu = fmax(nuA, nuB);
  m.f = mu - 1.0 / (nu + mu * m.rbar2);
  return m;
}

// Brent's bracketing root finder (Brent 1973): keeps a bracket [b, c] with
// f(b) f(c) <= 0 and |f(b)| <= |f(c)|, tries inverse quadratic interpolation
// (secant when only two distinct points are known) and falls back to
// bisection when the step is unsafe or the bracket shrinks too slowly.  Stops
// when |c - b| <= 4 eps_mach |b| + xtol or f(b) = 0.
template <class Fn>
real brent(Fn fn, real a, real b, real fa, real fb, int max_iter, double xtol, int* iters, bool* ok) {
  *ok = false;
  *iters = 0;
  if ((fa > 0.0 && fb > 0.0) || (fa < 0.0 && fb < 0.0)) return b;
  real c = a, fc = fa;
  real d = b - a, e = d;
  for (int it = 0; it <= max_iter; ++it) {
    if ((fb > 0.0 && fc > 0.0) || (fb < 0.0 && fc < 0.0)) {
      c = a;
      fc = fa;
      d = b - a;
      e = d;
    }
    if (fabs(fc) < fabs(fb)) {
      a = b;
      b = c;
      c = a;
      fa = fb;
      fb = fc;
      fc = fa;
    }
    real tol = 2.0 * DBL_EPSILON * fabs(b) + 0.5 * xtol;
    real m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) {
      *ok = true;
      *iters = it;
      return b;
    }
    if (it == max_iter) break;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      real s = fb / fa, p, q;
      if (a == c) {
        p = 2.0 * m * s;
        q = 1.0 - s;
      } else {
        real qa = fa / fc, r = fb / fc;
        p = s * (2.0 * m * qa * (qa - r) - (b - a) * (r - 1.0));
        q = (qa - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0.0)
        q = -q;
      else
        p = -p;
      real lim1 = 3.0 * m * q - fabs(tol * q);
      real lim2 = fabs(e * q);
      if (2.0 * p < fmin(lim1, lim2)) {
        e = d;
        d = p / q;
      } else {
        d = m;
        e = m;
      }
    } else {
      d = m;
      e = m;
    }
    a = b;
    fa = fb;
    if (fabs(d) > tol)
      b = b + d;
    else
      b = b + (m > 0.0 ? tol : -tol);
    fb = fn(b);
  }
  *iters = max_iter;
  return b;
}

}  // namespace

int c2p_point(const oracle_params* P, const oracle_eos_table* E, const double cb[10], const double gtp[6],
              double chip, double alpha, double prim[NP], double cons_out[10], int* iters_out) {
  return c2p_point_ext(P, E, cb, gtp, chip, alpha, prim, cons_out, iters_out, nullptr, 0.0, nullptr, nullptr);
}


int c2p_point_ext(const oracle_params* P, const oracle_eos_table* E, const double cb[10], const double gtp[6],
                  double chip, double alpha, double prim[NP], double cons_out[10], int* iters_out, const double* seed3,
                  double delta, double* roots3, int* seeded_ok) {
  for (int n = 0; n < 10; ++n) cons_out[n] = cb[n];
  if (roots3) roots3[0] = roots3[1] = roots3[2] = 0.0;
  if (seeded_ok) *seeded_ok = 0;
  *iters_out = 0;
  // Metric: gamma_ij = gt_ij / chi, gamma^ij = chi gt^ij, sqrt(gamma) = sqrt(det gt) chi^{-3/2}.
  real gt[6], gtu[6], gdd[6], guu[6];
  for (int n = 0; n < 6; ++n) gt[n] = gtp[n];
  real chi = chip;
  real dgt = det_sym(gt);
  inv_sym(gt, dgt, gtu);
  for (int n = 0; n < 6; ++n) {
    gdd[n] = gt[n] / chi;
    guu[n] = chi * gtu[n];
  }
  real sqrtg = sqrt(dgt) / (chi * sqrt(chi));
  bool finite = isfinite_r(sqrtg);
  for (int n = 0; n < 9; ++n) finite = finite && std::isfinite(cb[n]);
  for (int n = 0; n < NP; ++n) prim[n] = 0.0;
  if (!finite || !(sqrtg > 0.0)) return -5;

  real D = cb[0] / sqrtg, DYe = cb[1] / sqrtg, tau = cb[2] / sqrtg;
  real S[3] = {cb[3] / sqrtg, cb[4] / sqrtg, cb[5] / sqrtg};
  real B[3] = {cb[6] / sqrtg, cb[7] / sqrtg, cb[8] / sqrtg};
  bool low_or_bh;
  int status = 0;
  real rho, eps, p, T, cs2, W, ye;
  real v[3] = {0.0, 0.0, 0.0};

  if (D < P->rho_min) {
    // rho = D / W <= D < rho_min: atmosphere (policy item 1) without solving.
    status = 1;
  } else {
    // Step 1: rescaled variables.
    fixed_q F;
    F.D = D;
    F.Ye = DYe / D;
    F.h0 = P->h0;
    F.q = tau / D;
    real r[3] = {S[0] / D, S[1] / D, S[2] / D};
    real sD = sqrt(D);
    real Bc[3] = {B[0] / sD, B[1] / sD, B[2] / sD};
    real ru[3], Bcd[3];
    for (int i = 0; i < 3; ++i) {
      ru[i] = guu[sym(i, 0)] * r[0] + guu[sym(i, 1)] * r[1] + guu[sym(i, 2)] * r[2];
      Bcd[i] = gdd[sym(i, 0)] * Bc[0] + gdd[sym(i, 1)] * Bc[1] + gdd[sym(i, 2)] * Bc[2];
    }
    F.r2 = ru[0] * r[0] + ru[1] * r[1] + ru[2] * r[2];
    F.B2 = Bc[0] * Bcd[0] + Bc[1] * Bcd[1] + Bc[2] * Bcd[2];
    F.rB = r[0] * Bc[0] + r[1] * Bc[1] + r[2] * Bc[2];
    F.B2rp2 = F.B2 * F.r2 - F.rB * F.rB;
    F.v02 = F.r2 / (F.h0 * F.h0 + F.r2);

    // Step 2: mu_+ = root of f_a on (0, 1/h0].  f_a(1/h0) >= 0 analytically;
    // when rounding makes it <= 0 the root is the end point itself.
    // iters counts every evaluation of f_a and of the master function.
    //
    // With a seed s for mu (learned seeder, not part of the paper) the seed
    // bracket is [lo, up] = [s (1 - delta), min(s (1 + delta), 1/h0)].  mu_+
    // only bounds the bracket of Step 3, and f_a changes sign once, at mu_+:
    //  (a) f_a(up) < 0: [lo, up] lies below mu_+; Step 3 runs on it and mu_+
    //      is not solved;
    //  (b) f_a(up) >= 0: mu_+ lies in (0, up] and is solved there; Step 3
    //      runs on [lo, mu_+] when lo < mu_+, else on (0, mu_+].
    // When the master function keeps its sign on the seed bracket, its signs
    // narrow the plain bracket: f(lo) > 0 gives (0, lo]; in case (a) f(up) < 0
    // gives [up, mu_+], with mu_+ solved on [up, 1/h0].
    int it1 = 0, it2 = 0, ev = 0;
    bool ok1 = true, ok2 = true;
    real mu_hi = 1.0 / F.h0;
    auto fa_fn = [&](real mu) { return f_aux(F, mu); };
    auto fm_fn = [&](real x) { return f_master(P, E, F, x).f; };
    int sd = 0;
    real lo = 0.0, up = mu_hi;
    bool seeded = false;
    if (seed3 && std::isfinite(seed3[1]) && seed3[1] > 0.0 && delta > 0.0) {
      real l = seed3[1] * (1.0 - delta);
      real u = fmin(real(seed3[1] * (1.0 + delta)), mu_hi);
      if (l > 0.0 && l < u) {
        seeded = true;
        lo = l;
        up = u;
        sd |= 1;
      }
    }
    real fa_top = f_aux(F, up);
    ev += 1;
    bool case_a = seeded && fa_top < 0.0;
    bool have_plus = !case_a;
    real mu_plus = up;
    if (!case_a && fa_top > 0.0)
      mu_plus = brent(fa_fn, 0.0, up, -1.0, fa_top, P->max_iter, P->c2p_xtol, &it1, &ok1);
    // Step 3: root of the master function on (0, mu_+].  f(mu_+) >= 0
    // analytically (it is exactly 0 when the velocity bound v_0 is reached, as
    // for states with tau below the kinetic energy); a rounding-negative
    // value means the root is mu_+.
    real x_lo = 0.0, x_hi = mu_plus;
    if (case_a) {
      x_lo = lo;
      x_hi = up;
    } else if (seeded && lo < mu_plus) {
      x_lo = lo;
    }
    real f_lo = fm_fn(x_lo), f_hi = fm_fn(x_hi);
    ev += 2;
    bool from_seed = x_lo > 0.0;
    if (x_lo > 0.0 && f_lo > 0.0) {
      x_hi = x_lo;
      f_hi = f_lo;
      x_lo = 0.0;
      f_lo = fm_fn(0.0);
      ev += 1;
      from_seed = false;
    } else if (case_a && f_hi < 0.0) {
      real fa_max = f_aux(F, mu_hi);
      ev += 1;
      mu_plus = mu_hi;
      if (fa_max > 0.0) {
        int itx = 0;
        mu_plus = brent(fa_fn, up, mu_hi, fa_top, fa_max, P->max_iter, P->c2p_xtol, &itx, &ok1);
        it1 += itx;
      }
      have_plus = true;
      x_lo = up;
      f_lo = f_hi;
      x_hi = mu_plus;
      f_hi = fm_fn(mu_plus);
      ev += 1;
      from_seed = false;
    }
    real mu = x_hi;
    if (f_hi > 0.0) mu = brent(fm_fn, x_lo, x_hi, f_lo, f_hi, P->max_iter, P->c2p_xtol, &it2, &ok2);
    if (from_seed) sd |= 2;
    if (!have_plus) sd |= 4;
    if (seeded_ok) *seeded_ok = sd;
    *iters_out = it1 + it2 + ev;
    if (!ok1 || !ok2) return -5;
    // Step 4: primitives from the root.
    master_eval m = f_master(P, E, F, mu);
    if (roots3) {
      roots3[0] = have_plus ? dbl(mu_plus) : 0.0;
      roots3[1] = dbl(mu);
      roots3[2] = dbl(m.W);
    }
    rho = m.rho;
    eps = m.eps;
    p = m.p;
    T = m.T;
    cs2 = m.cs2;
    W = m.W;
    ye = F.Ye;
    for (int i = 0; i < 3; ++i) v[i] = mu * m.chi * (ru[i] + mu * F.rB * Bc[i]);

    // Error policy.
    low_or_bh = (rho < P->rho_low) || (alpha < P->alpha_bh);
    if (m.rho_raw < P->rho_min) {
      status = 1;
    } else {
      if (m.rho_raw > P->rho_max) return -1;
      real emin = eos_eps_min(P, E, rho, ye), emax = eos_eps_max(P, E, rho, ye);
      if (m.eps_raw < emin) status |= 2;
      if (m.eps_raw > emax) {
        if (!low_or_bh) return -2;
        status |= 2;
      }
      if (W > P->W_max) {
        if (!low_or_bh) return -3;
        // Rescale v to v_max keeping D fixed.
        real vmax = sqrt(1.0 - 1.0 / (P->W_max * P->W_max));
        real vd2 = 0.0;
        for (int i = 0; i < 3; ++i)
          vd2 += v[i] * (gdd[sym(i, 0)] * v[0] + gdd[sym(i, 1)] * v[1] + gdd[sym(i, 2)] * v[2]);
        real sc = vmax / sqrt(vd2);
        for (int i = 0; i < 3; ++i) v[i] = v[i] * sc;
        W = P->W_max;
        rho = D / W;
        status |= 4;
      }
      if (ye < P->ye_min || ye > P->ye_max) {
        if (!low_or_bh) return -4;
        ye = P->ye_atmo;
        status |= 8;
      }
      if (status & (4 | 8)) {
        // Thermodynamics at the corrected (rho, eps, ye).
        real e2 = fmax(fmin(eos_eps_max(P, E, rho, ye), eps), eos_eps_min(P, E, rho, ye));
        eos_state s = eos_from_eps(P, E, rho, e2, ye);
        eps = e2;
        p = s.p;
        T = s.T;
        cs2 = s.cs2;
      }
    }
  }
  if (status & 1) {
    eos_state s = eos_atmosphere(P, E);
    rho = P->rho_atmo;
    eps = s.eps;
    p = s.p;
    T = s.T;
    cs2 = s.cs2;
    W = 1.0;
    ye = P->ye_atmo;
    v[0] = v[1] = v[2] = 0.0;
    status = 1;
  }
  prim[P_RHO] = dbl(rho);
  prim[P_EPS] = dbl(eps);
  prim[P_P] = dbl(p);
  prim[P_VX] = dbl(v[0]);
  prim[P_VY] = dbl(v[1]);
  prim[P_VZ] = dbl(v[2]);
  prim[P_W] = dbl(W);
  prim[P_YE] = dbl(ye);
  prim[P_T] = dbl(T);
  prim[P_CS2] = dbl(cs2);
  if (status > 0) {
    // A correction fired: the conserved variables are recomputed from the
    // corrected primitives so that both stay consistent.
    real pr[NP];
    for (int n = 0; n < NP; ++n) pr[n] = prim[n];
    real cons[9];
    prim2con_point(pr, B, gdd, cons);
    for (int n = 0; n < 6; ++n) cons_out[n] = dbl(cons[n] * sqrtg);
  }
  return status;
}

// Master function of one flat-metric state sampled on a uniform grid, for the
// uniqueness pin: Kastaun et al. show that f(mu) changes sign exactly once on
// (0, mu_+], which makes the bracketed root unique.  Step 1 is redone for
// gamma_ij = delta_ij (S_i and B^i as given); Step 2 solves mu_+ as
// c2p_point_ext does without seeds.  Writes f(mu_k) for mu_k = mu_+ k / n,
// k = 1..n, and returns mu_+ (0 when D < rho_min: no solve).
double c2p_master_scan(const oracle_params* P, const oracle_eos_table* E, const double cb[10], long n, double* f_out) {
  real D = cb[0];
  if (!(D >= P->rho_min)) return 0.0;
  fixed_q F;
  F.D = D;
  F.Ye = cb[1] / D;
  F.h0 = P->h0;
  F.q = cb[2] / D;
  real r[3] = {cb[3] / D, cb[4] / D, cb[5] / D};
  real sD = sqrt(D);
  real Bc[3] = {cb[6] / sD, cb[7] / sD, cb[8] / sD};
  F.r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  F.B2 = Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2];
  F.rB = r[0] * Bc[0] + r[1] * Bc[1] + r[2] * Bc[2];
  F.B2rp2 = F.B2 * F.r2 - F.rB * F.rB;
  F.v02 = F.r2 / (F.h0 * F.h0 + F.r2);
  auto fa_fn = [&](real mu) { return f_aux(F, mu); };
  real up = 1.0 / F.h0;
  real fa_top = f_aux(F, up);
  real mu_plus = up;
  int it = 0;
  bool ok = true;
  if (fa_top > 0.0) mu_plus = brent(fa_fn, 0.0, up, -1.0, fa_top, P->max_iter, P->c2p_xtol, &it, &ok);
  for (long k = 1; k <= n; ++k) f_out[k - 1] = dbl(f_master(P, E, F, mu_plus * (real(k) / real(n))).f);
  return dbl(mu_plus);
}
