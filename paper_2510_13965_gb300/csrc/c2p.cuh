// Device EOS, prim2con and con2prim: Kastaun's two Brent root finds with the
// EOS validity clamps and the error policy, following the appendix
// "Conversion from conserved to primitive fields" (steps 1-4 and the policy
// list at its end); conserved variables as defined in Sec. II B
// (eq. def_con2prim); hybrid EOS as in Sec. II B.
//
// The master function is evaluated with the identities
//   eps_hat = W (qbar - mu rbar^2 + 1) - 1      (v^2 W^2 / (1 + W) = W - 1),
//   nu_A = h / W,  nu_B = h (1 + qbar - mu rbar^2) / (1 + eps),  h = 1 + eps + p / rho,
// and Brent's inverse-quadratic step is scaled by f_a f_c^2 so one division
// per iteration remains.  Results agree with the literal formulas to rounding.
#pragma once
#include "dev.cuh"

namespace gk {

struct EosOut {
  double p, eps, T, cs2;
};

struct Eos {
  int kind;
  double gam, K, eps_max;
  // hybrid: cold pieces (K_i, a_i, Gamma_i), dividing densities
  int npoly;
  double hK[4], ha[4], hg[4], hr[3];
  // table
  int nr, nt, ny;
  double lr0, idlr, lt0, dlt, idlt, ye0, idye;
  const double* p;
  const double* e;
  const double* c;
  // The atmosphere's state eos_T(rho_atmo, T_atmo, ye_atmo), evaluated once
  // on the device when atmo_set (a context's EOS); else per atmosphere point.
  int atmo_set;
  EosOut atmo;
};

DI void tab_loc(const Eos& E, double x, double x0, double idx, int n, int* i, double* w) {
  double f = (x - x0) * idx;
  double fl = floor(f);
  int ii = (int)fl;
  ii = ii < 0 ? 0 : (ii > n - 2 ? n - 2 : ii);
  double ww = f - (double)ii;
  *w = fmin(fmax(ww, 0.0), 1.0);
  *i = ii;
}

struct TabPos {
  long long b;  // node offset of (ir, 0, iy)
  double wr, wy;
  int sr, st, sy;
};

DI TabPos tab_pos(const Eos& E, double rho, double ye) {
  int ir, iy;
  TabPos t;
  tab_loc(E, log10(rho), E.lr0, E.idlr, E.nr, &ir, &t.wr);
  tab_loc(E, ye, E.ye0, E.idye, E.ny, &iy, &t.wy);
  t.sr = 1;
  t.st = E.nr;
  t.sy = E.nr * E.nt;
  t.b = (long long)iy * t.sy + ir;
  return t;
}
// Bilinear value in (rho, Ye) at temperature node it.
DI double tab_bl(const TabPos& t, const double* A, int it) {
  const double* q = A + t.b + (long long)it * t.st;
  double lo = fma(t.wr, ld(q + 1) - ld(q), ld(q));
  double hi = fma(t.wr, ld(q + t.sy + 1) - ld(q + t.sy), ld(q + t.sy));
  return fma(t.wy, hi - lo, lo);
}

// Hybrid EOS cold part on the piece holding rho: p_cold, eps_cold, Gamma_i.
struct HybCold {
  double p, eps, g;
};
DI HybCold hyb_cold(const Eos& E, double rho) {
  int i = 0;
  while (i < E.npoly - 1 && rho > E.hr[i]) ++i;
  HybCold c;
  c.g = E.hg[i];
  const double rg1 = pow(rho, c.g - 1.0);
  c.p = E.hK[i] * rg1 * rho;
  c.eps = fma(E.hK[i] / (c.g - 1.0), rg1, E.ha[i]);
  return c;
}
// Hybrid (p, cs2) at eps: p = p_c + (Gamma_th - 1) rho (eps - eps_c);
// c_s^2 h = dp/drho|_eps + p / rho^2 dp/deps|_rho with deps_c/drho = p_c / rho^2.
DI void hyb_eps(const Eos& E, const HybCold& c, double rho, double eps, double* p, double* cs2) {
  const double gth = E.gam - 1.0, de = eps - c.eps;
  *p = fma(gth * rho, de, c.p);
  if (cs2) {
    const double ir = 1.0 / rho;
    const double dpdr = fma(gth, de, (c.g - gth) * c.p * ir);
    *cs2 = fma(gth * ir, *p, dpdr) / (1.0 + eps + *p * ir);
  }
}

DI double eos_emin(const Eos& E, double rho, double ye) {
  if (E.kind == 0) return 0.0;
  if (E.kind == 2) return hyb_cold(E, rho).eps;
  return tab_bl(tab_pos(E, rho, ye), E.e, 0);
}
DI double eos_emax(const Eos& E, double rho, double ye) {
  if (E.kind != 1) return E.eps_max;
  return tab_bl(tab_pos(E, rho, ye), E.e, E.nt - 1);
}

// Temperature cell of the table at a (rho, Ye) location: the nodes lo, lo+1
// whose eps values (elo, ehi) bracket eps by binary search; the first or last
// cell when eps lies below or above the column.
DI void tab_tcell(const Eos& E, const TabPos& t, double eps, int* lo_, double* elo_, double* ehi_) {
  int lo = 0, hi = E.nt - 1;
  double elo = tab_bl(t, E.e, lo), ehi = tab_bl(t, E.e, hi);
  if (eps <= elo) {
    hi = 1;
    ehi = tab_bl(t, E.e, 1);
  } else if (eps >= ehi) {
    lo = E.nt - 2;
    elo = tab_bl(t, E.e, lo);
  } else {
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      double em = tab_bl(t, E.e, mid);
      if (em <= eps) {
        lo = mid;
        elo = em;
      } else {
        hi = mid;
        ehi = em;
      }
    }
  }
  *lo_ = lo;
  *elo_ = elo;
  *ehi_ = ehi;
}

// (p, T, cs2) from (rho, eps, ye); eps inside [eps_min, eps_max].
DI EosOut eos_eps(const Eos& E, double rho, double eps, double ye) {
  EosOut o;
  o.eps = eps;
  if (E.kind == 0) {
    o.p = (E.gam - 1.0) * rho * eps;
    o.T = 0.0;
    o.cs2 = E.gam * o.p / fma(rho, 1.0 + eps, o.p);
    return o;
  }
  if (E.kind == 2) {
    hyb_eps(E, hyb_cold(E, rho), rho, eps, &o.p, &o.cs2);
    o.T = 0.0;
    return o;
  }
  TabPos t = tab_pos(E, rho, ye);
  int lo;
  double elo, ehi;
  tab_tcell(E, t, eps, &lo, &elo, &ehi);
  double w = fmin(fmax((eps - elo) / (ehi - elo), 0.0), 1.0);
  double p0 = tab_bl(t, E.p, lo), p1 = tab_bl(t, E.p, lo + 1);
  double c0 = tab_bl(t, E.c, lo), c1 = tab_bl(t, E.c, lo + 1);
  o.p = fma(w, p1 - p0, p0);
  o.cs2 = fma(w, c1 - c0, c0);
  o.T = exp10(fma((double)lo + w, E.dlt, E.lt0));
  return o;
}

// The master function's EOS step in one table location: eps clamped to
// [eps_min(rho), eps_max(rho)], then (p, T, cs2) at the clamped eps.  For the
// table the temperature cell search starts at *cell (the previous
// evaluation's cell, or -1): eps increases strictly along T at fixed
// (rho, Ye), so the cell with e_k <= eps < e_{k+1} is unique and the result
// equals that of the full binary search.  *cell receives the cell used.
struct EosClamp {
  double eps, p, T, cs2, emin, emax;
};
template <bool FULL>
DI EosClamp eos_clamped(const Eos& E, double rho, double eps_raw, double ye, int* cell) {
  EosClamp o;
  if (E.kind == 0) {
    o.emin = 0.0;
    o.emax = E.eps_max;
    o.eps = fmax(fmin(o.emax, eps_raw), o.emin);
    o.p = (E.gam - 1.0) * rho * o.eps;
    o.T = 0.0;
    o.cs2 = FULL ? E.gam * o.p / fma(rho, 1.0 + o.eps, o.p) : 0.0;
    return o;
  }
  if (E.kind == 2) {
    const HybCold c = hyb_cold(E, rho);
    o.emin = c.eps;
    o.emax = E.eps_max;
    o.eps = fmax(fmin(o.emax, eps_raw), o.emin);
    o.T = 0.0;
    o.cs2 = 0.0;
    hyb_eps(E, c, rho, o.eps, &o.p, FULL ? &o.cs2 : nullptr);
    return o;
  }
  TabPos t = tab_pos(E, rho, ye);
  double elo = tab_bl(t, E.e, 0), ehi = tab_bl(t, E.e, E.nt - 1);
  o.emin = elo;
  o.emax = ehi;
  const double eps = fmax(fmin(ehi, eps_raw), elo);
  o.eps = eps;
  int lo = 0, hi = E.nt - 1;
  if (eps <= elo) {
    hi = 1;
    ehi = tab_bl(t, E.e, 1);
  } else if (eps >= ehi) {
    lo = E.nt - 2;
    elo = tab_bl(t, E.e, lo);
  } else {
    bool found = false;
    int k = *cell;
    if (k >= 0 && k <= E.nt - 2) {
      double ek = tab_bl(t, E.e, k), ek1 = tab_bl(t, E.e, k + 1);
      if (ek <= eps && eps < ek1) {
        lo = k;
        hi = k + 1;
        elo = ek;
        ehi = ek1;
        found = true;
      }
    }
    if (!found) {
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        double em = tab_bl(t, E.e, mid);
        if (em <= eps) {
          lo = mid;
          elo = em;
        } else {
          hi = mid;
          ehi = em;
        }
      }
    }
  }
  *cell = lo;
  double w = fmin(fmax((eps - elo) / (ehi - elo), 0.0), 1.0);
  double p0 = tab_bl(t, E.p, lo), p1 = tab_bl(t, E.p, lo + 1);
  o.p = fma(w, p1 - p0, p0);
  if (FULL) {
    double c0 = tab_bl(t, E.c, lo), c1 = tab_bl(t, E.c, lo + 1);
    o.cs2 = fma(w, c1 - c0, c0);
    o.T = exp10(fma((double)lo + w, E.dlt, E.lt0));
  } else {
    o.cs2 = o.T = 0.0;
  }
  return o;
}

// (p, eps, cs2) from (rho, T, ye) (table), the cold polytrope (ideal gas), or
// the cold part (hybrid).
DI EosOut eos_T(const Eos& E, double rho, double T, double ye) {
  EosOut o;
  if (E.kind == 2) {
    const HybCold c = hyb_cold(E, rho);
    o.eps = c.eps;
    o.T = 0.0;
    hyb_eps(E, c, rho, c.eps, &o.p, &o.cs2);
    return o;
  }
  if (E.kind == 0) {
    o.p = E.K * pow(rho, E.gam);
    o.eps = o.p / ((E.gam - 1.0) * rho);
    o.T = 0.0;
    o.cs2 = E.gam * o.p / fma(rho, 1.0 + o.eps, o.p);
    return o;
  }
  TabPos t = tab_pos(E, rho, ye);
  int it;
  double wt;
  tab_loc(E, log10(T), E.lt0, E.idlt, E.nt, &it, &wt);
  double a, b;
  a = tab_bl(t, E.p, it);
  b = tab_bl(t, E.p, it + 1);
  o.p = fma(wt, b - a, a);
  a = tab_bl(t, E.e, it);
  b = tab_bl(t, E.e, it + 1);
  o.eps = fma(wt, b - a, a);
  a = tab_bl(t, E.c, it);
  b = tab_bl(t, E.c, it + 1);
  o.cs2 = fma(wt, b - a, a);
  o.T = T;
  return o;
}

// Undensitized (D, DYe, tau, S_i) from primitives (Sec. II B, eq.
// def_con2prim, h = rho (1 + eps) + p); B^i given; gdd = gamma_ij.
DI void prim2con(const double gdd[6], double rho, double eps, double p, const double v[3], double ye,
                 const double B[3], double out[6]) {
  double vd[3], Bd[3];
  lower3(gdd, v, vd);
  lower3(gdd, B, Bd);
  double v2 = v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2];
  double B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  double Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
  double iW2 = 1.0 - v2;
  double W = rsqrt(iW2);
  // 1 / iW2, with the quotient at rest (v = 0: atmosphere points) taken
  // without the division sequence (1 / 1 is exactly 1).
  double W2 = iW2 == 1.0 ? 1.0 : 1.0 / iW2;
  double h = fma(rho, 1.0 + eps, p);
  double D = rho * W;
  double hW2 = h * W2;
  out[0] = D;
  out[1] = D * ye;
  out[2] = hW2 - p + B2 - 0.5 * fma(Bv, Bv, B2 * iW2) - D;
  double hb = hW2 + B2;
  for (int i = 0; i < 3; ++i) out[3 + i] = fma(hb, vd[i], -Bv * Bd[i]);
}

struct C2PFix {
  double D, iD, ye, q, r2, rB, B2, B2rp2, v02, h0;
};

struct C2PEval {
  double f, chi, W, iW, rho, rho_raw, eps, eps_raw, p, T, cs2;
};

// chi(mu) = 1 / (1 + mu B^2) and rbar^2(mu) of the con2prim appendix.
DI void c2p_chi_rbar(const C2PFix& F, double mu, double* chi, double* rbar2) {
  double c = 1.0 / fma(mu, F.B2, 1.0);
  *chi = c;
  *rbar2 = fma(F.r2 * c, c, mu * c * (1.0 + c) * F.rB * F.rB);
}

// Auxiliary function of step 2: f_a(mu) = mu sqrt(h0^2 + rbar^2(mu)) - 1.
DI double c2p_faux(const C2PFix& F, double mu) {
  double chi, rbar2;
  c2p_chi_rbar(F, mu, &chi, &rbar2);
  return fma(mu, sqrt(fma(F.h0, F.h0, rbar2)), -1.0);
}

// Master function of step 3, f(mu) = mu - 1 / (nu_hat + mu rbar^2), with
// the clamps of rho and eps to the EOS validity range.
template <bool FULL>
DI C2PEval c2p_master(const grmhd_params& P, const Eos& E, const C2PFix& F, double mu, int* cell) {
  C2PEval m;
  double rbar2;
  c2p_chi_rbar(F, mu, &m.chi, &rbar2);
  double mc = mu * m.chi;
  double qbar = fma(-0.5, F.B2, F.q) - 0.5 * mc * mc * F.B2rp2;
  double v2 = fmin(mu * mu * rbar2, F.v02);
  double s = 1.0 - v2;
  m.W = rsqrt(s);
  m.iW = s * m.W;
  m.rho_raw = F.D * m.iW;
  m.rho = fmax(fmin(P.rho_max, m.rho_raw), P.rho_min);
  double x = fma(-mu, rbar2, qbar);  // qbar - mu rbar^2
  m.eps_raw = fma(m.W, x + 1.0, -1.0);
  EosClamp eo = eos_clamped<FULL>(E, m.rho, m.eps_raw, F.ye, cell);
  m.eps = eo.eps;
  m.p = eo.p;
  if (FULL) {
    m.T = eo.T;
    m.cs2 = eo.cs2;
  }
  double pr = (E.kind == 0) ? (E.gam - 1.0) * m.eps : m.p / m.rho;  // p / rho
  double h = 1.0 + m.eps + pr;
  double nuA = h * m.iW;
  double nuB = h * (1.0 + x) / (1.0 + m.eps);
  double nu = fmax(nuA, nuB);
  m.f = mu - 1.0 / fma(mu, rbar2, nu);
  return m;
}

// Brent (1973) on [a, b] with f(a) fa, f(b) fb of opposite sign (or zero);
// the root finder the con2prim appendix names for both of its root finds.
// Stops when |c - b| <= 4 eps_mach |b| + xtol or f(b) = 0.  ok = 0 when the
// bracket is invalid or the iteration cap is reached.
template <class Fn>
DI double brent(Fn fn, double a, double b, double fa, double fb, int max_iter, double xtol, int* iters, int* ok) {
  *ok = 0;
  *iters = 0;
  if ((fa > 0.0 && fb > 0.0) || (fa < 0.0 && fb < 0.0)) return b;
  double c = a, fc = fa, d = b - a, e = d;
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
    double tol = fma(2.0 * 2.220446049250313e-16, fabs(b), 0.5 * xtol);
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) {
      *ok = 1;
      *iters = it;
      return b;
    }
    if (it == max_iter) break;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      // Interpolation step p/q (secant if a == c, else inverse quadratic),
      // both scaled by fa fc^2 (the comparisons below are invariant).
      double p, q;
      if (a == c) {
        p = 2.0 * m * fb;
        q = fa - fb;
      } else {
        p = fb * (2.0 * m * fa * (fa - fb) - (b - a) * (fb - fc) * fc);
        q = (fa - fc) * (fb - fc) * (fb - fa);
      }
      if (p > 0.0)
        q = -q;
      else
        p = -p;
      if (2.0 * p < fmin(3.0 * m * q - fabs(tol * q), fabs(e * q))) {
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
    b += (fabs(d) > tol) ? d : (m > 0.0 ? tol : -tol);
    fb = fn(b);
  }
  *iters = max_iter;
  return b;
}

struct C2POut {
  double prim[NP];
  double cons[6];  // corrected densitized D, DYe, tau, S_i (valid when status > 0)
  int status;
  int iters;       // evaluations of f_a and of the master function
  int seeded;      // bit 0: seed usable; bit 1: master bracket from the seed; bit 2: mu_+ not solved
  double mu_plus, mu, W_root;  // roots and W at mu (0 unless the root finds converged; mu_+ 0 if not solved)
  double isg;                  // 1 / sqrt(gamma), for the caller's flux epilogue
};

// con2prim at one point (appendix "Conversion from conserved to primitive
// fields": step 1 rescaled variables, step 2 mu_+ from f_a, step 3 the master
// function's root, step 4 primitives, then the error policy).
// cb: densitized (D, DYe, tau, S_i, B^i); gdd/guu:
// physical metric and inverse; sg = sqrt(gamma); alpha for the BH test.
DI void c2p_point(const grmhd_params& P, const Eos& E, const double cb[9], const double gdd[6], const double guu[6],
                  double sg, double alpha, C2POut& o, const double* seed = nullptr, double delta = 0.0) {
  for (int n = 0; n < NP; ++n) o.prim[n] = 0.0;
  o.iters = 0;
  o.seeded = 0;
  o.mu_plus = o.mu = o.W_root = 0.0;
  const double isg = 1.0 / sg;
  o.isg = isg;
  bool finite = isfinite(sg) && sg > 0.0;
  for (int n = 0; n < 9; ++n) finite = finite && isfinite(cb[n]);
  if (!finite) {
    o.status = -5;
    return;
  }
  double D = cb[0] * isg;
  double B[3] = {cb[6] * isg, cb[7] * isg, cb[8] * isg};
  int status = 0;
  double rho = 0, eps = 0, p = 0, T = 0, cs2 = 0, W = 1, ye = 0;
  double v[3] = {0.0, 0.0, 0.0};
  if (D < P.rho_min) {
    status = 1;
  } else {
    C2PFix F;
    F.D = D;
    F.iD = 1.0 / D;
    F.ye = cb[1] * isg * F.iD;
    F.h0 = P.h0;
    double sc = isg * F.iD;
    F.q = cb[2] * sc;
    double r[3] = {cb[3] * sc, cb[4] * sc, cb[5] * sc};
    double isD = rsqrt(D);
    double Bc[3] = {B[0] * isD, B[1] * isD, B[2] * isD};
    double ru[3], Bcd[3];
    lower3(guu, r, ru);
    lower3(gdd, Bc, Bcd);
    F.r2 = ru[0] * r[0] + ru[1] * r[1] + ru[2] * r[2];
    F.B2 = Bc[0] * Bcd[0] + Bc[1] * Bcd[1] + Bc[2] * Bcd[2];
    F.rB = r[0] * Bc[0] + r[1] * Bc[1] + r[2] * Bc[2];
    F.B2rp2 = fma(F.B2, F.r2, -F.rB * F.rB);
    F.v02 = F.r2 / fma(F.h0, F.h0, F.r2);
    // With a seed s for mu (learned seeder, not part of the paper) the seed
    // bracket is [lo, up] = [s (1 - delta), min(s (1 + delta), 1/h0)].  mu_+
    // only bounds the master root's bracket, and f_a changes sign once, at
    // mu_+: (a) f_a(up) < 0: [lo, up] lies below mu_+, which is not solved;
    // (b) f_a(up) >= 0: mu_+ is solved on (0, up] and the master bracket is
    // [lo, mu_+] (or (0, mu_+] when lo >= mu_+).  A master bracket without a
    // sign change is narrowed by the signs found: f(lo) > 0 gives (0, lo]; in
    // case (a) f(up) < 0 gives [up, mu_+] with mu_+ solved on [up, 1/h0].
    // Every lane goes through the same call sites (one f_a and one master
    // Brent, two bracket evaluations), so mixed warps do not serialise.
    // o.iters counts every evaluation of f_a and of the master function.
    int it1 = 0, it2 = 0, ok1 = 1, ok2 = 1, ev = 0, sd = 0;
    const double muh = 1.0 / F.h0;
    auto fa_fn = [&](double mu) { return c2p_faux(F, mu); };
    int tcell = -1;  // temperature cell of the previous master evaluation
    auto fm_fn = [&](double x) { return c2p_master<false>(P, E, F, x, &tcell).f; };
    double lo = 0.0, up = muh;
    bool seeded = false;
    if (seed && isfinite(seed[1]) && seed[1] > 0.0 && delta > 0.0) {
      double l = seed[1] * (1.0 - delta);
      double u = fmin(seed[1] * (1.0 + delta), muh);
      if (l > 0.0 && l < u) {
        seeded = true;
        lo = l;
        up = u;
        sd |= 1;
      }
    }
    double fa_top = c2p_faux(F, up);
    ev += 1;
    const bool case_a = seeded && fa_top < 0.0;
    bool have_plus = !case_a;
    double mup = up;
    // A non-positive f_a at the upper end (zero analytically, negative by
    // rounding at 1/h0) makes that end point the root.
    if (!case_a && fa_top > 0.0) mup = brent(fa_fn, 0.0, up, -1.0, fa_top, P.max_iter, P.c2p_xtol, &it1, &ok1);
    double x_lo = 0.0, x_hi = mup;
    if (case_a) {
      x_lo = lo;
      x_hi = up;
    } else if (seeded && lo < mup) {
      x_lo = lo;
    }
    double f_lo = fm_fn(x_lo), f_hi = fm_fn(x_hi);
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
      double fa_max = c2p_faux(F, muh);
      ev += 1;
      mup = muh;
      if (fa_max > 0.0) {
        int itx = 0;
        mup = brent(fa_fn, up, muh, fa_top, fa_max, P.max_iter, P.c2p_xtol, &itx, &ok1);
        it1 += itx;
      }
      have_plus = true;
      x_lo = up;
      f_lo = f_hi;
      x_hi = mup;
      f_hi = fm_fn(mup);
      ev += 1;
      from_seed = false;
    }
    // f(mu_+) >= 0 analytically; a rounding-negative value makes mu_+ the root.
    double mu = x_hi;
    if (f_hi > 0.0) mu = brent(fm_fn, x_lo, x_hi, f_lo, f_hi, P.max_iter, P.c2p_xtol, &it2, &ok2);
    if (from_seed) sd |= 2;
    if (!have_plus) sd |= 4;
    o.iters = it1 + it2 + ev;
    o.seeded = sd;
    if (!ok1 || !ok2) {
      o.status = -5;
      return;
    }
    C2PEval m = c2p_master<true>(P, E, F, mu, &tcell);
    o.mu_plus = have_plus ? mup : 0.0;
    o.mu = mu;
    o.W_root = m.W;
    rho = m.rho;
    eps = m.eps;
    p = m.p;
    T = m.T;
    cs2 = m.cs2;
    W = m.W;
    ye = F.ye;
    double mc = mu * m.chi, mrb = mu * F.rB;
    for (int i = 0; i < 3; ++i) v[i] = mc * fma(mrb, Bc[i], ru[i]);
    bool low = (rho < P.rho_low) || (alpha < P.alpha_bh);
    if (m.rho_raw < P.rho_min) {
      status = 1;
    } else {
      int fatal = 0;
      if (m.rho_raw > P.rho_max) fatal = -1;
      double emin = eos_emin(E, rho, ye), emax = eos_emax(E, rho, ye);
      if (!fatal && m.eps_raw < emin) status |= 2;
      if (!fatal && m.eps_raw > emax) {
        if (!low) fatal = -2;
        else status |= 2;
      }
      if (!fatal && W > P.W_max) {
        if (!low) {
          fatal = -3;
        } else {
          double vd[3];
          lower3(gdd, v, vd);
          double vmax = sqrt(1.0 - 1.0 / (P.W_max * P.W_max));
          double s = vmax * rsqrt(v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2]);
          for (int i = 0; i < 3; ++i) v[i] *= s;
          W = P.W_max;
          rho = D / W;
          status |= 4;
        }
      }
      if (!fatal && (ye < P.ye_min || ye > P.ye_max)) {
        if (!low) fatal = -4;
        else {
          ye = P.ye_atmo;
          status |= 8;
        }
      }
      if (fatal) {
        o.status = fatal;
        o.prim[RHO] = rho;
        o.prim[EPS] = eps;
        o.prim[PRS] = p;
        o.prim[VX] = v[0];
        o.prim[VY] = v[1];
        o.prim[VZ] = v[2];
        o.prim[WW] = W;
        o.prim[YE] = ye;
        o.prim[TT] = T;
        o.prim[CS2] = cs2;
        return;
      }
      if (status & (4 | 8)) {
        double e2 = fmax(fmin(eos_emax(E, rho, ye), eps), eos_emin(E, rho, ye));
        EosOut eo = eos_eps(E, rho, e2, ye);
        eps = e2;
        p = eo.p;
        T = eo.T;
        cs2 = eo.cs2;
      }
    }
  }
  if (status & 1) {
    const EosOut eo = E.atmo_set ? E.atmo : eos_T(E, P.rho_atmo, P.T_atmo, P.ye_atmo);
    rho = P.rho_atmo;
    eps = eo.eps;
    p = eo.p;
    T = eo.T;
    cs2 = eo.cs2;
    W = 1.0;
    ye = P.ye_atmo;
    v[0] = v[1] = v[2] = 0.0;
    status = 1;
  }
  o.status = status;
  o.prim[RHO] = rho;
  o.prim[EPS] = eps;
  o.prim[PRS] = p;
  o.prim[VX] = v[0];
  o.prim[VY] = v[1];
  o.prim[VZ] = v[2];
  o.prim[WW] = W;
  o.prim[YE] = ye;
  o.prim[TT] = T;
  o.prim[CS2] = cs2;
  if (status > 0) {
    double c6[6];
    prim2con(gdd, rho, eps, p, v, ye, B, c6);
    for (int n = 0; n < 6; ++n) o.cons[n] = c6[n] * sg;
  }
}

}  // namespace gk
