// Equations of state for the oracle.
//
// Ideal gas: p = (Gamma - 1) rho eps, the thermal part of the hybrid EOS of
// Sec. II B with no cold part; c_s^2 = Gamma p / h with h = rho (1 + eps) + p
// (the ideal-EOS sound speed quoted with the fast magnetosonic bound,
// Appendix "Characteristic speeds").
//
// Hybrid (eos_kind 2, Sec. II B): p = p_cold(rho) + p_th, eps = eps_cold(rho) +
// eps_th, p_th = (Gamma_th - 1) rho eps_th; the cold part a piecewise
// polytrope p_cold = K_i rho^Gamma_i, eps_cold = a_i + K_i rho^(Gamma_i - 1) /
// (Gamma_i - 1) on rho_{i-1} <= rho <= rho_i, with K_0 given, a_0 = 0 and the
// other K_i, a_i from continuity of p_cold and eps_cold (eq.
// piecewise_p_eps_cold).  eps >= eps_cold(rho) (no negative thermal energy).
//
// Table: p, eps, c_s^2 given at the nodes of a (log10 rho, log10 T, Ye) grid
// and interpolated trilinearly (the tabulated finite-temperature EOS of
// Sec. II B).  T(rho, eps, Ye) is inverted exactly: at fixed (rho, Ye) the
// trilinear interpolant of eps is piecewise linear in log10 T, so a binary
// search over the T nodes followed by one linear solve recovers it.
#include "oracle.hpp"
#include <cmath>

static void locate(real x, double x0, double dx, int n, int* i, real* w) {
  real f = (x - x0) / dx;
  int ii = (int)std::floor(dbl(f));
  if (ii < 0) ii = 0;
  if (ii > n - 2) ii = n - 2;
  real ww = f - (double)ii;
  if (ww < 0.0) ww = 0.0;
  if (ww > 1.0) ww = 1.0;
  *i = ii;
  *w = ww;
}

static inline real lerp(real a, real b, real w) { return a + w * (b - a); }

static inline long node(const oracle_eos_table* E, int ir, int it, int iy) {
  return ((long)iy * E->nt + it) * E->nr + ir;
}

// Bilinear value in (rho, Ye) of array A at temperature node it.
static real bilin(const oracle_eos_table* E, const double* A, int ir, real wr, int it, int iy, real wy) {
  real lo = lerp(A[node(E, ir, it, iy)], A[node(E, ir + 1, it, iy)], wr);
  real hi = lerp(A[node(E, ir, it, iy + 1)], A[node(E, ir + 1, it, iy + 1)], wr);
  return lerp(lo, hi, wy);
}

struct tab_loc {
  int ir, iy;
  real wr, wy;
};

static tab_loc tab_locate(const oracle_eos_table* E, real rho, real ye) {
  tab_loc L;
  locate(log10(rho), E->lr0, E->dlr, E->nr, &L.ir, &L.wr);
  locate(ye, E->ye0, E->dye, E->ny, &L.iy, &L.wy);
  return L;
}

// Piecewise-polytrope constants K_i, a_i from continuity at the dividing
// densities, and the cold part at rho.
struct cold_state {
  real p, eps, gamma;
};
static cold_state hybrid_cold(const oracle_params* P, real rho) {
  double K[4], a[4];
  K[0] = P->K_poly;
  a[0] = 0.0;
  for (int i = 1; i < P->npoly; ++i) {
    double rb = P->rho_poly[i - 1], g0 = P->gamma_poly[i - 1], g1 = P->gamma_poly[i];
    K[i] = K[i - 1] * std::pow(rb, g0 - g1);
    a[i] = a[i - 1] + K[i - 1] / (g0 - 1.0) * std::pow(rb, g0 - 1.0) - K[i] / (g1 - 1.0) * std::pow(rb, g1 - 1.0);
  }
  int i = 0;
  while (i < P->npoly - 1 && rho > P->rho_poly[i]) ++i;
  double g = P->gamma_poly[i];
  cold_state c;
  c.gamma = g;
  c.p = K[i] * pow(rho, g);
  c.eps = a[i] + K[i] / (g - 1.0) * pow(rho, g - 1.0);
  return c;
}

static eos_state hybrid_from_eps(const oracle_params* P, real rho, real eps) {
  cold_state c = hybrid_cold(P, rho);
  real gth = P->gamma_th - 1.0;
  eos_state s;
  s.eps = eps;
  s.p = c.p + gth * rho * (eps - c.eps);
  s.T = 0.0;
  // c_s^2 h = dp/drho|_eps + p / rho^2 dp/deps|_rho, with d eps_cold / d rho = p_cold / rho^2.
  real dpdrho = c.gamma * c.p / rho + gth * (eps - c.eps) - gth * c.p / rho;
  real h = 1.0 + eps + s.p / rho;
  s.cs2 = (dpdrho + gth * s.p / rho) / h;
  return s;
}

// Derivatives of the table's interpolant p(rho, eps, Ye) (the paper takes the
// tabulated EOS's derivatives numerically; these are the table's own): in the
// located cell p = p_lo + w (p_hi - p_lo), w = (eps - e_lo) / (e_hi - e_lo),
// with p_lo, p_hi, e_lo, e_hi the (log10 rho, Ye)-bilinear values at the T
// nodes bracketing eps, as in eos_from_eps.  Along a clamped coordinate
// (outside the table) the interpolant is constant.
static void table_derivs(const oracle_eos_table* E, real rho, real eps, real ye, real* dpdrho, real* dpdeps,
                         real* dpdye) {
  tab_loc L = tab_locate(E, rho, ye);
  const real fr = (log10(rho) - E->lr0) / E->dlr, fy = (ye - E->ye0) / E->dye;
  const bool in_r = fr >= 0.0 && fr <= E->nr - 1.0, in_y = fy >= 0.0 && fy <= E->ny - 1.0;
  int lo = 0, hi = E->nt - 1;
  real elo = bilin(E, E->eps, L.ir, L.wr, lo, L.iy, L.wy);
  real ehi = bilin(E, E->eps, L.ir, L.wr, hi, L.iy, L.wy);
  if (eps <= elo) {
    hi = 1;
    ehi = bilin(E, E->eps, L.ir, L.wr, 1, L.iy, L.wy);
  } else if (eps >= ehi) {
    lo = E->nt - 2;
    elo = bilin(E, E->eps, L.ir, L.wr, lo, L.iy, L.wy);
  } else {
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      real em = bilin(E, E->eps, L.ir, L.wr, mid, L.iy, L.wy);
      if (em <= eps) {
        lo = mid;
        elo = em;
      } else {
        hi = mid;
        ehi = em;
      }
    }
  }
  real wt = (eps - elo) / (ehi - elo);
  const bool in_t = wt >= 0.0 && wt <= 1.0;
  if (wt < 0.0) wt = 0.0;
  if (wt > 1.0) wt = 1.0;
  const real plo = bilin(E, E->p, L.ir, L.wr, lo, L.iy, L.wy);
  const real phi = bilin(E, E->p, L.ir, L.wr, lo + 1, L.iy, L.wy);
  // d/d(log10 rho) and d/dYe of the bilinear value of A at T node it.
  auto d_lr = [&](const double* A, int it) {
    real a = A[node(E, L.ir + 1, it, L.iy)] - A[node(E, L.ir, it, L.iy)];
    real b = A[node(E, L.ir + 1, it, L.iy + 1)] - A[node(E, L.ir, it, L.iy + 1)];
    return lerp(a, b, L.wy) / E->dlr;
  };
  auto d_ye = [&](const double* A, int it) {
    real a = A[node(E, L.ir, it, L.iy + 1)] - A[node(E, L.ir, it, L.iy)];
    real b = A[node(E, L.ir + 1, it, L.iy + 1)] - A[node(E, L.ir + 1, it, L.iy)];
    return lerp(a, b, L.wr) / E->dye;
  };
  auto along = [&](real dplo, real dphi, real delo, real dehi) {
    real dw = in_t ? -(delo + wt * (dehi - delo)) / (ehi - elo) : real(0.0);
    return dplo + wt * (dphi - dplo) + dw * (phi - plo);
  };
  *dpdeps = in_t ? (phi - plo) / (ehi - elo) : real(0.0);
  *dpdrho = in_r ? along(d_lr(E->p, lo), d_lr(E->p, lo + 1), d_lr(E->eps, lo), d_lr(E->eps, lo + 1)) /
                       (rho * std::log(10.0))
                 : real(0.0);
  *dpdye = in_y ? along(d_ye(E->p, lo), d_ye(E->p, lo + 1), d_ye(E->eps, lo), d_ye(E->eps, lo + 1)) : real(0.0);
}

int eos_derivs(const oracle_params* P, const oracle_eos_table* E, real rho, real eps, real ye, real* dpdrho,
               real* dpdeps, real* dpdye) {
  // Partial derivatives of p(rho, eps, Ye) (needed by the LES terms).
  if (P->eos_kind == 1) {
    if (!E) return -1;
    table_derivs(E, rho, eps, ye, dpdrho, dpdeps, dpdye);
    return 0;
  }
  *dpdye = 0.0;
  if (P->eos_kind == 0) {
    *dpdrho = (P->gamma_th - 1.0) * eps;
    *dpdeps = (P->gamma_th - 1.0) * rho;
    return 0;
  }
  if (P->eos_kind == 2) {
    // d/drho of p_c + (Gamma_th - 1) rho (eps - eps_c) with deps_c/drho = p_c / rho^2.
    cold_state c = hybrid_cold(P, rho);
    real gth = P->gamma_th - 1.0;
    *dpdrho = c.gamma * c.p / rho + gth * (eps - c.eps) - gth * c.p / rho;
    *dpdeps = gth * rho;
    return 0;
  }
  return -1;
}

real eos_eps_min(const oracle_params* P, const oracle_eos_table* E, real rho, real ye) {
  if (P->eos_kind == 0) return 0.0;
  if (P->eos_kind == 2) return hybrid_cold(P, rho).eps;
  tab_loc L = tab_locate(E, rho, ye);
  return bilin(E, E->eps, L.ir, L.wr, 0, L.iy, L.wy);
}

real eos_eps_max(const oracle_params* P, const oracle_eos_table* E, real rho, real ye) {
  if (P->eos_kind == 0 || P->eos_kind == 2) return P->eps_max;
  tab_loc L = tab_locate(E, rho, ye);
  return bilin(E, E->eps, L.ir, L.wr, E->nt - 1, L.iy, L.wy);
}

static eos_state ideal_from_eps(const oracle_params* P, real rho, real eps) {
  eos_state s;
  s.eps = eps;
  s.p = (P->gamma_th - 1.0) * rho * eps;
  s.T = 0.0;
  s.cs2 = P->gamma_th * s.p / (rho * (1.0 + eps) + s.p);
  return s;
}

eos_state eos_from_eps(const oracle_params* P, const oracle_eos_table* E, real rho, real eps, real ye) {
  if (P->eos_kind == 0) return ideal_from_eps(P, rho, eps);
  if (P->eos_kind == 2) return hybrid_from_eps(P, rho, eps);
  tab_loc L = tab_locate(E, rho, ye);
  // Binary search for the T interval whose node values bracket eps.
  int lo = 0, hi = E->nt - 1;
  real elo = bilin(E, E->eps, L.ir, L.wr, lo, L.iy, L.wy);
  real ehi = bilin(E, E->eps, L.ir, L.wr, hi, L.iy, L.wy);
  if (eps <= elo) {
    hi = 1;
    ehi = bilin(E, E->eps, L.ir, L.wr, 1, L.iy, L.wy);
  } else if (eps >= ehi) {
    lo = E->nt - 2;
    elo = bilin(E, E->eps, L.ir, L.wr, lo, L.iy, L.wy);
  } else {
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      real em = bilin(E, E->eps, L.ir, L.wr, mid, L.iy, L.wy);
      if (em <= eps) {
        lo = mid;
        elo = em;
      } else {
        hi = mid;
        ehi = em;
      }
    }
  }
  real wt = (eps - elo) / (ehi - elo);
  if (wt < 0.0) wt = 0.0;
  if (wt > 1.0) wt = 1.0;
  eos_state s;
  s.eps = eps;
  real plo = bilin(E, E->p, L.ir, L.wr, lo, L.iy, L.wy);
  real phi = bilin(E, E->p, L.ir, L.wr, lo + 1, L.iy, L.wy);
  s.p = lerp(plo, phi, wt);
  real clo = bilin(E, E->cs2, L.ir, L.wr, lo, L.iy, L.wy);
  real chi = bilin(E, E->cs2, L.ir, L.wr, lo + 1, L.iy, L.wy);
  s.cs2 = lerp(clo, chi, wt);
  s.T = pow(10.0, E->lt0 + (lo + wt) * E->dlt);
  return s;
}

eos_state eos_from_T(const oracle_params* P, const oracle_eos_table* E, real rho, real T, real ye) {
  if (P->eos_kind == 0) {
    // Ideal gas has no temperature: the cold polytrope p = K rho^Gamma is used.
    real p = P->K_atmo * pow(rho, P->gamma_th);
    return ideal_from_eps(P, rho, p / ((P->gamma_th - 1.0) * rho));
  }
  if (P->eos_kind == 2) return hybrid_from_eps(P, rho, hybrid_cold(P, rho).eps);  // cold: no temperature
  tab_loc L = tab_locate(E, rho, ye);
  int it;
  real wt;
  locate(log10(T), E->lt0, E->dlt, E->nt, &it, &wt);
  eos_state s;
  s.T = T;
  s.p = lerp(bilin(E, E->p, L.ir, L.wr, it, L.iy, L.wy), bilin(E, E->p, L.ir, L.wr, it + 1, L.iy, L.wy), wt);
  s.eps = lerp(bilin(E, E->eps, L.ir, L.wr, it, L.iy, L.wy), bilin(E, E->eps, L.ir, L.wr, it + 1, L.iy, L.wy), wt);
  s.cs2 = lerp(bilin(E, E->cs2, L.ir, L.wr, it, L.iy, L.wy), bilin(E, E->cs2, L.ir, L.wr, it + 1, L.iy, L.wy), wt);
  return s;
}

eos_state eos_atmosphere(const oracle_params* P, const oracle_eos_table* E) {
  return eos_from_T(P, E, P->rho_atmo, P->T_atmo, P->ye_atmo);
}

real det_sym(const real g[6]) {
  return g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
         g[2] * (g[1] * g[4] - g[3] * g[2]);
}

void inv_sym(const real g[6], real det, real gu[6]) {
  real id = 1.0 / det;
  gu[0] = (g[3] * g[5] - g[4] * g[4]) * id;
  gu[1] = (g[2] * g[4] - g[1] * g[5]) * id;
  gu[2] = (g[1] * g[4] - g[2] * g[3]) * id;
  gu[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gu[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gu[5] = (g[0] * g[3] - g[1] * g[1]) * id;
}
