// C entry points of the oracle, loaded through ctypes by oracle/__init__.py.
// Host pointers only.  Patch arrays are field-major [field][z][y][x] with
// ghosted extents (n0 + 6 padded to px, n1 + 6, n2 + 6).
#include <cstring>
#include <vector>
#include "oracle.hpp"
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_COUNT_FLOPS
long long oracle_flops = 0;
#endif

extern "C" {

// Host threads of the OpenMP build's point loops (n <= 0 keeps the default);
// returns the count in effect (1 in the serial builds).
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

long long oracle_flop_counter(int reset) {
#ifdef ORACLE_COUNT_FLOPS
  long long v = oracle_flops;
  if (reset) oracle_flops = 0;
  return v;
#else
  (void)reset;
  return -1;
#endif
}

int oracle_ghost_fill(const oracle_params* P, const int* n, int px, double* U, int nf) {
  ghost_fill(P, make_grid(n, px, 1.0), U, nf);
  return 0;
}

int oracle_init_state(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx,
                      const double* ID, double* U) {
  init_state(P, E, make_grid(n, px, dx), ID, U);
  return 0;
}

int oracle_con2prim_patch(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double* U,
                          double* prim, int8_t* status, long* iters) {
  return c2p_patch(P, E, make_grid(n, px, 1.0), U, prim, status, iters);
}

// E: the table (eos_kind 1; its pressure derivatives enter the LES terms) or null.
int oracle_rhs_patch(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx,
                     const double* U, const double* prim, double* rhs) {
  rhs_patch(P, E, make_grid(n, px, dx), U, prim, rhs, nullptr);
  return 0;
}

// Right-hand side at a list of interior points; out is [npts][32].
int oracle_rhs_points(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx,
                      const double* U, const double* prim, int npts, const int* ijk, double* out) {
  grid G = make_grid(n, px, dx);
  std::vector<double> aux;
  if (les_on(P)) {
    aux.assign((size_t)les_naux() * G.sf, 0.0);
    if (les_aux_patch(P, E, G, U, prim, aux.data())) return -1;
  }
  for (int q = 0; q < npts; ++q) {
    real r[NF];
    rhs_point(P, G, U, prim, ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2], r, aux.empty() ? nullptr : aux.data());
    for (int f = 0; f < NF; ++f) out[(long)q * NF + f] = dbl(r[f]);
  }
  return 0;
}

// dp/drho|eps, dp/deps|rho, dp/dYe at one state (out[3]); -1 when unavailable.
int oracle_eos_derivs(const oracle_params* P, const oracle_eos_table* E, double rho, double eps, double ye,
                      double* out) {
  real a, b, c;
  if (eos_derivs(P, E, rho, eps, ye, &a, &b, &c)) return -1;
  out[0] = dbl(a);
  out[1] = dbl(b);
  out[2] = dbl(c);
  return 0;
}

// LES SGS flux vectors along d (added to the MHD fluxes) at a list of points
// (interior, or ghost points along d); out is [npts][10].  Returns -1 when the
// EOS derivatives are unavailable (eos_kind 1 without its table).
int oracle_les_flux_points(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx,
                           const double* U, const double* prim, int npts, const int* ijk, int d, double* out) {
  grid G = make_grid(n, px, dx);
  std::vector<double> aux((size_t)les_naux() * G.sf, 0.0);
  if (les_aux_patch(P, E, G, U, prim, aux.data())) return -1;
  for (int q = 0; q < npts; ++q) {
    real F[10];
    les_flux_point(P, G, U, aux.data(), ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2], d, F);
    for (int m = 0; m < 10; ++m) out[(long)q * 10 + m] = dbl(F[m]);
  }
  return 0;
}

// Diagnostic geometry at one interior point: Rsum_ij = Rhat_ij + R^chi_ij
// (= R_ij + 2 D_(i Z_j)), its trace R + 2 D_i Z^i, and Gt^i.
int oracle_geom_point(const oracle_params* P, const int* n, int px, double dx, const double* U, const double* prim,
                      int i, int j, int k, double* Rsum6, double* Rtr, double* Gt3, double* Z3) {
  grid G = make_grid(n, px, dx);
  real r[NST];
  geom Gm;
  ccz4_rhs_point(P, G, U, prim, i, j, k, r, &Gm);
  for (int q = 0; q < 6; ++q) Rsum6[q] = dbl(Gm.Rsum[q]);
  *Rtr = dbl(Gm.Rtr);
  for (int a = 0; a < 3; ++a) {
    Gt3[a] = dbl(Gm.Gt[a]);
    Z3[a] = dbl(Gm.Z[a]);
  }
  return 0;
}

int oracle_substep(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx, int stage,
                   double dt, double* Un, double* Ua, double* Ub, double* acc, double* prim, int8_t* status) {
  grid G = make_grid(n, px, dx);
  std::vector<double> k((size_t)NF * G.sf, 0.0);
  return substep(P, E, G, stage, dt, Un, Ua, Ub, acc, prim, status, k.data(), nullptr);
}

// Same as oracle_substep; counts[5] receives the flops of [con2prim,
// pointwise fluxes, interface fluxes, local right-hand side, RK combination]
// (meaningful in the counting build only).
int oracle_substep_counted(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx,
                           int stage, double dt, double* Un, double* Ua, double* Ub, double* acc, double* prim,
                           int8_t* status, long long* counts) {
  grid G = make_grid(n, px, dx);
  std::vector<double> k((size_t)NF * G.sf, 0.0);
  return substep(P, E, G, stage, dt, Un, Ua, Ub, acc, prim, status, k.data(), counts);
}

int oracle_rk4_step(const oracle_params* P, const oracle_eos_table* E, const int* n, int px, double dx, double dt,
                    double* Un, double* Ua, double* Ub, double* acc, double* prim, int8_t* status) {
  grid G = make_grid(n, px, dx);
  std::vector<double> k((size_t)NF * G.sf, 0.0);
  int worst = 0;
  const int nsub = P->rk == 1 ? 3 : 4;
  for (int s = 0; s < nsub; ++s) {
    int w = substep(P, E, G, s, dt, Un, Ua, Ub, acc, prim, status, k.data(), nullptr);
    if (w < worst) worst = w;
  }
  return worst;
}

// ---- pointwise entry points used by the pins ------------------------------
int oracle_c2p_point(const oracle_params* P, const oracle_eos_table* E, const double* cons_bar, const double* gt,
                     double chi, double alpha, double* prim, double* cons_out, int* iters) {
  return c2p_point(P, E, cons_bar, gt, chi, alpha, prim, cons_out, iters);
}

// con2prim on n independent states with a flat metric: cons [n][10]
// (D, DYe, tau, S_i, B^i, phi), prim [n][NP].
int oracle_c2p_flat(const oracle_params* P, const oracle_eos_table* E, long n, const double* cons, double* prim,
                    int8_t* status, int* iters) {
  const double gt[6] = {1, 0, 0, 1, 0, 1};
  int worst = 0;
  ORACLE_PAR_FOR_STATES
  for (long q = 0; q < n; ++q) {
    double co[10];
    int it = 0;
    int st = c2p_point(P, E, cons + q * 10, gt, 1.0, 1.0, prim + q * NP, co, &it);
    if (status) status[q] = (int8_t)st;
    if (iters) iters[q] = it;
    if (st < worst) worst = st;
  }
  return worst;
}

// Master function of flat-metric state cons [10] at mu_+ k / n, k = 1..n,
// into f [n]; returns mu_+ (0: atmosphere, no solve).
double oracle_c2p_master_scan(const oracle_params* P, const oracle_eos_table* E, const double* cons, long n,
                              double* f) {
  return c2p_master_scan(P, E, cons, n, f);
}

// Flat-metric con2prim with optional seeds [n][3] (NULL: plain) and bracket
// half-width delta; roots [n][3] (mu_+, mu, W) and seeded [n] (bit mask of
// seed brackets used) may be NULL.
int oracle_c2p_flat_ext(const oracle_params* P, const oracle_eos_table* E, long n, const double* cons, double* prim,
                        int8_t* status, int* iters, const double* seeds, double delta, double* roots, int8_t* seeded) {
  const double gt[6] = {1, 0, 0, 1, 0, 1};
  int worst = 0;
  ORACLE_PAR_FOR_STATES
  for (long q = 0; q < n; ++q) {
    double co[10];
    int it = 0, sd = 0;
    int st = c2p_point_ext(P, E, cons + q * 10, gt, 1.0, 1.0, prim + q * NP, co, &it, seeds ? seeds + 3 * q : nullptr,
                           delta, roots ? roots + 3 * q : nullptr, &sd);
    if (status) status[q] = (int8_t)st;
    if (iters) iters[q] = it;
    if (seeded) seeded[q] = (int8_t)sd;
    if (st < worst) worst = st;
  }
  return worst;
}

// Undensitized conserved variables (D, DYe, tau, S_i, B^i) from primitives
// (rho, eps, p, v^i, ..., Ye) and the physical metric gamma_ij.
int oracle_prim2con_point(const double* prim, const double* B, const double* gdd, double* cons) {
  real pr[NP], b[3], g[6], c[9];
  for (int q = 0; q < NP; ++q) pr[q] = prim[q];
  for (int q = 0; q < 3; ++q) b[q] = B[q];
  for (int q = 0; q < 6; ++q) g[q] = gdd[q];
  prim2con_point(pr, b, g, c);
  for (int q = 0; q < 9; ++q) cons[q] = dbl(c[q]);
  return 0;
}

int oracle_eos_from_eps(const oracle_params* P, const oracle_eos_table* E, double rho, double eps, double ye,
                        double* out4) {
  eos_state s = eos_from_eps(P, E, rho, eps, ye);
  out4[0] = dbl(s.p);
  out4[1] = dbl(s.eps);
  out4[2] = dbl(s.T);
  out4[3] = dbl(s.cs2);
  return 0;
}

int oracle_eos_from_T(const oracle_params* P, const oracle_eos_table* E, double rho, double T, double ye,
                      double* out4) {
  eos_state s = eos_from_T(P, E, rho, T, ye);
  out4[0] = dbl(s.p);
  out4[1] = dbl(s.eps);
  out4[2] = dbl(s.T);
  out4[3] = dbl(s.cs2);
  return 0;
}

double oracle_fd_d1(const double* u, double dx) { return dbl(fd_d1(u, 1, 1.0 / (12.0 * dx))); }
double oracle_fd_d2(const double* u, double dx) { return dbl(fd_d2(u, 1, 1.0 / (12.0 * dx * dx))); }
// u points at the centre of a 2-D array with row stride ld (axis 2); returns D_2(D_1 u).
double oracle_fd_d11(const double* u, long ld, double dx) { return dbl(fd_d11(u, 1, ld, 1.0 / (144.0 * dx * dx))); }
double oracle_fd_up(const double* u, double beta, double dx) { return dbl(fd_up(u, 1, beta, 1.0 / (12.0 * dx))); }
double oracle_fd_ko(const double* u, double sigma, double dx) { return dbl(fd_ko(u, 1, sigma / (64.0 * dx))); }
double oracle_mp5(const double* f) { return dbl(mp5(f[0], f[1], f[2], f[3], f[4])); }
double oracle_minmod4(double a, double b, double c, double d) { return dbl(minmod4(a, b, c, d)); }

int oracle_fast_speeds(double alpha, double betad, double gudd, double vd, double v2, double a2, double* lp,
                       double* lm) {
  real p, m;
  fast_speeds(alpha, betad, gudd, vd, v2, a2, &p, &m);
  *lp = dbl(p);
  *lm = dbl(m);
  return 0;
}

// Pointwise flux vector along d at one point: U32 (32 evolved fields) and prim (NP).
int oracle_flux_point(const oracle_params* P, const double* U32, const double* prim, int d, double* F10,
                      double* lam) {
  real F[10], l;
  mhd_flux_point(P, U32, 1, prim, 1, d, F, &l);
  for (int q = 0; q < 10; ++q) F10[q] = dbl(F[q]);
  *lam = dbl(l);
  return 0;
}

// Matter projections at one point: E, S_i, S_ij.
int oracle_matter_point(const double* U32, const double* prim, double* E, double* Si, double* Sij) {
  real e, s[3], sij[6], gdd[6], guu[6], sg;
  matter_point(U32, 1, prim, 1, &e, s, sij, gdd, guu, &sg);
  *E = dbl(e);
  for (int q = 0; q < 3; ++q) Si[q] = dbl(s[q]);
  for (int q = 0; q < 6; ++q) Sij[q] = dbl(sij[q]);
  return 0;
}

}  // extern "C"
