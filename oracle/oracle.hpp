// CPU oracle for one Runge-Kutta substep of the GRMHD method of
// "MHDuet: a high-order GRRMHD code for CPU and GPU architectures"
// (arXiv 2510.13965): CCZ4 spacetime right-hand side (Sec. II A), ideal-MHD
// balance laws with Lax-Friedrichs splitting and MP5 reconstruction
// (Sec. II B, Sec. III C), Kastaun con2prim (Appendix "Conversion from
// conserved to primitive fields") and the explicit RK4 tableau (Table RK4).
//
// TEST INFRASTRUCTURE ONLY.  Plain, serial, FP64, compiled with
// -ffp-contract=off.  It shares no code with the CUDA path; only the tests,
// the smoke check and the benchmark's CPU-baseline leg may load it.
//
// Parity unpinned: the value of kappa_2 (named in the K and Theta equations,
// never defined; 0 here) and of the damping, gauge and cleaning constants
// (kappa_z, kappa_c, eta, c_b, kappa_b; the paper bounds some and fixes
// none): values, not formulas, that no closed form in the paper fixes.  Every
// function is pinned by the tests: the Z-term of the conformal Ricci part
// R^chi (taken literally from Sec. II A) and every Theta, Z and kappa_2 term
// of the spacetime equations by the covariant Z4 system they must reproduce.
#pragma once
#include <cstdint>
#include "real.hpp"

extern "C" {

// Physical and numerical parameters.  Field order is mirrored by the ctypes
// Structure in oracle/__init__.py.
struct oracle_params {
  double kappa_z, kappa_c, kappa_2, eta, sigma_ko;  // CCZ4 damping, gauge, KO
  double c_b, kappa_b;                              // divergence cleaning
  double gamma_th, K_atmo;                          // ideal gas Gamma; atmosphere polytrope K
  double rho_atmo, rho_min, rho_low, rho_max;       // con2prim error policy
  double alpha_bh, W_max, eps_max;
  double ye_min, ye_max, ye_atmo, T_atmo;
  double h0;                                        // specific-enthalpy lower bound of the EOS
  double c2p_xtol;                                  // absolute part of the Brent stop rule
  int eos_kind;                                     // 0 ideal gas, 1 table
  int bc;                                           // 0 periodic, 1 linear extrapolation, 2 frozen, 3 hierarchy
  int max_iter;                                     // Brent iteration cap
  int rk;                                           // 0 RK4 (Table RK4), 1 SSP-RK3 (Table RK3SSP)
  // Hybrid EOS (eos_kind 2, Sec. II B): piecewise-polytropic cold part with
  // npoly pieces, K_0 = K_poly, exponents gamma_poly[i], dividing densities
  // rho_poly[i] between pieces i and i + 1; thermal part (gamma_th - 1) rho eps_th.
  int npoly;
  int pad2_;
  double K_poly;
  double rho_poly[3];
  double gamma_poly[4];
  // LES gradient sub-grid-scale model (Sec. II B, Appendix on LES): the
  // coefficients C_N, C_Y, C_T, C_M of the D, DYe, S_i and B^i terms; all
  // zero: no LES terms.
  double les_c[4];
  // No SGS flux at a flux point whose rest-mass density is below this.
  double les_rho_min;
};

// Tabulated EOS on nodes of (log10 rho, log10 T[MeV], Ye); rho varies fastest:
// node (ir, it, iy) is at ((iy * nt) + it) * nr + ir.
struct oracle_eos_table {
  int nr, nt, ny, pad_;
  double lr0, dlr, lt0, dlt, ye0, dye;
  const double* p;
  const double* eps;
  const double* cs2;
};

}  // extern "C"

// ---------------------------------------------------------------------------
// Field indices.  Evolved state: 22 CCZ4 + gauge fields, 10 MHD conserved.
enum {
  F_GT = 0,    // conformal metric  gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz
  F_AT = 6,    // trace-free conformal extrinsic curvature, same ordering
  F_CHI = 12,  // conformal factor chi
  F_KH = 13,   // Khat = K - 2 Theta
  F_TH = 14,   // Theta
  F_GH = 15,   // Gammahat^i
  F_ALP = 18,  // lapse
  F_BET = 19,  // shift beta^i
  F_D = 22,    // densitized conserved: Dbar, DYebar, taubar, Sbar_i, Bbar^i, phibar
  F_DYE = 23,
  F_TAU = 24,
  F_S = 25,
  F_B = 28,
  F_PHI = 31,
  NF = 32,
  NST = 22  // number of spacetime fields
};
// Primitive variables stored per point.
enum { P_RHO = 0, P_EPS, P_P, P_VX, P_VY, P_VZ, P_W, P_YE, P_T, P_CS2, NP };
// Initial-data fields (ADM metric, lapse, shift, fluid primitives).
enum {
  I_G = 0,      // physical metric gamma_ij (6)
  I_K = 6,      // extrinsic curvature K_ij (6)
  I_ALP = 12,
  I_BET = 13,   // beta^i (3)
  I_RHO = 16,
  I_EPS = 17,
  I_V = 18,     // v^i (3), contravariant
  I_B = 21,     // B^i (3), not densitized
  I_YE = 24,
  I_T = 25,
  NID = 26
};
// Symmetric 3x3 index: xx xy xz yy yz zz
static inline int sym(int i, int j) {
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return t[i][j];
}

// Ghosted vertex-centred patch: interior points 0..n-1 per axis, 3 ghosts per side.
struct grid {
  int n[3];
  int px, py, pz;   // ghosted extents (px may be padded)
  long sy, sz, sf;  // strides of y, z and field
  double dx;
  long at(int i, int j, int k) const { return (long)(k + 3) * sz + (long)(j + 3) * sy + (i + 3); }
};
static const int NG = 3;

// Loops over grid points whose iterations are independent (each writes only
// its own point) may run on several host threads in the OpenMP build of the
// same sources (liboracle_omp.so).  No point's arithmetic changes, so that
// build's results are bitwise those of the serial one.
#ifdef _OPENMP
#define ORACLE_PAR_FOR _Pragma("omp parallel for collapse(2) schedule(static)")
#define ORACLE_PAR_FOR_C2P _Pragma("omp parallel for collapse(2) schedule(static) reduction(min : worst) reduction(+ : its)")
#define ORACLE_PAR_FOR_STATES _Pragma("omp parallel for schedule(static) reduction(min : worst)")
#else
#define ORACLE_PAR_FOR
#define ORACLE_PAR_FOR_C2P
#define ORACLE_PAR_FOR_STATES
#endif

// ---- patch-level steps (patch.cpp) ------------------------------------------
grid make_grid(const int n[3], int px, double dx);
// bc 0 periodic, 1 linear extrapolation; bc 2 (frozen) and 3 (mesh-refinement
// hierarchy, filled by amr.cpp) leave the ghosts to the caller.
void ghost_fill(const oracle_params* P, const grid& G, double* U, int nf);
void init_state(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* ID, double* U);
int c2p_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, double* U, double* prim,
              int8_t* status, long* iters_total);
void rhs_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* U, const double* prim,
               double* rhs, long long* counts);
int substep(const oracle_params* P, const oracle_eos_table* E, const grid& G, int stage, double dt, double* Un,
            double* Ua, double* Ub, double* acc, double* prim, int8_t* status, double* krhs, long long* counts);

// ---- EOS (eos.cpp) --------------------------------------------------------
struct eos_state {
  real p, eps, T, cs2;
};
real eos_eps_min(const oracle_params* P, const oracle_eos_table* E, real rho, real ye);
real eos_eps_max(const oracle_params* P, const oracle_eos_table* E, real rho, real ye);
// p, T, cs2 from (rho, eps, ye); eps must lie in [eps_min, eps_max].
eos_state eos_from_eps(const oracle_params* P, const oracle_eos_table* E, real rho, real eps, real ye);
// p, eps, cs2 from (rho, T, ye) (table) or the cold/atmosphere branch for the ideal gas.
eos_state eos_from_T(const oracle_params* P, const oracle_eos_table* E, real rho, real T, real ye);
eos_state eos_atmosphere(const oracle_params* P, const oracle_eos_table* E);
// dp/drho|eps, dp/deps|rho, dp/dYe: analytic for the ideal gas and the
// hybrid EOS, the derivatives of the table's interpolant otherwise (-1
// without a table).
int eos_derivs(const oracle_params* P, const oracle_eos_table* E, real rho, real eps, real ye, real* dpdrho,
               real* dpdeps, real* dpdye);

// ---- metric helpers -------------------------------------------------------
real det_sym(const real g[6]);
void inv_sym(const real g[6], real det, real gu[6]);

// ---- con2prim / prim2con (c2p.cpp) ----------------------------------------
// Undensitized conserved (D, DYe, tau, S_i, B^i) from primitives and gamma_ij.
void prim2con_point(const real prim[NP], const real B[3], const real gdd[6], real cons[9]);
// Full con2prim at one point from densitized conserved variables and the
// conformal metric (gt_ij, chi).  Returns the per-point status code.
int c2p_point(const oracle_params* P, const oracle_eos_table* E, const double cons_bar[10],
              const double gt[6], double chi, double alpha, double prim[NP], double cons_out[10],
              int* iters);
// Same, optionally starting from seeds (mu_+, mu, W) with relative bracket
// half-width delta (only the mu seed is used), and returning (mu_+, mu, W at
// mu) in roots3 (mu_+ is 0 when the seeded start made it unnecessary).
// seeded_ok: bit 0 the seed was usable, bit 1 the final master bracket came
// from the seed, bit 2 mu_+ was not solved.
int c2p_point_ext(const oracle_params* P, const oracle_eos_table* E, const double cons_bar[10],
                  const double gt[6], double chi, double alpha, double prim[NP], double cons_out[10],
                  int* iters, const double* seed3, double delta, double* roots3, int* seeded_ok);
// Master function f(mu) of a flat-metric state at mu_+ k / n, k = 1..n
// (uniqueness pin); returns mu_+, or 0 for a state below rho_min.
double c2p_master_scan(const oracle_params* P, const oracle_eos_table* E, const double cons[10], long n,
                       double* f_out);

// ---- finite differences and MP5 (fd.cpp) ----------------------------------
real fd_d1(const double* u, long s, real inv12dx);
real fd_d2(const double* u, long s, real inv12dx2);
real fd_d11(const double* u, long s1, long s2, real inv144dx2);  // D_2(D_1 u)
real fd_up(const double* u, long s, real beta, real inv12dx);
real fd_ko(const double* u, long s, real coef);
real mp5(real a, real b, real c, real d, real e);
real minmod2(real a, real b);
real minmod4(real a, real b, real c, real d);

// ---- right-hand sides -----------------------------------------------------
// Geometric quantities at one point shared by the CCZ4 and MHD right-hand sides.
struct geom {
  real g[6], gu[6], A[6], gdd[6], guu[6], Sij[6], dg[3][6], Rsum[6];
  real Gh[3], Z[3], Gt[3], dal[3], dchi[3], Si[3], dbe[3][3];
  real chi, alpha, Kh, Th, sqrtg, E, Rtr;
};
// CCZ4 + gauge + KO right-hand side at one interior point (ccz4.cpp).
void ccz4_rhs_point(const oracle_params* P, const grid& G, const double* U, const double* prim,
                    int i, int j, int k, real rhs[NST], geom* out);
// Pointwise MHD flux vector along direction d and max |lambda_fast^{+-}| (mhd.cpp).
void mhd_flux_point(const oracle_params* P, const double* Up, long sf, const double* prp, long spf,
                    int d, real F[10], real* lam);
void fast_speeds(real alpha, real betad, real gudd, real vd, real v2, real a2, real* lp, real* lm);
// Interface flux Fhat_{i+1/2} from pointwise fluxes/conserved/speeds at i-2..i+3.
void iface_flux(const real Fm[6][10], const real Um[6][10], const real lam[6], real Fhat[10]);
// MHD source terms at one interior point.
void mhd_source_point(const oracle_params* P, const geom& Gm, const double* Up, long sf, real src[10]);
// Matter projections: E, S_i, S_ij (lower indices, physical metric) at a point.
void matter_point(const double* Up, long sf, const double* prp, long spf, real* E, real Si[3],
                  real Sij[6], real gdd[6], real guu[6], real* sqrtg);
// Full 32-field right-hand side at one interior point, fluxes computed on the
// fly; aux: the LES point values of the patch (les_aux_patch) or null when
// the LES terms are off.
void rhs_point(const oracle_params* P, const grid& G, const double* U, const double* prim, int i,
               int j, int k, real rhs[NF], const double* aux);
// ---- LES gradient SGS model (les.cpp) ------------------------------------
bool les_on(const oracle_params* P);
long les_naux();
int les_aux_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* U,
                  const double* prim, double* aux);
void les_flux_point(const oracle_params* P, const grid& G, const double* U, const double* aux, int i, int j, int k,
                    int d, real F[10]);
