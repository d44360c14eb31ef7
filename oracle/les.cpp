// Large-eddy-simulation terms of the MHD fluxes: the gradient sub-grid-scale
// (SGS) model (Sec. II B; Appendix "Large Eddy Simulation techniques", eqs.
// sgs_gradient and the closed forms hTauv ... HT that follow it).
//
// TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Nothing in the product
// (the CUDA library and its Python binding) may include, link or call it.
//
// The filtered balance law (Appendix, eq. filtered_conservation_final) moves
// the SGS residual of each flux to the flux side; with the gradient model the
// residual of F^k is -xi H^k, H^k = grad(dF^k/dC) . grad C, so F^k gains
// xi H^k.  The paper gives H in closed form; it is evaluated here with
//   h = rho (1 + eps) + p (enthalpy density), cE = h W^2, Theta = cE + B^2,
//   E = v x B (E_i = sqrt(gamma) [ijk] v^j B^k), W^-2 = 1 / W^2,
//   grad f . grad g = gamma^{ab} d_a f d_b g, indices moved with gamma_ij,
//   xi = gamma^{1/3} dx^2 / 24,
// and the SGS fluxes along k: alpha C_N xi sqrt(gamma) H_N^k (D),
// alpha C_Y xi sqrt(gamma) H_NY^k (DYe), alpha C_T xi sqrt(gamma) H_T^k_i
// (S_i), alpha C_M xi sqrt(gamma) H_M^{ki} (B^i); tau and phi get none (the
// paper lists no tau term).  The derivative d_a of a point value is the
// fourth-order centred difference where its stencil fits in the ghosted
// patch, else the second-order centred one, else the second-order one-sided
// one (the patch's outermost ghost layer).  A flux point whose rest-mass
// density is below les_rho_min gets no SGS flux (the paper states no rule for
// low densities; there the gradient model acts on an almost massless,
// magnetised fluid).
#include <cmath>
#include <vector>

#include "oracle.hpp"

namespace {

enum {
  A_RHO = 0, A_EPS, A_YE, A_D, A_DY, A_IW2, A_H, A_CE, A_TH, A_VB, A_PR, A_PE, A_PY, A_P,
  A_VU, A_VD = A_VU + 3, A_BU = A_VD + 3, A_BD = A_BU + 3, A_EU = A_BD + 3, A_ED = A_EU + 3,
  NAUX = A_ED + 3
};

void metric_at(const double* U, long o, long sf, real gdd[6], real guu[6], real* sg, real* det) {
  real chi = U[F_CHI * sf + o];
  for (int n = 0; n < 6; ++n) gdd[n] = real(U[(F_GT + n) * sf + o]) / chi;
  *det = det_sym(gdd);
  inv_sym(gdd, *det, guu);
  *sg = sqrt(*det);
}

// The point values whose gradients the closed forms use.
int aux_point(const oracle_params* P, const oracle_eos_table* E, const double* U, const double* prim, long o, long sf,
              double* a, long sa) {
  real gdd[6], guu[6], sg, det;
  metric_at(U, o, sf, gdd, guu, &sg, &det);
  real rho = prim[P_RHO * sf + o], eps = prim[P_EPS * sf + o], p = prim[P_P * sf + o];
  real W = prim[P_W * sf + o], ye = prim[P_YE * sf + o];
  real v[3], B[3], vd[3], Bd[3];
  for (int i = 0; i < 3; ++i) {
    v[i] = prim[(P_VX + i) * sf + o];
    B[i] = real(U[(F_B + i) * sf + o]) / sg;
  }
  for (int i = 0; i < 3; ++i) {
    vd[i] = gdd[sym(i, 0)] * v[0] + gdd[sym(i, 1)] * v[1] + gdd[sym(i, 2)] * v[2];
    Bd[i] = gdd[sym(i, 0)] * B[0] + gdd[sym(i, 1)] * B[1] + gdd[sym(i, 2)] * B[2];
  }
  real B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  real vB = v[0] * Bd[0] + v[1] * Bd[1] + v[2] * Bd[2];
  real h = rho * (1.0 + eps) + p;
  real W2 = W * W;
  real cE = h * W2;
  real Ed[3] = {sg * (v[1] * B[2] - v[2] * B[1]), sg * (v[2] * B[0] - v[0] * B[2]), sg * (v[0] * B[1] - v[1] * B[0])};
  real Eu[3];
  for (int i = 0; i < 3; ++i) Eu[i] = guu[sym(i, 0)] * Ed[0] + guu[sym(i, 1)] * Ed[1] + guu[sym(i, 2)] * Ed[2];
  real dpdr, dpde, dpdy;
  if (eos_derivs(P, E, rho, eps, ye, &dpdr, &dpde, &dpdy)) return -1;
  real D = rho * W;
  real vals[NAUX];
  vals[A_RHO] = rho;
  vals[A_EPS] = eps;
  vals[A_YE] = ye;
  vals[A_D] = D;
  vals[A_DY] = D * ye;
  vals[A_IW2] = 1.0 / W2;
  vals[A_H] = h;
  vals[A_CE] = cE;
  vals[A_TH] = cE + B2;
  vals[A_VB] = vB;
  vals[A_PR] = dpdr;
  vals[A_PE] = dpde;
  vals[A_PY] = dpdy;
  vals[A_P] = p;
  for (int i = 0; i < 3; ++i) {
    vals[A_VU + i] = v[i];
    vals[A_VD + i] = vd[i];
    vals[A_BU + i] = B[i];
    vals[A_BD + i] = Bd[i];
    vals[A_EU + i] = Eu[i];
    vals[A_ED + i] = Ed[i];
  }
  for (int f = 0; f < NAUX; ++f) a[f * sa] = dbl(vals[f]);
  return 0;
}

// d_a of a point value A (stride s along a) at index c of an axis with n
// interior points and NG ghosts per side.
real dgrad(const double* A, long o, long s, int c, int n, real dx) {
  if (c - 2 >= -NG && c + 2 <= n + NG - 1)
    return (real(A[o - 2 * s]) - 8.0 * real(A[o - s]) + 8.0 * real(A[o + s]) - real(A[o + 2 * s])) / (12.0 * dx);
  if (c - 1 >= -NG && c + 1 <= n + NG - 1) return (real(A[o + s]) - real(A[o - s])) / (2.0 * dx);
  if (c == -NG) return (-3.0 * real(A[o]) + 4.0 * real(A[o + s]) - real(A[o + 2 * s])) / (2.0 * dx);
  return (3.0 * real(A[o]) - 4.0 * real(A[o - s]) + real(A[o - 2 * s])) / (2.0 * dx);
}

}  // namespace

bool les_on(const oracle_params* P) {
  return P->les_c[0] != 0.0 || P->les_c[1] != 0.0 || P->les_c[2] != 0.0 || P->les_c[3] != 0.0;
}

long les_naux() { return NAUX; }

// Auxiliary point values on every point of the ghosted patch; aux is
// [NAUX][sf].  Returns -1 when the EOS derivatives are unavailable (a table
// kind without its table).
int les_aux_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* U,
                  const double* prim, double* aux) {
  for (int k = -NG; k < G.n[2] + NG; ++k)
    for (int j = -NG; j < G.n[1] + NG; ++j)
      for (int i = -NG; i < G.n[0] + NG; ++i) {
        long o = G.at(i, j, k);
        if (aux_point(P, E, U, prim, o, G.sf, aux + o, G.sf)) return -1;
      }
  return 0;
}

// SGS flux vector along d at point (i, j, k) (added to the MHD flux F^d).
void les_flux_point(const oracle_params* P, const grid& G, const double* U, const double* aux, int i, int j, int k,
                    int d, real F[10]) {
  const long o = G.at(i, j, k);
  for (int n = 0; n < 10; ++n) F[n] = 0.0;
  if (aux[(long)A_RHO * G.sf + o] < P->les_rho_min) return;
  const long st[3] = {1, G.sy, G.sz};
  const int idx[3] = {i, j, k};
  real gr[3][NAUX];
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < NAUX; ++f) gr[a][f] = dgrad(aux + (long)f * G.sf, o, st[a], idx[a], G.n[a], G.dx);
  real gdd[6], guu[6], sg, det;
  metric_at(U, o, G.sf, gdd, guu, &sg, &det);
  auto val = [&](int f) { return real(aux[(long)f * G.sf + o]); };
  auto dot = [&](int f1, int f2) {
    real s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s = s + guu[sym(a, b)] * gr[a][f1] * gr[b][f2];
    return s;
  };
  real rho = val(A_RHO), p = val(A_P), D = val(A_D), DY = val(A_DY), cE = val(A_CE), Th = val(A_TH), vB = val(A_VB);
  real dpdr = val(A_PR), dpde = val(A_PE), dpdy = val(A_PY);
  real W2 = 1.0 / val(A_IW2);
  real vu[3], vd[3], Bu[3], Bd[3], Eu[3], Ed[3];
  for (int a = 0; a < 3; ++a) {
    vu[a] = val(A_VU + a);
    vd[a] = val(A_VD + a);
    Bu[a] = val(A_BU + a);
    Bd[a] = val(A_BD + a);
    Eu[a] = val(A_EU + a);
    Ed[a] = val(A_ED + a);
  }
  real E2 = Ed[0] * Eu[0] + Ed[1] * Eu[1] + Ed[2] * Eu[2];
  // Psi_v^k.
  real sBv = 0.0, sBvB = 0.0, sBvT = 0.0;
  for (int jj = 0; jj < 3; ++jj) {
    sBv = sBv + dot(A_BU + jj, A_VD + jj);
    sBvB = sBvB + Bd[jj] * dot(A_BU + jj, A_VB);
    sBvT = sBvT + Bu[jj] * dot(A_VD + jj, A_TH);
  }
  real Psi_v[3];
  for (int kk = 0; kk < 3; ++kk)
    Psi_v[kk] = 2.0 / Th *
                (dot(A_VB, A_BU + kk) - dot(A_TH, A_VU + kk) + Bu[kk] / cE * (Th * sBv + sBvB - sBvT));
  // Psi_M^{ki} (k: first index).
  real PsiM[3][3];
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii) {
      real t1 = 0.5 * (dot(A_BU + ii, A_VU + kk) - dot(A_BU + kk, A_VU + ii));
      real t2 = 0.5 * (Bu[ii] * dot(A_BU + kk, A_VB) - Bu[kk] * dot(A_BU + ii, A_VB));
      real t3 = 0.5 * (Bu[ii] * dot(A_VU + kk, A_TH) - Bu[kk] * dot(A_VU + ii, A_TH));
      PsiM[kk][ii] = 4.0 / Th * (Th * t1 + t2 - t3);
    }
  real BvPsi = 0.0;
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii) BvPsi = BvPsi + 0.5 * (Bd[ii] * vd[kk] - Bd[kk] * vd[ii]) * PsiM[kk][ii];
  real gBgB = 0.0, gEgE = 0.0, gvgv = 0.0, vPsi = 0.0;
  for (int jj = 0; jj < 3; ++jj) {
    gBgB = gBgB + dot(A_BD + jj, A_BU + jj);
    gEgE = gEgE + dot(A_ED + jj, A_EU + jj);
    gvgv = gvgv + dot(A_VD + jj, A_VU + jj);
    vPsi = vPsi + vd[jj] * Psi_v[jj];
  }
  real Psi_Th = Th / (Th - E2) * (gBgB - gEgE - BvPsi);
  real PsiA = W2 * (p * dpde + rho * rho * dpdr);
  // H_p.
  real giW2 = dot(A_IW2, A_IW2);
  // The Ye terms stand inside the braces with the factor rho, beside the rho
  // and eps terms (reading of the printed H_p, whose Ye line follows the
  // closing brace; that placement fails the gradient-model check).
  real brace = rho * (dot(A_PR, A_RHO) + dot(A_PE, A_EPS)) - 2.0 * dpde * dot(A_RHO, A_EPS) +
               rho * (dot(A_PY, A_YE) - 2.0 / D * dpdy * dot(A_YE, A_D)) -
               (cE * dpde - PsiA) * (W2 / 4.0 * giW2 + dot(A_IW2, A_RHO) / rho) -
               2.0 / W2 * dpde * (gBgB - W2 * W2 * dot(A_IW2, A_H)) -
               (cE * dpde + PsiA) * (vPsi + gvgv + W2 * giW2) +
               Psi_Th / (cE * Th) * ((cE * dpde + PsiA) * (Th - E2) - PsiA * Th / W2);
  real Hp = cE * W2 * (Th - E2) / ((rho * cE - PsiA) * (Th - E2) * W2 + PsiA * Th) * brace;
  real HTh = Psi_Th + Th / (Th - E2) * Hp;
  real Hv[3];
  for (int kk = 0; kk < 3; ++kk) Hv[kk] = Psi_v[kk] - (vu[kk] + vB / cE * Bu[kk]) * HTh / Th;
  // H_M^{ki} = 2 B^[i H_v^k] + 4 grad B^[i . grad v^k].
  real HM[3][3];
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii)
      HM[kk][ii] = 2.0 * 0.5 * (Bu[ii] * Hv[kk] - Bu[kk] * Hv[ii]) +
                   4.0 * 0.5 * (dot(A_BU + ii, A_VU + kk) - dot(A_BU + kk, A_VU + ii));
  // H_E^i = 1/2 eps^i_jk H_M^{jk}, eps_ljk = sqrt(gamma) [ljk].
  real HEd[3] = {sg * 0.5 * (HM[1][2] - HM[2][1]), sg * 0.5 * (HM[2][0] - HM[0][2]), sg * 0.5 * (HM[0][1] - HM[1][0])};
  real HE[3];
  for (int a = 0; a < 3; ++a) HE[a] = guu[sym(a, 0)] * HEd[0] + guu[sym(a, 1)] * HEd[1] + guu[sym(a, 2)] * HEd[2];
  real EHE = Ed[0] * HE[0] + Ed[1] * HE[1] + Ed[2] * HE[2];
  // H_T^{ki}; grad(v^k v^i) by the product rule.
  real HT[3][3];
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii) {
      real gEvv = vu[kk] * dot(A_CE, A_VU + ii) + vu[ii] * dot(A_CE, A_VU + kk);
      HT[kk][ii] = 2.0 * (gEvv + cE * (0.5 * (vu[kk] * Hv[ii] + vu[ii] * Hv[kk]) + dot(A_VU + kk, A_VU + ii)) +
                          vu[kk] * vu[ii] * Hp) -
                   2.0 * (dot(A_BU + kk, A_BU + ii) + dot(A_EU + kk, A_EU + ii) + 0.5 * (Eu[kk] * HE[ii] + Eu[ii] * HE[kk])) +
                   (guu[sym(kk, ii)] - vu[kk] * vu[ii]) * (Hp + gBgB + gEgE + EHE);
    }
  real alpha = U[F_ALP * G.sf + o];
  real xi = cbrt(det) * G.dx * G.dx / 24.0;
  real base = alpha * xi * sg;
  F[0] = base * P->les_c[0] * (2.0 * dot(A_D, A_VU + d) + D * Hv[d]);
  F[1] = base * P->les_c[1] * (2.0 * dot(A_DY, A_VU + d) + DY * Hv[d]);
  F[2] = 0.0;
  for (int a = 0; a < 3; ++a)
    F[3 + a] = base * P->les_c[2] * (gdd[sym(a, 0)] * HT[d][0] + gdd[sym(a, 1)] * HT[d][1] + gdd[sym(a, 2)] * HT[d][2]);
  for (int a = 0; a < 3; ++a) F[6 + a] = base * P->les_c[3] * HM[d][a];
  F[9] = 0.0;
}
