// Ideal-MHD right-hand side (Sec. II B, eq. mhd_system with the LES terms
// and the neutrino sources set to zero): flux vectors, fast magnetosonic
// speed bound (Appendix "Characteristic speeds", eq. fast_waves),
// Lax-Friedrichs splitting with MP5 reconstruction (Sec. III C, eqs.
// flux_decomposition and LLF2), conservative flux difference, and the
// geometric source terms.
#include "oracle.hpp"
#include <cmath>

// Matter projections at one point.  E = tau + D (the CCZ4 energy density),
// S_i, and the stress S_ij of eq. def_cont, all undensitized.
void matter_point(const double* Up, long sf, const double* prp, long spf, real* E, real Si[3], real Sij[6],
                  real gdd[6], real guu[6], real* sqrtg) {
  real gt[6], gtu[6];
  for (int n = 0; n < 6; ++n) gt[n] = Up[(F_GT + n) * sf];
  real chi = Up[F_CHI * sf];
  real det = det_sym(gt);
  inv_sym(gt, det, gtu);
  for (int n = 0; n < 6; ++n) {
    gdd[n] = gt[n] / chi;
    guu[n] = chi * gtu[n];
  }
  real sg = sqrt(det) / (chi * sqrt(chi));
  *sqrtg = sg;
  real isg = 1.0 / sg;
  *E = (real(Up[F_TAU * sf]) + real(Up[F_D * sf])) * isg;
  real v[3], B[3], vd[3], Bd[3];
  for (int a = 0; a < 3; ++a) {
    Si[a] = real(Up[(F_S + a) * sf]) * isg;
    B[a] = real(Up[(F_B + a) * sf]) * isg;
    v[a] = prp[(P_VX + a) * spf];
  }
  for (int a = 0; a < 3; ++a) {
    vd[a] = gdd[sym(a, 0)] * v[0] + gdd[sym(a, 1)] * v[1] + gdd[sym(a, 2)] * v[2];
    Bd[a] = gdd[sym(a, 0)] * B[0] + gdd[sym(a, 1)] * B[1] + gdd[sym(a, 2)] * B[2];
  }
  real B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  real Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
  real W = prp[P_W * spf], p = prp[P_P * spf];
  real iW2 = 1.0 / (W * W);
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      Sij[ab] = 0.5 * (vd[a] * Si[b] + vd[b] * Si[a]) + gdd[ab] * p - 0.5 * iW2 * (2.0 * Bd[a] * Bd[b] - gdd[ab] * B2) -
                0.5 * Bv * (Bd[a] * vd[b] + Bd[b] * vd[a] - gdd[ab] * Bv);
    }
}

// Fast magnetosonic speeds for normal propagation along one axis, eq. fast_waves.
void fast_speeds(real alpha, real betad, real gudd, real vd, real v2, real a2, real* lp, real* lm) {
  real den = 1.0 - v2 * a2;
  real rad = sqrt(a2 * (1.0 - v2) * (den * gudd - (1.0 - a2) * vd * vd));
  real pre = alpha / den;
  *lp = -betad + pre * ((1.0 - a2) * vd + rad);
  *lm = -betad + pre * ((1.0 - a2) * vd - rad);
}

// Flux vector F^d of the ten MHD conserved fields at one point, and the
// largest |lambda^{+-}_fast| along d.
void mhd_flux_point(const oracle_params* P, const double* Up, long sf, const double* prp, long spf, int d,
                    real F[10], real* lam) {
  real E, Si[3], Sij[6], gdd[6], guu[6], sg;
  matter_point(Up, sf, prp, spf, &E, Si, Sij, gdd, guu, &sg);
  real al = Up[F_ALP * sf];
  real be[3], v[3], Bb[3];
  for (int a = 0; a < 3; ++a) {
    be[a] = Up[(F_BET + a) * sf];
    v[a] = prp[(P_VX + a) * spf];
    Bb[a] = Up[(F_B + a) * sf];
  }
  real chi = Up[F_CHI * sf];
  real gt[6], gtu[6];
  for (int n = 0; n < 6; ++n) gt[n] = Up[(F_GT + n) * sf];
  inv_sym(gt, det_sym(gt), gtu);
  real Db = Up[F_D * sf], DYb = Up[F_DYE * sf], taub = Up[F_TAU * sf], phib = Up[F_PHI * sf];
  real Sb[3] = {Up[F_S * sf], Up[(F_S + 1) * sf], Up[(F_S + 2) * sf]};
  real vel = -be[d] + al * v[d];
  F[0] = vel * Db;
  F[1] = vel * DYb;
  real Sbu_d = guu[sym(d, 0)] * Sb[0] + guu[sym(d, 1)] * Sb[1] + guu[sym(d, 2)] * Sb[2];
  F[2] = -be[d] * taub + al * (Sbu_d - Db * v[d]);
  for (int a = 0; a < 3; ++a) {
    real Smix = guu[sym(d, 0)] * Sij[sym(0, a)] + guu[sym(d, 1)] * Sij[sym(1, a)] + guu[sym(d, 2)] * Sij[sym(2, a)];
    F[3 + a] = -be[d] * Sb[a] + al * sg * Smix;
  }
  for (int a = 0; a < 3; ++a)
    F[6 + a] = Bb[a] * (al * v[d] - be[d]) - Bb[d] * (al * v[a] - be[a]) + al * chi * gtu[sym(d, a)] * phib;
  F[9] = -be[d] * phib + al * P->c_b * P->c_b * Bb[d];

  // a^2 = c_s^2 + c_a^2 - c_s^2 c_a^2, c_a^2 = b^2 / (h + b^2), b^2 = B^2/W^2 + (v.B)^2.
  real isg = 1.0 / sg;
  real B[3] = {Bb[0] * isg, Bb[1] * isg, Bb[2] * isg};
  real vd[3], Bd[3];
  for (int a = 0; a < 3; ++a) {
    vd[a] = gdd[sym(a, 0)] * v[0] + gdd[sym(a, 1)] * v[1] + gdd[sym(a, 2)] * v[2];
    Bd[a] = gdd[sym(a, 0)] * B[0] + gdd[sym(a, 1)] * B[1] + gdd[sym(a, 2)] * B[2];
  }
  real v2 = v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2];
  real B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  real Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
  real W = prp[P_W * spf];
  real b2 = B2 / (W * W) + Bv * Bv;
  real h = real(prp[P_RHO * spf]) * (1.0 + real(prp[P_EPS * spf])) + real(prp[P_P * spf]);
  real ca2 = b2 / (h + b2);
  real cs2 = prp[P_CS2 * spf];
  real a2 = cs2 + ca2 - cs2 * ca2;
  real lp, lm;
  fast_speeds(al, be[d], guu[sym(d, d)], v[d], v2, a2, &lp, &lm);
  *lam = fmax(fabs(lp), fabs(lm));
}

// Fhat_{i+1/2} = F^L + F^R with F^L = MP5(F^+_{i-2..i+2}), F^R = MP5(F^-_{i+3..i-1}),
// F^{+-} = (F +- lambda U)/2 and lambda the largest speed over points i-2..i+3.
// Index m = 0..5 holds point i-2+m.
void iface_flux(const real Fm[6][10], const real Um[6][10], const real lam[6], real Fhat[10]) {
  real L = lam[0];
  for (int m = 1; m < 6; ++m) L = fmax(L, lam[m]);
  for (int n = 0; n < 10; ++n) {
    real fp[6], fm[6];
    for (int m = 0; m < 6; ++m) {
      fp[m] = 0.5 * (Fm[m][n] + L * Um[m][n]);
      fm[m] = 0.5 * (Fm[m][n] - L * Um[m][n]);
    }
    real FL = mp5(fp[0], fp[1], fp[2], fp[3], fp[4]);
    real FR = mp5(fm[5], fm[4], fm[3], fm[2], fm[1]);
    Fhat[n] = FL + FR;
  }
}

// Geometric sources of eq. mhd_system (neutrino and LES terms zero).
void mhd_source_point(const oracle_params* P, const geom& Gm, const double* Up, long sf, real src[10]) {
  real al = Gm.alpha, chi = Gm.chi, sg = Gm.sqrtg;
  // Sbar^{ij} = sqrt(gamma) gamma^ik gamma^jl S_kl; trSbar = gamma_jk Sbar^jk; Sbar^j = gamma^jk Sbar_k.
  real Sm[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Sm[a][b] = Gm.guu[sym(a, 0)] * Gm.Sij[sym(0, b)] + Gm.guu[sym(a, 1)] * Gm.Sij[sym(1, b)] +
                 Gm.guu[sym(a, 2)] * Gm.Sij[sym(2, b)];
  real Suu[6];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b)
      Suu[sym(a, b)] = sg * (Sm[a][0] * Gm.guu[sym(0, b)] + Sm[a][1] * Gm.guu[sym(1, b)] + Sm[a][2] * Gm.guu[sym(2, b)]);
  real trS = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) trS += Gm.gdd[sym(a, b)] * Suu[sym(a, b)];
  real Sb[3] = {Up[F_S * sf], Up[(F_S + 1) * sf], Up[(F_S + 2) * sf]};
  real Sbu[3];
  for (int a = 0; a < 3; ++a) Sbu[a] = Gm.guu[sym(a, 0)] * Sb[0] + Gm.guu[sym(a, 1)] * Sb[1] + Gm.guu[sym(a, 2)] * Sb[2];
  real Kt = Gm.Kh + 2.0 * Gm.Th;
  real taub = Up[F_TAU * sf], Db = Up[F_D * sf], phib = Up[F_PHI * sf];
  real Bb[3] = {Up[F_B * sf], Up[(F_B + 1) * sf], Up[(F_B + 2) * sf]};

  src[0] = 0.0;
  src[1] = 0.0;
  real SA = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) SA += Suu[sym(a, b)] * Gm.A[sym(a, b)];
  src[2] = (al / chi) * SA + (al / 3.0) * trS * Kt -
           (Sbu[0] * Gm.dal[0] + Sbu[1] * Gm.dal[1] + Sbu[2] * Gm.dal[2]);
  for (int c = 0; c < 3; ++c) {
    real Sdg = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Sdg += Suu[sym(a, b)] * Gm.dg[c][sym(a, b)];
    real Sdb = Sb[0] * Gm.dbe[0][c] + Sb[1] * Gm.dbe[1][c] + Sb[2] * Gm.dbe[2][c];
    src[3 + c] = (al / (2.0 * chi)) * (Sdg - trS * Gm.dchi[c]) + Sdb - (taub + Db) * Gm.dal[c];
  }
  const real cb2 = P->c_b * P->c_b;
  for (int a = 0; a < 3; ++a) {
    real s = 0.0;
    for (int kk = 0; kk < 3; ++kk) s += Gm.gu[sym(kk, a)] * (-0.5 * al * Gm.dchi[kk] + (chi / cb2) * Gm.dal[kk]);
    src[6 + a] = phib * (-al * (chi * Gm.Gh[a] - 2.0 * Gm.Z[a]) + s);
  }
  src[9] = -al * cb2 * phib * Kt + cb2 * (Bb[0] * Gm.dal[0] + Bb[1] * Gm.dal[1] + Bb[2] * Gm.dal[2]) -
           al * P->kappa_b * phib;
  (void)sg;
}

// Full right-hand side at one interior point with interface fluxes computed
// from scratch (used for sampled points; the patch driver precomputes them).
void rhs_point(const oracle_params* P, const grid& G, const double* U, const double* prim, int i, int j, int k,
               real rhs[NF], const double* aux) {
  geom Gm;
  ccz4_rhs_point(P, G, U, prim, i, j, k, rhs, &Gm);
  const long o = G.at(i, j, k);
  const long st[3] = {1, G.sy, G.sz};
  real src[10];
  mhd_source_point(P, Gm, U + o, G.sf, src);
  real idx = 1.0 / G.dx;
  for (int n = 0; n < 10; ++n) rhs[NST + n] = src[n];
  for (int d = 0; d < 3; ++d) {
    // Pointwise fluxes at i-3..i+3 along d; interfaces i-1/2 and i+1/2.
    real Fm[7][10], Um[7][10], lam[7];
    for (int m = 0; m < 7; ++m) {
      long q = o + (m - 3) * st[d];
      mhd_flux_point(P, U + q, G.sf, prim + q, G.sf, d, Fm[m], &lam[m]);
      if (aux) {
        int ijk[3] = {i, j, k};
        ijk[d] += m - 3;
        real Fs[10];
        les_flux_point(P, G, U, aux, ijk[0], ijk[1], ijk[2], d, Fs);
        for (int n = 0; n < 10; ++n) Fm[m][n] = Fm[m][n] + Fs[n];
      }
      for (int n = 0; n < 10; ++n) Um[m][n] = U[(NST + n) * G.sf + q];
    }
    real Fhm[10], Fhp[10];
    iface_flux((const real(*)[10])&Fm[0], (const real(*)[10])&Um[0], &lam[0], Fhm);  // i-1/2: points i-3..i+2
    iface_flux((const real(*)[10])&Fm[1], (const real(*)[10])&Um[1], &lam[1], Fhp);  // i+1/2: points i-2..i+3
    for (int n = 0; n < 10; ++n) rhs[NST + n] -= (Fhp[n] - Fhm[n]) * idx;
  }
}
