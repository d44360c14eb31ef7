// CCZ4 + gauge right-hand side at one interior point, Sec. II A
// (eqs. system1 ... system3 and the Ricci split that follows them), with the
// 4th-order operators of Sec. III B: centred D_i, compact D_ii, mixed
// D_ij = D_j(D_i), one-sided advection derivatives for every beta^k d_k term,
// and Kreiss-Oliger dissipation on all 22 spacetime fields.
#include "oracle.hpp"
#include <cmath>

static const double PI = 3.14159265358979323846;

// Sum over i, j of a^{ij} b_ij for symmetric a, b stored as xx xy xz yy yz zz.
static real contract(const real a[6], const real b[6]) {
  return a[0] * b[0] + a[3] * b[3] + a[5] * b[5] + 2.0 * (a[1] * b[1] + a[2] * b[2] + a[4] * b[4]);
}

void ccz4_rhs_point(const oracle_params* P, const grid& G, const double* U, const double* prim, int i,
                    int j, int k, real rhs[NST], geom* out) {
  const long o = G.at(i, j, k);
  const long sf = G.sf;
  const long st[3] = {1, G.sy, G.sz};
  const real dx = G.dx;
  const real inv12dx = 1.0 / (12.0 * dx);
  const real inv12dx2 = 1.0 / (12.0 * dx * dx);
  const real inv144dx2 = 1.0 / (144.0 * dx * dx);
  const real ko = P->sigma_ko / (64.0 * dx);
  auto F = [&](int f) { return U + (long)f * sf + o; };

  // Point values.
  real g[6], A[6], Gh[3], be[3];
  for (int n = 0; n < 6; ++n) {
    g[n] = *F(F_GT + n);
    A[n] = *F(F_AT + n);
  }
  real chi = *F(F_CHI), Kh = *F(F_KH), Th = *F(F_TH), al = *F(F_ALP);
  for (int a = 0; a < 3; ++a) {
    Gh[a] = *F(F_GH + a);
    be[a] = *F(F_BET + a);
  }

  // Centred first derivatives.
  real dg[3][6], dchi[3], dK[3], dTh[3], dGh[3][3], dal[3], dbe[3][3];
  for (int a = 0; a < 3; ++a) {
    for (int n = 0; n < 6; ++n) dg[a][n] = fd_d1(F(F_GT + n), st[a], inv12dx);
    dchi[a] = fd_d1(F(F_CHI), st[a], inv12dx);
    dK[a] = fd_d1(F(F_KH), st[a], inv12dx);
    dTh[a] = fd_d1(F(F_TH), st[a], inv12dx);
    dal[a] = fd_d1(F(F_ALP), st[a], inv12dx);
    for (int c = 0; c < 3; ++c) {
      dGh[c][a] = fd_d1(F(F_GH + c), st[a], inv12dx);  // d_a Gammahat^c
      dbe[c][a] = fd_d1(F(F_BET + c), st[a], inv12dx);  // d_a beta^c
    }
  }
  // Second derivatives: ddX[sym(a,b)] = d_a d_b X.
  real ddg[6][6], ddchi[6], ddal[6], ddbe[3][6];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      if (a == b) {
        for (int n = 0; n < 6; ++n) ddg[n][ab] = fd_d2(F(F_GT + n), st[a], inv12dx2);
        ddchi[ab] = fd_d2(F(F_CHI), st[a], inv12dx2);
        ddal[ab] = fd_d2(F(F_ALP), st[a], inv12dx2);
        for (int c = 0; c < 3; ++c) ddbe[c][ab] = fd_d2(F(F_BET + c), st[a], inv12dx2);
      } else {
        for (int n = 0; n < 6; ++n) ddg[n][ab] = fd_d11(F(F_GT + n), st[a], st[b], inv144dx2);
        ddchi[ab] = fd_d11(F(F_CHI), st[a], st[b], inv144dx2);
        ddal[ab] = fd_d11(F(F_ALP), st[a], st[b], inv144dx2);
        for (int c = 0; c < 3; ++c) ddbe[c][ab] = fd_d11(F(F_BET + c), st[a], st[b], inv144dx2);
      }
    }
  // Advection terms beta^k d_k u (upwinded) and KO dissipation for all fields.
  real adv[NST], diss[NST];
  for (int f = 0; f < NST; ++f) {
    adv[f] = be[0] * fd_up(F(f), st[0], be[0], inv12dx) + be[1] * fd_up(F(f), st[1], be[1], inv12dx) +
             be[2] * fd_up(F(f), st[2], be[2], inv12dx);
    diss[f] = fd_ko(F(f), st[0], ko) + fd_ko(F(f), st[1], ko) + fd_ko(F(f), st[2], ko);
  }

  // Conformal metric inverse and Christoffel symbols.
  real detg = det_sym(g);
  real gu[6];
  inv_sym(g, detg, gu);
  // Gl[k][sym(i,j)] = Gt_kij = 1/2 (d_i gt_kj + d_j gt_ki - d_k gt_ij), first index lowered.
  real Gl[3][6], Gu[3][6];
  for (int kk = 0; kk < 3; ++kk)
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b)
        Gl[kk][sym(a, b)] = 0.5 * (dg[a][sym(kk, b)] + dg[b][sym(kk, a)] - dg[kk][sym(a, b)]);
  for (int kk = 0; kk < 3; ++kk)
    for (int n = 0; n < 6; ++n)
      Gu[kk][n] = gu[sym(kk, 0)] * Gl[0][n] + gu[sym(kk, 1)] * Gl[1][n] + gu[sym(kk, 2)] * Gl[2][n];
  // Contracted Christoffel Gt^i = gt^{ij} gt^{kl} d_l gt_jk.
  real tj[3], Gt[3];
  for (int a = 0; a < 3; ++a) {
    real s = 0.0;
    for (int kk = 0; kk < 3; ++kk)
      for (int l = 0; l < 3; ++l) s += gu[sym(kk, l)] * dg[l][sym(a, kk)];
    tj[a] = s;
  }
  for (int a = 0; a < 3; ++a) Gt[a] = gu[sym(a, 0)] * tj[0] + gu[sym(a, 1)] * tj[1] + gu[sym(a, 2)] * tj[2];
  // Z^i from Gammahat^i = Gt^i + (2/chi) Z^i.
  real Z[3];
  for (int a = 0; a < 3; ++a) Z[a] = 0.5 * chi * (Gh[a] - Gt[a]);

  // Conformal Ricci Rhat_ij.
  real Rh[6];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      real t1 = -0.5 * contract(gu, ddg[ab]);
      real t2 = 0.0, t3 = 0.0, t4 = 0.0;
      for (int kk = 0; kk < 3; ++kk) {
        t2 += 0.5 * (g[sym(kk, a)] * dGh[kk][b] + g[sym(kk, b)] * dGh[kk][a]);
        t3 += Gh[kk] * 0.5 * (Gl[a][sym(b, kk)] + Gl[b][sym(a, kk)]);
      }
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          real s = 0.0;
          for (int kk = 0; kk < 3; ++kk)
            s += Gu[kk][sym(m, a)] * Gl[b][sym(kk, n)] + Gu[kk][sym(m, b)] * Gl[a][sym(kk, n)] +
                 Gu[kk][sym(m, a)] * Gl[kk][sym(n, b)];
          t4 += gu[sym(m, n)] * s;
        }
      Rh[ab] = t1 + t2 + t3 + t4;
    }
  // chi part R^chi_ij (the paper gives chi R^chi_ij).
  real c5b = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) c5b += gu[sym(a, b)] * (ddchi[sym(a, b)] - (1.5 / chi) * dchi[a] * dchi[b]);
  for (int kk = 0; kk < 3; ++kk) c5b -= Gh[kk] * dchi[kk];
  real Rchi[6];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      real c1 = 0.5 * ddchi[ab];
      real c2 = 0.0, c4 = 0.0;
      for (int kk = 0; kk < 3; ++kk) {
        c2 -= 0.5 * Gu[kk][ab] * dchi[kk];
        c4 += (2.0 / chi) * Z[kk] * 0.5 * (g[sym(kk, a)] * dchi[b] + g[sym(kk, b)] * dchi[a]);
      }
      real c3 = -(1.0 / (4.0 * chi)) * dchi[a] * dchi[b];
      real c5 = 0.5 * g[ab] * c5b;
      Rchi[ab] = (c1 + c2 + c3 + c4 + c5) / chi;
    }
  real Rsum[6];
  for (int n = 0; n < 6; ++n) Rsum[n] = Rh[n] + Rchi[n];
  real Rtr = chi * contract(gu, Rsum);  // R + 2 D_i Z^i

  // Second covariant derivative of the lapse and its trace.
  real gdchida = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) gdchida += gu[sym(a, b)] * dchi[a] * dal[b];
  real DDa[6];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      real s = ddal[ab];
      for (int kk = 0; kk < 3; ++kk) s -= Gu[kk][ab] * dal[kk];
      s += (0.5 / chi) * (dchi[a] * dal[b] + dchi[b] * dal[a] - g[ab] * gdchida);
      DDa[ab] = s;
    }
  real DDtr = chi * contract(gu, ddal);
  for (int kk = 0; kk < 3; ++kk) DDtr -= chi * Gt[kk] * dal[kk];
  DDtr -= 0.5 * gdchida;

  // Matter projections.
  real E, Si[3], Sij[6], gdd[6], guu[6], sqrtg;
  matter_point(U + o, sf, prim + o, sf, &E, Si, Sij, gdd, guu, &sqrtg);
  real Str = chi * contract(gu, Sij);

  // Traces and products of Atilde.
  real Am[3][3];  // Am[k][j] = A^k_j = gt^{kl} A_lj
  for (int kk = 0; kk < 3; ++kk)
    for (int b = 0; b < 3; ++b)
      Am[kk][b] = gu[sym(kk, 0)] * A[sym(0, b)] + gu[sym(kk, 1)] * A[sym(1, b)] + gu[sym(kk, 2)] * A[sym(2, b)];
  real Auu[6];  // A^{ij}
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b)
      Auu[sym(a, b)] = Am[a][0] * gu[sym(0, b)] + Am[a][1] * gu[sym(1, b)] + Am[a][2] * gu[sym(2, b)];
  real Atr = contract(gu, A);
  real AA = contract(Auu, A);
  real divb = dbe[0][0] + dbe[1][1] + dbe[2][2];
  real Kt = Kh + 2.0 * Th;  // K = Khat + 2 Theta
  real lndet = log(detg);
  real Zda = Z[0] * dal[0] + Z[1] * dal[1] + Z[2] * dal[2];

  // d_t gt_ij and d_t At_ij.
  real X[6];
  for (int n = 0; n < 6; ++n) X[n] = al * (Rsum[n] - 8.0 * PI * Sij[n]) - DDa[n];
  real Xtr = contract(gu, X);
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      int ab = sym(a, b);
      real lie_g = 0.0, lie_A = 0.0, AA2 = 0.0;
      for (int kk = 0; kk < 3; ++kk) {
        lie_g += g[sym(a, kk)] * dbe[kk][b] + g[sym(kk, b)] * dbe[kk][a];
        lie_A += A[sym(a, kk)] * dbe[kk][b] + A[sym(kk, b)] * dbe[kk][a];
        AA2 += A[sym(a, kk)] * Am[kk][b];
      }
      rhs[F_GT + ab] = adv[F_GT + ab] + lie_g - (2.0 / 3.0) * g[ab] * divb -
                       2.0 * al * (A[ab] - (1.0 / 3.0) * g[ab] * Atr) - (al / 3.0) * P->kappa_c * g[ab] * lndet;
      real XTF = X[ab] - (1.0 / 3.0) * g[ab] * Xtr;
      rhs[F_AT + ab] = adv[F_AT + ab] + lie_A - (2.0 / 3.0) * A[ab] * divb -
                       (al / 3.0) * P->kappa_c * g[ab] * Atr + chi * XTF + al * (Kh * A[ab] - 2.0 * AA2);
    }
  // d_t chi, d_t Khat, d_t Theta.
  rhs[F_CHI] = adv[F_CHI] + (2.0 / 3.0) * chi * (al * Kt - divb);
  rhs[F_KH] = adv[F_KH] - DDtr +
              al * ((1.0 / 3.0) * Kt * Kt + AA + 4.0 * PI * (E + Str) + P->kappa_z * (1.0 - P->kappa_2) * Th) +
              2.0 * Zda;
  rhs[F_TH] = adv[F_TH] +
              0.5 * al * (Rtr + (2.0 / 3.0) * Kh * Kh + (2.0 / 3.0) * Th * (Kh - 2.0 * Th) - AA) - Zda -
              al * (8.0 * PI * E + P->kappa_z * (2.0 + P->kappa_2) * Th);
  // d_t Gammahat^i.
  real dd_divb[3];  // d_j d_k beta^k
  for (int b = 0; b < 3; ++b) dd_divb[b] = ddbe[0][sym(b, 0)] + ddbe[1][sym(b, 1)] + ddbe[2][sym(b, 2)];
  for (int a = 0; a < 3; ++a) {
    real s = adv[F_GH + a];
    for (int b = 0; b < 3; ++b) s -= Gh[b] * dbe[a][b];
    s += (2.0 / 3.0) * Gh[a] * divb;
    s += contract(gu, ddbe[a]);
    real t = 0.0;
    for (int b = 0; b < 3; ++b) t += gu[sym(a, b)] * dd_divb[b];
    s += (1.0 / 3.0) * t;
    real Ada = 0.0, Adchi = 0.0, GA = contract(Auu, Gu[a]), gdK = 0.0, gS = 0.0, gTh = 0.0;
    for (int b = 0; b < 3; ++b) {
      Ada += Auu[sym(a, b)] * dal[b];
      Adchi += Auu[sym(a, b)] * dchi[b];
      gdK += gu[sym(a, b)] * dK[b];
      gS += gu[sym(a, b)] * Si[b];
      gTh += gu[sym(a, b)] * ((1.0 / 3.0) * dTh[b] + (Th / al) * dal[b]);
    }
    s -= 2.0 * Ada;
    s += 2.0 * al * (GA - (3.0 / (2.0 * chi)) * Adchi - (2.0 / 3.0) * gdK - 8.0 * PI * gS);
    s += 2.0 * al * (-gTh - (1.0 / chi) * Z[a] * (P->kappa_z + (2.0 / 3.0) * Kt));
    rhs[F_GH + a] = s;
  }
  // Gauge: 1+log slicing and the simplified Gamma-freezing shift (beta_0 = 0, f = 1).
  rhs[F_ALP] = adv[F_ALP] - 2.0 * al * Kh;
  for (int a = 0; a < 3; ++a) rhs[F_BET + a] = adv[F_BET + a] + 0.75 * Gh[a] - P->eta * be[a];
  for (int f = 0; f < NST; ++f) rhs[f] += diss[f];

  if (out) {
    for (int n = 0; n < 6; ++n) {
      out->g[n] = g[n];
      out->gu[n] = gu[n];
      out->A[n] = A[n];
      out->gdd[n] = gdd[n];
      out->guu[n] = guu[n];
      out->Sij[n] = Sij[n];
      for (int a = 0; a < 3; ++a) out->dg[a][n] = dg[a][n];
      out->Rsum[n] = Rsum[n];
    }
    for (int a = 0; a < 3; ++a) {
      out->Gh[a] = Gh[a];
      out->Z[a] = Z[a];
      out->Gt[a] = Gt[a];
      out->dal[a] = dal[a];
      out->dchi[a] = dchi[a];
      out->Si[a] = Si[a];
      for (int b = 0; b < 3; ++b) out->dbe[a][b] = dbe[a][b];
    }
    out->chi = chi;
    out->alpha = al;
    out->Kh = Kh;
    out->Th = Th;
    out->sqrtg = sqrtg;
    out->E = E;
    out->Rtr = Rtr;
  }
}
