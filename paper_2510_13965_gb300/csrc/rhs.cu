// Right-hand side kernel: CCZ4 + gauge + Kreiss-Oliger (Sec. II A, Sec. III B)
// and the MHD flux divergence + geometric sources (Sec. II B, Sec. III C) at
// every interior point, with the RK4 stage combination fused as epilogue.
//
// One thread per point.  The kernel is bound by the FP64 pipe, so the
// algebra is arranged for few FP64 operations: second derivatives are
// contracted as soon as they are formed, the Christoffel-product term of
// Rhat_ij is computed through C^n_ka = gt^mn Gt^k_ma, divisions are shared.
#include "kern.cuh"

namespace gk {

constexpr double PI = 3.14159265358979323846;

// One block per work item.  TILED: the items may be tile-shaped (see
// work_point); otherwise every item is a linear chunk of the interior, whose
// decode needs fewer registers (the tile decode adds ~0.1 KB to the spill
// frame at 255 registers).  A loop over items (a persistent pool of blocks)
// is not offered: it raised the spill frame from 0.9 to 1.3 KB.
template <int MODE, int BS, bool TILED>  // MODE 0: write L(U) to rhs[patch]; 1: fused RK stage combination
__global__ void __launch_bounds__(BS) k_rhs(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int reg,
                                                 int stage, double dt, grmhd_params P, double* const* rhs_out) {
  constexpr int LB = BS == 64 ? 6 : (BS == 128 ? 7 : 8);
  {
  Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  int pi, pj, pk;
  if constexpr (TILED) {
    if (!work_point(DOM_INT, G, wk.block, threadIdx.x, LB, pi, pj, pk)) return;
  } else {
    const long long q = (long long)wk.block * blockDim.x + threadIdx.x;
    if (q >= dom_count(DOM_INT, G)) return;
    dom_decode(DOM_INT, G, q, pi, pj, pk);
  }
  const long long o = at(G, pi, pj, pk), sf = G.sf;
  const long long st[3] = {1, G.sy, G.sz};
  const double* U = PD.U[reg] + o;
  const double i12 = G.i12, i12s = G.i12s, i144 = G.i144;
  const double kof = P.sigma_ko * (12.0 / 64.0) * i12;  // sigma / (64 dx)
#define FP(f) (U + (long long)(f) * sf)

  double r[NF];

  // ---- point values ----------------------------------------------------
  double g[6], A[6], Gh[3], be[3];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    g[n] = ld(FP(GT + n));
    A[n] = ld(FP(AT + n));
  }
  const double chi = ld(FP(CHI)), Kh = ld(FP(KH)), Th = ld(FP(TH)), al = ld(FP(ALP));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Gh[a] = ld(FP(GH + a));
    be[a] = ld(FP(BET + a));
  }
  const double detg = det3(g);
  double gu[6];
  inv3(g, 1.0 / detg, gu);

  // ---- one pass over fields and axes: the six centre differences of each
  // (field, axis) feed the one-sided advection derivative, the KO operator
  // and, where the equations need them, D_a and D_aa. ------------------------
  double dg[3][6], dchi[3], dK[3], dTh[3], dGh[3][3], dal[3], dbe[3][3];  // dGh[c][a] = d_a Gh^c
  double Rs[6];               // Rhat_ij, starting with -1/2 gt^mn d_m d_n gt_ij
  double ddchi[6], ddal[6];
  double lb[3], ddb[3];       // gt^jk d_j d_k beta^i ; d_j d_k beta^k
#pragma unroll
  for (int n = 0; n < 6; ++n) Rs[n] = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) lb[c] = ddb[c] = 0.0;
  bool upw[3];
  double wadv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    upw[a] = ipos(be[a]);
    wadv[a] = __longlong_as_double(__double_as_longlong(be[a]) & 0x7fffffffffffffffLL) * i12;  // |beta^a| / (12 dx)
  }
#pragma unroll
  for (int f = 0; f < NST; ++f) {
    const double* u = FP(f);
    const double c = ld(u);
    const bool need_d1 = !(f >= AT && f < AT + 6);
    const bool need_d2 = (f < GT + 6) || f == CHI || f == ALP || (f >= BET && f < BET + 3);
    double adv = 0.0, ko = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long s = st[a];
      const double t1p = ld(u + s) - c, t1m = ld(u - s) - c;
      const double t2p = ld(u + 2 * s) - c, t2m = ld(u - 2 * s) - c;
      const double t3p = ld(u + 3 * s) - c, t3m = ld(u - 3 * s) - c;
      const double s1 = t1p + t1m, s2 = t2p + t2m, s3 = t3p + t3m;
      ko += fma(15.0, s1, fma(-6.0, s2, s3));
      const double x3 = upw[a] ? t3p : t3m, x2 = upw[a] ? t2p : t2m;
      const double x1 = upw[a] ? t1p : t1m, y1 = upw[a] ? t1m : t1p;
      adv = fma(wadv[a], fma(-3.0, y1, fma(18.0, x1, fma(-6.0, x2, x3))), adv);
      if (need_d1) {
        const double d1 = fma(8.0, t1p - t1m, -(t2p - t2m)) * i12;
        if (f < GT + 6) dg[a][f - GT] = d1;
        if (f == CHI) dchi[a] = d1;
        if (f == KH) dK[a] = d1;
        if (f == TH) dTh[a] = d1;
        if (f >= GH && f < GH + 3) dGh[f - GH][a] = d1;
        if (f == ALP) dal[a] = d1;
        if (f >= BET && f < BET + 3) dbe[f - BET][a] = d1;
      }
      if (need_d2) {
        const double d2 = fma(16.0, s1, -s2) * i12s;
        if (f < GT + 6) Rs[f - GT] = fma(-0.5 * gu[S6(a, a)], d2, Rs[f - GT]);
        if (f == CHI) ddchi[S6(a, a)] = d2;
        if (f == ALP) ddal[S6(a, a)] = d2;
        if (f >= BET && f < BET + 3) {
          lb[f - BET] = fma(gu[S6(a, a)], d2, lb[f - BET]);
          if (f - BET == a) ddb[a] += d2;
        }
      }
    }
    r[f] = fma(kof, ko, adv);
  }
  // Mixed second derivatives D_ab = D_b(D_a).
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b) {
      const int ab = S6(a, b);
      const double wgt = -gu[ab] * i144;
#pragma unroll
      for (int n = 0; n < 6; ++n) Rs[n] = fma(wgt, fd11(FP(GT + n), st[a], st[b]), Rs[n]);
      ddchi[ab] = fd11(FP(CHI), st[a], st[b]) * i144;
      ddal[ab] = fd11(FP(ALP), st[a], st[b]) * i144;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double d2 = fd11(FP(BET + c), st[a], st[b]) * i144;
        lb[c] = fma(2.0 * gu[ab], d2, lb[c]);
        if (c == b) ddb[a] += d2;
        if (c == a) ddb[b] += d2;
      }
    }

  // ---- Christoffels ---------------------------------------------------------------
  double Gl[3][6], Gu[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) Gl[k][S6(a, b)] = 0.5 * (dg[a][S6(k, b)] + dg[b][S6(k, a)] - dg[k][S6(a, b)]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int n = 0; n < 6; ++n) Gu[k][n] = fma(gu[S6(k, 0)], Gl[0][n], fma(gu[S6(k, 1)], Gl[1][n], gu[S6(k, 2)] * Gl[2][n]));
  double Gt[3], Z[3];
  {
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double sacc = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) sacc = fma(gu[S6(k, l)], dg[l][S6(a, k)], sacc);
      t[a] = sacc;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Gt[a] = fma(gu[S6(a, 0)], t[0], fma(gu[S6(a, 1)], t[1], gu[S6(a, 2)] * t[2]));
      Z[a] = 0.5 * chi * (Gh[a] - Gt[a]);
    }
  }

  // ---- rest of Rhat_ij: Gammahat terms and Christoffel products --------------------
  {
    // C[n][k][a] = gt^{mn} Gt^k_{ma}
    double C[3][3][3];
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          C[n][k][a] = fma(gu[S6(0, n)], Gu[k][S6(0, a)], fma(gu[S6(1, n)], Gu[k][S6(1, a)], gu[S6(2, n)] * Gu[k][S6(2, a)]));
    // X[a][b] = sum_nk C^n_ka Gt_bkn
    double X[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double sacc = 0.0;
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
          for (int k = 0; k < 3; ++k) sacc = fma(C[n][k][a], Gl[b][S6(k, n)], sacc);
        X[a][b] = sacc;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        double y = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
          for (int k = 0; k < 3; ++k) y = fma(C[n][k][a], Gl[k][S6(n, b)], y);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          t2 = fma(g[S6(k, a)], dGh[k][b], fma(g[S6(k, b)], dGh[k][a], t2));
          t3 = fma(Gh[k], Gl[a][S6(b, k)] + Gl[b][S6(a, k)], t3);
        }
        Rs[S6(a, b)] += 0.5 * (t2 + t3) + X[a][b] + X[b][a] + y;
      }
  }

  // ---- R^chi_ij, D_i D_j alpha ------------------------------------------------
  const double ichi = 1.0 / chi;
  double gdchi[3], gdal[3];  // gt^ij d_j chi, gt^ij d_j alpha
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gdchi[a] = fma(gu[S6(a, 0)], dchi[0], fma(gu[S6(a, 1)], dchi[1], gu[S6(a, 2)] * dchi[2]));
    gdal[a] = fma(gu[S6(a, 0)], dal[0], fma(gu[S6(a, 1)], dal[1], gu[S6(a, 2)] * dal[2]));
  }
  const double dchi2 = dchi[0] * gdchi[0] + dchi[1] * gdchi[1] + dchi[2] * gdchi[2];  // gt^km d_k chi d_m chi
  const double dchida = dal[0] * gdchi[0] + dal[1] * gdchi[1] + dal[2] * gdchi[2];
  const double c5 = 0.5 * (tr6(gu, ddchi) - 1.5 * ichi * dchi2 - (Gh[0] * dchi[0] + Gh[1] * dchi[1] + Gh[2] * dchi[2]));
  double DDa[6];
  {
    double Zl[3];  // Z^k gt_ki
    lower3(g, Z, Zl);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        int ab = S6(a, b);
        double Gdchi = Gu[0][ab] * dchi[0] + Gu[1][ab] * dchi[1] + Gu[2][ab] * dchi[2];
        double Gdal = Gu[0][ab] * dal[0] + Gu[1][ab] * dal[1] + Gu[2][ab] * dal[2];
        double cR = 0.5 * (ddchi[ab] - Gdchi) - 0.25 * ichi * dchi[a] * dchi[b] +
                    ichi * (Zl[a] * dchi[b] + Zl[b] * dchi[a]) + g[ab] * c5;
        Rs[ab] = fma(cR, ichi, Rs[ab]);
        DDa[ab] = ddal[ab] - Gdal + 0.5 * ichi * (dchi[a] * dal[b] + dchi[b] * dal[a] - g[ab] * dchida);
      }
  }
  const double Rtr = chi * tr6(gu, Rs);
  const double DDtr = chi * (tr6(gu, ddal) - (Gt[0] * dal[0] + Gt[1] * dal[1] + Gt[2] * dal[2])) - 0.5 * dchida;

  // ---- matter: E, S_i, S_ij from conserved + primitives -------------------------
  const double* PR = PD.prim + o;
  double gdd[6], guu[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    gdd[n] = g[n] * ichi;
    guu[n] = gu[n] * chi;
  }
  const double sg = sqrt(detg) * ichi * sqrt(ichi);
  const double isg = 1.0 / sg;
  double Sb[3], Bb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Sb[a] = ld(FP(SS + a));
    Bb[a] = ld(FP(BB + a));
  }
  const double Db = ld(FP(DD)), taub = ld(FP(TAU)), phib = ld(FP(PHI));
  const double E = (taub + Db) * isg;
  double Sl[3], Sij[6];
  {
    double v[3] = {ld(PR + VX * sf), ld(PR + VY * sf), ld(PR + VZ * sf)};
    double B[3] = {Bb[0] * isg, Bb[1] * isg, Bb[2] * isg};
    double vd[3], Bd[3];
    lower3(gdd, v, vd);
    lower3(gdd, B, Bd);
    double B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
    double Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
    double W = ld(PR + WW * sf);
    double iW2 = 1.0 / (W * W);
    double piso = ld(PR + PRS * sf) + 0.5 * fma(iW2, B2, Bv * Bv);
#pragma unroll
    for (int a = 0; a < 3; ++a) Sl[a] = Sb[a] * isg;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        double t = 0.5 * fma(vd[a], Sl[b], vd[b] * Sl[a]) - iW2 * Bd[a] * Bd[b] - 0.5 * Bv * fma(Bd[a], vd[b], Bd[b] * vd[a]);
        Sij[S6(a, b)] = fma(gdd[S6(a, b)], piso, t);
      }
  }
  const double Str = chi * tr6(gu, Sij);

  // ---- At algebra ------------------------------------------------------------
  double Am[3][3];  // A^k_j
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int b = 0; b < 3; ++b) Am[k][b] = fma(gu[S6(k, 0)], A[S6(0, b)], fma(gu[S6(k, 1)], A[S6(1, b)], gu[S6(k, 2)] * A[S6(2, b)]));
  double Auu[6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) Auu[S6(a, b)] = fma(Am[a][0], gu[S6(0, b)], fma(Am[a][1], gu[S6(1, b)], Am[a][2] * gu[S6(2, b)]));
  const double Atr = Am[0][0] + Am[1][1] + Am[2][2];
  const double AA = tr6(Auu, A);
  const double divb = dbe[0][0] + dbe[1][1] + dbe[2][2];
  const double Kt = Kh + 2.0 * Th;
  const double Zda = Z[0] * dal[0] + Z[1] * dal[1] + Z[2] * dal[2];
  const double lnd = log(detg);

  // ---- d_t gt_ij, d_t At_ij ----------------------------------------------------
  {
    double X[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) X[n] = fma(al, fma(-8.0 * PI, Sij[n], Rs[n]), -DDa[n]);
    const double Xtr3 = tr6(gu, X) * (1.0 / 3.0);
    const double c_g = al * (2.0 / 3.0) * Atr - (al / 3.0) * P.kappa_c * lnd - (2.0 / 3.0) * divb;  // x gt_ij
    const double c_A = -(al / 3.0) * P.kappa_c * Atr;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        int ab = S6(a, b);
        double lg = 0.0, lA = 0.0, AA2 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          lg = fma(g[S6(a, k)], dbe[k][b], fma(g[S6(k, b)], dbe[k][a], lg));
          lA = fma(A[S6(a, k)], dbe[k][b], fma(A[S6(k, b)], dbe[k][a], lA));
          AA2 = fma(A[S6(a, k)], Am[k][b], AA2);
        }
        r[GT + ab] += lg + fma(g[ab], c_g, -2.0 * al * A[ab]);
        double XTF = fma(-g[ab], Xtr3, X[ab]);
        r[AT + ab] += lA - (2.0 / 3.0) * A[ab] * divb + fma(g[ab], c_A, chi * XTF) + al * fma(Kh, A[ab], -2.0 * AA2);
      }
  }
  // ---- d_t chi, d_t Khat, d_t Theta ---------------------------------------------
  r[CHI] += (2.0 / 3.0) * chi * fma(al, Kt, -divb);
  r[KH] += -DDtr + al * ((1.0 / 3.0) * Kt * Kt + AA + 4.0 * PI * (E + Str) + P.kappa_z * (1.0 - P.kappa_2) * Th) + 2.0 * Zda;
  r[TH] += 0.5 * al * (Rtr + (2.0 / 3.0) * Kh * Kh + (2.0 / 3.0) * Th * (Kh - 2.0 * Th) - AA) - Zda -
           al * (8.0 * PI * E + P.kappa_z * (2.0 + P.kappa_2) * Th);

  // ---- d_t Gammahat^i ---------------------------------------------------------
  {
    const double k23 = (2.0 / 3.0) * divb;
    const double zfac = -2.0 * al * ichi * (P.kappa_z + (2.0 / 3.0) * Kt);
    const double thfac = 2.0 * Th;  // 2 alpha (Theta / alpha) d_j alpha = 2 Theta d_j alpha
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = r[GH + a];
      s -= Gh[0] * dbe[a][0] + Gh[1] * dbe[a][1] + Gh[2] * dbe[a][2];
      s = fma(Gh[a], k23, s);
      s += lb[a] + (1.0 / 3.0) * (gu[S6(a, 0)] * ddb[0] + gu[S6(a, 1)] * ddb[1] + gu[S6(a, 2)] * ddb[2]);
      double Ada = Auu[S6(a, 0)] * dal[0] + Auu[S6(a, 1)] * dal[1] + Auu[S6(a, 2)] * dal[2];
      double Adc = Auu[S6(a, 0)] * dchi[0] + Auu[S6(a, 1)] * dchi[1] + Auu[S6(a, 2)] * dchi[2];
      double gdK = gu[S6(a, 0)] * dK[0] + gu[S6(a, 1)] * dK[1] + gu[S6(a, 2)] * dK[2];
      double gdT = gu[S6(a, 0)] * dTh[0] + gu[S6(a, 1)] * dTh[1] + gu[S6(a, 2)] * dTh[2];
      double gS = guu[S6(a, 0)] * Sl[0] + guu[S6(a, 1)] * Sl[1] + guu[S6(a, 2)] * Sl[2];  // chi gt^ij S_j
      double GA = tr6(Auu, Gu[a]);
      s -= 2.0 * Ada;
      s += 2.0 * al * (GA - 1.5 * ichi * Adc - (2.0 / 3.0) * gdK - 8.0 * PI * ichi * gS - (1.0 / 3.0) * gdT);
      s -= thfac * gdal[a];
      s = fma(zfac, Z[a], s);
      r[GH + a] = s;
    }
  }
  // ---- gauge ---------------------------------------------------------------------
  r[ALP] -= 2.0 * al * Kh;
#pragma unroll
  for (int a = 0; a < 3; ++a) r[BET + a] += fma(0.75, Gh[a], -P.eta * be[a]);

  // ---- MHD: flux divergence and sources -------------------------------------------
  {
    const double idx = G.ihdx;  // 1/(2 dx): the interface arrays hold 2 Fhat
#pragma unroll
    for (int n = 0; n < 10; ++n) r[NST + n] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double* Fh = PD.Fh + (long long)d * 10 * sf + o;
#pragma unroll
      for (int n = 0; n < 10; ++n) r[NST + n] += ld(Fh + n * sf - st[d]) - ld(Fh + n * sf);
    }
#pragma unroll
    for (int n = 0; n < 10; ++n) r[NST + n] *= idx;
    // Sbar^ij = sqrt(gamma) gamma^ik gamma^jl S_kl
    double Sm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Sm[a][b] = fma(guu[S6(a, 0)], Sij[S6(0, b)], fma(guu[S6(a, 1)], Sij[S6(1, b)], guu[S6(a, 2)] * Sij[S6(2, b)]));
    double Suu[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) Suu[S6(a, b)] = sg * fma(Sm[a][0], guu[S6(0, b)], fma(Sm[a][1], guu[S6(1, b)], Sm[a][2] * guu[S6(2, b)]));
    const double trS = sg * (Sm[0][0] + Sm[1][1] + Sm[2][2]);
    double Sbu[3];
    lower3(guu, Sb, Sbu);
    r[TAU] += al * ichi * tr6(Suu, A) + (al / 3.0) * trS * Kt - (Sbu[0] * dal[0] + Sbu[1] * dal[1] + Sbu[2] * dal[2]);
    const double tD = taub + Db;
    const double ac2 = 0.5 * al * ichi;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double Sdg = tr6(Suu, dg[c]);
      double Sdb = Sb[0] * dbe[0][c] + Sb[1] * dbe[1][c] + Sb[2] * dbe[2][c];
      r[SS + c] += ac2 * fma(-trS, dchi[c], Sdg) + Sdb - tD * dal[c];
    }
    const double cb2 = P.c_b * P.c_b;
    const double icb2 = 1.0 / cb2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = fma(-0.5 * al, gdchi[a], chi * icb2 * gdal[a]);
      r[BB + a] += phib * (s - al * (chi * Gh[a] - 2.0 * Z[a]));
    }
    r[PHI] += -al * cb2 * phib * Kt + cb2 * (Bb[0] * dal[0] + Bb[1] * dal[1] + Bb[2] * dal[2]) - al * P.kappa_b * phib;
  }

  // ---- output ------------------------------------------------------------------------
  if (MODE == 0) {
    double* out = rhs_out[wk.patch] + o;
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * sf] = r[f];
  } else if (P.rk == 1) {
    // SSP-RK3 (Table RK3SSP): Y2 = U^n + dt k1 into U[1], Y3 = U^n + dt/4 k1 +
    // dt/4 k2 built in U[2], U[3] = U^n + dt/6 (k1 + k2), U^{n+1} = U[3] + 2 dt/3 k3.
    double* Un = PD.U[0] + o;
    double* Y2 = PD.U[1] + o;
    double* Y3 = PD.U[2] + o;
    double* acc = PD.U[3] + o;
    const double q = 0.25 * dt, s6 = dt / 6.0, t23 = 2.0 * dt / 3.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      long long x = f * sf;
      if (stage == 0) {
        double u = Un[x];
        Y2[x] = fma(dt, r[f], u);
        Y3[x] = fma(q, r[f], u);
        acc[x] = fma(s6, r[f], u);
      } else if (stage == 1) {
        Y3[x] = fma(q, r[f], Y3[x]);
        acc[x] = fma(s6, r[f], acc[x]);
      } else {
        Un[x] = fma(t23, r[f], acc[x]);
      }
    }
  } else {
    double* Un = PD.U[0] + o;
    double* acc = PD.U[3] + o;
    double* out = PD.U[stage == 0 ? 1 : (stage == 1 ? 2 : (stage == 2 ? 1 : 0))] + o;
    const double a1 = stage == 2 ? dt : 0.5 * dt;  // U^(i+1) = U^n + a dt k
    const double bsub = stage == 0 || stage == 3 ? dt / 6.0 : dt / 3.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      long long x = f * sf;
      if (stage == 0) {
        double u = Un[x];
        out[x] = fma(a1, r[f], u);
        acc[x] = fma(bsub, r[f], u);
      } else if (stage < 3) {
        out[x] = fma(a1, r[f], Un[x]);
        acc[x] = fma(bsub, r[f], acc[x]);
      } else {
        out[x] = fma(bsub, r[f], acc[x]);
      }
    }
  }
#undef FP
  }
}

template <int BS, bool TILED>
static void launch_rhs_bs(const PatchDev* pd, const Work* w, int nblk, int reg, int mode, int stage, double dt,
                          const grmhd_params& P, double* const* rhs_dev, cudaStream_t st) {
  if (mode == 0)
    k_rhs<0, BS, TILED><<<nblk, BS, 0, st>>>(pd, w, reg, stage, dt, P, rhs_dev);
  else
    k_rhs<1, BS, TILED><<<nblk, BS, 0, st>>>(pd, w, reg, stage, dt, P, rhs_dev);
}

void launch_rhs(const PatchDev* pd, const Work* w, int nblk, int reg, int mode, int stage, double dt,
                const grmhd_params& P, double* const* rhs_dev, cudaStream_t st, int bs, bool tiled) {
  if (nblk <= 0) return;
  if (tiled) {
    if (bs == 64) launch_rhs_bs<64, true>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
    else if (bs == 256) launch_rhs_bs<256, true>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
    else launch_rhs_bs<128, true>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
  } else if (bs == 64) {
    launch_rhs_bs<64, false>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
  } else if (bs == 256) {
    launch_rhs_bs<256, false>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
  } else {
    launch_rhs_bs<128, false>(pd, w, nblk, reg, mode, stage, dt, P, rhs_dev, st);
  }
}

}  // namespace gk
