// LES gradient sub-grid-scale (SGS) model (Sec. II B; Appendix "Large Eddy
// Simulation techniques": eq. sgs_gradient and the closed forms of H that
// follow it), added to the pointwise MHD fluxes before the reconstruction.
//
// Per the appendix's filtered balance law, flux F^k gains xi H^k with the
// gradient model's H^k = grad(dF^k/dC) . grad C, scaled by the coefficient of
// its equation.  The closed forms are evaluated with
//   h = rho (1 + eps) + p (enthalpy density), cE = h W^2, Theta = cE + B^2,
//   E = v x B (E_i = sqrt(gamma) [ijk] v^j B^k), W^-2 = 1 / W^2,
//   grad f . grad g = gamma^{ab} d_a f d_b g, indices moved with gamma_ij,
//   xi = gamma^{1/3} dx^2 / 24,
// and the fluxes along k gain alpha C xi sqrt(gamma) times H_N^k (D, C_N),
// H_NY^k (DYe, C_Y), H_T^k_i (S_i, C_T), H_M^{ki} (B^i, C_M).  d_a of a point
// value: fourth-order centred where the stencil fits in the ghosted patch,
// else second-order centred, else second-order one-sided (outermost ghosts).
// A flux point whose rest-mass density is below les_rho_min gets no SGS flux
// (the paper states no rule for low densities; in an atmosphere the model
// acts on an almost massless, magnetised fluid).
//
// Two passes after con2prim: k_les_aux writes the point values whose
// gradients are needed ([NAUX][sf] per patch), k_les_flux evaluates the
// closed forms once per flux point and adds the SGS flux for every direction
// the point serves.
#include "kern.cuh"

namespace gk {

namespace {

enum : int {
  A_RHO = 0, A_EPS, A_YE, A_D, A_DY, A_IW2, A_H, A_CE, A_TH, A_VB, A_PR, A_PE, A_PY, A_P,
  A_VU, A_VD = A_VU + 3, A_BU = A_VD + 3, A_BD = A_BU + 3, A_EU = A_BD + 3, A_ED = A_EU + 3,
  NAUX_ = A_ED + 3
};
static_assert(NAUX_ == LES_NAUX, "LES point-value count");

DI void metric(const double* U, long long o, long long sf, double gdd[6], double guu[6], double* sg, double* det) {
  const double ichi = 1.0 / U[CHI * sf + o];
  for (int n = 0; n < 6; ++n) gdd[n] = U[(GT + n) * sf + o] * ichi;
  *det = det3(gdd);
  inv3(gdd, 1.0 / *det, guu);
  *sg = sqrt(*det);
}

// Partial derivatives of the table's interpolant p(rho, eps, Ye): p is
// linear in eps between the two temperature nodes that bracket it, and each
// node value is bilinear in (log10 rho, Ye); moving rho or Ye at fixed eps
// also moves the weight along T through the nodes' eps values.  Along a
// coordinate clamped at the table's edge the interpolant is constant.
DI void tab_derivs(const Eos& E, double rho, double eps, double ye, double* dpdr, double* dpde, double* dpdy) {
  const double fr = (log10(rho) - E.lr0) * E.idlr, fy = (ye - E.ye0) * E.idye;
  const bool in_r = fr >= 0.0 && fr <= E.nr - 1.0, in_y = fy >= 0.0 && fy <= E.ny - 1.0;
  const TabPos t = tab_pos(E, rho, ye);
  int lo;
  double elo, ehi;
  tab_tcell(E, t, eps, &lo, &elo, &ehi);
  const double ide = 1.0 / (ehi - elo);
  double wt = (eps - elo) * ide;
  const bool in_t = wt >= 0.0 && wt <= 1.0;
  wt = fmin(fmax(wt, 0.0), 1.0);
  const double plo = tab_bl(t, E.p, lo), phi = tab_bl(t, E.p, lo + 1);
  // d/d(log10 rho) and d/dYe of the bilinear node value of A at T node it
  auto d_lr = [&](const double* A, int it) {
    const double* q = A + t.b + (long long)it * t.st;
    const double a = ld(q + 1) - ld(q), b = ld(q + t.sy + 1) - ld(q + t.sy);
    return fma(t.wy, b - a, a) * E.idlr;
  };
  auto d_ye = [&](const double* A, int it) {
    const double* q = A + t.b + (long long)it * t.st;
    const double a = ld(q + t.sy) - ld(q), b = ld(q + t.sy + 1) - ld(q + 1);
    return fma(t.wr, b - a, a) * E.idye;
  };
  auto along = [&](double dplo, double dphi, double delo, double dehi) {
    const double dw = in_t ? -fma(wt, dehi - delo, delo) * ide : 0.0;
    return fma(dw, phi - plo, fma(wt, dphi - dplo, dplo));
  };
  *dpde = in_t ? (phi - plo) * ide : 0.0;
  *dpdr = in_r ? along(d_lr(E.p, lo), d_lr(E.p, lo + 1), d_lr(E.e, lo), d_lr(E.e, lo + 1)) / (rho * M_LN10) : 0.0;
  *dpdy = in_y ? along(d_ye(E.p, lo), d_ye(E.p, lo + 1), d_ye(E.e, lo), d_ye(E.e, lo + 1)) : 0.0;
}

// dp/drho|eps, dp/deps|rho and dp/dYe: analytic for the ideal gas and the
// hybrid EOS (the hybrid's cold part: deps_c/drho = p_c / rho^2; dp/dYe = 0);
// for the table (whose derivatives the paper takes numerically) those of the
// interpolant that defines its p(rho, eps, Ye).
DI void eos_derivs(const Eos& E, double rho, double eps, double ye, double* dpdr, double* dpde, double* dpdy) {
  if (E.kind == 1) {
    tab_derivs(E, rho, eps, ye, dpdr, dpde, dpdy);
    return;
  }
  const double gth = E.gam - 1.0;
  if (E.kind == 2) {
    const HybCold c = hyb_cold(E, rho);
    *dpdr = c.g * c.p / rho + gth * (eps - c.eps) - gth * c.p / rho;
  } else {
    *dpdr = gth * eps;
  }
  *dpde = gth * rho;
  *dpdy = 0.0;
}

__global__ void __launch_bounds__(128) k_les_aux(const PatchDev* __restrict__ pd, const Work* __restrict__ w, Eos E,
                                                 int reg) {
  const Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  const long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_ALL, G)) return;
  int i, j, k;
  dom_decode(DOM_ALL, G, q, i, j, k);
  const long long o = at(G, i, j, k), sf = G.sf;
  const double* U = PD.U[reg];
  const double* pr = PD.prim;
  double gdd[6], guu[6], sg, det;
  metric(U, o, sf, gdd, guu, &sg, &det);
  const double rho = pr[RHO * sf + o], eps = pr[EPS * sf + o], p = pr[PRS * sf + o], W = pr[WW * sf + o];
  const double ye = pr[YE * sf + o];
  double v[3], B[3], vd[3], Bd[3];
  const double isg = 1.0 / sg;
  for (int a = 0; a < 3; ++a) {
    v[a] = pr[(VX + a) * sf + o];
    B[a] = U[(BB + a) * sf + o] * isg;
  }
  lower3(gdd, v, vd);
  lower3(gdd, B, Bd);
  const double B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
  const double vB = v[0] * Bd[0] + v[1] * Bd[1] + v[2] * Bd[2];
  const double h = rho * (1.0 + eps) + p;
  const double W2 = W * W;
  const double cE = h * W2;
  const double Ed[3] = {sg * (v[1] * B[2] - v[2] * B[1]), sg * (v[2] * B[0] - v[0] * B[2]),
                        sg * (v[0] * B[1] - v[1] * B[0])};
  double Eu[3];
  lower3(guu, Ed, Eu);
  double dpdr, dpde, dpdy;
  eos_derivs(E, rho, eps, ye, &dpdr, &dpde, &dpdy);
  const double D = rho * W;
  double* A = PD.les + o;
  A[A_RHO * sf] = rho;
  A[A_EPS * sf] = eps;
  A[A_YE * sf] = ye;
  A[A_D * sf] = D;
  A[A_DY * sf] = D * ye;
  A[A_IW2 * sf] = 1.0 / W2;
  A[A_H * sf] = h;
  A[A_CE * sf] = cE;
  A[A_TH * sf] = cE + B2;
  A[A_VB * sf] = vB;
  A[A_PR * sf] = dpdr;
  A[A_PE * sf] = dpde;
  A[A_PY * sf] = dpdy;
  A[A_P * sf] = p;
  for (int a = 0; a < 3; ++a) {
    A[(A_VU + a) * sf] = v[a];
    A[(A_VD + a) * sf] = vd[a];
    A[(A_BU + a) * sf] = B[a];
    A[(A_BD + a) * sf] = Bd[a];
    A[(A_EU + a) * sf] = Eu[a];
    A[(A_ED + a) * sf] = Ed[a];
  }
}

// Stencil of d_a at index c on an axis with n interior points: 0 the
// fourth-order centred difference where it fits in the ghosted patch, else
// 1 the second-order centred one, else the second-order one-sided one at the
// low (2) or high (3) end.  dnum gives the stencil's numerator; the factor
// 1/(12 dx) or 1/(2 dx) is applied with the metric transform.
DI int dkind(int c, int n) {
  if (c - 2 >= -3 && c + 2 <= n + 2) return 0;
  if (c - 1 >= -3 && c + 1 <= n + 2) return 1;
  return c == -3 ? 2 : 3;
}
DI double dnum(const double* A, long long s, int kind) {
  if (kind == 0) return ld(A - 2 * s) - 8.0 * ld(A - s) + 8.0 * ld(A + s) - ld(A + 2 * s);
  if (kind == 1) return ld(A + s) - ld(A - s);
  if (kind == 2) return -3.0 * ld(A) + 4.0 * ld(A + s) - ld(A + 2 * s);
  return 3.0 * ld(A) - 4.0 * ld(A - s) + ld(A - 2 * s);
}

__global__ void __launch_bounds__(128) k_les_flux(const PatchDev* __restrict__ pd, const Work* __restrict__ w,
                                                  int reg, double cN, double cY, double cT, double cM,
                                                  double rho_min) {
  const Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  const long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_ALL, G)) return;
  int i, j, k;
  dom_decode(DOM_ALL, G, q, i, j, k);
  const bool inx = i >= 0 && i < G.n0, iny = j >= 0 && j < G.n1, inz = k >= 0 && k < G.n2;
  const bool need[3] = {iny && inz, inx && inz, inx && iny};
  if (!(need[0] || need[1] || need[2])) return;
  const long long o = at(G, i, j, k), sf = G.sf;
  const double* U = PD.U[reg];
  const double* A = PD.les + o;
  if (A[A_RHO * sf] < rho_min) return;
  const long long st[3] = {1, G.sy, G.sz};
  const int ic[3] = {i, j, k}, nn[3] = {G.n0, G.n1, G.n2};
  int kd[3];
  double sc[3];
  const double idx = 1.0 / G.dx;
  for (int a = 0; a < 3; ++a) {
    kd[a] = dkind(ic[a], nn[a]);
    sc[a] = kd[a] == 0 ? (1.0 / 12.0) * idx : 0.5 * idx;
  }
  double gr[3][LES_NAUX];
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < LES_NAUX; ++f) gr[a][f] = dnum(A + f * sf, st[a], kd[a]);
  double gdd[6], guu[6], sg, det;
  metric(U, o, sf, gdd, guu, &sg, &det);
  // gamma^{ab} = L L^T (Cholesky); with each gradient replaced by L^T d f,
  // grad f . grad g = gamma^{ab} d_a f d_b g is a plain three-term sum.  The
  // stencils' factors sc_a scale L's rows.
  const double L00 = sqrt(guu[0]), L10 = guu[1] / L00, L20 = guu[2] / L00;
  const double L11 = sqrt(guu[3] - L10 * L10), L21 = (guu[4] - L20 * L10) / L11;
  const double L22 = sqrt(guu[5] - L20 * L20 - L21 * L21);
  const double M00 = L00 * sc[0], M10 = L10 * sc[1], M20 = L20 * sc[2];
  const double M11 = L11 * sc[1], M21 = L21 * sc[2], M22 = L22 * sc[2];
  for (int f = 0; f < LES_NAUX; ++f) {
    const double d0 = gr[0][f], d1 = gr[1][f], d2 = gr[2][f];
    gr[0][f] = M00 * d0 + M10 * d1 + M20 * d2;
    gr[1][f] = M11 * d1 + M21 * d2;
    gr[2][f] = M22 * d2;
  }
  auto dot = [&](int f1, int f2) { return gr[0][f1] * gr[0][f2] + gr[1][f1] * gr[1][f2] + gr[2][f1] * gr[2][f2]; };
  auto val = [&](int f) { return A[f * sf]; };
  const double rho = val(A_RHO), p = val(A_P), D = val(A_D), DY = val(A_DY), cE = val(A_CE), Th = val(A_TH);
  const double vB = val(A_VB), dpdr = val(A_PR), dpde = val(A_PE), dpdy = val(A_PY);
  const double W2 = 1.0 / val(A_IW2);
  double vu[3], vd[3], Bu[3], Bd[3], Eu[3], Ed[3];
  for (int a = 0; a < 3; ++a) {
    vu[a] = val(A_VU + a);
    vd[a] = val(A_VD + a);
    Bu[a] = val(A_BU + a);
    Bd[a] = val(A_BD + a);
    Eu[a] = val(A_EU + a);
    Ed[a] = val(A_ED + a);
  }
  const double E2 = Ed[0] * Eu[0] + Ed[1] * Eu[1] + Ed[2] * Eu[2];
  const double iTh = 1.0 / Th, icE = 1.0 / cE;
  double sBv = 0.0, sBvB = 0.0, sBvT = 0.0;
  for (int a = 0; a < 3; ++a) {
    sBv += dot(A_BU + a, A_VD + a);
    sBvB += Bd[a] * dot(A_BU + a, A_VB);
    sBvT += Bu[a] * dot(A_VD + a, A_TH);
  }
  double Psi_v[3];
  for (int a = 0; a < 3; ++a)
    Psi_v[a] = 2.0 * iTh * (dot(A_VB, A_BU + a) - dot(A_TH, A_VU + a) + Bu[a] * icE * (Th * sBv + sBvB - sBvT));
  // grad B^i . grad v^k (all pairs), grad B^k . grad (v.B), grad v^k . grad Theta.
  double gBv[3][3], gBvB[3], gvT[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) gBv[a][b] = dot(A_BU + a, A_VU + b);
    gBvB[a] = dot(A_BU + a, A_VB);
    gvT[a] = dot(A_VU + a, A_TH);
  }
  // B_[i v_k] Psi_M^{ki}, Psi_M^{ki} = 4/Theta [Theta gB^[i.gv^k] + B^[i gB^k].g(vB) - B^[i gv^k].gTheta].
  double BvPsi = 0.0;
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii) {
      const double t1 = 0.5 * (gBv[ii][kk] - gBv[kk][ii]);
      const double t2 = 0.5 * (Bu[ii] * gBvB[kk] - Bu[kk] * gBvB[ii]);
      const double t3 = 0.5 * (Bu[ii] * gvT[kk] - Bu[kk] * gvT[ii]);
      const double PsiM = 4.0 * iTh * (Th * t1 + t2 - t3);
      BvPsi += 0.5 * (Bd[ii] * vd[kk] - Bd[kk] * vd[ii]) * PsiM;
    }
  double gBgB = 0.0, gEgE = 0.0, gvgv = 0.0, vPsi = 0.0;
  for (int a = 0; a < 3; ++a) {
    gBgB += dot(A_BD + a, A_BU + a);
    gEgE += dot(A_ED + a, A_EU + a);
    gvgv += dot(A_VD + a, A_VU + a);
    vPsi += vd[a] * Psi_v[a];
  }
  const double Psi_Th = Th / (Th - E2) * (gBgB - gEgE - BvPsi);
  const double PsiA = W2 * (p * dpde + rho * rho * dpdr);
  const double giW2 = dot(A_IW2, A_IW2);
  // H_p's Ye terms stand inside the braces with the factor rho, beside the
  // rho and eps terms (where the gradient model puts them).
  const double brace = rho * (dot(A_PR, A_RHO) + dot(A_PE, A_EPS)) - 2.0 * dpde * dot(A_RHO, A_EPS) +
                       rho * (dot(A_PY, A_YE) - 2.0 / D * dpdy * dot(A_YE, A_D)) -
                       (cE * dpde - PsiA) * (W2 / 4.0 * giW2 + dot(A_IW2, A_RHO) / rho) -
                       2.0 / W2 * dpde * (gBgB - W2 * W2 * dot(A_IW2, A_H)) -
                       (cE * dpde + PsiA) * (vPsi + gvgv + W2 * giW2) +
                       Psi_Th * icE * iTh * ((cE * dpde + PsiA) * (Th - E2) - PsiA * Th / W2);
  const double Hp = cE * W2 * (Th - E2) / ((rho * cE - PsiA) * (Th - E2) * W2 + PsiA * Th) * brace;
  const double HTh = Psi_Th + Th / (Th - E2) * Hp;
  double Hv[3];
  for (int a = 0; a < 3; ++a) Hv[a] = Psi_v[a] - (vu[a] + vB * icE * Bu[a]) * HTh * iTh;
  double HM[3][3];
  for (int kk = 0; kk < 3; ++kk)
    for (int ii = 0; ii < 3; ++ii)
      HM[kk][ii] = 2.0 * 0.5 * (Bu[ii] * Hv[kk] - Bu[kk] * Hv[ii]) + 4.0 * 0.5 * (gBv[ii][kk] - gBv[kk][ii]);
  const double HEd[3] = {sg * 0.5 * (HM[1][2] - HM[2][1]), sg * 0.5 * (HM[2][0] - HM[0][2]),
                         sg * 0.5 * (HM[0][1] - HM[1][0])};
  double HE[3];
  lower3(guu, HEd, HE);
  const double EHE = Ed[0] * HE[0] + Ed[1] * HE[1] + Ed[2] * HE[2];
  const double xi = cbrt(det) * G.dx * G.dx / 24.0;
  const double base = U[ALP * sf + o] * xi * sg;
  for (int d = 0; d < 3; ++d) {
    if (!need[d]) continue;
    double* F = PD.Fp + (long long)d * 10 * sf + o;
    if (cN != 0.0) F[0] += base * cN * (2.0 * dot(A_D, A_VU + d) + D * Hv[d]);
    if (cY != 0.0) F[sf] += base * cY * (2.0 * dot(A_DY, A_VU + d) + DY * Hv[d]);
    if (cT != 0.0) {
      double HT[3];
      for (int ii = 0; ii < 3; ++ii) {
        const double gEvv = vu[d] * dot(A_CE, A_VU + ii) + vu[ii] * dot(A_CE, A_VU + d);
        HT[ii] = 2.0 * (gEvv + cE * (0.5 * (vu[d] * Hv[ii] + vu[ii] * Hv[d]) + dot(A_VU + d, A_VU + ii)) +
                        vu[d] * vu[ii] * Hp) -
                 2.0 * (dot(A_BU + d, A_BU + ii) + dot(A_EU + d, A_EU + ii) + 0.5 * (Eu[d] * HE[ii] + Eu[ii] * HE[d])) +
                 (guu[S6(d, ii)] - vu[d] * vu[ii]) * (Hp + gBgB + gEgE + EHE);
      }
      double HTl[3];
      lower3(gdd, HT, HTl);
      for (int a = 0; a < 3; ++a) F[(3 + a) * sf] += base * cT * HTl[a];
    }
    if (cM != 0.0)
      for (int a = 0; a < 3; ++a) F[(6 + a) * sf] += base * cM * HM[d][a];
  }
}

}  // namespace

bool les_on(const grmhd_params& P) {
  return P.les_c[0] != 0.0 || P.les_c[1] != 0.0 || P.les_c[2] != 0.0 || P.les_c[3] != 0.0;
}

void launch_les(const PatchDev* pd, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                cudaStream_t st) {
  if (nblk <= 0) return;
  k_les_aux<<<nblk, 128, 0, st>>>(pd, w, E, reg);
  k_les_flux<<<nblk, 128, 0, st>>>(pd, w, reg, P.les_c[0], P.les_c[1], P.les_c[2], P.les_c[3], P.les_rho_min);
}

}  // namespace gk
