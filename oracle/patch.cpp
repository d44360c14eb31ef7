// Patch-level drivers of the oracle: ghost fill, initial-data conversion,
// con2prim over a patch, the right-hand side over a patch, and the explicit
// RK4 substep (Table RK4, explicit tableau) of the method of lines (Sec. III A).
#include "oracle.hpp"
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

grid make_grid(const int n[3], int px, double dx) {
  grid G;
  for (int a = 0; a < 3; ++a) G.n[a] = n[a];
  G.px = px;
  G.py = n[1] + 2 * NG;
  G.pz = n[2] + 2 * NG;
  G.sy = px;
  G.sz = (long)px * G.py;
  G.sf = G.sz * G.pz;
  G.dx = dx;
  return G;
}

// Ghost zones, three deep, filled axis by axis (x, then y over the x-extended
// range, then z over the x- and y-extended range) so corners are consistent.
// bc 0: periodic copy.  bc 1: linear extrapolation from the two outermost
// interior points, U_{-m} = (1+m) U_0 - m U_1 (the outer-boundary ghost
// extrapolation of Sec. IV B, taken at first order).
// bc 2: frozen ghosts (the initial data's ghost values, kept by every
// register; see substep) -- nothing to fill here.
// bc 3: ghosts of a mesh-refinement hierarchy, filled by amr.cpp before each
// substep -- nothing to fill here.
static void ghost_fill_bc(int bc, const grid& G, double* U, int nf);

void ghost_fill(const oracle_params* P, const grid& G, double* U, int nf) {
  if (P->bc == 2 || P->bc == 3) return;
  ghost_fill_bc(P->bc, G, U, nf);
}

static void ghost_fill_bc(int bc, const grid& G, double* U, int nf) {
  const long st[3] = {1, G.sy, G.sz};
  for (int ax = 0; ax < 3; ++ax) {
    int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
    int lo1 = (b1 < ax) ? -NG : 0, hi1 = (b1 < ax) ? G.n[b1] + NG : G.n[b1];
    int lo2 = (b2 < ax) ? -NG : 0, hi2 = (b2 < ax) ? G.n[b2] + NG : G.n[b2];
    int n = G.n[ax];
    for (int f = 0; f < nf; ++f)
      for (int c2 = lo2; c2 < hi2; ++c2)
        for (int c1 = lo1; c1 < hi1; ++c1) {
          int idx[3];
          idx[ax] = 0;
          idx[b1] = c1;
          idx[b2] = c2;
          double* base = U + (long)f * G.sf + G.at(idx[0], idx[1], idx[2]);
          long s = st[ax];
          for (int m = 1; m <= NG; ++m) {
            if (bc == 0) {
              base[-m * s] = base[(n - m) * s];
              base[(n - 1 + m) * s] = base[(m - 1) * s];
            } else {
              real lo = (1.0 + m) * real(base[0]) - (double)m * real(base[s]);
              real hi = (1.0 + m) * real(base[(n - 1) * s]) - (double)m * real(base[(n - 2) * s]);
              base[-m * s] = dbl(lo);
              base[(n - 1 + m) * s] = dbl(hi);
            }
          }
        }
  }
}

// Initial data: ADM metric, extrinsic curvature, lapse, shift and fluid
// primitives at every point (ghosts included) -> CCZ4 variables (Sec. II A
// field definitions, Theta = 0, Khat = K) and densitized conserved variables
// (eq. def_con2prim), phi = 0.  Gammahat^i = Gt^i from the same centred D_i
// as the right-hand side, so Z^i = 0 on the grid; then all ghosts are refilled.
void init_state(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* ID, double* U) {
  ORACLE_PAR_FOR
  for (int k = -NG; k < G.n[2] + NG; ++k)
    for (int j = -NG; j < G.n[1] + NG; ++j)
      for (int i = -NG; i < G.n[0] + NG; ++i) {
        long o = G.at(i, j, k);
        auto id = [&](int f) { return real(ID[(long)f * G.sf + o]); };
        real g[6], K[6], gu[6];
        for (int n = 0; n < 6; ++n) {
          g[n] = id(I_G + n);
          K[n] = id(I_K + n);
        }
        real det = det_sym(g);
        inv_sym(g, det, gu);
        real chi = pow(det, -1.0 / 3.0);
        real trK = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) trK += gu[sym(a, b)] * K[sym(a, b)];
        for (int n = 0; n < 6; ++n) {
          U[(F_GT + n) * G.sf + o] = dbl(chi * g[n]);
          U[(F_AT + n) * G.sf + o] = dbl(chi * (K[n] - g[n] * trK / 3.0));
        }
        U[F_CHI * G.sf + o] = dbl(chi);
        U[F_KH * G.sf + o] = dbl(trK);
        U[F_TH * G.sf + o] = 0.0;
        U[F_ALP * G.sf + o] = dbl(id(I_ALP));
        for (int a = 0; a < 3; ++a) U[(F_BET + a) * G.sf + o] = dbl(id(I_BET + a));
        // Fluid.
        real pr[NP];
        real rho = id(I_RHO), ye = id(I_YE);
        eos_state s;
        if (P->eos_kind == 0) {
          s.eps = id(I_EPS);
          s.p = (P->gamma_th - 1.0) * rho * s.eps;
        } else if (P->eos_kind == 2) {
          s = eos_from_eps(P, E, rho, id(I_EPS), ye);
        } else {
          s = eos_from_T(P, E, rho, id(I_T), ye);
        }
        pr[P_RHO] = rho;
        pr[P_EPS] = s.eps;
        pr[P_P] = s.p;
        for (int a = 0; a < 3; ++a) pr[P_VX + a] = id(I_V + a);
        pr[P_YE] = ye;
        real B[3] = {id(I_B), id(I_B + 1), id(I_B + 2)};
        real cons[9];
        prim2con_point(pr, B, g, cons);
        real sg = sqrt(det);
        for (int n = 0; n < 9; ++n) U[(F_D + n) * G.sf + o] = dbl(cons[n] * sg);
        U[F_PHI * G.sf + o] = 0.0;
      }
  // Gammahat^i = gt^{ij} gt^{kl} d_l gt_jk at interior points.
  const long st[3] = {1, G.sy, G.sz};
  const real inv12dx = 1.0 / (12.0 * G.dx);
  ORACLE_PAR_FOR
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long o = G.at(i, j, k);
        real g[6], gu[6], dg[3][6];
        for (int n = 0; n < 6; ++n) {
          g[n] = U[(F_GT + n) * G.sf + o];
          for (int a = 0; a < 3; ++a) dg[a][n] = fd_d1(U + (F_GT + n) * G.sf + o, st[a], inv12dx);
        }
        inv_sym(g, det_sym(g), gu);
        real tj[3];
        for (int a = 0; a < 3; ++a) {
          real s = 0.0;
          for (int kk = 0; kk < 3; ++kk)
            for (int l = 0; l < 3; ++l) s += gu[sym(kk, l)] * dg[l][sym(a, kk)];
          tj[a] = s;
        }
        for (int a = 0; a < 3; ++a)
          U[(F_GH + a) * G.sf + o] = dbl(gu[sym(a, 0)] * tj[0] + gu[sym(a, 1)] * tj[1] + gu[sym(a, 2)] * tj[2]);
      }
  if (P->bc == 2)  // frozen ghosts keep the initial data; Gammahat is extrapolated into them
    ghost_fill_bc(1, G, U + (long)F_GH * G.sf, 3);
  else  // a hierarchy's patch (bc 3) is extrapolated like an outer boundary until its first ghost fill
    ghost_fill_bc(P->bc == 3 ? 1 : P->bc, G, U, NF);
}

// con2prim at every point of the patch, ghosts included; corrected conserved
// variables are written back into U.  Returns the most negative status seen
// (0 when no point failed).
int c2p_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, double* U, double* prim,
              int8_t* status, long* iters_total) {
  int worst = 0;
  long its = 0;
  ORACLE_PAR_FOR_C2P
  for (int k = -NG; k < G.n[2] + NG; ++k)
    for (int j = -NG; j < G.n[1] + NG; ++j)
      for (int i = -NG; i < G.n[0] + NG; ++i) {
        long o = G.at(i, j, k);
        double cb[10], gt[6], pr[NP], co[10];
        for (int n = 0; n < 10; ++n) cb[n] = U[(F_D + n) * G.sf + o];
        for (int n = 0; n < 6; ++n) gt[n] = U[(F_GT + n) * G.sf + o];
        int it = 0;
        int st = c2p_point(P, E, cb, gt, U[F_CHI * G.sf + o], U[F_ALP * G.sf + o], pr, co, &it);
        its += it;
        for (int n = 0; n < NP; ++n) prim[(long)n * G.sf + o] = pr[n];
        for (int n = 0; n < 10; ++n) U[(F_D + n) * G.sf + o] = co[n];
        if (status) status[o] = (int8_t)st;
        if (st < worst) worst = st;
      }
  if (iters_total) *iters_total = its;
  return worst;
}

// Right-hand side at every interior point (rhs has the layout of U; ghost
// entries are left untouched).  Pointwise fluxes and interface fluxes are
// computed once per point / interface, then differenced.
#ifdef ORACLE_COUNT_FLOPS
static long long flops_now() { return oracle_flops; }
#else
static long long flops_now() { return 0; }
#endif

// counts (optional): flops of [pointwise fluxes, interface fluxes, local terms
// (CCZ4 + sources + flux difference)] in the counting build.
void rhs_patch(const oracle_params* P, const oracle_eos_table* E, const grid& G, const double* U, const double* prim,
               double* rhs, long long* counts) {
  long long c0 = flops_now(), c_pt = 0, c_if = 0;
  const long st[3] = {1, G.sy, G.sz};
  const long npts = G.sf;
  // Fhat[d][n][o]: flux at the interface between point o and o + st[d].
  std::vector<double> Fhat((size_t)3 * 10 * npts, 0.0);
  std::vector<double> Fp((size_t)10 * npts), Lp((size_t)npts);
  // LES gradient SGS model: point values whose gradients the SGS fluxes use.
  std::vector<double> aux;
  if (les_on(P)) {
    aux.assign((size_t)les_naux() * npts, 0.0);
    les_aux_patch(P, E, G, U, prim, aux.data());
  }
  for (int d = 0; d < 3; ++d) {
    int lo[3] = {0, 0, 0}, hi[3] = {G.n[0], G.n[1], G.n[2]};
    lo[d] = -NG;
    hi[d] = G.n[d] + NG;
    ORACLE_PAR_FOR
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          long o = G.at(i, j, k);
          real Fv[10], lam;
          mhd_flux_point(P, U + o, G.sf, prim + o, G.sf, d, Fv, &lam);
          if (!aux.empty()) {
            real Fs[10];
            les_flux_point(P, G, U, aux.data(), i, j, k, d, Fs);
            for (int n = 0; n < 10; ++n) Fv[n] = Fv[n] + Fs[n];
          }
          for (int n = 0; n < 10; ++n) Fp[(size_t)n * npts + o] = dbl(Fv[n]);
          Lp[o] = dbl(lam);
        }
    long long c1 = flops_now();
    c_pt += c1 - c0;
    lo[d] = -1;
    hi[d] = G.n[d];
    ORACLE_PAR_FOR
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          long o = G.at(i, j, k);
          real Fm[6][10], Um[6][10], lam[6];
          for (int m = 0; m < 6; ++m) {
            long q = o + (m - 2) * st[d];
            for (int n = 0; n < 10; ++n) {
              Fm[m][n] = Fp[(size_t)n * npts + q];
              Um[m][n] = U[(NST + n) * G.sf + q];
            }
            lam[m] = Lp[q];
          }
          real Fh[10];
          iface_flux(Fm, Um, lam, Fh);
          for (int n = 0; n < 10; ++n) Fhat[((size_t)d * 10 + n) * npts + o] = dbl(Fh[n]);
        }
    c0 = flops_now();
    c_if += c0 - c1;
  }
  real idx = 1.0 / G.dx;
  ORACLE_PAR_FOR
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long o = G.at(i, j, k);
        real r[NF];
        geom Gm;
        ccz4_rhs_point(P, G, U, prim, i, j, k, r, &Gm);
        real src[10];
        mhd_source_point(P, Gm, U + o, G.sf, src);
        for (int n = 0; n < 10; ++n) {
          real v = src[n];
          for (int d = 0; d < 3; ++d) {
            real fp = Fhat[((size_t)d * 10 + n) * npts + o];
            real fm = Fhat[((size_t)d * 10 + n) * npts + o - st[d]];
            v -= (fp - fm) * idx;
          }
          r[NST + n] = v;
        }
        for (int f = 0; f < NF; ++f) rhs[(long)f * G.sf + o] = dbl(r[f]);
      }
  if (counts) {
    counts[0] = c_pt;
    counts[1] = c_if;
    counts[2] = flops_now() - c0;
  }
}

// One substep of explicit RK4 on registers Un, Ua, Ub (stage values) and acc:
//   stage 0: in Un -> Ua = Un + dt/2 k1, acc = Un + dt/6 k1
//   stage 1: in Ua -> Ub = Un + dt/2 k2, acc += dt/3 k2
//   stage 2: in Ub -> Ua = Un + dt k3,   acc += dt/3 k3
//   stage 3: in Ua -> Un = acc + dt/6 k4
// Each stage first fills ghosts and runs con2prim on its input register.
// counts (optional, counting build): [con2prim, pointwise fluxes, interface
// fluxes, local right-hand side, RK combination].
// One Runge-Kutta substep (Sec. III A).  RK4 (Table RK4, explicit part):
// stage inputs U^n, Ua, Ub, Ua; the stages' outputs U^n + dt/2 k1, U^n + dt/2 k2,
// U^n + dt k3 and the accumulator acc = U^n + dt (k1/6 + k2/3 + k3/3), then
// U^{n+1} = acc + dt k4/6.  SSP-RK3 (Table RK3SSP, explicit part; rk = 1):
// stage inputs Y1 = U^n, Y2 = Ua, Y3 = Ub with Y2 = U^n + dt k1,
// Y3 = U^n + dt/4 k1 + dt/4 k2, U^{n+1} = U^n + dt (k1/6 + k2/6 + 2 k3/3)
// (acc collects the first two terms).
int substep(const oracle_params* P, const oracle_eos_table* E, const grid& G, int stage, double dt, double* Un,
            double* Ua, double* Ub, double* acc, double* prim, int8_t* status, double* krhs, long long* counts) {
  const bool rk3 = P->rk == 1;
  double* in = stage == 0 ? Un : stage == 1 ? Ua : stage == 2 ? Ub : Ua;
  double* out = stage == 0 ? Ua : stage == 1 ? Ub : stage == 2 ? Ua : Un;
  ghost_fill(P, G, in, NF);
  if (P->bc == 2 && in != Un) {
    // Frozen ghosts: the stage register carries U^n's ghost values.
    for (int f = 0; f < NF; ++f)
      for (int k = -NG; k < G.n[2] + NG; ++k)
        for (int j = -NG; j < G.n[1] + NG; ++j)
          for (int i = -NG; i < G.n[0] + NG; ++i) {
            bool inner = i >= 0 && i < G.n[0] && j >= 0 && j < G.n[1] && k >= 0 && k < G.n[2];
            if (!inner) in[(long)f * G.sf + G.at(i, j, k)] = Un[(long)f * G.sf + G.at(i, j, k)];
          }
  }
  long long t0 = flops_now();
  int worst = c2p_patch(P, E, G, in, prim, status, nullptr);
  long long t1 = flops_now();
  rhs_patch(P, E, G, in, prim, krhs, counts ? counts + 1 : nullptr);
  long long t2 = flops_now();
  real hdt = 0.5 * dt, sdt = dt / 6.0, tdt = dt / 3.0;
  ORACLE_PAR_FOR
  for (int f = 0; f < NF; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          long o = (long)f * G.sf + G.at(i, j, k);
          real kk = krhs[o];
          if (rk3) {
            if (stage == 0) {
              Ua[o] = dbl(real(Un[o]) + dt * kk);
              Ub[o] = dbl(real(Un[o]) + (0.25 * dt) * kk);
              acc[o] = dbl(real(Un[o]) + sdt * kk);
            } else if (stage == 1) {
              Ub[o] = dbl(real(Ub[o]) + (0.25 * dt) * kk);
              acc[o] = dbl(real(acc[o]) + sdt * kk);
            } else {
              Un[o] = dbl(real(acc[o]) + (2.0 * dt / 3.0) * kk);
            }
          } else if (stage == 0) {
            out[o] = dbl(real(Un[o]) + hdt * kk);
            acc[o] = dbl(real(Un[o]) + sdt * kk);
          } else if (stage == 1) {
            out[o] = dbl(real(Un[o]) + hdt * kk);
            acc[o] = dbl(real(acc[o]) + tdt * kk);
          } else if (stage == 2) {
            out[o] = dbl(real(Un[o]) + dt * kk);
            acc[o] = dbl(real(acc[o]) + tdt * kk);
          } else {
            out[o] = dbl(real(acc[o]) + sdt * kk);
          }
        }
  if (counts) {
    counts[0] = t1 - t0;
    counts[4] = flops_now() - t2;
  }
  return worst;
}
