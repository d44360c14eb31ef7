// Point-wise and interface kernels of the substep: initial-data conversion
// to the CCZ4 variables (Sec. II A), ghost fill (periodic, or the outer
// boundary's extrapolation of Sec. IV B), con2prim with the point-wise MHD
// fluxes and characteristic speeds (Sec. II B; appendix on the
// characteristic structure), interface fluxes (Lax-Friedrichs splitting and
// MP5 reconstruction, Sec. III C), the unfused RK stage combination
// (Sec. III A, explicit tableaux) and the flat-metric con2prim of independent
// states.
#include <cmath>
#include "kern.cuh"

namespace gk {

Eos make_eos(const grmhd_params& P, const grmhd_eos_table* T) {
  Eos E;
  E.kind = P.eos_kind;
  E.gam = P.gamma_th;
  E.K = P.K_atmo;
  E.eps_max = P.eps_max;
  E.nr = E.nt = E.ny = 0;
  E.lr0 = E.idlr = E.lt0 = E.dlt = E.idlt = E.ye0 = E.idye = 0.0;
  E.p = E.e = E.c = nullptr;
  E.atmo_set = 0;
  E.atmo = EosOut{0.0, 0.0, 0.0, 0.0};
  E.npoly = 0;
  for (int i = 0; i < 4; ++i) E.hK[i] = E.ha[i] = E.hg[i] = 0.0;
  for (int i = 0; i < 3; ++i) E.hr[i] = 0.0;
  if (P.eos_kind == 2) {
    // Piece constants of the hybrid EOS's cold part (Sec. II B): K_0 given,
    // a_0 = 0; p_cold and eps_cold continuous at each dividing density.
    E.npoly = P.npoly;
    E.hK[0] = P.K_poly;
    E.hg[0] = P.gamma_poly[0];
    for (int i = 1; i < P.npoly; ++i) {
      const double rb = P.rho_poly[i - 1], g0 = P.gamma_poly[i - 1], g1 = P.gamma_poly[i];
      E.hg[i] = g1;
      E.hK[i] = E.hK[i - 1] * std::pow(rb, g0 - g1);
      E.ha[i] = E.ha[i - 1] + E.hK[i - 1] / (g0 - 1.0) * std::pow(rb, g0 - 1.0) -
                E.hK[i] / (g1 - 1.0) * std::pow(rb, g1 - 1.0);
      E.hr[i - 1] = rb;
    }
  }
  if (T && P.eos_kind == 1) {
    E.nr = T->nr;
    E.nt = T->nt;
    E.ny = T->ny;
    E.lr0 = T->lr0;
    E.idlr = 1.0 / T->dlr;
    E.lt0 = T->lt0;
    E.dlt = T->dlt;
    E.idlt = 1.0 / T->dlt;
    E.ye0 = T->ye0;
    E.idye = 1.0 / T->dye;
    E.p = T->p;
    E.e = T->eps;
    E.c = T->cs2;
  }
  return E;
}

// The atmosphere's EOS state, evaluated once by the same device code that
// con2prim would run at every atmosphere point (so the stored values are
// those it would compute).
__global__ void k_atmo_state(grmhd_params P, Eos E, EosOut* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = eos_T(E, P.rho_atmo, P.T_atmo, P.ye_atmo);
}

int eos_set_atmo(const grmhd_params& P, Eos& E, cudaStream_t st) {
  EosOut* d = nullptr;
  EosOut h;
  if (cudaMalloc(&d, sizeof(EosOut)) != cudaSuccess) return GRMHD_ERR_NOMEM;
  k_atmo_state<<<1, 32, 0, st>>>(P, E, d);
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(&h, d, sizeof(EosOut), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d);
  if (!ok) return GRMHD_ERR_CUDA;
  E.atmo = h;
  E.atmo_set = 1;
  return GRMHD_OK;
}

int eos_check(const grmhd_params& P, const grmhd_eos_table* T) {
  if (P.eos_kind == 0) return GRMHD_OK;
  if (P.eos_kind == 1)
    return (T && T->p && T->eps && T->cs2 && T->nr >= 2 && T->nt >= 2 && T->ny >= 2) ? GRMHD_OK : GRMHD_ERR_ARG;
  if (P.eos_kind != 2 || P.npoly < 1 || P.npoly > 4 || !(P.K_poly > 0.0)) return GRMHD_ERR_ARG;
  for (int i = 0; i < P.npoly; ++i)
    if (!(P.gamma_poly[i] > 1.0)) return GRMHD_ERR_ARG;
  for (int i = 0; i + 1 < P.npoly; ++i)
    if (!(P.rho_poly[i] > 0.0) || (i > 0 && !(P.rho_poly[i] > P.rho_poly[i - 1]))) return GRMHD_ERR_ARG;
  return GRMHD_OK;
}

// ---------------------------------------------------------------------------
// Initial data -> CCZ4 variables and conserved variables at every point.
__global__ void k_init(Geo G, grmhd_params P, Eos E, const double* __restrict__ id, double* __restrict__ U) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_ALL, G)) return;
  int i, j, k;
  dom_decode(DOM_ALL, G, q, i, j, k);
  long long o = at(G, i, j, k);
  const long long sf = G.sf;
  double g[6], K[6], gu[6];
  for (int n = 0; n < 6; ++n) {
    g[n] = id[(IG + n) * sf + o];
    K[n] = id[(IK + n) * sf + o];
  }
  double det = det3(g);
  inv3(g, 1.0 / det, gu);
  double chi = 1.0 / cbrt(det);
  double trK = tr6(gu, K);
  for (int n = 0; n < 6; ++n) {
    U[(GT + n) * sf + o] = chi * g[n];
    U[(AT + n) * sf + o] = chi * fma(-g[n], trK * (1.0 / 3.0), K[n]);
  }
  U[CHI * sf + o] = chi;
  U[KH * sf + o] = trK;
  U[TH * sf + o] = 0.0;
  U[ALP * sf + o] = id[IALP * sf + o];
  for (int a = 0; a < 3; ++a) U[(BET + a) * sf + o] = id[(IBET + a) * sf + o];
  double rho = id[IRHO * sf + o], ye = id[IYE * sf + o];
  double eps, p;
  if (P.eos_kind == 0) {
    eps = id[IEPS * sf + o];
    p = (P.gamma_th - 1.0) * rho * eps;
  } else if (P.eos_kind == 2) {
    eps = id[IEPS * sf + o];
    p = eos_eps(E, rho, eps, ye).p;
  } else {
    EosOut eo = eos_T(E, rho, id[IT * sf + o], ye);
    eps = eo.eps;
    p = eo.p;
  }
  double v[3] = {id[IV * sf + o], id[(IV + 1) * sf + o], id[(IV + 2) * sf + o]};
  double B[3] = {id[IB * sf + o], id[(IB + 1) * sf + o], id[(IB + 2) * sf + o]};
  double c6[6];
  prim2con(g, rho, eps, p, v, ye, B, c6);
  double sg = sqrt(det);
  for (int n = 0; n < 6; ++n) U[(DD + n) * sf + o] = c6[n] * sg;
  for (int a = 0; a < 3; ++a) U[(BB + a) * sf + o] = B[a] * sg;
  U[PHI * sf + o] = 0.0;
}

// Gammahat^i = gt^ij gt^kl d_l gt_jk at interior points (same D_i as the RHS).
__global__ void k_init_gh(Geo G, double* __restrict__ U) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_INT, G)) return;
  int i, j, k;
  dom_decode(DOM_INT, G, q, i, j, k);
  long long o = at(G, i, j, k);
  const long long sf = G.sf;
  const long long st[3] = {1, G.sy, G.sz};
  const double i12 = 1.0 / (12.0 * G.dx);
  double g[6], gu[6], dg[3][6];
  for (int n = 0; n < 6; ++n) {
    g[n] = U[(GT + n) * sf + o];
    for (int a = 0; a < 3; ++a) dg[a][n] = fd1(U + (GT + n) * sf + o, st[a]) * i12;
  }
  inv3(g, 1.0 / det3(g), gu);
  double t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
      for (int l = 0; l < 3; ++l) s = fma(gu[S6(kk, l)], dg[l][S6(a, kk)], s);
    t[a] = s;
  }
  for (int a = 0; a < 3; ++a)
    U[(GH + a) * sf + o] = gu[S6(a, 0)] * t[0] + gu[S6(a, 1)] * t[1] + gu[S6(a, 2)] * t[2];
}

void launch_init(const PatchDev*, int, const Geo& G, const grmhd_params& P, const Eos& E, const double* id, double* U,
                 cudaStream_t st) {
  long long n = dom_count(DOM_ALL, G);
  k_init<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(G, P, E, id, U);
  long long m = dom_count(DOM_INT, G);
  k_init_gh<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(G, U);
}

// ---------------------------------------------------------------------------
// Ghost fill along one axis: each thread owns one line and fills its 3 + 3
// ghost points for all 32 fields.
template <int AX>
__global__ void k_ghost(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int reg, int bc, int f0, int f1) {
  Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo& G = PD.G;
  constexpr int dom = AX == 0 ? DOM_GX : (AX == 1 ? DOM_GY : DOM_GZ);
  long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(dom, G)) return;
  int i, j, k;
  dom_decode(dom, G, q, i, j, k);
  long long o = at(G, i, j, k);
  const long long s = AX == 0 ? 1 : (AX == 1 ? G.sy : G.sz);
  const int n = AX == 0 ? G.n0 : (AX == 1 ? G.n1 : G.n2);
  double* U = PD.U[reg];
  for (int f = f0; f < f1; ++f) {
    double* b = U + f * G.sf + o;
    if (bc == 0) {
#pragma unroll
      for (int m = 1; m <= 3; ++m) {
        b[-m * s] = b[(n - m) * s];
        b[(n - 1 + m) * s] = b[(m - 1) * s];
      }
    } else {
      double u0 = b[0], u1 = b[s], v0 = b[(n - 1) * s], v1 = b[(n - 2) * s];
#pragma unroll
      for (int m = 1; m <= 3; ++m) {
        b[-m * s] = fma(1.0 + m, u0, -(double)m * u1);
        b[(n - 1 + m) * s] = fma(1.0 + m, v0, -(double)m * v1);
      }
    }
  }
}

void launch_ghost(const PatchDev* pd, const Work* w, int nblk, int reg, int axis, int bc, cudaStream_t st, int f0,
                  int f1) {
  if (nblk <= 0) return;
  if (axis == 0) k_ghost<0><<<nblk, BS_ALL, 0, st>>>(pd, w, reg, bc, f0, f1);
  if (axis == 1) k_ghost<1><<<nblk, BS_ALL, 0, st>>>(pd, w, reg, bc, f0, f1);
  if (axis == 2) k_ghost<2><<<nblk, BS_ALL, 0, st>>>(pd, w, reg, bc, f0, f1);
}

// ---------------------------------------------------------------------------
// con2prim at every point, then the point-wise flux vectors F^d (10 fields)
// and max |lambda^{+-}_fast| along d for the directions whose interface
// stencils use this point.
// con2prim and point-wise fluxes of one work item (see k_c2p); adds the
// item's iteration, correction, failure and point counts to acc.
template <bool SEEDED, int LB>
DI void c2p_item(const PatchDev* __restrict__ pd, const Work wk, int reg, const grmhd_params& P, const Eos& E,
                 DevFlags* flags, double delta, unsigned long long acc[4]) {
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  int i, j, k;
  const bool active = work_point(DOM_ALL, G, wk.block, threadIdx.x, LB, i, j, k);
  int st_code = 0, iters = 0;
  if (active) {
    const long long o = at(G, i, j, k), sf = G.sf;
    double* U = PD.U[reg];
    double gt[6], gtu[6], gdd[6], guu[6];
    for (int n = 0; n < 6; ++n) gt[n] = U[(GT + n) * sf + o];
    double chi = U[CHI * sf + o];
    double det = det3(gt);
    inv3(gt, 1.0 / det, gtu);
    double ichi = 1.0 / chi;
    for (int n = 0; n < 6; ++n) {
      gdd[n] = gt[n] * ichi;
      guu[n] = chi * gtu[n];
    }
    double sg = sqrt(det) * ichi * sqrt(ichi);
    double cb[9];
    for (int n = 0; n < 9; ++n) cb[n] = U[(DD + n) * sf + o];
    double al = U[ALP * sf + o];
    C2POut r;
    if (SEEDED) {
      double sq[3];
      for (int m = 0; m < 3; ++m) sq[m] = (double)PD.seed[m * sf + o];
      c2p_point(P, E, cb, gdd, guu, sg, al, r, sq, delta);
    } else {
      c2p_point(P, E, cb, gdd, guu, sg, al, r);
    }
    st_code = r.status;
    iters = r.iters;
    for (int n = 0; n < NP; ++n) PD.prim[n * sf + o] = r.prim[n];
    PD.status[o] = (int8_t)r.status;
    if (r.status > 0)
      for (int n = 0; n < 6; ++n) {
        U[(DD + n) * sf + o] = r.cons[n];
        cb[n] = r.cons[n];
      }
    if (r.status < 0) atomicOr(&flags->flags, r.status == -5 ? 2 : 1);

    // Which directions need this point: interior in the two other axes.
    bool inx = (i >= 0 && i < G.n0), iny = (j >= 0 && j < G.n1), inz = (k >= 0 && k < G.n2);
    bool need[3] = {iny && inz, inx && inz, inx && iny};
    if (need[0] || need[1] || need[2]) {
      const double* pr = r.prim;
      double v[3] = {pr[VX], pr[VY], pr[VZ]};
      const double isg = r.isg;  // 1 / sg, formed once by c2p_point
      double B[3] = {cb[6] * isg, cb[7] * isg, cb[8] * isg};
      double Sl[3] = {cb[3] * isg, cb[4] * isg, cb[5] * isg};
      double vd[3], Bd[3];
      lower3(gdd, v, vd);
      lower3(gdd, B, Bd);
      double v2 = v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2];
      double B2 = B[0] * Bd[0] + B[1] * Bd[1] + B[2] * Bd[2];
      double Bv = B[0] * vd[0] + B[1] * vd[1] + B[2] * vd[2];
      double W = pr[WW];
      // At rest (W = 1, v = 0: atmosphere points) the quotients 1 / W^2 and
      // al / den are exact without their division sequences.
      double iW2 = W == 1.0 ? 1.0 : 1.0 / (W * W);
      double piso = pr[PRS] + 0.5 * fma(iW2, B2, Bv * Bv);
      double Sij[6];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
          double t = 0.5 * fma(vd[a], Sl[b], vd[b] * Sl[a]) - iW2 * Bd[a] * Bd[b] -
                     0.5 * Bv * fma(Bd[a], vd[b], Bd[b] * vd[a]);
          Sij[S6(a, b)] = fma(gdd[S6(a, b)], piso, t);
        }
      double be[3] = {U[BET * sf + o], U[(BET + 1) * sf + o], U[(BET + 2) * sf + o]};
      double phib = U[PHI * sf + o];
      double b2 = fma(B2, iW2, Bv * Bv);
      double h = fma(pr[RHO], 1.0 + pr[EPS], pr[PRS]);
      double ca2 = b2 == 0.0 ? 0.0 : b2 / (h + b2);  // no field (the atmosphere outside a star): exactly 0
      double cs2 = pr[CS2];
      double a2 = cs2 + ca2 - cs2 * ca2;
      double den = fma(-v2, a2, 1.0);
      double pre = den == 1.0 ? al : al / den;
      double a2w = a2 * (1.0 - v2);
      double oma2 = 1.0 - a2;
      const double cb2 = P.c_b * P.c_b;
      double avb[3];
      for (int a = 0; a < 3; ++a) avb[a] = fma(al, v[a], -be[a]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!need[d]) continue;
        double* F = PD.Fp + (long long)d * 10 * sf + o;
        F[0 * sf] = avb[d] * cb[0];
        F[1 * sf] = avb[d] * cb[1];
        double Sbu = guu[S6(d, 0)] * cb[3] + guu[S6(d, 1)] * cb[4] + guu[S6(d, 2)] * cb[5];
        F[2 * sf] = fma(-be[d], cb[2], al * fma(-cb[0], v[d], Sbu));
        double asg = al * sg;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          double Sm = guu[S6(d, 0)] * Sij[S6(0, a)] + guu[S6(d, 1)] * Sij[S6(1, a)] + guu[S6(d, 2)] * Sij[S6(2, a)];
          F[(3 + a) * sf] = fma(-be[d], cb[3 + a], asg * Sm);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
          F[(6 + a) * sf] = fma(cb[6 + a], avb[d], fma(-cb[6 + d], avb[a], al * chi * gtu[S6(d, a)] * phib));
        F[9 * sf] = fma(-be[d], phib, al * cb2 * cb[6 + d]);
        double rad = sqrt(a2w * fma(den, guu[S6(d, d)], -oma2 * v[d] * v[d]));
        double c = fma(pre * oma2, v[d], -be[d]);
        PD.lam[(long long)d * sf + o] = fma(pre, rad, fabs(c));
      }
    }
  }
  acc[0] += iters;
  acc[1] += st_code > 0;
  acc[2] += st_code < 0;
  acc[3] += active;
}

// PERS: a persistent pool of blocks loops over the work items with stride
// gridDim.x; otherwise one block per item (the loop costs registers, so it
// exists only in the persistent instantiations).
template <bool STATS, int BS, bool SEEDED, bool PERS>
__global__ void __launch_bounds__(BS) k_c2p(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int nitems,
                                                 int reg, grmhd_params P, Eos E, DevFlags* flags, C2PStats* stats,
                                                 double delta) {
  constexpr int LB = BS == 64 ? 6 : (BS == 128 ? 7 : 8);
  unsigned long long acc[4] = {0, 0, 0, 0};
  if constexpr (PERS) {
    for (int item = blockIdx.x; item < nitems; item += gridDim.x)
      c2p_item<SEEDED, LB>(pd, w[item], reg, P, E, flags, delta, acc);
  } else {
    c2p_item<SEEDED, LB>(pd, w[blockIdx.x], reg, P, E, flags, delta, acc);
  }
  if (STATS) {
    unsigned long long it = acc[0], cor = acc[1], bad = acc[2], pts = acc[3];
    for (int off = 16; off > 0; off >>= 1) {
      it += __shfl_down_sync(0xffffffffu, it, off);
      cor += __shfl_down_sync(0xffffffffu, cor, off);
      bad += __shfl_down_sync(0xffffffffu, bad, off);
      pts += __shfl_down_sync(0xffffffffu, pts, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats->iters, it);
      atomicAdd(&stats->corrected, cor);
      atomicAdd(&stats->failed, bad);
      atomicAdd(&stats->points, pts);
    }
  }
}

template <int BS, bool PERS>
static void launch_c2p_bs(const PatchDev* pd, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                          DevFlags* flags, C2PStats* stats, cudaStream_t st, bool seeded, double delta) {
  if (seeded) {
    if (stats) {
      auto k = k_c2p<true, BS, true, PERS>;
      k<<<grid_for(k, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg, P, E, flags, stats, delta);
    } else {
      auto k = k_c2p<false, BS, true, PERS>;
      k<<<grid_for(k, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg, P, E, flags, stats, delta);
    }
  } else if (stats) {
    auto k = k_c2p<true, BS, false, PERS>;
    k<<<grid_for(k, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg, P, E, flags, stats, 0.0);
  } else {
    auto k = k_c2p<false, BS, false, PERS>;
    k<<<grid_for(k, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg, P, E, flags, stats, 0.0);
  }
}

void launch_c2p(const PatchDev* pd, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                DevFlags* flags, C2PStats* stats, cudaStream_t st, int bs, bool seeded, double delta, bool pers) {
  if (nblk <= 0) return;
  if (pers) {
    if (bs == 64) launch_c2p_bs<64, true>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
    else if (bs == 256) launch_c2p_bs<256, true>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
    else launch_c2p_bs<128, true>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
  } else if (bs == 64) {
    launch_c2p_bs<64, false>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
  } else if (bs == 256) {
    launch_c2p_bs<256, false>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
  } else {
    launch_c2p_bs<128, false>(pd, w, nblk, reg, P, E, flags, stats, st, seeded, delta);
  }
}

// ---------------------------------------------------------------------------
// Interface fluxes along direction D: lambda = max over points i-2 .. i+3,
// g^{+-} = F +- lambda U, F^L = MP5(g^+_{i-2..i+2}), F^R = MP5(g^-_{i+3..i-1}),
// stored as 2 Fhat = F^L + F^R (MP5 commutes with the positive factor 1/2;
// the right-hand side folds the 1/2 into 1/dx, a power-of-two scaling that
// changes no rounding).
// Interface fluxes of one work item along direction D (see k_iflux).
template <int D, int LB>
DI void iflux_item(const PatchDev* __restrict__ pd, const Work wk, int reg) {
  constexpr int dom = D == 0 ? DOM_IFX : (D == 1 ? DOM_IFY : DOM_IFZ);
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  int i, j, k;
  if (!work_point(dom, G, wk.block, threadIdx.x, LB, i, j, k)) return;
  const long long o = at(G, i, j, k), sf = G.sf;
  const long long s = D == 0 ? 1 : (D == 1 ? G.sy : G.sz);
  const double* lam = PD.lam + (long long)D * sf + o;
  // The maximum on the integer pipe (imax: the order of the doubles' keys).
  double L = ld(lam - 2 * s);
#pragma unroll
  for (int m = -1; m <= 3; ++m) L = imax(L, ld(lam + m * s));
  const double* Fp = PD.Fp + (long long)D * 10 * sf + o;
  const double* Uc = PD.U[reg] + (long long)DD * sf + o;
  double* Fh = PD.Fh + (long long)D * 10 * sf + o;
#pragma unroll 1
  for (int f = 0; f < 10; ++f) {
    double gp[6], gm[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      double Fv = ld(Fp + f * sf + (m - 2) * s), Uv = ld(Uc + f * sf + (m - 2) * s);
      gp[m] = fma(L, Uv, Fv);
      gm[m] = fma(-L, Uv, Fv);
    }
    double FL = mp5(gp[0], gp[1], gp[2], gp[3], gp[4]);
    double FR = mp5(gm[5], gm[4], gm[3], gm[2], gm[1]);
    Fh[f * sf] = FL + FR;
  }
}

// PERS: a persistent pool of blocks loops over the work items (see k_c2p).
template <int D, int BS, bool PERS>
__global__ void __launch_bounds__(BS) k_iflux(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int nitems,
                                                   int reg) {
  constexpr int LB = BS == 64 ? 6 : (BS == 128 ? 7 : 8);
  if constexpr (PERS) {
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) iflux_item<D, LB>(pd, w[item], reg);
  } else {
    iflux_item<D, LB>(pd, w[blockIdx.x], reg);
  }
}

template <int BS, bool PERS>
static void launch_iflux_bs(const PatchDev* pd, const Work* w, int nblk, int reg, int dir, cudaStream_t st) {
  if (dir == 0) k_iflux<0, BS, PERS><<<grid_for(k_iflux<0, BS, PERS>, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg);
  if (dir == 1) k_iflux<1, BS, PERS><<<grid_for(k_iflux<1, BS, PERS>, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg);
  if (dir == 2) k_iflux<2, BS, PERS><<<grid_for(k_iflux<2, BS, PERS>, BS, nblk, PERS), BS, 0, st>>>(pd, w, nblk, reg);
}

void launch_iflux(const PatchDev* pd, const Work* w, int nblk, int reg, int dir, cudaStream_t st, int bs, bool pers) {
  if (nblk <= 0) return;
  if (pers) {
    if (bs == 64) launch_iflux_bs<64, true>(pd, w, nblk, reg, dir, st);
    else if (bs == 256) launch_iflux_bs<256, true>(pd, w, nblk, reg, dir, st);
    else launch_iflux_bs<128, true>(pd, w, nblk, reg, dir, st);
  } else if (bs == 64) {
    launch_iflux_bs<64, false>(pd, w, nblk, reg, dir, st);
  } else if (bs == 256) {
    launch_iflux_bs<256, false>(pd, w, nblk, reg, dir, st);
  } else {
    launch_iflux_bs<128, false>(pd, w, nblk, reg, dir, st);
  }
}

// Frozen ghosts (bc 2): the ghost zones of every register hold the ghost values
// of U^n, which no step changes.
__global__ void k_ghost_copy(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int reg) {
  Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo& G = PD.G;
  long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_ALL, G)) return;
  int i, j, k;
  dom_decode(DOM_ALL, G, q, i, j, k);
  if (i >= 0 && i < G.n0 && j >= 0 && j < G.n1 && k >= 0 && k < G.n2) return;
  const long long o = at(G, i, j, k);
  for (int f = 0; f < NF; ++f) PD.U[reg][f * G.sf + o] = PD.U[0][f * G.sf + o];
}

void launch_ghost_copy(const PatchDev* pd, const Work* w, int nblk, int reg, cudaStream_t st) {
  if (nblk <= 0 || reg == 0) return;
  k_ghost_copy<<<nblk, BS_ALL, 0, st>>>(pd, w, reg);
}

// ---------------------------------------------------------------------------
// Unfused RK4 stage combination at interior points.
__global__ void k_rk(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int stage, double dt,
                     double* const* __restrict__ rhs, int rk) {
  Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_INT, G)) return;
  int i, j, k;
  dom_decode(DOM_INT, G, q, i, j, k);
  const long long o = at(G, i, j, k), sf = G.sf;
  const double* K = rhs[wk.patch];
  double *Un = PD.U[0], *Ua = PD.U[1], *Ub = PD.U[2], *acc = PD.U[3];
  if (rk == 1) {  // SSP-RK3
    for (int f = 0; f < NF; ++f) {
      long long x = f * sf + o;
      double kk = K[x];
      if (stage == 0) {
        double u = Un[x];
        Ua[x] = fma(dt, kk, u);
        Ub[x] = fma(0.25 * dt, kk, u);
        acc[x] = fma(dt / 6.0, kk, u);
      } else if (stage == 1) {
        Ub[x] = fma(0.25 * dt, kk, Ub[x]);
        acc[x] = fma(dt / 6.0, kk, acc[x]);
      } else {
        Un[x] = fma(2.0 * dt / 3.0, kk, acc[x]);
      }
    }
    return;
  }
  for (int f = 0; f < NF; ++f) {
    long long x = f * sf + o;
    double kk = K[x];
    if (stage == 0) {
      double u = Un[x];
      Ua[x] = fma(0.5 * dt, kk, u);
      acc[x] = fma(dt / 6.0, kk, u);
    } else if (stage == 1) {
      Ub[x] = fma(0.5 * dt, kk, Un[x]);
      acc[x] = fma(dt / 3.0, kk, acc[x]);
    } else if (stage == 2) {
      Ua[x] = fma(dt, kk, Un[x]);
      acc[x] = fma(dt / 3.0, kk, acc[x]);
    } else {
      Un[x] = fma(dt / 6.0, kk, acc[x]);
    }
  }
}

void launch_rk(const PatchDev* pd, const Work* w, int nblk, int stage, double dt, double* const* rhs, cudaStream_t st,
               int rk) {
  if (nblk <= 0) return;
  k_rk<<<nblk, BS_INT, 0, st>>>(pd, w, stage, dt, rhs, rk);
}

// ---------------------------------------------------------------------------
// Order of independent states for con2prim.  The root finder's evaluation
// count varies from state to state (8 to 27 on the isolated workload), and a
// warp runs as long as its slowest lane: on states in random order 70 % of the
// lanes are busy.  The count follows b^2 / rho closely, so the states are
// grouped by the binary exponent of B^2 / D (2 e(max |B^i|) - e(D), integer
// operations on the bit patterns only) in a counting sort over 64 bins; in
// that order 84 % of the lanes are busy (oracle counts, 2^16 states).  Each
// state's arithmetic is unchanged, so the results are bitwise those in the
// given order.
constexpr int ORDER_BINS = 64;
constexpr int ORDER_BLOCK = 256, ORDER_PER_THREAD = 4;

DI int order_bin(const double* __restrict__ c) {
  auto ex = [](double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); };
  const int eb = max(ex(ld(c + 6)), max(ex(ld(c + 7)), ex(ld(c + 8))));
  const int key = eb == 0 ? -1000 : 2 * eb - ex(ld(c)) - 1023;  // unbiased 2 e(B) - e(D)
  return min(max(key + 40, 0), ORDER_BINS - 1);
}

// Pass 1: bin counts (block histograms in shared memory, one global atomic per bin and block).
__global__ void __launch_bounds__(ORDER_BLOCK) k_order_count(long long n, const double* __restrict__ cons,
                                                             unsigned* __restrict__ hist) {
  __shared__ unsigned h[ORDER_BINS];
  if (threadIdx.x < ORDER_BINS) h[threadIdx.x] = 0;
  __syncthreads();
  const long long q0 = (long long)blockIdx.x * ORDER_BLOCK * ORDER_PER_THREAD;
  for (int k = 0; k < ORDER_PER_THREAD; ++k) {
    const long long q = q0 + (long long)k * ORDER_BLOCK + threadIdx.x;
    if (q < n) atomicAdd(&h[order_bin(cons + q * 10)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < ORDER_BINS && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Exclusive scan of the 64 counts into the bins' write cursors (one warp).
__global__ void k_order_scan(unsigned* __restrict__ hist) {
  const int l = threadIdx.x;
  unsigned a = hist[2 * l], b = hist[2 * l + 1], s = a + b, t = s;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned u = __shfl_up_sync(0xffffffffu, t, o);
    if (l >= o) t += u;
  }
  const unsigned ex = t - s;
  hist[2 * l] = ex;
  hist[2 * l + 1] = ex + a;
}

// Pass 2: each block reserves a range per bin (one atomic per bin) and writes
// its states' indices there; the order within a bin is free.
__global__ void __launch_bounds__(ORDER_BLOCK) k_order_scatter(long long n, const double* __restrict__ cons,
                                                               unsigned* __restrict__ cursor,
                                                               int32_t* __restrict__ order) {
  __shared__ unsigned h[ORDER_BINS], base[ORDER_BINS];
  if (threadIdx.x < ORDER_BINS) h[threadIdx.x] = 0;
  __syncthreads();
  const long long q0 = (long long)blockIdx.x * ORDER_BLOCK * ORDER_PER_THREAD;
  int bin[ORDER_PER_THREAD];
  unsigned rank[ORDER_PER_THREAD];
#pragma unroll
  for (int k = 0; k < ORDER_PER_THREAD; ++k) {
    const long long q = q0 + (long long)k * ORDER_BLOCK + threadIdx.x;
    bin[k] = q < n ? order_bin(cons + q * 10) : -1;
    rank[k] = bin[k] >= 0 ? atomicAdd(&h[bin[k]], 1u) : 0u;
  }
  __syncthreads();
  if (threadIdx.x < ORDER_BINS) base[threadIdx.x] = h[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], h[threadIdx.x]) : 0u;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ORDER_PER_THREAD; ++k)
    if (bin[k] >= 0) order[base[bin[k]] + rank[k]] = (int32_t)(q0 + (long long)k * ORDER_BLOCK + threadIdx.x);
}

int32_t* c2p_flat_order(long long n, const double* cons, cudaStream_t st) {
  if (n < ORDER_MIN_STATES || n > 0x7fffffffLL) return nullptr;
  void* mem = nullptr;
  const size_t bytes = (size_t)n * sizeof(int32_t) + 256 + ORDER_BINS * sizeof(unsigned);
  if (cudaMallocAsync(&mem, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;  // the caller solves in the given order
  }
  int32_t* order = static_cast<int32_t*>(mem);
  unsigned* hist = reinterpret_cast<unsigned*>(static_cast<char*>(mem) + (((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255));
  const unsigned blocks = (unsigned)((n + ORDER_BLOCK * ORDER_PER_THREAD - 1) / (ORDER_BLOCK * ORDER_PER_THREAD));
  cudaMemsetAsync(hist, 0, ORDER_BINS * sizeof(unsigned), st);
  k_order_count<<<blocks, ORDER_BLOCK, 0, st>>>(n, cons, hist);
  k_order_scan<<<1, 32, 0, st>>>(hist);
  k_order_scatter<<<blocks, ORDER_BLOCK, 0, st>>>(n, cons, hist, order);
  return order;
}

void c2p_flat_order_free(int32_t* order, cudaStream_t st) {
  if (order) cudaFreeAsync(order, st);
}

// ---------------------------------------------------------------------------
// con2prim of independent states with a flat metric (alpha = 1); thread i
// solves state order[i] (or i).
__global__ void __launch_bounds__(128) k_c2p_flat(grmhd_params P, Eos E, long long n, const double* __restrict__ cons,
                                                   double* __restrict__ prim, int8_t* __restrict__ status,
                                                   int32_t* __restrict__ iters, const int32_t* __restrict__ order) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (order) q = order[q];
  const double g[6] = {1.0, 0.0, 0.0, 1.0, 0.0, 1.0};
  double cb[9];
  for (int m = 0; m < 9; ++m) cb[m] = ld(cons + q * 10 + m);
  C2POut r;
  c2p_point(P, E, cb, g, g, 1.0, 1.0, r);
  for (int m = 0; m < NP; ++m) prim[q * NP + m] = r.prim[m];
  status[q] = (int8_t)r.status;
  if (iters) iters[q] = r.iters;
}

__global__ void k_prim2con_flat(grmhd_params P, Eos E, long long n, const double* __restrict__ prim,
                                const double* __restrict__ B, double* __restrict__ cons) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double g[6] = {1.0, 0.0, 0.0, 1.0, 0.0, 1.0};
  const double* pr = prim + q * NP;
  double rho = pr[RHO], ye = pr[YE], eps, p;
  if (P.eos_kind == 1) {
    EosOut eo = eos_T(E, rho, pr[TT], ye);
    eps = eo.eps;
    p = eo.p;
  } else if (P.eos_kind == 2) {
    eps = pr[EPS];
    p = eos_eps(E, rho, eps, ye).p;
  } else {
    eps = pr[EPS];
    p = (P.gamma_th - 1.0) * rho * eps;
  }
  double v[3] = {pr[VX], pr[VY], pr[VZ]};
  double b[3] = {B[q * 3], B[q * 3 + 1], B[q * 3 + 2]};
  double c6[6];
  prim2con(g, rho, eps, p, v, ye, b, c6);
  for (int m = 0; m < 6; ++m) cons[q * 10 + m] = c6[m];
  for (int m = 0; m < 3; ++m) cons[q * 10 + 6 + m] = b[m];
  cons[q * 10 + 9] = 0.0;
}

void launch_c2p_flat(const grmhd_params& P, const Eos& E, long long n, const double* cons, double* prim,
                     int8_t* status, int32_t* iters, cudaStream_t st) {
  if (n <= 0) return;
  int32_t* order = c2p_flat_order(n, cons, st);
  k_c2p_flat<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, E, n, cons, prim, status, iters, order);
  c2p_flat_order_free(order, st);
}

void launch_prim2con_flat(const grmhd_params& P, const Eos& E, long long n, const double* prim, const double* B,
                          double* cons, cudaStream_t st) {
  if (n <= 0) return;
  k_prim2con_flat<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, E, n, prim, B, cons);
}

}  // namespace gk

namespace gk {

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: every thread runs CH independent FMA
// recurrences a <- a m + b (m, b per chain, in registers), unrolled four
// times, so the FP64 pipe, not the latency of one chain or the loop
// arithmetic, limits the rate.  The sum is stored only if it equals an
// impossible value, which keeps the compiler from dropping the work without
// any memory traffic.
// ADD: the chains are additions a <- a + b instead (the FP64 add rate).
template <int CH, bool ADD>
__global__ void __launch_bounds__(256) k_dfma_probe(long long iters, double* __restrict__ sink) {
  double a[CH], m[CH], b[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    a[c] = 1.0 + c * 1e-3 + threadIdx.x * 1e-9;
    m[c] = 0.9999999999 - c * 1e-13;
    b[c] = 1e-12 * (1 + threadIdx.x + c);
  }
  for (long long it = 0; it < iters; it += 4)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) a[c] = ADD ? a[c] + b[c] : fma(a[c], m[c], b[c]);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

long long launch_dfma_probe(int blocks, int chains, long long iters, double* sink, cudaStream_t st, bool add) {
  iters = (iters + 3) / 4 * 4;
  if (add) {
    if (chains == 16)
      k_dfma_probe<16, true><<<blocks, 256, 0, st>>>(iters, sink);
    else if (chains == 4)
      k_dfma_probe<4, true><<<blocks, 256, 0, st>>>(iters, sink);
    else
      k_dfma_probe<8, true><<<blocks, 256, 0, st>>>(iters, sink);
  } else if (chains == 16) {
    k_dfma_probe<16, false><<<blocks, 256, 0, st>>>(iters, sink);
  } else if (chains == 4) {
    k_dfma_probe<4, false><<<blocks, 256, 0, st>>>(iters, sink);
  } else {
    k_dfma_probe<8, false><<<blocks, 256, 0, st>>>(iters, sink);
  }
  return (long long)blocks * 256 * (chains == 16 ? 16 : (chains == 4 ? 4 : 8)) * iters;
}

}  // namespace gk
