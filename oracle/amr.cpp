// Oracle of the mesh-refinement ghost fill and restriction (Sec. IV B,
// "Mesh Refinement: refinement criteria, prolongation and restriction"), for
// a fixed hierarchy advanced without sub-cycling (every level takes the same
// time step).  Test infrastructure only: plain loops over points, FP64.
//
// Hierarchy: level 0 is one patch whose outer ghosts are extrapolated as in
// ghost_fill (bc 1).  A patch of level l >= 1 has spacing dx_0 / 2^l and an
// origin at integer index o (per axis) of the level-l grid that starts at the
// level-0 origin; level-l grid point g coincides with level-(l-1) point g / 2
// when g is even and lies midway between points (g - 1) / 2 and (g + 1) / 2
// when g is odd (vertex-centred refinement by two).
//
// Ghost point g of a level-l patch (l >= 1), filled level by level:
//   1. if g is an interior point of another level-l patch: copied from it;
//   2. otherwise from the level-(l-1) patch whose interior holds c = floor(g/2):
//      along each axis where g is even the coarse value at c is taken, along
//      each axis where g is odd the paper's six-point Lagrange midpoint
//      formula  U_{c+1/2} = [150 (U_c + U_{c+1}) - 25 (U_{c-1} + U_{c+2})
//      + 3 (U_{c-2} + U_{c+3})] / 256  is applied, x first, then y, then z.
//      The stencil reaches three coarse points beyond the interior, inside the
//      coarse patch's ghosts, which were filled first.
// Restriction (after each full step, finest level first): every interior
// point of a level-l patch at even g overwrites the coarse interior point
// g / 2 (direct copy, the paper's restriction operator).
//
// Sub-cycling in time (Sec. IV C, "Sub-cycling in time", BOR scheme): level l
// takes steps of dt_0 / 2^l; after each step of level l, level l+1 takes two
// steps and is restricted into level l.  The ghost points of level l+1 during
// its steps come from level l's dense output (Sec. III A, dense output
// interpolator) U^{n+theta} = U^n + sum_j b_j(theta) k_j, k_j = dt f(U^(j)):
// its time derivatives at t^n, D_m = dt^m d^m U / dt^m = sum_j b_j^(m)(0) k_j,
// give the Taylor data of the interpolant at the start t0 = t^n + theta0 dt
// of the fine step (theta0 = 0 or 1/2, fine step h = dt / 2):
//   U(t0) = U^n + sum_m theta0^m / m! D_m,
//   h^i U^(i)(t0) = (h / dt)^i sum_{m >= i} theta0^(m-i) / (m-i)! D_m,
// and the fine stage values are the RK scheme's stages expanded in these
// derivatives.  With P_i = h^i U^(i)(t0) and, for a nonlinear f, the term
// P_J = h^3 f_U U'' that the expansion of RK4's third and fourth stages keeps
// at third order:
//   RK4:     Y1 = U0,  Y2 = U0 + P1/2,  Y3 = U0 + P1/2 + P2/4 + (P3 - P_J)/16,
//            Y4 = U0 + P1 + P2/2 + (P3 + P_J)/8;
//   SSP-RK3: Y1 = U0,  Y2 = U0 + P1,    Y3 = U0 + P1/2 + P2/4.
// dt^3 f_U U'' is taken from the coarse step's own stages, J = 4 (k3 - k2)
// (= dt^3 f_U U'' + O(dt^4)), and P_J = J / R^3.  The time expression is
// formed at every coarse point of the prolongation stencil, then the spatial
// prolongation above is applied to it.  Level l's U^n, D_m and J carry ghost
// values: level 0 extrapolates them like its registers, finer levels copy
// them from the same-level patches that hold those points (other ghost
// points are undefined; a stencil that reaches one is an error).
#include <cmath>
#include <cstdint>
#include <vector>

#include "oracle.hpp"
#include <algorithm>

namespace {

struct hpatch {
  int n[3];
  int px;
  int level;
  long o[3];
  grid G;
};

std::vector<hpatch> parse(int np, const int* meta, const double* dx) {
  std::vector<hpatch> H(np);
  for (int p = 0; p < np; ++p) {
    const int* m = meta + 8 * p;
    hpatch& h = H[p];
    for (int a = 0; a < 3; ++a) h.n[a] = m[a];
    h.px = m[3];
    h.level = m[4];
    for (int a = 0; a < 3; ++a) h.o[a] = m[5 + a];
    h.G = make_grid(h.n, h.px, dx[p]);
  }
  return H;
}

bool interior(const hpatch& h, const long g[3]) {
  for (int a = 0; a < 3; ++a)
    if (g[a] < h.o[a] || g[a] >= h.o[a] + h.n[a]) return false;
  return true;
}

int find_patch(const std::vector<hpatch>& H, int level, const long g[3], int except) {
  for (int q = 0; q < (int)H.size(); ++q)
    if (q != except && H[q].level == level && interior(H[q], g)) return q;
  return -1;
}

long floor_half(long g) { return g >= 0 ? g / 2 : -((-g + 1) / 2); }

// The paper's midpoint formula on U_{c-2..c+3}.
real midpoint(const real u[6]) {
  return (150.0 * (u[2] + u[3]) - 25.0 * (u[1] + u[4]) + 3.0 * (u[0] + u[5])) / 256.0;
}

// Coarse value at c (odd[a]: the midpoint c + 1/2 along axis a) of field f.
real prolong(const hpatch& r, const double* U, int f, const long c[3], const int odd[3]) {
  long i0 = c[0] - r.o[0], j0 = c[1] - r.o[1], k0 = c[2] - r.o[2];
  const double* F = U + (long)f * r.G.sf;
  real zline[6];
  int nz = odd[2] ? 6 : 1, ny = odd[1] ? 6 : 1, nx = odd[0] ? 6 : 1;
  for (int c2 = 0; c2 < nz; ++c2) {
    long k = k0 + (odd[2] ? c2 - 2 : 0);
    real yline[6];
    for (int c1 = 0; c1 < ny; ++c1) {
      long j = j0 + (odd[1] ? c1 - 2 : 0);
      real xline[6];
      for (int c0 = 0; c0 < nx; ++c0) {
        long i = i0 + (odd[0] ? c0 - 2 : 0);
        xline[c0] = F[r.G.at((int)i, (int)j, (int)k)];
      }
      yline[c1] = odd[0] ? midpoint(xline) : xline[0];
    }
    zline[c2] = odd[1] ? midpoint(yline) : yline[0];
  }
  return odd[2] ? midpoint(zline) : zline[0];
}

int ghost_fill_hier(const oracle_params* P, std::vector<hpatch>& H, double* const* U, int lmin) {
  int maxl = 0, nl0 = 0, p0 = -1;
  for (int p = 0; p < (int)H.size(); ++p) {
    if (H[p].level > maxl) maxl = H[p].level;
    if (H[p].level == 0) {
      ++nl0;
      p0 = p;
    }
  }
  if (nl0 != 1) return -1;
  oracle_params P1 = *P;
  P1.bc = 1;
  if (lmin <= 0) ghost_fill(&P1, H[p0].G, U[p0], NF);
  for (int l = std::max(1, lmin); l <= maxl; ++l) {
    for (int p = 0; p < (int)H.size(); ++p) {
      const hpatch& h = H[p];
      if (h.level != l) continue;
      for (int k = -NG; k < h.n[2] + NG; ++k)
        for (int j = -NG; j < h.n[1] + NG; ++j)
          for (int i = -NG; i < h.n[0] + NG; ++i) {
            if (i >= 0 && i < h.n[0] && j >= 0 && j < h.n[1] && k >= 0 && k < h.n[2]) continue;
            long g[3] = {h.o[0] + i, h.o[1] + j, h.o[2] + k};
            long dst = h.G.at(i, j, k);
            int q = find_patch(H, l, g, p);
            if (q >= 0) {
              long src = H[q].G.at((int)(g[0] - H[q].o[0]), (int)(g[1] - H[q].o[1]), (int)(g[2] - H[q].o[2]));
              for (int f = 0; f < NF; ++f) U[p][(long)f * h.G.sf + dst] = U[q][(long)f * H[q].G.sf + src];
              continue;
            }
            long c[3];
            int odd[3];
            for (int a = 0; a < 3; ++a) {
              c[a] = floor_half(g[a]);
              odd[a] = (int)(g[a] - 2 * c[a]);
            }
            int r = find_patch(H, l - 1, c, -1);
            if (r < 0) return -2;
            for (int f = 0; f < NF; ++f) U[p][(long)f * h.G.sf + dst] = dbl(prolong(H[r], U[r], f, c, odd));
          }
    }
  }
  return 0;
}

int restrict_hier(std::vector<hpatch>& H, double* const* U) {
  int maxl = 0;
  for (const auto& h : H)
    if (h.level > maxl) maxl = h.level;
  for (int l = maxl; l >= 1; --l)
    for (int p = 0; p < (int)H.size(); ++p) {
      const hpatch& h = H[p];
      if (h.level != l) continue;
      for (int k = 0; k < h.n[2]; ++k)
        for (int j = 0; j < h.n[1]; ++j)
          for (int i = 0; i < h.n[0]; ++i) {
            long g[3] = {h.o[0] + i, h.o[1] + j, h.o[2] + k};
            if ((g[0] & 1) || (g[1] & 1) || (g[2] & 1)) continue;
            long c[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
            int r = find_patch(H, l - 1, c, -1);
            if (r < 0) continue;
            long dst = H[r].G.at((int)(c[0] - H[r].o[0]), (int)(c[1] - H[r].o[1]), (int)(c[2] - H[r].o[2]));
            long src = h.G.at(i, j, k);
            for (int f = 0; f < NF; ++f) U[r][(long)f * H[r].G.sf + dst] = U[p][(long)f * h.G.sf + src];
          }
    }
  return 0;
}

// Dense-output polynomials b_j(theta) = sum_p bcoef[j][p] theta^p (Sec. III A):
// RK4 with the third-order interpolator, SSP-RK3 with the second-order one.
const double kDenseRk4[4][4] = {
    {0.0, 1.0, -1.5, 2.0 / 3.0}, {0.0, 0.0, 1.0, -2.0 / 3.0}, {0.0, 0.0, 1.0, -2.0 / 3.0}, {0.0, 0.0, -0.5, 2.0 / 3.0}};
const double kDenseRk3[3][4] = {{0.0, 1.0, -5.0 / 6.0, 0.0}, {0.0, 0.0, 1.0 / 6.0, 0.0}, {0.0, 0.0, 4.0 / 6.0, 0.0}};

double bcoef(int rk, int j, int p) { return rk == 1 ? kDenseRk3[j][p] : kDenseRk4[j][p]; }
double fact(int m) { return m <= 1 ? 1.0 : m * fact(m - 1); }

// D_m (m = 1..3) from the stages' k_j: D[m-1] = m! sum_j bcoef[j][m] k_j;
// D[3] = J = 4 (k3 - k2) for RK4 (0 for SSP-RK3).
void dense_derivs(int rk, const double* k, double* D) {
  const int ns = rk == 1 ? 3 : 4;
  for (int m = 1; m <= 3; ++m) {
    real s = 0.0;
    for (int j = 0; j < ns; ++j) s = s + fact(m) * bcoef(rk, j, m) * real(k[j]);
    D[m - 1] = dbl(s);
  }
  D[3] = rk == 1 ? 0.0 : dbl(4.0 * (real(k[2]) - real(k[1])));
}

// Coefficients c[0..4] of (U^n, D_1, D_2, D_3, J) in the stage value Y_s of
// fine step msub of R (theta0 = msub / R, h = dt / R).
void bor_coeffs(int rk, int msub, int R, int s, double c[5]) {
  const double th = (double)msub / R, r = 1.0 / R;
  // T[i][m]: coefficient of D_m (D_0 = U^n) in P_i = h^i U^(i)(t0).
  double T[4][4] = {};
  for (int m = 0; m < 4; ++m) T[0][m] = std::pow(th, m) / fact(m);
  for (int i = 1; i < 4; ++i)
    for (int m = i; m < 4; ++m) T[i][m] = std::pow(r, i) * std::pow(th, m - i) / fact(m - i);
  // Y_s = sum_i w[i] P_i + wj P_J.
  double w[4] = {1.0, 0.0, 0.0, 0.0}, wj = 0.0;
  if (rk == 1) {
    if (s == 1) w[1] = 1.0;
    if (s == 2) {
      w[1] = 0.5;
      w[2] = 0.25;
    }
  } else {
    if (s == 1) w[1] = 0.5;
    if (s == 2) {
      w[1] = 0.5;
      w[2] = 0.25;
      w[3] = 1.0 / 16.0;
      wj = -1.0 / 16.0;
    }
    if (s == 3) {
      w[1] = 1.0;
      w[2] = 0.5;
      w[3] = 0.125;
      wj = 0.125;
    }
  }
  for (int m = 0; m < 4; ++m) {
    double v = 0.0;
    for (int i = 0; i < 4; ++i) v += w[i] * T[i][m];
    c[m] = v;
  }
  c[4] = wj * r * r * r;
}

void restrict_level(std::vector<hpatch>& H, int l, double* const* U) {
  for (int p = 0; p < (int)H.size(); ++p) {
    const hpatch& h = H[p];
    if (h.level != l) continue;
    for (int k = 0; k < h.n[2]; ++k)
      for (int j = 0; j < h.n[1]; ++j)
        for (int i = 0; i < h.n[0]; ++i) {
          long g[3] = {h.o[0] + i, h.o[1] + j, h.o[2] + k};
          if ((g[0] & 1) || (g[1] & 1) || (g[2] & 1)) continue;
          long c[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
          int r = find_patch(H, l - 1, c, -1);
          if (r < 0) continue;
          long dst = H[r].G.at((int)(c[0] - H[r].o[0]), (int)(c[1] - H[r].o[1]), (int)(c[2] - H[r].o[2]));
          long src = h.G.at(i, j, k);
          for (int f = 0; f < NF; ++f) U[r][(long)f * H[r].G.sf + dst] = U[p][(long)f * h.G.sf + src];
        }
  }
}

struct sub_state {
  const oracle_params* P;
  const oracle_eos_table* E;
  std::vector<hpatch>* H;
  int maxl, p0;
  double* const* U[4];
  double* const* prim;
  int8_t* const* status;
  // per patch: U^n, D_1, D_2, D_3, J (levels below the finest), and dt * RHS per stage
  std::vector<std::vector<double>> dense[5];
  std::vector<std::vector<double>> k[4];
};

// Ghost points of level l's dense arrays: extrapolation on level 0, copies from
// same-level interiors on finer levels, NaN elsewhere.
void dense_ghosts(sub_state& S, int l) {
  std::vector<hpatch>& H = *S.H;
  oracle_params P1 = *S.P;
  P1.bc = 1;
  for (int p = 0; p < (int)H.size(); ++p) {
    const hpatch& h = H[p];
    if (h.level != l) continue;
    for (int d = 0; d < 5; ++d) {
      double* A = S.dense[d][p].data();
      if (l == 0) {
        ghost_fill(&P1, h.G, A, NF);
        continue;
      }
      for (int k = -NG; k < h.n[2] + NG; ++k)
        for (int j = -NG; j < h.n[1] + NG; ++j)
          for (int i = -NG; i < h.n[0] + NG; ++i) {
            if (i >= 0 && i < h.n[0] && j >= 0 && j < h.n[1] && k >= 0 && k < h.n[2]) continue;
            long g[3] = {h.o[0] + i, h.o[1] + j, h.o[2] + k};
            long dst = h.G.at(i, j, k);
            int q = find_patch(H, l, g, p);
            for (int f = 0; f < NF; ++f) {
              double v = std::nan("");
              if (q >= 0)
                v = S.dense[d][q][(long)f * H[q].G.sf +
                                  H[q].G.at((int)(g[0] - H[q].o[0]), (int)(g[1] - H[q].o[1]), (int)(g[2] - H[q].o[2]))];
              A[(long)f * h.G.sf + dst] = v;
            }
          }
    }
  }
}

// Ghost fill of register `in` of the level-l patches (l >= 1) for fine step
// msub, stage s: same-level copies, else the prolongation of the parent's
// stage value c0 U^n + c1 D_1 + c2 D_2 + c3 D_3.
int fill_level_sub(sub_state& S, int l, double* const* in, int msub, int s) {
  std::vector<hpatch>& H = *S.H;
  double c[5];
  bor_coeffs(S.P->rk, msub, 2, s, c);
  // The parent level's stage value on its whole ghosted patches.
  std::vector<std::vector<double>> T(H.size());
  for (int r = 0; r < (int)H.size(); ++r) {
    if (H[r].level != l - 1) continue;
    const size_t n = (size_t)NF * H[r].G.sf;
    T[r].resize(n);
    for (size_t o = 0; o < n; ++o)
      T[r][o] = dbl((((c[0] * real(S.dense[0][r][o]) + c[1] * real(S.dense[1][r][o])) + c[2] * real(S.dense[2][r][o])) +
                     c[3] * real(S.dense[3][r][o])) +
                    c[4] * real(S.dense[4][r][o]));
  }
  for (int p = 0; p < (int)H.size(); ++p) {
    const hpatch& h = H[p];
    if (h.level != l) continue;
    for (int k = -NG; k < h.n[2] + NG; ++k)
      for (int j = -NG; j < h.n[1] + NG; ++j)
        for (int i = -NG; i < h.n[0] + NG; ++i) {
          if (i >= 0 && i < h.n[0] && j >= 0 && j < h.n[1] && k >= 0 && k < h.n[2]) continue;
          long g[3] = {h.o[0] + i, h.o[1] + j, h.o[2] + k};
          long dst = h.G.at(i, j, k);
          int q = find_patch(H, l, g, p);
          if (q >= 0) {
            long src = H[q].G.at((int)(g[0] - H[q].o[0]), (int)(g[1] - H[q].o[1]), (int)(g[2] - H[q].o[2]));
            for (int f = 0; f < NF; ++f) in[p][(long)f * h.G.sf + dst] = in[q][(long)f * H[q].G.sf + src];
            continue;
          }
          long cc[3];
          int odd[3];
          for (int a = 0; a < 3; ++a) {
            cc[a] = floor_half(g[a]);
            odd[a] = (int)(g[a] - 2 * cc[a]);
          }
          int r = find_patch(H, l - 1, cc, -1);
          if (r < 0) return -2;
          for (int f = 0; f < NF; ++f) {
            double v = dbl(prolong(H[r], T[r].data(), f, cc, odd));
            if (!std::isfinite(v)) return -4;
            in[p][(long)f * h.G.sf + dst] = v;
          }
        }
  }
  return 0;
}

// One step of level l (fine step msub of its parent's step), then the
// recursion into level l + 1 and its restriction.
int advance(sub_state& S, int l, int msub, double dt, int* worst) {
  std::vector<hpatch>& H = *S.H;
  const int rk = S.P->rk, ns = rk == 1 ? 3 : 4;
  const bool parent = l < S.maxl;
  static const int in_rk4[4] = {0, 1, 2, 1}, in_rk3[3] = {0, 1, 2};
  for (int s = 0; s < ns; ++s) {
    double* const* in = S.U[rk == 1 ? in_rk3[s] : in_rk4[s]];
    if (l == 0) {
      oracle_params P1 = *S.P;
      P1.bc = 1;
      ghost_fill(&P1, H[S.p0].G, in[S.p0], NF);
    } else {
      int rc = fill_level_sub(S, l, in, msub, s);
      if (rc) return rc;
    }
    for (int p = 0; p < (int)H.size(); ++p) {
      if (H[p].level != l) continue;
      const size_t n = (size_t)NF * H[p].G.sf;
      if (parent && s == 0) S.dense[0][p].assign(S.U[0][p], S.U[0][p] + n);
      std::vector<double> krhs(n, 0.0);
      int w = substep(S.P, S.E, H[p].G, s, dt, S.U[0][p], S.U[1][p], S.U[2][p], S.U[3][p], S.prim[p], S.status[p],
                      krhs.data(), nullptr);
      if (w < *worst) *worst = w;
      if (parent) {
        S.k[s][p].resize(n);
        for (size_t o = 0; o < n; ++o) S.k[s][p][o] = dbl(dt * real(krhs[o]));
      }
    }
  }
  if (!parent) return 0;
  for (int p = 0; p < (int)H.size(); ++p) {
    if (H[p].level != l) continue;
    const size_t n = (size_t)NF * H[p].G.sf;
    for (int d = 1; d < 5; ++d) S.dense[d][p].assign(n, 0.0);
    for (int f = 0; f < NF; ++f)
      for (int k = 0; k < H[p].n[2]; ++k)
        for (int j = 0; j < H[p].n[1]; ++j)
          for (int i = 0; i < H[p].n[0]; ++i) {
            const long o = (long)f * H[p].G.sf + H[p].G.at(i, j, k);
            double kk[4] = {0, 0, 0, 0}, D[4];
            for (int s = 0; s < ns; ++s) kk[s] = S.k[s][p][o];
            dense_derivs(rk, kk, D);
            for (int d = 1; d < 5; ++d) S.dense[d][p][o] = D[d - 1];
          }
  }
  dense_ghosts(S, l);
  for (int m = 0; m < 2; ++m) {
    int rc = advance(S, l + 1, m, 0.5 * dt, worst);
    if (rc) return rc;
  }
  restrict_level(H, l + 1, S.U[0]);
  return 0;
}

}  // namespace

extern "C" {

// Dense-output time derivatives (D_1, D_2, D_3) and J of one step from its
// k_j = dt f (rk 0: RK4, four k; rk 1: SSP-RK3, three k); D[4].
void oracle_dense_derivs(int rk, const double* k, double* D) { dense_derivs(rk, k, D); }

// Coefficients of (U^n, D_1, D_2, D_3, J) in stage s of fine step msub of R; c[5].
void oracle_bor_coeffs(int rk, int msub, int R, int s, double* c) { bor_coeffs(rk, msub, R, s, c); }

// One step of the whole hierarchy with sub-cycling: level 0 advances by dt0,
// level l by 2^l steps of dt0 / 2^l (Sec. IV C, BOR).  P->bc must be 3.
// Returns the worst con2prim status, or -2 (uncovered ghost point), -3 (bc),
// -4 (a prolongation stencil reached an undefined dense-output ghost point).
int oracle_hier_subcycle_step(const oracle_params* P, const oracle_eos_table* E, int np, const int* meta,
                              const double* dx, double dt0, double* const* U0, double* const* U1, double* const* U2,
                              double* const* U3, double* const* prim, int8_t* const* status) {
  if (P->bc != 3) return -3;
  std::vector<hpatch> H = parse(np, meta, dx);
  sub_state S;
  S.P = P;
  S.E = E;
  S.H = &H;
  S.maxl = 0;
  S.p0 = -1;
  int nl0 = 0;
  for (int p = 0; p < np; ++p) {
    if (H[p].level > S.maxl) S.maxl = H[p].level;
    if (H[p].level == 0) {
      S.p0 = p;
      ++nl0;
    }
  }
  if (nl0 != 1) return -1;
  S.U[0] = U0;
  S.U[1] = U1;
  S.U[2] = U2;
  S.U[3] = U3;
  S.prim = prim;
  S.status = status;
  for (int d = 0; d < 5; ++d) S.dense[d].resize(np);
  for (int d = 0; d < 4; ++d) S.k[d].resize(np);
  int worst = 0;
  int rc = advance(S, 0, 0, dt0, &worst);
  return rc ? rc : worst;
}


// meta[np][8] = (n0, n1, n2, px, level, o0, o1, o2); dx[np]; U[np] the
// register to fill.  Returns 0, or -1 (not exactly one level-0 patch), -2 (a
// ghost point covered by neither its level nor the next coarser one).
int oracle_hier_ghost_fill(const oracle_params* P, int np, const int* meta, const double* dx, double* const* U) {
  std::vector<hpatch> H = parse(np, meta, dx);
  return ghost_fill_hier(P, H, U, 0);
}

// The same from level lmin on: lmin >= 1 leaves the level-0 patch's outer
// ghosts as they are.
int oracle_hier_ghost_fill_from(const oracle_params* P, int np, const int* meta, const double* dx, double* const* U,
                                int lmin) {
  std::vector<hpatch> H = parse(np, meta, dx);
  return ghost_fill_hier(P, H, U, lmin);
}

int oracle_hier_restrict(int np, const int* meta, const double* dx, double* const* U) {
  std::vector<hpatch> H = parse(np, meta, dx);
  return restrict_hier(H, U);
}

// One Runge-Kutta step (RK4, or SSP-RK3 when P->rk = 1) of the whole
// hierarchy with time step dt on every level: per
// substep the hierarchy ghost fill of the stage's input register, then each
// patch's con2prim, right-hand side and stage update; finally the restriction
// of U^{n+1}.  P->bc must be 3 (ghosts are filled here, not per patch).
int oracle_hier_rk4_step_mask(const oracle_params* P, const oracle_eos_table* E, int np, const int* meta,
                              const double* dx, double dt, double* const* U0, double* const* U1,
                              double* const* U2, double* const* U3, double* const* prim, int8_t* const* status,
                              int rmask);

int oracle_hier_rk4_step(const oracle_params* P, const oracle_eos_table* E, int np, const int* meta,
                         const double* dx, double dt, double* const* U0, double* const* U1, double* const* U2,
                         double* const* U3, double* const* prim, int8_t* const* status) {
  return oracle_hier_rk4_step_mask(P, E, np, meta, dx, dt, U0, U1, U2, U3, prim, status, -1);
}

// As oracle_hier_rk4_step, restricting after the step only the levels l >= 1
// whose bit (1 << l) is set in rmask (finest first).
int oracle_hier_rk4_step_mask(const oracle_params* P, const oracle_eos_table* E, int np, const int* meta,
                              const double* dx, double dt, double* const* U0, double* const* U1,
                              double* const* U2, double* const* U3, double* const* prim, int8_t* const* status,
                              int rmask) {
  if (P->bc != 3) return -3;
  std::vector<hpatch> H = parse(np, meta, dx);
  int worst = 0;
  const int nsub = P->rk == 1 ? 3 : 4;
  for (int s = 0; s < nsub; ++s) {
    double* const* in = s == 0 ? U0 : s == 1 ? U1 : s == 2 ? U2 : U1;
    int rc = ghost_fill_hier(P, H, in, 0);
    if (rc) return rc;
    for (int p = 0; p < np; ++p) {
      std::vector<double> k((size_t)NF * H[p].G.sf, 0.0);
      int w = substep(P, E, H[p].G, s, dt, U0[p], U1[p], U2[p], U3[p], prim[p], status[p], k.data(), nullptr);
      if (w < worst) worst = w;
    }
  }
  int maxl = 0;
  for (const auto& h : H)
    if (h.level > maxl) maxl = h.level;
  for (int l = maxl; l >= 1; --l)
    if (rmask & (1 << l)) restrict_level(H, l, U0);
  return worst;
}

}  // extern "C"
