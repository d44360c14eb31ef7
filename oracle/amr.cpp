// Oracle of the mesh-refinement ghost fill and restriction (Sec. III D,
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
#include <cmath>
#include <cstdint>
#include <vector>

#include "oracle.hpp"

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

int ghost_fill_hier(const oracle_params* P, std::vector<hpatch>& H, double* const* U) {
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
  ghost_fill(&P1, H[p0].G, U[p0], NF);
  for (int l = 1; l <= maxl; ++l) {
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

}  // namespace

extern "C" {

// meta[np][8] = (n0, n1, n2, px, level, o0, o1, o2); dx[np]; U[np] the
// register to fill.  Returns 0, or -1 (not exactly one level-0 patch), -2 (a
// ghost point covered by neither its level nor the next coarser one).
int oracle_hier_ghost_fill(const oracle_params* P, int np, const int* meta, const double* dx, double* const* U) {
  std::vector<hpatch> H = parse(np, meta, dx);
  return ghost_fill_hier(P, H, U);
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
int oracle_hier_rk4_step(const oracle_params* P, const oracle_eos_table* E, int np, const int* meta,
                         const double* dx, double dt, double* const* U0, double* const* U1, double* const* U2,
                         double* const* U3, double* const* prim, int8_t* const* status) {
  if (P->bc != 3) return -3;
  std::vector<hpatch> H = parse(np, meta, dx);
  int worst = 0;
  const int nsub = P->rk == 1 ? 3 : 4;
  for (int s = 0; s < nsub; ++s) {
    double* const* in = s == 0 ? U0 : s == 1 ? U1 : s == 2 ? U2 : U1;
    int rc = ghost_fill_hier(P, H, in);
    if (rc) return rc;
    for (int p = 0; p < np; ++p) {
      std::vector<double> k((size_t)NF * H[p].G.sf, 0.0);
      int w = substep(P, E, H[p].G, s, dt, U0[p], U1[p], U2[p], U3[p], prim[p], status[p], k.data(), nullptr);
      if (w < worst) worst = w;
    }
  }
  restrict_hier(H, U0);
  return worst;
}

}  // extern "C"
