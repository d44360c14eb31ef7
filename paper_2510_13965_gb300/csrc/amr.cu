// Mesh-refinement ghost fill and restriction for a fixed hierarchy advanced
// without sub-cycling (Sec. III D, prolongation and restriction).
//
// The host turns the patch layout into task lists once, at context creation:
// every ghost point of a level-l patch (l >= 1) becomes one task, a copy from
// the interior of another level-l patch when one covers it, else a
// prolongation from the level-(l-1) patch whose interior holds floor(g/2);
// every interior point of a level-l patch at even level-l coordinates becomes
// one restriction task (copy into the coarse interior point g/2).  One thread
// executes one task for all 32 fields; tasks of one kind are contiguous so
// warps do not diverge between kinds.  Level l's ghost tasks read only
// level-l interiors and level-(l-1) data (ghosts included), so the levels are
// filled in order, one launch each, after the level-0 patch's outer
// extrapolation.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>
#include "kern.cuh"

namespace gk {

// The paper's six-point Lagrange midpoint formula on u[0..5] = U_{c-2..c+3}:
//   U_{c+1/2} = [150 (U_c + U_{c+1}) - 25 (U_{c-1} + U_{c+2}) + 3 (U_{c-2} + U_{c+3})] / 256,
// rounded operation by operation in this order (no contraction).
DI double mid6(const double* u) {
  double a = __dmul_rn(150.0, __dadd_rn(u[2], u[3]));
  double b = __dmul_rn(25.0, __dadd_rn(u[1], u[4]));
  double c = __dmul_rn(3.0, __dadd_rn(u[0], u[5]));
  return __dmul_rn(__dadd_rn(__dsub_rn(a, b), c), 0.00390625);
}

// Tensor-product prolongation from base point p (the coarse point c) of one
// field: along each axis with its bit set in odd, the midpoint formula over
// offsets -2..3; x first, then y, then z.
DI double prolong(const double* p, long long sy, long long sz, int odd) {
  const bool ox = odd & 1, oy = odd & 2, oz = odd & 4;
  double zl[6];
  const int nz = oz ? 6 : 1, ny = oy ? 6 : 1;
  for (int c2 = 0; c2 < nz; ++c2) {
    const double* pz = p + (oz ? (c2 - 2) * sz : 0);
    double yl[6];
    for (int c1 = 0; c1 < ny; ++c1) {
      const double* py = pz + (oy ? (c1 - 2) * sy : 0);
      if (ox) {
        double xl[6];
#pragma unroll
        for (int c0 = 0; c0 < 6; ++c0) xl[c0] = py[c0 - 2];
        yl[c1] = mid6(xl);
      } else {
        yl[c1] = py[0];
      }
    }
    zl[c2] = oy ? mid6(yl) : yl[0];
  }
  return oz ? mid6(zl) : zl[0];
}

__global__ void __launch_bounds__(256) k_amr(const PatchDev* __restrict__ pd, const AmrTask* __restrict__ t,
                                              long long n, int reg) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrTask T = t[q];
  const PatchDev& D = pd[T.dst];
  const PatchDev& S = pd[T.src];
  double* d = D.U[reg] + T.dofs;
  const double* s = S.U[reg] + T.sofs;
  if (T.odd == 0) {
    for (int f = 0; f < NF; ++f) d[f * D.G.sf] = s[f * S.G.sf];
  } else {
    for (int f = 0; f < NF; ++f) d[f * D.G.sf] = prolong(s + f * S.G.sf, S.G.sy, S.G.sz, T.odd);
  }
}

void launch_amr(const PatchDev* pd, const AmrTask* t, long long n, int reg, cudaStream_t st) {
  if (n <= 0) return;
  k_amr<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, t, n, reg);
}

namespace {

long long floor_half(long long g) { return g >= 0 ? g / 2 : -((-g + 1) / 2); }

// Dense owner map of the interiors of one level's patches.
struct LevelMap {
  long long lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0};
  std::vector<int> owner;
  int at(const long long g[3]) const {
    long long r[3];
    for (int a = 0; a < 3; ++a) {
      r[a] = g[a] - lo[a];
      if (r[a] < 0 || r[a] >= ext[a]) return -1;
    }
    return owner[(size_t)((r[2] * ext[1] + r[1]) * ext[0] + r[0])];
  }
};

long long offset(const Geo& G, long long i, long long j, long long k) {
  return (k + 3) * G.sz + (j + 3) * G.sy + (i + 3);
}

}  // namespace

int amr_plan(const grmhd_patch_desc* d, const std::vector<Geo>& geo, int np, AmrPlan& P) {
  P = AmrPlan();
  int nl0 = 0, maxl = 0;
  for (int p = 0; p < np; ++p) {
    if (d[p].level < 0 || d[p].level > 20) {
      P.err = "hierarchy: level out of range";
      return GRMHD_ERR_ARG;
    }
    if (d[p].level == 0) {
      ++nl0;
      P.level0 = p;
    }
    if (d[p].level > maxl) maxl = d[p].level;
  }
  if (nl0 != 1) {
    P.err = "hierarchy: exactly one level-0 patch is required";
    return GRMHD_ERR_ARG;
  }
  P.nlev = maxl + 1;
  const grmhd_patch_desc& d0 = d[P.level0];
  std::vector<std::array<long long, 3>> org(np);
  for (int p = 0; p < np; ++p) {
    double dxl = d0.dx / std::ldexp(1.0, d[p].level);
    if (std::fabs(d[p].dx - dxl) > 1e-12 * dxl) {
      P.err = "hierarchy: patch spacing is not dx0 / 2^level";
      return GRMHD_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a) {
      double f = (d[p].x0[a] - d0.x0[a]) / dxl;
      long long o = std::llround(f);
      if (std::fabs(f - (double)o) > 1e-6) {
        P.err = "hierarchy: patch origin is not on its level's grid";
        return GRMHD_ERR_ARG;
      }
      org[p][a] = o;
    }
  }
  // Owner maps per level.
  std::vector<LevelMap> maps(P.nlev);
  for (int l = 0; l < P.nlev; ++l) {
    LevelMap& M = maps[l];
    bool any = false;
    long long hi[3] = {0, 0, 0};
    for (int p = 0; p < np; ++p) {
      if (d[p].level != l) continue;
      for (int a = 0; a < 3; ++a) {
        long long a0 = org[p][a], a1 = org[p][a] + d[p].n[a];
        if (!any || a0 < M.lo[a]) M.lo[a] = a0;
        if (!any || a1 > hi[a]) hi[a] = a1;
      }
      any = true;
    }
    if (!any) {
      P.err = "hierarchy: a level between 0 and the finest has no patch";
      return GRMHD_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a) M.ext[a] = hi[a] - M.lo[a];
    double cells = (double)M.ext[0] * (double)M.ext[1] * (double)M.ext[2];
    if (cells > 2e9) {
      P.err = "hierarchy: level bounding box too large";
      return GRMHD_ERR_ARG;
    }
    M.owner.assign((size_t)cells, -1);
    for (int p = 0; p < np; ++p) {
      if (d[p].level != l) continue;
      for (long long k = 0; k < d[p].n[2]; ++k)
        for (long long j = 0; j < d[p].n[1]; ++j)
          for (long long i = 0; i < d[p].n[0]; ++i) {
            long long r0 = org[p][0] + i - M.lo[0], r1 = org[p][1] + j - M.lo[1], r2 = org[p][2] + k - M.lo[2];
            int& o = M.owner[(size_t)((r2 * M.ext[1] + r1) * M.ext[0] + r0)];
            if (o >= 0) {
              P.err = "hierarchy: patches of one level overlap";
              return GRMHD_ERR_ARG;
            }
            o = p;
          }
    }
  }
  P.ghost.assign(P.nlev, {});
  P.restr.assign(P.nlev, {});
  for (int p = 0; p < np; ++p) {
    const int l = d[p].level;
    if (l == 0) continue;
    const Geo& Gp = geo[p];
    const int n0 = d[p].n[0], n1 = d[p].n[1], n2 = d[p].n[2];
    for (int k = -3; k < n2 + 3; ++k)
      for (int j = -3; j < n1 + 3; ++j)
        for (int i = -3; i < n0 + 3; ++i) {
          bool inner = i >= 0 && i < n0 && j >= 0 && j < n1 && k >= 0 && k < n2;
          long long g[3] = {org[p][0] + i, org[p][1] + j, org[p][2] + k};
          if (inner) {
            if ((g[0] & 1) || (g[1] & 1) || (g[2] & 1)) continue;
            long long c[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
            int r = maps[l - 1].at(c);
            if (r < 0) continue;
            P.restr[l].push_back(AmrTask{r, (int)offset(geo[r], c[0] - org[r][0], c[1] - org[r][1], c[2] - org[r][2]),
                                         p, (int)offset(Gp, i, j, k), 0});
            continue;
          }
          int q = maps[l].at(g);
          if (q >= 0) {
            P.ghost[l].push_back(AmrTask{p, (int)offset(Gp, i, j, k), q,
                                         (int)offset(geo[q], g[0] - org[q][0], g[1] - org[q][1], g[2] - org[q][2]),
                                         0});
            continue;
          }
          long long c[3];
          int odd = 0;
          for (int a = 0; a < 3; ++a) {
            c[a] = floor_half(g[a]);
            if (g[a] - 2 * c[a]) odd |= 1 << a;
          }
          int r = maps[l - 1].at(c);
          if (r < 0) {
            P.err = "hierarchy: a ghost point of a fine patch lies outside the next coarser level";
            return GRMHD_ERR_ARG;
          }
          P.ghost[l].push_back(AmrTask{p, (int)offset(Gp, i, j, k), r,
                                       (int)offset(geo[r], c[0] - org[r][0], c[1] - org[r][1], c[2] - org[r][2]), odd});
        }
  }
  // Group each level's ghost tasks by kind (copy, then each set of midpoint
  // axes), keeping their spatial order: the kinds cost 0 to ~390 FP64
  // operations per field, and a warp of mixed kinds runs all their paths.
  for (auto& v : P.ghost)
    std::stable_sort(v.begin(), v.end(), [](const AmrTask& a, const AmrTask& b) {
      int ka = __builtin_popcount(a.odd), kb = __builtin_popcount(b.odd);
      return ka != kb ? ka < kb : a.odd < b.odd;
    });
  return GRMHD_OK;
}

}  // namespace gk
