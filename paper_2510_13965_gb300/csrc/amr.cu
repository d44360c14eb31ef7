// Mesh-refinement ghost fill and restriction for a fixed hierarchy advanced
// without sub-cycling (Sec. IV B, prolongation and restriction).
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

// Tensor-product prolongation around the coarse base point of one field:
// along each axis with its bit set in odd, the midpoint formula over offsets
// -2..3; x first, then y, then z.  rd(off) reads the coarse value at offset
// off (in points of the coarse patch's layout) from the base point.
template <bool XPRE, class Rd, class RdX>
DI double prolong(Rd rd, RdX rdx, long long sy, long long sz, int odd) {
  const bool ox = odd & 1, oy = odd & 2, oz = odd & 4;
  double zl[6];
  const int nz = oz ? 6 : 1, ny = oy ? 6 : 1;
#pragma unroll 1
  for (int c2 = 0; c2 < nz; ++c2) {
    const long long pz = oz ? (c2 - 2) * sz : 0;
    double yl[6];
    for (int c1 = 0; c1 < ny; ++c1) {
      const long long py = pz + (oy ? (c1 - 2) * sy : 0);
      if (ox) {
        if (XPRE) {
          yl[c1] = rdx(py);  // the x-midpoint of this row, computed by k_amr_xmid
        } else {
          double xl[6];
#pragma unroll
          for (int c0 = 0; c0 < 6; ++c0) xl[c0] = rd(py + c0 - 2);
          yl[c1] = mid6(xl);
        }
      } else {
        yl[c1] = rd(py);
      }
    }
    zl[c2] = oy ? mid6(yl) : yl[0];
  }
  return oz ? mid6(zl) : zl[0];
}

// x-midpoints of a coarse level, once per coarse row that the finer level's
// stencils read: X(c) = mid6(U(c-2 .. c+3)) along x, into the patch's
// pointwise-flux scratch (free during a ghost fill; 33 doubles per point).
__global__ void __launch_bounds__(256) k_amr_xmid(const PatchDev* __restrict__ pd, const AmrPoint* __restrict__ p,
                                                   long long n, int reg) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrPoint P = p[q];
  const PatchDev& S = pd[P.patch];
  const double* u = S.U[reg] + P.ofs;
  double* x = S.Fp + P.ofs;
  for (int f = 0; f < NF; ++f) {
    const double* uf = u + f * S.G.sf;
    double xl[6];
#pragma unroll
    for (int c0 = 0; c0 < 6; ++c0) xl[c0] = uf[c0 - 2];
    x[f * S.G.sf] = mid6(xl);
  }
}

void launch_amr_xmid(const PatchDev* pd, const AmrPoint* pts, long long n, int reg, cudaStream_t st) {
  if (n <= 0) return;
  k_amr_xmid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, pts, n, reg);
}

template <bool XPRE>
__global__ void __launch_bounds__(256) k_amr(const PatchDev* __restrict__ pd, const AmrTask* __restrict__ t,
                                              long long n, int reg, int reg_coarse) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrTask T = t[q];
  const PatchDev& D = pd[T.dst];
  const PatchDev& S = pd[T.src];
  double* d = D.U[reg] + T.dofs;
  const double* s = S.U[(T.odd & AMR_COARSE) ? reg_coarse : reg] + T.sofs;
  const int odd = T.odd & 7;
  if (odd == 0) {
    for (int f = 0; f < NF; ++f) d[f * D.G.sf] = s[f * S.G.sf];
  } else {
    const double* xs = S.Fp + T.sofs;
    for (int f = 0; f < NF; ++f) {
      const double* sf = s + f * S.G.sf;
      const double* xf = xs + f * S.G.sf;
      d[f * D.G.sf] = prolong<XPRE>([sf](long long off) { return sf[off]; }, [xf](long long off) { return xf[off]; },
                                    S.G.sy, S.G.sz, odd);
    }
  }
}

void launch_amr(const PatchDev* pd, const AmrTask* t, long long n, int reg, cudaStream_t st, int reg_coarse,
                bool xpre) {
  if (n <= 0) return;
  const int rc = reg_coarse < 0 ? reg : reg_coarse;
  if (xpre)
    k_amr<true><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, t, n, reg, rc);
  else
    k_amr<false><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, t, n, reg, rc);
}

// Sub-cycled ghost fill (Sec. IV C, BOR), first pass: at every coarse point
// that the level's prolongation stencils read, the stage value
// ((((c0 U^n + c1 D_1) + c2 D_2) + c3 D_3) + c4 J) of the coarse level's dense
// output, rounded operation by operation, into register reg_t (the coarse
// patch's RK accumulator, free between its steps).  The ghost fill proper then
// prolongates from reg_t.
struct DenseCoef {
  double c[NDENSE];
};
__global__ void __launch_bounds__(256) k_amr_time(const PatchDev* __restrict__ pd, const AmrPoint* __restrict__ p,
                                                   long long n, DenseCoef K, int nd, int reg_t) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrPoint P = p[q];
  const PatchDev& S = pd[P.patch];
  double* out = S.U[reg_t] + P.ofs;
  const double* src[NDENSE];
#pragma unroll
  for (int e = 0; e < NDENSE; ++e) src[e] = e < nd ? S.U[REG_DENSE + e] + P.ofs : nullptr;
  for (int f = 0; f < NF; ++f) {
    const long long fo = f * S.G.sf;
    double v = __dmul_rn(K.c[0], src[0][fo]);
    for (int e = 1; e < nd; ++e) v = __dadd_rn(v, __dmul_rn(K.c[e], src[e][fo]));
    out[fo] = v;
  }
}

void launch_amr_time(const PatchDev* pd, const AmrPoint* pts, long long n, const double coef[NDENSE], int nd,
                     int reg_t, cudaStream_t st) {
  if (n <= 0) return;
  DenseCoef K;
  for (int e = 0; e < NDENSE; ++e) K.c[e] = coef[e];
  k_amr_time<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, pts, n, K, nd, reg_t);
}

// Dense output of a step (Sec. III A) recorded from the RK registers after
// each substep, without storing k: with k_j = dt f(Y_j),
//   RK4 (stage inputs U^n, Y2 = U^n + k1/2, Y3 = U^n + k2/2, Y4 = U^n + k3):
//     after substep 0: U^n, k1 = 2 (Y2 - U^n);  1: k2 = 2 (Y3 - U^n);
//     2: k3 = Y4 - U^n;  3: k4 = 6 (U^{n+1} - U^n) - k1 - 2 k2 - 2 k3, then
//     D_2 = -3 k1 + 2 k2 + 2 k3 - k4, D_3 = 4 (k1 - k2 - k3 + k4), J = 4 (k3 - k2);
//   SSP-RK3 (Y2 = U^n + k1, Y3 = U^n + k1/4 + k2/4):
//     0: U^n, k1 = Y2 - U^n;  1: k2 = 4 (Y3 - U^n) - k1;
//     2: k3 = 3/2 (U^{n+1} - U^n) - (k1 + k2)/4, D_2 = -5/3 k1 + 1/3 k2 + 4/3 k3.
// D_1 = k1; the D_m are the derivatives at theta = 0 of the paper's b_j(theta).
__global__ void k_dense_rec(const PatchDev* __restrict__ pd, const Work* __restrict__ w, int stage, int rk) {
  Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const Geo G = PD.G;
  long long q = (long long)wk.block * blockDim.x + threadIdx.x;
  if (q >= dom_count(DOM_INT, G)) return;
  int i, j, k;
  dom_decode(DOM_INT, G, q, i, j, k);
  const long long o = at(G, i, j, k), sf = G.sf;
  const double *U0 = PD.U[0], *U1 = PD.U[1], *U2 = PD.U[2];
  double *Sn = PD.U[REG_DENSE], *S1 = PD.U[REG_DENSE + 1], *S2 = PD.U[REG_DENSE + 2], *S3 = PD.U[REG_DENSE + 3],
         *SJ = PD.U[REG_DENSE + 4];
  for (int f = 0; f < NF; ++f) {
    const long long x = f * sf + o;
    if (rk == 1) {
      if (stage == 0) {
        const double un = U0[x];
        Sn[x] = un;
        S1[x] = U1[x] - un;
      } else if (stage == 1) {
        S2[x] = 4.0 * (U2[x] - Sn[x]) - S1[x];
      } else {
        const double k1 = S1[x], k2 = S2[x];
        const double k3 = 1.5 * (U0[x] - Sn[x]) - 0.25 * (k1 + k2);
        S2[x] = (-5.0 * k1 + k2 + 4.0 * k3) * (1.0 / 3.0);
      }
      continue;
    }
    if (stage == 0) {
      const double un = U0[x];
      Sn[x] = un;
      S1[x] = 2.0 * (U1[x] - un);
    } else if (stage == 1) {
      S2[x] = 2.0 * (U2[x] - Sn[x]);
    } else if (stage == 2) {
      S3[x] = U1[x] - Sn[x];
    } else {
      const double k1 = S1[x], k2 = S2[x], k3 = S3[x];
      const double k4 = 6.0 * (U0[x] - Sn[x]) - k1 - 2.0 * (k2 + k3);
      S2[x] = -3.0 * k1 + 2.0 * (k2 + k3) - k4;
      S3[x] = 4.0 * ((k1 - k2) - (k3 - k4));
      SJ[x] = 4.0 * (k3 - k2);
    }
  }
}

void launch_dense_rec(const PatchDev* pd, const Work* w, int nblk, int stage, int rk, cudaStream_t st) {
  if (nblk <= 0) return;
  k_dense_rec<<<nblk, BS_INT, 0, st>>>(pd, w, stage, rk);
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

// 3-D prefix sums of the points of a level's bounding box that no patch
// interior covers: box_covered answers whether a box holds none.
struct Uncovered {
  long long lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0};
  std::vector<int> ps;  // (ext0 + 1) (ext1 + 1) (ext2 + 1)
  void build(const LevelMap& M) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = M.lo[a];
      ext[a] = M.ext[a];
    }
    const long long X = ext[0] + 1, Y = ext[1] + 1;
    ps.assign((size_t)(X * Y * (ext[2] + 1)), 0);
    for (long long k = 0; k < ext[2]; ++k)
      for (long long j = 0; j < ext[1]; ++j)
        for (long long i = 0; i < ext[0]; ++i) {
          int u = M.owner[(size_t)((k * ext[1] + j) * ext[0] + i)] < 0;
          ps[(size_t)(((k + 1) * Y + (j + 1)) * X + (i + 1))] =
              u + ps[(size_t)(((k)*Y + (j + 1)) * X + (i + 1))] + ps[(size_t)(((k + 1) * Y + (j)) * X + (i + 1))] +
              ps[(size_t)(((k + 1) * Y + (j + 1)) * X + (i))] - ps[(size_t)(((k)*Y + (j)) * X + (i + 1))] -
              ps[(size_t)(((k)*Y + (j + 1)) * X + (i))] - ps[(size_t)(((k + 1) * Y + (j)) * X + (i))] +
              ps[(size_t)(((k)*Y + (j)) * X + (i))];
        }
  }
  // Inclusive box [a, b] in level coordinates.
  bool box_covered(const long long a[3], const long long b[3]) const {
    long long r0[3], r1[3];
    for (int d = 0; d < 3; ++d) {
      r0[d] = a[d] - lo[d];
      r1[d] = b[d] - lo[d] + 1;
      if (r0[d] < 0 || r1[d] > ext[d]) return false;
    }
    const long long X = ext[0] + 1, Y = ext[1] + 1;
    auto S = [&](long long i, long long j, long long k) { return (long long)ps[(size_t)((k * Y + j) * X + i)]; };
    long long n = S(r1[0], r1[1], r1[2]) - S(r0[0], r1[1], r1[2]) - S(r1[0], r0[1], r1[2]) - S(r1[0], r1[1], r0[2]) +
                  S(r0[0], r0[1], r1[2]) + S(r0[0], r1[1], r0[2]) + S(r1[0], r0[1], r0[2]) - S(r0[0], r0[1], r0[2]);
    return n == 0;
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
  P.nsame.assign(P.nlev, 0);
  // Prefix sums of uncovered points of each level's bounding box.
  std::vector<Uncovered> uncov(P.nlev);
  for (int l = 1; l + 1 < P.nlev; ++l) uncov[l].build(maps[l]);
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
                                       (int)offset(geo[r], c[0] - org[r][0], c[1] - org[r][1], c[2] - org[r][2]),
                                       odd | AMR_COARSE});
          // Sub-cycling reads the coarse level's dense output on the stencil,
          // which exists on coarse interiors (and the level-0 ghosts) only.
          if (l >= 2 && P.sub_err.empty()) {
            long long lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
              lo[a] = c[a] - ((odd >> a) & 1 ? 2 : 0);
              hi[a] = c[a] + ((odd >> a) & 1 ? 3 : 0);
            }
            if (!uncov[l - 1].box_covered(lo, hi))
              P.sub_err = "hierarchy: a prolongation stencil of level " + std::to_string(l) +
                          " leaves the interiors of level " + std::to_string(l - 1) + " (sub-cycling needs nesting)";
          }
        }
  }
  // Group each level's ghost tasks by kind (copy, then each set of midpoint
  // axes), keeping their spatial order: the kinds cost 0 to ~390 FP64
  // operations per field, and a warp of mixed kinds runs all their paths.
  // Coarse points read by each level's coarse-source tasks (unique, in patch
  // and offset order).
  P.tpts.assign(P.nlev, {});
  {
    std::vector<std::vector<uint8_t>> mark(np);
    for (int l = 1; l < P.nlev; ++l) {
      for (const auto& t : P.ghost[l]) {
        if (!(t.odd & AMR_COARSE)) continue;
        const Geo& G = geo[t.src];
        auto& m = mark[t.src];
        if (m.empty()) m.assign((size_t)G.sf, 0);
        const int ox = t.odd & 1, oy = (t.odd >> 1) & 1, oz = (t.odd >> 2) & 1;
        for (int dz = oz ? -2 : 0; dz <= (oz ? 3 : 0); ++dz)
          for (int dy = oy ? -2 : 0; dy <= (oy ? 3 : 0); ++dy)
            for (int dx = ox ? -2 : 0; dx <= (ox ? 3 : 0); ++dx)
              m[(size_t)(t.sofs + dz * G.sz + dy * G.sy + dx)] = 1;
      }
      for (int r = 0; r < np; ++r) {
        auto& m = mark[r];
        if (m.empty()) continue;
        for (size_t o = 0; o < m.size(); ++o)
          if (m[o]) P.tpts[l].push_back(AmrPoint{r, (int)o});
        m.clear();
      }
    }
    // Coarse rows whose x-midpoint the level's x-odd tasks read: base points
    // (c_x, c_y + dy, c_z + dz) over the task's y and z stencil offsets.
    P.xpts.assign(P.nlev, {});
    for (int l = 1; l < P.nlev; ++l) {
      for (const auto& t : P.ghost[l]) {
        if (!(t.odd & AMR_COARSE) || !(t.odd & 1)) continue;
        const Geo& G = geo[t.src];
        auto& m = mark[t.src];
        if (m.empty()) m.assign((size_t)G.sf, 0);
        const int oy = (t.odd >> 1) & 1, oz = (t.odd >> 2) & 1;
        for (int dz = oz ? -2 : 0; dz <= (oz ? 3 : 0); ++dz)
          for (int dy = oy ? -2 : 0; dy <= (oy ? 3 : 0); ++dy) m[(size_t)(t.sofs + dz * G.sz + dy * G.sy)] = 1;
      }
      for (int r = 0; r < np; ++r) {
        auto& m = mark[r];
        if (m.empty()) continue;
        for (size_t o = 0; o < m.size(); ++o)
          if (m[o]) P.xpts[l].push_back(AmrPoint{r, (int)o});
        m.clear();
      }
    }
  }
  // Same-level copies come first (sub-cycling fills the dense registers'
  // ghosts from them alone), then the coarse-source kinds.
  for (int l = 0; l < P.nlev; ++l) {
    auto& v = P.ghost[l];
    std::stable_sort(v.begin(), v.end(), [](const AmrTask& a, const AmrTask& b) {
      int ca = a.odd >> 3, cb = b.odd >> 3;
      if (ca != cb) return ca < cb;
      int ka = __builtin_popcount(a.odd & 7), kb = __builtin_popcount(b.odd & 7);
      return ka != kb ? ka < kb : a.odd < b.odd;
    });
    for (const auto& t : v)
      if (!(t.odd & AMR_COARSE)) ++P.nsame[l];
  }
  return GRMHD_OK;
}

}  // namespace gk
