// Patch sharding across ranks (one GPU each) for a mesh-refinement hierarchy:
// the partition of the patches and the point-to-point exchange plan.  This is
// the GPU-native counterpart of the paper's MPI box decomposition (Sec. IV A):
// every rank advances its own patches, and per Runge-Kutta substep one
// exchange of source points precedes the ghost fill.
//
// Partition: patches in Morton order of their centres (finest-level grid
// units), cut into nranks contiguous runs of about equal interior point count.
//
// Exchange plan, for a nested hierarchy (every prolongation stencil point of
// a level l >= 2 lies in an interior of level l-1; the level-0 ghosts are
// filled by extrapolation on the level-0 patch's owner first):
//  - ghost phase: every point that a rank's ghost tasks read is resolved to
//    its authoritative source: an interior point of some patch, or a level-0
//    ghost point.  A point of another patch's ghost zone (inside a
//    prolongation stencil) resolves to the interior point of the same level
//    that covers it, whose value the ghost fill would copy there.  Sources on
//    other ranks are exchanged once per substep, before the local ghost fill,
//    into mirror arrays of their patches at the points where the tasks read
//    them;
//  - restriction: every restricted coarse point takes the value of the finest
//    interior point that coincides with it (the cascade of direct copies,
//    finest level first, in one step); sources on other ranks are exchanged
//    once per step into mirrors, then copied.
// Every list is built identically on every rank from the global layout.
#include <algorithm>
#include <cstdint>
#include <map>
#include <string>
#include <unordered_set>
#include <vector>
#include "kern.cuh"

namespace gk {

namespace {

uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

}  // namespace

int shard_partition(const grmhd_patch_desc* d, int np, int nranks, int* owner) {
  if (!d || !owner || np < 1 || nranks < 1) return GRMHD_ERR_ARG;
  int L = 0;
  for (int p = 0; p < np; ++p) L = std::max(L, d[p].level);
  double x0[3] = {d[0].x0[0], d[0].x0[1], d[0].x0[2]}, fdx = d[0].dx;
  for (int p = 0; p < np; ++p) {
    fdx = std::min(fdx, d[p].dx);
    for (int a = 0; a < 3; ++a) x0[a] = std::min(x0[a], d[p].x0[a]);
  }
  std::vector<std::pair<uint64_t, int>> key(np);
  for (int p = 0; p < np; ++p) {
    uint64_t m = 0;
    for (int a = 0; a < 3; ++a) {
      double c = (d[p].x0[a] - x0[a] + 0.5 * (d[p].n[a] - 1) * d[p].dx) / fdx;
      m |= spread3((uint64_t)std::max(0.0, c)) << a;
    }
    key[p] = {m, p};
  }
  std::stable_sort(key.begin(), key.end());
  long long total = 0;
  for (int p = 0; p < np; ++p) total += (long long)d[p].n[0] * d[p].n[1] * d[p].n[2];
  long long acc = 0;
  int r = 0;
  for (const auto& kp : key) {
    const int p = kp.second;
    const long long w = (long long)d[p].n[0] * d[p].n[1] * d[p].n[2];
    // Move to the next rank once this one holds its share (centre of the
    // patch past the cut), keeping every rank non-empty while patches last.
    while (r + 1 < nranks && 2 * (acc + w / 2) * nranks > 2 * total * (r + 1) / 1) ++r;
    owner[p] = r;
    acc += w;
  }
  return GRMHD_OK;
}


namespace {

// Dense map of one level's interiors: level-grid point -> patch, or -1.
struct LevelOwner {
  long long lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0};
  std::vector<int> own;
  int at(const long long g[3]) const {
    long long r[3];
    for (int a = 0; a < 3; ++a) {
      r[a] = g[a] - lo[a];
      if (r[a] < 0 || r[a] >= ext[a]) return -1;
    }
    return own[(size_t)((r[2] * ext[1] + r[1]) * ext[0] + r[0])];
  }
};

uint64_t pkey(int p, long long o) { return ((uint64_t)(uint32_t)p << 36) | (uint64_t)o; }

}  // namespace

int shard_plan(const grmhd_patch_desc* d, const std::vector<Geo>& geo, int np, const int* owner, int nranks, int rank,
               ShardPlan& S) {
  S = ShardPlan();
  if (!d || !owner || nranks < 1 || rank < 0 || rank >= nranks) {
    S.err = "shard: arguments";
    return GRMHD_ERR_ARG;
  }
  for (int p = 0; p < np; ++p)
    if (owner[p] < 0 || owner[p] >= nranks) {
      S.err = "shard: owner out of range";
      return GRMHD_ERR_ARG;
    }
  AmrPlan P;
  if (amr_plan(d, geo, np, P) != GRMHD_OK) {
    S.err = P.err;
    return GRMHD_ERR_ARG;
  }
  S.level0 = P.level0;
  S.nlev = P.nlev;
  std::vector<std::array<long long, 3>> org(np);
  for (int p = 0; p < np; ++p) {
    const double dxl = d[P.level0].dx / std::ldexp(1.0, d[p].level);
    for (int a = 0; a < 3; ++a) org[p][a] = std::llround((d[p].x0[a] - d[P.level0].x0[a]) / dxl);
  }
  std::vector<LevelOwner> lv(P.nlev);
  for (int l = 0; l < P.nlev; ++l) {
    LevelOwner& M = lv[l];
    bool any = false;
    long long hi[3] = {0, 0, 0};
    for (int p = 0; p < np; ++p) {
      if (d[p].level != l) continue;
      for (int a = 0; a < 3; ++a) {
        if (!any || org[p][a] < M.lo[a]) M.lo[a] = org[p][a];
        if (!any || org[p][a] + d[p].n[a] > hi[a]) hi[a] = org[p][a] + d[p].n[a];
      }
      any = true;
    }
    for (int a = 0; a < 3; ++a) M.ext[a] = hi[a] - M.lo[a];
    M.own.assign((size_t)(M.ext[0] * M.ext[1] * M.ext[2]), -1);
    for (int p = 0; p < np; ++p) {
      if (d[p].level != l) continue;
      for (long long k = 0; k < d[p].n[2]; ++k)
        for (long long j = 0; j < d[p].n[1]; ++j)
          for (long long i = 0; i < d[p].n[0]; ++i)
            M.own[(size_t)(((org[p][2] + k - M.lo[2]) * M.ext[1] + (org[p][1] + j - M.lo[1])) * M.ext[0] +
                           (org[p][0] + i - M.lo[0]))] = p;
    }
  }
  // Authoritative source of point o of patch p at the time of the exchange.
  auto resolve = [&](int p, long long o, int& sp, long long& so) -> bool {
    const Geo& G = geo[p];
    const long long k = o / G.sz - 3, j = (o % G.sz) / G.sy - 3, i = o % G.sy - 3;
    const bool inner = i >= 0 && i < G.n0 && j >= 0 && j < G.n1 && k >= 0 && k < G.n2;
    if (inner || d[p].level == 0) {
      sp = p;
      so = o;
      return true;
    }
    const long long g[3] = {org[p][0] + i, org[p][1] + j, org[p][2] + k};
    const int q = lv[d[p].level].at(g);
    if (q < 0) return false;
    const Geo& Q = geo[q];
    sp = q;
    so = (g[2] - org[q][2] + 3) * Q.sz + (g[1] - org[q][1] + 3) * Q.sy + (g[0] - org[q][0] + 3);
    return true;
  };
  S.role.assign(np, 0);
  for (int p = 0; p < np; ++p)
    if (owner[p] == rank) S.role[p] = 1;
  S.gsend.assign(nranks, {});
  S.grecv.assign(nranks, {});
  S.rsend.assign(nranks, {});
  S.rrecv.assign(nranks, {});
  // One pass over every rank's ghost tasks: each point of another rank's
  // patch that a task reads is a mirror point fed by the owner of its source.
  std::vector<std::unordered_set<uint64_t>> seen(nranks);
  bool ok = true;
  auto want = [&](int rr, int p, long long o) {
    if (owner[p] == rr || !seen[rr].insert(pkey(p, o)).second) return;
    int sp;
    long long so;
    if (!resolve(p, o, sp, so)) {
      ok = false;
      return;
    }
    const int sr = owner[sp];
    if (rr == rank) {
      S.grecv[sr].push_back(AmrPoint{p, (int)o});
      if (S.role[p] == 0) S.role[p] = 2;
    }
    if (sr == rank) S.gsend[rr].push_back(AmrPoint{sp, (int)so});
  };
  for (int l = 1; l < P.nlev && ok; ++l)
    for (const auto& t : P.ghost[l]) {
      const int rr = owner[t.dst];
      if (!(t.odd & AMR_COARSE)) {
        want(rr, t.src, t.sofs);
        continue;
      }
      const Geo& G = geo[t.src];
      const int ox = t.odd & 1, oy = (t.odd >> 1) & 1, oz = (t.odd >> 2) & 1;
      for (int dz = oz ? -2 : 0; dz <= (oz ? 3 : 0); ++dz)
        for (int dy = oy ? -2 : 0; dy <= (oy ? 3 : 0); ++dy)
          for (int dx = ox ? -2 : 0; dx <= (ox ? 3 : 0); ++dx) want(rr, t.src, t.sofs + dz * G.sz + dy * G.sy + dx);
    }
  if (!ok) {
    S.err = "shard: a ghost stencil reads a point of another rank's patch that no interior covers (the hierarchy "
            "must be nested: stencils of level l >= 2 inside interiors of level l-1)";
    return GRMHD_ERR_ARG;
  }
  // The rank's own ghost tasks; the coarse points and x-midpoint rows their
  // stencils read.
  S.gofs.assign(P.nlev + 1, 0);
  S.tpts.assign(P.nlev, {});
  S.xpts.assign(P.nlev, {});
  for (int l = 1; l < P.nlev; ++l) {
    S.gofs[l] = (long long)S.ghost.size();
    std::unordered_set<uint64_t> rows, pts;
    for (const auto& t : P.ghost[l]) {
      if (owner[t.dst] != rank) continue;
      S.ghost.push_back(t);
      if (S.role[t.src] == 0) S.role[t.src] = 2;
      if (!(t.odd & AMR_COARSE)) continue;
      const Geo& G = geo[t.src];
      const int ox = t.odd & 1, oy = (t.odd >> 1) & 1, oz = (t.odd >> 2) & 1;
      for (int dz = oz ? -2 : 0; dz <= (oz ? 3 : 0); ++dz)
        for (int dy = oy ? -2 : 0; dy <= (oy ? 3 : 0); ++dy) {
          const long long base = t.sofs + dz * G.sz + dy * G.sy;
          if (ox && rows.insert(pkey(t.src, base)).second) S.xpts[l].push_back(AmrPoint{t.src, (int)base});
          for (int dx = ox ? -2 : 0; dx <= (ox ? 3 : 0); ++dx)
            if (pts.insert(pkey(t.src, base + dx)).second) S.tpts[l].push_back(AmrPoint{t.src, (int)(base + dx)});
        }
    }
  }
  S.gofs[P.nlev] = (long long)S.ghost.size();
  // Restriction: the finest source of every restricted point, in the order
  // of the coarse points (by patch and offset).
  std::map<std::pair<int, int>, std::pair<int, int>> src_of;  // coarse point -> fine point
  for (int l = 1; l < P.nlev; ++l)
    for (const auto& t : P.restr[l]) src_of[{t.dst, t.dofs}] = {t.src, t.sofs};
  for (const auto& kv : src_of) {
    const int dp = kv.first.first;
    std::pair<int, int> f = kv.second;
    for (auto it = src_of.find(f); it != src_of.end(); it = src_of.find(f)) f = it->second;
    const int sr = owner[f.first], dr = owner[dp];
    if (dr == rank) {
      S.restr.push_back(AmrTask{dp, kv.first.second, f.first, f.second, 0});
      if (sr != rank) {
        S.rrecv[sr].push_back(AmrPoint{f.first, f.second});
        if (S.role[f.first] == 0) S.role[f.first] = 2;
      }
    }
    if (sr == rank && dr != rank) S.rsend[dr].push_back(AmrPoint{f.first, f.second});
  }
  return GRMHD_OK;
}

// Gather / scatter of the 32 fields of register reg at listed points: buffer
// layout [32][n] (field-major, so a warp's accesses to the buffer coalesce).
__global__ void k_shard_pack(const PatchDev* __restrict__ pd, const AmrPoint* __restrict__ pts, long long n, int reg,
                             double* __restrict__ buf) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrPoint P = pts[q];
  const PatchDev& S = pd[P.patch];
  const double* u = S.U[reg] + P.ofs;
  for (int f = 0; f < NF; ++f) buf[f * n + q] = u[f * S.G.sf];
}

__global__ void k_shard_unpack(const PatchDev* __restrict__ pd, const AmrPoint* __restrict__ pts, long long n, int reg,
                               const double* __restrict__ buf) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const AmrPoint P = pts[q];
  const PatchDev& D = pd[P.patch];
  double* u = D.U[reg] + P.ofs;
  for (int f = 0; f < NF; ++f) u[f * D.G.sf] = buf[f * n + q];
}

void launch_shard_pack(const PatchDev* pd, const AmrPoint* pts, long long n, int reg, double* buf, cudaStream_t st) {
  if (n <= 0) return;
  k_shard_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, pts, n, reg, buf);
}

void launch_shard_unpack(const PatchDev* pd, const AmrPoint* pts, long long n, int reg, const double* buf,
                         cudaStream_t st) {
  if (n <= 0) return;
  k_shard_unpack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pd, pts, n, reg, buf);
}

}  // namespace gk
