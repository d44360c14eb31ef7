// Host side of the C ABI declared in include/grmhd.h.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "kern.cuh"

using namespace gk;

struct grmhd_ctx {
  grmhd_params P;
  Eos E;
  cudaStream_t st;
  int np;
  std::vector<grmhd_patch_desc> desc;
  std::vector<PatchDev> pd_host;
  PatchDev* pd = nullptr;
  // work lists per group, block size and domain, concatenated; group 0 holds
  // every patch, group 1 + l the level-l patches of a hierarchy (bc 3)
  Work* work = nullptr;
  std::vector<std::array<std::array<int, NDOM + 1>, NBS>> wofs;
  int bs_c2p = 128, bs_if = 128, bs_rhs = 128;  // chosen block sizes
  // Per-patch slices of every work list, [group][block size][domain] -> for
  // each patch of the group in order, (first item, item count) relative to the
  // list's start; used when per_patch launches are on.
  std::vector<std::array<std::array<std::vector<std::pair<int, int>>, NDOM>, NBS>> pslice;
  bool per_patch = false;
  // Schedule of the con2prim (kind 0), interface-flux (1) and right-hand-side
  // (2) launches: a tile shape per patch and kind (0 = linear chunks, see
  // work_point) and a persistent flag per kind (kinds 0 and 1); their work
  // lists live in twork, laid out like work (empty for the ghost-line domains).
  std::vector<std::array<int, 3>> shape;
  bool pers[3] = {false, false, false};
  bool rhs_tiled = false;
  Work* twork = nullptr;
  std::vector<std::array<std::array<int, NDOM + 1>, NBS>> twofs;
  std::vector<std::array<std::array<std::vector<std::pair<int, int>>, NDOM>, NBS>> tpslice;
  std::vector<int> group_of;  // per group: -1 all patches, else the level
  // Sharded contexts (grmhd_init_shard): per patch 0 absent, 1 local
  // (evolved), 2 mirror (holds exchanged source points only); all 1 otherwise.
  std::vector<int> role;
  bool shard = false;
  double* scratch = nullptr;
  DevFlags* flags = nullptr;
  C2PStats* stats = nullptr;
  double** rhs_ptrs = nullptr;  // device array of npatch pointers
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // mesh-refinement hierarchy (bc 3): ghost tasks per level 1..L, then
  // restriction tasks per level L..1, in one device array
  AmrTask* amr = nullptr;
  // learned con2prim seeder (grmhd_set_seeder): seeds [3][sf] per patch
  const grmhd_seeder* seeder = nullptr;
  double seed_delta = 0.0;
  float* seed_buf = nullptr;
  // points to seed (the seeder's first pass): (patch, point offset) and the count
  int2* seed_list = nullptr;
  int* seed_count = nullptr;
  long long seed_cap = 0;
  int amr_level0 = -1, amr_nlev = 0;
  std::vector<long long> amr_gofs, amr_gcnt, amr_rofs, amr_rcnt, amr_gsame;
  // per level: coarse points its prolongation stencils read (sub-cycling)
  AmrPoint* amr_tp = nullptr;
  std::vector<long long> amr_tofs, amr_tcnt;
  // per level: coarse rows whose x-midpoints its prolongations read (in amr_tp)
  std::vector<long long> amr_xofs, amr_xcnt;
  std::string amr_sub_err;
  // sub-cycling in time (grmhd_set_subcycling): dense-output registers
  bool subcycle = false;
  double* dense_buf = nullptr;
  double* les_buf = nullptr;  // LES point values of every patch
  long long launches = 0;
  long long graph_kernels = 0;
  std::string err;
  // CUDA-event profiling per kernel kind (eager launches only).
  bool profiling = false;
  struct Rec {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

enum { K_GHOST = 0, K_C2P = 1, K_IFLUX = 2, K_RHS = 3, K_RK = 4, K_INIT = 5, K_SEED = 6, K_DENSE = 7, K_LES = 8, NKIND = 9 };

static cudaEvent_t ev_get(grmhd_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch with events on the context's stream when profiling is
// on and the stream is not being captured.
struct ProfScope {
  grmhd_ctx* c;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(grmhd_ctx* c_, int k) : c(c_), kind(k) {
    if (!c->profiling) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cs);
    if (cs != cudaStreamCaptureStatusNone) return;
    a = ev_get(c);
    cudaEventRecord(a, c->st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = ev_get(c);
    cudaEventRecord(b, c->st);
    c->recs.push_back(grmhd_ctx::Rec{a, b, kind});
  }
};

static const char* kNoCtx = "no context";

static int fail(grmhd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int cuda_ok(grmhd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GRMHD_OK;
  return fail(c, GRMHD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static int check_launch(grmhd_ctx* c, const char* what) {
  return cuda_ok(c, cudaGetLastError(), what);
}

static int bs_index(int bs) { return bs == 64 ? 0 : (bs == 256 ? 2 : 1); }

// Calls fn(work items, count) once for the whole list of a domain (batched
// launches) or once per patch of the group (per-patch launches).
template <class Fn>
static void for_slices(grmhd_ctx* c, int dom, int bs, int grp, Fn fn) {
  const int b = bs_index(bs);
  const Work* w = c->work + c->wofs[grp][b][dom];
  if (!c->per_patch) {
    fn(w, c->wofs[grp][b][dom + 1] - c->wofs[grp][b][dom]);
    return;
  }
  for (const auto& sl : c->pslice[grp][b][dom]) fn(w + sl.first, sl.second);
}

// The same over the tuned lists of the con2prim, interface-flux and
// right-hand-side launches.
template <class Fn>
static void for_tslices(grmhd_ctx* c, int dom, int bs, int grp, Fn fn) {
  const int b = bs_index(bs);
  const Work* w = c->twork + c->twofs[grp][b][dom];
  if (!c->per_patch) {
    fn(w, c->twofs[grp][b][dom + 1] - c->twofs[grp][b][dom]);
    return;
  }
  for (const auto& sl : c->tpslice[grp][b][dom]) fn(w + sl.first, sl.second);
}

static int kind_of(int dom) {
  return dom == DOM_ALL ? 0 : (dom >= DOM_IFX && dom <= DOM_IFZ ? 1 : (dom == DOM_INT ? 2 : -1));
}
static int log2_bs(int bs) { return bs == 64 ? 6 : (bs == 256 ? 8 : 7); }

// (Re)builds the tuned work lists from the schedule and uploads them; a
// captured graph refers to the old lists, so it is discarded.
static int build_tuned(grmhd_ctx* c) {
  std::vector<Work> wl;
  const int ngrp = (int)c->group_of.size();
  c->twofs.assign(ngrp, {});
  c->tpslice.assign(ngrp, {});
  bool tiled = false;
  for (int i = 0; i < c->np; ++i) tiled = tiled || c->shape[i][2] != 0;
  for (int g = 0; g < ngrp; ++g)
    for (int b = 0; b < NBS; ++b) {
      const int lb = log2_bs(BS_CAND[b]);
      for (int dom = 0; dom < NDOM; ++dom) {
        c->twofs[g][b][dom] = (int)wl.size();
        const int kind = kind_of(dom);
        if (kind < 0) continue;
        for (int i = 0; i < c->np; ++i) {
          if (c->role[i] != 1 || (c->group_of[g] >= 0 && c->desc[i].level != c->group_of[g])) continue;
          const int sh = c->shape[i][kind];
          const long long nt = dom_tiles(dom, c->pd_host[i].G, lb, sh);
          c->tpslice[g][b][dom].push_back({(int)wl.size() - c->twofs[g][b][dom], (int)nt});
          for (long long t = 0; t < nt; ++t) wl.push_back(Work{i, (int)t | (sh << TILE_BITS)});
        }
      }
      c->twofs[g][b][NDOM] = (int)wl.size();
    }
  int rc;
  if ((rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync"))) return rc;
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  if (c->graph) {
    cudaGraphDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaFree(c->twork);
  c->twork = nullptr;
  if ((rc = cuda_ok(c, cudaMalloc(&c->twork, (wl.size() + 1) * sizeof(Work)), "cudaMalloc tuned work")))
    return GRMHD_ERR_NOMEM;
  if (!wl.empty() &&
      (rc = cuda_ok(c, cudaMemcpy(c->twork, wl.data(), wl.size() * sizeof(Work), cudaMemcpyHostToDevice),
                    "copy tuned work")))
    return rc;
  c->rhs_tiled = tiled;
  return GRMHD_OK;
}

extern "C" {

int grmhd_abi_version(void) { return 2; }

const char* grmhd_last_error(grmhd_ctx* c) { return c ? c->err.c_str() : kNoCtx; }

long long grmhd_launch_count(grmhd_ctx* c) { return c ? c->launches : -1; }

void grmhd_destroy(grmhd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  cudaFree(c->pd);
  cudaFree(c->work);
  cudaFree(c->twork);
  cudaFree(c->dense_buf);
  cudaFree(c->les_buf);
  cudaFree(c->amr_tp);
  cudaFree(c->scratch);
  cudaFree(c->flags);
  cudaFree(c->stats);
  cudaFree(c->rhs_ptrs);
  cudaFree(c->amr);
  cudaFree(c->seed_buf);
  cudaFree(c->seed_list);
  delete c;
}

static Geo geo_of(const grmhd_patch_desc& d) {
  Geo G;
  G.n0 = d.n[0];
  G.n1 = d.n[1];
  G.n2 = d.n[2];
  G.px = d.px;
  G.sy = d.px;
  G.sz = G.sy * (G.n1 + 6);
  G.sf = G.sz * (G.n2 + 6);
  G.dx = d.dx;
  G.i12 = 1.0 / (12.0 * G.dx);
  G.i12s = 1.0 / (12.0 * G.dx * G.dx);
  G.i144 = 1.0 / (144.0 * G.dx * G.dx);
  G.ihdx = 0.5 / G.dx;
  return G;
}

// Context creation; S: the plan of one rank of a sharded hierarchy, or null
// (every patch local).
static int init_impl(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d,
                     const grmhd_eos_table* eos, void* stream, const ShardPlan* S) {
  if (!out) return GRMHD_ERR_ARG;
  *out = nullptr;
  if (!p || !d || npatch <= 0) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  if (p->bc < 0 || p->bc > 3) return GRMHD_ERR_ARG;
  if (p->max_iter < 1 || !(p->h0 > 0.0)) return GRMHD_ERR_ARG;
  if (p->rk != 0 && p->rk != 1) return GRMHD_ERR_ARG;
  std::vector<int> role(npatch, 1);
  if (S) role = S->role;
  for (int i = 0; i < npatch; ++i) {
    const grmhd_patch_desc& q = d[i];
    if (q.n[0] < 4 || q.n[1] < 4 || q.n[2] < 4 || q.px < q.n[0] + 6 || !(q.dx > 0.0)) return GRMHD_ERR_ARG;
    if (role[i] == 0) continue;  // absent from this rank: its arrays are not touched
    for (int r = 0; r < 4; ++r)
      if (!q.U[r] || ((uintptr_t)q.U[r] & 7)) return GRMHD_ERR_ARG;
    if (!q.prim || ((uintptr_t)q.prim & 7) || !q.status) return GRMHD_ERR_ARG;
  }
  grmhd_ctx* c = new grmhd_ctx();
  c->P = *p;
  c->E = make_eos(*p, eos);
  c->st = (cudaStream_t)stream;
  c->np = npatch;
  c->desc.assign(d, d + npatch);
  c->pd_host.resize(npatch);
  c->role = role;
  c->shard = S != nullptr;
  // scratch: Fp (30) + lam (3) + Fh (30) doubles per ghosted point of every
  // patch this rank holds (mirrors too: the x-midpoint pre-pass of a ghost
  // fill writes into the coarse patch's Fp)
  size_t total = 0;
  std::vector<size_t> ofs(npatch);
  for (int i = 0; i < npatch; ++i) {
    c->pd_host[i] = PatchDev();
    c->pd_host[i].G = geo_of(d[i]);
    ofs[i] = total;
    if (role[i]) total += (size_t)63 * c->pd_host[i].G.sf;
  }
  int rc;
  if ((rc = cuda_ok(c, cudaMalloc(&c->scratch, total * sizeof(double)), "cudaMalloc scratch")) != GRMHD_OK) {
    grmhd_destroy(c);
    return GRMHD_ERR_NOMEM;
  }
  if ((rc = eos_set_atmo(c->P, c->E, c->st)) != GRMHD_OK) {
    grmhd_destroy(c);
    return rc;
  }
  for (int i = 0; i < npatch; ++i) {
    PatchDev& q = c->pd_host[i];
    for (int r = 0; r < REG_DENSE + NDENSE; ++r) q.U[r] = nullptr;
    q.seed = nullptr;
    q.les = nullptr;
    q.prim = nullptr;
    q.status = nullptr;
    q.Fp = q.lam = q.Fh = nullptr;
    if (!role[i]) continue;
    for (int r = 0; r < 4; ++r) q.U[r] = d[i].U[r];
    q.prim = d[i].prim;
    q.status = d[i].status;
    q.Fp = c->scratch + ofs[i];
    q.lam = q.Fp + 30 * q.G.sf;
    q.Fh = q.lam + 3 * q.G.sf;
  }
  if (les_on(*p)) {
    size_t ltot = 0;
    for (int i = 0; i < npatch; ++i)
      if (role[i] == 1) ltot += (size_t)LES_NAUX * c->pd_host[i].G.sf;
    if ((rc = cuda_ok(c, cudaMalloc(&c->les_buf, ltot * sizeof(double)), "cudaMalloc LES values")) != GRMHD_OK) {
      grmhd_destroy(c);
      return GRMHD_ERR_NOMEM;
    }
    size_t lo = 0;
    for (int i = 0; i < npatch; ++i) {
      if (role[i] != 1) continue;
      c->pd_host[i].les = c->les_buf + lo;
      lo += (size_t)LES_NAUX * c->pd_host[i].G.sf;
    }
  }
  // work lists: for each group, block size and domain, the blocks of patch
  // 0, then patch 1, ... (group 0: every patch; group 1 + l: level l)
  int ngrp = 1;
  if (p->bc == 3) {
    int maxl = 0;
    bool ok = true;
    for (int i = 0; i < npatch; ++i) {
      ok = ok && d[i].level >= 0 && d[i].level <= 20;
      if (d[i].level > maxl) maxl = d[i].level;
    }
    if (ok) ngrp = 2 + maxl;  // otherwise the hierarchy plan below rejects the layout
  }
  c->wofs.assign(ngrp, {});
  c->pslice.assign(ngrp, {});
  c->group_of.assign(ngrp, -1);
  for (int g = 1; g < ngrp; ++g) c->group_of[g] = g - 1;
  c->shape.assign(npatch, {0, 0, 0});
  std::vector<Work> wl;
  for (int g = 0; g < ngrp; ++g)
    for (int b = 0; b < NBS; ++b) {
      int bs = BS_CAND[b];
      for (int dom = 0; dom < NDOM; ++dom) {
        c->wofs[g][b][dom] = (int)wl.size();
        for (int i = 0; i < npatch; ++i) {
          if (role[i] != 1 || (g > 0 && d[i].level != g - 1)) continue;
          long long n = dom_count(dom, c->pd_host[i].G);
          long long nb = (n + bs - 1) / bs;
          c->pslice[g][b][dom].push_back({(int)wl.size() - c->wofs[g][b][dom], (int)nb});
          for (long long k = 0; k < nb; ++k) wl.push_back(Work{i, (int)k});
        }
      }
      c->wofs[g][b][NDOM] = (int)wl.size();
    }
  if ((rc = cuda_ok(c, cudaMalloc(&c->work, wl.size() * sizeof(Work)), "cudaMalloc work")) ||
      (rc = cuda_ok(c, cudaMalloc(&c->pd, npatch * sizeof(PatchDev)), "cudaMalloc pd")) ||
      (rc = cuda_ok(c, cudaMalloc(&c->flags, sizeof(DevFlags)), "cudaMalloc flags")) ||
      (rc = cuda_ok(c, cudaMalloc(&c->stats, sizeof(C2PStats)), "cudaMalloc stats")) ||
      (rc = cuda_ok(c, cudaMalloc(&c->rhs_ptrs, npatch * sizeof(double*)), "cudaMalloc rhs ptrs"))) {
    grmhd_destroy(c);
    return rc == GRMHD_ERR_CUDA ? GRMHD_ERR_NOMEM : rc;
  }
  if (p->bc == 3) {
    std::vector<Geo> geo(npatch);
    for (int i = 0; i < npatch; ++i) geo[i] = c->pd_host[i].G;
    AmrPlan plan;
    if (amr_plan(d, geo, npatch, plan) != GRMHD_OK) {
      std::fprintf(stderr, "grmhd_init_patches: %s\n", plan.err.c_str());
      grmhd_destroy(c);
      return GRMHD_ERR_ARG;
    }
    if (S) {
      // This rank's ghost tasks, stencil points and composed restriction
      // copies (all under level 1: they are independent of one another).
      for (int l = 1; l < plan.nlev; ++l) {
        plan.ghost[l].assign(S->ghost.begin() + S->gofs[l], S->ghost.begin() + S->gofs[l + 1]);
        plan.restr[l].clear();
        plan.tpts[l] = S->tpts[l];
        plan.xpts[l] = S->xpts[l];
        plan.nsame[l] = 0;
        for (const auto& t : plan.ghost[l])
          if (!(t.odd & AMR_COARSE)) ++plan.nsame[l];
      }
      if (plan.nlev > 1) plan.restr[1] = S->restr;
      plan.sub_err = "sharded hierarchy (sub-cycling is not available across ranks)";
    }
    c->amr_level0 = plan.level0;
    c->amr_nlev = plan.nlev;
    c->amr_gsame = plan.nsame;
    c->amr_sub_err = plan.sub_err;
    std::vector<AmrTask> all;
    c->amr_gofs.assign(plan.nlev, 0);
    c->amr_gcnt.assign(plan.nlev, 0);
    c->amr_rofs.assign(plan.nlev, 0);
    c->amr_rcnt.assign(plan.nlev, 0);
    for (int l = 1; l < plan.nlev; ++l) {
      c->amr_gofs[l] = (long long)all.size();
      c->amr_gcnt[l] = (long long)plan.ghost[l].size();
      all.insert(all.end(), plan.ghost[l].begin(), plan.ghost[l].end());
    }
    for (int l = plan.nlev - 1; l >= 1; --l) {
      c->amr_rofs[l] = (long long)all.size();
      c->amr_rcnt[l] = (long long)plan.restr[l].size();
      all.insert(all.end(), plan.restr[l].begin(), plan.restr[l].end());
    }
    std::vector<AmrPoint> tp;
    c->amr_tofs.assign(plan.nlev, 0);
    c->amr_tcnt.assign(plan.nlev, 0);
    for (int l = 1; l < plan.nlev; ++l) {
      c->amr_tofs[l] = (long long)tp.size();
      c->amr_tcnt[l] = (long long)plan.tpts[l].size();
      tp.insert(tp.end(), plan.tpts[l].begin(), plan.tpts[l].end());
    }
    c->amr_xofs.assign(plan.nlev, 0);
    c->amr_xcnt.assign(plan.nlev, 0);
    for (int l = 1; l < plan.nlev; ++l) {
      c->amr_xofs[l] = (long long)tp.size();
      c->amr_xcnt[l] = (long long)plan.xpts[l].size();
      tp.insert(tp.end(), plan.xpts[l].begin(), plan.xpts[l].end());
    }
    if (!tp.empty()) {
      if ((rc = cuda_ok(c, cudaMalloc(&c->amr_tp, tp.size() * sizeof(AmrPoint)), "cudaMalloc amr points"))) {
        grmhd_destroy(c);
        return GRMHD_ERR_NOMEM;
      }
      if ((rc = cuda_ok(c, cudaMemcpy(c->amr_tp, tp.data(), tp.size() * sizeof(AmrPoint), cudaMemcpyHostToDevice),
                        "copy amr points"))) {
        grmhd_destroy(c);
        return rc;
      }
    }
    if (!all.empty()) {
      if ((rc = cuda_ok(c, cudaMalloc(&c->amr, all.size() * sizeof(AmrTask)), "cudaMalloc amr tasks"))) {
        grmhd_destroy(c);
        return GRMHD_ERR_NOMEM;
      }
      if ((rc = cuda_ok(c, cudaMemcpy(c->amr, all.data(), all.size() * sizeof(AmrTask), cudaMemcpyHostToDevice),
                        "copy amr tasks"))) {
        grmhd_destroy(c);
        return rc;
      }
    }
  }
  if ((rc = cuda_ok(c, cudaMemcpyAsync(c->work, wl.data(), wl.size() * sizeof(Work), cudaMemcpyHostToDevice, c->st),
                    "copy work")) ||
      (rc = cuda_ok(c, cudaMemcpyAsync(c->pd, c->pd_host.data(), npatch * sizeof(PatchDev), cudaMemcpyHostToDevice,
                                       c->st), "copy pd")) ||
      (rc = cuda_ok(c, cudaMemsetAsync(c->flags, 0, sizeof(DevFlags), c->st), "clear flags")) ||
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")) || (rc = build_tuned(c))) {
    grmhd_destroy(c);
    return rc;
  }
  *out = c;
  return GRMHD_OK;
}

int grmhd_init_patches(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d,
                       const grmhd_eos_table* eos, void* stream) {
  return init_impl(out, p, npatch, d, eos, stream, nullptr);
}

int grmhd_shard_partition(int npatch, const grmhd_patch_desc* d, int nranks, int* owner) {
  return shard_partition(d, npatch, nranks, owner);
}

int grmhd_shard_plan(int npatch, const grmhd_patch_desc* d, const int* owner, int nranks, int rank, int* role,
                     long long* counts, int* lists, long long cap) {
  if (!d || !owner || npatch < 1 || nranks < 1 || rank < 0 || rank >= nranks || !counts) return GRMHD_ERR_ARG;
  std::vector<Geo> geo(npatch);
  for (int i = 0; i < npatch; ++i) geo[i] = geo_of(d[i]);
  ShardPlan S;
  if (shard_plan(d, geo, npatch, owner, nranks, rank, S) != GRMHD_OK) {
    std::fprintf(stderr, "grmhd_shard_plan: %s\n", S.err.c_str());
    return GRMHD_ERR_ARG;
  }
  if (role)
    for (int i = 0; i < npatch; ++i) role[i] = S.role[i];
  long long need = 0;
  for (int q = 0; q < nranks; ++q) {
    counts[4 * q + 0] = (long long)S.gsend[q].size();
    counts[4 * q + 1] = (long long)S.grecv[q].size();
    counts[4 * q + 2] = (long long)S.rsend[q].size();
    counts[4 * q + 3] = (long long)S.rrecv[q].size();
    need += counts[4 * q] + counts[4 * q + 1] + counts[4 * q + 2] + counts[4 * q + 3];
  }
  if (!lists) return GRMHD_OK;
  if (cap < 2 * need) return GRMHD_ERR_SIZE;
  long long o = 0;
  for (int q = 0; q < nranks; ++q)
    for (const auto* v : {&S.gsend[q], &S.grecv[q], &S.rsend[q], &S.rrecv[q]})
      for (const auto& pt : *v) {
        lists[o++] = pt.patch;
        lists[o++] = pt.ofs;
      }
  return GRMHD_OK;
}

int grmhd_init_shard(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d, const int* owner,
                     int nranks, int rank, const grmhd_eos_table* eos, void* stream) {
  if (!out) return GRMHD_ERR_ARG;
  *out = nullptr;
  if (!p || !d || !owner || npatch < 1 || p->bc != 3) return GRMHD_ERR_ARG;
  std::vector<Geo> geo(npatch);
  for (int i = 0; i < npatch; ++i) geo[i] = geo_of(d[i]);
  ShardPlan S;
  if (shard_plan(d, geo, npatch, owner, nranks, rank, S) != GRMHD_OK) {
    std::fprintf(stderr, "grmhd_init_shard: %s\n", S.err.c_str());
    return GRMHD_ERR_ARG;
  }
  return init_impl(out, p, npatch, d, eos, stream, &S);
}

static int nblk(grmhd_ctx* c, int dom, int bs = 128, int grp = 0) {
  int b = bs_index(bs);
  return c->wofs[grp][b][dom + 1] - c->wofs[grp][b][dom];
}
static const Work* wl(grmhd_ctx* c, int dom, int bs = 128, int grp = 0) {
  return c->work + c->wofs[grp][bs_index(bs)][dom];
}

// The contiguous slice of a ghost-line work list (block size 128) that belongs
// to one patch: work items are grouped by patch in increasing order.
static void patch_range(grmhd_ctx* c, int dom, int patch, int* first, int* cnt) {
  long long before = 0;
  for (int i = 0; i < patch; ++i)
    if (c->role[i] == 1) before += (dom_count(dom, c->pd_host[i].G) + BS_ALL - 1) / BS_ALL;
  *first = (int)before;
  *cnt = (int)((dom_count(dom, c->pd_host[patch].G) + BS_ALL - 1) / BS_ALL);
}

int grmhd_init_state(grmhd_ctx* c, int patch, const double* id) {
  if (!c) return GRMHD_ERR_ARG;
  if (patch < 0 || patch >= c->np || !id || c->role[patch] != 1)
    return fail(c, GRMHD_ERR_ARG, "init_state: bad patch (or not evolved on this rank) or id");
  const PatchDev& q = c->pd_host[patch];
  {
    ProfScope ps(c, K_INIT);
    launch_init(c->pd, patch, q.G, c->P, c->E, id, q.U[0], c->st);
  }
  c->launches += 2;
  int rc = check_launch(c, "init");
  if (rc) return rc;
  for (int ax = 0; ax < 3; ++ax) {
    // ghost fill of this patch only: its own slice of the work list
    int dom = DOM_GX + ax;
    const Work* w = wl(c, dom);
    int n = nblk(c, dom);
    // find the contiguous range of this patch
    int first = -1, cnt = 0;
    patch_range(c, dom, patch, &first, &cnt);
    if (first + cnt > n) return fail(c, GRMHD_ERR_ARG, "init_state: work list");
    if (c->P.bc == 2)  // frozen ghosts keep the initial data; only Gammahat is extrapolated
      launch_ghost(c->pd, w + first, cnt, 0, ax, 1, c->st, GH, GH + 3);
    else
      launch_ghost(c->pd, w + first, cnt, 0, ax, c->P.bc, c->st);
    c->launches += 1;
  }
  return check_launch(c, "init ghost");
}

// Ghost fill of hierarchy levels 1.. in order (bc 3).
static int fill_levels(grmhd_ctx* c, int reg) {
  for (int l = 1; l < c->amr_nlev; ++l) {
    // The coarser level's x-midpoints once per row, then the fill (uses the
    // coarser level's pointwise-flux scratch).
    ProfScope ps(c, K_GHOST);
    launch_amr_xmid(c->pd, c->amr_tp + c->amr_xofs[l], c->amr_xcnt[l], reg, c->st);
    launch_amr(c->pd, c->amr + c->amr_gofs[l], c->amr_gcnt[l], reg, c->st, -1, true);
    c->launches += 2;
  }
  return check_launch(c, "ghost hierarchy");
}

int grmhd_ghost_fill(grmhd_ctx* c, int reg) {
  if (!c) return GRMHD_ERR_ARG;
  if (reg < 0 || reg > 3) return fail(c, GRMHD_ERR_ARG, "ghost_fill: reg");
  if (c->P.bc == 3) {
    // Level 0: outer boundary extrapolation of its single patch (on the rank
    // that evolves it); then each finer level from its own interiors and the
    // next coarser level.
    for (int ax = 0; ax < 3 && c->role[c->amr_level0] == 1; ++ax) {
      int first, cnt;
      patch_range(c, DOM_GX + ax, c->amr_level0, &first, &cnt);
      ProfScope ps(c, K_GHOST);
      launch_ghost(c->pd, wl(c, DOM_GX + ax) + first, cnt, reg, ax, 1, c->st);
      c->launches += 1;
    }
    return fill_levels(c, reg);
  }
  if (c->P.bc == 2) {
    if (reg != 0) {
      ProfScope ps(c, K_GHOST);
      launch_ghost_copy(c->pd, wl(c, DOM_ALL), nblk(c, DOM_ALL), reg, c->st);
      c->launches += 1;
    }
    return check_launch(c, "ghost copy");
  }
  for (int ax = 0; ax < 3; ++ax) {
    ProfScope ps(c, K_GHOST);
    launch_ghost(c->pd, wl(c, DOM_GX + ax), nblk(c, DOM_GX + ax), reg, ax, c->P.bc, c->st);
    c->launches += 1;
  }
  return check_launch(c, "ghost");
}

static int c2p_and_fluxes(grmhd_ctx* c, int reg, bool stats, int grp = 0) {
  if (c->seeder) {
    ProfScope ps(c, K_SEED);
    int rc = GRMHD_OK;
    for_slices(c, DOM_ALL, 128, grp, [&](const Work* w, int n) {
      int r = launch_seeder_patches(c->seeder, c->pd, w, n, reg, c->P.rho_min, c->seed_list, c->seed_count,
                                    c->seed_cap, &c->flags->flags, c->st);
      if (r && !rc) rc = r;
      c->launches += 2;
    });
    if (rc) return fail(c, rc, "seeder launch");
  }
  {
    ProfScope ps(c, K_C2P);
    for_tslices(c, DOM_ALL, c->bs_c2p, grp, [&](const Work* w, int n) {
      launch_c2p(c->pd, w, n, reg, c->P, c->E, c->flags, stats ? c->stats : nullptr, c->st, c->bs_c2p,
                 c->seeder != nullptr, c->seed_delta, c->pers[0]);
      c->launches += 1;
    });
  }
  if (c->les_buf) {
    ProfScope ps(c, K_LES);
    for_slices(c, DOM_ALL, 128, grp, [&](const Work* w, int n) {
      launch_les(c->pd, w, n, reg, c->P, c->E, c->st);
      c->launches += 2;
    });
  }
  return check_launch(c, "con2prim");
}

int grmhd_set_seeder(grmhd_ctx* c, const grmhd_seeder* s, double delta) {
  if (!c) return GRMHD_ERR_ARG;
  if (!s) {
    c->seeder = nullptr;
    return GRMHD_OK;
  }
  if (!(delta > 0.0 && delta < 1.0)) return fail(c, GRMHD_ERR_ARG, "set_seeder: delta in (0, 1)");
  int rc;
  if (!c->seed_buf) {
    size_t total = 0;
    for (int i = 0; i < c->np; ++i)
      if (c->role[i] == 1) total += 3 * (size_t)c->pd_host[i].G.sf;
    // The list holds every local point (point offsets fit an int: a patch's
    // field has fewer than 2^31 points) and, after it, the count.
    const long long cap = (long long)(total / 3);
    for (int i = 0; i < c->np; ++i)
      if (c->role[i] == 1 && c->pd_host[i].G.sf >= (1LL << 31))
        return fail(c, GRMHD_ERR_ARG, "set_seeder: a patch has 2^31 or more points");
    if ((rc = cuda_ok(c, cudaMalloc(&c->seed_list, (size_t)cap * sizeof(int2) + 16), "cudaMalloc seed list")))
      return GRMHD_ERR_NOMEM;
    if ((rc = cuda_ok(c, cudaMalloc(&c->seed_buf, total * sizeof(float)), "cudaMalloc seeds"))) {
      cudaFree(c->seed_list);
      c->seed_list = nullptr;
      return GRMHD_ERR_NOMEM;
    }
    c->seed_cap = cap;
    c->seed_count = reinterpret_cast<int*>(c->seed_list + cap);
    size_t o = 0;
    for (int i = 0; i < c->np; ++i) {
      if (c->role[i] != 1) continue;
      c->pd_host[i].seed = c->seed_buf + o;
      o += 3 * (size_t)c->pd_host[i].G.sf;
    }
    if ((rc = cuda_ok(c, cudaMemcpyAsync(c->pd, c->pd_host.data(), c->np * sizeof(PatchDev), cudaMemcpyHostToDevice,
                                         c->st), "copy pd")) ||
        (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
      return rc;
  }
  c->seeder = s;
  c->seed_delta = delta;
  return GRMHD_OK;
}

static int iflux(grmhd_ctx* c, int reg, int grp = 0) {
  for (int d = 0; d < 3; ++d) {
    ProfScope ps(c, K_IFLUX);
    for_tslices(c, DOM_IFX + d, c->bs_if, grp, [&](const Work* w, int n) {
      launch_iflux(c->pd, w, n, reg, d, c->st, c->bs_if, c->pers[1]);
      c->launches += 1;
    });
  }
  return check_launch(c, "iflux");
}

int grmhd_con2prim(grmhd_ctx* c, int reg, grmhd_c2p_stats* s) {
  if (!c) return GRMHD_ERR_ARG;
  if (reg < 0 || reg > 3) return fail(c, GRMHD_ERR_ARG, "con2prim: reg");
  int rc;
  if (s && (rc = cuda_ok(c, cudaMemsetAsync(c->stats, 0, sizeof(C2PStats), c->st), "clear stats"))) return rc;
  if ((rc = c2p_and_fluxes(c, reg, s != nullptr))) return rc;
  if (s) {
    C2PStats h;
    if ((rc = cuda_ok(c, cudaMemcpyAsync(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->st), "stats copy")) ||
        (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
      return rc;
    s->points = (long long)h.points;
    s->iterations = (long long)h.iters;
    s->corrected = (long long)h.corrected;
    s->failed = (long long)h.failed;
  }
  return GRMHD_OK;
}

int grmhd_rhs_eval(grmhd_ctx* c, int reg, double* const* rhs) {
  if (!c) return GRMHD_ERR_ARG;
  if (reg < 0 || reg > 3 || !rhs) return fail(c, GRMHD_ERR_ARG, "rhs_eval: args");
  for (int i = 0; i < c->np; ++i)
    if (c->role[i] == 1 && !rhs[i]) return fail(c, GRMHD_ERR_ARG, "rhs_eval: null rhs");
  int rc;
  if ((rc = cuda_ok(c, cudaMemcpyAsync(c->rhs_ptrs, rhs, c->np * sizeof(double*), cudaMemcpyHostToDevice, c->st),
                    "rhs ptrs")) ||
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
    return rc;
  if ((rc = iflux(c, reg))) return rc;
  {
    ProfScope ps(c, K_RHS);
    for_tslices(c, DOM_INT, c->bs_rhs, 0, [&](const Work* w, int n) {
      launch_rhs(c->pd, w, n, reg, 0, 0, 0.0, c->P, c->rhs_ptrs, c->st, c->bs_rhs, c->rhs_tiled);
      c->launches += 1;
    });
  }
  return check_launch(c, "rhs");
}

int grmhd_rk_update(grmhd_ctx* c, int stage, double dt, double* const* rhs) {
  if (!c) return GRMHD_ERR_ARG;
  if (stage < 0 || stage > (c->P.rk == 1 ? 2 : 3) || !rhs) return fail(c, GRMHD_ERR_ARG, "rk_update: args");
  int rc;
  if ((rc = cuda_ok(c, cudaMemcpyAsync(c->rhs_ptrs, rhs, c->np * sizeof(double*), cudaMemcpyHostToDevice, c->st),
                    "rhs ptrs")) ||
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
    return rc;
  {
    ProfScope ps(c, K_RK);
    launch_rk(c->pd, wl(c, DOM_INT), nblk(c, DOM_INT), stage, dt, c->rhs_ptrs, c->st, c->P.rk);
  }
  c->launches += 1;
  return check_launch(c, "rk");
}

static const int kStageIn[4] = {0, 1, 2, 1};    // RK4
static const int kStageInRk3[3] = {0, 1, 2};    // SSP-RK3

int grmhd_rhs_substep(grmhd_ctx* c, int stage, double dt) {
  if (!c) return GRMHD_ERR_ARG;
  const bool rk3 = c->P.rk == 1;
  if (stage < 0 || stage > (rk3 ? 2 : 3)) return fail(c, GRMHD_ERR_ARG, "rhs_substep: stage");
  int reg = rk3 ? kStageInRk3[stage] : kStageIn[stage];
  int rc;
  // A sharded context fills levels 1.. only: level 0's ghosts come from
  // grmhd_shard_ghost0 on its own rank, before the exchange.
  if ((rc = c->shard ? fill_levels(c, reg) : grmhd_ghost_fill(c, reg))) return rc;
  if ((rc = c2p_and_fluxes(c, reg, false))) return rc;
  if ((rc = iflux(c, reg))) return rc;
  {
    ProfScope ps(c, K_RHS);
    for_tslices(c, DOM_INT, c->bs_rhs, 0, [&](const Work* w, int n) {
      launch_rhs(c->pd, w, n, reg, 1, stage, dt, c->P, nullptr, c->st, c->bs_rhs, c->rhs_tiled);
      c->launches += 1;
    });
  }
  return check_launch(c, "rhs fused");
}

int grmhd_restrict(grmhd_ctx* c, int reg) {
  if (!c) return GRMHD_ERR_ARG;
  if (reg < 0 || reg > 3) return fail(c, GRMHD_ERR_ARG, "restrict: reg");
  if (c->P.bc != 3) return GRMHD_OK;
  for (int l = c->amr_nlev - 1; l >= 1; --l) {
    ProfScope ps(c, K_GHOST);
    launch_amr(c->pd, c->amr + c->amr_rofs[l], c->amr_rcnt[l], reg, c->st);
    c->launches += 1;
  }
  return check_launch(c, "restrict");
}

// Coefficients of (U^n, D_1, D_2, D_3, J) in the BOR stage value (Sec. IV C,
// sub-cycling; Sec. III A, dense output) of stage s of fine step msub (0, 1)
// of a coarse step, refinement ratio 2.  With the Taylor data of the
// dense-output cubic at t0 = t^n + msub dt/2 and h = dt/2,
//   P_0 = sum_m th^m/m! D_m, P_1 = (D_1 + th D_2 + th^2/2 D_3)/2,
//   P_2 = (D_2 + th D_3)/4, P_3 = D_3/8, P_J = J/8  (th = msub/2),
// the fine stages are Y = sum_i w_i P_i + w_J P_J with, for RK4,
//   w = (1), (1, 1/2), (1, 1/2, 1/4, 1/16; w_J -1/16), (1, 1, 1/2, 1/8; w_J 1/8),
// and for SSP-RK3 (1), (1, 1), (1, 1/2, 1/4).
static void bor_coef(int rk, int msub, int s, double c[NDENSE]) {
  const double th = 0.5 * msub;
  const double P[4][4] = {{1.0, th, 0.5 * th * th, th * th * th / 6.0},
                          {0.0, 0.5, 0.5 * th, 0.25 * th * th},
                          {0.0, 0.0, 0.25, 0.25 * th},
                          {0.0, 0.0, 0.0, 0.125}};
  double w[4] = {1.0, 0.0, 0.0, 0.0}, wj = 0.0;
  if (rk == 1) {
    if (s == 1) w[1] = 1.0;
    if (s == 2) w[1] = 0.5, w[2] = 0.25;
  } else if (s == 1) {
    w[1] = 0.5;
  } else if (s == 2) {
    w[1] = 0.5, w[2] = 0.25, w[3] = 1.0 / 16.0, wj = -1.0 / 16.0;
  } else if (s == 3) {
    w[1] = 1.0, w[2] = 0.5, w[3] = 0.125, wj = 0.125;
  }
  for (int m = 0; m < 4; ++m) {
    double v = 0.0;
    for (int i = 0; i < 4; ++i) v += w[i] * P[i][m];
    c[m] = v;
  }
  c[4] = wj * 0.125;
}

// Outer-boundary extrapolation of register reg of the level-0 patch.
static void ghost_level0(grmhd_ctx* c, int reg) {
  for (int ax = 0; ax < 3; ++ax) {
    int first, cnt;
    patch_range(c, DOM_GX + ax, c->amr_level0, &first, &cnt);
    launch_ghost(c->pd, wl(c, DOM_GX + ax) + first, cnt, reg, ax, 1, c->st);
    c->launches += 1;
  }
}

// One step of dt of level l (fine step msub of its parent's step), then two
// steps of level l + 1 and its restriction into level l (Sec. IV C, BOR).
static int sub_advance(grmhd_ctx* c, int l, int msub, double dt) {
  const bool rk3 = c->P.rk == 1;
  const int ns = rk3 ? 3 : 4, nd = rk3 ? 3 : NDENSE, grp = 1 + l;
  const bool parent = l + 1 < c->amr_nlev;
  int rc;
  for (int s = 0; s < ns; ++s) {
    const int reg = rk3 ? kStageInRk3[s] : kStageIn[s];
    {
      ProfScope ps(c, K_GHOST);
      if (l == 0) {
        ghost_level0(c, reg);
      } else {
        // The parent's stage value at the coarse points the stencils read,
        // into the parent's accumulator register (free between its steps),
        // then the ghost fill from it.
        double cf[NDENSE];
        bor_coef(c->P.rk, msub, s, cf);
        launch_amr_time(c->pd, c->amr_tp + c->amr_tofs[l], c->amr_tcnt[l], cf, nd, 3, c->st);
        launch_amr_xmid(c->pd, c->amr_tp + c->amr_xofs[l], c->amr_xcnt[l], 3, c->st);
        launch_amr(c->pd, c->amr + c->amr_gofs[l], c->amr_gcnt[l], reg, c->st, 3, true);
        c->launches += 3;
      }
    }
    if ((rc = check_launch(c, "sub-cycled ghost fill"))) return rc;
    if ((rc = c2p_and_fluxes(c, reg, false, grp))) return rc;
    if ((rc = iflux(c, reg, grp))) return rc;
    {
      ProfScope ps(c, K_RHS);
      for_tslices(c, DOM_INT, c->bs_rhs, grp, [&](const Work* w, int n) {
        launch_rhs(c->pd, w, n, reg, 1, s, dt, c->P, nullptr, c->st, c->bs_rhs, c->rhs_tiled);
        c->launches += 1;
      });
    }
    if (parent) {
      ProfScope ps(c, K_DENSE);
      launch_dense_rec(c->pd, wl(c, DOM_INT, 128, grp), nblk(c, DOM_INT, 128, grp), s, c->P.rk, c->st);
      c->launches += 1;
    }
    if ((rc = check_launch(c, "sub-cycled substep"))) return rc;
  }
  if (!parent) return GRMHD_OK;
  // Ghosts of the dense registers: extrapolated on level 0, same-level
  // copies on finer levels (the prolongation stencils need no others).
  for (int e = 0; e < nd; ++e) {
    ProfScope ps(c, K_DENSE);
    if (l == 0) {
      ghost_level0(c, REG_DENSE + e);
    } else {
      launch_amr(c->pd, c->amr + c->amr_gofs[l], c->amr_gsame[l], REG_DENSE + e, c->st);
      c->launches += 1;
    }
  }
  for (int m = 0; m < 2; ++m)
    if ((rc = sub_advance(c, l + 1, m, 0.5 * dt))) return rc;
  {
    ProfScope ps(c, K_GHOST);
    launch_amr(c->pd, c->amr + c->amr_rofs[l + 1], c->amr_rcnt[l + 1], 0, c->st);
    c->launches += 1;
  }
  return check_launch(c, "restrict");
}

int grmhd_set_subcycling(grmhd_ctx* c, int on) {
  if (!c) return GRMHD_ERR_ARG;
  if (!on) {
    c->subcycle = false;
    return GRMHD_OK;
  }
  if (c->P.bc != 3) return fail(c, GRMHD_ERR_ARG, "set_subcycling: needs a mesh-refinement hierarchy (bc 3)");
  if (!c->amr_sub_err.empty()) return fail(c, GRMHD_ERR_ARG, "set_subcycling: " + c->amr_sub_err);
  if (!c->dense_buf && c->amr_nlev > 1) {
    const int nd = c->P.rk == 1 ? 3 : NDENSE;
    size_t total = 0;
    for (int i = 0; i < c->np; ++i)
      if (c->desc[i].level + 1 < c->amr_nlev) total += (size_t)nd * NF * c->pd_host[i].G.sf;
    int rc;
    if ((rc = cuda_ok(c, cudaMalloc(&c->dense_buf, total * sizeof(double)), "cudaMalloc dense registers")))
      return GRMHD_ERR_NOMEM;
    size_t o = 0;
    for (int i = 0; i < c->np; ++i) {
      if (c->desc[i].level + 1 >= c->amr_nlev) continue;
      for (int e = 0; e < nd; ++e) {
        c->pd_host[i].U[REG_DENSE + e] = c->dense_buf + o;
        o += (size_t)NF * c->pd_host[i].G.sf;
      }
    }
    if ((rc = cuda_ok(c, cudaMemcpyAsync(c->pd, c->pd_host.data(), c->np * sizeof(PatchDev), cudaMemcpyHostToDevice,
                                         c->st), "copy pd")) ||
        (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
      return rc;
  }
  c->subcycle = true;
  return GRMHD_OK;
}

int grmhd_shard_ghost0(grmhd_ctx* c, int reg) {
  if (!c || !c->shard || reg < 0 || reg > 3) return GRMHD_ERR_ARG;
  for (int ax = 0; ax < 3 && c->role[c->amr_level0] == 1; ++ax) {
    int first, cnt;
    patch_range(c, DOM_GX + ax, c->amr_level0, &first, &cnt);
    ProfScope ps(c, K_GHOST);
    launch_ghost(c->pd, wl(c, DOM_GX + ax) + first, cnt, reg, ax, 1, c->st);
    c->launches += 1;
  }
  return check_launch(c, "level-0 ghosts");
}

int grmhd_shard_pack(grmhd_ctx* c, int reg, const int* pts, long long n, double* buf) {
  if (!c || reg < 0 || reg > 3 || n < 0 || (n > 0 && (!pts || !buf))) return GRMHD_ERR_ARG;
  launch_shard_pack(c->pd, reinterpret_cast<const AmrPoint*>(pts), n, reg, buf, c->st);
  c->launches += n > 0;
  return check_launch(c, "shard pack");
}

int grmhd_shard_unpack(grmhd_ctx* c, int reg, const int* pts, long long n, const double* buf) {
  if (!c || reg < 0 || reg > 3 || n < 0 || (n > 0 && (!pts || !buf))) return GRMHD_ERR_ARG;
  launch_shard_unpack(c->pd, reinterpret_cast<const AmrPoint*>(pts), n, reg, buf, c->st);
  c->launches += n > 0;
  return check_launch(c, "shard unpack");
}

int grmhd_step(grmhd_ctx* c, double dt) {
  if (!c) return GRMHD_ERR_ARG;
  if (c->shard) return fail(c, GRMHD_ERR_ARG, "step: a sharded context steps through the exchange protocol");
  if (c->subcycle) return sub_advance(c, 0, 0, dt);
  const int nsub = c->P.rk == 1 ? 3 : 4;
  for (int s = 0; s < nsub; ++s) {
    int rc = grmhd_rhs_substep(c, s, dt);
    if (rc) return rc;
  }
  return grmhd_restrict(c, 0);
}

int grmhd_capture_graph(grmhd_ctx* c, int nsteps, double dt) {
  if (!c) return GRMHD_ERR_ARG;
  if (nsteps < 1) return fail(c, GRMHD_ERR_ARG, "capture: nsteps");
  if (c->st == nullptr) return fail(c, GRMHD_ERR_ARG, "capture: needs a non-default stream");
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  if (c->graph) {
    cudaGraphDestroy(c->graph);
    c->graph = nullptr;
  }
  int rc;
  if ((rc = cuda_ok(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return rc;
  long long before = c->launches;
  int inner = GRMHD_OK;
  for (int s = 0; s < nsteps && inner == GRMHD_OK; ++s) inner = grmhd_step(c, dt);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  c->graph_kernels = c->launches - before;
  c->launches = before;  // captured launches run at replay
  if (inner) {
    if (g) cudaGraphDestroy(g);
    return inner;
  }
  if ((rc = cuda_ok(c, e, "end capture"))) return rc;
  c->graph = g;
  if ((rc = cuda_ok(c, cudaGraphInstantiate(&c->gexec, g, 0), "instantiate"))) return rc;
  return GRMHD_OK;
}

int grmhd_graph_launch(grmhd_ctx* c) {
  if (!c) return GRMHD_ERR_ARG;
  if (!c->gexec) return fail(c, GRMHD_ERR_ARG, "graph_launch: no graph");
  c->launches += c->graph_kernels;
  return cuda_ok(c, cudaGraphLaunch(c->gexec, c->st), "graph launch");
}

int grmhd_set_per_patch(grmhd_ctx* c, int on) {
  if (!c) return GRMHD_ERR_ARG;
  c->per_patch = on != 0;
  return GRMHD_OK;
}

int grmhd_set_block_sizes(grmhd_ctx* c, int bs_c2p, int bs_iflux, int bs_rhs) {
  if (!c) return GRMHD_ERR_ARG;
  auto ok = [](int b) { return b == 64 || b == 128 || b == 256; };
  if (!ok(bs_c2p) || !ok(bs_iflux) || !ok(bs_rhs)) return fail(c, GRMHD_ERR_ARG, "block sizes: 64, 128 or 256");
  c->bs_c2p = bs_c2p;
  c->bs_if = bs_iflux;
  c->bs_rhs = bs_rhs;
  return GRMHD_OK;
}

int grmhd_set_schedule(grmhd_ctx* c, const int* shapes, const int* pers) {
  if (!c) return GRMHD_ERR_ARG;
  if (shapes)
    for (int i = 0; i < 3 * c->np; ++i)
      if (shapes[i] < 0 || shapes[i] >= NSHAPE) return fail(c, GRMHD_ERR_ARG, "set_schedule: shape 0..4");
  if (pers && pers[2]) return fail(c, GRMHD_ERR_ARG, "set_schedule: the right-hand side has no persistent form");
  if (shapes)
    for (int i = 0; i < c->np; ++i)
      for (int k = 0; k < 3; ++k) c->shape[i][k] = shapes[3 * i + k];
  if (pers)
    for (int k = 0; k < 2; ++k) c->pers[k] = pers[k] != 0;
  return build_tuned(c);
}

int grmhd_get_schedule(grmhd_ctx* c, int* shapes, int* pers) {
  if (!c) return GRMHD_ERR_ARG;
  if (shapes)
    for (int i = 0; i < c->np; ++i)
      for (int k = 0; k < 3; ++k) shapes[3 * i + k] = c->shape[i][k];
  if (pers)
    for (int k = 0; k < 3; ++k) pers[k] = c->pers[k] ? 1 : 0;
  return GRMHD_OK;
}

// Size class of a patch for the tile-shape search: its longest edge, in the
// bins <= 16, 24, 32, 48, 64, 96, 128, larger.
static int size_class(const grmhd_patch_desc& d) {
  const int e = std::max(d.n[0], std::max(d.n[1], d.n[2]));
  const int lim[7] = {16, 24, 32, 48, 64, 96, 128};
  for (int k = 0; k < 7; ++k)
    if (e <= lim[k]) return k;
  return 7;
}

// Times `reps` launches of kernel kind `kind` (after one untimed launch) over
// the given patches with tile shape sh, on stage-0 data (register 0 in, the
// fused stage-0 outputs U[1], U[3] out: repeated launches change nothing).
static double time_kind(grmhd_ctx* c, int kind, const std::vector<int>& patches, int sh, int reps, Work* tmp,
                        size_t cap, cudaEvent_t e0, cudaEvent_t e1) {
  const int bs = kind == 0 ? c->bs_c2p : (kind == 1 ? c->bs_if : c->bs_rhs);
  const int lb = log2_bs(bs);
  double total = 0.0;
  const int ndir = kind == 1 ? 3 : 1;
  for (int d = 0; d < ndir; ++d) {
    const int dom = kind == 0 ? DOM_ALL : (kind == 1 ? DOM_IFX + d : DOM_INT);
    std::vector<Work> wl;
    for (int i : patches) {
      const long long nt = dom_tiles(dom, c->pd_host[i].G, lb, sh);
      for (long long t = 0; t < nt; ++t) wl.push_back(Work{i, (int)t | (sh << TILE_BITS)});
    }
    if (wl.empty()) continue;
    if (wl.size() > cap) return -1.0;  // cannot happen: the buffer holds the largest trial list
    if (cudaMemcpy(tmp, wl.data(), wl.size() * sizeof(Work), cudaMemcpyHostToDevice) != cudaSuccess) return -1.0;
    const int n = (int)wl.size();
    for (int r = 0; r <= reps; ++r) {
      if (r == 1) cudaEventRecord(e0, c->st);
      if (kind == 0)
        launch_c2p(c->pd, tmp, n, 0, c->P, c->E, c->flags, nullptr, c->st, bs, c->seeder != nullptr, c->seed_delta);
      else if (kind == 1)
        launch_iflux(c->pd, tmp, n, 0, d, c->st, bs);
      else
        launch_rhs(c->pd, tmp, n, 0, 1, 0, 0.0, c->P, nullptr, c->st, bs, sh != 0);
    }
    cudaEventRecord(e1, c->st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
    total += ms;
  }
  return total;
}

int grmhd_autotune(grmhd_ctx* c, double dt, int reps, int* chosen) {
  if (!c) return GRMHD_ERR_ARG;
  if (reps < 1) return fail(c, GRMHD_ERR_ARG, "autotune: reps");
  bool was = c->profiling;
  // Phase 1: block size per kernel kind, from whole substeps with the
  // current schedule.
  double best[3] = {1e300, 1e300, 1e300};
  int pick[3] = {128, 128, 128};
  int rc = GRMHD_OK;
  for (int b = 0; b < NBS && rc == GRMHD_OK; ++b) {
    c->bs_c2p = c->bs_if = c->bs_rhs = BS_CAND[b];
    if ((rc = grmhd_rhs_substep(c, 0, dt))) break;  // warm-up of this variant
    if ((rc = grmhd_profile(c, 1))) break;
    for (int r = 0; r < reps && rc == GRMHD_OK; ++r) rc = grmhd_rhs_substep(c, 0, dt);
    if (rc) break;
    double ms[NKIND];
    long long cnt[NKIND];
    if ((rc = grmhd_profile_read(c, ms, cnt, NKIND))) break;
    const int kinds[3] = {K_C2P, K_IFLUX, K_RHS};
    for (int k = 0; k < 3; ++k)
      if (ms[kinds[k]] < best[k]) {
        best[k] = ms[kinds[k]];
        pick[k] = BS_CAND[b];
      }
  }
  grmhd_profile(c, was ? 1 : 0);
  c->bs_c2p = pick[0];
  c->bs_if = pick[1];
  c->bs_rhs = pick[2];
  if (chosen) {
    chosen[0] = pick[0];
    chosen[1] = pick[1];
    chosen[2] = pick[2];
  }
  if (rc) return rc;
  // Phase 2: tile shape per patch-size class and kernel kind, each kind timed
  // alone on the class's patches (con2prim, then interface fluxes, then the
  // right-hand side, so every kernel reads current inputs).
  if ((rc = grmhd_rhs_substep(c, 0, dt)) || (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync"))) return rc;
  std::vector<std::vector<int>> cls(8);
  for (int i = 0; i < c->np; ++i)
    if (c->role[i] == 1) cls[size_class(c->desc[i])].push_back(i);
  // The largest trial list: one domain, one class, one shape at a time.
  size_t maxw = 1;
  for (int kind = 0; kind < 3; ++kind) {
    const int lb = log2_bs(kind == 0 ? c->bs_c2p : (kind == 1 ? c->bs_if : c->bs_rhs));
    for (const auto& pl : cls)
      for (int dom = 0; dom < NDOM; ++dom) {
        if (kind_of(dom) != kind) continue;
        for (int sh = 0; sh < NSHAPE; ++sh) {
          size_t m = 0;
          for (int i : pl) m += (size_t)dom_tiles(dom, c->pd_host[i].G, lb, sh);
          maxw = std::max(maxw, m);
        }
      }
  }
  Work* tmp = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((rc = cuda_ok(c, cudaMalloc(&tmp, maxw * sizeof(Work)), "cudaMalloc autotune list"))) return GRMHD_ERR_NOMEM;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int kind = 0; kind < 3 && rc == GRMHD_OK; ++kind)
    for (const auto& pl : cls) {
      if (pl.empty()) continue;
      double tbest = 1e300;
      int sbest = 0;
      for (int sh = 0; sh < NSHAPE; ++sh) {
        double t = time_kind(c, kind, pl, sh, reps, tmp, maxw, e0, e1);
        if (t < 0.0) {
          rc = fail(c, GRMHD_ERR_CUDA, "autotune: tile timing");
          break;
        }
        if (t < tbest) {
          tbest = t;
          sbest = sh;
        }
      }
      for (int i : pl) c->shape[i][kind] = sbest;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tmp);
  if (rc || (rc = build_tuned(c))) return rc;
  // Phase 3: persistent pool or one block per item, for con2prim and the
  // interface fluxes, from whole substeps with the chosen shapes.
  for (int kind = 0; kind < 2 && rc == GRMHD_OK; ++kind) {
    double t[2] = {0.0, 0.0};
    for (int p = 0; p < 2 && rc == GRMHD_OK; ++p) {
      c->pers[kind] = p != 0;
      if ((rc = grmhd_rhs_substep(c, 0, dt)) || (rc = grmhd_profile(c, 1))) break;
      for (int r = 0; r < reps && rc == GRMHD_OK; ++r) rc = grmhd_rhs_substep(c, 0, dt);
      double ms[NKIND];
      long long cnt[NKIND];
      if (rc || (rc = grmhd_profile_read(c, ms, cnt, NKIND))) break;
      t[p] = ms[kind == 0 ? K_C2P : K_IFLUX];
    }
    c->pers[kind] = t[1] < t[0];
  }
  grmhd_profile(c, was ? 1 : 0);
  return rc;
}

int grmhd_profile(grmhd_ctx* c, int on) {
  if (!c) return GRMHD_ERR_ARG;
  int rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync");
  for (auto& r : c->recs) {
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  c->profiling = on != 0;
  return rc;
}

int grmhd_profile_read(grmhd_ctx* c, double* ms, long long* count, int nkinds) {
  if (!c || !ms || !count || nkinds < 1) return GRMHD_ERR_ARG;
  int rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync");
  if (rc) return rc;
  for (int k = 0; k < nkinds; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  for (auto& r : c->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return fail(c, GRMHD_ERR_CUDA, "event elapsed");
    if (r.kind < nkinds) {
      ms[r.kind] += t;
      count[r.kind] += 1;
    }
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  return GRMHD_OK;
}

int grmhd_sync_status(grmhd_ctx* c) {
  if (!c) return GRMHD_ERR_ARG;
  DevFlags h;
  int rc;
  if ((rc = cuda_ok(c, cudaMemcpyAsync(&h, c->flags, sizeof(h), cudaMemcpyDeviceToHost, c->st), "flags copy")) ||
      (rc = cuda_ok(c, cudaMemsetAsync(c->flags, 0, sizeof(DevFlags), c->st), "flags clear")) ||
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
    return rc;
  if (h.flags & 4) return fail(c, GRMHD_ERR_TIMEOUT, "seeder tensor-core wait timed out");
  if (h.flags & 2) return fail(c, GRMHD_ERR_NONFINITE, "non-finite state reached con2prim");
  if (h.flags & 1) return fail(c, GRMHD_ERR_C2P_FATAL, "fatal con2prim point");
  return GRMHD_OK;
}

int grmhd_dfma_probe(int blocks_per_sm, int chains, long long iters, double* sink, long long* fmas, void* stream) {
  // chains < 0: addition chains of |chains| (the FP64 add rate)
  const bool add = chains < 0;
  if (add) chains = -chains;
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || (chains != 4 && chains != 8 && chains != 16) || iters < 1 || !sink ||
      !fmas)
    return GRMHD_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return GRMHD_ERR_CUDA;
  *fmas = launch_dfma_probe(nsm * blocks_per_sm, chains, iters, sink, (cudaStream_t)stream, add);
  return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

int grmhd_prim2con_flat(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* prim,
                        const double* B, double* cons, void* stream) {
  if (!p || n < 0 || (n > 0 && (!prim || !B || !cons))) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  launch_prim2con_flat(*p, make_eos(*p, eos), n, prim, B, cons, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

int grmhd_c2p_flat(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* cons, double* prim,
                   int8_t* status, int32_t* iters, void* stream) {
  if (!p || n < 0 || (n > 0 && (!cons || !prim || !status))) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  if (p->max_iter < 1 || !(p->h0 > 0.0)) return GRMHD_ERR_ARG;
  launch_c2p_flat(*p, make_eos(*p, eos), n, cons, prim, status, iters, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}

}  // extern "C"
