// Host side of the C ABI declared in include/grmhd.h.
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
  cudaFree(c->dense_buf);
  cudaFree(c->les_buf);
  cudaFree(c->amr_tp);
  cudaFree(c->scratch);
  cudaFree(c->flags);
  cudaFree(c->stats);
  cudaFree(c->rhs_ptrs);
  cudaFree(c->amr);
  cudaFree(c->seed_buf);
  delete c;
}

int grmhd_init_patches(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d,
                       const grmhd_eos_table* eos, void* stream) {
  if (!out) return GRMHD_ERR_ARG;
  *out = nullptr;
  if (!p || !d || npatch <= 0) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  if (p->bc < 0 || p->bc > 3) return GRMHD_ERR_ARG;
  if (p->max_iter < 1 || !(p->h0 > 0.0)) return GRMHD_ERR_ARG;
  if (p->rk != 0 && p->rk != 1) return GRMHD_ERR_ARG;
  for (int i = 0; i < npatch; ++i) {
    const grmhd_patch_desc& q = d[i];
    if (q.n[0] < 4 || q.n[1] < 4 || q.n[2] < 4 || q.px < q.n[0] + 6 || !(q.dx > 0.0)) return GRMHD_ERR_ARG;
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
  // scratch: Fp (30) + lam (3) + Fh (30) doubles per ghosted point
  size_t total = 0;
  std::vector<size_t> ofs(npatch);
  for (int i = 0; i < npatch; ++i) {
    Geo G;
    G.n0 = d[i].n[0];
    G.n1 = d[i].n[1];
    G.n2 = d[i].n[2];
    G.px = d[i].px;
    G.sy = d[i].px;
    G.sz = G.sy * (G.n1 + 6);
    G.sf = G.sz * (G.n2 + 6);
    G.dx = d[i].dx;
    G.i12 = 1.0 / (12.0 * G.dx);
    G.i12s = 1.0 / (12.0 * G.dx * G.dx);
    G.i144 = 1.0 / (144.0 * G.dx * G.dx);
    G.idx = 1.0 / G.dx;
    c->pd_host[i].G = G;
    ofs[i] = total;
    total += (size_t)63 * G.sf;
  }
  int rc;
  if ((rc = cuda_ok(c, cudaMalloc(&c->scratch, total * sizeof(double)), "cudaMalloc scratch")) != GRMHD_OK) {
    grmhd_destroy(c);
    return GRMHD_ERR_NOMEM;
  }
  for (int i = 0; i < npatch; ++i) {
    PatchDev& q = c->pd_host[i];
    for (int r = 0; r < 4; ++r) q.U[r] = d[i].U[r];
    q.prim = d[i].prim;
    q.status = d[i].status;
    q.Fp = c->scratch + ofs[i];
    q.lam = q.Fp + 30 * q.G.sf;
    q.Fh = q.lam + 3 * q.G.sf;
    q.seed = nullptr;
    q.les = nullptr;
  }
  if (les_on(*p)) {
    size_t ltot = 0;
    for (int i = 0; i < npatch; ++i) ltot += (size_t)LES_NAUX * c->pd_host[i].G.sf;
    if ((rc = cuda_ok(c, cudaMalloc(&c->les_buf, ltot * sizeof(double)), "cudaMalloc LES values")) != GRMHD_OK) {
      grmhd_destroy(c);
      return GRMHD_ERR_NOMEM;
    }
    size_t lo = 0;
    for (int i = 0; i < npatch; ++i) {
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
  std::vector<Work> wl;
  for (int g = 0; g < ngrp; ++g)
    for (int b = 0; b < NBS; ++b) {
      int bs = BS_CAND[b];
      for (int dom = 0; dom < NDOM; ++dom) {
        c->wofs[g][b][dom] = (int)wl.size();
        for (int i = 0; i < npatch; ++i) {
          if (g > 0 && d[i].level != g - 1) continue;
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
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync"))) {
    grmhd_destroy(c);
    return rc;
  }
  *out = c;
  return GRMHD_OK;
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
  for (int i = 0; i < patch; ++i) before += (dom_count(dom, c->pd_host[i].G) + BS_ALL - 1) / BS_ALL;
  *first = (int)before;
  *cnt = (int)((dom_count(dom, c->pd_host[patch].G) + BS_ALL - 1) / BS_ALL);
}

int grmhd_init_state(grmhd_ctx* c, int patch, const double* id) {
  if (!c) return GRMHD_ERR_ARG;
  if (patch < 0 || patch >= c->np || !id) return fail(c, GRMHD_ERR_ARG, "init_state: bad patch or id");
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

int grmhd_ghost_fill(grmhd_ctx* c, int reg) {
  if (!c) return GRMHD_ERR_ARG;
  if (reg < 0 || reg > 3) return fail(c, GRMHD_ERR_ARG, "ghost_fill: reg");
  if (c->P.bc == 3) {
    // Level 0: outer boundary extrapolation of its single patch; then each
    // finer level from its own interiors and the next coarser level.
    for (int ax = 0; ax < 3; ++ax) {
      int first, cnt;
      patch_range(c, DOM_GX + ax, c->amr_level0, &first, &cnt);
      ProfScope ps(c, K_GHOST);
      launch_ghost(c->pd, wl(c, DOM_GX + ax) + first, cnt, reg, ax, 1, c->st);
      c->launches += 1;
    }
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
      int r = launch_seeder_patches(c->seeder, c->pd, w, n, reg, c->P.rho_min, &c->flags->flags, c->st);
      if (r && !rc) rc = r;
      c->launches += 1;
    });
    if (rc) return fail(c, rc, "seeder launch");
  }
  {
    ProfScope ps(c, K_C2P);
    for_slices(c, DOM_ALL, c->bs_c2p, grp, [&](const Work* w, int n) {
      launch_c2p(c->pd, w, n, reg, c->P, c->E, c->flags, stats ? c->stats : nullptr, c->st, c->bs_c2p,
                 c->seeder != nullptr, c->seed_delta);
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
    for (int i = 0; i < c->np; ++i) total += 3 * (size_t)c->pd_host[i].G.sf;
    if ((rc = cuda_ok(c, cudaMalloc(&c->seed_buf, total * sizeof(float)), "cudaMalloc seeds"))) return GRMHD_ERR_NOMEM;
    size_t o = 0;
    for (int i = 0; i < c->np; ++i) {
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
    for_slices(c, DOM_IFX + d, c->bs_if, grp, [&](const Work* w, int n) {
      launch_iflux(c->pd, w, n, reg, d, c->st, c->bs_if);
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
    if (!rhs[i]) return fail(c, GRMHD_ERR_ARG, "rhs_eval: null rhs");
  int rc;
  if ((rc = cuda_ok(c, cudaMemcpyAsync(c->rhs_ptrs, rhs, c->np * sizeof(double*), cudaMemcpyHostToDevice, c->st),
                    "rhs ptrs")) ||
      (rc = cuda_ok(c, cudaStreamSynchronize(c->st), "sync")))
    return rc;
  if ((rc = iflux(c, reg))) return rc;
  {
    ProfScope ps(c, K_RHS);
    for_slices(c, DOM_INT, c->bs_rhs, 0, [&](const Work* w, int n) {
      launch_rhs(c->pd, w, n, reg, 0, 0, 0.0, c->P, c->rhs_ptrs, c->st, c->bs_rhs);
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
  if ((rc = grmhd_ghost_fill(c, reg))) return rc;
  if ((rc = c2p_and_fluxes(c, reg, false))) return rc;
  if ((rc = iflux(c, reg))) return rc;
  {
    ProfScope ps(c, K_RHS);
    for_slices(c, DOM_INT, c->bs_rhs, 0, [&](const Work* w, int n) {
      launch_rhs(c->pd, w, n, reg, 1, stage, dt, c->P, nullptr, c->st, c->bs_rhs);
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
      for_slices(c, DOM_INT, c->bs_rhs, grp, [&](const Work* w, int n) {
        launch_rhs(c->pd, w, n, reg, 1, s, dt, c->P, nullptr, c->st, c->bs_rhs);
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

int grmhd_step(grmhd_ctx* c, double dt) {
  if (!c) return GRMHD_ERR_ARG;
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

int grmhd_autotune(grmhd_ctx* c, double dt, int reps, int* chosen) {
  if (!c) return GRMHD_ERR_ARG;
  if (reps < 1) return fail(c, GRMHD_ERR_ARG, "autotune: reps");
  bool was = c->profiling;
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

int grmhd_dfma_probe(int blocks_per_sm, long long iters, double* sink, long long* fmas, void* stream) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !sink || !fmas) return GRMHD_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return GRMHD_ERR_CUDA;
  *fmas = launch_dfma_probe(nsm * blocks_per_sm, iters, sink, (cudaStream_t)stream);
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
