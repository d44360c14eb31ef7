// Kernel declarations and the device-side patch descriptor shared by the
// kernel translation units and the host API.
#pragma once
#include <cuda_runtime.h>
#include <array>
#include <string>
#include <vector>
#include "c2p.cuh"

namespace gk {

// Registers 0..3: RK registers (U^n, two stage values, accumulator).
// Registers 4..8 (levels with a finer level, under sub-cycling): the dense
// output of the level's last step, U^n, D_1, D_2, D_3, J; otherwise null.
constexpr int REG_DENSE = 4;
constexpr int LES_NAUX = 32;  // point values whose gradients the LES closed forms use
constexpr int NDENSE = 5;
struct PatchDev {
  Geo G;
  double* U[REG_DENSE + NDENSE];
  double* prim;
  int8_t* status;
  double* Fp;   // pointwise fluxes [3][10][sf]
  double* lam;  // pointwise max |lambda_fast| [3][sf]
  double* Fh;   // interface fluxes [3][10][sf] at the interface between o and o + s_d
  float* seed;  // learned con2prim seeds [3][sf] (mu_+, mu, W) or null
  double* les;  // LES point values [LES_NAUX][sf] (LES terms on) or null
};

// Work item of a launch: patch index and block index within that patch's domain.
struct Work {
  int patch;
  int block;
};

enum Domain : int {
  DOM_ALL = 0,  // every point, ghosts included
  DOM_INT = 1,  // interior points
  DOM_IFX = 2,  // interfaces i+1/2, i = -1 .. n0-1, interior in y, z (likewise IFY, IFZ)
  DOM_IFY = 3,
  DOM_IFZ = 4,
  DOM_GX = 5,   // ghost-fill lines along x over interior (y, z)
  DOM_GY = 6,   // lines along y over (x incl. ghosts, interior z)
  DOM_GZ = 7,   // lines along z over (x, y incl. ghosts)
  NDOM = 8
};

// Number of work items of a domain.
inline __host__ __device__ long long dom_count(int dom, const Geo& G) {
  long long a = G.n0, b = G.n1, c = G.n2;
  switch (dom) {
    case DOM_ALL: return (a + 6) * (b + 6) * (c + 6);
    case DOM_INT: return a * b * c;
    case DOM_IFX: return (a + 1) * b * c;
    case DOM_IFY: return a * (b + 1) * c;
    case DOM_IFZ: return a * b * (c + 1);
    case DOM_GX: return b * c;
    case DOM_GY: return (a + 6) * c;
    default: return (a + 6) * (b + 6);
  }
}

// Linear work index -> point (i, j, k) of the domain (for ghost lines: the line's base point).
DI void dom_decode(int dom, const Geo& G, long long q, int& i, int& j, int& k) {
  long long ex, ey;
  int ox = 0, oy = 0, oz = 0;
  switch (dom) {
    case DOM_ALL: ex = G.n0 + 6; ey = G.n1 + 6; ox = oy = oz = -3; break;
    case DOM_INT: ex = G.n0; ey = G.n1; break;
    case DOM_IFX: ex = G.n0 + 1; ey = G.n1; ox = -1; break;
    case DOM_IFY: ex = G.n0; ey = G.n1 + 1; oy = -1; break;
    case DOM_IFZ: ex = G.n0; ey = G.n1; oz = -1; break;
    case DOM_GX: i = 0; j = (int)(q % G.n1); k = (int)(q / G.n1); return;
    case DOM_GY: i = (int)(q % (G.n0 + 6)) - 3; j = 0; k = (int)(q / (G.n0 + 6)); return;
    default: i = (int)(q % (G.n0 + 6)) - 3; j = (int)(q / (G.n0 + 6)) - 3; k = 0; return;
  }
  i = (int)(q % ex) + ox;
  q /= ex;
  j = (int)(q % ey) + oy;
  k = (int)(q / ey) + oz;
}

// ---- tile-shaped work items -------------------------------------------------
// A work item's `block` field holds a tile index in bits 0-23 and a tile shape
// in bits 24-30.  Shape 0: the domain's points in linear chunks of the block
// size (x fastest, wrapping across rows).  Shape s >= 1: boxes of
// 2^lx x 2^ly x 2^lz points, lx + ly + lz = log2(block size), tiles numbered x
// fastest over the domain; points of a box outside the domain are idle.
constexpr int NSHAPE = 5;
constexpr int TILE_BITS = 24;
constexpr int TILE_MASK = (1 << TILE_BITS) - 1;

// log2 extents of shape s (1..4) for a block of 2^b threads (b = 6, 7, 8):
// 1: a row segment 2^b x 1 x 1; 2: 32 x 2 x 2^(b-6); 3: 16 x 4 x 2^(b-6);
// 4: 8 x 8 x 2^(b-6).
inline __host__ __device__ void shape_log2(int b, int s, int& lx, int& ly, int& lz) {
  switch (s) {
    case 1: lx = b; ly = 0; lz = 0; break;
    case 2: lx = 5; ly = 1; lz = b - 6; break;
    case 3: lx = 4; ly = 2; lz = b - 6; break;
    default: lx = 3; ly = 3; lz = b - 6; break;
  }
}

// Extents and origin of a domain's point box (not for the ghost-line domains).
inline __host__ __device__ void dom_box(int dom, const Geo& G, int ex[3], int o[3]) {
  ex[0] = G.n0; ex[1] = G.n1; ex[2] = G.n2;
  o[0] = o[1] = o[2] = 0;
  if (dom == DOM_ALL) {
    for (int a = 0; a < 3; ++a) ex[a] += 6, o[a] = -3;
  } else if (dom >= DOM_IFX && dom <= DOM_IFZ) {
    ex[dom - DOM_IFX] += 1;
    o[dom - DOM_IFX] = -1;
  }
}

// Number of work items of a domain in shape s for blocks of 2^b threads.
inline long long dom_tiles(int dom, const Geo& G, int b, int s) {
  if (s == 0) return (dom_count(dom, G) + (1 << b) - 1) >> b;
  int ex[3], o[3], l[3];
  dom_box(dom, G, ex, o);
  shape_log2(b, s, l[0], l[1], l[2]);
  long long n = 1;
  for (int a = 0; a < 3; ++a) n *= (ex[a] + (1 << l[a]) - 1) >> l[a];
  return n;
}

// Point (i, j, k) of thread tid of a work item; false when the thread is idle.
DI bool work_point(int dom, const Geo& G, int blk, int tid, int bs_log2, int& i, int& j, int& k) {
  const int s = blk >> TILE_BITS, t = blk & TILE_MASK;
  if (s == 0) {
    long long q = ((long long)t << bs_log2) + tid;
    if (q >= dom_count(dom, G)) return false;
    dom_decode(dom, G, q, i, j, k);
    return true;
  }
  int ex[3], o[3], l0, l1, l2;
  dom_box(dom, G, ex, o);
  shape_log2(bs_log2, s, l0, l1, l2);
  const int ntx = (ex[0] + (1 << l0) - 1) >> l0, nty = (ex[1] + (1 << l1) - 1) >> l1;
  const int bx = t % ntx, r = t / ntx, by = r % nty, bz = r / nty;
  const int x = (bx << l0) + (tid & ((1 << l0) - 1));
  const int y = (by << l1) + ((tid >> l0) & ((1 << l1) - 1));
  const int z = (bz << l2) + (tid >> (l0 + l1));
  if (x >= ex[0] || y >= ex[1] || z >= ex[2]) return false;
  i = x + o[0];
  j = y + o[1];
  k = z + o[2];
  return true;
}

// Grid of a launch over nitems work items: one block per item, or (pers) a
// persistent pool of at most as many blocks as are resident on the GPU at
// once, each looping over the items with stride gridDim.x.
template <class K>
inline int grid_for(K kernel, int bs, int nitems, bool pers) {
  if (!pers) return nitems;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bs, 0);
  long long g = (long long)(nsm > 0 ? nsm : 1) * (per > 0 ? per : 1);
  return (int)(g < nitems ? g : nitems);
}

struct C2PStats {
  unsigned long long points, iters, corrected, failed;
};

// Device error flags: bit 0 fatal con2prim point, bit 1 non-finite input.
struct DevFlags {
  int flags;
  int worst_status;
};

Eos make_eos(const grmhd_params& P, const grmhd_eos_table* T);
// Evaluates the atmosphere's EOS state once on the device into E (synchronous).
int eos_set_atmo(const grmhd_params& P, Eos& E, cudaStream_t st);
// GRMHD_OK when the EOS kind and its parameters (table pointers and sizes,
// hybrid pieces) are usable, else GRMHD_ERR_ARG.
int eos_check(const grmhd_params& P, const grmhd_eos_table* T);

// Launchers (host functions in the .cu files; all enqueue on `st`).
void launch_init(const PatchDev* pd, int p, const Geo& G, const grmhd_params& P, const Eos& E, const double* id,
                 double* U, cudaStream_t st);
void launch_ghost(const PatchDev* pd_dev, const Work* w, int nblk, int reg, int axis, int bc, cudaStream_t st,
                  int f0 = 0, int f1 = NF);
// bs: threads per block of the launch (64, 128 or 256); the work list must
// have been built for the same block size.
// Work lists of the con2prim, interface-flux and right-hand-side launches may
// hold tile-shaped items (see work_point); pers: persistent launch (grid_for).
void launch_c2p(const PatchDev* pd_dev, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                DevFlags* flags, C2PStats* stats, cudaStream_t st, int bs = 128, bool seeded = false, double delta = 0.0,
                bool pers = false);
void launch_iflux(const PatchDev* pd_dev, const Work* w, int nblk, int reg, int dir, cudaStream_t st, int bs = 128,
                  bool pers = false);
// tiled: the work list may hold tile-shaped items (shape >= 1); otherwise
// all items are linear chunks (shape 0).
void launch_rhs(const PatchDev* pd_dev, const Work* w, int nblk, int reg, int mode, int stage, double dt,
                const grmhd_params& P, double* const* rhs_dev, cudaStream_t st, int bs = 128, bool tiled = false);
void launch_ghost_copy(const PatchDev* pd_dev, const Work* w, int nblk, int reg, cudaStream_t st);
void launch_rk(const PatchDev* pd_dev, const Work* w, int nblk, int stage, double dt, double* const* rhs_dev,
               cudaStream_t st, int rk = 0);
// Flat-state con2prim processing order grouped by the binary exponent of
// B^2 / D (a counting sort on the device into stream-ordered memory), or null
// below ORDER_MIN_STATES states (or when the memory is not available: the
// states are then solved in the given order).  Free with c2p_flat_order_free
// on the same stream after the solve's launch.
constexpr long long ORDER_MIN_STATES = 1 << 16;
int32_t* c2p_flat_order(long long n, const double* cons, cudaStream_t st);
void c2p_flat_order_free(int32_t* order, cudaStream_t st);
void launch_c2p_flat(const grmhd_params& P, const Eos& E, long long n, const double* cons, double* prim,
                     int8_t* status, int32_t* iters, cudaStream_t st);
void launch_prim2con_flat(const grmhd_params& P, const Eos& E, long long n, const double* prim, const double* B,
                          double* cons, cudaStream_t st);

// LES gradient SGS model (les.cu): true when any coefficient is nonzero;
// launch_les adds the SGS fluxes to PatchDev::Fp after con2prim of register
// reg over the DOM_ALL work list (block size 128).
bool les_on(const grmhd_params& P);
void launch_les(const PatchDev* pd_dev, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                cudaStream_t st);

// Block sizes of the launches (threads per block).
constexpr int BS_ALL = 128;
constexpr int BS_INT = 128;
constexpr int BS_IF = 128;
// Mesh-refinement hierarchy (amr.cu).  One task moves one point for all
// fields: a copy (odd & 7 == 0) or a prolongation from the coarse base point
// sofs of patch src (bit a of odd: midpoint along axis a); bit 3 of odd marks
// a source on the coarser level (else a same-level copy).
constexpr int AMR_COARSE = 8;
struct AmrTask {
  int dst, dofs, src, sofs, odd;
};
// One coarse point (patch, offset in its ghosted layout) that a level's
// prolongation stencils read.
struct AmrPoint {
  int patch, ofs;
};
struct AmrPlan {
  int level0 = -1, nlev = 0;
  std::vector<std::vector<AmrTask>> ghost;  // per level (0 unused): ghost tasks
  std::vector<std::vector<AmrTask>> restr;  // per level (0 unused): restriction into level - 1
  std::vector<long long> nsame;             // per level: leading same-level copies among its ghost tasks
  std::vector<std::vector<AmrPoint>> tpts;  // per level (0 unused): coarse points its stencils read, unique
  std::vector<std::vector<AmrPoint>> xpts;  // per level (0 unused): coarse rows whose x-midpoints it reads
  std::string err;
  // Empty when every prolongation stencil point lies in an interior of the
  // coarser level (or in the level-0 patch's ghosts), which sub-cycling needs.
  std::string sub_err;
};
int amr_plan(const grmhd_patch_desc* d, const std::vector<Geo>& geo, int np, AmrPlan& P);
// Ghost fill or restriction tasks on register reg; coarse-source tasks read
// register reg_coarse of their source (reg_coarse < 0: reg).  xpre: the
// x-midpoints of the coarse rows were computed by launch_amr_xmid into the
// source patches' Fp scratch (same values, computed once per row).
void launch_amr(const PatchDev* pd_dev, const AmrTask* t, long long n, int reg, cudaStream_t st, int reg_coarse = -1,
                bool xpre = false);
// x-midpoints of register reg at the listed coarse rows into PatchDev::Fp.
void launch_amr_xmid(const PatchDev* pd_dev, const AmrPoint* pts, long long n, int reg, cudaStream_t st);
// Sub-cycling: register reg_t of each listed coarse point receives the
// stage value sum_d coef[d] U[REG_DENSE + d] (nd terms).
void launch_amr_time(const PatchDev* pd_dev, const AmrPoint* pts, long long n, const double coef[NDENSE], int nd,
                     int reg_t, cudaStream_t st);
// Dense-output record after substep `stage` of a step (rk 0 RK4, 1 SSP-RK3)
// at the interior points of the work list (block size 128).
void launch_dense_rec(const PatchDev* pd_dev, const Work* w, int nblk, int stage, int rk, cudaStream_t st);

// ---- sharding across ranks (shard.cu) ----------------------------------------
// Owner rank of every patch: Morton order of the patch centres cut into
// nranks runs of about equal interior point count.
int shard_partition(const grmhd_patch_desc* d, int np, int nranks, int* owner);
// Sharding plan of one rank; see the file comment.
struct ShardPlan {
  std::vector<int> role;                          // per patch: 0 absent, 1 local, 2 mirror
  std::vector<std::vector<AmrPoint>> gsend, grecv;  // per peer: ghost-phase sources / their mirror points
  std::vector<std::vector<AmrPoint>> rsend, rrecv;  // per peer: restriction sources / their mirror points
  std::vector<AmrTask> ghost;                     // the rank's ghost tasks, levels 1.., in level order
  std::vector<long long> gofs;                    // per level: first ghost task (size nlev + 1)
  std::vector<AmrTask> restr;                     // composed restriction copies into local patches
  std::vector<std::vector<AmrPoint>> tpts, xpts;  // per level: coarse stencil points, x-midpoint rows
  int level0 = -1, nlev = 0;
  std::string err;
};
// The plan of rank `rank` (GRMHD_ERR_ARG with S.err when the hierarchy is not
// nested as the single exchange per substep needs).
int shard_plan(const grmhd_patch_desc* d, const std::vector<Geo>& geo, int np, const int* owner, int nranks, int rank,
               ShardPlan& S);
// Gather / scatter of register reg at n listed points into / from a [32][n] buffer.
void launch_shard_pack(const PatchDev* pd, const AmrPoint* pts, long long n, int reg, double* buf, cudaStream_t st);
void launch_shard_unpack(const PatchDev* pd, const AmrPoint* pts, long long n, int reg, const double* buf,
                         cudaStream_t st);

// Learned seeder over patch points (seeder.cu): seeds of every point of the
// work list (blocks of 128 points) of register reg into PatchDev::seed, in
// two passes: the atmosphere test lists the points to solve (list of
// capacity cap, its length in *count), then the network runs on the list.
int launch_seeder_patches(const grmhd_seeder* s, const PatchDev* pd_dev, const Work* w, int nblk, int reg,
                          double rho_min, int2* list, int* count, long long cap, int* err, cudaStream_t st);

// FP64 throughput probe: `blocks` blocks of 256 threads, each thread running
// `chains` (4, 8 or 16) independent FMA (or, add, addition) chains; returns
// the thread-level instructions one launch executes.
long long launch_dfma_probe(int blocks, int chains, long long iters, double* sink, cudaStream_t st, bool add);

// Block sizes the autotuner chooses from.
constexpr int NBS = 3;
constexpr int BS_CAND[NBS] = {64, 128, 256};

}  // namespace gk
