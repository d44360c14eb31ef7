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

struct C2PStats {
  unsigned long long points, iters, corrected, failed;
};

// Device error flags: bit 0 fatal con2prim point, bit 1 non-finite input.
struct DevFlags {
  int flags;
  int worst_status;
};

Eos make_eos(const grmhd_params& P, const grmhd_eos_table* T);
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
void launch_c2p(const PatchDev* pd_dev, const Work* w, int nblk, int reg, const grmhd_params& P, const Eos& E,
                DevFlags* flags, C2PStats* stats, cudaStream_t st, int bs = 128, bool seeded = false, double delta = 0.0);
void launch_iflux(const PatchDev* pd_dev, const Work* w, int nblk, int reg, int dir, cudaStream_t st, int bs = 128);
void launch_rhs(const PatchDev* pd_dev, const Work* w, int nblk, int reg, int mode, int stage, double dt,
                const grmhd_params& P, double* const* rhs_dev, cudaStream_t st, int bs = 128);
void launch_ghost_copy(const PatchDev* pd_dev, const Work* w, int nblk, int reg, cudaStream_t st);
void launch_rk(const PatchDev* pd_dev, const Work* w, int nblk, int stage, double dt, double* const* rhs_dev,
               cudaStream_t st, int rk = 0);
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

// Learned seeder over patch points (seeder.cu): seeds of every point of the
// work list (blocks of 128 points) of register reg into PatchDev::seed.
int launch_seeder_patches(const grmhd_seeder* s, const PatchDev* pd_dev, const Work* w, int nblk, int reg,
                          double rho_min, int* err, cudaStream_t st);

// FP64 FMA throughput probe: `blocks` blocks of 256 threads; returns the
// thread-level FMAs one launch executes.
long long launch_dfma_probe(int blocks, long long iters, double* sink, cudaStream_t st);

// Block sizes the autotuner chooses from.
constexpr int NBS = 3;
constexpr int BS_CAND[NBS] = {64, 128, 256};

}  // namespace gk
