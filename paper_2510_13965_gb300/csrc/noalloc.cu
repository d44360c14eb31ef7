// Allocation-free right-hand-side evaluation of one patch.
//
// Some callers cannot let a library call cudaMalloc: applications that have
// handed all device memory to their own pool allocator (a raw cudaMalloc would
// fail or fragment the pool), code paths that must not pay the device-wide
// synchronisation cudaMalloc / cudaFree can imply, and host frameworks that
// only permit allocation through their own allocator.  grmhd_rhs_eval_static
// serves them: it runs the same kernels as grmhd_con2prim + grmhd_rhs_eval on
// a one-patch context, but every piece of device memory it needs besides the
// caller's arrays lives in the file-scope array below.
//
// The array is part of the library image, so every GPU that loads the library
// reserves it (kStaticBytes, about 27.7 MB) until the process exits.  All calls
// on one device share it, and it keeps whatever the last call left there:
// calls that may overlap on the GPU (for example on two streams of the same
// device) race on it and must be serialised by the caller.  Calls on the same
// stream are ordered and safe.
//
// Nothing is copied from host memory: the descriptor, the output pointer and
// the work list are written into the array by a set-up kernel that receives
// them as launch arguments, and the same kernel clears the device flags.
#include <cstdint>
#include <mutex>
#include "kern.cuh"

namespace gk {
namespace {

// Largest patch accepted: 54,872 ghosted points (a 32^3 patch with its three
// ghost layers per side, or any shape with px (n1+6)(n2+6) <= that).
constexpr long long kMaxPoints = 54872;
constexpr long long kScratchDoubles = 63 * kMaxPoints;  // pointwise + interface fluxes
constexpr int kMaxWork = 8 * 432;                       // work items, 8 domains
constexpr size_t kWorkOfs = (size_t)kScratchDoubles * sizeof(double);
constexpr size_t kPdOfs = kWorkOfs + (size_t)kMaxWork * sizeof(Work);
constexpr size_t kFlagsOfs = kPdOfs + 256;
constexpr size_t kRhsPtrOfs = kFlagsOfs + 256;
constexpr size_t kStaticBytes = kRhsPtrOfs + 256;
static_assert(sizeof(PatchDev) <= 256, "descriptor slot");
static_assert(kWorkOfs % 16 == 0 && kPdOfs % 16 == 0 && kFlagsOfs % 16 == 0, "slot alignment");

static __device__ __align__(256) unsigned char g_static_area[kStaticBytes];

constexpr int kMaxDevices = 64;
void* g_area_ptr[kMaxDevices] = {nullptr};
std::mutex g_area_mu;

// Device address of g_static_area on the current device, looked up on the
// first call made with that device current (one lookup per device, also when
// several host threads make their first calls at once).
int area_on_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GRMHD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_area_mu);
  if (!g_area_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_area) != cudaSuccess || !p) return GRMHD_ERR_CUDA;
    g_area_ptr[dev] = p;
  }
  *out = (unsigned char*)g_area_ptr[dev];
  return GRMHD_OK;
}

// Block counts per domain, passed by value to the set-up kernel.
struct Blocks {
  int ofs[NDOM + 1];
};

// Writes the descriptor, the output pointer and the work list (patch 0,
// blocks 0 .. nb-1 of each domain, domains in order) into the static array
// and clears the device flags.
__global__ void k_static_setup(PatchDev pd, double* rhs, Blocks b) {
  PatchDev* pd_dev = (PatchDev*)(g_static_area + kPdOfs);
  Work* w = (Work*)(g_static_area + kWorkOfs);
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *pd_dev = pd;
    *(double**)(g_static_area + kRhsPtrOfs) = rhs;
    DevFlags* f = (DevFlags*)(g_static_area + kFlagsOfs);
    f->flags = 0;
    f->worst_status = 0;
  }
  for (int dom = 0; dom < NDOM; ++dom)
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < b.ofs[dom + 1] - b.ofs[dom];
         q += gridDim.x * blockDim.x)
      w[b.ofs[dom] + q] = Work{0, q};
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" int grmhd_rhs_eval_static(const grmhd_params* p, const grmhd_patch_desc* d, const grmhd_eos_table* eos,
                                     int reg, double* rhs, int* dev_flags, void* stream) {
  if (!p || !d || !rhs || reg < 0 || reg > 3) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  if (les_on(*p)) return GRMHD_ERR_ARG;  // the LES point values need scratch memory
  if (p->bc != 0 && p->bc != 1) return GRMHD_ERR_ARG;
  if (p->max_iter < 1 || !(p->h0 > 0.0)) return GRMHD_ERR_ARG;
  if (d->n[0] < 4 || d->n[1] < 4 || d->n[2] < 4 || d->px < d->n[0] + 6 || !(d->dx > 0.0)) return GRMHD_ERR_ARG;
  if (!d->U[reg] || ((uintptr_t)d->U[reg] & 7) || !d->prim || ((uintptr_t)d->prim & 7) || !d->status ||
      ((uintptr_t)rhs & 7) || ((uintptr_t)dev_flags & 3))
    return GRMHD_ERR_ARG;
  Geo G;
  G.n0 = d->n[0];
  G.n1 = d->n[1];
  G.n2 = d->n[2];
  G.px = d->px;
  G.sy = d->px;
  G.sz = G.sy * (G.n1 + 6);
  G.sf = G.sz * (G.n2 + 6);
  G.dx = d->dx;
  G.i12 = 1.0 / (12.0 * G.dx);
  G.i12s = 1.0 / (12.0 * G.dx * G.dx);
  G.i144 = 1.0 / (144.0 * G.dx * G.dx);
  G.ihdx = 0.5 / G.dx;
  if (G.sf > kMaxPoints) return GRMHD_ERR_SIZE;

  Blocks b;
  int nw = 0;
  for (int dom = 0; dom < NDOM; ++dom) {
    b.ofs[dom] = nw;
    int bs = (dom == DOM_INT) ? BS_INT : ((dom >= DOM_IFX && dom <= DOM_IFZ) ? BS_IF : BS_ALL);
    long long nb = (dom_count(dom, G) + bs - 1) / bs;
    if (nw + nb > kMaxWork) return GRMHD_ERR_SIZE;
    nw += (int)nb;
  }
  b.ofs[NDOM] = nw;

  unsigned char* area = nullptr;
  int rc = area_on_current_device(&area);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;

  PatchDev pd;
  pd.G = G;
  for (int r = 0; r < 4; ++r) pd.U[r] = d->U[r] ? d->U[r] : d->U[reg];
  for (int r = 4; r < REG_DENSE + NDENSE; ++r) pd.U[r] = nullptr;
  pd.les = nullptr;
  pd.prim = d->prim;
  pd.status = d->status;
  pd.Fp = (double*)area;
  pd.lam = pd.Fp + 30 * G.sf;
  pd.Fh = pd.lam + 3 * G.sf;
  pd.seed = nullptr;

  const PatchDev* pd_dev = (const PatchDev*)(area + kPdOfs);
  const Work* w_dev = (const Work*)(area + kWorkOfs);
  DevFlags* flags_dev = (DevFlags*)(area + kFlagsOfs);
  double* const* rhs_dev = (double* const*)(area + kRhsPtrOfs);
  k_static_setup<<<4, 256, 0, st>>>(pd, rhs, b);
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;

  Eos E = make_eos(*p, eos);
  launch_c2p(pd_dev, w_dev + b.ofs[DOM_ALL], b.ofs[DOM_ALL + 1] - b.ofs[DOM_ALL], reg, *p, E, flags_dev, nullptr, st);
  for (int dd = 0; dd < 3; ++dd)
    launch_iflux(pd_dev, w_dev + b.ofs[DOM_IFX + dd], b.ofs[DOM_IFX + dd + 1] - b.ofs[DOM_IFX + dd], reg, dd, st);
  launch_rhs(pd_dev, w_dev + b.ofs[DOM_INT], b.ofs[DOM_INT + 1] - b.ofs[DOM_INT], reg, 0, 0, 0.0, *p, rhs_dev, st);
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  if (dev_flags &&
      cudaMemcpyAsync(dev_flags, &flags_dev->flags, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}
