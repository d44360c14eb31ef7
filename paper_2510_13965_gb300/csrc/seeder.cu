// Learned con2prim seeder (no counterpart in the paper) and the seeded flat
// con2prim.
//
// Network 8 -> 64 -> 64 -> 64 -> 3 (ReLU).  One CTA of 128 threads (4 warps)
// owns a tile of 128 samples.  Every product of inference and training is a
// tcgen05.mma with M = 128 samples: BF16 operands in shared memory, FP32
// accumulator in tensor memory, read back with tcgen05.ld (namespace tc:
// inference; namespace tt: forward, backward and weight gradients).  A
// training tile's partial gradient goes to its own slot of a partial-gradient
// array; the Adam kernel sums the slots in a fixed order, so training is
// deterministic.
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>
#include <cstring>
#include "kern.cuh"

namespace gk {
namespace sd {

constexpr int NI = 8, NH = 64, NO = 3;
constexpr int OW1 = 0, OB1 = OW1 + NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH * NO, NPAR = OB4 + NO;
static_assert(NPAR == GRMHD_SEEDER_NPARAMS, "parameter count");
constexpr int NNORM = 2 * NI + 2 * NO;
static_assert(NNORM == GRMHD_SEEDER_NNORM, "normalisation count");
constexpr int TM = 128;    // samples per CTA
constexpr int MAX_BATCH = 65536;
constexpr int MAX_TILES = MAX_BATCH / TM;

typedef unsigned short u16;

DI u16 bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
DI uint32_t pk(u16 lo, u16 hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
DI uint32_t pkf(float lo, float hi) { return pk(bf(lo), bf(hi)); }

// Features of one conserved state from its undensitized D, DYe, tau and the
// invariants S2 = S_i S^i, B2 = B_i B^i, SB = S_i B^i (Kastaun's scalars: the
// features do not depend on the metric otherwise).  The quantities whose
// cancellation BF16 inputs could not resolve ((1 + q)^2 - r^2 at large
// Lorentz factors, r and q themselves) are formed in FP64; the logarithms of
// the formed quantities, whose results are FP32 features, run in FP32.
// Returns sqrt(1 + r^2) and max(1 + q, 1e-30) for the seed map.
DI void features_sc(double D, double DYe, double tau, double S2, double B2, double SB, float f[NI], double* sr,
                    double* Qo) {
  double iD = 1.0 / D;
  double q = tau * iD;
  double r = sqrt(S2) * iD, b2 = B2 * iD;
  double Q = fmax(1.0 + q, 1e-30);
  double X = fmax((1.0 + q - r) * (1.0 + q + r), 1e-30);
  // Past the cancellation, FP32 is enough for what becomes an FP32 feature.
  const float rf = (float)r, Qf = (float)Q, b2f = (float)b2;
  float den = sqrtf((float)S2) * sqrtf((float)B2);
  f[0] = log10f((float)D);
  f[1] = (float)(DYe * iD);
  f[2] = logf(Qf);
  f[3] = logf((float)X);
  f[4] = rf / Qf;
  f[5] = log10f(fmaxf(b2f, 1e-30f));
  f[6] = den > 0.f ? (float)SB / den : 0.f;
  f[7] = b2f / Qf;
  *sr = (double)sqrtf(fmaf(rf, rf, 1.f));
  *Qo = Q;
}

// Flat-metric state (D, DYe, tau, S_i, B^i).
DI void features(const double* c, float f[NI]) {
  double sr, Q;
  features_sc(c[0], c[1], c[2], c[3] * c[3] + c[4] * c[4] + c[5] * c[5], c[6] * c[6] + c[7] * c[7] + c[8] * c[8],
              c[3] * c[6] + c[4] * c[7] + c[5] * c[8], f, &sr, &Q);
}

// ---- FP32 feature path of the inference kernels ------------------------------
// At inference the features are rounded to BF16 (relative 2^-9) and the seeds
// are polished by the FP64 root finder, so FP32 carries enough of them: the
// inference kernels read the FP64 state, narrow it to FP32 on the integer
// pipe and form features and seeds in FP32, leaving the narrow FP64 pipe to
// the con2prim and flux kernels.  (1 + q)^2 - r^2 loses about 2 W^2 ulps to
// cancellation, below the BF16 rounding for W < 100.

// FP64 -> FP32 with the mantissa truncated (relative error below 2^-23);
// magnitudes below FP32's normal range give a signed zero, above it a signed
// infinity; NaN stays NaN.
DI float narrow(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sgn = hi & 0x80000000u, mh = hi & 0xfffffu, ex = (hi >> 20) & 0x7ffu;
  const int e = (int)ex - 1023 + 127;
  if (e >= 255) return __uint_as_float(sgn | 0x7f800000u | ((ex == 0x7ffu && (mh | lo)) ? 0x400000u : 0u));
  if (e <= 0) return __uint_as_float(sgn);
  return __uint_as_float(sgn | ((unsigned)e << 23) | (mh << 3) | (lo >> 29));
}
// FP32 -> FP64, exact for normal numbers, zeros, infinities and NaN (FP32
// subnormals give a signed zero).
DI double widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sgn = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi;
  if (e == 0xffu) hi = sgn | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else if (e == 0u) hi = sgn;
  else hi = sgn | ((e + (1023u - 127u)) << 20) | (m >> 3);
  const unsigned lo = e == 0u ? 0u : (m & 7u) << 29;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

DI float det3f(const float g[6]) {
  return g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2]);
}
DI void inv3f(const float g[6], float idet, float u[6]) {
  u[0] = (g[3] * g[5] - g[4] * g[4]) * idet;
  u[1] = (g[2] * g[4] - g[1] * g[5]) * idet;
  u[2] = (g[1] * g[4] - g[2] * g[3]) * idet;
  u[3] = (g[0] * g[5] - g[2] * g[2]) * idet;
  u[4] = (g[1] * g[2] - g[0] * g[4]) * idet;
  u[5] = (g[0] * g[3] - g[1] * g[1]) * idet;
}
DI void lower3f(const float g[6], const float v[3], float o[3]) {
  o[0] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  o[1] = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  o[2] = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
}

// The features of features_sc in FP32 (the same formulas); sr = sqrt(1 + r^2)
// and Q = max(1 + q, 1e-30) for the seed map.
DI void features_f32(float D, float DYe, float tau, float S2, float B2, float SB, float f[NI], float* sr, float* Qo) {
  const float iD = 1.0f / D;
  const float q = tau * iD, s = sqrtf(S2), r = s * iD, b2 = B2 * iD;
  const float Q = fmaxf(1.0f + q, 1e-30f);
  const float X = fmaxf((1.0f + q - r) * (1.0f + q + r), 1e-30f);
  const float den = s * sqrtf(B2);
  f[0] = log10f(D);
  f[1] = DYe * iD;
  f[2] = logf(Q);
  f[3] = logf(X);
  f[4] = r / Q;
  f[5] = log10f(fmaxf(b2, 1e-30f));
  f[6] = den > 0.f ? SB / den : 0.f;
  f[7] = b2 / Q;
  *sr = sqrtf(fmaf(r, r, 1.f));
  *Qo = Q;
}

// (sqrt(1 + r^2), max(1 + q, 1e-30)) of a flat-metric state: the scalings of
// the mu_+ and mu targets.
DI void target_scales(const double* c, double* sr, double* Q) {
  double D = c[0];
  double r = sqrt(c[3] * c[3] + c[4] * c[4] + c[5] * c[5]) / D;
  *sr = sqrt(1.0 + r * r);
  *Q = fmax(1.0 + c[2] / D, 1e-30);
}

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor cores (tcgen05).  One CTA of 128
// threads owns a tile of 128 samples: thread r writes row r of the input and
// of each hidden activation into shared memory, one elected thread issues the
// layer's tcgen05.mma (M = 128 samples, N = 64 units or 16 for the 3 outputs,
// K in steps of 16; BF16 operands from shared memory, FP32 accumulator in 64
// TMEM columns), commits it to an mbarrier, and every warp reads its 32 rows
// of the accumulator back with tcgen05.ld for the bias + ReLU + BF16 epilogue.
// Operands use the no-swizzle K-major core-matrix layout: 8 rows x 16 bytes
// per core matrix, slabs of K = 16; within a slab the core matrix of row group
// g and K half h sits at g * 256 + h * 128 bytes, so a matrix descriptor has
// leading (K) byte offset 128 and stride (row group) byte offset 256.
// Persistent: the weights are converted once per CTA.
namespace tc {
constexpr int W1_B = 0;                      // B operand of layer 1: 64 units x K 16 (inputs 8..15 zero)
constexpr int W2_B = W1_B + 64 * 16 * 2;     // 64 x 64
constexpr int W3_B = W2_B + 64 * 64 * 2;     // 64 x 64
constexpr int W4_B = W3_B + 64 * 64 * 2;     // 16 x 64 (outputs 3..15 zero)
constexpr int X_B = W4_B + 16 * 64 * 2;      // A operand of layer 1: 128 x 16
constexpr int H_B = X_B + 128 * 16 * 2;      // A operand of layers 2-4: 128 x 64 (reused)
constexpr int FL_B = H_B + 128 * 64 * 2;     // floats: biases (3 x 64 + 4), normalisation (22 + 2)
constexpr int MBAR_B = FL_B + (3 * NH + 4 + NNORM + 2) * 4;
constexpr int TADDR_B = MBAR_B + 8;
constexpr int SMEM = TADDR_B + 8;
static_assert(MBAR_B % 8 == 0, "mbarrier alignment");
constexpr uint32_t TMEM_COLS = 64;
constexpr uint32_t IDESC_BASE = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);  // f32 <- bf16 x bf16, M 128
constexpr uint32_t IDESC_N64 = IDESC_BASE | ((uint32_t)(64 >> 3) << 17);
constexpr uint32_t IDESC_N16 = IDESC_BASE | ((uint32_t)(16 >> 3) << 17);
constexpr long WAIT_LIMIT = 20000000;

// Byte offset of element (r, k) in an operand of `rows` rows (K-major core layout).
__host__ __device__ inline int core_off(int r, int k, int rows) {
  int kk = k & 15;
  return (k >> 4) * (rows * 32) + (r >> 3) * 256 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2;
}
DI uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
DI uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}
DI void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
DI void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// Bounded wait for the mbarrier phase with the given parity (at most `limit`
// polls); false on timeout.
DI bool wait(uint32_t mbar, uint32_t parity, long limit = WAIT_LIMIT) {
  uint32_t done = 0;
  for (long it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  return done != 0;
}
DI void ld64(uint32_t ta, float* f) {
  uint32_t v[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
      "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
        "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
        "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
        "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 64; ++c) f[c] = __uint_as_float(v[c]);
}
DI void ld16(uint32_t ta, float* f) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) f[c] = __uint_as_float(v[c]);
}

// Weights (BF16, core layout), biases and normalisation into shared memory.
DI void load(const float* __restrict__ w, const float* __restrict__ norm, unsigned char* sm) {
  for (int q = threadIdx.x; q < 64 * 16; q += blockDim.x) {
    int n = q >> 4, k = q & 15;
    *reinterpret_cast<u16*>(sm + W1_B + core_off(n, k, 64)) = k < NI ? bf(w[OW1 + k * NH + n]) : 0;
  }
  for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
    int n = q >> 6, k = q & 63;
    *reinterpret_cast<u16*>(sm + W2_B + core_off(n, k, 64)) = bf(w[OW2 + k * NH + n]);
    *reinterpret_cast<u16*>(sm + W3_B + core_off(n, k, 64)) = bf(w[OW3 + k * NH + n]);
  }
  for (int q = threadIdx.x; q < 16 * 64; q += blockDim.x) {
    int n = q >> 6, k = q & 63;
    *reinterpret_cast<u16*>(sm + W4_B + core_off(n, k, 16)) = n < NO ? bf(w[OW4 + k * NO + n]) : 0;
  }
  float* F = reinterpret_cast<float*>(sm + FL_B);
  for (int q = threadIdx.x; q < NH; q += blockDim.x) {
    F[q] = w[OB1 + q];
    F[NH + q] = w[OB2 + q];
    F[2 * NH + q] = w[OB3 + q];
  }
  if (threadIdx.x < 4) F[3 * NH + threadIdx.x] = threadIdx.x < NO ? w[OB4 + threadIdx.x] : 0.f;
  if (threadIdx.x < NNORM) F[3 * NH + 4 + threadIdx.x] = norm[threadIdx.x];
}

// Row r of the input operand: standardized features as BF16, zeros beyond 8.
DI void put_x(unsigned char* sm, int r, const float f[NI], const float* nrm, bool valid) {
  uint32_t p[4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    p[c] = valid ? pk(bf((f[2 * c] - nrm[2 * c]) / nrm[NI + 2 * c]), bf((f[2 * c + 1] - nrm[2 * c + 1]) / nrm[NI + 2 * c + 1]))
                 : 0u;
  *reinterpret_cast<uint4*>(sm + X_B + core_off(r, 0, 128)) = make_uint4(p[0], p[1], p[2], p[3]);
  *reinterpret_cast<uint4*>(sm + X_B + core_off(r, 8, 128)) = make_uint4(0u, 0u, 0u, 0u);
}

// Epilogue of a hidden layer: row r = bf16(relu(acc + bias)) into the activation operand.
DI void put_h(unsigned char* sm, int r, const float* acc, const float* bias) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t p[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int k = 8 * c + 2 * e;
      p[e] = pkf(fmaxf(acc[k] + bias[k], 0.f), fmaxf(acc[k + 1] + bias[k + 1], 0.f));
    }
    *reinterpret_cast<uint4*>(sm + H_B + core_off(r, 8 * c, 128)) = make_uint4(p[0], p[1], p[2], p[3]);
  }
}

// The four layers of one tile whose inputs are in place; y = network outputs
// of this thread's row.  Returns false (in every thread) when a wait timed out.
// hold > 0 (test hook): no product is issued, so the barrier never completes
// and each wait gives up after `hold` polls with nothing in flight.
DI bool forward(unsigned char* sm, uint32_t tmem, uint32_t& phase, float y[NO], int hold = 0) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mbar = su32(sm + MBAR_B);
  const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
  const float* F = reinterpret_cast<const float*>(sm + FL_B);
  bool ok = true;
  float acc[64];
#pragma unroll 1
  for (int layer = 0; layer < 4; ++layer) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && hold == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (layer == 0) {
        mma(tmem, sdesc(su32(sm + X_B)), sdesc(su32(sm + W1_B)), IDESC_N64, 0u);
      } else {
        const int wb = layer == 1 ? W2_B : layer == 2 ? W3_B : W4_B, nrows = layer == 3 ? 16 : 64;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma(tmem, sdesc(su32(sm + H_B + ks * 128 * 32)), sdesc(su32(sm + wb + ks * nrows * 32)),
              layer == 3 ? IDESC_N16 : IDESC_N64, ks > 0 ? 1u : 0u);
      }
      commit(mbar);
    }
    const long limit = hold > 0 ? (long)hold : WAIT_LIMIT;
    bool done = wait(mbar, phase, limit);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      // Timed out: let the MMA finish (bounded) before the caller frees TMEM.
      wait(mbar, phase ^ 1u, limit);
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (layer < 3) {
      ld64(ta, acc);
      put_h(sm, tid, acc, F + layer * NH);
    } else {
      ld16(ta, acc);
#pragma unroll
      for (int j = 0; j < NO; ++j) y[j] = acc[j] + F[3 * NH + j];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  return ok;
}

// TMEM and mbarrier set-up / tear-down of a CTA.
DI uint32_t begin(unsigned char* sm) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(sm + MBAR_B)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(sm + TADDR_B)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *reinterpret_cast<volatile uint32_t*>(sm + TADDR_B);
}
DI void end(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}
}  // namespace tc

// ---------------------------------------------------------------------------
// Training on the tcgen05 tensor cores.  One CTA of 128 threads owns a tile
// of 128 samples; every product is a tcgen05.mma with M = 128, BF16 operands
// in shared memory (K-major no-swizzle core layout, as for inference) and an
// FP32 accumulator in tensor memory:
//   forward         H_l = relu(H_{l-1} W_l + b_l)        A = H_{l-1} [128 x K], B = W_l^T [N x K]
//   backward data   dZ_l = [H_l > 0] (dZ_{l+1} W_{l+1}^T)  A = dZ_{l+1}, B = W_{l+1} [in x out]
//   weight grads    two stacked products over K = 128 samples:
//     [dZ3^T; dZ2^T] [H2^T; H1^T]^T  -> dW3^T and dW2^T on its diagonal blocks,
//     [dZ1^T; dY^T]  [X^T; H3^T]^T    -> dW1^T and dW4^T on its diagonal blocks,
//   so no operand is padded to M = 128 with zeros beyond dY's 3 rows.
// The epilogues write each activation and gradient twice: as the next
// product's A operand (row = sample) and transposed (row = unit) for the
// weight-gradient products; the ReLU masks are kept as bits.  Bias gradients
// are exact FP32 column sums of the unrounded dz (warp reduce-scatter, then
// a fixed-order sum over the warps), as in the oracle.
namespace tt {
using tc::core_off;
using tc::sdesc;
using tc::su32;
constexpr uint32_t COLS = 256;
constexpr int WF1 = 0;              // B fwd 1: 64 out x 16 in (inputs 8..15 zero)
constexpr int WF2 = WF1 + 2048;     // B fwd 2: 64 x 64
constexpr int WF3 = WF2 + 8192;     // B fwd 3
constexpr int WF4 = WF3 + 8192;     // B fwd 4: 16 out (3 used) x 64 in
constexpr int WB2 = WF4 + 2048;     // B bwd 2: 64 in x 64 out
constexpr int WB3 = WB2 + 8192;     // B bwd 3
constexpr int WB4 = WB3 + 8192;     // B bwd 4: 64 in x 16 out (3 used)
constexpr int XA = WB4 + 2048;      // A fwd 1: 128 x 16
constexpr int HA = XA + 4096;       // A fwd 2 / 4: 128 x 64 (H1, then H3)
constexpr int HB = HA + 16384;      // A fwd 3: H2
constexpr int DYA = HB + 16384;     // A bwd 4: 128 x 16 (3 used)
constexpr int DZA = DYA + 4096;     // A bwd 3 / 2: 128 x 64 (dZ3, then dZ2)
constexpr int A1 = DZA + 16384;     // 128 x K 128: rows 0-63 dZ3^T, 64-127 dZ2^T
constexpr int B1 = A1 + 32768;      // 128 x K 128: rows 0-63 H2^T, 64-127 H1^T
constexpr int A2 = B1 + 32768;      // 128 x K 128: rows 0-63 dZ1^T, 64-66 dY^T, rest 0
constexpr int B2 = A2 + 32768;      // 80 x K 128: rows 0-7 X^T, 8-15 0, 16-79 H3^T
constexpr int MASK = B2 + 20480;    // ReLU masks: uint64 [3][128]
constexpr int FL = MASK + 3 * 128 * 8;
// floats at FL: biases b1 b2 b3 (3 x 64) + b4 (4); normalisation (22 + 2);
// bias-gradient partials [4 warps][196]; loss partials (4 doubles).
constexpr int TF_B = 0, TF_NORM = 3 * NH + 4, TF_GB = TF_NORM + NNORM + 2, TF_LOSS = TF_GB + 4 * (3 * NH + 4);
constexpr int NFL = TF_LOSS + 8;
constexpr int MBAR = FL + NFL * 4;
constexpr int TADDR = MBAR + 8;
constexpr int SMEM = TADDR + 8;
static_assert(MBAR % 8 == 0, "mbarrier alignment");
static_assert(SMEM <= 227 * 1024, "shared memory");
constexpr uint32_t idesc_n(int n) { return tc::IDESC_BASE | ((uint32_t)(n >> 3) << 17); }

DI void st16(unsigned char* sm, int off, float v) { *reinterpret_cast<u16*>(sm + off) = bf(v); }
// Row r of a 128-row K-major operand, K = 0..63, as BF16, 16 bytes at a time.
DI void put_row64(unsigned char* sm, int base, int r, const float* v) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *reinterpret_cast<uint4*>(sm + base + core_off(r, 8 * c, 128)) =
        make_uint4(pkf(v[8 * c], v[8 * c + 1]), pkf(v[8 * c + 2], v[8 * c + 3]), pkf(v[8 * c + 4], v[8 * c + 5]),
                   pkf(v[8 * c + 6], v[8 * c + 7]));
}
// Element (row0 + k, s) of a K-major operand of `rows` rows (row0 a multiple
// of 8, s the K index) sits at col_base(base, s, rows, row0) + col_off(k):
// core_off split into its part fixed by the thread and its part fixed by k.
DI int col_base(int base, int s, int rows, int row0) {
  return base + (s >> 4) * (rows * 32) + row0 * 32 + ((s >> 3) & 1) * 128 + (s & 7) * 2;
}
DI int col_off(int k) { return (k >> 3) * 256 + (k & 7) * 16; }

// Issues ksteps MMAs of K = 16 (A rows 128, B rows brows) into TMEM column col.
DI void issue(unsigned char* sm, uint32_t tmem, int col, int a, int b, int brows, int ksteps, uint32_t idesc) {
  for (int ks = 0; ks < ksteps; ++ks)
    tc::mma(tmem + (uint32_t)col, sdesc(su32(sm + a + ks * 128 * 32)), sdesc(su32(sm + b + ks * brows * 32)), idesc,
            ks > 0 ? 1u : 0u);
}

// Makes the threads' shared-memory writes visible to the tensor cores.
DI void pre_issue() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}

// Commits the issued products, waits for them (bounded) and makes TMEM
// readable; false in every thread on timeout (after a second bounded wait).
DI bool finish(unsigned char* sm, uint32_t& phase) {
  const uint32_t mbar = su32(sm + MBAR);
  if (threadIdx.x == 0) tc::commit(mbar);
  bool done = tc::wait(mbar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!done)) {
    tc::wait(mbar, phase ^ 1u);
    return false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

// Warp reduce-scatter of v[64] (column values of the warp's 32 rows): lane l
// returns the sums over the warp of columns 2l and 2l + 1, in a fixed order.
DI void reduce_scatter64(const float v[64], float out[2], int lane) {
  float a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const bool hi = lane & 16;
    float keep = hi ? v[32 + i] : v[i], send = hi ? v[i] : v[32 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const bool hi = lane & 8;
    float keep = hi ? a[16 + i] : a[i], send = hi ? a[i] : a[16 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 4;
    float keep = hi ? a[8 + i] : a[i], send = hi ? a[i] : a[8 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 2;
    float keep = hi ? a[4 + i] : a[i], send = hi ? a[i] : a[4 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 1;
    float keep = hi ? a[2 + i] : a[i], send = hi ? a[i] : a[2 + i];
    out[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
}

}  // namespace tt

// Forward and backward over one tile of the batch [off, off + nb) on the
// tcgen05 tensor cores; writes the tile's partial gradient (gpart[tile][NPAR])
// and sum of squared errors (lpart[tile]).  off = (step[0] mod nbatch) * nb
// when step is given, else 0.  A tensor-core wait that runs out sets bit 2 of
// *err and the tile's outputs are left unwritten.
__global__ void __launch_bounds__(TM) k_mlp_train_tc(long long n, const float* __restrict__ X,
                                                     const float* __restrict__ T, int nb, long long nbatch,
                                                     const unsigned long long* __restrict__ step,
                                                     const float* __restrict__ w, const float* __restrict__ norm,
                                                     float* __restrict__ gpart, double* __restrict__ lpart, float scale,
                                                     int* __restrict__ err) {
  using namespace tt;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sm = smem;
  const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
  float* F = reinterpret_cast<float*>(sm + FL);
  uint64_t* mask = reinterpret_cast<uint64_t*>(sm + MASK);
  // Weights in both orientations.  Every parameter is read once, coalesced
  // (consecutive threads read consecutive floats), with all of a thread's
  // loads in flight together; the padding of WF1, WF4, WB4 and the stacked
  // A2 / B2 operands is zeroed first.
  for (int q = s; q < 2048 / 16; q += TM) {
    reinterpret_cast<uint4*>(sm + WF1)[q] = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4*>(sm + WF4)[q] = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4*>(sm + WB4)[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int q = s; q < (32768 + 20480) / 16; q += TM)  // A2 and B2 (contiguous)
    reinterpret_cast<uint4*>(sm + A2)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  {
    static_assert(NH * NH % TM == 0 && NI * NH % TM == 0 && NH * NO <= 2 * TM, "weight split over the threads");
    float v2[NH * NH / TM], v3[NH * NH / TM], v1[NI * NH / TM], v4[2];
#pragma unroll
    for (int t = 0; t < NH * NH / TM; ++t) {
      v2[t] = __ldg(w + OW2 + s + TM * t);
      v3[t] = __ldg(w + OW3 + s + TM * t);
    }
#pragma unroll
    for (int t = 0; t < NI * NH / TM; ++t) v1[t] = __ldg(w + OW1 + s + TM * t);
#pragma unroll
    for (int t = 0; t < 2; ++t) v4[t] = s + TM * t < NH * NO ? __ldg(w + OW4 + s + TM * t) : 0.f;
#pragma unroll
    for (int t = 0; t < NH * NH / TM; ++t) {
      const int e = s + TM * t, in = e >> 6, out = e & 63;  // W[in][out]
      st16(sm, WF2 + core_off(out, in, 64), v2[t]);
      st16(sm, WB2 + core_off(in, out, 64), v2[t]);
      st16(sm, WF3 + core_off(out, in, 64), v3[t]);
      st16(sm, WB3 + core_off(in, out, 64), v3[t]);
    }
#pragma unroll
    for (int t = 0; t < NI * NH / TM; ++t) {
      const int e = s + TM * t;
      st16(sm, WF1 + core_off(e & 63, e >> 6, 64), v1[t]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = s + TM * t, in = e / NO, out = e - in * NO;
      if (e < NH * NO) {
        st16(sm, WF4 + core_off(out, in, 16), v4[t]);
        st16(sm, WB4 + core_off(in, out, 64), v4[t]);
      }
    }
  }
  for (int q = s; q < NH; q += TM) {
    F[TF_B + q] = w[OB1 + q];
    F[TF_B + NH + q] = w[OB2 + q];
    F[TF_B + 2 * NH + q] = w[OB3 + q];
  }
  if (s < 4) F[TF_B + 3 * NH + s] = s < NO ? w[OB4 + s] : 0.f;
  if (s < NNORM) F[TF_NORM + s] = norm[s];
  if (s == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(sm + MBAR)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(sm + TADDR)), "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + TADDR);
  const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  uint32_t phase = 0;
  bool ok = true;

  // Input row s: standardized features into X (A operand) and X^T (B2 rows 0-7).
  long long off = step ? (long long)(step[0] % (unsigned long long)nbatch) * nb : 0;
  long long i = (long long)blockIdx.x * TM + s;
  const bool valid = i < nb && off + i < n;
  const long long q = off + i;
  const float* nm = F + TF_NORM;
  float xr[NI];
  static_assert(NI == 8, "two float4 per sample");
  if (valid && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    const float4 p0 = reinterpret_cast<const float4*>(X + q * NI)[0], p1 = reinterpret_cast<const float4*>(X + q * NI)[1];
    xr[0] = p0.x, xr[1] = p0.y, xr[2] = p0.z, xr[3] = p0.w, xr[4] = p1.x, xr[5] = p1.y, xr[6] = p1.z, xr[7] = p1.w;
  } else {
#pragma unroll
    for (int k = 0; k < NI; ++k) xr[k] = valid ? X[q * NI + k] : 0.f;
  }
  {
    float x[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) x[k] = valid ? (xr[k] - nm[k]) / nm[NI + k] : 0.f;
    *reinterpret_cast<uint4*>(sm + XA + core_off(s, 0, 128)) =
        make_uint4(pkf(x[0], x[1]), pkf(x[2], x[3]), pkf(x[4], x[5]), pkf(x[6], x[7]));
    *reinterpret_cast<uint4*>(sm + XA + core_off(s, 8, 128)) = make_uint4(0u, 0u, 0u, 0u);
    const int tb = col_base(B2, s, 80, 0);
#pragma unroll
    for (int k = 0; k < NI; ++k) st16(sm, tb + col_off(k), x[k]);
  }
  float v[64];
  // ---- forward: three hidden layers ----
#pragma unroll 1
  for (int l = 0; l < 3 && ok; ++l) {
    pre_issue();
    if (s == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(sm, tmem, 0, l == 0 ? XA : (l == 1 ? HA : HB), l == 0 ? WF1 : (l == 1 ? WF2 : WF3), 64, l == 0 ? 1 : 4,
            idesc_n(64));
    }
    if (!(ok = finish(sm, phase))) break;
    tc::ld64(ta, v);
    uint64_t m = 0;
#pragma unroll
    for (int k = 0; k < 64; ++k) {
      v[k] = fmaxf(v[k] + F[TF_B + l * NH + k], 0.f);
      m |= (uint64_t)(v[k] > 0.f) << k;
    }
    put_row64(sm, l == 1 ? HB : HA, s, v);
    // transposed copies: H1 -> B1 rows 64-127, H2 -> B1 rows 0-63, H3 -> B2 rows 16-79
    const int tb = l == 0 ? col_base(B1, s, 128, 64) : (l == 1 ? col_base(B1, s, 128, 0) : col_base(B2, s, 80, 16));
#pragma unroll
    for (int k = 0; k < 64; ++k) st16(sm, tb + col_off(k), v[k]);
    mask[l * 128 + s] = m;
  }
  // ---- output layer and error ----
  double se = 0.0;
  if (ok) {
    pre_issue();
    if (s == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(sm, tmem, 0, HA, WF4, 16, 4, idesc_n(16));
    }
    ok = finish(sm, phase);
  }
  if (ok) {
    float y[16];
    tc::ld16(ta, y);
    const float* tn = nm + 2 * NI;
    float dy[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      float e = 0.f;
      if (valid) e = y[j] + F[TF_B + 3 * NH + j] - (T[q * NO + j] - tn[j]) / tn[NO + j];
      se += (double)e * (double)e;
      dy[j] = scale * e;
    }
    static_assert(NO == 3, "dy packing");
    *reinterpret_cast<uint4*>(sm + DYA + core_off(s, 0, 128)) =
        make_uint4(pkf(dy[0], dy[1]), pkf(dy[2], 0.f), 0u, 0u);
    *reinterpret_cast<uint4*>(sm + DYA + core_off(s, 8, 128)) = make_uint4(0u, 0u, 0u, 0u);
    const int tb = col_base(A2, s, 128, 64);
#pragma unroll
    for (int j = 0; j < NO; ++j) st16(sm, tb + col_off(j), dy[j]);
    float* gbw = F + TF_GB + warp * (3 * NH + 4);
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      float t = dy[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) gbw[3 * NH + j] = t;
    }
  }
  // ---- backward data: dZ3, dZ2, dZ1 ----
#pragma unroll 1
  for (int l = 2; l >= 0 && ok; --l) {  // dZ of hidden layer l + 1
    const int c = 2 - l;
    pre_issue();
    if (s == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(sm, tmem, 0, c == 0 ? DYA : DZA, c == 0 ? WB4 : (c == 1 ? WB3 : WB2), 64, c == 0 ? 1 : 4, idesc_n(64));
    }
    if (!(ok = finish(sm, phase))) break;
    tc::ld64(ta, v);
    const uint64_t m = mask[l * 128 + s];
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = (m >> k) & 1 ? v[k] : 0.f;
    // dZ3 / dZ2: A operand of the next product; all three transposed into the
    // stacked operands (dZ3 -> A1 rows 0-63, dZ2 -> A1 rows 64-127, dZ1 -> A2 rows 0-63).
    if (l > 0) put_row64(sm, DZA, s, v);
    const int tb = l == 2 ? col_base(A1, s, 128, 0) : (l == 1 ? col_base(A1, s, 128, 64) : col_base(A2, s, 128, 0));
#pragma unroll
    for (int k = 0; k < 64; ++k) st16(sm, tb + col_off(k), v[k]);
    float sum2[2];
    tt::reduce_scatter64(v, sum2, lane);
    float* gbw = F + TF_GB + warp * (3 * NH + 4) + l * NH;
    gbw[2 * lane] = sum2[0];
    gbw[2 * lane + 1] = sum2[1];
  }
  // ---- weight gradients: the two stacked products ----
  if (ok) {
    pre_issue();
    if (s == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(sm, tmem, 128, A1, B1, 128, 8, idesc_n(128));
      issue(sm, tmem, 0, A2, B2, 80, 8, idesc_n(80));
    }
    ok = finish(sm, phase);
  }
  float* gp = gpart + (size_t)blockIdx.x * NPAR;
  if (ok) {
    const int m = warp * 32 + lane;  // row of both products
    if (warp < 2) {
      tc::ld64(ta + 128, v);  // dW3^T row m: columns = H2 units (in)
#pragma unroll
      for (int k = 0; k < 64; ++k) gp[OW3 + k * NH + m] = v[k];
      float d1[16];
      tc::ld16(ta, d1);  // dW1^T row m: columns 0-7 = input features
#pragma unroll
      for (int k = 0; k < NI; ++k) gp[OW1 + k * NH + m] = d1[k];
    } else {
      tc::ld64(ta + 192, v);  // dW2^T row m - 64
#pragma unroll
      for (int k = 0; k < 64; ++k) gp[OW2 + k * NH + (m - 64)] = v[k];
      tc::ld64(ta + 16, v);  // dW4^T rows 64-66: columns 16-79 = H3 units
      if (m < 64 + NO)
#pragma unroll
        for (int k = 0; k < 64; ++k) gp[OW4 + k * NO + (m - 64)] = v[k];
    }
  }
  // ---- bias gradients and loss: fixed-order sums of the warp partials ----
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  double* lw = reinterpret_cast<double*>(F + TF_LOSS);
  if (lane == 0) lw[warp] = se;
  __syncthreads();
  if (ok) {
    for (int c = s; c < 3 * NH + NO; c += TM) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < 4; ++ww) t += F[TF_GB + ww * (3 * NH + 4) + c];
      int dst = c < NH ? OB1 + c : c < 2 * NH ? OB2 + (c - NH) : c < 3 * NH ? OB3 + (c - 2 * NH) : OB4 + (c - 3 * NH);
      gp[dst] = t;
    }
    if (s == 0) lpart[blockIdx.x] = ((lw[0] + lw[1]) + lw[2]) + lw[3];
  } else if (s == 0) {
    atomicOr(err, 4);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  }
}

// MODE 0: inference from conserved states to seeds (double [n][3]).
// MODE 1: forward from raw features to targets (float [n][3]).
template <int MODE>
__global__ void __launch_bounds__(TM) k_mlp_fwd(long long n, const void* __restrict__ in, const float* __restrict__ w,
                                                const float* __restrict__ norm, void* __restrict__ out,
                                                int* __restrict__ err, int hold) {
  extern __shared__ __align__(1024) unsigned char smem[];
  tc::load(w, norm, smem);
  const uint32_t tmem = tc::begin(smem);
  const float* F = reinterpret_cast<const float*>(smem + tc::FL_B);
  const float* nm = F + 3 * NH + 4;  // features mean/scale, then targets
  const float* tn = nm + 2 * NI;
  const int s = threadIdx.x;
  uint32_t phase = 0;
  const long long ntiles = (n + TM - 1) / TM;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    long long q = tile * TM + s;
    bool valid = q < n;
    float f[NI];
    float sr = 1.f, Q = 1.f;
    if (valid) {
      if (MODE == 0) {
        float c[9];
        const double* cp = static_cast<const double*>(in) + q * 10;
#pragma unroll
        for (int m = 0; m < 9; ++m) c[m] = narrow(cp[m]);
        features_f32(c[0], c[1], c[2], c[3] * c[3] + c[4] * c[4] + c[5] * c[5],
                     c[6] * c[6] + c[7] * c[7] + c[8] * c[8], c[3] * c[6] + c[4] * c[7] + c[5] * c[8], f, &sr, &Q);
      } else {
        const float* fp = static_cast<const float*>(in) + q * NI;
#pragma unroll
        for (int k = 0; k < NI; ++k) f[k] = fp[k];
      }
    }
    tc::put_x(smem, s, f, nm, valid);
    float y[NO];
    if (!tc::forward(smem, tmem, phase, y, hold)) {
      if (s == 0) atomicOr(err, 1);
      break;
    }
    if (!valid) continue;
    float t0 = fmaf(y[0], tn[NO + 0], tn[0]);
    float t1 = fmaf(y[1], tn[NO + 1], tn[1]);
    float t2 = fmaf(y[2], tn[NO + 2], tn[2]);
    if (MODE == 0) {
      // Seeds need no more than FP32 accuracy: the FP64 root finder polishes them.
      double* o = static_cast<double*>(out) + q * 3;
      o[0] = widen(expf(t0) / sr);
      o[1] = widen(expf(t1) / Q);
      o[2] = widen(expf(t2));
    } else {
      float* o = static_cast<float*>(out) + q * 3;
      o[0] = t0;
      o[1] = t1;
      o[2] = t2;
    }
  }
  tc::end(tmem);
}

// ---- seeds for the points of patches ---------------------------------------
// Features of patch point o from the conserved variables of register reg and
// the metric (gamma_ij = gt_ij / chi, gamma^ij = chi gt^ij, sqrt(gamma) =
// sqrt(det gt) chi^(-3/2)), in FP32.  False for atmosphere points (D <
// rho_min, which con2prim resets without solving) and non-finite states: a
// decision rounded the other way at the threshold only changes whether the
// point gets a seed.
DI bool patch_point(const PatchDev& PD, long long o, int reg, float rho_min, float f[NI], float* sr, float* Q) {
  const long long sf = PD.G.sf;
  const double* U = PD.U[reg];
  float gt[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) gt[m] = narrow(U[(GT + m) * sf + o]);
  const float chi = narrow(U[CHI * sf + o]);
  const float det = det3f(gt);
  const float ichi = 1.0f / chi;
  const float isg = 1.0f / (sqrtf(det) * ichi * sqrtf(ichi));
  const float D = narrow(U[DD * sf + o]) * isg;
  if (!(D >= rho_min && isfinite(D))) return false;
  float gtu[6];
  inv3f(gt, 1.0f / det, gtu);
  float Sd[3], Bu[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Sd[a] = narrow(U[(DD + 3 + a) * sf + o]) * isg;
    Bu[a] = narrow(U[(DD + 6 + a) * sf + o]) * isg;
  }
  float Su[3], Bd[3];
  lower3f(gtu, Sd, Su);  // gt^ij S_j; times chi below
  lower3f(gt, Bu, Bd);   // gt_ij B^j; times 1/chi below
  const float S2 = chi * (Sd[0] * Su[0] + Sd[1] * Su[1] + Sd[2] * Su[2]);
  const float B2 = ichi * (Bu[0] * Bd[0] + Bu[1] * Bd[1] + Bu[2] * Bd[2]);
  const float SB = Sd[0] * Bu[0] + Sd[1] * Bu[1] + Sd[2] * Bu[2];
  features_f32(D, narrow(U[(DD + 1) * sf + o]) * isg, narrow(U[(DD + 2) * sf + o]) * isg, S2, B2, SB, f, sr, Q);
  return true;
}

DI void nan_seed(const PatchDev& PD, long long o) {
  float* sd = PD.seed + o;
  sd[0] = sd[PD.G.sf] = sd[2 * PD.G.sf] = __int_as_float(0x7fc00000);
}

// Pass 1 over the points of patch work items (blocks of 128 points, DOM_ALL):
// the atmosphere test; points to solve are appended to `list` (patch, point
// offset; warp-aggregated, in no particular order), the others get NaN seeds
// (which con2prim ignores).  Most points of a star's hierarchy are
// atmosphere, so the network then runs on full tiles of fluid points only.
__global__ void __launch_bounds__(TM) k_seed_scan(const PatchDev* __restrict__ pd, const Work* __restrict__ w,
                                                  int reg, double rho_min, int2* __restrict__ list,
                                                  int* __restrict__ count, long long cap) {
  const Work wk = w[blockIdx.x];
  const PatchDev& PD = pd[wk.patch];
  const long long q = (long long)wk.block * TM + threadIdx.x;
  bool solve = false;
  long long o = 0;
  if (q < dom_count(DOM_ALL, PD.G)) {
    int i, j, k;
    dom_decode(DOM_ALL, PD.G, q, i, j, k);
    o = at(PD.G, i, j, k);
    // D = Dbar chi^(3/2) / sqrt(det gt), with det gt = 1 (the conformal
    // metric's determinant, 1 up to truncation error): two loads per point
    // instead of eight.  The second pass tests again with the determinant.
    const double* U = PD.U[reg];
    const float chi = narrow(U[CHI * PD.G.sf + o]);
    const float D = narrow(U[DD * PD.G.sf + o]) * chi * sqrtf(chi);
    solve = D >= narrow(rho_min) && isfinite(D);
    if (!solve) nan_seed(PD, o);
  }
  const unsigned m = __ballot_sync(0xffffffffu, solve);
  if (!m) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (solve) {
    const long long e = (long long)base + __popc(m & ((1u << lane) - 1u));
    if (e < cap) list[e] = make_int2(wk.patch, (int)o);
    else nan_seed(PD, o);  // cannot happen: the list holds every point
  }
}

// Pass 2: seeds of the listed points (count written by pass 1), tiles of 128
// list entries on the tcgen05 tensor cores; seeds (float) into
// PatchDev::seed.  Persistent; CTAs without a tile return before any set-up.
__global__ void __launch_bounds__(TM) k_mlp_list(const PatchDev* __restrict__ pd, const int2* __restrict__ list,
                                                 const int* __restrict__ count, long long cap, int reg,
                                                 double rho_min, const float* __restrict__ wts,
                                                 const float* __restrict__ norm, int* __restrict__ err, int hold) {
  const int nl = (int)((long long)*count < cap ? (long long)*count : cap);
  const int ntiles = (nl + TM - 1) / TM;
  if ((int)blockIdx.x >= ntiles) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  tc::load(wts, norm, smem);
  const uint32_t tmem = tc::begin(smem);
  const float* F = reinterpret_cast<const float*>(smem + tc::FL_B);
  const float* nm = F + 3 * NH + 4;
  const float* tn = nm + 2 * NI;
  const int s = threadIdx.x;
  const float rho_min_f = narrow(rho_min);
  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e = tile * TM + s;
    int2 it = make_int2(0, 0);
    bool solve = false;
    float f[NI];
    float sr = 1.f, Q = 1.f;
    if (e < nl) {
      it = list[e];
      solve = patch_point(pd[it.x], it.y, reg, rho_min_f, f, &sr, &Q);
    }
    tc::put_x(smem, s, f, nm, solve);
    float y[NO];
    if (!tc::forward(smem, tmem, phase, y, hold)) {
      if (s == 0) atomicOr(err, 4);
      break;
    }
    if (e < nl) {
      const PatchDev& PD = pd[it.x];
      if (solve) {
        float* sd = PD.seed + it.y;
        const long long sf = PD.G.sf;
        sd[0] = expf(fmaf(y[0], tn[NO + 0], tn[0])) / sr;
        sd[sf] = expf(fmaf(y[1], tn[NO + 1], tn[1])) / Q;
        sd[2 * sf] = expf(fmaf(y[2], tn[NO + 2], tn[2]));
      } else {
        nan_seed(PD, it.y);
      }
    }
  }
  tc::end(tmem);
}

// Sums nparts partial gradients (fixed order) into grad and the loss partials into loss.
__global__ void k_reduce_grad(const float* __restrict__ gpart, int nparts, const double* __restrict__ lpart,
                              float* __restrict__ grad, double* __restrict__ loss, double lscale) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < NPAR) {
    float g = 0.f;
    for (int p = 0; p < nparts; ++p) g += gpart[(size_t)p * NPAR + q];
    grad[q] = g;
  }
  if (q == 0 && loss) {
    double l = 0.0;
    for (int p = 0; p < nparts; ++p) l += lpart[p];
    *loss = l * lscale;
  }
}

// Adam on the FP32 master weights.  The gradient is the fixed-order sum of
// nparts partials.  With ctr: step s = ctr[0] (then ctr[0] += 1 once every
// block is done), learning rate on a half cosine from lr0 to lr1 over total
// steps, and the step's mean loss added to loss_hist[s / spe]; without ctr:
// step s = fixed_step - 1, learning rate lr0.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ gpart, int nparts, unsigned long long* ctr, long long fixed_step,
                       long long total, long long spe, float lr0, float lr1, float b1, float b2, float eps,
                       const double* __restrict__ lpart, double* __restrict__ loss_hist, double lscale) {
  long long s = ctr ? (long long)ctr[0] : fixed_step - 1;
  float lr = lr0;
  if (ctr && total > 1)
    lr = lr1 + 0.5f * (lr0 - lr1) * (1.f + cospif((float)((double)s / (double)(total - 1))));
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < NPAR) {
    float g = 0.f;
    for (int p = 0; p < nparts; ++p) g += gpart[(size_t)p * NPAR + q];
    // Bias corrections in FP64: 1 - beta2^t in FP32 loses ~5 digits to cancellation.
    double t = (double)(s + 1);
    float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    float mm = b1 * m[q] + (1.f - b1) * g;
    float vv = b2 * v[q] + (1.f - b2) * g * g;
    m[q] = mm;
    v[q] = vv;
    float mh = mm / c1;
    float vh = vv / c2;
    w[q] -= lr * mh / (sqrtf(vh) + eps);
  }
  if (ctr) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss_hist) {
      double l = 0.0;
      for (int p = 0; p < nparts; ++p) l += lpart[p];
      loss_hist[s / spe] += l * lscale;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      unsigned long long tk = atomicAdd(&ctr[1], 1ull);
      if (tk == gridDim.x - 1) {
        ctr[1] = 0ull;
        ctr[0] = (unsigned long long)(s + 1);
        __threadfence();
      }
    }
  }
}

// Per-channel sums of the 11 channels (8 features, 3 targets): block b writes
// part[b][22] = (sum x, sum x^2) per channel.
constexpr int STAT_BLOCKS = 304, STAT_THREADS = 256;
__global__ void __launch_bounds__(STAT_THREADS) k_stats(long long n, const float* __restrict__ X,
                                                        const float* __restrict__ T, double* __restrict__ part) {
  __shared__ double red[STAT_THREADS / 32][2 * (NI + NO)];
  double acc[2 * (NI + NO)];
#pragma unroll
  for (int c = 0; c < 2 * (NI + NO); ++c) acc[c] = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < NI + NO; ++c) {
      double x = c < NI ? X[q * NI + c] : T[q * NO + (c - NI)];
      acc[2 * c] += x;
      acc[2 * c + 1] += x * x;
    }
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 2 * (NI + NO); ++c) {
    double x = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][c] = x;
  }
  __syncthreads();
  if (threadIdx.x < 2 * (NI + NO)) {
    double x = 0.0;
    for (int ww = 0; ww < STAT_THREADS / 32; ++ww) x += red[ww][threadIdx.x];
    part[blockIdx.x * 2 * (NI + NO) + threadIdx.x] = x;
  }
}

// Normalisation from the block sums: mean and standard deviation (scale 1
// for a channel that does not vary).
__global__ void k_norm(long long n, const double* __restrict__ part, float* __restrict__ norm) {
  int c = threadIdx.x;
  if (c >= NI + NO) return;
  double s1 = 0.0, s2 = 0.0;
  for (int b = 0; b < STAT_BLOCKS; ++b) {
    s1 += part[b * 2 * (NI + NO) + 2 * c];
    s2 += part[b * 2 * (NI + NO) + 2 * c + 1];
  }
  double mean = s1 / (double)n;
  double var = fmax(s2 / (double)n - mean * mean, 0.0);
  double sdv = sqrt(var);
  if (!(sdv > 1e-6 * (1.0 + fabs(mean)))) sdv = 1.0;
  if (c < NI) {
    norm[c] = (float)mean;
    norm[NI + c] = (float)sdv;
  } else {
    norm[2 * NI + (c - NI)] = (float)mean;
    norm[2 * NI + NO + (c - NI)] = (float)sdv;
  }
}

__global__ void k_features(long long n, const double* __restrict__ cons, float* __restrict__ f) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  double c[9];
#pragma unroll
  for (int m = 0; m < 9; ++m) c[m] = cons[q * 10 + m];
  float o[NI];
  features(c, o);
#pragma unroll
  for (int k = 0; k < NI; ++k) f[q * NI + k] = o[k];
}

__global__ void k_targets(long long n, const double* __restrict__ cons, const double* __restrict__ roots,
                          float* __restrict__ t) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  double sr, Q;
  target_scales(cons + q * 10, &sr, &Q);
  t[q * 3] = (float)log(roots[q * 3] * sr);
  t[q * 3 + 1] = (float)log(roots[q * 3 + 1] * Q);
  t[q * 3 + 2] = (float)log(roots[q * 3 + 2]);
}

__global__ void __launch_bounds__(128) k_c2p_flat_seeded(grmhd_params P, Eos E, long long n,
                                                          const double* __restrict__ cons,
                                                          const double* __restrict__ seeds, double delta,
                                                          double* __restrict__ prim, int8_t* __restrict__ status,
                                                          int32_t* __restrict__ iters, double* __restrict__ roots,
                                                          int8_t* __restrict__ seeded,
                                                          const int32_t* __restrict__ order) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (order) q = order[q];  // thread i solves state order[i]
  const double g[6] = {1.0, 0.0, 0.0, 1.0, 0.0, 1.0};
  double cb[9];
  for (int m = 0; m < 9; ++m) cb[m] = ld(cons + q * 10 + m);
  double sq[3];
  if (seeds)
    for (int m = 0; m < 3; ++m) sq[m] = ld(seeds + q * 3 + m);
  C2POut r;
  c2p_point(P, E, cb, g, g, 1.0, 1.0, r, seeds ? sq : nullptr, delta);
  for (int m = 0; m < NP; ++m) prim[q * NP + m] = r.prim[m];
  status[q] = (int8_t)r.status;
  if (iters) iters[q] = r.iters;
  if (seeded) seeded[q] = (int8_t)r.seeded;
  if (roots) {
    roots[q * 3] = r.mu_plus;
    roots[q * 3 + 1] = r.mu;
    roots[q * 3 + 2] = r.W_root;
  }
}

// splitmix64 (Steele, Lea and Flood 2014) for the weight initialisation.
inline uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace sd
}  // namespace gk

using namespace gk;
using namespace gk::sd;

struct grmhd_seeder {
  int dev = 0;
  float* w = nullptr;  // [NPAR] master weights
  float* m = nullptr;  // [NPAR] Adam first moment
  float* v = nullptr;  // [NPAR] Adam second moment
  float* norm = nullptr;  // [NNORM]
  unsigned long long* ctr = nullptr;  // [2] step, ticket
  int* err = nullptr;                 // tensor-core wait timed out (inference kernels)
  double* stats = nullptr;            // [STAT_BLOCKS][22]
  float* gpart = nullptr;             // [MAX_TILES][NPAR]
  double* lpart = nullptr;            // [MAX_TILES]
  void* block = nullptr;              // one allocation for all of the above
  cudaStream_t cap = nullptr;         // stream used for graph capture
  int hold = 0;                       // test hook: polls per product wait with no product issued
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool attr_set = false;
int set_smem_attrs() {
  if (attr_set) return GRMHD_OK;
  if (cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tt::SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_fwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_list, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  attr_set = true;
  return GRMHD_OK;
}

unsigned grid_of(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Resident CTAs per SM of a tensor-core inference kernel, from its registers
// and shared memory, at most 5 (each CTA holds 64 of the SM's 512 TMEM
// columns; 5 leaves 192 for other work).
int tc_ctas_per_sm(const void* fn, int dev) {
  cudaFuncAttributes fa;
  int smem_sm = 0;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return 1;
  int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * TM) : 4;
  int by_smem = smem_sm / (tc::SMEM + 1024);
  int n = by_regs < by_smem ? by_regs : by_smem;
  return n < 1 ? 1 : (n > 5 ? 5 : n);
}

// Persistent grid of the forward kernels: resident CTAs per SM x SMs, at most
// one CTA per tile.
template <int MODE>
unsigned fwd_grid(long long n) {
  static int per_dev[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!per_dev[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    per_dev[dev] = (sms > 0 ? sms : 1) * tc_ctas_per_sm((const void*)k_mlp_fwd<MODE>, dev);
  }
  long long tiles = (n + TM - 1) / TM;
  return (unsigned)(tiles < per_dev[dev] ? tiles : per_dev[dev]);
}

int last_rc() { return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA; }

}  // namespace

namespace gk {
int launch_seeder_patches(const grmhd_seeder* s, const PatchDev* pd, const Work* w, int nblk, int reg, double rho_min,
                          int2* list, int* count, long long cap, int* err, cudaStream_t st) {
  if (!s || nblk <= 0) return nblk <= 0 ? GRMHD_OK : GRMHD_ERR_ARG;
  if (!list || !count || cap < 1) return GRMHD_ERR_ARG;
  static int per_dev[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!per_dev[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    per_dev[dev] = (sms > 0 ? sms : 1) * tc_ctas_per_sm((const void*)k_mlp_list, dev);
  }
  if (cudaMemsetAsync(count, 0, sizeof(int), st) != cudaSuccess) return GRMHD_ERR_CUDA;
  k_seed_scan<<<nblk, TM, 0, st>>>(pd, w, reg, rho_min, list, count, cap);
  // The grid covers every listed point however many pass 1 finds (at most
  // one tile per block and round).
  const long long tiles = ((long long)nblk * TM + TM - 1) / TM;
  const int grid = (int)(tiles < per_dev[dev] ? tiles : per_dev[dev]);
  k_mlp_list<<<grid, TM, tc::SMEM, st>>>(pd, list, count, cap, reg, rho_min, s->w, s->norm, err, s->hold);
  return last_rc();
}
}  // namespace gk

extern "C" {

int grmhd_seeder_create(grmhd_seeder** out, unsigned long long seed) {
  if (!out) return GRMHD_ERR_ARG;
  *out = nullptr;
  if (set_smem_attrs()) return GRMHD_ERR_CUDA;
  grmhd_seeder* s = new grmhd_seeder();
  cudaGetDevice(&s->dev);
  size_t o_w = 0, o_m = align256(o_w + NPAR * 4), o_v = align256(o_m + NPAR * 4), o_n = align256(o_v + NPAR * 4),
         o_c = align256(o_n + NNORM * 4), o_s = align256(o_c + 32), o_g = align256(o_s + STAT_BLOCKS * 22 * 8),
         o_l = align256(o_g + (size_t)MAX_TILES * NPAR * 4), total = align256(o_l + MAX_TILES * 8);
  if (cudaMalloc(&s->block, total) != cudaSuccess) {
    delete s;
    return GRMHD_ERR_CUDA;
  }
  char* b = static_cast<char*>(s->block);
  s->w = (float*)(b + o_w);
  s->m = (float*)(b + o_m);
  s->v = (float*)(b + o_v);
  s->norm = (float*)(b + o_n);
  s->ctr = (unsigned long long*)(b + o_c);
  s->err = (int*)(b + o_c + 16);
  s->stats = (double*)(b + o_s);
  s->gpart = (float*)(b + o_g);
  s->lpart = (double*)(b + o_l);
  if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(s->block);
    delete s;
    return GRMHD_ERR_CUDA;
  }
  // He-uniform weights, zero biases.
  float h[NPAR];
  uint64_t st = seed;
  const int offs[4] = {OW1, OW2, OW3, OW4}, fan[4] = {NI, NH, NH, NH}, cnt[4] = {NI * NH, NH * NH, NH * NH, NH * NO};
  for (int q = 0; q < NPAR; ++q) h[q] = 0.f;
  for (int l = 0; l < 4; ++l) {
    float a = sqrtf(6.f / (float)fan[l]);
    for (int q = 0; q < cnt[l]; ++q) {
      double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      h[offs[l] + q] = (float)((2.0 * u - 1.0) * a);
    }
  }
  float nm[NNORM];
  for (int c = 0; c < NNORM; ++c) nm[c] = 0.f;
  for (int c = 0; c < NI; ++c) nm[NI + c] = 1.f;
  for (int c = 0; c < NO; ++c) nm[2 * NI + NO + c] = 1.f;
  int rc = grmhd_seeder_set_params(s, h, nm);
  if (!rc && (cudaMemset(s->err, 0, sizeof(int)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess))
    rc = GRMHD_ERR_CUDA;
  if (rc) {
    grmhd_seeder_destroy(s);
    return rc;
  }
  *out = s;
  return GRMHD_OK;
}

int grmhd_seeder_set_params(grmhd_seeder* s, const float* params, const float* norm) {
  if (!s) return GRMHD_ERR_ARG;
  if (params && cudaMemcpy(s->w, params, NPAR * 4, cudaMemcpyHostToDevice) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (norm) {
    for (int c = 0; c < NI; ++c)
      if (!(norm[NI + c] != 0.f)) return GRMHD_ERR_ARG;
    for (int c = 0; c < NO; ++c)
      if (!(norm[2 * NI + NO + c] != 0.f)) return GRMHD_ERR_ARG;
    if (cudaMemcpy(s->norm, norm, NNORM * 4, cudaMemcpyHostToDevice) != cudaSuccess) return GRMHD_ERR_CUDA;
  }
  if (cudaMemset(s->m, 0, NPAR * 4) != cudaSuccess || cudaMemset(s->v, 0, NPAR * 4) != cudaSuccess ||
      cudaMemset(s->ctr, 0, 16) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

int grmhd_seeder_get_params(grmhd_seeder* s, float* params, float* norm) {
  if (!s) return GRMHD_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return GRMHD_ERR_CUDA;
  if (params && cudaMemcpy(params, s->w, NPAR * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (norm && cudaMemcpy(norm, s->norm, NNORM * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

int grmhd_seeder_features(long long n, const double* cons, float* f, void* stream) {
  if (n < 0 || (n > 0 && (!cons || !f))) return GRMHD_ERR_ARG;
  if (n == 0) return GRMHD_OK;
  k_features<<<grid_of(n, 256), 256, 0, (cudaStream_t)stream>>>(n, cons, f);
  return last_rc();
}

int grmhd_seeder_targets(long long n, const double* cons, const double* roots, float* t, void* stream) {
  if (n < 0 || (n > 0 && (!cons || !roots || !t))) return GRMHD_ERR_ARG;
  if (n == 0) return GRMHD_OK;
  k_targets<<<grid_of(n, 256), 256, 0, (cudaStream_t)stream>>>(n, cons, roots, t);
  return last_rc();
}

int grmhd_seeder_forward(grmhd_seeder* s, long long n, const float* f, float* t_out, void* stream) {
  if (!s || n < 0 || (n > 0 && (!f || !t_out))) return GRMHD_ERR_ARG;
  if (n == 0) return GRMHD_OK;
  k_mlp_fwd<1><<<fwd_grid<1>(n), TM, tc::SMEM, (cudaStream_t)stream>>>(n, f, s->w, s->norm, t_out, s->err, s->hold);
  return last_rc();
}

int grmhd_seeder_infer(grmhd_seeder* s, long long n, const double* cons, double* seeds, void* stream) {
  if (!s || n < 0 || (n > 0 && (!cons || !seeds))) return GRMHD_ERR_ARG;
  if (n == 0) return GRMHD_OK;
  k_mlp_fwd<0><<<fwd_grid<0>(n), TM, tc::SMEM, (cudaStream_t)stream>>>(n, cons, s->w, s->norm, seeds, s->err,
                                                                        s->hold);
  return last_rc();
}

int grmhd_seeder_grad(grmhd_seeder* s, long long n, const float* f, const float* t, float* grad, double* loss,
                      void* stream) {
  if (!s || n < 1 || n > MAX_BATCH || !f || !t || !grad) return GRMHD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int tiles = (int)grid_of(n, TM);
  k_mlp_train_tc<<<tiles, TM, tt::SMEM, st>>>(n, f, t, (int)n, 1, nullptr, s->w, s->norm, s->gpart, s->lpart,
                                              (float)(2.0 / (3.0 * (double)n)), s->err);
  k_reduce_grad<<<grid_of(NPAR, 256), 256, 0, st>>>(s->gpart, tiles, s->lpart, grad, loss, 1.0 / (3.0 * (double)n));
  return last_rc();
}

int grmhd_seeder_adam(grmhd_seeder* s, const float* grad, long long step, float lr, float beta1, float beta2,
                      float eps, void* stream) {
  if (!s || !grad || step < 1) return GRMHD_ERR_ARG;
  k_adam<<<grid_of(NPAR, 256), 256, 0, (cudaStream_t)stream>>>(s->w, s->m, s->v, grad, 1, nullptr, step, 0, 1, lr,
                                                               lr, beta1, beta2, eps, nullptr, nullptr, 0.0);
  return last_rc();
}

int grmhd_seeder_train(grmhd_seeder* s, long long n, const float* f, const float* t, const grmhd_train_cfg* cfg,
                       double* loss_hist, void* stream) {
  if (!s || !cfg || !f || !t) return GRMHD_ERR_ARG;
  const int bsz = cfg->batch;
  if (bsz < TM || bsz > MAX_BATCH || bsz % TM || cfg->epochs < 1 || n < bsz) return GRMHD_ERR_ARG;
  if (!(cfg->lr > 0.f) || !(cfg->lr_final >= 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
    return GRMHD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nbatch = n / bsz, total = nbatch * cfg->epochs;
  const int tiles = bsz / TM;
  if (cfg->fit_norm) {
    k_stats<<<STAT_BLOCKS, STAT_THREADS, 0, st>>>(n, f, t, s->stats);
    k_norm<<<1, 32, 0, st>>>(n, s->stats, s->norm);
  }
  if (cudaMemsetAsync(s->m, 0, NPAR * 4, st) != cudaSuccess || cudaMemsetAsync(s->v, 0, NPAR * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->ctr, 0, 16, st) != cudaSuccess ||
      (loss_hist && cudaMemsetAsync(loss_hist, 0, sizeof(double) * cfg->epochs, st) != cudaSuccess))
    return GRMHD_ERR_CUDA;
  // One epoch as a graph: nbatch x (forward/backward, Adam).
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GRMHD_ERR_CUDA;
  const float scale = (float)(2.0 / (3.0 * (double)bsz));
  const double lscale = 1.0 / (3.0 * (double)bsz * (double)nbatch);
  for (long long b = 0; b < nbatch; ++b) {
    k_mlp_train_tc<<<tiles, TM, tt::SMEM, s->cap>>>(n, f, t, bsz, nbatch, s->ctr, s->w, s->norm, s->gpart,
                                                    s->lpart, scale, s->err);
    k_adam<<<grid_of(NPAR, 256), 256, 0, s->cap>>>(s->w, s->m, s->v, s->gpart, tiles, s->ctr, 0, total, nbatch,
                                                    cfg->lr, cfg->lr_final, cfg->beta1, cfg->beta2, cfg->eps, s->lpart,
                                                    loss_hist, lscale);
  }
  cudaError_t e1 = cudaStreamEndCapture(s->cap, &g);
  if (e1 != cudaSuccess || !g) return GRMHD_ERR_CUDA;
  cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return GRMHD_ERR_CUDA;
  int rc = GRMHD_OK;
  for (int e = 0; e < cfg->epochs && rc == GRMHD_OK; ++e)
    if (cudaGraphLaunch(ge, st) != cudaSuccess) rc = GRMHD_ERR_CUDA;
  // The executable graph may be destroyed while its launches are pending.
  cudaGraphExecDestroy(ge);
  return rc;
}

int grmhd_seeder_hold_products(grmhd_seeder* s, int polls) {
  if (!s || polls < 0) return GRMHD_ERR_ARG;
  s->hold = polls;
  return GRMHD_OK;
}

int grmhd_seeder_status(grmhd_seeder* s) {
  if (!s) return GRMHD_ERR_ARG;
  int e = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(s->err, 0, sizeof(int)) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return e ? GRMHD_ERR_TIMEOUT : GRMHD_OK;
}

void grmhd_seeder_destroy(grmhd_seeder* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->block) cudaFree(s->block);
  delete s;
}

int grmhd_c2p_flat_seeded(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* cons,
                          const double* seeds, double delta, double* prim, int8_t* status, int32_t* iters,
                          double* roots, int8_t* seeded, void* stream) {
  if (!p || n < 0 || (n > 0 && (!cons || !prim || !status))) return GRMHD_ERR_ARG;
  if (eos_check(*p, eos) != GRMHD_OK) return GRMHD_ERR_ARG;
  if (p->max_iter < 1 || !(p->h0 > 0.0)) return GRMHD_ERR_ARG;
  if (seeds && !(delta > 0.0 && delta < 1.0)) return GRMHD_ERR_ARG;
  if (n == 0) return GRMHD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* order = c2p_flat_order(n, cons, st);
  k_c2p_flat_seeded<<<grid_of(n, 128), 128, 0, st>>>(*p, make_eos(*p, eos), n, cons, seeds, delta, prim, status,
                                                      iters, roots, seeded, order);
  c2p_flat_order_free(order, st);
  return last_rc();
}

}  // extern "C"
