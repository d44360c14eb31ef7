// Oracle of the learned con2prim seeder's network (not part of the paper):
// MLP 8 -> 64 -> 64 -> 64 -> 3 with ReLU, forward, backward of the mean-squared
// error and one Adam step, in FP64.  With `bf16` set, every operand that the
// GPU feeds to its BF16 tensor-core products (inputs, weights, hidden
// activations, output and hidden-layer gradients) is rounded to BF16
// (round-to-nearest-even of the FP32 value) first; sums and biases stay exact.
//
// Parameter layout (floats, 9091): W1[8][64], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], W4[64][3], b4[3]; W[k][j] multiplies input k into unit j.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const int NI = 8, NH = 64, NO = 3;
const int OW1 = 0, OB1 = OW1 + NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH * NH,
          OW4 = OB3 + NH, OB4 = OW4 + NH * NO, NPAR = OB4 + NO;

double bf16(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

struct Net {
  const float* p;
  bool round;
  double r(double x) const { return round ? bf16(x) : x; }
  double W(int off, int k, int j, int nj) const { return r(p[off + k * nj + j]); }
  double b(int off, int j) const { return p[off + j]; }
};

// Forward of one sample; keeps the (rounded) activations for the backward.
void forward(const Net& N, const float* x, double in[NI], double h1[NH], double h2[NH], double h3[NH], double y[NO]) {
  for (int k = 0; k < NI; ++k) in[k] = N.r(x[k]);
  for (int j = 0; j < NH; ++j) {
    double z = N.b(OB1, j);
    for (int k = 0; k < NI; ++k) z += in[k] * N.W(OW1, k, j, NH);
    h1[j] = N.r(z > 0.0 ? z : 0.0);
  }
  for (int j = 0; j < NH; ++j) {
    double z = N.b(OB2, j);
    for (int k = 0; k < NH; ++k) z += h1[k] * N.W(OW2, k, j, NH);
    h2[j] = N.r(z > 0.0 ? z : 0.0);
  }
  for (int j = 0; j < NH; ++j) {
    double z = N.b(OB3, j);
    for (int k = 0; k < NH; ++k) z += h2[k] * N.W(OW3, k, j, NH);
    h3[j] = N.r(z > 0.0 ? z : 0.0);
  }
  for (int j = 0; j < NO; ++j) {
    double z = N.b(OB4, j);
    for (int k = 0; k < NH; ++k) z += h3[k] * N.W(OW4, k, j, NO);
    y[j] = z;
  }
}

}  // namespace

extern "C" {

int oracle_mlp_nparams(void) { return NPAR; }

// y[n][3] = net(x[n][8]).
int oracle_mlp_forward(const float* params, long n, const float* x, double* y, int bf16_operands) {
  Net N{params, bf16_operands != 0};
  double in[NI], h1[NH], h2[NH], h3[NH];
  for (long s = 0; s < n; ++s) forward(N, x + s * NI, in, h1, h2, h3, y + s * NO);
  return 0;
}

// Loss L = mean over samples and outputs of (y - t)^2, and dL/dparams (grad[NPAR]).
double oracle_mlp_grad(const float* params, long n, const float* x, const float* t, double* grad, int bf16_operands) {
  Net N{params, bf16_operands != 0};
  std::vector<double> g(NPAR, 0.0);
  double loss = 0.0;
  const double sc = 2.0 / (3.0 * (double)n);
  double in[NI], h1[NH], h2[NH], h3[NH], y[NO];
  for (long s = 0; s < n; ++s) {
    forward(N, x + s * NI, in, h1, h2, h3, y);
    double dy[NO], dyr[NO];
    for (int j = 0; j < NO; ++j) {
      double e = y[j] - t[s * NO + j];
      loss += e * e;
      dy[j] = sc * e;
      dyr[j] = N.r(dy[j]);
    }
    // Output layer.
    for (int j = 0; j < NO; ++j) {
      g[OB4 + j] += dy[j];
      for (int k = 0; k < NH; ++k) g[OW4 + k * NO + j] += h3[k] * dyr[j];
    }
    // Hidden layers: dz = (dh * [h > 0]); the rounded dz feeds the products.
    double dz3[NH], dz3r[NH], dz2[NH], dz2r[NH], dz1[NH], dz1r[NH];
    for (int k = 0; k < NH; ++k) {
      double d = 0.0;
      for (int j = 0; j < NO; ++j) d += dyr[j] * N.W(OW4, k, j, NO);
      dz3[k] = h3[k] > 0.0 ? d : 0.0;
      dz3r[k] = N.r(dz3[k]);
    }
    for (int j = 0; j < NH; ++j) {
      g[OB3 + j] += dz3[j];
      for (int k = 0; k < NH; ++k) g[OW3 + k * NH + j] += h2[k] * dz3r[j];
    }
    for (int k = 0; k < NH; ++k) {
      double d = 0.0;
      for (int j = 0; j < NH; ++j) d += dz3r[j] * N.W(OW3, k, j, NH);
      dz2[k] = h2[k] > 0.0 ? d : 0.0;
      dz2r[k] = N.r(dz2[k]);
    }
    for (int j = 0; j < NH; ++j) {
      g[OB2 + j] += dz2[j];
      for (int k = 0; k < NH; ++k) g[OW2 + k * NH + j] += h1[k] * dz2r[j];
    }
    for (int k = 0; k < NH; ++k) {
      double d = 0.0;
      for (int j = 0; j < NH; ++j) d += dz2r[j] * N.W(OW2, k, j, NH);
      dz1[k] = h1[k] > 0.0 ? d : 0.0;
      dz1r[k] = N.r(dz1[k]);
    }
    for (int j = 0; j < NH; ++j) {
      g[OB1 + j] += dz1[j];
      for (int k = 0; k < NI; ++k) g[OW1 + k * NH + j] += in[k] * dz1r[j];
    }
  }
  for (int q = 0; q < NPAR; ++q) grad[q] = g[q];
  return loss / (3.0 * (double)n);
}

// Seeder features of flat-metric conserved states cons[n][10] (D, DYe, tau,
// S_i, B^i): with q = tau / D, r = |S| / D, b2 = |B|^2 / D and
// Q = max(1 + q, 1e-30),
//   (log10 D, DYe / D, ln Q, ln max((1 + q - r)(1 + q + r), 1e-30), r / Q,
//    log10 max(b2, 1e-30), S.B / (|S| |B|) or 0, b2 / Q).
int oracle_seeder_features(long n, const double* cons, double* f) {
  for (long s = 0; s < n; ++s) {
    const double* c = cons + 10 * s;
    double D = c[0];
    double Smag = std::sqrt(c[3] * c[3] + c[4] * c[4] + c[5] * c[5]);
    double Bmag = std::sqrt(c[6] * c[6] + c[7] * c[7] + c[8] * c[8]);
    double q = c[2] / D, r = Smag / D, b2 = Bmag * Bmag / D;
    double Q = std::max(1.0 + q, 1e-30);
    double* o = f + NI * s;
    o[0] = std::log10(D);
    o[1] = c[1] / D;
    o[2] = std::log(Q);
    o[3] = std::log(std::max((1.0 + q - r) * (1.0 + q + r), 1e-30));
    o[4] = r / Q;
    o[5] = std::log10(std::max(b2, 1e-30));
    o[6] = (Smag > 0.0 && Bmag > 0.0) ? (c[3] * c[6] + c[4] * c[7] + c[5] * c[8]) / (Smag * Bmag) : 0.0;
    o[7] = b2 / Q;
  }
  return 0;
}

// Seeder targets from the states cons[n][10] and roots[n][3] = (mu_+, mu, W):
//   (ln(mu_+ sqrt(1 + r^2)), ln(mu max(1 + q, 1e-30)), ln W).
// For B = 0 and h0 = 1, mu_+ = 1 / sqrt(1 + r^2) and mu (1 + q) = 1 - p / (rho h W^2),
// so the targets are corrections to those closed forms.
int oracle_seeder_targets(long n, const double* cons, const double* roots, double* t) {
  for (long s = 0; s < n; ++s) {
    const double* c = cons + 10 * s;
    const double* r = roots + 3 * s;
    double D = c[0];
    double rr = std::sqrt(c[3] * c[3] + c[4] * c[4] + c[5] * c[5]) / D;
    double Q = std::max(1.0 + c[2] / D, 1e-30);
    t[3 * s] = std::log(r[0] * std::sqrt(1.0 + rr * rr));
    t[3 * s + 1] = std::log(r[1] * Q);
    t[3 * s + 2] = std::log(r[2]);
  }
  return 0;
}

// One Adam step (step number t >= 1) on FP64 copies of the state.
int oracle_adam(double* w, double* m, double* v, const double* g, long n, double lr, double b1, double b2, double eps,
                int t) {
  double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (long q = 0; q < n; ++q) {
    m[q] = b1 * m[q] + (1.0 - b1) * g[q];
    v[q] = b2 * v[q] + (1.0 - b2) * g[q] * g[q];
    double mh = m[q] / c1, vh = v[q] / c2;
    w[q] -= lr * mh / (std::sqrt(vh) + eps);
  }
  return 0;
}

}  // extern "C"
