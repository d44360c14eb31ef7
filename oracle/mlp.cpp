// Oracle of the learned con2prim seeder's network (not part of the paper):
// MLP 8 -> 64 -> 64 -> 64 -> 3 with ReLU, forward, backward of the mean-squared
// error and one Adam step, in FP64.  With `bf16` set, every operand that the
// GPU feeds to its BF16 tensor-core products (inputs, weights, hidden
// activations, output and hidden-layer gradients) is rounded to BF16
// (round-to-nearest-even of the FP32 value) first; sums and biases stay exact.
//
// Parameter layout (floats, 9091): W1[8][64], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], W4[64][3], b4[3]; W[k][j] multiplies input k into unit j.
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
