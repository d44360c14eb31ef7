// Scalar type of the CPU oracle.
//
// TEST INFRASTRUCTURE ONLY: the oracle is a plain, serial, FP64 restatement of
// the paper's method used to check the CUDA path.  Nothing in the product
// (the CUDA library and its Python binding) may include, link or call it.
//
// In the normal build `real` is `double`.  Built with -DORACLE_COUNT_FLOPS,
// `real` becomes a wrapper that counts every floating-point add, subtract,
// multiply, divide and square root (one flop each; transcendental calls count
// one; negation, fabs, fmin, fmax and comparisons count zero).  The counting
// build gives the algorithmic flop count per grid point that the roofline uses.
#pragma once
#include <cmath>

#ifdef ORACLE_COUNT_FLOPS
extern long long oracle_flops;

struct counted {
  double v;
  counted() : v(0.0) {}
  counted(double x) : v(x) {}
  explicit operator double() const { return v; }
  counted& operator+=(counted o) { ++oracle_flops; v += o.v; return *this; }
  counted& operator-=(counted o) { ++oracle_flops; v -= o.v; return *this; }
  counted& operator*=(counted o) { ++oracle_flops; v *= o.v; return *this; }
  counted& operator/=(counted o) { ++oracle_flops; v /= o.v; return *this; }
};
inline counted operator+(counted a, counted b) { ++oracle_flops; return counted(a.v + b.v); }
inline counted operator-(counted a, counted b) { ++oracle_flops; return counted(a.v - b.v); }
inline counted operator*(counted a, counted b) { ++oracle_flops; return counted(a.v * b.v); }
inline counted operator/(counted a, counted b) { ++oracle_flops; return counted(a.v / b.v); }
inline counted operator-(counted a) { return counted(-a.v); }
inline bool operator<(counted a, counted b) { return a.v < b.v; }
inline bool operator>(counted a, counted b) { return a.v > b.v; }
inline bool operator<=(counted a, counted b) { return a.v <= b.v; }
inline bool operator>=(counted a, counted b) { return a.v >= b.v; }
inline bool operator==(counted a, counted b) { return a.v == b.v; }
inline bool operator!=(counted a, counted b) { return a.v != b.v; }
inline counted sqrt(counted a) { ++oracle_flops; return counted(std::sqrt(a.v)); }
inline counted log(counted a) { ++oracle_flops; return counted(std::log(a.v)); }
inline counted log10(counted a) { ++oracle_flops; return counted(std::log10(a.v)); }
inline counted exp(counted a) { ++oracle_flops; return counted(std::exp(a.v)); }
inline counted cbrt(counted a) { ++oracle_flops; return counted(std::cbrt(a.v)); }
inline counted pow(counted a, counted b) { ++oracle_flops; return counted(std::pow(a.v, b.v)); }
inline counted fabs(counted a) { return counted(std::fabs(a.v)); }
inline counted fmin(counted a, counted b) { return counted(std::fmin(a.v, b.v)); }
inline counted fmax(counted a, counted b) { return counted(std::fmax(a.v, b.v)); }
inline bool isfinite_r(counted a) { return std::isfinite(a.v); }
inline double dbl(counted a) { return a.v; }
typedef counted real;
#else
typedef double real;
inline bool isfinite_r(double a) { return std::isfinite(a); }
inline double dbl(double a) { return a; }
#endif
