// Test infrastructure (CPU oracle): second-order forward-mode automatic differentiation.
//
// An `AD` value carries f, its gradient and its full Hessian with respect to 12 inputs
// (the stacked positions of the four vertices of a contact stencil).  Every arithmetic
// operation applies the chain rule exactly, so derivatives of the barrier and friction
// potentials come out of the same code that evaluates them, with no hand-derived formula.
// Used only by the oracle; the CUDA path derives its derivatives in closed form.
#pragma once
#include <cmath>

namespace orc {

constexpr int NV = 12;

struct AD {
  double v;
  double g[NV];
  double h[NV][NV];

  AD() : v(0) { zero(); }
  AD(double c) : v(c) { zero(); }  // NOLINT: constants convert implicitly
  void zero() {
    for (int i = 0; i < NV; ++i) {
      g[i] = 0;
      for (int j = 0; j < NV; ++j) h[i][j] = 0;
    }
  }
  static AD var(double value, int index) {
    AD a(value);
    a.g[index] = 1.0;
    return a;
  }
};

// unary chain rule: y = f(a), f' = d1, f'' = d2
inline AD chain(const AD& a, double fv, double d1, double d2) {
  AD r(fv);
  for (int i = 0; i < NV; ++i) r.g[i] = d1 * a.g[i];
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j) r.h[i][j] = d1 * a.h[i][j] + d2 * a.g[i] * a.g[j];
  return r;
}

inline AD operator+(const AD& a, const AD& b) {
  AD r(a.v + b.v);
  for (int i = 0; i < NV; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];
  return r;
}
inline AD operator-(const AD& a, const AD& b) {
  AD r(a.v - b.v);
  for (int i = 0; i < NV; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j];
  return r;
}
inline AD operator-(const AD& a) { return AD(0.0) - a; }
inline AD operator*(const AD& a, const AD& b) {
  AD r(a.v * b.v);
  for (int i = 0; i < NV; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j)
      r.h[i][j] = a.h[i][j] * b.v + a.v * b.h[i][j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
  return r;
}
inline AD inv(const AD& a) {
  double x = a.v;
  return chain(a, 1.0 / x, -1.0 / (x * x), 2.0 / (x * x * x));
}
inline AD operator/(const AD& a, const AD& b) { return a * inv(b); }
inline AD sqrt(const AD& a) {
  double s = std::sqrt(a.v);
  return chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}
inline AD log(const AD& a) { return chain(a, std::log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v)); }

inline double val(const AD& a) { return a.v; }
inline double val(double a) { return a; }

}  // namespace orc
