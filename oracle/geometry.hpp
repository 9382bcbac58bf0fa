// Test infrastructure (CPU oracle): unsigned point-triangle and edge-edge distances.
//
// The contact pairs of Sec. III-B are point-triangle (PT) and edge-edge (EE) pairs with
// unsigned distance d_k(x); the paper defers the distance itself to the IPC paper it cites.
// Here d^2 is written out as the minimum of |p - y|^2 over the closed triangle (PT) or of
// |y_a - y_b|^2 over the two closed segments (EE), in the plainest form that is evidently
// that minimum:
//   PT: project p onto the triangle's plane; if the projection's barycentrics are all
//       >= 0 the projection is the closest point, otherwise the minimum lies on the
//       boundary and is the smallest of the three point-segment distances.  (A triangle
//       with collinear vertices has no plane: the smallest edge distance decides.)
//   EE: the squared distance is a convex quadratic in the segment parameters (s,t); if
//       its unconstrained minimiser lies in [0,1]^2 it is the answer, otherwise (or if the
//       segments are parallel to within |ea x eb|^2 <= 1e-20 |ea|^2 |eb|^2) the minimum is
//       on the boundary of the square: the smallest of the four endpoint-segment distances.
// Ties between boundary candidates keep the first in the listed order.
// Templated on the scalar so that the same code gives values (double) and exact first and
// second derivatives (AD).  Each routine also reports the closest-point stencil c[4] with
// r = sum_a c_a x_a = (point on side A) - (point on side B), used for lagged friction.
#pragma once
#include <algorithm>
#include <cmath>

#include "ad.hpp"

namespace orc {

template <class T>
struct V3 {
  T x, y, z;
};
template <class T>
inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T>
inline V3<T> operator*(const V3<T>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T>
inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Region codes.  PT: 0 face, 1..3 edge (t0t1, t1t2, t2t0), 4..6 vertex t0, t1, t2.
// EE: 0 interior-interior, 1..4 endpoint a0, a1, b0, b1 against the other segment's
// interior, 5..8 endpoint-endpoint (a0b0, a0b1, a1b0, a1b1).
enum { PT_FACE = 0 };

// |p - (a + t (b - a))|^2 minimised over t in [0,1]; returns d^2, writes t (clamped).
template <class T>
T point_segment_d2(const V3<T>& p, const V3<T>& a, const V3<T>& b, double* tout) {
  V3<T> e = b - a;
  if (val(dot(e, e)) == 0.0) {  // a segment of zero length is its point
    *tout = 0.0;
    V3<T> r = p - a;
    return dot(r, r);
  }
  T t = dot(p - a, e) / dot(e, e);
  if (val(t) <= 0.0) {
    t = T(0.0);
  } else if (val(t) >= 1.0) {
    t = T(1.0);
  }
  *tout = val(t);
  V3<T> r = p - (a + e * t);
  return dot(r, r);
}

template <class T>
T pt_d2(const V3<T>& p, const V3<T>& t0, const V3<T>& t1, const V3<T>& t2, int* region,
        double c[4]) {
  V3<T> e1 = t1 - t0, e2 = t2 - t0, r0 = p - t0;
  T a = dot(e1, e1), b = dot(e1, e2), cc = dot(e2, e2);
  T d = dot(e1, r0), e = dot(e2, r0);
  T det = a * cc - b * b;
  T b1 = (cc * d - b * e) / det;
  T b2 = (a * e - b * d) / det;
  if (val(b1) >= 0.0 && val(b2) >= 0.0 && val(b1) + val(b2) <= 1.0) {
    V3<T> r = r0 - e1 * b1 - e2 * b2;
    T d2 = dot(r, r);
    // The face point lies in the closed triangle, so no edge is closer unless the solve
    // was singular (a triangle with collinear vertices, where det is rounding noise and
    // any point of the triangle can come out).  The distance is the minimum over the
    // closed triangle: an edge closer by more than rounding (1e-13 relative; a regular
    // triangle's edges are never closer than its face point) wins.
    double t_unused;
    const V3<double> pv = {val(p.x), val(p.y), val(p.z)};
    const V3<double> q0 = {val(t0.x), val(t0.y), val(t0.z)}, q1 = {val(t1.x), val(t1.y), val(t1.z)},
                     q2 = {val(t2.x), val(t2.y), val(t2.z)};
    const double edges = std::min(point_segment_d2(pv, q0, q1, &t_unused),
                                  std::min(point_segment_d2(pv, q1, q2, &t_unused),
                                           point_segment_d2(pv, q2, q0, &t_unused)));
    if (!(edges < val(d2) * (1.0 - 1e-13))) {
      *region = PT_FACE;
      c[0] = 1.0; c[1] = -(1.0 - val(b1) - val(b2)); c[2] = -val(b1); c[3] = -val(b2);
      return d2;
    }
  }
  const V3<T>* tv[3] = {&t0, &t1, &t2};
  T best(0.0);
  int best_k = -1;
  double best_t = 0;
  for (int k = 0; k < 3; ++k) {
    double tp;
    T d2 = point_segment_d2(p, *tv[k], *tv[(k + 1) % 3], &tp);
    if (best_k < 0 || val(d2) < val(best)) {
      best = d2; best_k = k; best_t = tp;
    }
  }
  c[0] = 1.0; c[1] = c[2] = c[3] = 0.0;
  int ia = 1 + best_k, ib = 1 + (best_k + 1) % 3;
  if (best_t <= 0.0) {
    *region = 4 + best_k;
    c[ia] = -1.0;
  } else if (best_t >= 1.0) {
    *region = 4 + (best_k + 1) % 3;
    c[ib] = -1.0;
  } else {
    *region = 1 + best_k;
    c[ia] = -(1.0 - best_t);
    c[ib] = -best_t;
  }
  return best;
}

template <class T>
T ee_d2(const V3<T>& a0, const V3<T>& a1, const V3<T>& b0, const V3<T>& b1, int* region,
        double c[4]) {
  V3<T> ea = a1 - a0, eb = b1 - b0, r0 = a0 - b0;
  T A = dot(ea, ea), B = dot(ea, eb), C = dot(eb, eb);
  T D = dot(ea, r0), E = dot(eb, r0);
  V3<T> n = cross(ea, eb);
  T nn = dot(n, n);
  if (val(nn) > 1e-20 * val(A) * val(C)) {
    // stationarity: A s - B t = -D, -B s + C t = E; determinant A C - B^2 = |ea x eb|^2
    T s = (B * E - C * D) / nn;
    T t = (A * E - B * D) / nn;
    if (val(s) >= 0.0 && val(s) <= 1.0 && val(t) >= 0.0 && val(t) <= 1.0) {
      V3<T> r = r0 + ea * s - eb * t;
      *region = 0;
      c[0] = 1.0 - val(s); c[1] = val(s); c[2] = -(1.0 - val(t)); c[3] = -val(t);
      return dot(r, r);
    }
  }
  // boundary of the parameter square: endpoints against the other segment
  double tp[4];
  T d2[4] = {point_segment_d2(a0, b0, b1, &tp[0]), point_segment_d2(a1, b0, b1, &tp[1]),
             point_segment_d2(b0, a0, a1, &tp[2]), point_segment_d2(b1, a0, a1, &tp[3])};
  int k = 0;
  for (int i = 1; i < 4; ++i)
    if (val(d2[i]) < val(d2[k])) k = i;
  double t = tp[k];
  c[0] = c[1] = c[2] = c[3] = 0.0;
  if (k < 2) {            // endpoint a_k against segment b: r = a_k - (b0 + t eb)
    c[k] = 1.0;
    c[2] = -(1.0 - t); c[3] = -t;
  } else {                // endpoint b_{k-2} against segment a: r = (a0 + t ea) - b
    c[0] = 1.0 - t; c[1] = t;
    c[k] = -1.0;
  }
  bool end = (t <= 0.0 || t >= 1.0);
  if (!end) {
    *region = 1 + k;
  } else {
    int other = (t <= 0.0) ? 0 : 1;   // which endpoint of the other segment
    int ia = (k < 2) ? k : other;     // endpoint of a
    int ib = (k < 2) ? other : k - 2; // endpoint of b
    *region = 5 + ia * 2 + ib;
    if (k < 2) { c[2] = (ib == 0) ? -1.0 : 0.0; c[3] = (ib == 1) ? -1.0 : 0.0; }
    else { c[0] = (ia == 0) ? 1.0 : 0.0; c[1] = (ia == 1) ? 1.0 : 0.0; }
  }
  return d2[k];
}

// IPC log barrier, Eq. 7: b(d) = -(d - dhat)^2 log(d / dhat) on (0, dhat), else 0.
template <class T>
T barrier(const T& d, double dhat) {
  if (val(d) <= 0.0 || val(d) >= dhat) return T(0.0);
  T m = d - T(dhat);
  return -(m * m) * log(d / T(dhat));
}

// f0 of the lagged friction (Sec. III-B): f0(y) = integral_{eps}^{y} f1 + eps with f1 of
// Eq. 9; for y < eps this is -y^3/(3 eps^2) + y^2/eps + eps/3, and y otherwise.
template <class T>
T friction_f0(const T& y, double eps) {
  if (val(y) >= eps) return y;
  return -(y * y * y) / T(3.0 * eps * eps) + (y * y) / T(eps) + T(eps / 3.0);
}

}  // namespace orc
