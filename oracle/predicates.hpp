// Test infrastructure (CPU oracle): exact orientation predicates by floating-point
// expansion arithmetic (Shewchuk 1997, "Adaptive precision floating-point arithmetic and
// fast robust geometric predicates"), written from the method's description.
//
// An expansion is a sum of doubles whose components do not overlap; its sign is the sign
// of its largest-magnitude nonzero component.  two_sum / two_prod give the exact error of
// one addition / multiplication, so sums and products of expansions are exact and the
// sign of a determinant of double inputs is decided without rounding.  This is the
// penetration checker behind the "no intersection after an accepted step" invariant.
#pragma once
#include <cmath>
#include <vector>

namespace orc {

using Expansion = std::vector<double>;

inline void two_sum(double a, double b, double& x, double& y) {
  x = a + b;
  double bv = x - a;
  double av = x - bv;
  y = (a - av) + (b - bv);
}

inline void two_prod(double a, double b, double& x, double& y) {
  x = a * b;
  y = std::fma(a, b, -x);
}

// e + b, components kept in increasing magnitude, zeros dropped
inline Expansion grow(const Expansion& e, double b) {
  Expansion h;
  h.reserve(e.size() + 1);
  double q = b;
  for (double ei : e) {
    double s, err;
    two_sum(q, ei, s, err);
    if (err != 0.0) h.push_back(err);
    q = s;
  }
  if (q != 0.0 || h.empty()) h.push_back(q);
  return h;
}

inline Expansion add(const Expansion& e, const Expansion& f) {
  Expansion h = e;
  for (double fi : f) h = grow(h, fi);
  return h;
}

inline Expansion neg(const Expansion& e) {
  Expansion h(e);
  for (double& v : h) v = -v;
  return h;
}

inline Expansion scale(const Expansion& e, double b) {
  Expansion h{0.0};
  for (double ei : e) {
    double p, err;
    two_prod(ei, b, p, err);
    h = grow(h, err);
    h = grow(h, p);
  }
  return h;
}

inline Expansion mul(const Expansion& e, const Expansion& f) {
  Expansion h{0.0};
  for (double fi : f) h = add(h, scale(e, fi));
  return h;
}

inline Expansion diff(double a, double b) {
  double x, y;
  two_sum(a, -b, x, y);
  Expansion e;
  if (y != 0.0) e.push_back(y);
  e.push_back(x);
  return e;
}

inline int sign(const Expansion& e) {
  for (size_t i = e.size(); i-- > 0;)
    if (e[i] != 0.0) return e[i] > 0 ? 1 : -1;
  return 0;
}

// sign of det[a-d; b-d; c-d] (positive when d lies below the plane of a,b,c oriented
// counter-clockwise seen from above)
inline int orient3d(const double* a, const double* b, const double* c, const double* d) {
  Expansion ad[3], bd[3], cd[3];
  for (int k = 0; k < 3; ++k) {
    ad[k] = diff(a[k], d[k]);
    bd[k] = diff(b[k], d[k]);
    cd[k] = diff(c[k], d[k]);
  }
  Expansion cx = add(mul(bd[1], cd[2]), neg(mul(bd[2], cd[1])));
  Expansion cy = add(mul(bd[2], cd[0]), neg(mul(bd[0], cd[2])));
  Expansion cz = add(mul(bd[0], cd[1]), neg(mul(bd[1], cd[0])));
  Expansion det = add(add(mul(ad[0], cx), mul(ad[1], cy)), mul(ad[2], cz));
  return sign(det);
}

// sign of det[a-c; b-c] in the plane spanned by axes (i, j)
inline int orient2d(const double* a, const double* b, const double* c, int i, int j) {
  Expansion acx = diff(a[i], c[i]), acy = diff(a[j], c[j]);
  Expansion bcx = diff(b[i], c[i]), bcy = diff(b[j], c[j]);
  return sign(add(mul(acx, bcy), neg(mul(acy, bcx))));
}

// Closed segments p-q and r-s in the plane (i,j): do they share a point?
inline bool segments_meet_2d(const double* p, const double* q, const double* r, const double* s,
                             int i, int j) {
  int o1 = orient2d(p, q, r, i, j), o2 = orient2d(p, q, s, i, j);
  int o3 = orient2d(r, s, p, i, j), o4 = orient2d(r, s, q, i, j);
  if (o1 * o2 < 0 && o3 * o4 < 0) return true;
  auto on = [&](const double* a, const double* b, const double* x) {
    return std::fmin(a[i], b[i]) <= x[i] && x[i] <= std::fmax(a[i], b[i]) &&
           std::fmin(a[j], b[j]) <= x[j] && x[j] <= std::fmax(a[j], b[j]);
  };
  if (o1 == 0 && on(p, q, r)) return true;
  if (o2 == 0 && on(p, q, s)) return true;
  if (o3 == 0 && on(r, s, p)) return true;
  if (o4 == 0 && on(r, s, q)) return true;
  return false;
}

// Does the closed segment p-q meet the closed triangle a,b,c?
inline bool segment_meets_triangle(const double* p, const double* q, const double* a,
                                   const double* b, const double* c) {
  int sp = orient3d(a, b, c, p), sq = orient3d(a, b, c, q);
  if (sp * sq > 0) return false;
  if (sp == 0 && sq == 0) {
    // coplanar: pick a projection plane in which the triangle is not degenerate
    for (int drop = 0; drop < 3; ++drop) {
      int i = (drop + 1) % 3, j = (drop + 2) % 3;
      int o = orient2d(a, b, c, i, j);
      if (o == 0) continue;
      auto inside = [&](const double* x) {
        int s0 = orient2d(a, b, x, i, j), s1 = orient2d(b, c, x, i, j), s2 = orient2d(c, a, x, i, j);
        return s0 * o >= 0 && s1 * o >= 0 && s2 * o >= 0;
      };
      if (inside(p) || inside(q)) return true;
      return segments_meet_2d(p, q, a, b, i, j) || segments_meet_2d(p, q, b, c, i, j) ||
             segments_meet_2d(p, q, c, a, i, j);
    }
    return false;  // degenerate triangle
  }
  // the segment crosses (or touches) the plane: it meets the triangle iff the three
  // orientations of (p, q, edge) do not disagree in sign
  int s0 = orient3d(p, q, a, b), s1 = orient3d(p, q, b, c), s2 = orient3d(p, q, c, a);
  bool has_pos = s0 > 0 || s1 > 0 || s2 > 0;
  bool has_neg = s0 < 0 || s1 < 0 || s2 < 0;
  return !(has_pos && has_neg);
}

}  // namespace orc
