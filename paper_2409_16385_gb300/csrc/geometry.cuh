// Device-side unsigned distance of point-triangle (PT) and edge-edge (EE) stencils
// (Sec. III-B, d_k(x)) with the closest-feature stencil needed by the closed-form
// derivatives.
//
// A stencil's squared distance is a partial minimum s(x) = min_beta |r(x, beta)|^2 with
// r = sum_a c_a(beta) x_a affine in beta (beta: barycentric / segment parameters of the
// closest feature).  For each region we report
//   c[4]      the coefficients at the minimiser (r = sum c_a x_a),
//   m         the number of free parameters of that feature (0, 1 or 2),
//   a[j][4]   dc/dbeta_j (constant per region),
// from which eval.cu builds the exact gradient and Hessian of s by the Schur complement of
// the inner minimisation.  Region choice: PT -- projection inside the triangle, else the
// nearest of the three edges (t0t1, t1t2, t2t0); EE -- unconstrained segment-parameter
// minimiser inside [0,1]^2 (and the segments not parallel to within 1e-20 relative),
// else the nearest of (a0, seg b), (a1, seg b), (b0, seg a), (b1, seg a); ties keep the
// first in that order.
#pragma once
#include "common.cuh"

namespace eipc {

struct Stencil {
  double c[4];
  double a[2][4];
  int m;
  double d2;
};

// |p - (e0 + t (e1 - e0))|^2 over t in [0,1].  t = clamp((w.e) / (e.e), 0, 1), with the
// division taken only inside (0, 1): w.e <= 0 gives 0 and w.e >= e.e gives 1, the values the
// correctly rounded quotient clamps to (also for e = 0 and NaN).
__device__ __forceinline__ double seg_point_d2(V3 p, V3 e0, V3 e1, double* t_out) {
  V3 e = e1 - e0, w = p - e0;
  const double we = dot(w, e), ee = dot(e, e);
  double t;
  if (!(we > 0.0)) t = 0.0;
  else if (we >= ee) t = 1.0;
  else t = we / ee;
  V3 r = w - e * t;
  *t_out = t;
  return dot(r, r);
}

__device__ __forceinline__ void set_zero(Stencil& S) {
#pragma unroll
  for (int k = 0; k < 4; ++k) { S.c[k] = 0.0; S.a[0][k] = 0.0; S.a[1][k] = 0.0; }
}

// closest feature on segment (ia, ib) at parameter t, seen from a fixed point slot `ip`
// with sign +1 (point on side A) -- used for PT edges and EE endpoint cases
__device__ __forceinline__ void point_segment_stencil(Stencil& S, int ip, double sp, int ia, int ib,
                                                      double t) {
  set_zero(S);
  S.c[ip] = sp;
  if (t <= 0.0) {
    S.c[ia] = -sp; S.m = 0;
  } else if (t >= 1.0) {
    S.c[ib] = -sp; S.m = 0;
  } else {
    S.c[ia] = -sp * (1.0 - t);
    S.c[ib] = -sp * t;
    S.a[0][ia] = sp;
    S.a[0][ib] = -sp;
    S.m = 1;
  }
}

template <bool kStencil>
__device__ __forceinline__ double pt_distance(V3 p, V3 t0, V3 t1, V3 t2, Stencil* S) {
  V3 e1 = t1 - t0, e2 = t2 - t0, w = p - t0;
  V3 n = cross(e1, e2);
  double nn = dot(n, n);
  // barycentric coordinates of the projection: beta1 = ((w x e2) . n)/nn, etc., with one
  // reciprocal of nn for the three quotients (nn = 0 gives infinite or NaN barycentrics,
  // which fail the face test, as the quotients would)
  const double inv_nn = 1.0 / nn;
  double b1 = dot(cross(w, e2), n) * inv_nn;
  double b2 = dot(cross(e1, w), n) * inv_nn;
  if (b1 >= 0.0 && b2 >= 0.0 && b1 + b2 <= 1.0) {
    double h = dot(w, n);
    double d2 = h * h * inv_nn;
    if (kStencil) {
      set_zero(*S);
      S->c[0] = 1.0; S->c[1] = -(1.0 - b1 - b2); S->c[2] = -b1; S->c[3] = -b2;
      S->a[0][1] = 1.0; S->a[0][2] = -1.0;
      S->a[1][1] = 1.0; S->a[1][3] = -1.0;
      S->m = 2;
      S->d2 = d2;
    }
    return d2;
  }
  double ta, tb, tc;
  double da = seg_point_d2(p, t0, t1, &ta);
  double db = seg_point_d2(p, t1, t2, &tb);
  double dc = seg_point_d2(p, t2, t0, &tc);
  int k = 0;
  double best = da, tbest = ta;
  if (db < best) { best = db; tbest = tb; k = 1; }
  if (dc < best) { best = dc; tbest = tc; k = 2; }
  if (kStencil) {
    point_segment_stencil(*S, 0, 1.0, 1 + k, 1 + (k + 1) % 3, tbest);
    S->d2 = best;
  }
  return best;
}

template <bool kStencil>
__device__ __forceinline__ double ee_distance(V3 a0, V3 a1, V3 b0, V3 b1, Stencil* S) {
  V3 ea = a1 - a0, eb = b1 - b0, w = a0 - b0;
  double A = dot(ea, ea), B = dot(ea, eb), C = dot(eb, eb);
  double D = dot(ea, w), E = dot(eb, w);
  V3 n = cross(ea, eb);
  double nn = dot(n, n);
  if (nn > 1e-20 * A * C) {
    const double inv_nn = 1.0 / nn;
    double s = (B * E - C * D) * inv_nn;
    double t = (A * E - B * D) * inv_nn;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      double h = dot(w, n);
      double d2 = h * h * inv_nn;
      if (kStencil) {
        set_zero(*S);
        S->c[0] = 1.0 - s; S->c[1] = s; S->c[2] = -(1.0 - t); S->c[3] = -t;
        S->a[0][0] = -1.0; S->a[0][1] = 1.0;
        S->a[1][2] = 1.0; S->a[1][3] = -1.0;
        S->m = 2;
        S->d2 = d2;
      }
      return d2;
    }
  }
  double t0, t1, t2, t3;
  double d0 = seg_point_d2(a0, b0, b1, &t0);
  double d1 = seg_point_d2(a1, b0, b1, &t1);
  double d2 = seg_point_d2(b0, a0, a1, &t2);
  double d3 = seg_point_d2(b1, a0, a1, &t3);
  int k = 0;
  double best = d0, tb = t0;
  if (d1 < best) { best = d1; tb = t1; k = 1; }
  if (d2 < best) { best = d2; tb = t2; k = 2; }
  if (d3 < best) { best = d3; tb = t3; k = 3; }
  if (kStencil) {
    if (k < 2) point_segment_stencil(*S, k, 1.0, 2, 3, tb);      // a_k - point on b
    else point_segment_stencil(*S, k, -1.0, 0, 1, tb);          // point on a - b_{k-2}
    S->d2 = best;
  }
  return best;
}

// ---------------------------------------------------------------- FP32 screen
// "Certainly farther than r" tests in FP32 only (62x the FP64 rate on GB300), on FP32 copies
// of the positions.  With M the largest coordinate of the candidate's points, each FP32
// coordinate is off by <= M 2^-24 and the FP32 distance by a small multiple of that (taken
// as 40 M 2^-24).  The callers prove far with a radius grown by twice that, 80 M 2^-24, and
// declare a pair far only if its FP32 squared distance also exceeds r^2 (1 + 4e-3), i.e.
// d > r (1 + 2e-3): the margin holds at any scene size.  Misclassifying the closest
// region can only (a) report a lower bound (plane / line distance when the projection is
// wrongly found inside), or (b) report a boundary value whose excess is bounded by the
// curvature times the squared parameter error.  Stencils whose parameter solve is not
// well conditioned (|n|^2 <= 0.1 |e1|^2 |e2|^2) are screened by a bound that needs no
// parameter solve: edges within 18 degrees of parallel by their segment-to-line distances
// (seg_line_far_f32); skinny triangles not at all.  Every pair not screened goes through
// the exact FP64 test, so the kept set is unchanged.
struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 load_xf(const float* __restrict__ x4f, int32_t v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(x4f) + v);
  return {a.x, a.y, a.z};
}
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(F3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float fdot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 fcross(F3 a, F3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// |w - t e|^2 over t in [0,1] (w relative to the segment start)
__device__ __forceinline__ float fseg_d2(F3 w, F3 e) {
  float t = fdot(w, e) / fdot(e, e);
  t = fminf(fmaxf(t, 0.f), 1.f);
  const F3 r = w - e * t;
  return fdot(r, r);
}

__device__ __forceinline__ bool pt_far_f32(F3 p, F3 t0, F3 t1, F3 t2, float r2m) {
  const F3 e1 = t1 - t0, e2 = t2 - t0, w = p - t0;
  const F3 n = fcross(e1, e2);
  const float nn = fdot(n, n);
  if (!(nn > 0.1f * fdot(e1, e1) * fdot(e2, e2))) return false;
  const float b1 = fdot(fcross(w, e2), n) / nn;
  const float b2 = fdot(fcross(e1, w), n) / nn;
  float d2;
  if (b1 >= 0.f && b2 >= 0.f && b1 + b2 <= 1.f) {
    const float h = fdot(w, n);
    d2 = h * h / nn;
  } else {
    d2 = fminf(fseg_d2(w, e1), fminf(fseg_d2(w - e1, e2 - e1), fseg_d2(w, e2)));
  }
  return d2 > r2m;
}

// Segment-to-line lower bound for near-parallel edges: with U = (segment start - line
// point) x e_line and V = e_seg x e_line, the squared distance from the point at parameter
// s of the segment to the line is |U + s V|^2 / L (L = |e_line|^2).  Its minimum over
// s in [0, 1] is |U|^2 (U.V >= 0), |U + V|^2 (U.V <= -|V|^2), else |U x V|^2 / |V|^2
// (Lagrange's identity, free of the cancellation in |U|^2 - (U.V)^2 / |V|^2).  A case
// chosen wrongly through rounding of U.V overestimates by at most (err U.V)^2 / |V|^2,
// of order eps^2 |U|^2: negligible against the margin.  The segments' distance is at least
// this (the other segment lies on the line), so "far" here proves the pair far.  The
// interior case needs |V|^2 > 1e-12 |e_seg|^2 L (edges not parallel to within 1e-6 rad),
// else nothing is proven.
__device__ __forceinline__ bool seg_line_far_f32(F3 U, F3 V, float Lseg, float L, float r2m) {
  const float uv = fdot(U, V), vv = fdot(V, V);
  float g;
  if (uv >= 0.f) {
    g = fdot(U, U);
  } else if (uv <= -vv) {
    const F3 W = {U.x + V.x, U.y + V.y, U.z + V.z};
    g = fdot(W, W);
  } else {
    if (!(vv > 1e-12f * Lseg * L)) return false;
    const F3 X = fcross(U, V);
    g = fdot(X, X) / vv;
  }
  return g > r2m * L;
}

__device__ __forceinline__ bool ee_far_f32(F3 a0, F3 a1, F3 b0, F3 b1, float r2m) {
  const F3 ea = a1 - a0, eb = b1 - b0, w = a0 - b0;
  const float A = fdot(ea, ea), C = fdot(eb, eb);
  const F3 n = fcross(ea, eb);
  const float nn = fdot(n, n);
  if (!(nn > 0.1f * A * C)) {
    // near-parallel: segment a against line b, segment b against line a
    const F3 wb = b0 - a0;
    return seg_line_far_f32(fcross(w, eb), n, A, C, r2m) || seg_line_far_f32(fcross(wb, ea), n * -1.f, C, A, r2m);
  }
  const float B = fdot(ea, eb), D = fdot(ea, w), E = fdot(eb, w);
  const float s = (B * E - C * D) / nn, t = (A * E - B * D) / nn;
  float d2;
  if (s >= 0.f && s <= 1.f && t >= 0.f && t <= 1.f) {
    const float h = fdot(w, n);
    d2 = h * h / nn;
  } else {
    d2 = fminf(fminf(fseg_d2(w, eb), fseg_d2(a1 - b0, eb)), fminf(fseg_d2(b0 - a0, ea), fseg_d2(b1 - a0, ea)));
  }
  return d2 > r2m;
}

}  // namespace eipc
