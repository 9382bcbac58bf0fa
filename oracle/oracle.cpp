// Test infrastructure: the CPU oracle of the Embedded-IPC contact stage.
//
// A plain, slow FP64 implementation written straight from the paper (arxiv 2409.16385):
//   * embedding x = phi(q) = J q, x_k = sum_j w^k_j q_{i^j(k)}          (Sec. III-D, Eq. 14)
//   * contact set B: every point-triangle and edge-edge pair with 0 < d_k < dhat,
//     enumerated by brute force over all pairs                            (Sec. III-B)
//   * barrier kappa * b(d_k) with b of Eq. 7; lagged friction
//     D_k = mu lambda_k^n f0(|u_k|) with f0, f1 of Sec. III-B
//   * exact gradient / Hessian by forward-mode AD (ad.hpp), per-pair barrier Hessian
//     projected to the nearest PSD matrix (projected Newton, Sec. III-C) by cyclic Jacobi
//   * reduced gradient / Hessian  grad_q = J^T grad_x,  hess_q = J^T hess_x J   (Eq. 17)
//   * step bound by conservative advancement over every pair whose swept boxes overlap
//     (the CCD clamp of Sec. III-C; x = J q is linear so a reduced step is a straight
//     full-space motion)
//   * exact edge-triangle intersection test (predicates.hpp) for the no-penetration check.
// Only tests, the smoke check and the CPU-baseline leg of the benchmark call this code;
// it shares nothing with the CUDA library.  Compile with -ffp-contract=off.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "ad.hpp"
#include "geometry.hpp"
#include "predicates.hpp"

using namespace orc;

namespace {

// ------------------------------------------------------------------ symmetric eigen / P+
// Cyclic Jacobi: rotate away every off-diagonal entry in turn until the off-diagonal mass
// is below (1e-17 ||A||_F)^2; the diagonal then holds the eigenvalues, V the eigenvectors.
void jacobi_eigen(int n, double* A, double* V, double* lam) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off <= 1e-34 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t;
        if (std::fabs(theta) > 1e150) {
          t = 0.5 / theta;
        } else {
          t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        }
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

// nearest PSD matrix in the Frobenius norm: V max(Lambda, 0) V^T
void psd_project(int n, const double* H, double* out) {
  std::vector<double> A(H, H + n * n), V(n * n), lam(n);
  jacobi_eigen(n, A.data(), V.data(), lam.data());
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int k = 0; k < n; ++k)
        if (lam[k] > 0) s += V[i * n + k] * lam[k] * V[j * n + k];
      out[i * n + j] = s;
    }
}

// ------------------------------------------------------------------ pair stencils
// Pair type 0 = PT (i = vertex, j = triangle), 1 = EE (i < j edge ids).
struct Mesh {
  int64_t nv, nf, ne;
  const double* x;       // [nv,3]
  const int32_t* tris;   // [nf,3]
  const int32_t* edges;  // [ne,2]
  const uint8_t* kin;    // [nv] 1 = kinematic
};

inline void stencil(const Mesh& m, int type, int64_t i, int64_t j, int32_t v[4]) {
  if (type == 0) {
    v[0] = (int32_t)i;
    v[1] = m.tris[3 * j]; v[2] = m.tris[3 * j + 1]; v[3] = m.tris[3 * j + 2];
  } else {
    v[0] = m.edges[2 * i]; v[1] = m.edges[2 * i + 1];
    v[2] = m.edges[2 * j]; v[3] = m.edges[2 * j + 1];
  }
}

inline V3<double> P(const double* x, int32_t v) { return {x[3 * v], x[3 * v + 1], x[3 * v + 2]}; }

double pair_d2(int type, const V3<double> p[4], int* region, double c[4]) {
  if (type == 0) return pt_d2(p[0], p[1], p[2], p[3], region, c);
  return ee_d2(p[0], p[1], p[2], p[3], region, c);
}

AD pair_d2_ad(int type, const double* x4, int* region, double c[4]) {
  V3<AD> p[4];
  for (int a = 0; a < 4; ++a)
    p[a] = {AD::var(x4[3 * a], 3 * a), AD::var(x4[3 * a + 1], 3 * a + 1), AD::var(x4[3 * a + 2], 3 * a + 2)};
  if (type == 0) return pt_d2(p[0], p[1], p[2], p[3], region, c);
  return ee_d2(p[0], p[1], p[2], p[3], region, c);
}

bool incident(int type, const int32_t v[4]) {
  if (type == 0) return v[0] == v[1] || v[0] == v[2] || v[0] == v[3];
  return v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3];
}

bool all_kinematic(const Mesh& m, const int32_t v[4]) {
  return m.kin[v[0]] && m.kin[v[1]] && m.kin[v[2]] && m.kin[v[3]];
}

struct Box {
  double lo[3], hi[3];
};

Box prim_box(const Mesh& m, int type, int64_t i, bool side_a, const double* x) {
  int32_t v[3];
  int nvx;
  if (type == 0 && side_a) { v[0] = (int32_t)i; nvx = 1; }
  else if (type == 0) { v[0] = m.tris[3 * i]; v[1] = m.tris[3 * i + 1]; v[2] = m.tris[3 * i + 2]; nvx = 3; }
  else { v[0] = m.edges[2 * i]; v[1] = m.edges[2 * i + 1]; nvx = 2; }
  Box b;
  for (int k = 0; k < 3; ++k) { b.lo[k] = x[3 * v[0] + k]; b.hi[k] = b.lo[k]; }
  for (int t = 1; t < nvx; ++t)
    for (int k = 0; k < 3; ++k) {
      b.lo[k] = std::min(b.lo[k], x[3 * v[t] + k]);
      b.hi[k] = std::max(b.hi[k], x[3 * v[t] + k]);
    }
  return b;
}

inline bool overlap(const Box& a, const Box& b, double pad) {
  for (int k = 0; k < 3; ++k)
    if (a.lo[k] - pad > b.hi[k] || b.lo[k] - pad > a.hi[k]) return false;
  return true;
}

struct PairRec {
  int32_t type, i, j;
  double d;
  bool operator<(const PairRec& o) const {
    if (type != o.type) return type < o.type;
    if (i != o.i) return i < o.i;
    return j < o.j;
  }
};

// All pairs of B with 0 < d < dhat; returns false if some pair has d <= 0.
// The box test only skips pairs that are certainly farther than dhat apart.
bool enumerate_pairs(const Mesh& m, double dhat, std::vector<PairRec>& out) {
  std::vector<Box> vb(m.nv), fb(m.nf), eb(m.ne);
  for (int64_t v = 0; v < m.nv; ++v) vb[v] = prim_box(m, 0, v, true, m.x);
  for (int64_t f = 0; f < m.nf; ++f) fb[f] = prim_box(m, 0, f, false, m.x);
  for (int64_t e = 0; e < m.ne; ++e) eb[e] = prim_box(m, 1, e, true, m.x);
  const double pad = dhat * (1.0 + 1e-9);
  bool ok = true;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<std::vector<PairRec>> part(nth);
#pragma omp parallel for schedule(dynamic, 64) reduction(&& : ok)
  for (int64_t v = 0; v < m.nv; ++v) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    for (int64_t f = 0; f < m.nf; ++f) {
      if (!overlap(vb[v], fb[f], pad)) continue;
      int32_t s[4];
      stencil(m, 0, v, f, s);
      if (incident(0, s) || all_kinematic(m, s)) continue;
      V3<double> p[4] = {P(m.x, s[0]), P(m.x, s[1]), P(m.x, s[2]), P(m.x, s[3])};
      int reg; double c[4];
      double d = std::sqrt(pair_d2(0, p, &reg, c));
      if (d <= 0.0) ok = false;
      else if (d < dhat) part[tid].push_back({0, (int32_t)v, (int32_t)f, d});
    }
  }
#pragma omp parallel for schedule(dynamic, 64) reduction(&& : ok)
  for (int64_t e = 0; e < m.ne; ++e) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    for (int64_t g = e + 1; g < m.ne; ++g) {
      if (!overlap(eb[e], eb[g], pad)) continue;
      int32_t s[4];
      stencil(m, 1, e, g, s);
      if (incident(1, s) || all_kinematic(m, s)) continue;
      V3<double> p[4] = {P(m.x, s[0]), P(m.x, s[1]), P(m.x, s[2]), P(m.x, s[3])};
      int reg; double c[4];
      double d = std::sqrt(pair_d2(1, p, &reg, c));
      if (d <= 0.0) ok = false;
      else if (d < dhat) part[tid].push_back({1, (int32_t)e, (int32_t)g, d});
    }
  }
  out.clear();
  for (auto& p : part) out.insert(out.end(), p.begin(), p.end());
  std::sort(out.begin(), out.end());
  return ok;
}

// ------------------------------------------------------------------ per-pair potentials
struct Local {
  double E;
  double g[12];
  double H[144];
};

// EE mollifier (the IPC-style variant; the paper applies none): per-edge rest squared
// lengths and the factor of eps_x = factor |e_i^rest|^2 |e_j^rest|^2; factor <= 0 = off.
std::vector<double> g_rest_len2;
double g_moll_factor = 0.0;

// m(c) = -c^2 / eps^2 + 2 c / eps for c = |e_i x e_j|^2 < eps, else 1
template <class T>
T mollifier(const T& c, double eps) {
  if (val(c) >= eps) return T(1.0);
  return c * (T(2.0 / eps) - c * T(1.0 / (eps * eps)));
}

double moll_eps(int type, int64_t i, int64_t j) {
  if (type != 1 || g_moll_factor <= 0.0 || g_rest_len2.empty() || i < 0 || j < 0) return 0.0;
  return g_moll_factor * g_rest_len2[i] * g_rest_len2[j];
}

// kappa m(x) b(d(x)) with exact derivatives (m = 1 unless an EE pair is mollified); H is
// the raw (unprojected) Hessian
void barrier_local(int type, int64_t pi, int64_t pj, const double* x4, double dhat, double kappa, Local& out) {
  int reg; double c[4];
  AD s = pair_d2_ad(type, x4, &reg, c);
  AD d = sqrt(s);
  AD b = barrier(d, dhat);
  const double eps = moll_eps(type, pi, pj);
  if (eps > 0.0) {
    V3<AD> p[4];
    for (int a = 0; a < 4; ++a)
      p[a] = {AD::var(x4[3 * a], 3 * a), AD::var(x4[3 * a + 1], 3 * a + 1), AD::var(x4[3 * a + 2], 3 * a + 2)};
    V3<AD> n = cross(p[1] - p[0], p[3] - p[2]);
    b = mollifier(dot(n, n), eps) * b;
  }
  out.E = kappa * b.v;
  for (int i = 0; i < 12; ++i) out.g[i] = kappa * b.g[i];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) out.H[i * 12 + j] = kappa * b.h[i][j];
}

struct Lag {
  int32_t v[4];
  double gamma[4];
  double n[3];
  double anchor[3];
  double lambda;
};

// lagged friction mu lambda f0(|u|), u the tangential part of sum_a gamma_a (x_a - x_a^n)
void friction_local(const Lag& L, const double* x4, double mu, double eps, Local& out) {
  AD xv[12];
  for (int i = 0; i < 12; ++i) xv[i] = AD::var(x4[i], i);
  AD v[3];
  for (int k = 0; k < 3; ++k) {
    AD s(0.0);
    for (int a = 0; a < 4; ++a)
      if (L.gamma[a] != 0.0) s = s + AD(L.gamma[a]) * xv[3 * a + k];
    v[k] = s - AD(L.anchor[k]);
  }
  AD vn = v[0] * AD(L.n[0]) + v[1] * AD(L.n[1]) + v[2] * AD(L.n[2]);
  AD w[3];
  for (int k = 0; k < 3; ++k) w[k] = v[k] - vn * AD(L.n[k]);
  AD y2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double ml = mu * L.lambda;
  if (y2.v == 0.0) {
    // limit u -> 0: f0 -> eps/3, gradient 0, Hessian (2/eps) mu lambda (gamma gamma^T) (x) (I - n n^T)
    out.E = ml * eps / 3.0;
    for (int i = 0; i < 12; ++i) out.g[i] = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            out.H[(3 * a + k) * 12 + 3 * b + l] =
                ml * (2.0 / eps) * L.gamma[a] * L.gamma[b] * ((k == l ? 1.0 : 0.0) - L.n[k] * L.n[l]);
    return;
  }
  AD y = sqrt(y2);
  AD f = friction_f0(y, eps);
  out.E = ml * f.v;
  for (int i = 0; i < 12; ++i) out.g[i] = ml * f.g[i];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) out.H[i * 12 + j] = ml * f.h[i][j];
}

void gather4(const double* x, const int32_t v[4], double* x4) {
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) x4[3 * a + k] = x[3 * v[a] + k];
}

// ------------------------------------------------------------------ reduced assembly
struct Reduced {
  double E = 0;
  std::vector<double> g;                                   // [ns*3]
  std::map<std::pair<int32_t, int32_t>, std::array<double, 9>> H;
};

// g_r += J^T g_local, H_r += J^T H_local J over the cage nodes of the four vertices
void scatter(const int32_t v[4], const int32_t* idx, const double* w, const Local& L, Reduced& R) {
  for (int a = 0; a < 4; ++a) {
    if (idx[4 * v[a]] < 0) continue;  // kinematic: no reduced DoF
    for (int i = 0; i < 4; ++i) {
      int32_t I = idx[4 * v[a] + i];
      double wa = w[4 * v[a] + i];
      for (int k = 0; k < 3; ++k) R.g[3 * I + k] += wa * L.g[3 * a + k];
      for (int b = 0; b < 4; ++b) {
        if (idx[4 * v[b]] < 0) continue;
        for (int j = 0; j < 4; ++j) {
          int32_t Jn = idx[4 * v[b] + j];
          double wb = w[4 * v[b] + j];
          auto& blk = R.H[{I, Jn}];
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) blk[3 * k + l] += wa * wb * L.H[(3 * a + k) * 12 + 3 * b + l];
        }
      }
    }
  }
}

// ------------------------------------------------------------------ step bound (CCD)
// Conservative advancement for one pair moving linearly by dx over t in [0,1]:
// the common mean displacement is removed; L bounds how fast the distance can shrink
// (largest relative speed on side A plus largest on side B), so advancing t by
// (1 - s) d(t) / L never closes more than (1 - s) d(t).  Stop once d(t) <= s d(0).
double ca_pair(int type, const double* x4, const double* dx4, double s, int max_iter, int* iters,
               bool* capped) {
  double mean[3] = {0, 0, 0};
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) mean[k] += dx4[3 * a + k];
  for (int k = 0; k < 3; ++k) mean[k] /= 4.0;
  double rel[12];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) rel[3 * a + k] = dx4[3 * a + k] - mean[k];
  auto norm3 = [&](int a) {
    return std::sqrt(rel[3 * a] * rel[3 * a] + rel[3 * a + 1] * rel[3 * a + 1] + rel[3 * a + 2] * rel[3 * a + 2]);
  };
  double La, Lb;
  if (type == 0) {
    La = norm3(0);
    Lb = std::max(norm3(1), std::max(norm3(2), norm3(3)));
  } else {
    La = std::max(norm3(0), norm3(1));
    Lb = std::max(norm3(2), norm3(3));
  }
  double L = La + Lb;
  *iters = 0;
  *capped = false;
  if (L == 0.0) return 1.0;
  auto dist = [&](double t) {
    V3<double> p[4];
    for (int a = 0; a < 4; ++a)
      p[a] = {x4[3 * a] + t * rel[3 * a], x4[3 * a + 1] + t * rel[3 * a + 1], x4[3 * a + 2] + t * rel[3 * a + 2]};
    int reg; double c[4];
    return std::sqrt(pair_d2(type, p, &reg, c));
  };
  double d0 = dist(0.0);
  if (d0 <= 0.0) return 0.0;
  double t = 0.0, d = d0;
  while (true) {
    double tn = t + (1.0 - s) * d / L;
    if (tn >= 1.0) return 1.0;
    t = tn;
    d = dist(t);
    ++*iters;
    if (d <= s * d0) return t;
    if (*iters >= max_iter) { *capped = true; return t; }
  }
}

}  // namespace

// ====================================================================== C interface
extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// x_k = sum_j w_kj q_{idx_kj} (Sec. III-D); kinematic rows (idx = -1) copy x_kin
void orc_embed(int64_t nv, const int32_t* idx, const double* w, const double* x_kin,
               const double* q, double* x) {
  for (int64_t v = 0; v < nv; ++v) {
    if (idx[4 * v] < 0) {
      for (int k = 0; k < 3; ++k) x[3 * v + k] = x_kin[3 * v + k];
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int j = 0; j < 4; ++j) s += w[4 * v + j] * q[3 * idx[4 * v + j] + k];
      x[3 * v + k] = s;
    }
  }
}

// squared distance of one PT (type 0) or EE (type 1) stencil, region code and stencil c
double orc_pair_d2(int type, const double* x4, int32_t* region, double* c) {
  V3<double> p[4];
  for (int a = 0; a < 4; ++a) p[a] = {x4[3 * a], x4[3 * a + 1], x4[3 * a + 2]};
  int reg;
  double d2 = pair_d2(type, p, &reg, c);
  *region = reg;
  return d2;
}

// b, b', b'' at d (one-variable AD)
void orc_barrier(double d, double dhat, double* out3) {
  AD x = AD::var(d, 0);
  AD b = barrier(x, dhat);
  out3[0] = b.v; out3[1] = b.g[0]; out3[2] = b.h[0][0];
}

// f0, f0', f0'' at y
void orc_f0(double y, double eps, double* out3) {
  AD x = AD::var(y, 0);
  AD f = friction_f0(x, eps);
  out3[0] = f.v; out3[1] = f.g[0]; out3[2] = f.h[0][0];
}

// local barrier energy, gradient, raw Hessian and projected Hessian of one stencil
void orc_pair_barrier(int type, const double* x4, double dhat, double kappa, double* E,
                      double* g12, double* H144, double* Hp144) {
  Local L;
  barrier_local(type, -1, -1, x4, dhat, kappa, L);
  *E = L.E;
  std::memcpy(g12, L.g, sizeof(L.g));
  std::memcpy(H144, L.H, sizeof(L.H));
  psd_project(12, L.H, Hp144);
}

void orc_psd_project(int n, const double* H, double* out) { psd_project(n, H, out); }

void orc_eigen(int n, const double* H, double* lam, double* V) {
  std::vector<double> A(H, H + n * n);
  jacobi_eigen(n, A.data(), V, lam);
}

// Brute-force contact set B.  Writes up to `cap` pairs ordered by (type, i, j);
// returns the total count, or -1 if some pair has d <= 0 (penetration).
int64_t orc_pairs(int64_t nv, const double* x, const uint8_t* kin, int64_t nf, const int32_t* tris,
                  int64_t ne, const int32_t* edges, double dhat, int64_t cap, int32_t* type,
                  int32_t* pi, int32_t* pj, double* pd) {
  Mesh m{nv, nf, ne, x, tris, edges, kin};
  std::vector<PairRec> out;
  if (!enumerate_pairs(m, dhat, out)) return -1;
  for (int64_t k = 0; k < (int64_t)out.size() && k < cap; ++k) {
    type[k] = out[k].type; pi[k] = out[k].i; pj[k] = out[k].j; pd[k] = out[k].d;
  }
  return (int64_t)out.size();
}

// Candidate pairs of B restricted to given queries (for sampled checks on large scenes):
// PT pairs of vertices vq[0..nq) or EE pairs having edge eq[k] as one side.
int64_t orc_pairs_of(int64_t nv, const double* x, const uint8_t* kin, int64_t nf,
                     const int32_t* tris, int64_t ne, const int32_t* edges, double dhat, int type,
                     int64_t nq, const int32_t* queries, int64_t cap, int32_t* pi, int32_t* pj,
                     double* pd) {
  Mesh m{nv, nf, ne, x, tris, edges, kin};
  std::vector<PairRec> out;
  const double pad = dhat * (1.0 + 1e-9);
  for (int64_t qi = 0; qi < nq; ++qi) {
    int64_t a = queries[qi];
    Box ba = prim_box(m, type, a, true, x);
    int64_t nb = type == 0 ? nf : ne;
    for (int64_t b = 0; b < nb; ++b) {
      if (type == 1 && b == a) continue;
      Box bb = prim_box(m, type, b, type == 1, x);
      if (!overlap(ba, bb, pad)) continue;
      int64_t i = a, j = b;
      if (type == 1 && j < i) std::swap(i, j);
      int32_t s[4];
      stencil(m, type, i, j, s);
      if (incident(type, s) || all_kinematic(m, s)) continue;
      V3<double> p[4] = {P(x, s[0]), P(x, s[1]), P(x, s[2]), P(x, s[3])};
      int reg; double c[4];
      double d = std::sqrt(pair_d2(type, p, &reg, c));
      if (d > 0.0 && d < dhat) out.push_back({type, (int32_t)i, (int32_t)j, d});
    }
  }
  std::sort(out.begin(), out.end());
  for (int64_t k = 0; k < (int64_t)out.size() && k < cap; ++k) {
    pi[k] = out[k].i; pj[k] = out[k].j; pd[k] = out[k].d;
  }
  return (int64_t)out.size();
}

// Lagged friction state at x^n for a pair list (Sec. III-B): lambda = kappa |b'(d)|,
// closest-point stencil gamma, contact normal n and anchor sum_a gamma_a x^n_a.
void orc_friction_lag(int64_t nv, const double* xn, int64_t nf, const int32_t* tris, int64_t ne,
                      const int32_t* edges, int64_t np, const int32_t* type, const int32_t* pi,
                      const int32_t* pj, double dhat, double kappa, int32_t* lv, double* lgamma,
                      double* ln, double* lanchor, double* llambda) {
  Mesh m{nv, nf, ne, xn, tris, edges, nullptr};
  for (int64_t k = 0; k < np; ++k) {
    int32_t s[4];
    stencil(m, type[k], pi[k], pj[k], s);
    V3<double> p[4] = {P(xn, s[0]), P(xn, s[1]), P(xn, s[2]), P(xn, s[3])};
    int reg; double c[4];
    double d = std::sqrt(pair_d2(type[k], p, &reg, c));
    double r[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int q = 0; q < 3; ++q) r[q] += c[a] * xn[3 * s[a] + q];
    double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double bb[3];
    orc_barrier(d, dhat, bb);
    for (int a = 0; a < 4; ++a) { lv[4 * k + a] = s[a]; lgamma[4 * k + a] = c[a]; }
    for (int q = 0; q < 3; ++q) { ln[3 * k + q] = r[q] / rn; lanchor[3 * k + q] = r[q]; }
    // lagged normal force magnitude; a mollified EE pair scales it by m(x^n)
    double mk = 1.0;
    const double eps = moll_eps(type[k], pi[k], pj[k]);
    if (eps > 0.0) {
      V3<double> n = cross(p[1] - p[0], p[3] - p[2]);
      mk = mollifier(dot(n, n), eps);
    }
    llambda[k] = kappa * mk * std::fabs(bb[1]);
  }
}

struct orc_eval_result {
  Reduced R;
  std::vector<double> Ek;   // per barrier pair energy
};

// Contact potential and its reduced derivatives:
//   E   = kappa sum_k b(d_k) + sum_f mu lambda_f f0(|u_f|)
//   g_r = J^T grad_x E,  H_r = J^T (sum_k P+(kappa hess b_k) + sum_f hess D_f) J
orc_eval_result* orc_eval(int64_t nv, const double* x, int64_t nf, const int32_t* tris, int64_t ne,
                          const int32_t* edges, const int32_t* idx, const double* w, int64_t ns,
                          int64_t np, const int32_t* type, const int32_t* pi, const int32_t* pj,
                          int64_t nfr, const int32_t* lv, const double* lgamma, const double* ln,
                          const double* lanchor, const double* llambda, double dhat, double kappa,
                          double mu, double eps, int project) {
  Mesh m{nv, nf, ne, x, tris, edges, nullptr};
  auto* res = new orc_eval_result;
  res->R.g.assign(3 * ns, 0.0);
  res->Ek.assign(np, 0.0);
  std::vector<Local> loc(np);
  std::vector<std::array<int32_t, 4>> st(np);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < np; ++k) {
    stencil(m, type[k], pi[k], pj[k], st[k].data());
    double x4[12];
    gather4(x, st[k].data(), x4);
    Local L;
    barrier_local(type[k], pi[k], pj[k], x4, dhat, kappa, L);
    if (project) {
      double Hp[144];
      psd_project(12, L.H, Hp);
      std::memcpy(L.H, Hp, sizeof(Hp));
    }
    loc[k] = L;
  }
  for (int64_t k = 0; k < np; ++k) {
    res->R.E += loc[k].E;
    res->Ek[k] = loc[k].E;
    scatter(st[k].data(), idx, w, loc[k], res->R);
  }
  if (mu > 0.0) {
    for (int64_t f = 0; f < nfr; ++f) {
      Lag L;
      for (int a = 0; a < 4; ++a) { L.v[a] = lv[4 * f + a]; L.gamma[a] = lgamma[4 * f + a]; }
      for (int q = 0; q < 3; ++q) { L.n[q] = ln[3 * f + q]; L.anchor[q] = lanchor[3 * f + q]; }
      L.lambda = llambda[f];
      double x4[12];
      gather4(x, L.v, x4);
      Local F;
      friction_local(L, x4, mu, eps, F);
      res->R.E += F.E;
      scatter(L.v, idx, w, F, res->R);
    }
  }
  return res;
}

// Hessian-vector product of the contact potential without PSD projection, for a full-space
// direction u (one 3-vector per vertex, kinematic vertices included):
//   y = (sum_k kappa hess b_k + sum_f hess D_f) u
//   out_r = J^T y over the embedded vertices (reduced, [ns*3]);
//   out_kin = sum of y over the kinematic vertices ([3]).
// With u = J v this is H_r v for the unprojected H_r of orc_eval; with u nonzero on the
// kinematic vertices it is the mixed derivative of g_r with respect to their positions.
void orc_hvp(int64_t nv, const double* x, int64_t nf, const int32_t* tris, int64_t ne, const int32_t* edges,
             const int32_t* idx, const double* w, int64_t ns, int64_t np, const int32_t* type, const int32_t* pi,
             const int32_t* pj, int64_t nfr, const int32_t* lv, const double* lgamma, const double* ln,
             const double* lanchor, const double* llambda, double dhat, double kappa, double mu, double eps,
             const double* u, double* out_r, double* out_kin) {
  Mesh m{nv, nf, ne, x, tris, edges, nullptr};
  std::vector<double> y(3 * nv, 0.0);
  auto apply = [&](const int32_t v[4], const Local& L) {
    double u4[12], y4[12];
    gather4(u, v, u4);
    for (int i = 0; i < 12; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 12; ++j) acc += L.H[i * 12 + j] * u4[j];
      y4[i] = acc;
    }
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) y[3 * v[a] + k] += y4[3 * a + k];
  };
  for (int64_t k = 0; k < np; ++k) {
    int32_t v[4];
    stencil(m, type[k], pi[k], pj[k], v);
    double x4[12];
    gather4(x, v, x4);
    Local L;
    barrier_local(type[k], pi[k], pj[k], x4, dhat, kappa, L);
    apply(v, L);
  }
  if (mu > 0.0) {
    for (int64_t f = 0; f < nfr; ++f) {
      Lag L;
      for (int a = 0; a < 4; ++a) { L.v[a] = lv[4 * f + a]; L.gamma[a] = lgamma[4 * f + a]; }
      for (int q = 0; q < 3; ++q) { L.n[q] = ln[3 * f + q]; L.anchor[q] = lanchor[3 * f + q]; }
      L.lambda = llambda[f];
      double x4[12];
      gather4(x, L.v, x4);
      Local F;
      friction_local(L, x4, mu, eps, F);
      apply(L.v, F);
    }
  }
  for (int64_t i = 0; i < 3 * ns; ++i) out_r[i] = 0.0;
  for (int k = 0; k < 3; ++k) out_kin[k] = 0.0;
  for (int64_t a = 0; a < nv; ++a) {
    if (idx[4 * a] < 0) {
      for (int k = 0; k < 3; ++k) out_kin[k] += y[3 * a + k];
      continue;
    }
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 3; ++k) out_r[3 * idx[4 * a + i] + k] += w[4 * a + i] * y[3 * a + k];
  }
}

// Deduplicated contact set, the IPC-style alternative to the paper's literal set B (which
// counts every pair): each pair stands for the pair of mesh features that realises its
// distance -- face and vertex, vertex and edge, two vertices, or two edges in their
// interiors -- and pairs realising the same feature pair count once.  Pairs are visited
// in the given order (callers pass (type, i, j) order); keep[k] = 1 for the first pair of
// each feature pair, 0 for the rest.
void orc_dedup(int64_t nv, const double* x, int64_t nf, const int32_t* tris, int64_t ne, const int32_t* edges,
               int64_t np, const int32_t* type, const int32_t* pi, const int32_t* pj, int32_t* keep) {
  Mesh m{nv, nf, ne, x, tris, edges, nullptr};
  std::map<std::pair<int32_t, int32_t>, int32_t> edge_of;
  for (int64_t e = 0; e < ne; ++e)
    edge_of[{std::min(edges[2 * e], edges[2 * e + 1]), std::max(edges[2 * e], edges[2 * e + 1])}] = (int32_t)e;
  auto edge_id = [&](int32_t a, int32_t b) {
    auto it = edge_of.find({std::min(a, b), std::max(a, b)});
    return it == edge_of.end() ? -1 : it->second;
  };
  std::map<std::array<int64_t, 3>, int64_t> seen;
  for (int64_t k = 0; k < np; ++k) {
    int32_t v[4];
    stencil(m, type[k], pi[k], pj[k], v);
    V3<double> p[4];
    for (int a = 0; a < 4; ++a) p[a] = P(x, v[a]);
    int reg; double c[4];
    pair_d2(type[k], p, &reg, c);
    std::array<int64_t, 3> key;
    if (type[k] == 0) {
      if (reg == PT_FACE) {
        key = {0, pj[k], pi[k]};                                  // face, vertex
      } else if (reg <= 3) {
        const int e = reg - 1;                                    // edge (t_e, t_e+1)
        key = {1, pi[k], edge_id(v[1 + e], v[1 + (e + 1) % 3])};
      } else {
        const int32_t t = v[1 + (reg - 4)];                       // vertex t_(reg-4)
        key = {2, std::min(v[0], t), std::max(v[0], t)};
      }
    } else {
      if (reg == 0) {
        key = {3, pi[k], pj[k]};                                  // two edge interiors
      } else if (reg <= 4) {
        const int e = reg - 1;                                    // endpoint e against the other edge
        key = e < 2 ? std::array<int64_t, 3>{1, v[e], pj[k]} : std::array<int64_t, 3>{1, v[e], pi[k]};
      } else {
        const int ia = (reg - 5) / 2, ib = (reg - 5) % 2;          // endpoint against endpoint
        key = {2, std::min(v[ia], v[2 + ib]), std::max(v[ia], v[2 + ib])};
      }
    }
    keep[k] = seen.emplace(key, k).second ? 1 : 0;
  }
}

// EE mollifier: rest squared lengths of the ne edges and the factor of eps_x (<= 0: off)
void orc_set_mollifier(int64_t ne, const double* rest_len2, double factor) {
  g_rest_len2.assign(rest_len2, rest_len2 + (factor > 0.0 ? ne : 0));
  g_moll_factor = factor;
}

// one mollified EE stencil with eps_x given: energy, gradient, raw Hessian (for pins)
void orc_pair_barrier_mollified(const double* x4, double eps, double dhat, double kappa, double* E, double* g12,
                                double* H144) {
  const std::vector<double> keep = g_rest_len2;
  const double keep_f = g_moll_factor;
  g_rest_len2.assign(2, 1.0);
  g_moll_factor = eps;
  Local L;
  barrier_local(1, 0, 1, x4, dhat, kappa, L);
  g_rest_len2 = keep;
  g_moll_factor = keep_f;
  *E = L.E;
  std::memcpy(g12, L.g, sizeof(L.g));
  std::memcpy(H144, L.H, sizeof(L.H));
}

int64_t orc_result_nnzb(const orc_eval_result* r) { return (int64_t)r->R.H.size(); }

void orc_result_copy(const orc_eval_result* r, double* E, double* g, int32_t* I, int32_t* J,
                     double* vals, double* Ek) {
  *E = r->R.E;
  std::memcpy(g, r->R.g.data(), r->R.g.size() * sizeof(double));
  int64_t k = 0;
  for (const auto& kv : r->R.H) {
    I[k] = kv.first.first;
    J[k] = kv.first.second;
    std::memcpy(vals + 9 * k, kv.second.data(), 9 * sizeof(double));
    ++k;
  }
  if (Ek) std::memcpy(Ek, r->Ek.data(), r->Ek.size() * sizeof(double));
}

void orc_result_free(orc_eval_result* r) { delete r; }

// Local friction potential of one stencil (for pins)
void orc_pair_friction(const int32_t* v4, const double* gamma4, const double* n3,
                       const double* anchor3, double lambda, const double* x4, double mu,
                       double eps, double* E, double* g12, double* H144) {
  Lag L;
  for (int a = 0; a < 4; ++a) { L.v[a] = v4[a]; L.gamma[a] = gamma4[a]; }
  for (int q = 0; q < 3; ++q) { L.n[q] = n3[q]; L.anchor[q] = anchor3[q]; }
  L.lambda = lambda;
  Local F;
  friction_local(L, x4, mu, eps, F);
  *E = F.E;
  std::memcpy(g12, F.g, sizeof(F.g));
  std::memcpy(H144, F.H, sizeof(F.H));
}

// Conservative-advancement time of impact of one stencil (for pins)
double orc_ca_pair(int type, const double* x4, const double* dx4, double s, int max_iter,
                   int32_t* iters, int32_t* capped) {
  int it; bool cap;
  double t = ca_pair(type, x4, dx4, s, max_iter, &it, &cap);
  *iters = it; *capped = cap ? 1 : 0;
  return t;
}

// Step bound alpha = min(1, min_k t_k) over every PT / EE pair (not incident, not all
// kinematic) whose closed swept boxes over [x, x + dx] overlap.
double orc_accd(int64_t nv, const double* x, const double* dx, const uint8_t* kin, int64_t nf,
                const int32_t* tris, int64_t ne, const int32_t* edges, double s, int max_iter,
                int64_t* n_candidates, int64_t* total_iters, int32_t* any_capped) {
  std::vector<double> x1(3 * nv);
  for (int64_t i = 0; i < 3 * nv; ++i) x1[i] = x[i] + dx[i];
  Mesh m0{nv, nf, ne, x, tris, edges, kin};
  Mesh m1{nv, nf, ne, x1.data(), tris, edges, kin};
  auto swept = [&](int type, int64_t i, bool side_a) {
    Box a = prim_box(m0, type, i, side_a, x), b = prim_box(m1, type, i, side_a, x1.data());
    for (int k = 0; k < 3; ++k) { a.lo[k] = std::min(a.lo[k], b.lo[k]); a.hi[k] = std::max(a.hi[k], b.hi[k]); }
    return a;
  };
  std::vector<Box> vb(nv), fb(nf), eb(ne);
  for (int64_t v = 0; v < nv; ++v) vb[v] = swept(0, v, true);
  for (int64_t f = 0; f < nf; ++f) fb[f] = swept(0, f, false);
  for (int64_t e = 0; e < ne; ++e) eb[e] = swept(1, e, true);
  double alpha = 1.0;
  int64_t ncand = 0, iters = 0;
  int capped = 0;
  auto run = [&](int type, int64_t i, int64_t j, double& a, int64_t& nc, int64_t& it, int& cp) {
    int32_t st[4];
    stencil(m0, type, i, j, st);
    if (incident(type, st) || all_kinematic(m0, st)) return;
    double x4[12], dx4[12];
    gather4(x, st, x4);
    gather4(dx, st, dx4);
    int n; bool c;
    double t = ca_pair(type, x4, dx4, s, max_iter, &n, &c);
    ++nc; it += n; if (c) cp = 1;
    if (t < a) a = t;
  };
#pragma omp parallel for schedule(dynamic, 64) reduction(min : alpha) reduction(+ : ncand, iters) reduction(| : capped)
  for (int64_t v = 0; v < nv; ++v)
    for (int64_t f = 0; f < nf; ++f)
      if (overlap(vb[v], fb[f], 0.0)) run(0, v, f, alpha, ncand, iters, capped);
#pragma omp parallel for schedule(dynamic, 64) reduction(min : alpha) reduction(+ : ncand, iters) reduction(| : capped)
  for (int64_t e = 0; e < ne; ++e)
    for (int64_t g = e + 1; g < ne; ++g)
      if (overlap(eb[e], eb[g], 0.0)) run(1, e, g, alpha, ncand, iters, capped);
  if (n_candidates) *n_candidates = ncand;
  if (total_iters) *total_iters = iters;
  if (any_capped) *any_capped = capped;
  return alpha;
}

// Step bound restricted to the pairs that have one of the given query primitives as a
// side (type 0: query vertices against all triangles; type 1: query edges against all
// other edges) -- a bounded sample of orc_accd's work.
double orc_accd_of(int64_t nv, const double* x, const double* dx, const uint8_t* kin, int64_t nf,
                   const int32_t* tris, int64_t ne, const int32_t* edges, double s, int max_iter, int type,
                   int64_t nq, const int32_t* queries, int64_t* n_candidates, int64_t* total_iters) {
  std::vector<double> x1(3 * nv);
  for (int64_t i = 0; i < 3 * nv; ++i) x1[i] = x[i] + dx[i];
  Mesh m0{nv, nf, ne, x, tris, edges, kin};
  Mesh m1{nv, nf, ne, x1.data(), tris, edges, kin};
  auto swept = [&](int t, int64_t i, bool side_a) {
    Box a = prim_box(m0, t, i, side_a, x), b = prim_box(m1, t, i, side_a, x1.data());
    for (int k = 0; k < 3; ++k) { a.lo[k] = std::min(a.lo[k], b.lo[k]); a.hi[k] = std::max(a.hi[k], b.hi[k]); }
    return a;
  };
  int64_t nb = type == 0 ? nf : ne;
  std::vector<Box> other(nb);
  for (int64_t b = 0; b < nb; ++b) other[b] = swept(type, b, type == 1);
  double alpha = 1.0;
  int64_t ncand = 0, iters = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(min : alpha) reduction(+ : ncand, iters)
  for (int64_t qi = 0; qi < nq; ++qi) {
    int64_t a = queries[qi];
    Box ba = swept(type, a, true);
    for (int64_t b = 0; b < nb; ++b) {
      if (type == 1 && b == a) continue;
      if (!overlap(ba, other[b], 0.0)) continue;
      int64_t i = a, j = b;
      if (type == 1 && j < i) std::swap(i, j);
      int32_t st[4];
      stencil(m0, type, i, j, st);
      if (incident(type, st) || all_kinematic(m0, st)) continue;
      double x4[12], dx4[12];
      gather4(x, st, x4);
      gather4(dx, st, dx4);
      int n; bool c;
      double t = ca_pair(type, x4, dx4, s, max_iter, &n, &c);
      ++ncand; iters += n;
      if (t < alpha) alpha = t;
    }
  }
  if (n_candidates) *n_candidates = ncand;
  if (total_iters) *total_iters = iters;
  return alpha;
}

// Step bound over a given candidate list (the CPU-baseline stage timing feeds the same
// candidates the GPU found); returns alpha and accumulates iterations.
double orc_accd_list(int64_t nc, const int32_t* type, const int32_t* pi, const int32_t* pj,
                     int64_t nv, const double* x, const double* dx, int64_t nf, const int32_t* tris,
                     int64_t ne, const int32_t* edges, double s, int max_iter, int64_t* total_iters) {
  Mesh m{nv, nf, ne, x, tris, edges, nullptr};
  double alpha = 1.0;
  int64_t iters = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(min : alpha) reduction(+ : iters)
  for (int64_t k = 0; k < nc; ++k) {
    int32_t st[4];
    stencil(m, type[k], pi[k], pj[k], st);
    double x4[12], dx4[12];
    gather4(x, st, x4);
    gather4(dx, st, dx4);
    int n; bool c;
    double t = ca_pair(type[k], x4, dx4, s, max_iter, &n, &c);
    iters += n;
    if (t < alpha) alpha = t;
  }
  if (total_iters) *total_iters = iters;
  return alpha;
}

// 1 if no edge meets a non-incident triangle and no PT / EE pair is at distance 0.
int orc_intersection_free(int64_t nv, const double* x, int64_t nf, const int32_t* tris, int64_t ne,
                          const int32_t* edges) {
  std::vector<uint8_t> nokin(nv, 0);
  Mesh m{nv, nf, ne, x, tris, edges, nokin.data()};
  std::vector<Box> fb(nf), eb(ne);
  for (int64_t f = 0; f < nf; ++f) fb[f] = prim_box(m, 0, f, false, x);
  for (int64_t e = 0; e < ne; ++e) eb[e] = prim_box(m, 1, e, true, x);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t e = 0; e < ne; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    for (int64_t f = 0; f < nf; ++f) {
      if (!overlap(eb[e], fb[f], 0.0)) continue;
      const int32_t* t = tris + 3 * f;
      if (a == t[0] || a == t[1] || a == t[2] || b == t[0] || b == t[1] || b == t[2]) continue;
      if (segment_meets_triangle(x + 3 * a, x + 3 * b, x + 3 * t[0], x + 3 * t[1], x + 3 * t[2]))
        bad = 1;
    }
  }
  return bad ? 0 : 1;
}

}  // extern "C"
