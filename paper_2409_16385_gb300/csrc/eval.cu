// Per-pair contact potentials and their reduction into the subspace.
//
// Barrier (Eq. 7): E_k = kappa b(d), b = -(d - dhat)^2 log(d / dhat).
// With s = d^2 the partial minimum min_beta |r(x,beta)|^2 (geometry.cuh):
//   grad s   = 2 c (x) r
//   hess s   = 2 (c c^T) (x) I3 - G M^-1 G^T,  G_j = 2 (c (x) v_j + a_j (x) r),
//              v_j = sum_a a_j[a] x_a, M = 2 [v_j . v_l]
// (Schur complement of the inner minimisation), so
//   hess E = kappa [(b'' - b'/d) (c c^T) (x) (r^ r^T) + (b'/d) (c c^T) (x) I3]
//            - (kappa b' / (2d)) G M^-1 G^T.
// Every term lies in the span of {c^ (x) e_x, c^ (x) e_y, c^ (x) e_z, a^_1 (x) r^, a^_2 (x) r^}
// (a^_j: a_j orthonormalised against c), an orthonormal basis Q of at most 5 columns.  The
// 12x12 Hessian is Q K Q^T with K (<= 5x5) in closed form; its projection onto the PSD cone
// (projected Newton, Sec. III-C) is Q K+ Q^T with K+ from a 5x5 Jacobi eigensolve -- the
// same matrix as projecting the 12x12 itself, because P+ acts on eigenpairs and the
// complement of span(Q) is the zero eigenspace.
//
// Reduction (Eq. 17): g_r = J^T g, H_r = J^T H J.  J restricted to a stencil maps the
// stencil's unique cage nodes I to the 4 vertices with weights w_aI, so Q's columns map to
// per-node scalars omega_I = sum_a c^_a w_aI, alpha_jI = sum_a a^_j[a] w_aI, and
//   block(I, J) = A_I K+ A_J^T,   A_I = [omega_I I3 | alpha_1I r^ | alpha_2I r^]  (3x5).
// Friction (Sec. III-B, lagged): D = mu lambda f0(|u|), u = (I - n n^T)(sum gamma_a x_a - anchor),
//   grad = mu lambda f1(y)/y gamma (x) u,   hess = (gamma gamma^T) (x) F,
//   F = mu lambda [(f1/y)(I - n n^T) + (f1' - f1/y) u^ u^T]   (PSD as written).
// Records (key = I * Ns + J, 3x3 block): the keys depend only on each item's cage nodes, so
// they are written and stably sorted before the evaluation, which then writes every block to
// its sorted position; each key's records are summed in a fixed order that depends only on
// that key's own records (32-record units, then a fixed warp tree), so the result is bitwise
// repeatable and the same for a scene alone or inside a batch.
#include "geometry.cuh"
#include "scene.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

constexpr int kMaxNodes = 16;
constexpr int kEvalThreads = 128;

// Key of the upper block (I, J), I <= J < ns: its row-major position in the upper triangle,
// I ns - I (I - 1) / 2 + (J - I).  Ordered like (I, J), and below ns (ns + 1) / 2, so the
// record sort covers fewer bits than with I ns + J (24 instead of 25 for 5,664 nodes).
__host__ __device__ __forceinline__ uint64_t upper_key(uint64_t I, uint64_t J, uint64_t ns) {
  return I * ns - I * (I - 1) / 2 + (J - I);
}

// (I, J) of an upper key: I is the last row whose first key is at most the key; an FP64
// estimate from the quadratic, then exact integer correction
__device__ __forceinline__ void upper_decode(uint64_t key, uint64_t ns, uint64_t* I, uint64_t* J) {
  const double b = 2.0 * (double)ns + 1.0;
  double r = 0.5 * (b - sqrt(fmax(b * b - 8.0 * (double)key, 0.0)));
  int64_t i = (int64_t)r;
  if (i < 0) i = 0;
  if (i > (int64_t)ns - 1) i = (int64_t)ns - 1;
  while (i > 0 && upper_key((uint64_t)i, (uint64_t)i, ns) > key) --i;
  while (i + 1 < (int64_t)ns && upper_key((uint64_t)(i + 1), (uint64_t)(i + 1), ns) <= key) ++i;
  *I = (uint64_t)i;
  *J = key - upper_key((uint64_t)i, (uint64_t)i, ns) + (uint64_t)i;
}

// stencil vertex ids of pair (type, i, j)
__device__ __forceinline__ void stencil_vertices(const Topo& T, int type, int32_t i, int32_t j, int32_t v[4]) {
  if (type == 0) {
    v[0] = i;
    v[1] = T.tris[3 * (int64_t)j]; v[2] = T.tris[3 * (int64_t)j + 1]; v[3] = T.tris[3 * (int64_t)j + 2];
  } else {
    v[0] = T.edges[2 * (int64_t)i]; v[1] = T.edges[2 * (int64_t)i + 1];
    v[2] = T.edges[2 * (int64_t)j]; v[3] = T.edges[2 * (int64_t)j + 1];
  }
}

// item k < P: barrier pair k; P <= k < P + L: friction pair k - P
__device__ __forceinline__ bool item_vertices(const Topo& T, const eipc_pairs& pr, int64_t P, const int32_t* lag_v,
                                              int64_t L, int64_t k, int32_t v[4]) {
  if (k < P) {
    stencil_vertices(T, pr.type[k], pr.i[k], pr.j[k], v);
    return true;
  }
  if (k < P + L) {
    const int4 q = reinterpret_cast<const int4*>(lag_v)[k - P];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    return true;
  }
  return false;
}

// Friction merged into contact pairs with the same stencil: for pair k,
// fric_of_pair[k] = INT32_MAX - f when lagged friction item f takes k's records (0: none);
// pair_of_fric[f] = that pair + 1 (0: none).  The claim holds only if both agree.
// friction item f rides on pair kp's records (both arrays as in EvalArgs)
__device__ __forceinline__ bool friction_merged(const int32_t* __restrict__ fric_of_pair,
                                                const int32_t* __restrict__ pair_of_fric, int64_t f) {
  if (!pair_of_fric) return false;
  const int32_t kp = pair_of_fric[f] - 1;
  return kp >= 0 && fric_of_pair[kp] == INT32_MAX - (int32_t)f;
}

// (type, i, j) of a pair as one ordered 64-bit key (i, j < 2^31)
__device__ __forceinline__ uint64_t lag_pair_key(int type, int32_t i, int32_t j) {
  return ((uint64_t)(type & 1) << 62) | ((uint64_t)(uint32_t)i << 31) | (uint64_t)(uint32_t)j;
}

// first pair position k in [0, P) with (type[k], i[k]) >= (type, i) (the pair list is in
// (type, i, j) order)
__device__ __forceinline__ int64_t pair_lower_bound(const eipc_pairs& pr, int64_t P, int type, int32_t i) {
  int64_t lo = 0, hi = P;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int t = pr.type[mid];
    if (t < type || (t == type && pr.i[mid] < i)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Friction items that ride on a contact pair: lagged item f and pair k share their records
// when their stencils have the same four vertices in the same order (then the same cage
// nodes in the same order, so the same record keys).  The candidates are the PT pairs of
// vertex v0 and the EE pairs of edge (v0, v1).  When several items find the same pair (a
// lag list with repeated stencils), the lowest f wins; the others keep their own records.
__global__ void __launch_bounds__(kBlock) k_fric_match(Topo T, eipc_pairs pr, eipc_lag lag, int64_t item_cap,
                                                       const uint64_t* __restrict__ ekey,
                                                       const int32_t* __restrict__ eid,
                                                       const uint64_t* __restrict__ lag_key,
                                                       int32_t* __restrict__ fric_of_pair,
                                                       int32_t* __restrict__ pair_of_fric) {
  pdl_entry();
  int64_t P = clamp_count(pr.count, pr.capacity);
  if (P > item_cap) P = item_cap;
  int64_t L = clamp_count(lag.count, lag.capacity);
  if (P + L > item_cap) L = item_cap - P;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < L; f += grid_stride()) {
    const int4 q = reinterpret_cast<const int4*>(lag.v)[f];
    int64_t found = -1;
    if (lag_key) {
      // the item's own pair key (type, i, j), recorded when the scene built this lag state:
      // one search in the pair list's order, then the same check of the four vertices
      const uint64_t key = lag_key[f];
      int64_t lo = 0, hi = P;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (lag_pair_key(pr.type[mid], pr.i[mid], pr.j[mid]) < key) lo = mid + 1;
        else hi = mid;
      }
      if (lo < P && lag_pair_key(pr.type[lo], pr.i[lo], pr.j[lo]) == key) {
        int32_t v[4];
        stencil_vertices(T, pr.type[lo], pr.i[lo], pr.j[lo], v);
        if (v[0] == q.x && v[1] == q.y && v[2] == q.z && v[3] == q.w) found = lo;
      }
      pair_of_fric[f] = (int32_t)(found + 1);
      if (found >= 0) atomicMax(fric_of_pair + found, INT32_MAX - (int32_t)f);
      continue;
    }
    for (int64_t k = pair_lower_bound(pr, P, 0, q.x); k < P && found < 0; ++k) {
      if (pr.type[k] != 0 || pr.i[k] != q.x) break;
      const int64_t j = pr.j[k];
      if (T.tris[3 * j] == q.y && T.tris[3 * j + 1] == q.z && T.tris[3 * j + 2] == q.w) found = k;
    }
    if (found < 0) {
      const int32_t e = edge_id_of(q.x, q.y, T.nv, ekey, eid, T.ne);
      if (e >= 0 && T.edges[2 * (int64_t)e] == q.x) {
        for (int64_t k = pair_lower_bound(pr, P, 1, e); k < P && found < 0; ++k) {
          if (pr.type[k] != 1 || pr.i[k] != e) break;
          const int64_t j = pr.j[k];
          if (T.edges[2 * j] == q.z && T.edges[2 * j + 1] == q.w) found = k;
        }
      }
    }
    pair_of_fric[f] = (int32_t)(found + 1);
    if (found >= 0) atomicMax(fric_of_pair + found, INT32_MAX - (int32_t)f);
  }
}

// unique cage nodes of each item (kinematic vertices carry none), record counts
__global__ void __launch_bounds__(kBlock) k_item_nodes(Topo T, eipc_pairs pr, const int32_t* lag_v,
                                                       const int64_t* lag_count, int64_t lag_cap,
                                                       const int32_t* __restrict__ cage_idx, int64_t item_cap,
                                                       int32_t* __restrict__ item_nodes, int32_t* __restrict__ item_n,
                                                       int32_t* __restrict__ item_group, const int32_t* __restrict__ vgroup,
                                                       int64_t* __restrict__ rc_h, int64_t* __restrict__ rc_g,
                                                       int64_t* n_items, DevStatus* st,
                                                       const int32_t* __restrict__ fric_of_pair,
                                                       const int32_t* __restrict__ pair_of_fric) {
  pdl_entry();
  const int64_t P = clamp_count(pr.count, pr.capacity);
  const int64_t L = lag_v ? clamp_count(lag_count, lag_cap) : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t n = P + L;
    if (n > item_cap) {
      raise_flag(st, EIPC_FLAG_REC_OVERFLOW);
      n = item_cap;
    }
    *n_items = n;
  }
  const int64_t n = (P + L) < item_cap ? (P + L) : item_cap;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    int32_t v[4];
    item_vertices(T, pr, P, lag_v, L, k, v);
    item_group[k] = vgroup[v[0]];
    if (k >= P && friction_merged(fric_of_pair, pair_of_fric, k - P)) {
      item_n[k] = 0;               // evaluated in its contact pair's records
      rc_h[k] = 0;
      rc_g[k] = 0;
      continue;
    }
    int32_t nodes[kMaxNodes];
    int cnt = 0;
    for (int a = 0; a < 4; ++a) {
      const int4 id = __ldg(reinterpret_cast<const int4*>(cage_idx) + v[a]);
      if (id.x < 0) continue;
      const int32_t ids[4] = {id.x, id.y, id.z, id.w};
      for (int s = 0; s < 4; ++s) {
        bool seen = false;
        for (int u = 0; u < cnt; ++u) seen |= (nodes[u] == ids[s]);
        if (!seen) nodes[cnt++] = ids[s];
      }
    }
    for (int u = 0; u < cnt; ++u) item_nodes[kMaxNodes * k + u] = nodes[u];
    item_n[k] = cnt;
    rc_h[k] = (int64_t)cnt * (cnt + 1) / 2;
    rc_g[k] = cnt;
  }
}

// per-node weights of a stencil basis: out[u] = sum over (a, slot) with idx == node_u of
// coef[a] * w[a][slot]
__device__ __forceinline__ void node_weights(const int32_t v[4], const int32_t* __restrict__ cage_idx,
                                             const double* __restrict__ w, const int32_t* nodes, int n,
                                             const double coef[3][4], int ncoef, double out[kMaxNodes][3]) {
  for (int u = 0; u < n; ++u)
    for (int c = 0; c < 3; ++c) out[u][c] = 0.0;
  for (int a = 0; a < 4; ++a) {
    const int4 id = __ldg(reinterpret_cast<const int4*>(cage_idx) + v[a]);
    if (id.x < 0) continue;
    const int ids[4] = {id.x, id.y, id.z, id.w};
    const double2 w01 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a]);
    const double2 w23 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a] + 1);
    const double ws[4] = {w01.x, w01.y, w23.x, w23.y};
    for (int s = 0; s < 4; ++s) {
      int u = 0;
      while (u < n - 1 && nodes[u] != ids[s]) ++u;
      for (int c = 0; c < ncoef; ++c) out[u][c] += coef[c][a] * ws[s];
    }
  }
}

// node_weights for NC (3 or 4) coefficient sets into rows of four: the barrier's c^, a^_1,
// a^_2 and, with NC = 4, the lagged friction's gamma, in one pass over the stencil's cage
// slots
template <int NC>
__device__ __forceinline__ void node_weights4(const int32_t v[4], const int32_t* __restrict__ cage_idx,
                                              const double* __restrict__ w, const int32_t* nodes, int n,
                                              const double coef[4][4], double out[kMaxNodes][4]) {
  for (int u = 0; u < n; ++u)
    for (int c = 0; c < NC; ++c) out[u][c] = 0.0;
  for (int a = 0; a < 4; ++a) {
    const int4 id = __ldg(reinterpret_cast<const int4*>(cage_idx) + v[a]);
    if (id.x < 0) continue;
    const int ids[4] = {id.x, id.y, id.z, id.w};
    const double2 w01 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a]);
    const double2 w23 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a] + 1);
    const double ws[4] = {w01.x, w01.y, w23.x, w23.y};
    for (int s = 0; s < 4; ++s) {
      int u = 0;
      while (u < n - 1 && nodes[u] != ids[s]) ++u;
#pragma unroll
      for (int c = 0; c < NC; ++c) out[u][c] += coef[c][a] * ws[s];
    }
  }
}

// node_weights for one coefficient set: out[u] = sum over (a, slot) with idx == node_u of
// coef[a] * w[a][slot]
__device__ __forceinline__ void node_weights1(const int32_t v[4], const int32_t* __restrict__ cage_idx,
                                              const double* __restrict__ w, const int32_t* nodes, int n,
                                              const double coef[4], double out[kMaxNodes]) {
  for (int u = 0; u < n; ++u) out[u] = 0.0;
  for (int a = 0; a < 4; ++a) {
    const int4 id = __ldg(reinterpret_cast<const int4*>(cage_idx) + v[a]);
    if (id.x < 0) continue;
    const int ids[4] = {id.x, id.y, id.z, id.w};
    const double2 w01 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a]);
    const double2 w23 = __ldg(reinterpret_cast<const double2*>(w) + 2 * (int64_t)v[a] + 1);
    const double ws[4] = {w01.x, w01.y, w23.x, w23.y};
    for (int s = 0; s < 4; ++s) {
      int u = 0;
      while (u < n - 1 && nodes[u] != ids[s]) ++u;
      out[u] += coef[a] * ws[s];
    }
  }
}

// One Jacobi rotation J (c, s = t c in rows/columns p, q) of the symmetric A held in full,
// A <- J^T A J, and V <- V J.  The entries outside rows and columns p, q are unchanged; the
// (p, q) block takes the closed form of the rotation that zeroes a_pq (a_pp - t a_pq,
// a_qq + t a_pq, 0), so each pair of mirrored entries is computed once.
template <class T, int N>
__device__ __forceinline__ void rotate_sym(T A[N][N], T V[N][N], int p, int q, T c, T s, T t, T apq) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k == p || k == q) continue;
    const T akp = A[k][p], akq = A[k][q];
    const T np = c * akp - s * akq, nq = s * akp + c * akq;
    A[k][p] = np; A[p][k] = np;
    A[k][q] = nq; A[q][k] = nq;
  }
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = T(0);
  A[q][p] = T(0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const T vkp = V[k][p], vkq = V[k][q];
    V[k][p] = c * vkp - s * vkq;
    V[k][q] = s * vkp + c * vkq;
  }
}

// Sweep orders of the Jacobi solvers: rounds of two rotations in disjoint planes covering
// every index pair once (a round-robin schedule: 5 rounds for N = 5, 3 for N = 4).  The
// rotations of a round commute, so their order inside the round does not matter.
__device__ constexpr int kRound5[5][2][2] = {{{1, 4}, {2, 3}}, {{0, 4}, {1, 2}}, {{0, 3}, {2, 4}},
                                             {{0, 2}, {1, 3}}, {{0, 1}, {3, 4}}};
__device__ constexpr int kRound4[3][2][2] = {{{0, 1}, {2, 3}}, {{0, 2}, {1, 3}}, {{0, 3}, {1, 2}}};
template <int N>
__device__ __forceinline__ int round_entry(int r, int h, int w) {
  return N == 5 ? kRound5[r][h][w] : kRound4[r][h][w];
}
template <int N>
constexpr int kRounds = N == 5 ? 5 : 3;

// FP32 rotation angle zeroing a_pq: t = tan, c = cos, s = sin; false when a_pq is negligible
__device__ __forceinline__ bool angle_f32(float app, float aqq, float apq, float* t, float* c, float* s) {
  if (!(fabsf(apq) > 1e-30f)) return false;
  const float theta = (aqq - app) / (2.f * apq);
  const float at = fabsf(theta);
  float tt = at > 1e18f ? 0.5f / at : 1.f / (at + sqrtf(at * at + 1.f));
  tt = theta < 0.f ? -tt : tt;
  *t = tt;
  *c = 1.f / sqrtf(tt * tt + 1.f);
  *s = tt * *c;
  return true;
}

// Fixed number of Jacobi sweeps in FP32 (62x the FP64 rate on this part): a cheap
// approximate eigenbasis V of the symmetric N x N matrix A (scaled to unit norm beforehand).
template <int N>
__device__ __forceinline__ void jacobi_f32(float A[N][N], float V[N][N], int sweeps) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) V[i][j] = (i == j) ? 1.f : 0.f;
  for (int sweep = 0; sweep < sweeps; ++sweep) {
#pragma unroll
    for (int r = 0; r < kRounds<N>; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = round_entry<N>(r, h, 0), q = round_entry<N>(r, h, 1);
        const float apq = A[p][q];
        float t, c, sn;
        if (angle_f32(A[p][p], A[q][q], apq, &t, &c, &sn)) rotate_sym<float, N>(A, V, p, q, c, sn, t, apq);
      }
  }
}

// FP64 rotation angle zeroing a_pq (t, c), false when a_pq is exactly zero.  The zero test
// and the small-angle test read the exponent fields with integer instructions, keeping them
// off the FP64 pipe.
__device__ __forceinline__ bool angle_f64(double app, double aqq, double apq, double* t_out, double* c_out) {
  const int hi_a = __double2hiint(apq);
  if (((hi_a & 0x7fffffff) | __double2loint(apq)) == 0) return false;
  const double gap = aqq - app;
  const int ea = (hi_a >> 20) & 0x7ff, eg = (__double2hiint(gap) >> 20) & 0x7ff;
  double t, c;
  if (eg - ea >= 21 && eg > 1023 - 120 && eg < 1023 + 120) {
    // small angle, |apq| < 2^-20 |gap| (the usual case after the FP32
    // pre-diagonalisation): t = apq / gap to relative O(t^2) <= 2^-40, with 1/gap to FP32
    // precision (the exponent range check keeps gap a normal float).  Any t gives an exact
    // rotation (c = 1 - t^2 / 2 and s = t c are orthonormal to O(t^4)); the approximate t
    // leaves an off-diagonal residual of about 2^-24 |apq|, far below the sweep's stopping
    // threshold
    t = apq * (double)__frcp_rn((float)gap);
    c = 1.0 - 0.5 * t * t;
  } else {
    const double theta = gap / (2.0 * apq);
    const double at = fabs(theta);
    t = at > 1e150 ? 0.5 / at : 1.0 / (at + sqrt(at * at + 1.0));
    t = theta < 0.0 ? -t : t;
    c = rsqrt(t * t + 1.0);
  }
  *t_out = t;
  *c_out = c;
  return true;
}

// Jacobi on the symmetric N x N A held in registers, from the basis V the caller has
// already rotated A into; A becomes diagonal (eigenvalues), V accumulates the rotations
// (columns = eigenvectors).
template <int N>
__device__ __forceinline__ void jacobi(double A[N][N], double V[N][N]) {
  double fro = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) fro += A[i][j] * A[i][j];
  // stop once the off-diagonal norm is below 1e-13 of the matrix norm
  const double tol = 1e-26 * fro;
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = 0.0;
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) off += A[p][q] * A[p][q];
    if (off <= tol) break;
#pragma unroll
    for (int r = 0; r < kRounds<N>; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = round_entry<N>(r, h, 0), q = round_entry<N>(r, h, 1);
        const double apq = A[p][q];
        double t, c;
        if (angle_f64(A[p][p], A[q][q], apq, &t, &c)) rotate_sym<double, N>(A, V, p, q, c, t * c, t, apq);
      }
  }
}

struct EvalArgs {
  Topo T;
  eipc_pairs pr;
  const int32_t* cage_idx;
  const double* w;
  const double* x4;
  int64_t ns;
  double dhat, kappa;
  const int32_t* item_nodes;
  const int32_t* item_n;
  const int64_t* ro_h;
  const int64_t* ro_g;
  const int64_t* n_items;
  int64_t rec_cap, gcap;
  uint64_t* hkeys;
  uint32_t* hvals;
  double* hrec;
  uint64_t* gkeys;
  uint32_t* gvals;
  double* grec;
  double* item_E;
  DevStatus* st;
  bool project;            // PSD-project the barrier Hessians (projected Newton)
  const uint32_t* order;   // processing order of the barrier items (null: index order)
  const double* moll_r2;   // EE mollifier: rest squared edge lengths (null: off)
  double moll_factor;      // eps_x = moll_factor |e_i|^2 |e_j|^2
  int64_t* queue;          // next unclaimed position of `order` (work queue)
  int tile;                // items a warp claims from the queue at a time (multiple of 32)
  const double* hv_dir;    // Hessian-vector product: reduced direction [ns*3]
  double kin_dir[3];       // ... and the rigid direction of the kinematic vertices
  // Presorted Hessian records (energy/gradient/Hessian evaluation): the keys were written
  // and sorted before the evaluation, and record r goes to its sorted position hinv[r]
  // without a key.  Gradient records (Hessian-vector products only) are written at r with
  // their key.
  const uint32_t* hinv;
  // friction merged into contact pairs (friction_merged; null: no merging); lag, mu and
  // eps_f are the friction parameters
  const int32_t* fric_of_pair;
  const int32_t* pair_of_fric;
  eipc_lag lag;
  double mu, eps_f;
};

// Lagged friction of item f at the current positions (Sec. III-B, Eq. 8-9): energy
// mu lambda f0(|u|), the gradient scale mu lambda f1(y)/y along u, the symmetric 3 x 3
// F = mu lambda (f1(y)/y (I - n n^T) + (f1'(y) - f1(y)/y) u u^T / y^2), and the per-node
// weights of gamma for the item's cage nodes.
struct FrictionTerms {
  double E, gs;
  double u[3];
  double F[3][3];
};

__device__ __forceinline__ void friction_terms(const double* __restrict__ x4, const eipc_lag& lag, int64_t f,
                                               const int32_t v[4], double mu, double eps, FrictionTerms& R,
                                               double gam[4]) {
  for (int a = 0; a < 4; ++a) gam[a] = lag.gamma[4 * f + a];
  const V3 nrm = {lag.n[3 * f], lag.n[3 * f + 1], lag.n[3 * f + 2]};
  const V3 anc = {lag.anchor[3 * f], lag.anchor[3 * f + 1], lag.anchor[3 * f + 2]};
  const double ml = mu * lag.lambda[f];
  V3 vs = {0.0, 0.0, 0.0};
  for (int a = 0; a < 4; ++a) vs = vs + load_x(x4, v[a]) * gam[a];
  vs = vs - anc;
  const V3 u = vs - nrm * dot(nrm, vs);
  const double y2 = dot(u, u);
  // f0(y), f1(y)/y and (f1'(y) - f1(y)/y) / y^2, with one division for 1/eps (or 1/y)
  // and one for 1/y^2
  double f0, f1y, c2;
  if (y2 == 0.0) {
    f0 = eps / 3.0; f1y = 2.0 / eps; c2 = 0.0;
  } else {
    const double y = sqrt(y2);
    double f1p_minus;
    if (y < eps) {
      const double ie = 1.0 / eps, yie2 = y * ie * ie;
      f0 = y2 * (ie - yie2 / 3.0) + eps / 3.0;    // -y^3 / (3 eps^2) + y^2 / eps + eps / 3
      f1y = 2.0 * ie - yie2;
      f1p_minus = -yie2;                          // (2/eps - 2y/eps^2) - (2/eps - y/eps^2)
    } else {
      const double iy = 1.0 / y;
      f0 = y; f1y = iy; f1p_minus = -iy;
    }
    c2 = f1p_minus / y2;
  }
  R.E = ml * f0;
  R.gs = ml * f1y;
  R.u[0] = u.x; R.u[1] = u.y; R.u[2] = u.z;
  const double nn[3] = {nrm.x, nrm.y, nrm.z};
  for (int p = 0; p < 3; ++p)
    for (int q = p; q < 3; ++q) {
      const double s = ml * (f1y * ((p == q ? 1.0 : 0.0) - nn[p] * nn[q]) + c2 * R.u[p] * R.u[q]);
      R.F[p][q] = s;
      R.F[q][p] = s;
    }
}

// Eigen-decomposition of the symmetric N x N K (N = 5, or 4 when the span has four
// dimensions): an FP32 Jacobi pre-diagonalisation of K/|K|, its eigenvectors
// re-orthonormalised in FP64 (modified Gram-Schmidt), K rotated into that basis in FP64,
// then FP64 Jacobi sweeps to full precision (quadratic convergence from the ~1e-7 residual
// leaves one or two sweeps).  On return K is diagonal, V its eigenvectors.
template <int N>
__device__ __forceinline__ void eigen_sym(double K[N][N], double V[N][N]) {
  double fro = 0.0;
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int q = 0; q < N; ++q) fro += K[p][q] * K[p][q];
  if (fro == 0.0) {
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = 0; q < N; ++q) V[p][q] = (p == q) ? 1.0 : 0.0;
    return;
  }
  // 1/|K| only scales the FP32 stage: FP32 precision is enough when |K|^2 is a normal float
  const double inv = (fro > 1e-36 && fro < 1e36) ? (double)rsqrtf((float)fro) : rsqrt(fro);
  float Af[N][N], Vf[N][N];
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int q = 0; q < N; ++q) Af[p][q] = (float)(K[p][q] * inv);
  jacobi_f32<N>(Af, Vf, 4);
  // FP64 orthonormal basis from the FP32 eigenvectors (columns)
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int p = 0; p < N; ++p) V[p][j] = (double)Vf[p][j];
#pragma unroll
    for (int i = 0; i < j; ++i) {
      double pr = 0.0;
#pragma unroll
      for (int p = 0; p < N; ++p) pr += V[p][i] * V[p][j];
#pragma unroll
      for (int p = 0; p < N; ++p) V[p][j] -= pr * V[p][i];
    }
    double nn = 0.0;
#pragma unroll
    for (int p = 0; p < N; ++p) nn += V[p][j] * V[p][j];
    // the FP32 eigenvectors are orthonormal to FP32 precision, so |nn - 1| is about 1e-7:
    // two Newton steps for 1/sqrt(nn) from 1 leave an error of order (nn - 1)^4
    double r = 1.5 - 0.5 * nn;
    r = r * (1.5 - 0.5 * nn * r * r);
#pragma unroll
    for (int p = 0; p < N; ++p) V[p][j] *= r;
  }
  // K <- V^T K V
  double T[N][N];
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < N; ++q) s += K[p][q] * V[q][j];
      T[p][j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int p = 0; p < N; ++p) s += V[p][i] * T[p][j];
      K[i][j] = s;
      K[j][i] = s;
    }
  jacobi<N>(K, V);
}

// K+ = (V max(Lambda, 0)) V^T of the leading N x N block of the 5 x 5 K (rows and columns
// beyond N are zero in K and in K+)
template <int N>
__device__ __forceinline__ void psd_span_inl(const double K[5][5], double Kp[5][5]) {
  double Kn[N][N], V[N][N];
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int q = 0; q < N; ++q) Kn[p][q] = K[p][q];
  eigen_sym<N>(Kn, V);
  double W[N][N];
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const double le = Kn[e][e] > 0.0 ? Kn[e][e] : 0.0;
#pragma unroll
    for (int p = 0; p < N; ++p) W[p][e] = V[p][e] * le;
  }
#pragma unroll
  for (int p = 0; p < 5; ++p)
#pragma unroll
    for (int q = p; q < 5; ++q) {
      double s = 0.0;
      if (p < N && q < N) {
#pragma unroll
        for (int e = 0; e < N; ++e) s += W[p][e] * V[q][e];
      }
      Kp[p][q] = s;
      Kp[q][p] = s;
    }
}

// The 4 x 4 projection (99 % of the pairs of the benchmark workloads) is inlined; the
// 5 x 5 one, for pairs with two free closest-point parameters, is a separate function, so
// its larger register footprint (the 5 x 5 eigensolver's matrices) does not set the
// register allocation of the common path: under a register cap only the rare call spills.
__device__ __noinline__ void psd_span5(const double K[5][5], double Kp[5][5]) { psd_span_inl<5>(K, Kp); }
__device__ __forceinline__ void psd_span4(const double K[5][5], double Kp[5][5]) { psd_span_inl<4>(K, Kp); }

// one upper-triangle record: key (min, max) of the two cage nodes, block transposed when
// the first node is the larger one.  With presorted records the sorted position is
// hinv[pos]; a caller that has already loaded it passes it as `pre` (else pass -1).
__device__ __forceinline__ void emit_upper(const EvalArgs& A, int64_t pos, int32_t Iu, int32_t Iv,
                                           const double B[3][3], int64_t pre = -1) {
  const bool swap = Iu > Iv;
  int64_t dst = pos;
  if (A.hinv) {
    dst = pre >= 0 ? pre : (int64_t)A.hinv[pos];
  } else {
    A.hkeys[pos] = swap ? upper_key((uint64_t)Iv, (uint64_t)Iu, (uint64_t)A.ns)
                        : upper_key((uint64_t)Iu, (uint64_t)Iv, (uint64_t)A.ns);
    A.hvals[pos] = (uint32_t)pos;
  }
  double v[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) v[3 * a + b] = swap ? B[b][a] : B[a][b];
  double2* p = reinterpret_cast<double2*>(A.hrec + kHRecStride * dst);
#pragma unroll
  for (int c = 0; c < 4; ++c) p[c] = make_double2(v[2 * c], v[2 * c + 1]);
  A.hrec[kHRecStride * dst + 8] = v[8];
}

// The diagonal record (I, I) of a presorted item: the block is symmetric, so its six
// upper entries B00 B01 B02 B11 B12 B22 take the first six values of the row and the item's
// gradient at node I the next three.  The segment sums of the diagonal records are then
// the reduced Hessian's diagonal blocks and g_r together, with no gradient records, sort or
// reduction of their own.
__device__ __forceinline__ void emit_diag(const EvalArgs& A, int64_t pos, const double B[3][3], double g0, double g1,
                                          double g2, int64_t pre = -1) {
  const int64_t dst = pre >= 0 ? pre : (int64_t)A.hinv[pos];
  double2* p = reinterpret_cast<double2*>(A.hrec + kHRecStride * dst);
  p[0] = make_double2(B[0][0], B[0][1]);
  p[1] = make_double2(B[0][2], B[1][1]);
  p[2] = make_double2(B[1][2], B[2][2]);
  p[3] = make_double2(g0, g1);
  A.hrec[kHRecStride * dst + 8] = g2;
}

// one keyed gradient record (Hessian-vector products)
__device__ __forceinline__ void emit_grad(const EvalArgs& A, int64_t pos, uint64_t key, double y0, double y1, double y2) {
  A.gkeys[pos] = key;
  A.gvals[pos] = (uint32_t)pos;
  *reinterpret_cast<double2*>(A.grec + kGRecStride * pos) = make_double2(y0, y1);
  A.grec[kGRecStride * pos + 2] = y2;
}

// The barrier Hessian of one active pair in its span (Sec. III-B, Eq. 7; the 12 x 12
// Hessian of kappa b(d(x)) lies in the span of c^ (x) e_xyz and a^_j (x) r^): the
// orthonormal 4-vectors basis[0] = c^, basis[1..2] = a^_1, a^_2, the unit direction r^
// between the closest points, and the 5 x 5 matrix K of the Hessian in that basis,
// unprojected and symmetric.  Also the energy kappa b(d) and b'(d).
struct BarrierSpan {
  double E, b1, cn;
  V3 rh;
  double basis[3][4];
  double K[5][5];
};

__device__ __forceinline__ void barrier_span(const V3 Y[4], const Stencil& S, double d, double dhat, double kappa,
                                             BarrierSpan& B) {
  const double lg = log(d / dhat);
  const double m = d - dhat;
  const double inv_d = 1.0 / d;
  const double md = m * inv_d;
  const double b = -m * m * lg;
  const double b1 = -2.0 * m * lg - m * md;
  const double b2 = -2.0 * lg - 4.0 * md + md * md;
  B.E = kappa * b;
  B.b1 = b1;
  // r and r^
  V3 r = {0.0, 0.0, 0.0};
  for (int a = 0; a < 4; ++a) r = r + Y[a] * S.c[a];
  B.rh = r * rsqrt(dot(r, r));
  const V3 rh = B.rh;
  // orthonormal 4-vectors c^, a^_1, a^_2
  const double cc = S.c[0] * S.c[0] + S.c[1] * S.c[1] + S.c[2] * S.c[2] + S.c[3] * S.c[3];
  const double inv_cn = rsqrt(cc);
  const double cn = cc * inv_cn;
  B.cn = cn;
  for (int a = 0; a < 4; ++a) B.basis[0][a] = S.c[a] * inv_cn;
  for (int j = 0; j < 2; ++j) {
    if (j < S.m) {
      double t[4];
      for (int a = 0; a < 4; ++a) t[a] = S.a[j][a];
      for (int i = 0; i <= j; ++i) {
        double pr = 0.0;
        for (int a = 0; a < 4; ++a) pr += B.basis[i][a] * t[a];
        for (int a = 0; a < 4; ++a) t[a] -= pr * B.basis[i][a];
      }
      const double inv_tn = rsqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
      for (int a = 0; a < 4; ++a) B.basis[1 + j][a] = t[a] * inv_tn;
    } else {
      for (int a = 0; a < 4; ++a) B.basis[1 + j][a] = 0.0;
    }
  }
  // v_j, M = 2 [v_j . v_l], g_j = Q^T G_j
  V3 vj[2];
  for (int j = 0; j < 2; ++j) {
    vj[j] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) vj[j] = vj[j] + Y[a] * S.a[j][a];
  }
  double (&K)[5][5] = B.K;
  const double kb = kappa * cn * cn;
  const double rr = kappa * (b2 - b1 * inv_d);
  const double kd = kb * b1 * inv_d;
  const double rhv[3] = {rh.x, rh.y, rh.z};
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) K[p][q] = cn * cn * (rr * rhv[p] * rhv[q]) + (p == q ? kd : 0.0);
  for (int p = 0; p < 5; ++p)
    for (int q = 3; q < 5; ++q) { K[p][q] = 0.0; K[q][p] = 0.0; }
  if (S.m > 0) {
    double g[2][5];
    for (int j = 0; j < S.m; ++j) {
      double ca = 0.0;
      for (int a = 0; a < 4; ++a) ca += B.basis[0][a] * S.a[j][a];
      const double vv[3] = {vj[j].x, vj[j].y, vj[j].z};
      for (int p = 0; p < 3; ++p) g[j][p] = 2.0 * cn * vv[p] + 2.0 * d * ca * rhv[p];
      for (int l = 0; l < 2; ++l) {
        double al = 0.0;
        for (int a = 0; a < 4; ++a) al += B.basis[1 + l][a] * S.a[j][a];
        g[j][3 + l] = 2.0 * d * al;
      }
    }
    double Mi[2][2];
    if (S.m == 1) {
      Mi[0][0] = 0.5 / dot(vj[0], vj[0]);
    } else {
      const double m00 = 2.0 * dot(vj[0], vj[0]), m01 = 2.0 * dot(vj[0], vj[1]), m11 = 2.0 * dot(vj[1], vj[1]);
      const double inv_det = 1.0 / (m00 * m11 - m01 * m01);
      Mi[0][0] = m11 * inv_det; Mi[1][1] = m00 * inv_det; Mi[0][1] = Mi[1][0] = -m01 * inv_det;
    }
    const double beta = -0.5 * kappa * b1 * inv_d;
    for (int p = 0; p < 5; ++p)
      for (int q = 0; q < 5; ++q) {
        double s2 = 0.0;
        for (int j = 0; j < S.m; ++j)
          for (int l = 0; l < S.m; ++l) s2 += g[j][p] * Mi[j][l] * g[l][q];
        K[p][q] += beta * s2;
      }
  }
  // symmetrise against rounding
  for (int p = 0; p < 5; ++p)
    for (int q = p + 1; q < 5; ++q) { const double t = 0.5 * (K[p][q] + K[q][p]); K[p][q] = t; K[q][p] = t; }
}

// ------------------------------------------------------------------ EE mollifier
// IPC-style variant (the paper applies none): an edge-edge pair whose edges are nearly
// parallel, c = |e_i x e_j|^2 < eps_x = factor |e_i^rest|^2 |e_j^rest|^2, carries
// kappa m(c) b(d) with m(c) = c (2 / eps - c / eps^2), which is C1 at c = eps and vanishes
// as the edges become parallel.  Its Hessian leaves the 5-dimensional span, so these rare
// pairs take a full 12 x 12 path (exact Hessian; Jacobi projection for projected Newton).

__device__ __forceinline__ bool ee_mollified(const EvalArgs& A, int type, int32_t i, int32_t j, const V3 Y[4],
                                             double* eps, double* c) {
  if (type != 1 || !A.moll_r2) return false;
  const V3 nn = cross(Y[1] - Y[0], Y[3] - Y[2]);
  *c = dot(nn, nn);
  *eps = A.moll_factor * A.moll_r2[i] * A.moll_r2[j];
  return *c < *eps;
}

// energy, gradient and exact Hessian (node-major 3a + k) of kappa m(c(x)) b(d(x))
__device__ __noinline__ void mollified_local(const V3* Y, const Stencil& S, double d, double dhat, double kappa,
                                             double eps, double c, double* E, double* g, double* H) {
  BarrierSpan B;
  barrier_span(Y, S, d, dhat, kappa, B);
  const double rhv[3] = {B.rh.x, B.rh.y, B.rh.z};
  double Q[12][5];
#pragma unroll 1
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) {
      for (int p = 0; p < 3; ++p) Q[3 * a + k][p] = (k == p) ? B.basis[0][a] : 0.0;
      Q[3 * a + k][3] = B.basis[1][a] * rhv[k];
      Q[3 * a + k][4] = B.basis[2][a] * rhv[k];
    }
  double QK[12][5];
#pragma unroll 1
  for (int r = 0; r < 12; ++r)
    for (int p = 0; p < 5; ++p) {
      double acc = 0.0;
      for (int q = 0; q < 5; ++q) acc += Q[r][q] * B.K[q][p];
      QK[r][p] = acc;
    }
  // kappa grad b = kappa b' c_a r^ (c_a = |c| basis0_a)
  double gb[12];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) gb[3 * a + k] = kappa * B.b1 * B.cn * B.basis[0][a] * rhv[k];
  // c = |e0 x e1|^2: gradient and Hessian blocks in (e0, e1)
  const V3 e0 = Y[1] - Y[0], e1 = Y[3] - Y[2];
  const double s00 = dot(e0, e0), s11 = dot(e1, e1), s01 = dot(e0, e1);
  const double E0[3] = {e0.x, e0.y, e0.z}, E1[3] = {e1.x, e1.y, e1.z};
  double ge[2][3];
  for (int k = 0; k < 3; ++k) {
    ge[0][k] = 2.0 * (s11 * E0[k] - s01 * E1[k]);
    ge[1][k] = 2.0 * (s00 * E1[k] - s01 * E0[k]);
  }
  double gc[12];
  for (int k = 0; k < 3; ++k) {
    gc[k] = -ge[0][k]; gc[3 + k] = ge[0][k]; gc[6 + k] = -ge[1][k]; gc[9 + k] = ge[1][k];
  }
  const double m = c * (2.0 / eps - c / (eps * eps));
  const double m1 = 2.0 / eps - 2.0 * c / (eps * eps);
  const double m2 = -2.0 / (eps * eps);
  const double kb = B.E;                 // kappa b
  *E = m * kb;
  for (int r = 0; r < 12; ++r) g[r] = m * gb[r] + kb * m1 * gc[r];
  // the e-blocks of the Hessian of c
  auto hc = [&](int ea, int eb, int k, int l) -> double {
    const double dl = (k == l) ? 1.0 : 0.0;
    if (ea == 0 && eb == 0) return 2.0 * (s11 * dl - E1[k] * E1[l]);
    if (ea == 1 && eb == 1) return 2.0 * (s00 * dl - E0[k] * E0[l]);
    if (ea == 0) return 4.0 * E0[k] * E1[l] - 2.0 * E1[k] * E0[l] - 2.0 * s01 * dl;
    return 4.0 * E1[k] * E0[l] - 2.0 * E0[k] * E1[l] - 2.0 * s01 * dl;
  };
  const int edge_of[4] = {0, 0, 1, 1};
  const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
#pragma unroll 1
  for (int r = 0; r < 12; ++r) {
    const int a = r / 3, k = r % 3;
    for (int q = 0; q < 12; ++q) {
      const int b2 = q / 3, l = q % 3;
      double hb = 0.0;
      for (int p = 0; p < 5; ++p) hb += QK[r][p] * Q[q][p];
      const double hcv = sgn[a] * sgn[b2] * hc(edge_of[a], edge_of[b2], k, l);
      H[12 * r + q] = m * hb + kb * (m2 * gc[r] * gc[q] + m1 * hcv) + m1 * (gb[r] * gc[q] + gc[r] * gb[q]);
    }
  }
  for (int r = 0; r < 12; ++r)
    for (int q = r + 1; q < 12; ++q) {
      const double t = 0.5 * (H[12 * r + q] + H[12 * q + r]);
      H[12 * r + q] = t; H[12 * q + r] = t;
    }
}

// cyclic Jacobi on an N x N symmetric matrix in memory, then A <- V max(Lambda, 0) V^T
__device__ __noinline__ void psd_project_mem(double* A, int N) {
  double V[144];
  for (int i = 0; i < N * N; ++i) V[i] = (i / N == i % N) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < N * N; ++i) fro += A[i] * A[i];
  const double tol = 1e-28 * fro;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) off += A[p * N + q] * A[p * N + q];
    if (off <= tol) break;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = A[p * N + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * N + q] - A[p * N + p]) / (2.0 * apq);
        const double at = fabs(theta);
        double t = at > 1e150 ? 0.5 / at : 1.0 / (at + sqrt(at * at + 1.0));
        t = theta < 0.0 ? -t : t;
        const double cs = rsqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < N; ++k) {
          const double akp = A[k * N + p], akq = A[k * N + q];
          A[k * N + p] = cs * akp - sn * akq;
          A[k * N + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < N; ++k) {
          const double apk = A[p * N + k], aqk = A[q * N + k];
          A[p * N + k] = cs * apk - sn * aqk;
          A[q * N + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < N; ++k) {
          const double vkp = V[k * N + p], vkq = V[k * N + q];
          V[k * N + p] = cs * vkp - sn * vkq;
          V[k * N + q] = sn * vkp + cs * vkq;
        }
      }
  }
  double lam[12];
  for (int e = 0; e < N; ++e) lam[e] = A[e * N + e] > 0.0 ? A[e * N + e] : 0.0;
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      double acc = 0.0;
      for (int e = 0; e < N; ++e) acc += V[p * N + e] * lam[e] * V[q * N + e];
      A[p * N + q] = acc;
    }
}

// weight of each stencil vertex on each of the item's cage nodes (0 for kinematic)
__device__ __forceinline__ void vertex_node_weights(const int32_t v[4], const int32_t* __restrict__ cage_idx,
                                                    const double* __restrict__ w, const int32_t* nodes, int n,
                                                    double W[4][kMaxNodes]) {
  for (int a = 0; a < 4; ++a) {
    for (int u = 0; u < n; ++u) W[a][u] = 0.0;
    const int4 id = __ldg(reinterpret_cast<const int4*>(cage_idx) + v[a]);
    if (id.x < 0) continue;
    const int ids[4] = {id.x, id.y, id.z, id.w};
    for (int s2 = 0; s2 < 4; ++s2) {
      int u = 0;
      while (u < n - 1 && nodes[u] != ids[s2]) ++u;
      W[a][u] += __ldg(w + 4 * (int64_t)v[a] + s2);
    }
  }
}

// One barrier item: distance, span Hessian (projected unless A.project is false), energy,
// and its upper-triangle Hessian records, the diagonal ones carrying the gradient, each
// written at its presorted position hinv[pos].
__device__ __forceinline__ void eval_barrier_item(const EvalArgs& A, int64_t k) {
  int32_t v[4];
  const int type = A.pr.type[k];
  stencil_vertices(A.T, type, A.pr.i[k], A.pr.j[k], v);
  V3 X[4];
  for (int a = 0; a < 4; ++a) X[a] = load_x(A.x4, v[a]);
  // positions relative to the first vertex (distance and derivatives are translation
  // invariant; this keeps the differences exact-ish)
  V3 Y[4];
  for (int a = 0; a < 4; ++a) Y[a] = X[a] - X[0];
  Stencil S;
  if (type == 0) pt_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
  else ee_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
  const int n = A.item_n[k];
  const int32_t* nodes = A.item_nodes + kMaxNodes * k;
  const int64_t oh = A.ro_h[k];
  double E = 0.0;
  double Kp[5][5];
  double cn = 0.0, b1 = 0.0;
  V3 rh = {0.0, 0.0, 0.0};
  double basis[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};  // c^, a^_1, a^_2
  bool active = false;
  if (!(S.d2 > 0.0)) {
    raise_flag(A.st, EIPC_FLAG_PENETRATION);
  } else {
    const double d = sqrt(S.d2);
    active = d < A.dhat;
    double eps_m, c_m;
    if (active && ee_mollified(A, type, A.pr.i[k], A.pr.j[k], Y, &eps_m, &c_m)) return;   // k_eval_mollified
    if (active) {
      BarrierSpan B;
      barrier_span(Y, S, d, A.dhat, A.kappa, B);
      E = B.E; b1 = B.b1; cn = B.cn; rh = B.rh;
      for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 4; ++a) basis[c][a] = B.basis[c][a];
      if (A.project) {
        // K+ in the span.  With fewer than two free closest-point parameters (an edge or a
        // vertex of the triangle, an endpoint against an edge or two endpoints) the fifth
        // basis vector is zero, so K's last row and column are zero and the projection is a
        // 4 x 4 eigenproblem
        if (S.m == 2) psd_span5(B.K, Kp);
        else psd_span4(B.K, Kp);
      } else {
        for (int p = 0; p < 5; ++p)
          for (int q = 0; q < 5; ++q) Kp[p][q] = B.K[p][q];
      }
    }
  }
  // the lagged friction item on this pair's stencil, if any, goes into the same records:
  // its blocks w_u w_v F are added to the barrier blocks (Sec. III-B, Eq. 8-9)
  const int32_t fenc = A.fric_of_pair ? A.fric_of_pair[k] : 0;
  const bool fr = fenc > 0;
  FrictionTerms R;
  // per-node scalars omega, alpha_1, alpha_2 and the friction weight w_u (nw[u][3])
  double coef[4][4];
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 4; ++a) coef[c][a] = basis[c][a];      // zero when not active
  if (fr) {
    friction_terms(A.x4, A.lag, (int64_t)(INT32_MAX - fenc), v, A.mu, A.eps_f, R, coef[3]);
    E += R.E;
  }
  A.item_E[k] = E;
  double nw[kMaxNodes][4];
  if (fr) {
    node_weights4<4>(v, A.cage_idx, A.w, nodes, n, coef, nw);
  } else if (active) {
    node_weights4<3>(v, A.cage_idx, A.w, nodes, n, coef, nw);
  } else {
    for (int u = 0; u < n; ++u) nw[u][0] = nw[u][1] = nw[u][2] = 0.0;
  }
  // Hessian records, upper triangle only: block(u,v) = A_u K+ A_v^T for u <= v, keyed by
  // (min(I_u, I_v), max(I_u, I_v)) and transposed when I_u > I_v
  const double rhv[3] = {rh.x, rh.y, rh.z};
  int64_t pos = oh;
  // the sorted position of the next record is loaded one record ahead, so its latency
  // overlaps the current block's arithmetic
  const int64_t pend = min(oh + (int64_t)n * (n + 1) / 2, A.rec_cap);
  int64_t nxt = (A.hinv && pos < pend) ? (int64_t)__ldg(A.hinv + pos) : -1;
  auto advance = [&]() {
    const int64_t cur = nxt;
    nxt = (A.hinv && pos + 1 < pend) ? (int64_t)__ldg(A.hinv + pos + 1) : -1;
    return cur;
  };
  for (int u = 0; u < n; ++u) {
    double Bu[3][5];
    if (active) {
      double t[5];
      for (int q = 0; q < 5; ++q) t[q] = nw[u][1] * Kp[3][q] + nw[u][2] * Kp[4][q];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 5; ++q) Bu[p][q] = nw[u][0] * Kp[p][q] + rhv[p] * t[q];
    }
    // the diagonal block (u, u) is symmetric: its upper triangle, mirrored
    if (pos < A.rec_cap) {
      const int64_t dst = advance();
      double B[3][3];
      if (active) {
        for (int p = 0; p < 3; ++p) {
          const double s = nw[u][1] * Bu[p][3] + nw[u][2] * Bu[p][4];
          for (int q = p; q < 3; ++q) {
            B[p][q] = nw[u][0] * Bu[p][q] + s * rhv[q];
            B[q][p] = B[p][q];
          }
        }
      } else {
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) B[p][q] = 0.0;
      }
      if (fr) {
        const double ww = nw[u][3] * nw[u][3];
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) B[p][q] += ww * R.F[p][q];
      }
      // the gradient at node u: kappa b' |c| omega_u r^ (+ mu lambda f1/y w_u u)
      const double s = active ? A.kappa * b1 * cn * nw[u][0] : 0.0;
      double gx = s * rh.x, gy = s * rh.y, gz = s * rh.z;
      if (fr) {
        const double sf = R.gs * nw[u][3];
        gx += sf * R.u[0]; gy += sf * R.u[1]; gz += sf * R.u[2];
      }
      emit_diag(A, pos, B, gx, gy, gz, dst);
    }
    ++pos;
    for (int w2 = u + 1; w2 < n; ++w2, ++pos) {
      if (pos >= A.rec_cap) continue;
      const int64_t dst = advance();
      double B[3][3];
      if (active) {
        for (int p = 0; p < 3; ++p) {
          const double s = nw[w2][1] * Bu[p][3] + nw[w2][2] * Bu[p][4];
          for (int q = 0; q < 3; ++q) B[p][q] = nw[w2][0] * Bu[p][q] + s * rhv[q];
        }
      } else {
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) B[p][q] = 0.0;
      }
      if (fr) {
        const double ww = nw[u][3] * nw[w2][3];
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) B[p][q] += ww * R.F[p][q];
      }
      emit_upper(A, pos, nodes[u], nodes[w2], B, dst);
    }
  }
}

// MINB = 2: no register cap (about 200 registers, 2 blocks of 128 per SM); MINB = 3: at
// most 170 registers (3 blocks per SM, a few hundred bytes of spills); MINB = 4: at most
// 128 registers (4 blocks per SM, spilling a few KB to L1-resident local memory).  Chosen at
// run time.  With A.project false the pair Hessians are kept as they are (no PSD
// projection).
template <int MINB>
__global__ void __launch_bounds__(kEvalThreads, MINB) k_eval_barrier(EvalArgs A) {
  pdl_entry();
  const int64_t P = clamp_count(A.pr.count, A.pr.capacity);
  const int64_t nit = *A.n_items;
  const int64_t np = P < nit ? P : nit;
  if (!A.order) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np; k += grid_stride())
      eval_barrier_item(A, k);
    return;
  }
  // scheduled: a persistent work queue over pair tiles -- each warp claims the next
  // A.tile items of the order (one to several per lane), so warps that drew light items come
  // back for more (dynamic balance); in a batch the tiles run across scene boundaries
  const int lane = threadIdx.x & 31;
  const int tile = A.tile >= 32 ? (A.tile & ~31) : 32;
  int64_t base = 0;
  int left = 0;                  // items of the claimed tile not yet taken (a multiple of 32)
  // a warp takes 32 items per round, so np / 32 + 2 rounds cover every claim it can make
  const int64_t max_rounds = np / 32 + 2;
  for (int64_t round = 0;; ++round) {
    if (round > max_rounds) {
      raise_flag(A.st, EIPC_FLAG_STACK_OVERFLOW);
      break;
    }
    if (left == 0) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(reinterpret_cast<unsigned long long*>(A.queue), (unsigned long long)tile);
      base = (int64_t)__shfl_sync(0xffffffffu, b, 0);
      left = tile;
    }
    if (base >= np) break;
    const int64_t idx = base + lane;
    if (idx < np) eval_barrier_item(A, (int64_t)A.order[idx]);
    base += 32;
    left -= 32;
  }
}

__global__ void __launch_bounds__(kEvalThreads) k_eval_friction(EvalArgs A, eipc_lag lag, double mu, double eps) {
  pdl_entry();
  const int64_t P = clamp_count(A.pr.count, A.pr.capacity);
  const int64_t nit = *A.n_items;
  const int64_t L = nit - P;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < L; f += grid_stride()) {
    const int64_t k = P + f;
    if (friction_merged(A.fric_of_pair, A.pair_of_fric, f)) {
      A.item_E[k] = 0.0;           // evaluated with its contact pair, in that pair's records
      continue;
    }
    const int4 q4 = reinterpret_cast<const int4*>(lag.v)[f];
    const int32_t v[4] = {q4.x, q4.y, q4.z, q4.w};
    FrictionTerms R;
    double gam[4];
    friction_terms(A.x4, lag, f, v, mu, eps, R, gam);
    A.item_E[k] = R.E;
    const int n = A.item_n[k];
    const int32_t* nodes = A.item_nodes + kMaxNodes * k;
    double nw[kMaxNodes];
    node_weights1(v, A.cage_idx, A.w, nodes, n, gam, nw);
    const int64_t oh = A.ro_h[k];
    int64_t pos2 = oh;
    for (int a = 0; a < n; ++a) {
      for (int b = a; b < n; ++b, ++pos2) {
        if (pos2 >= A.rec_cap) continue;
        double B[3][3];
        const double ww = nw[a] * nw[b];
        for (int p = 0; p < 3; ++p)
          for (int q = p; q < 3; ++q) {
            B[p][q] = ww * R.F[p][q];
            B[q][p] = B[p][q];
          }
        if (b == a) {
          const double s = R.gs * nw[a];
          emit_diag(A, pos2, B, s * R.u[0], s * R.u[1], s * R.u[2]);
        } else {
          emit_upper(A, pos2, nodes[a], nodes[b], B);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ Hessian-vector product
// y = H u for the unprojected contact Hessian H and the full-space direction u = J v on the
// embedded vertices, u = kin_dir on the kinematic ones.  Each item emits one record per
// cage node of its stencil (J^T y restricted to the item) and, if it touches kinematic
// vertices, one record holding the sum of y over them under key ns + (item mod 64); the
// gradient reduction sums the records, and the 64 kinematic partials are added in order.
constexpr int kKinSlots = 64;

__device__ __forceinline__ bool item_has_kinematic(const Topo& T, const eipc_pairs& pr, int64_t P, const int32_t* lag_v,
                                                   int64_t L, int64_t k, const int32_t* __restrict__ cage_idx) {
  int32_t v[4];
  item_vertices(T, pr, P, lag_v, L, k, v);
  bool any = false;
  for (int a = 0; a < 4; ++a) any |= __ldg(cage_idx + 4 * (int64_t)v[a]) < 0;
  return any;
}

__global__ void k_hvp_counts(Topo T, eipc_pairs pr, const int32_t* lag_v, const int64_t* lag_count, int64_t lag_cap,
                             const int32_t* __restrict__ cage_idx, const int32_t* __restrict__ item_n,
                             const int64_t* n_items, int64_t cap, int64_t* __restrict__ rc_g) {
  pdl_entry();
  const int64_t n = clamp_count(n_items, cap);
  const int64_t P = clamp_count(pr.count, pr.capacity);
  const int64_t L = lag_v ? clamp_count(lag_count, lag_cap) : 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride())
    rc_g[k] = (int64_t)item_n[k] + (item_has_kinematic(T, pr, P, lag_v, L, k, cage_idx) ? 1 : 0);
}

__global__ void k_hvp_kin_sum(const double* __restrict__ rows, double* __restrict__ out_kin) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < kKinSlots; ++s)
      for (int c = 0; c < 3; ++c) a[c] += rows[3 * s + c];
    for (int c = 0; c < 3; ++c) out_kin[c] = a[c];
  }
}

// coefficient sums over the kinematic vertices of a stencil
__device__ __forceinline__ void kinematic_sums(const int32_t v[4], const int32_t* __restrict__ cage_idx,
                                               const double coef[3][4], int ncoef, double out[3]) {
  for (int c = 0; c < 3; ++c) out[c] = 0.0;
  for (int a = 0; a < 4; ++a) {
    if (__ldg(cage_idx + 4 * (int64_t)v[a]) >= 0) continue;
    for (int c = 0; c < ncoef; ++c) out[c] += coef[c][a];
  }
}

__device__ __forceinline__ V3 load_dir(const double* __restrict__ v, int32_t node) {
  return {v[3 * (int64_t)node], v[3 * (int64_t)node + 1], v[3 * (int64_t)node + 2]};
}

__device__ __forceinline__ void emit_g(const EvalArgs& A, int64_t pos, uint64_t key, V3 y) {
  if (pos >= A.gcap) return;
  emit_grad(A, pos, key, y.x, y.y, y.z);
}

__global__ void __launch_bounds__(kEvalThreads) k_hvp_barrier(EvalArgs A) {
  pdl_entry();
  const int64_t P = clamp_count(A.pr.count, A.pr.capacity);
  const int64_t nit = *A.n_items;
  const int64_t np = P < nit ? P : nit;
  const V3 kd = {A.kin_dir[0], A.kin_dir[1], A.kin_dir[2]};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np; k += grid_stride()) {
    int32_t v[4];
    const int type = A.pr.type[k];
    stencil_vertices(A.T, type, A.pr.i[k], A.pr.j[k], v);
    V3 Y[4];
    const V3 X0 = load_x(A.x4, v[0]);
    for (int a = 0; a < 4; ++a) Y[a] = load_x(A.x4, v[a]) - X0;
    Stencil S;
    if (type == 0) pt_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
    else ee_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
    const int n = A.item_n[k];
    const int32_t* nodes = A.item_nodes + kMaxNodes * k;
    const int64_t og = A.ro_g[k];
    bool active = false;
    double t[5] = {0, 0, 0, 0, 0};
    double nw[kMaxNodes][3];
    double ks[3] = {0, 0, 0};
    V3 rh = {0.0, 0.0, 0.0};
    if (!(S.d2 > 0.0)) {
      raise_flag(A.st, EIPC_FLAG_PENETRATION);
    } else {
      const double d = sqrt(S.d2);
      active = d < A.dhat;
      double eps_m, c_m;
      if (active && ee_mollified(A, type, A.pr.i[k], A.pr.j[k], Y, &eps_m, &c_m)) continue;   // k_hvp_mollified
      if (active) {
        BarrierSpan B;
        barrier_span(Y, S, d, A.dhat, A.kappa, B);
        rh = B.rh;
        node_weights(v, A.cage_idx, A.w, nodes, n, B.basis, 3, nw);
        kinematic_sums(v, A.cage_idx, B.basis, 3, ks);
        // the direction in the span: Q^T u
        V3 uc = kd * ks[0];
        double ur[2] = {ks[1] * dot(kd, rh), ks[2] * dot(kd, rh)};
        for (int u = 0; u < n; ++u) {
          const V3 vu = load_dir(A.hv_dir, nodes[u]);
          uc = uc + vu * nw[u][0];
          const double vr = dot(vu, rh);
          ur[0] += nw[u][1] * vr;
          ur[1] += nw[u][2] * vr;
        }
        const double in5[5] = {uc.x, uc.y, uc.z, ur[0], ur[1]};
        for (int p = 0; p < 5; ++p) {
          double acc = 0.0;
          for (int q = 0; q < 5; ++q) acc += B.K[p][q] * in5[q];
          t[p] = acc;
        }
      }
    }
    const V3 tc = {t[0], t[1], t[2]};
    for (int u = 0; u < n; ++u) {
      V3 y = {0.0, 0.0, 0.0};
      if (active) y = tc * nw[u][0] + rh * (nw[u][1] * t[3] + nw[u][2] * t[4]);
      emit_g(A, og + u, (uint64_t)nodes[u], y);
    }
    bool kin = false;
    for (int a = 0; a < 4; ++a) kin |= __ldg(A.cage_idx + 4 * (int64_t)v[a]) < 0;
    if (kin) {
      V3 yk = {0.0, 0.0, 0.0};
      if (active) yk = tc * ks[0] + rh * (ks[1] * t[3] + ks[2] * t[4]);
      emit_g(A, og + n, (uint64_t)(A.ns + (k & (kKinSlots - 1))), yk);
    }
  }
}

__global__ void __launch_bounds__(kEvalThreads) k_hvp_friction(EvalArgs A, eipc_lag lag, double mu, double eps) {
  pdl_entry();
  const int64_t P = clamp_count(A.pr.count, A.pr.capacity);
  const int64_t nit = *A.n_items;
  const int64_t L = nit - P;
  const V3 kd = {A.kin_dir[0], A.kin_dir[1], A.kin_dir[2]};
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < L; f += grid_stride()) {
    const int64_t k = P + f;
    const int4 q4 = reinterpret_cast<const int4*>(lag.v)[f];
    const int32_t v[4] = {q4.x, q4.y, q4.z, q4.w};
    double gam[4];
    for (int a = 0; a < 4; ++a) gam[a] = lag.gamma[4 * f + a];
    const V3 nrm = {lag.n[3 * f], lag.n[3 * f + 1], lag.n[3 * f + 2]};
    const V3 anc = {lag.anchor[3 * f], lag.anchor[3 * f + 1], lag.anchor[3 * f + 2]};
    const double ml = mu * lag.lambda[f];
    V3 vs = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) vs = vs + load_x(A.x4, v[a]) * gam[a];
    vs = vs - anc;
    const V3 u = vs - nrm * dot(nrm, vs);
    const double y2 = dot(u, u);
    double f1y, f1p_minus;   // f1(y)/y, f1'(y) - f1(y)/y
    if (y2 == 0.0) {
      f1y = 2.0 / eps; f1p_minus = 0.0;
    } else {
      const double y = sqrt(y2);
      if (y < eps) { f1y = 2.0 / eps - y / (eps * eps); f1p_minus = -y / (eps * eps); }
      else { f1y = 1.0 / y; f1p_minus = -1.0 / y; }
    }
    const int n = A.item_n[k];
    const int32_t* nodes = A.item_nodes + kMaxNodes * k;
    const double coef[3][4] = {{gam[0], gam[1], gam[2], gam[3]}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    double nw[kMaxNodes][3];
    node_weights(v, A.cage_idx, A.w, nodes, n, coef, 1, nw);
    double ks[3];
    kinematic_sums(v, A.cage_idx, coef, 1, ks);
    // s = sum_a gamma_a u_a, then F s with F = mu lambda [f1/y (I - n n^T) + (f1' - f1/y) u u^T / y^2]
    V3 sd = kd * ks[0];
    for (int a = 0; a < n; ++a) sd = sd + load_dir(A.hv_dir, nodes[a]) * nw[a][0];
    const V3 sp = sd - nrm * dot(nrm, sd);
    V3 Fs = sp * (ml * f1y);
    if (y2 > 0.0) Fs = Fs + u * (ml * f1p_minus * dot(u, sd) / y2);
    const int64_t og = A.ro_g[k];
    for (int a = 0; a < n; ++a) emit_g(A, og + a, (uint64_t)nodes[a], Fs * nw[a][0]);
    bool kin = false;
    for (int a = 0; a < 4; ++a) kin |= __ldg(A.cage_idx + 4 * (int64_t)v[a]) < 0;
    if (kin) emit_g(A, og + n, (uint64_t)(A.ns + (k & (kKinSlots - 1))), Fs * ks[0]);
  }
}

// Mollified EE pairs (the main kernels skip them): the full 12 x 12 path, one thread per
// item, launched only when the mollifier is on.  The records go to the item's own offsets,
// as for every other item.
template <bool hvp>
__global__ void __launch_bounds__(kEvalThreads) k_mollified(EvalArgs A) {
  pdl_entry();
  const int64_t P = clamp_count(A.pr.count, A.pr.capacity);
  const int64_t nit = *A.n_items;
  const int64_t np = P < nit ? P : nit;
  const V3 kd = {A.kin_dir[0], A.kin_dir[1], A.kin_dir[2]};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np; k += grid_stride()) {
    const int type = A.pr.type[k];
    if (type != 1) continue;
    int32_t v[4];
    stencil_vertices(A.T, type, A.pr.i[k], A.pr.j[k], v);
    V3 Y[4];
    const V3 X0 = load_x(A.x4, v[0]);
    for (int a = 0; a < 4; ++a) Y[a] = load_x(A.x4, v[a]) - X0;
    double eps_m, c_m;
    if (!ee_mollified(A, type, A.pr.i[k], A.pr.j[k], Y, &eps_m, &c_m)) continue;
    Stencil S;
    ee_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
    if (!(S.d2 > 0.0)) continue;             // flagged by the main kernel
    const double d = sqrt(S.d2);
    if (!(d < A.dhat)) continue;
    const int n = A.item_n[k];
    const int32_t* nodes = A.item_nodes + kMaxNodes * k;
    const int64_t og = A.ro_g[k];
    double g12[12], H12[144], Em;
    mollified_local(Y, S, d, A.dhat, A.kappa, eps_m, c_m, &Em, g12, H12);
    double W[4][kMaxNodes];
    vertex_node_weights(v, A.cage_idx, A.w, nodes, n, W);
    if (hvp) {
      double u12[12], y12[12];
      bool kin = false;
      for (int a = 0; a < 4; ++a) {
        const bool ka = __ldg(A.cage_idx + 4 * (int64_t)v[a]) < 0;
        kin |= ka;
        V3 ua = ka ? kd : V3{0.0, 0.0, 0.0};
        for (int u = 0; u < n; ++u) ua = ua + load_dir(A.hv_dir, nodes[u]) * W[a][u];
        u12[3 * a] = ua.x; u12[3 * a + 1] = ua.y; u12[3 * a + 2] = ua.z;
      }
      for (int r = 0; r < 12; ++r) {
        double acc = 0.0;
        for (int q = 0; q < 12; ++q) acc += H12[12 * r + q] * u12[q];
        y12[r] = acc;
      }
      for (int u = 0; u < n; ++u) {
        V3 y = {0.0, 0.0, 0.0};
        for (int a = 0; a < 4; ++a) y = y + V3{y12[3 * a], y12[3 * a + 1], y12[3 * a + 2]} * W[a][u];
        emit_g(A, og + u, (uint64_t)nodes[u], y);
      }
      if (kin) {
        V3 yk = {0.0, 0.0, 0.0};
        for (int a = 0; a < 4; ++a)
          if (__ldg(A.cage_idx + 4 * (int64_t)v[a]) < 0) yk = yk + V3{y12[3 * a], y12[3 * a + 1], y12[3 * a + 2]};
        emit_g(A, og + n, (uint64_t)(A.ns + (k & (kKinSlots - 1))), yk);
      }
      continue;
    }
    if (A.project) psd_project_mem(H12, 12);
    A.item_E[k] = Em;
    int64_t pos = A.ro_h[k];
    for (int u = 0; u < n; ++u)
      for (int w2 = u; w2 < n; ++w2, ++pos) {
        if (pos >= A.rec_cap) continue;
        double Bk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            const double ww = W[a][u] * W[b][w2];
            if (ww == 0.0) continue;
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) Bk[p][q] += ww * H12[12 * (3 * a + p) + 3 * b + q];
          }
        if (w2 == u) {
          // the diagonal record carries the gradient at node u
          double y[3] = {0.0, 0.0, 0.0};
          for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) y[c] += W[a][u] * g12[3 * a + c];
          emit_diag(A, pos, Bk, y[0], y[1], y[2]);
        } else {
          emit_upper(A, pos, nodes[u], nodes[w2], Bk);
        }
      }
  }
}

// FP32 guess of a stencil's number of free closest-point parameters (2: projection inside
// the triangle / both segment parameters inside; 1: an edge interior; 0: two vertices), by
// the same region rules as pt_distance / ee_distance.  Only a scheduling hint: a wrong
// guess near a region boundary costs a divergent branch, never a different result.
__device__ __forceinline__ int seg_hint_f32(F3 w, F3 e, float* d2) {
  const float we = fdot(w, e), ee = fdot(e, e);
  const float t = we > 0.f ? (we < ee ? we / ee : 1.f) : 0.f;
  const F3 r = w - e * t;
  *d2 = fdot(r, r);
  return (t > 0.f && t < 1.f) ? 1 : 0;
}

__device__ __forceinline__ int span_hint_f32(const Topo& T, const double* __restrict__ x4, int type, int32_t i,
                                             int32_t j) {
  int32_t v[4];
  stencil_vertices(T, type, i, j, v);
  const V3 X0 = load_x(x4, v[0]);
  F3 Y[4];
  Y[0] = {0.f, 0.f, 0.f};
  for (int a = 1; a < 4; ++a) {
    const V3 d = load_x(x4, v[a]) - X0;
    Y[a] = {(float)d.x, (float)d.y, (float)d.z};
  }
  float best, d2;
  int m, mk;
  if (type == 0) {
    const F3 e1 = Y[2] - Y[1], e2 = Y[3] - Y[1], w = Y[0] - Y[1];
    const F3 n = fcross(e1, e2);
    const float nn = fdot(n, n);
    const float b1 = fdot(fcross(w, e2), n) / nn, b2 = fdot(fcross(e1, w), n) / nn;
    if (b1 >= 0.f && b2 >= 0.f && b1 + b2 <= 1.f) return 2;
    m = seg_hint_f32(w, e1, &best);
    mk = seg_hint_f32(Y[0] - Y[2], Y[3] - Y[2], &d2);
    if (d2 < best) { best = d2; m = mk; }
    mk = seg_hint_f32(Y[0] - Y[3], Y[1] - Y[3], &d2);
    if (d2 < best) m = mk;
    return m;
  }
  const F3 ea = Y[1] - Y[0], eb = Y[3] - Y[2], w = Y[0] - Y[2];
  const float A = fdot(ea, ea), B = fdot(ea, eb), C = fdot(eb, eb), D = fdot(ea, w), E = fdot(eb, w);
  const F3 n = fcross(ea, eb);
  const float nn = fdot(n, n);
  if (nn > 1e-12f * A * C) {
    const float sa = (B * E - C * D) / nn, tb = (A * E - B * D) / nn;
    if (sa >= 0.f && sa <= 1.f && tb >= 0.f && tb <= 1.f) return 2;
  }
  m = seg_hint_f32(Y[0] - Y[2], eb, &best);
  mk = seg_hint_f32(Y[1] - Y[2], eb, &d2);
  if (d2 < best) { best = d2; m = mk; }
  mk = seg_hint_f32(Y[2] - Y[0], ea, &d2);
  if (d2 < best) { best = d2; m = mk; }
  mk = seg_hint_f32(Y[3] - Y[0], ea, &d2);
  if (d2 < best) m = mk;
  return m;
}

// Schedule of the barrier evaluation: items keyed by (number of cage nodes, descending;
// a merged friction item or not; pair type; two free closest-point parameters (hinted) or
// fewer), friction items last.  A warp's lanes then take the same branches, project in the
// same dimension and emit the same number of blocks, and the heaviest items go first so
// the tail is light.  Only the processing order changes: every item writes its records at
// offsets fixed by its own index.  Keys fit in 8 bits: (16 - n) << 3 | fr << 2 | type << 1
// | (m == 2) with 1 <= n <= 16, and 128 for friction items.
__global__ void __launch_bounds__(kBlock) k_eval_order_keys(Topo T, const double* __restrict__ x4, eipc_pairs pr,
                                                            const int32_t* __restrict__ item_n, const int64_t* n_items,
                                                            const int32_t* __restrict__ fric_of_pair,
                                                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  pdl_entry();
  const int64_t P = clamp_count(pr.count, pr.capacity);
  const int64_t n = *n_items;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    uint64_t key = 128;
    if (k < P) {
      const int ty = pr.type[k] & 1;
      const int nn = min(max(item_n[k], 1), kMaxNodes);
      const int fr = (fric_of_pair && fric_of_pair[k] > 0) ? 1 : 0;
      const int m2 = span_hint_f32(T, x4, ty, pr.i[k], pr.j[k]) == 2 ? 1 : 0;
      key = (uint64_t)((kMaxNodes - nn) << 3 | fr << 2 | ty << 1 | m2);
    }
    keys[k] = key;
    vals[k] = (uint32_t)k;
  }
}

// record totals -> overflow flags and clamped sort counts
__global__ void k_rec_check(const int64_t* rh_total, const int64_t* rg_total, int64_t rec_cap, int64_t gcap,
                            int64_t* n_rh, int64_t* n_rg, DevStatus* st) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t a = *rh_total, b = *rg_total;
    if (a > rec_cap || b > gcap) {
      raise_flag(st, EIPC_FLAG_REC_OVERFLOW);
      raise_need(st, &st->need_rec, a > b ? a : b);
    }
    *n_rh = a < rec_cap ? a : rec_cap;
    *n_rg = b < gcap ? b : gcap;
  }
}

// Segment sums, one warp per segment: lane l adds records b+l, b+l+32, ... in order and a
// fixed shuffle tree combines the lanes, so the result depends only on the sorted order.
template <int W>
__device__ __forceinline__ void warp_tree_sum(double acc[W]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
}

// every upper block (I, J) becomes the full-pattern entry (I, J) and, off the diagonal,
// the transposed entry (J, I); diagonal blocks get a sentinel twin that sorts last.  Entry
// keys are row | col << br (br a whole number of radix digits): the upper blocks arrive in
// (I, J) order, so every transposed
// entry (r, I) of a row r (I < r) precedes the row's own upper entries, in increasing I;
// a stable sort on the row bits alone then leaves each row's columns increasing.
__global__ void __launch_bounds__(kBlock) k_full_entries(const uint64_t* __restrict__ ukey, const int64_t* n_seg,
                                                         int64_t ns, int br, int64_t cap,
                                                         uint64_t* __restrict__ fkey, uint32_t* __restrict__ fval,
                                                         int64_t* n_full_sort, int64_t* n_diag, DevStatus* st,
                                                         int32_t* __restrict__ dst) {
  pdl_entry();
  const int64_t S0 = *n_seg;
  const int64_t S = (2 * S0 <= cap) ? S0 : cap / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_full_sort = 2 * S;
    if (S < S0) raise_flag(st, EIPC_FLAG_REC_OVERFLOW);
  }
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += grid_stride()) {
    const uint64_t key = ukey[s];
    uint64_t I, J;
    upper_decode(key, (uint64_t)ns, &I, &J);
    fkey[2 * s] = I | (J << br);
    fval[2 * s] = (uint32_t)(s << 1);
    if (I != J) {
      fkey[2 * s + 1] = J | (I << br);
      fval[2 * s + 1] = (uint32_t)((s << 1) | 1);
    } else {
      fkey[2 * s + 1] = (1ull << br) - 1;           // row bits above every row: sorts last
      fval[2 * s + 1] = 0;
      dst[2 * s + 1] = -1;
      atomicAdd(reinterpret_cast<unsigned long long*>(n_diag), 1ull);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_seg_sum_g(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                      const double* __restrict__ rec, const int64_t* __restrict__ start,
                                                      const int64_t* n_rec, const int64_t* n_seg, int64_t cap,
                                                      double* __restrict__ g) {
  pdl_entry();
  const int64_t R = clamp_count(n_rec, cap);
  const int64_t S = *n_seg;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const int64_t b = start[s], e = (s + 1 < S) ? start[s + 1] : R;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t r = b + lane; r < e; r += 32) {
      const double* p = rec + kGRecStride * (int64_t)vals[r];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += p[c];
    }
    warp_tree_sum<3>(acc);
    if (lane == 0) {
      const int64_t node = (int64_t)keys[b];
#pragma unroll
      for (int c = 0; c < 3; ++c) g[3 * node + c] = acc[c];
    }
  }
}

// ---- presorted reduction: the record keys of the energy/gradient/Hessian evaluation
// depend only on each item's cage nodes, so they are written, sorted and turned into the
// BSR pattern before the evaluation; the evaluation then writes every record straight to
// its sorted position and the sums read contiguous records.

// keys of item k's Hessian records in the order the evaluation emits them: record (u, v),
// u <= v, keyed by the upper-triangle position of its nodes (min, max).  One warp per item,
// lanes on consecutive records.
__global__ void __launch_bounds__(kBlock) k_rec_keys(const int32_t* __restrict__ item_nodes,
                                                     const int32_t* __restrict__ item_n, const int64_t* __restrict__ ro_h,
                                                     const int64_t* n_items, int64_t rec_cap, int64_t ns,
                                                     uint64_t* __restrict__ hkeys, uint32_t* __restrict__ hvals) {
  pdl_entry();
  const int64_t nit = *n_items;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nit; k += nw) {
    const int n = item_n[k];
    const int32_t* nodes = item_nodes + kMaxNodes * k;
    const int64_t oh = ro_h[k];
    const int nrec = n * (n + 1) / 2;
    for (int l = lane; l < nrec; l += 32) {
      // row u of the upper triangle holds n - u records
      int u = 0, before = 0;
      while (before + (n - u) <= l) { before += n - u; ++u; }
      const int w2 = u + (l - before);
      const int64_t pos = oh + l;
      if (pos >= rec_cap) continue;
      const uint64_t Iu = (uint64_t)nodes[u], Iv = (uint64_t)nodes[w2];
      hkeys[pos] = Iu <= Iv ? upper_key(Iu, Iv, (uint64_t)ns) : upper_key(Iv, Iu, (uint64_t)ns);
      hvals[pos] = (uint32_t)pos;
    }
  }
}



// sorted full entries -> BSR columns, row counts, and for each upper segment s the BSR
// entry of its block (dst[2s]) and of its transpose (dst[2s+1]; -1 on the diagonal or
// beyond the capacity)
__global__ void __launch_bounds__(kBlock) k_bsr_pattern(const uint64_t* __restrict__ fkey, const uint32_t* __restrict__ fval,
                                                        const int64_t* n_full_sort, const int64_t* n_diag, int br,
                                                        int64_t ns, eipc_bsr H, int32_t* __restrict__ dst,
                                                        DevStatus* st, int64_t* __restrict__ n_gnodes) {
  pdl_entry();
  const int64_t nnzb = *n_full_sort - *n_diag;
  const uint64_t rmask = (1ull << br) - 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *H.nnzb = nnzb;
    *n_gnodes = *n_diag;           // nodes with a gradient: one diagonal block each
    if (nnzb > H.capacity) {
      raise_flag(st, EIPC_FLAG_BSR_OVERFLOW);
      raise_need(st, &st->need_bsr, nnzb);
    }
    if (nnzb == 0)
      for (int64_t r = 0; r <= ns; ++r) H.row_ptr[r] = 0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzb; e += grid_stride()) {
    const uint64_t key = fkey[e];
    const int64_t row = (int64_t)(key & rmask);
    // the entries are sorted by row: entry e starts every row after the previous entry's
    // row up to its own, and the last entry closes the rows after its own
    const int64_t prev = e > 0 ? (int64_t)(fkey[e - 1] & rmask) : -1;
    for (int64_t r = prev + 1; r <= row; ++r) H.row_ptr[r] = (int32_t)e;
    if (e == nnzb - 1)
      for (int64_t r = row + 1; r <= ns; ++r) H.row_ptr[r] = (int32_t)nnzb;
    const uint32_t v = fval[e];
    dst[2 * (int64_t)(v >> 1) + (v & 1u)] = e < H.capacity ? (int32_t)e : -1;
    if (e < H.capacity) H.col[e] = (int32_t)(key >> br);
  }
}

// Segment sums over contiguous presorted records in two passes.  Each segment is cut into
// units of kSegChunk consecutive records counted from its own first record; pass 1 adds
// each unit's records in order (one thread per unit, every lane doing useful FP64 adds,
// no shuffle tree), pass 2 adds a segment's unit sums in order (one thread per segment).
// The grouping depends only on the segment's own records, so a scene's sums are the same
// bits whether it is evaluated alone or inside a batch, and a long segment is spread over
// many threads.
constexpr int kSegChunk = 32;

// units per segment: unit[s] = ceil(len_s / kSegChunk) (exclusive-scanned afterwards),
// and, when keys is given, the segment's key ukey[s]
__global__ void __launch_bounds__(kBlock) k_seg_units(const int64_t* __restrict__ start, const int64_t* n_rec,
                                                      const int64_t* n_seg, int64_t cap, int64_t* __restrict__ unit,
                                                      const uint64_t* __restrict__ keys, uint64_t* __restrict__ ukey) {
  pdl_entry();
  const int64_t R = clamp_count(n_rec, cap);
  const int64_t S = *n_seg;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += grid_stride()) {
    const int64_t b = start[s];
    const int64_t len = ((s + 1 < S) ? start[s + 1] : R) - b;
    unit[s] = (len + kSegChunk - 1) / kSegChunk;
    if (keys) ukey[s] = keys[b];
  }
}

// the segment owning unit u: largest s with unit[s] <= u (unit exclusive-scanned, S >= 1)
__device__ __forceinline__ int64_t segment_of_unit(const int64_t* __restrict__ unit, int64_t S, int64_t u) {
  int64_t lo = 0, hi = S - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (unit[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// row r of a record array with rows of W values at a 16-byte aligned stride P, loaded
// two values at a time
template <int W, int P>
__device__ __forceinline__ void load_row(const double* __restrict__ x, int64_t r, double v[W]) {
  const double2* p = reinterpret_cast<const double2*>(x + P * r);
#pragma unroll
  for (int c = 0; c + 1 < W; c += 2) {
    const double2 t = __ldg(p + c / 2);
    v[c] = t.x;
    v[c + 1] = t.y;
  }
  if (W & 1) v[W - 1] = __ldg(x + P * r + W - 1);
}

// acc += x[r] for r = b, b+1, ..., e-1 in that order; the loads of four consecutive rows
// are issued before their adds so that a thread has several loads in flight
template <int W, int P>
__device__ __forceinline__ void add_in_order(const double* __restrict__ x, int64_t b, int64_t e, double acc[W]) {
  int64_t r = b;
  for (; r + 4 <= e; r += 4) {
    double v[4][W];
#pragma unroll
    for (int q = 0; q < 4; ++q) load_row<W, P>(x, r + q, v[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[c] += v[q][c];
  }
  for (; r < e; ++r) {
    double v[W];
    load_row<W, P>(x, r, v);
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] += v[c];
  }
}

template <int W, int P>
__global__ void __launch_bounds__(kBlock) k_seg_pieces(const double* __restrict__ rec, const int64_t* __restrict__ start,
                                                       const int64_t* __restrict__ unit, const int64_t* n_units,
                                                       const int64_t* n_rec, const int64_t* n_seg, int64_t cap,
                                                       double* __restrict__ piece) {
  pdl_entry();
  const int64_t R = clamp_count(n_rec, cap);
  const int64_t S = *n_seg;
  const int64_t U = *n_units;
  if (S <= 0) return;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U; u += grid_stride()) {
    const int64_t s = segment_of_unit(unit, S, u);
    const int64_t end = (s + 1 < S) ? start[s + 1] : R;
    const int64_t b = start[s] + (u - unit[s]) * kSegChunk;
    const int64_t e = (b + kSegChunk < end) ? b + kSegChunk : end;
    double acc[W];
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = 0.0;
    add_in_order<W, P>(rec, b, e, acc);
    double* p = piece + W * u;
#pragma unroll
    for (int c = 0; c < W; ++c) p[c] = acc[c];
  }
}

// Sum over the 32 lanes of a warp of the L-vectors a (L a power of two <= 16) by
// reduce-scatter: at each step the lanes pair up across one lane bit, each keeps half of
// the vector and adds its partner's copy of that half; when one entry is left, plain
// butterfly adds finish.  8 + 4 + 2 + 1 + 1 adds for L = 16 instead of 5 L.  Returns
// the full sum of component (lane >> (5 - log2 L)); the order of the adds is fixed.
template <int L>
__device__ __forceinline__ double warp_reduce_scatter(double (&a)[L], int lane) {
  int o = 16;
#pragma unroll
  for (int len = L; len > 1; len >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < len / 2; ++i) {
      const double send = hi ? a[i] : a[i + len / 2];
      const double keep = hi ? a[i + len / 2] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double v = a[0];
#pragma unroll
  for (; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Hessian pass 2, one warp per segment: lane l adds unit sums l, l+32, ... of its segment
// in order, then warp_reduce_scatter; the block goes into the BSR values at dst[2s] and,
// transposed, at dst[2s+1].  A diagonal segment (I, I) holds the six upper entries of its
// symmetric block and then the gradient at node I (emit_diag): the block is written whole
// and the gradient goes to g_r[I].
__global__ void __launch_bounds__(kBlock) k_seg_sum_h_pieces(const double* __restrict__ piece,
                                                             const int64_t* __restrict__ unit, const int64_t* n_units,
                                                             const int64_t* n_seg, int64_t cap,
                                                             const int32_t* __restrict__ dst, eipc_bsr H,
                                                             const uint64_t* __restrict__ ukey, int64_t ns,
                                                             double* __restrict__ g_r) {
  pdl_entry();
  const int64_t S0 = *n_seg;
  const int64_t S = (2 * S0 <= cap) ? S0 : cap / 2;      // the segments k_full_entries kept
  const int64_t U = *n_units;
  const int64_t nnzb = *H.nnzb;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const int64_t u1 = (s + 1 < S0) ? unit[s + 1] : U;
    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;
    for (int64_t k = unit[s] + lane; k < u1; k += 32) {
#pragma unroll
      for (int c = 0; c < 9; ++c) acc[c] += __ldg(piece + 9 * k + c);
    }
    const double v = warp_reduce_scatter<16>(acc, lane);
    const int c = lane >> 1;
    if ((lane & 1) == 0 && c < 9) {
      const int32_t du = dst[2 * s], dl = dst[2 * s + 1];
      const uint64_t key = ukey[s];
      uint64_t I, J;
      upper_decode(key, (uint64_t)ns, &I, &J);
      if (I != J) {
        if (du >= 0 && du < nnzb) H.val[9 * (int64_t)du + c] = v;
        if (dl >= 0 && dl < nnzb) H.val[9 * (int64_t)dl + 3 * (c % 3) + c / 3] = v;
      } else if (c < 6) {
        // upper entry c of the symmetric block: (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
        const int p = c < 3 ? 0 : (c < 5 ? 1 : 2);
        const int q = c < 3 ? c : (c < 5 ? c - 2 : 2);
        if (du >= 0 && du < nnzb) {
          H.val[9 * (int64_t)du + 3 * p + q] = v;
          H.val[9 * (int64_t)du + 3 * q + p] = v;
        }
      } else {
        g_r[3 * I + (c - 6)] = v;
      }
    }
  }
}

// deterministic sum: fixed chunk per block, fixed in-block tree, partials summed in order
__global__ void __launch_bounds__(kBlock) k_sum_partial(const double* __restrict__ x, const int64_t* n_dev,
                                                        int64_t cap, double* __restrict__ partial) {
  pdl_entry();
  const int64_t n = clamp_count(n_dev, cap);
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b = blockIdx.x * per, e = (b + per < n) ? b + per : n;
  double s = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) s += x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[kBlock / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// one warp: lane l adds partials l, l + 32, ... in order, then a fixed shuffle tree
__global__ void k_sum_final(const double* __restrict__ partial, int nb, double* out) {
  pdl_entry();
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double t = 0.0;
  for (int b = lane; b < nb; b += 32) t += partial[b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) *out = t;
}

// ------------------------------------------------------------------ friction lag
__global__ void __launch_bounds__(kEvalThreads) k_lag(Topo T, const double* __restrict__ x4, eipc_pairs pr,
                                                      double dhat, double kappa, eipc_lag out, DevStatus* st,
                                                      const double* __restrict__ moll_r2, double moll_factor,
                                                      uint64_t* __restrict__ key_out, int64_t key_cap) {
  pdl_entry();
  const int64_t P = clamp_count(pr.count, pr.capacity);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *out.count = P < out.capacity ? P : out.capacity;
    if (P > out.capacity) raise_flag(st, EIPC_FLAG_LAG_OVERFLOW);
  }
  const int64_t n = P < out.capacity ? P : out.capacity;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    int32_t v[4];
    const int type = pr.type[k];
    stencil_vertices(T, type, pr.i[k], pr.j[k], v);
    V3 X[4], Y[4];
    for (int a = 0; a < 4; ++a) X[a] = load_x(x4, v[a]);
    for (int a = 0; a < 4; ++a) Y[a] = X[a] - X[0];
    Stencil S;
    if (type == 0) pt_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
    else ee_distance<true>(Y[0], Y[1], Y[2], Y[3], &S);
    const double d = sqrt(S.d2);
    double b1 = 0.0;
    if (d > 0.0 && d < dhat) {
      const double lg = log(d / dhat), m = d - dhat;
      b1 = -2.0 * m * lg - m * m / d;
    }
    V3 rrel = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) rrel = rrel + Y[a] * S.c[a];
    const double rn = sqrt(dot(rrel, rrel));
    // anchor with the same arithmetic the evaluation uses for sum_a gamma_a x_a
    V3 anc = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) anc = anc + X[a] * S.c[a];
    reinterpret_cast<int4*>(out.v)[k] = make_int4(v[0], v[1], v[2], v[3]);
    if (k < key_cap) key_out[k] = lag_pair_key(type, pr.i[k], pr.j[k]);
    for (int a = 0; a < 4; ++a) out.gamma[4 * k + a] = S.c[a];
    out.n[3 * k] = rrel.x / rn; out.n[3 * k + 1] = rrel.y / rn; out.n[3 * k + 2] = rrel.z / rn;
    out.anchor[3 * k] = anc.x; out.anchor[3 * k + 1] = anc.y; out.anchor[3 * k + 2] = anc.z;
    // a mollified EE pair's lagged normal force is scaled by m(x^n)
    double mk = 1.0;
    if (type == 1 && moll_r2) {
      const V3 nn = cross(Y[1] - Y[0], Y[3] - Y[2]);
      const double c = dot(nn, nn);
      const double eps = moll_factor * moll_r2[pr.i[k]] * moll_r2[pr.j[k]];
      if (c < eps) mk = c * (2.0 / eps - c / (eps * eps));
    }
    out.lambda[k] = kappa * mk * fabs(b1);
  }
}

}  // namespace

int bits_for(uint64_t maxval) {
  int b = 1;
  while (b < 63 && (1ull << b) <= maxval) ++b;
  return b;
}

void lag_launch(eipc_scene* sc, const double* q_n, const eipc_pairs& pr, const eipc_params& p, const eipc_lag& out,
                cudaStream_t s) {
  EIPC_TIMED(sc, kKEmbed, s, embed_launch(sc, q_n, sc->x4, 1, 0, s));
  EIPC_TIMED(sc, kKLag, s,
             (launch(k_lag, blocks_for(pr.capacity, 8, kEvalThreads), kEvalThreads, 0, s, sc->topo, sc->x4, pr, p.dhat,
                     p.kappa, out, sc->status, static_cast<const double*>(sc->moll_factor > 0.0 ? sc->moll_r2 : nullptr),
                     sc->moll_factor, sc->lag_key, sc->item_cap)));
  sc->lag_src = out.v;   // the lag state whose pair keys lag_key now holds
}

void eval_launch(eipc_scene* sc, const double* q, const eipc_pairs& pr, const eipc_lag* lag, const eipc_params& p,
                 double* E, double* g_r, const eipc_bsr& H, cudaStream_t s) {
  EIPC_TIMED(sc, kKEmbed, s, embed_launch(sc, q, sc->x4, 1, 0, s));
  const bool fr = lag && p.mu > 0.0;
  // friction items ride on the contact pairs with the same stencil (not with the EE
  // mollifier, whose pairs are evaluated by their own kernel)
  const bool merge = fr && !(sc->moll_factor > 0.0);
  int64_t* cnt = sc->counters;
  int64_t* n_full = cnt + 13;
  int64_t* n_diag = cnt + 14;
  const int64_t item_cap = sc->item_cap;
  const int64_t pcap = pr.capacity < item_cap ? pr.capacity : item_cap;
  // counters, the evaluation queue, g_r and the friction claims, all reset up front
  zero_ranges(s, {{cnt + kCntItems, 5 * sizeof(int64_t)}, {n_diag, sizeof(int64_t)},
                  {cnt + kCntEvalQueue, sizeof(int64_t)}, {g_r, sizeof(double) * 3 * sc->ns},
                  {merge ? sc->fric_of_pair : nullptr, sizeof(int32_t) * pcap}});
  const int32_t* fop = merge ? sc->fric_of_pair : nullptr;
  const int32_t* pof = merge ? sc->pair_of_fric : nullptr;
  sc->timers->start(kKItems, s);
  if (merge)
    launch(k_fric_match, blocks_for(lag->capacity, 8), kBlock, 0, s, sc->topo, pr, *lag, item_cap,
           static_cast<const uint64_t*>(sc->edge_key), static_cast<const int32_t*>(sc->edge_id),
           static_cast<const uint64_t*>(lag->v == sc->lag_src ? sc->lag_key : nullptr), sc->fric_of_pair,
           sc->pair_of_fric);
  launch(k_item_nodes, blocks_for(item_cap, 8), kBlock, 0, s, sc->topo, pr, fr ? lag->v : nullptr, fr ? lag->count : nullptr,
                                                           fr ? lag->capacity : 0, sc->cage_idx, item_cap,
                                                           sc->item_nodes, sc->item_n, sc->item_group, sc->vgroup,
                                                           sc->rc_h, sc->rc_g,
                                                           cnt + kCntItems, sc->status, fop, pof);
  int64_t* tot_h = cnt + 9;
  int64_t* tot_g = cnt + 10;
  exclusive_scan2_i64(sc->rc_h, sc->ro_h, tot_h, sc->rc_g, sc->ro_g, tot_g, cnt + kCntItems, item_cap,
                      sc->scan_partial, s);
  launch(k_rec_check, 1, 32, 0, s, tot_h, tot_g, sc->rec_cap, sc->gcap, cnt + kCntRecH, cnt + kCntRecG, sc->status);
  sc->timers->stop(kKItems, s);

  // Hessian pattern before the evaluation: record keys (I, J) from the items' cage nodes,
  // stable sort, segments (one per BSR upper block), the inverse permutation that sends
  // each record to its sorted position, then the full symmetric pattern (every
  // off-diagonal upper block also at (J, I)), columns and row pointers
  sc->timers->start(kKHReduce, s);
  launch(k_rec_keys, blocks_for(32 * item_cap, 8), kBlock, 0, s, static_cast<const int32_t*>(sc->item_nodes),
         static_cast<const int32_t*>(sc->item_n), static_cast<const int64_t*>(sc->ro_h),
         static_cast<const int64_t*>(cnt + kCntItems), sc->rec_cap, sc->ns, sc->hkeys, sc->hvals);
  const int wh = radix_sort_u64(sc->hkeys, sc->hvals, sc->hkeys_alt, sc->hvals_alt, cnt + kCntRecH, sc->rec_cap,
                                sc->bits_h, sc->sort_hist, s);
  const uint64_t* hk = wh ? sc->hkeys_alt : sc->hkeys;
  const uint32_t* hv = wh ? sc->hvals_alt : sc->hvals;
  // segment starts, and the inverse permutation (each record's sorted position)
  segment_starts(hk, cnt + kCntRecH, sc->rec_cap, sc->seg_start, cnt + kCntSegH, sc->scan_partial, s, hv, sc->hinv);
  // seg_flag and seg_id hold the segment keys and the segments' BSR entries
  uint64_t* ukey = reinterpret_cast<uint64_t*>(sc->seg_flag);
  int32_t* dst = reinterpret_cast<int32_t*>(sc->seg_id);
  launch(k_seg_units, blocks_for(sc->rec_cap), kBlock, 0, s, static_cast<const int64_t*>(sc->seg_start),
         static_cast<const int64_t*>(cnt + kCntRecH), static_cast<const int64_t*>(cnt + kCntSegH), sc->rec_cap, sc->hunit,
         hk, ukey);
  exclusive_scan_i64(sc->hunit, sc->hunit, cnt + kCntSegH, sc->rec_cap, cnt + kCntUnitsH, sc->scan_partial, s);
  // row field: bits_g rounded up to whole radix digits (the sort passes cover whole bytes,
  // so the column must start on a byte); 2^bits_g > ns, so the all-ones row of the
  // diagonal twins is above every row
  const int rb = ((sc->bits_g + 7) / 8) * 8;
  launch(k_full_entries, blocks_for(sc->rec_cap), kBlock, 0, s, static_cast<const uint64_t*>(ukey),
         static_cast<const int64_t*>(cnt + kCntSegH), sc->ns, rb, sc->rec_cap, sc->hkeys, sc->hvals, n_full, n_diag,
         sc->status, dst);
  const int wf = radix_sort_u64(sc->hkeys, sc->hvals, sc->hkeys_alt, sc->hvals_alt, n_full, sc->rec_cap, rb,
                                sc->sort_hist, s);
  const uint64_t* fk = wf ? sc->hkeys_alt : sc->hkeys;
  const uint32_t* fv = wf ? sc->hvals_alt : sc->hvals;
  launch(k_bsr_pattern, blocks_for(sc->rec_cap), kBlock, 0, s, fk, fv, static_cast<const int64_t*>(n_full),
         static_cast<const int64_t*>(n_diag), rb, sc->ns, H, dst, sc->status, cnt + kCntSegG);
  sc->timers->stop(kKHReduce, s);

  EvalArgs A;
  A.T = sc->topo; A.pr = pr; A.cage_idx = sc->cage_idx; A.w = sc->w; A.x4 = sc->x4; A.ns = sc->ns;
  A.dhat = p.dhat; A.kappa = p.kappa; A.item_nodes = sc->item_nodes; A.item_n = sc->item_n;
  A.ro_h = sc->ro_h; A.ro_g = sc->ro_g; A.n_items = cnt + kCntItems; A.rec_cap = sc->rec_cap; A.gcap = sc->gcap;
  A.hkeys = nullptr; A.hvals = nullptr; A.hrec = sc->hrec; A.gkeys = nullptr; A.gvals = nullptr;
  A.grec = sc->grec; A.item_E = sc->item_E; A.st = sc->status;
  A.project = (p.flags & EIPC_PARAM_NO_PROJECTION) == 0;
  A.moll_r2 = sc->moll_factor > 0.0 ? sc->moll_r2 : nullptr;
  A.moll_factor = sc->moll_factor;
  A.hv_dir = nullptr; A.kin_dir[0] = A.kin_dir[1] = A.kin_dir[2] = 0.0;
  A.hinv = sc->hinv;                         // gradients ride in the diagonal records
  A.fric_of_pair = fop; A.pair_of_fric = pof;
  A.lag = fr ? *lag : eipc_lag{};
  A.mu = p.mu; A.eps_f = p.eps_v * p.h;
  {
    // (node count, type) schedule; the pair-sort buffers are free once the pairs are built
    launch(k_eval_order_keys, blocks_for(item_cap, 8), kBlock, 0, s, sc->topo, static_cast<const double*>(sc->x4), pr,
           static_cast<const int32_t*>(sc->item_n), static_cast<const int64_t*>(cnt + kCntItems), fop, sc->skeys,
           sc->svals);
    const int wo = radix_sort_u64(sc->skeys, sc->svals, sc->skeys_alt, sc->svals_alt, cnt + kCntItems, item_cap, 8,
                                  sc->sort_hist, s);
    A.order = wo ? sc->svals_alt : sc->svals;
    A.queue = cnt + kCntEvalQueue;
    A.tile = sc->tune.eval_tile;
  }
  // friction items on the scene's second stream, beside the barrier items: the two
  // kernels write disjoint records and item energies, and the barrier kernel leaves most
  // warp slots and part of the FP64 pipe free
  sc->timers->start(kKEvalPair, s);
  if (fr) {
    cudaEventRecord(sc->ev_fork, s);
    cudaStreamWaitEvent(sc->aux, sc->ev_fork, 0);
    EIPC_TIMED(sc, kKEvalFriction, sc->aux,
               (launch(k_eval_friction, blocks_for(lag->capacity, 8, kEvalThreads), kEvalThreads, 0, sc->aux, A,
                       *lag, p.mu, p.eps_v * p.h)));
    cudaEventRecord(sc->ev_join, sc->aux);
  }
  EIPC_TIMED(sc, kKEvalBarrier, s,
             (sc->tune.eval_variant == 4
                  ? launch(k_eval_barrier<4>, blocks_for(pr.capacity, sc->tune.eval_bps, sc->tune.eval_threads),
                           sc->tune.eval_threads, 0, s, A)
              : sc->tune.eval_variant == 3
                  ? launch(k_eval_barrier<3>, blocks_for(pr.capacity, sc->tune.eval_bps, sc->tune.eval_threads),
                           sc->tune.eval_threads, 0, s, A)
                  : launch(k_eval_barrier<2>, blocks_for(pr.capacity, sc->tune.eval_bps, sc->tune.eval_threads),
                           sc->tune.eval_threads, 0, s, A)));
  if (A.moll_r2)
    EIPC_TIMED(sc, kKEvalBarrier, s, (launch(k_mollified<false>, blocks_for(pr.capacity, 8, kEvalThreads), kEvalThreads, 0, s, A)));
  if (fr) cudaStreamWaitEvent(s, sc->ev_join, 0);
  sc->timers->stop(kKEvalPair, s);
  // sums over the contiguous presorted records, in sorted order
  sc->timers->start(kKHReduce, s);
  launch(k_seg_pieces<9, kHRecStride>, blocks_for(sc->rec_cap / kSegChunk + 1, 8), kBlock, 0, s, static_cast<const double*>(sc->hrec),
         static_cast<const int64_t*>(sc->seg_start), static_cast<const int64_t*>(sc->hunit),
         static_cast<const int64_t*>(cnt + kCntUnitsH), static_cast<const int64_t*>(cnt + kCntRecH),
         static_cast<const int64_t*>(cnt + kCntSegH), sc->rec_cap, sc->piece);
  // blocks into the BSR values; the diagonal segments' gradients into g_r
  launch(k_seg_sum_h_pieces, blocks_for(32 * sc->rec_cap, 8), kBlock, 0, s, static_cast<const double*>(sc->piece),
         static_cast<const int64_t*>(sc->hunit), static_cast<const int64_t*>(cnt + kCntUnitsH),
         static_cast<const int64_t*>(cnt + kCntSegH), sc->rec_cap, static_cast<const int32_t*>(dst), H,
         static_cast<const uint64_t*>(ukey), sc->ns, g_r);
  sc->timers->stop(kKHReduce, s);
  // energy
  sc->timers->start(kKEnergy, s);
  launch(k_sum_partial, kScanBlocks, kBlock, 0, s, sc->item_E, cnt + kCntItems, item_cap, sc->sum_partial);
  launch(k_sum_final, 1, 32, 0, s, sc->sum_partial, kScanBlocks, E);
  sc->timers->stop(kKEnergy, s);
}

void hvp_launch(eipc_scene* sc, const double* q, const eipc_pairs& pr, const eipc_lag* lag, const eipc_params& p,
                const double* v, const double* kin_dir, double* out_r, double* out_kin, cudaStream_t s) {
  EIPC_TIMED(sc, kKEmbed, s, embed_launch(sc, q, sc->x4, 1, 0, s));
  const bool fr = lag && p.mu > 0.0;
  int64_t* cnt = sc->counters;
  zero_ranges(s, {{cnt + kCntItems, 5 * sizeof(int64_t)}, {cnt + kCntZero, sizeof(int64_t)}});
  const int64_t item_cap = sc->item_cap;
  launch(k_item_nodes, blocks_for(item_cap, 8), kBlock, 0, s, sc->topo, pr, fr ? lag->v : nullptr, fr ? lag->count : nullptr,
         fr ? lag->capacity : 0, sc->cage_idx, item_cap, sc->item_nodes, sc->item_n, sc->item_group, sc->vgroup,
         sc->rc_h, sc->rc_g, cnt + kCntItems, sc->status, static_cast<const int32_t*>(nullptr),
         static_cast<const int32_t*>(nullptr));
  launch(k_hvp_counts, blocks_for(item_cap, 8), kBlock, 0, s, sc->topo, pr, fr ? lag->v : nullptr,
         fr ? static_cast<const int64_t*>(lag->count) : nullptr, fr ? lag->capacity : 0,
         static_cast<const int32_t*>(sc->cage_idx), static_cast<const int32_t*>(sc->item_n),
         static_cast<const int64_t*>(cnt + kCntItems), item_cap, sc->rc_g);
  int64_t* tot_g = cnt + 10;
  exclusive_scan_i64(sc->rc_g, sc->ro_g, cnt + kCntItems, item_cap, tot_g, sc->scan_partial, s);
  launch(k_rec_check, 1, 32, 0, s, static_cast<const int64_t*>(cnt + kCntZero), static_cast<const int64_t*>(tot_g),
         sc->rec_cap, sc->gcap, cnt + kCntRecH, cnt + kCntRecG, sc->status);
  EvalArgs A;
  A.T = sc->topo; A.pr = pr; A.cage_idx = sc->cage_idx; A.w = sc->w; A.x4 = sc->x4; A.ns = sc->ns;
  A.dhat = p.dhat; A.kappa = p.kappa; A.item_nodes = sc->item_nodes; A.item_n = sc->item_n;
  A.ro_h = sc->ro_h; A.ro_g = sc->ro_g; A.n_items = cnt + kCntItems; A.rec_cap = sc->rec_cap; A.gcap = sc->gcap;
  A.hkeys = sc->hkeys; A.hvals = sc->hvals; A.hrec = sc->hrec; A.gkeys = sc->gkeys; A.gvals = sc->gvals;
  A.grec = sc->grec; A.item_E = sc->item_E; A.st = sc->status;
  A.project = false;
  A.moll_r2 = sc->moll_factor > 0.0 ? sc->moll_r2 : nullptr;
  A.moll_factor = sc->moll_factor;
  A.order = nullptr;
  A.queue = nullptr;
  A.tile = 32;
  A.hv_dir = v;
  for (int c = 0; c < 3; ++c) A.kin_dir[c] = kin_dir ? kin_dir[c] : 0.0;
  A.hinv = nullptr;
  A.fric_of_pair = nullptr; A.pair_of_fric = nullptr;
  A.lag = fr ? *lag : eipc_lag{};
  A.mu = p.mu; A.eps_f = p.eps_v * p.h;
  EIPC_TIMED(sc, kKEvalBarrier, s,
             (launch(k_hvp_barrier, blocks_for(pr.capacity, 8, kEvalThreads), kEvalThreads, 0, s, A)));
  if (A.moll_r2)
    EIPC_TIMED(sc, kKEvalBarrier, s, (launch(k_mollified<true>, blocks_for(pr.capacity, 8, kEvalThreads), kEvalThreads, 0, s, A)));
  if (fr)
    EIPC_TIMED(sc, kKEvalFriction, s,
               (launch(k_hvp_friction, blocks_for(lag->capacity, 8, kEvalThreads), kEvalThreads, 0, s, A, *lag, p.mu,
                       p.eps_v * p.h)));
  sc->timers->start(kKGReduce, s);
  int wg = radix_sort_u64(sc->gkeys, sc->gvals, sc->gkeys_alt, sc->gvals_alt, cnt + kCntRecG, sc->gcap,
                          bits_for((uint64_t)(sc->ns + kKinSlots)), sc->sort_hist, s);
  const uint64_t* gk = wg ? sc->gkeys_alt : sc->gkeys;
  const uint32_t* gv = wg ? sc->gvals_alt : sc->gvals;
  segment_starts(gk, cnt + kCntRecG, sc->gcap, sc->gseg_start, cnt + kCntSegG, sc->scan_partial, s);
  zero_ranges(s, {{sc->hvp_out, sizeof(double) * 3 * (sc->ns + kKinSlots)}});
  launch(k_seg_sum_g, blocks_for(sc->gcap, 16), kBlock, 0, s, gk, gv, sc->grec, sc->gseg_start, cnt + kCntRecG,
         cnt + kCntSegG, sc->gcap, sc->hvp_out);
  cudaMemcpyAsync(out_r, sc->hvp_out, sizeof(double) * 3 * sc->ns, cudaMemcpyDeviceToDevice, s);
  if (out_kin)
    launch(k_hvp_kin_sum, 1, 32, 0, s, static_cast<const double*>(sc->hvp_out + 3 * sc->ns), out_kin);
  sc->timers->stop(kKGReduce, s);
}

}  // namespace eipc
