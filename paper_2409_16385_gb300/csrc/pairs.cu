// Embedding x = J q (Sec. III-D) and the contact set B (Sec. III-B): LBVH candidates,
// exact FP64 distance filter 0 < d < dhat, canonical (type, i, j) order.
#include "geometry.cuh"
#include "scene.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

// x_k = sum_j w_kj q_{idx_kj}; kinematic rows take x_kin (or 0 for a displacement).
// One thread per vertex; writes either the padded internal layout or a caller [Nv,3] array.
__global__ void __launch_bounds__(kBlock) k_embed(int64_t nv, const int32_t* __restrict__ idx,
                                                  const double* __restrict__ w, const double* __restrict__ xk4,
                                                  const double* __restrict__ q, double* __restrict__ out,
                                                  int padded, int displacement, float* __restrict__ outf,
                                                  DevStatus* st) {
  pdl_entry();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += grid_stride()) {
    const int4 id = __ldg(reinterpret_cast<const int4*>(idx) + v);
    double r[3];
    if (id.x < 0) {
      for (int k = 0; k < 3; ++k) r[k] = displacement ? 0.0 : xk4[4 * v + k];
    } else {
      const double2 w01 = __ldg(reinterpret_cast<const double2*>(w) + 2 * v);
      const double2 w23 = __ldg(reinterpret_cast<const double2*>(w) + 2 * v + 1);
      const int ids[4] = {id.x, id.y, id.z, id.w};
      const double ws[4] = {w01.x, w01.y, w23.x, w23.y};
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) s += ws[j] * __ldg(q + 3 * (int64_t)ids[j] + k);
        r[k] = s;
      }
      if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) raise_flag(st, EIPC_FLAG_NONFINITE);
    }
    if (padded) {
      reinterpret_cast<double2*>(out)[2 * v] = make_double2(r[0], r[1]);
      reinterpret_cast<double2*>(out)[2 * v + 1] = make_double2(r[2], 0.0);
      if (outf)
        reinterpret_cast<float4*>(outf)[v] =
            make_float4(__double2float_rn(r[0]), __double2float_rn(r[1]), __double2float_rn(r[2]), 0.f);
    } else {
      for (int k = 0; k < 3; ++k) out[3 * v + k] = r[k];
    }
  }
}

__device__ __forceinline__ void unpack(uint64_t key, int bi, int bj, int* type, int32_t* i, int32_t* j) {
  *j = (int32_t)(key & ((1ull << bj) - 1));
  *i = (int32_t)((key >> bj) & ((1ull << bi) - 1));
  *type = (int)(key >> (bi + bj));
}

__device__ __forceinline__ double stencil_d2(const Topo& T, const double* __restrict__ x4, int type, int32_t i,
                                             int32_t j) {
  if (type == 0) {
    const int32_t* f = T.tris + 3 * (int64_t)j;
    return pt_distance<false>(load_x(x4, i), load_x(x4, f[0]), load_x(x4, f[1]), load_x(x4, f[2]), nullptr);
  }
  const int32_t* ea = T.edges + 2 * (int64_t)i;
  const int32_t* eb = T.edges + 2 * (int64_t)j;
  return ee_distance<false>(load_x(x4, ea[0]), load_x(x4, ea[1]), load_x(x4, eb[0]), load_x(x4, eb[1]), nullptr);
}


// FP32 screen (geometry.cuh) over all candidates; the ones it cannot prove farther than
// dhat are compacted into `out` for the exact FP64 test.  The radius carries, besides the
// relative margin of the far tests, an absolute margin of twice their distance error
// budget, 80 M 2^-24 with M the candidate's largest coordinate, so the screen holds at any
// scene size.
__global__ void __launch_bounds__(kBlock) k_screen(Topo T, const float* __restrict__ x4f,
                                                   const uint64_t* __restrict__ cand,
                                                   const int64_t* n_cand, int64_t cap, double dhat,
                                                   uint64_t* __restrict__ out, int64_t* n_out) {
  pdl_entry();
  const int64_t n = clamp_count(n_cand, cap);
  const float dhat_up = __double2float_ru(dhat);
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += grid_stride()) {
    const int64_t k = base + threadIdx.x;
    bool pass = false;
    uint64_t key = 0;
    if (k < n) {
      key = cand[k];
      const int32_t j = (int32_t)(key & ((1ull << T.bits_j) - 1));
      const int32_t i = (int32_t)((key >> T.bits_j) & ((1ull << T.bits_i) - 1));
      const int type = (int)(key >> (T.bits_i + T.bits_j));
      F3 P[4];
      if (type == 0) {
        const int32_t* f = T.tris + 3 * (int64_t)j;
        P[0] = load_xf(x4f, i); P[1] = load_xf(x4f, f[0]); P[2] = load_xf(x4f, f[1]); P[3] = load_xf(x4f, f[2]);
      } else {
        const int32_t* ea = T.edges + 2 * (int64_t)i;
        const int32_t* eb = T.edges + 2 * (int64_t)j;
        P[0] = load_xf(x4f, ea[0]); P[1] = load_xf(x4f, ea[1]); P[2] = load_xf(x4f, eb[0]); P[3] = load_xf(x4f, eb[1]);
      }
      float M = 0.f;
      for (int a = 0; a < 4; ++a) M = fmaxf(M, fmaxf(fabsf(P[a].x), fmaxf(fabsf(P[a].y), fabsf(P[a].z))));
      const float r = __fadd_ru(dhat_up, 80.f * M * 5.9604645e-8f);
      const float r2m = r * r * 1.004f;
      pass = type == 0 ? !pt_far_f32(P[0], P[1], P[2], P[3], r2m) : !ee_far_f32(P[0], P[1], P[2], P[3], r2m);
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, pass);
    if (mask) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(reinterpret_cast<unsigned long long*>(n_out), (unsigned long long)__popc(mask));
      b = __shfl_sync(0xffffffffu, b, 0);
      if (pass) out[(int64_t)b + __popc(mask & ((1u << lane) - 1u))] = key;
    }
  }
}

// Exact filter of the broad-phase candidates: keep 0 < d < dhat, flag d <= 0.
__global__ void __launch_bounds__(kBlock) k_narrow(Topo T, const double* __restrict__ x4,
                                                   const uint64_t* __restrict__ cand, const int64_t* n_cand,
                                                   int64_t cand_cap, double dhat, uint64_t* __restrict__ skeys,
                                                   uint32_t* __restrict__ svals, double* __restrict__ sd,
                                                   int64_t* n_surv, DevStatus* st) {
  pdl_entry();
  const int64_t n = clamp_count(n_cand, cand_cap);
  const int lane = threadIdx.x & 31;
  // d2 at or above this has sqrt(d2) > dhat: rejected without the square root, the rest
  // take the test 0 < sqrt(d2) < dhat as it stands
  const double d2_reject = dhat * dhat * (1.0 + 1e-12);
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += grid_stride()) {
    const int64_t k = base + threadIdx.x;
    bool keep = false;
    uint64_t key = 0;
    double d = 0.0;
    if (k < n) {
      key = cand[k];
      int type; int32_t i, j;
      unpack(key, T.bits_i, T.bits_j, &type, &i, &j);
      const double d2 = stencil_d2(T, x4, type, i, j);
      if (!(d2 > 0.0)) {
        raise_flag(st, EIPC_FLAG_PENETRATION);
      } else if (d2 < d2_reject) {
        d = sqrt(d2);
        keep = d < dhat;
      }
    }
    uint32_t mask = __ballot_sync(0xffffffffu, keep);
    if (mask) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(reinterpret_cast<unsigned long long*>(n_surv), (unsigned long long)__popc(mask));
      b = __shfl_sync(0xffffffffu, b, 0);
      if (keep) {
        int64_t pos = (int64_t)b + __popc(mask & ((1u << lane) - 1u));
        // survivors never outnumber candidates, so pos < cand_cap
        skeys[pos] = key;
        svals[pos] = (uint32_t)pos;
        sd[pos] = d;
      }
    }
  }
}

// ---------------------------------------------------------------- constraint deduplication
// IPC-style reading of the pair set: a pair stands for the feature pair that realises its
// distance (face-vertex, vertex-edge, vertex-vertex, or edge-edge interior), and pairs that
// realise the same feature pair count once, represented by the first in (type, i, j) order.
// Feature keys: kind << 2B | id1 << B | id2, B bits per id.
enum { kFeatFV = 0, kFeatVE = 1, kFeatVV = 2, kFeatEE = 3 };

__device__ __forceinline__ uint64_t feature_key(int kind, uint32_t a, uint32_t b, int B) {
  return ((uint64_t)kind << (2 * B)) | ((uint64_t)a << B) | (uint64_t)b;
}

__global__ void __launch_bounds__(kBlock) k_feature_keys(Topo T, const double* __restrict__ x4,
                                                         const uint64_t* __restrict__ keys, const int64_t* n_surv,
                                                         int64_t cap, const uint64_t* __restrict__ ekey,
                                                         const int32_t* __restrict__ eid, int B,
                                                         uint64_t* __restrict__ fkeys, uint32_t* __restrict__ fvals,
                                                         DevStatus* st) {
  pdl_entry();
  const int64_t n = clamp_count(n_surv, cap);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    int type; int32_t i, j;
    unpack(keys[k], T.bits_i, T.bits_j, &type, &i, &j);
    int32_t v[4];
    if (type == 0) {
      v[0] = i; v[1] = T.tris[3 * (int64_t)j]; v[2] = T.tris[3 * (int64_t)j + 1]; v[3] = T.tris[3 * (int64_t)j + 2];
    } else {
      v[0] = T.edges[2 * (int64_t)i]; v[1] = T.edges[2 * (int64_t)i + 1];
      v[2] = T.edges[2 * (int64_t)j]; v[3] = T.edges[2 * (int64_t)j + 1];
    }
    V3 X[4];
    for (int a = 0; a < 4; ++a) X[a] = load_x(x4, v[a]);
    Stencil S;
    if (type == 0) pt_distance<true>(X[0] - X[0], X[1] - X[0], X[2] - X[0], X[3] - X[0], &S);
    else ee_distance<true>(X[0] - X[0], X[1] - X[0], X[2] - X[0], X[3] - X[0], &S);
    // the stencil's nonzero weights name the realising features
    int nz[4], m = 0;
    for (int a = 0; a < 4; ++a)
      if (S.c[a] != 0.0) nz[m++] = a;
    uint64_t f;
    if (S.m == 2) {
      f = type == 0 ? feature_key(kFeatFV, (uint32_t)j, (uint32_t)i, B) : feature_key(kFeatEE, (uint32_t)i, (uint32_t)j, B);
    } else if (S.m == 1) {
      // one point (the weight +-1 alone on its side) against the interior of a segment
      int pnt, s0, s1;
      if (type == 0) { pnt = 0; s0 = nz[1]; s1 = nz[2]; }
      else if ((S.c[0] != 0.0) != (S.c[1] != 0.0)) { pnt = S.c[0] != 0.0 ? 0 : 1; s0 = 2; s1 = 3; }
      else { pnt = S.c[2] != 0.0 ? 2 : 3; s0 = 0; s1 = 1; }
      int32_t e;
      if (type == 1) e = (s0 == 2) ? j : i;
      else e = edge_id_of(v[s0], v[s1], T.nv, ekey, eid, T.ne);
      if (e < 0) { raise_flag(st, EIPC_FLAG_BAD_INDEX); e = 0; }
      f = feature_key(kFeatVE, (uint32_t)v[pnt], (uint32_t)e, B);
    } else {
      int32_t a = v[nz[0]], b = v[m > 1 ? nz[1] : nz[0]];
      if (a > b) { const int32_t t = a; a = b; b = t; }
      f = feature_key(kFeatVV, (uint32_t)a, (uint32_t)b, B);
    }
    fkeys[k] = f;
    fvals[k] = (uint32_t)k;
  }
}

// sorted by feature: the first pair of each feature (lowest pair position, the sort being
// stable) is kept
__global__ void __launch_bounds__(kBlock) k_feature_firsts(const uint64_t* __restrict__ fkeys,
                                                           const uint32_t* __restrict__ fvals, const int64_t* n_surv,
                                                           int64_t cap, int64_t* __restrict__ keep) {
  pdl_entry();
  const int64_t n = clamp_count(n_surv, cap);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += grid_stride())
    keep[fvals[s]] = (s == 0 || fkeys[s] != fkeys[s - 1]) ? 1 : 0;
}

__global__ void __launch_bounds__(kBlock) k_feature_compact(const uint64_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ vals,
                                                            const int64_t* __restrict__ keep,
                                                            const int64_t* __restrict__ pos, const int64_t* n_surv,
                                                            int64_t cap, uint64_t* __restrict__ keys2,
                                                            uint32_t* __restrict__ vals2) {
  pdl_entry();
  const int64_t n = clamp_count(n_surv, cap);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride())
    if (keep[k]) {
      keys2[pos[k]] = keys[k];
      vals2[pos[k]] = vals[k];
    }
}

// Sorted survivors -> caller's pair arrays.
// The pair keys after a stable sort by (type, i) only: each run of one (type, i) -- the
// pairs one query found, a handful -- is put in j order by the thread at its head, in
// place (key order within a run is the whole key's order).  Runs longer than kRunMax are
// sorted the same way with a selection pass per element.
constexpr int kRunMax = 32;

__global__ void __launch_bounds__(kBlock) k_sort_runs(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                      const int64_t* n_dev, int64_t cap, int shift) {
  pdl_entry();
  const int64_t n = clamp_count(n_dev, cap);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    const uint64_t head = keys[k] >> shift;
    if (k > 0 && (keys[k - 1] >> shift) == head) continue;
    int64_t e = k + 1;
    while (e < n && (keys[e] >> shift) == head) ++e;
    const int64_t len = e - k;
    if (len == 1) continue;
    if (len <= kRunMax) {
      uint64_t kk[kRunMax];
      uint32_t vv[kRunMax];
      for (int a = 0; a < (int)len; ++a) {
        const uint64_t x = keys[k + a];
        const uint32_t y = vals[k + a];
        int b = a;
        while (b > 0 && kk[b - 1] > x) {
          kk[b] = kk[b - 1];
          vv[b] = vv[b - 1];
          --b;
        }
        kk[b] = x;
        vv[b] = y;
      }
      for (int a = 0; a < (int)len; ++a) {
        keys[k + a] = kk[a];
        vals[k + a] = vv[a];
      }
    } else {
      // in-place selection sort (keys are distinct)
      for (int64_t a = k; a < e; ++a) {
        int64_t m = a;
        for (int64_t b = a + 1; b < e; ++b)
          if (keys[b] < keys[m]) m = b;
        if (m != a) {
          const uint64_t tk = keys[a]; keys[a] = keys[m]; keys[m] = tk;
          const uint32_t tv = vals[a]; vals[a] = vals[m]; vals[m] = tv;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_emit_pairs(Topo T, const uint64_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ vals, const double* __restrict__ sd,
                                                       const int64_t* n_surv, int64_t cand_cap, eipc_pairs out,
                                                       DevStatus* st) {
  pdl_entry();
  const int64_t n = clamp_count(n_surv, cand_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *out.count = n;
    if (n > out.capacity) {
      raise_flag(st, EIPC_FLAG_PAIR_OVERFLOW);
      raise_need(st, &st->need_pairs, n);
    }
  }
  const int64_t m = n < out.capacity ? n : out.capacity;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += grid_stride()) {
    int type; int32_t i, j;
    unpack(keys[k], T.bits_i, T.bits_j, &type, &i, &j);
    out.type[k] = type;
    out.i[k] = i;
    out.j[k] = j;
    out.d[k] = sd[vals[k]];
  }
}

}  // namespace

void embed_launch(const eipc_scene* sc, const double* q, double* out, int out_padded, int displacement,
                  cudaStream_t s) {
  float* outf = (out_padded && out == sc->x4) ? sc->x4f : nullptr;   // FP32 copy for the screen
  launch(k_embed, blocks_for(sc->nv), kBlock, 0, s, sc->nv, sc->cage_idx, sc->w, sc->x_kin4, q, out, out_padded,
         displacement, outf, sc->status);
}

namespace {
// new prescribed positions for the kinematic rows (cage_idx[4v] < 0) only
__global__ void __launch_bounds__(kBlock) k_set_kinematic(int64_t nv, const int32_t* __restrict__ cage_idx,
                                                          const double* __restrict__ x_kin, double* __restrict__ x_kin4) {
  pdl_entry();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += grid_stride()) {
    if (cage_idx[4 * v] >= 0) continue;
    x_kin4[4 * v] = x_kin[3 * v];
    x_kin4[4 * v + 1] = x_kin[3 * v + 1];
    x_kin4[4 * v + 2] = x_kin[3 * v + 2];
  }
}
// squared rest length of every edge, |x_b - x_a|^2 from rest positions x_rest [nv*3]; bad
// counts the edges whose squared length is not a positive finite number
__global__ void __launch_bounds__(kBlock) k_edge_rest_len2(int64_t ne, const int32_t* __restrict__ edges,
                                                           const double* __restrict__ x_rest, double* __restrict__ r2,
                                                           int64_t* bad) {
  pdl_entry();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += grid_stride()) {
    const int64_t a = edges[2 * e], b = edges[2 * e + 1];
    const double dx = x_rest[3 * b] - x_rest[3 * a];
    const double dy = x_rest[3 * b + 1] - x_rest[3 * a + 1];
    const double dz = x_rest[3 * b + 2] - x_rest[3 * a + 2];
    const double l2 = dx * dx + dy * dy + dz * dz;
    r2[e] = l2;
    if (!(l2 > 0.0 && l2 <= 1.7976931348623157e308)) atomicAdd(reinterpret_cast<unsigned long long*>(bad), 1ull);
  }
}

// candidate keys (type << (bits_i + bits_j) | i << bits_j | j) decoded into three arrays
__global__ void __launch_bounds__(kBlock) k_decode_candidates(Topo T, const uint64_t* __restrict__ cand,
                                                              const int64_t* n_cand, int64_t cand_cap, int64_t out_cap,
                                                              int32_t* __restrict__ type, int32_t* __restrict__ ci,
                                                              int32_t* __restrict__ cj, int64_t* n_out) {
  pdl_entry();
  const int64_t n = clamp_count(n_cand, cand_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = n;
  const int64_t m = n < out_cap ? n : out_cap;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += grid_stride()) {
    const uint64_t key = cand[k];
    cj[k] = (int32_t)(key & ((1ull << T.bits_j) - 1));
    ci[k] = (int32_t)((key >> T.bits_j) & ((1ull << T.bits_i) - 1));
    type[k] = (int32_t)(key >> (T.bits_i + T.bits_j));
  }
}
}  // namespace

void mollifier_rest_launch(eipc_scene* sc, const double* x_rest, int64_t* bad, cudaStream_t s) {
  launch(k_edge_rest_len2, blocks_for(sc->ne), kBlock, 0, s, sc->ne, static_cast<const int32_t*>(sc->edges), x_rest,
         sc->moll_r2, bad);
}

void candidates_launch(eipc_scene* sc, int32_t* type, int32_t* ci, int32_t* cj, int64_t cap, int64_t* n,
                       cudaStream_t s) {
  launch(k_decode_candidates, blocks_for(sc->cand_cap), kBlock, 0, s, sc->topo,
         static_cast<const uint64_t*>(sc->cand), static_cast<const int64_t*>(sc->counters + kCntCand), sc->cand_cap,
         cap, type, ci, cj, n);
}

void set_kinematic_launch(eipc_scene* sc, const double* x_kin, cudaStream_t s) {
  launch(k_set_kinematic, blocks_for(sc->nv), kBlock, 0, s, sc->nv, static_cast<const int32_t*>(sc->cage_idx), x_kin,
         sc->x_kin4);
}

void pairs_launch(eipc_scene* sc, const double* q, const eipc_params& p, const eipc_pairs& out, cudaStream_t s) {
  EIPC_TIMED(sc, kKEmbed, s, embed_launch(sc, q, sc->x4, 1, 0, s));
  int64_t* n_cand = sc->counters + kCntCand;
  int64_t* n_surv = sc->counters + kCntSurv;
  int64_t* n_cand2 = sc->counters + kCntScreened;
  zero_ranges(s, {{sc->counters + kCntCand, 2 * sizeof(int64_t)}, {n_cand2, sizeof(int64_t)}});
  // LBVHs over triangles and edges, then one traversal: vertex boxes grown by dhat against
  // the triangle tree (PT) and edge boxes grown by dhat against the edge tree (EE, j > i)
  // full rebuild every `rebuild_interval` calls, refit of the same hierarchy in between (the
  // candidate set is exact for any hierarchy; only traversal cost depends on its quality)
  const bool rebuild = !sc->tri_bvh.built || !sc->edge_bvh.built || sc->contact_refits + 1 >= sc->rebuild_interval;
  // per-vertex boxes: unpadded for the leaves, grown by dhat for the queries
  EIPC_TIMED(sc, kKBvh, s, vertex_boxes(sc->topo, sc->x4, nullptr, p.dhat, sc->vbox, sc->vbox_pad, s));
  if (rebuild) {
    EIPC_TIMED(sc, kKBvh, s, bvh_build(sc->tri_bvh, kTri, sc->topo, sc->x4, nullptr, sc->vbox, sc->bounds_ws, sc->sort_hist, s,
                                      sc->tune.refit_variant));
    EIPC_TIMED(sc, kKBvh, s, bvh_build(sc->edge_bvh, kEdge, sc->topo, sc->x4, nullptr, sc->vbox, sc->bounds_ws, sc->sort_hist, s,
                                      sc->tune.refit_variant));
    sc->contact_refits = 0;
  } else {
    EIPC_TIMED(sc, kKBvh, s,
               bvh_refit_pair(sc->tri_bvh, kTri, sc->edge_bvh, kEdge, sc->topo, sc->vbox, s, sc->tune.refit_variant));
    ++sc->contact_refits;
  }
  EIPC_TIMED(sc, kKQuery, s,
             bvh_query(sc->tri_bvh, sc->edge_bvh, sc->topo, sc->vbox_pad, sc->cand, n_cand, sc->cand_cap,
                       sc->status, s, sc->tune.query_threads, sc->tune.query_bps,
                       sc->tune.query_variant));
  sc->timers->start(kKNarrow, s);
  launch(k_screen, blocks_for(sc->cand_cap, 16), kBlock, 0, s, sc->topo, static_cast<const float*>(sc->x4f),
         static_cast<const uint64_t*>(sc->cand),
         static_cast<const int64_t*>(n_cand), sc->cand_cap, p.dhat, sc->cand2, n_cand2);
  launch(k_narrow, blocks_for(sc->cand_cap, 16), kBlock, 0, s, sc->topo, sc->x4, sc->cand2, n_cand2, sc->cand_cap,
         p.dhat, sc->skeys, sc->svals, sc->sd, n_surv, sc->status);
  sc->timers->stop(kKNarrow, s);
  sc->timers->start(kKPairSort, s);
  // (type, i, j) order: a stable sort by (type, i), the key's bits above j, then each
  // run of one (type, i) sorted by j in place (three passes instead of five)
  const int bj = sc->topo.bits_j;
  int which = radix_sort_u64(sc->skeys, sc->svals, sc->skeys_alt, sc->svals_alt, n_surv, sc->cand_cap,
                             1 + sc->topo.bits_i, sc->sort_hist, s, bj);
  uint64_t* ks = which ? sc->skeys_alt : sc->skeys;
  uint32_t* vs = which ? sc->svals_alt : sc->svals;
  launch(k_sort_runs, blocks_for(sc->cand_cap, 8), kBlock, 0, s, ks, vs, static_cast<const int64_t*>(n_surv),
         sc->cand_cap, bj);
  const uint64_t* k = ks;
  const uint32_t* v = vs;
  const int64_t* n_out = n_surv;
  if (p.flags & EIPC_PARAM_DEDUP) {
    // feature keys in the record buffers (free until the evaluation), stable sort, firsts,
    // compaction back into (type, i, j) order in the other half of the pair-sort buffers
    const int64_t cap = sc->rec_cap < sc->cand_cap ? sc->rec_cap : sc->cand_cap;
    launch(k_feature_keys, blocks_for(cap, 8), kBlock, 0, s, sc->topo, static_cast<const double*>(sc->x4), k,
           static_cast<const int64_t*>(n_surv), cap, static_cast<const uint64_t*>(sc->edge_key),
           static_cast<const int32_t*>(sc->edge_id), sc->feat_bits, sc->hkeys, sc->hvals, sc->status);
    const int wf = radix_sort_u64(sc->hkeys, sc->hvals, sc->hkeys_alt, sc->hvals_alt, n_surv, cap, 2 + 2 * sc->feat_bits,
                                  sc->sort_hist, s);
    launch(k_feature_firsts, blocks_for(cap, 8), kBlock, 0, s, static_cast<const uint64_t*>(wf ? sc->hkeys_alt : sc->hkeys),
           static_cast<const uint32_t*>(wf ? sc->hvals_alt : sc->hvals), static_cast<const int64_t*>(n_surv), cap,
           sc->seg_flag);
    int64_t* n_kept = sc->counters + kCntDedup;
    exclusive_scan_i64(sc->seg_flag, sc->seg_id, n_surv, cap, n_kept, sc->scan_partial, s);
    uint64_t* k2 = which ? sc->skeys : sc->skeys_alt;
    uint32_t* v2 = which ? sc->svals : sc->svals_alt;
    launch(k_feature_compact, blocks_for(cap, 8), kBlock, 0, s, k, v, static_cast<const int64_t*>(sc->seg_flag),
           static_cast<const int64_t*>(sc->seg_id), static_cast<const int64_t*>(n_surv), cap, k2, v2);
    k = k2; v = v2; n_out = n_kept;
  }
  launch(k_emit_pairs, blocks_for(out.capacity, 8), kBlock, 0, s, sc->topo, k, v, sc->sd, n_out, sc->cand_cap, out,
                                                               sc->status);
  sc->timers->stop(kKPairSort, s);
}

}  // namespace eipc
