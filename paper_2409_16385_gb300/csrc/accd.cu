// Step bound for the straight full-space motion x + t dx (Sec. III-C: phi is linear, so a
// reduced step is a straight motion of every surface vertex and linear CCD is exact).
//
// Candidates: PT / EE pairs (not incident, not all kinematic) whose closed FP64 swept
// boxes over [x, x + dx] overlap -- found with an LBVH over FP32 swept boxes rounded
// outward, then confirmed with the exact FP64 box test.  Per candidate, conservative
// advancement: remove the stencil's mean displacement; L = (largest relative speed on side
// A) + (largest on side B) bounds how fast the distance can shrink, so advancing t by
// (1 - s) d(t) / L keeps d > 0 on the whole advance; stop once d(t) <= s d(0), at t >= 1
// (then t = 1) or after accd_max_iter advances (the t reached is still safe).
// alpha = min(1, min_k t_k): exact minimum via atomicMin on the IEEE bit pattern (t >= 0),
// so the result does not depend on thread order.  A pair's t is scaled by (1 - 2^-30)
// before the minimum: a deliberate margin that keeps alpha on the safe side of rounding
// differences between this FP64 arithmetic and any other evaluation of the same bound.
#include "geometry.cuh"
#include "scene.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

constexpr int kAccdThreads = 128;
constexpr double kMargin = 1.0 - 9.313225746154785e-10;   // 1 - 2^-30

__global__ void __launch_bounds__(kBlock) k_pad(const double* __restrict__ x, const double* __restrict__ dx,
                                                int64_t nv, double* __restrict__ x4, double* __restrict__ dx4,
                                                DevStatus* st) {
  pdl_entry();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += grid_stride()) {
    const double a = x[3 * v], b = x[3 * v + 1], c = x[3 * v + 2];
    const double e = dx[3 * v], f = dx[3 * v + 1], g = dx[3 * v + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(e) && isfinite(f) && isfinite(g)))
      raise_flag(st, EIPC_FLAG_NONFINITE);
    reinterpret_cast<double2*>(x4)[2 * v] = make_double2(a, b);
    reinterpret_cast<double2*>(x4)[2 * v + 1] = make_double2(c, 0.0);
    reinterpret_cast<double2*>(dx4)[2 * v] = make_double2(e, f);
    reinterpret_cast<double2*>(dx4)[2 * v + 1] = make_double2(g, 0.0);
  }
}

__global__ void k_alpha_init(unsigned long long* bits, unsigned long long* group_bits, int32_t ng) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) *bits = __double_as_longlong(1.0);
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
    group_bits[g] = __double_as_longlong(1.0);
}

__device__ __forceinline__ double pair_distance(int type, const V3 p[4]) {
  // relative to the first vertex: distance is translation invariant
  const V3 o = p[0];
  if (type == 0) return sqrt(pt_distance<false>(p[0] - o, p[1] - o, p[2] - o, p[3] - o, nullptr));
  return sqrt(ee_distance<false>(p[0] - o, p[1] - o, p[2] - o, p[3] - o, nullptr));
}

__global__ void __launch_bounds__(kAccdThreads) k_ca(Topo T, const double* __restrict__ x4,
                                                     const double* __restrict__ dx4, const uint64_t* __restrict__ cand,
                                                     const int64_t* n_cand, int64_t cap, double s, int max_iter,
                                                     unsigned long long* alpha_bits,
                                                     unsigned long long* __restrict__ group_bits, int64_t* n_adv,
                                                     DevStatus* st, int64_t* queue, int tile_req) {
  pdl_entry();
  const int64_t n = clamp_count(n_cand, cap);
  const int tile = tile_req >= 32 ? (tile_req & ~31) : 32;
  const int lane = threadIdx.x & 31;
  // persistent work queue over candidate tiles: each warp claims the next `tile`
  // candidates (tile / 32 per lane), so warps whose candidates settled at once come back for
  // more while a few run long advancements
  // every claim takes `tile` candidates, so n / tile + 2 claims cover all a warp can make
  const int64_t max_rounds = n / tile + 2;
  for (int64_t round = 0;; ++round) {
    if (round > max_rounds) {
      raise_flag(st, EIPC_FLAG_STACK_OVERFLOW);
      break;
    }
    unsigned long long qb = 0;
    if (lane == 0) qb = atomicAdd(reinterpret_cast<unsigned long long*>(queue), (unsigned long long)tile);
    const int64_t tbase = (int64_t)__shfl_sync(0xffffffffu, qb, 0);
    if (tbase >= n) break;
  for (int o = 0; o < tile; o += 32) {
    const int64_t k = tbase + o + lane;
    bool adv = false;
    int iters = 0;
    if (k < n) {
      const uint64_t key = cand[k];
      const int32_t j = (int32_t)(key & ((1ull << T.bits_j) - 1));
      const int32_t i = (int32_t)((key >> T.bits_j) & ((1ull << T.bits_i) - 1));
      const int type = (int)(key >> (T.bits_i + T.bits_j));
      int32_t v[4];
      if (type == 0) {
        v[0] = i;
        v[1] = T.tris[3 * (int64_t)j]; v[2] = T.tris[3 * (int64_t)j + 1]; v[3] = T.tris[3 * (int64_t)j + 2];
      } else {
        v[0] = T.edges[2 * (int64_t)i]; v[1] = T.edges[2 * (int64_t)i + 1];
        v[2] = T.edges[2 * (int64_t)j]; v[3] = T.edges[2 * (int64_t)j + 1];
      }
      V3 X[4], D[4];
      for (int a = 0; a < 4; ++a) { X[a] = load_x(x4, v[a]); D[a] = load_x(dx4, v[a]); }
      // exact closed swept-box overlap in FP64
      const int na = type == 0 ? 1 : 2;
      double lo[2][3], hi[2][3];
      for (int sd = 0; sd < 2; ++sd)
        for (int c = 0; c < 3; ++c) { lo[sd][c] = INFINITY; hi[sd][c] = -INFINITY; }
      for (int a = 0; a < 4; ++a) {
        const int sd = a < na ? 0 : 1;
        const double p0[3] = {X[a].x, X[a].y, X[a].z};
        const double p1[3] = {X[a].x + D[a].x, X[a].y + D[a].y, X[a].z + D[a].z};
        for (int c = 0; c < 3; ++c) {
          lo[sd][c] = fmin(lo[sd][c], fmin(p0[c], p1[c]));
          hi[sd][c] = fmax(hi[sd][c], fmax(p0[c], p1[c]));
        }
      }
      bool ov = true;
      for (int c = 0; c < 3; ++c) ov &= !(lo[0][c] > hi[1][c] || lo[1][c] > hi[0][c]);
      if (ov) {
        adv = true;
        V3 mean = (D[0] + D[1] + D[2] + D[3]) * 0.25;
        V3 R[4];
        for (int a = 0; a < 4; ++a) R[a] = D[a] - mean;
        // FP32 shortcut: the first advancement reaches t = 1 exactly when d0 >= L / (1 - s).
        // An upward-rounded bound L_hi >= L and a conservative FP32 far test proving
        // d0 > L_hi / (1 - s) give that result without the FP64 distance.  The far radius
        // carries twice the FP32 tests' distance error budget, 40 M 2^-24 (M: the candidate's
        // largest coordinate), as an absolute margin, so it holds for any motion size.
        bool far = false;
        {
          float la_f = 0.f, lb_f = 0.f, Mf = 0.f;
          F3 Xf[4];
          for (int a = 0; a < 4; ++a) {
            const float sp = __fsqrt_ru(__double2float_ru(dot(R[a], R[a])));
            if (a < na) la_f = fmaxf(la_f, sp); else lb_f = fmaxf(lb_f, sp);
            Xf[a] = F3{(float)X[a].x, (float)X[a].y, (float)X[a].z};
            Mf = fmaxf(Mf, fmaxf(fabsf(Xf[a].x), fmaxf(fabsf(Xf[a].y), fabsf(Xf[a].z))));
          }
          const float err = 80.f * Mf * 5.9604645e-8f;
          const float r = __fadd_ru(__fmul_ru(__fdiv_ru(__fadd_ru(la_f, lb_f), __double2float_rd(1.0 - s)), 1.000001f),
                                    err);
          const float r2m = r * r * 1.004f;
          far = type == 0 ? pt_far_f32(Xf[0], Xf[1], Xf[2], Xf[3], r2m) : ee_far_f32(Xf[0], Xf[1], Xf[2], Xf[3], r2m);
        }
        double la = 0.0, lb = 0.0;
        if (!far) {
          for (int a = 0; a < 4; ++a) {
            const double sp = sqrt(dot(R[a], R[a]));
            if (a < na) la = fmax(la, sp); else lb = fmax(lb, sp);
          }
        }
        const double L = la + lb;              // 0 when proven far: t stays 1
        double t = 1.0;
        if (L > 0.0) {
          const double d0 = pair_distance(type, X);
          if (!(d0 > 0.0)) {
            raise_flag(st, EIPC_FLAG_PENETRATION);
            t = 0.0;
          } else {
            double d = d0;
            t = 0.0;
            while (true) {
              const double tn = t + (1.0 - s) * d / L;
              if (tn >= 1.0) { t = 1.0; break; }
              t = tn;
              V3 P[4];
              for (int a = 0; a < 4; ++a) P[a] = X[a] + R[a] * t;
              d = pair_distance(type, P);
              ++iters;
              if (d <= s * d0) break;
              if (iters >= max_iter) { raise_flag(st, EIPC_FLAG_ACCD_CAP); break; }
            }
          }
        }
        if (t < 1.0) {
          const unsigned long long tb = (unsigned long long)__double_as_longlong(t * kMargin);
          atomicMin(alpha_bits, tb);
          atomicMin(group_bits + T.vgroup[v[0]], tb);   // per-scene bound of a batch
        }
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, adv);
    int tot = iters;
    for (int sh = 16; sh > 0; sh >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, sh);
    if (lane == 0) {
      if (m) atomicAdd(reinterpret_cast<unsigned long long*>(n_adv), (unsigned long long)__popc(m));
      if (tot) atomicAdd(&st->accd_iters, (unsigned long long)tot);
    }
  }
  }
}

__global__ void k_alpha_out(const unsigned long long* bits, double* alpha, const int64_t* n_adv, int64_t* n_out) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *alpha = __longlong_as_double((long long)*bits);
    if (n_out) *n_out = *n_adv;
  }
}

}  // namespace

void accd_launch(eipc_scene* sc, const double* x, const double* dx, const eipc_params& p, double* alpha,
                 int64_t* n_candidates, cudaStream_t s) {
  EIPC_TIMED(sc, kKEmbed, s, (launch(k_pad, blocks_for(sc->nv), kBlock, 0, s, x, dx, sc->nv, sc->x4, sc->dx4, sc->status)));
  int64_t* n_cand = sc->counters + kCntCand;
  int64_t* n_adv = sc->counters + kCntAccd;
  unsigned long long* abits = reinterpret_cast<unsigned long long*>(sc->counters + 12);
  int64_t* queue = sc->counters + kCntCcdQueue;
  zero_ranges(s, {{n_cand, sizeof(int64_t)}, {n_adv, sizeof(int64_t)}, {queue, sizeof(int64_t)}});
  launch(k_alpha_init, blocks_for(sc->n_groups), kBlock, 0, s, abits, sc->group_alpha_bits, sc->n_groups);
  // swept per-vertex boxes over [x, x + dx]; the hierarchies of the last contact-set build
  // are refitted with them when they exist (the topology is reused; only the boxes change)
  EIPC_TIMED(sc, kKBvh, s, vertex_boxes(sc->topo, sc->x4, sc->dx4, 0.0, sc->vbox, nullptr, s));
  if (sc->tri_bvh.built && sc->edge_bvh.built) {
    EIPC_TIMED(sc, kKBvh, s, bvh_refit_pair(sc->tri_bvh, kTri, sc->edge_bvh, kEdge, sc->topo, sc->vbox, s,
                                           sc->tune.refit_variant));
  } else {
    if (sc->tri_bvh.built)
      EIPC_TIMED(sc, kKBvh, s, bvh_refit(sc->tri_bvh, kTri, sc->topo, sc->vbox, s, sc->tune.refit_variant));
    else
      EIPC_TIMED(sc, kKBvh, s, bvh_build(sc->tri_bvh, kTri, sc->topo, sc->x4, sc->dx4, sc->vbox, sc->bounds_ws, sc->sort_hist, s,
                                        sc->tune.refit_variant));
    if (sc->edge_bvh.built)
      EIPC_TIMED(sc, kKBvh, s, bvh_refit(sc->edge_bvh, kEdge, sc->topo, sc->vbox, s, sc->tune.refit_variant));
    else
      EIPC_TIMED(sc, kKBvh, s, bvh_build(sc->edge_bvh, kEdge, sc->topo, sc->x4, sc->dx4, sc->vbox, sc->bounds_ws, sc->sort_hist, s,
                                        sc->tune.refit_variant));
  }
  EIPC_TIMED(sc, kKQuery, s,
             bvh_query(sc->tri_bvh, sc->edge_bvh, sc->topo, sc->vbox, sc->cand, n_cand, sc->cand_cap,
                       sc->status, s, sc->tune.query_threads, sc->tune.query_bps,
                       sc->tune.query_variant));
  EIPC_TIMED(sc, kKCa, s,
             (launch(k_ca, blocks_for(sc->cand_cap, 16, kAccdThreads), kAccdThreads, 0, s, 
                 sc->topo, sc->x4, sc->dx4, sc->cand, n_cand, sc->cand_cap, p.accd_s, p.accd_max_iter, abits, sc->group_alpha_bits, n_adv,
                 sc->status, queue, sc->tune.ccd_tile)));
  launch(k_alpha_out, 1, 32, 0, s, abits, alpha, n_adv, n_candidates);
}

}  // namespace eipc
