// C ABI entry points (include/embipc.h): argument checks, scene creation and workspace
// sizing, and the enqueueing of each call's kernels on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "scene.cuh"
#include "sort.cuh"

using namespace eipc;

namespace {

template <class T>
cudaError_t dalloc(T** p, int64_t n) {
  if (n < 1) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
}

void free_scene(eipc_scene* s) {
  if (!s) return;
  void* ptrs[] = {s->tris, s->edges, s->cage_idx, s->w, s->x_kin4, s->hvp_out, s->edge_key, s->edge_id, s->moll_r2, s->vkin, s->ekin, s->fkin, s->vgroup, s->group_alpha_bits, s->group_count, s->item_group, s->fric_of_pair, s->pair_of_fric, s->lag_key, s->x4, s->dx4, s->x4f, s->vbox, s->vbox_pad, s->cand2,
                  s->tri_bvh.n_dev, s->tri_bvh.nodes, s->tri_bvh.parent, s->tri_bvh.leaf_prim, s->tri_bvh.leaf_info,
                  s->tri_bvh.leaf_box, s->tri_bvh.refit_flag, s->tri_bvh.keys, s->tri_bvh.vals,
                  s->tri_bvh.keys_alt, s->tri_bvh.vals_alt, s->tri_bvh.range, s->tri_bvh.tl_root, s->tri_bvh.up_start,
                  s->tri_bvh.tl_count, s->edge_bvh.n_dev, s->edge_bvh.nodes, s->edge_bvh.leaf_info,
                  s->edge_bvh.parent, s->edge_bvh.leaf_prim, s->edge_bvh.leaf_box, s->edge_bvh.refit_flag,
                  s->edge_bvh.keys, s->edge_bvh.vals, s->edge_bvh.keys_alt, s->edge_bvh.vals_alt, s->edge_bvh.range,
                  s->edge_bvh.tl_root, s->edge_bvh.up_start, s->edge_bvh.tl_count, s->bounds_ws,
                  s->sort_hist, s->cand, s->counters, s->skeys, s->skeys_alt, s->svals, s->svals_alt, s->sd,
                  s->item_nodes, s->item_n, s->rc_h, s->ro_h, s->rc_g, s->ro_g, s->item_E, s->hkeys,
                  s->hkeys_alt, s->hvals, s->hvals_alt, s->hrec, s->seg_flag, s->seg_id, s->seg_start, s->hinv, s->piece, s->hunit,
                  s->gkeys, s->gkeys_alt, s->gvals, s->gvals_alt, s->grec,
                  s->gseg_start, s->scan_partial, s->sum_partial, s->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->timers) {
    s->timers->destroy();
    delete s->timers;
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->aux) cudaStreamDestroy(s->aux);
  delete s;
}

cudaError_t alloc_bvh(Bvh& t, int64_t n) {
  t.n = n;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
  ok(dalloc(&t.n_dev, 1));
  ok(dalloc(&t.nodes, n > 1 ? n - 1 : 1));
  ok(dalloc(&t.parent, 2 * n));
  ok(dalloc(&t.leaf_prim, n));
  ok(dalloc(&t.leaf_info, n));
  ok(dalloc(&t.leaf_box, 6 * n));
  ok(dalloc(&t.refit_flag, n));
  ok(dalloc(&t.keys, n));
  ok(dalloc(&t.vals, n));
  ok(dalloc(&t.keys_alt, n));
  ok(dalloc(&t.vals_alt, n));
  ok(dalloc(&t.range, n > 1 ? n - 1 : 1));
  ok(dalloc(&t.tl_root, n));
  ok(dalloc(&t.up_start, n));
  ok(dalloc(&t.tl_count, 2));
  if (e == cudaSuccess) e = cudaMemcpy(t.n_dev, &n, sizeof(int64_t), cudaMemcpyHostToDevice);
  return e;
}

bool params_ok(const eipc_params* p) {
  return p && p->dhat > 0.0 && p->kappa > 0.0 && p->mu >= 0.0 && p->eps_v > 0.0 && p->h > 0.0 && p->accd_s > 0.0 &&
         p->accd_s < 1.0 && p->accd_max_iter > 0 && (p->flags & ~(EIPC_PARAM_NO_PROJECTION | EIPC_PARAM_DEDUP)) == 0;
}

bool pairs_ok(const eipc_pairs* p) {
  return p && p->capacity >= 0 && p->capacity < (1ll << 31) && p->count &&
         (p->capacity == 0 || (p->type && p->i && p->j && p->d));
}

}  // namespace

extern "C" {

const char* eipc_version(void) { return "embipc 0.1 (sm_103a)"; }

eipc_status eipc_scene_create(int64_t Nv, int64_t F, int64_t E, int64_t Ns, const int32_t* tris,
                              const int32_t* edges, const int32_t* cage_idx, const double* w, const double* x_kin,
                              int64_t cand_capacity, int64_t rec_capacity, eipc_scene** out) {
  if (!out) return EIPC_ERR_INVALID;
  *out = nullptr;
  if (Nv <= 0 || F < 0 || E < 0 || Ns < 0 || Nv >= (1ll << 30) || F >= (1ll << 30) || E >= (1ll << 30) ||
      Ns >= (1ll << 24))
    return EIPC_ERR_INVALID;
  if ((F > 0 && !tris) || (E > 0 && !edges) || !cage_idx || !w || !x_kin) return EIPC_ERR_INVALID;
  // host-side validation of ids
  for (int64_t k = 0; k < 3 * F; ++k)
    if (tris[k] < 0 || tris[k] >= Nv) return EIPC_ERR_INVALID;
  for (int64_t k = 0; k < E; ++k)
    if (edges[2 * k] < 0 || edges[2 * k] >= Nv || edges[2 * k + 1] < 0 || edges[2 * k + 1] >= Nv ||
        edges[2 * k] >= edges[2 * k + 1])
      return EIPC_ERR_INVALID;
  std::vector<uint8_t> vkin(Nv), ekin(E > 0 ? E : 1), fkin(F > 0 ? F : 1);
  for (int64_t v = 0; v < Nv; ++v) {
    bool kin = cage_idx[4 * v] < 0;
    vkin[v] = kin;
    for (int s = 0; s < 4; ++s) {
      int32_t id = cage_idx[4 * v + s];
      if (kin ? (id != -1) : (id < 0 || id >= Ns)) return EIPC_ERR_INVALID;
    }
  }
  for (int64_t e = 0; e < E; ++e) ekin[e] = vkin[edges[2 * e]] && vkin[edges[2 * e + 1]];
  for (int64_t f = 0; f < F; ++f) fkin[f] = vkin[tris[3 * f]] && vkin[tris[3 * f + 1]] && vkin[tris[3 * f + 2]];
  std::vector<double> xk4(4 * Nv, 0.0);
  for (int64_t v = 0; v < Nv; ++v)
    for (int k = 0; k < 3; ++k) xk4[4 * v + k] = vkin[v] ? x_kin[3 * v + k] : 0.0;

  auto* s = new eipc_scene;
  std::memset(s, 0, sizeof(eipc_scene));
  s->timers = new Timers();
  s->nv = Nv; s->nf = F; s->ne = E; s->ns = Ns;
  if (cand_capacity <= 0) cand_capacity = 48 * (Nv + E);
  if (cand_capacity >= (1ll << 31)) cand_capacity = (1ll << 31) - 1;
  if (rec_capacity <= 0) rec_capacity = 1ll << 24;
  if (rec_capacity >= (1ll << 31)) rec_capacity = (1ll << 31) - 1;
  s->cand_cap = cand_capacity;
  // items (contact pairs + lagged friction pairs) each emit at least one record, usually
  // tens: a quarter of the record capacity, at least 4M, bounded by the candidates
  {
    const int64_t want = (rec_capacity / 4) > (1ll << 22) ? (rec_capacity / 4) : (1ll << 22);
    s->item_cap = cand_capacity < want ? cand_capacity : want;
  }
  s->rec_cap = rec_capacity;
  // the gradient records and the per-group energy sort (one key per item) share these
  s->gcap = rec_capacity > s->item_cap ? rec_capacity : s->item_cap;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
  ok(dalloc(&s->tris, 3 * F)); ok(dalloc(&s->edges, 2 * E)); ok(dalloc(&s->cage_idx, 4 * Nv));
  ok(dalloc(&s->w, 4 * Nv)); ok(dalloc(&s->x_kin4, 4 * Nv));
  ok(dalloc(&s->vkin, Nv)); ok(dalloc(&s->ekin, E)); ok(dalloc(&s->fkin, F));
  ok(dalloc(&s->vgroup, Nv)); ok(dalloc(&s->group_alpha_bits, 1)); ok(dalloc(&s->group_count, 4));
  ok(dalloc(&s->x4, 4 * Nv)); ok(dalloc(&s->dx4, 4 * Nv)); ok(dalloc(&s->x4f, 4 * Nv));
  ok(dalloc(&s->vbox, 8 * Nv)); ok(dalloc(&s->vbox_pad, 8 * Nv));
  ok(alloc_bvh(s->tri_bvh, F));
  ok(alloc_bvh(s->edge_bvh, E));
  ok(dalloc(&s->bounds_ws, 8));
  ok(dalloc(&s->sort_hist, (int64_t)sort_hist_entries()));
  ok(dalloc(&s->cand, s->cand_cap));
  ok(dalloc(&s->cand2, s->cand_cap));
  ok(dalloc(&s->counters, kCntN));
  ok(dalloc(&s->skeys, s->cand_cap)); ok(dalloc(&s->skeys_alt, s->cand_cap));
  ok(dalloc(&s->svals, s->cand_cap)); ok(dalloc(&s->svals_alt, s->cand_cap)); ok(dalloc(&s->sd, s->cand_cap));
  ok(dalloc(&s->item_nodes, 16 * s->item_cap)); ok(dalloc(&s->item_n, s->item_cap));
  ok(dalloc(&s->item_group, s->item_cap));
  ok(dalloc(&s->fric_of_pair, s->item_cap)); ok(dalloc(&s->pair_of_fric, s->item_cap));
  ok(dalloc(&s->lag_key, s->item_cap));
  ok(dalloc(&s->rc_h, s->item_cap)); ok(dalloc(&s->ro_h, s->item_cap));
  ok(dalloc(&s->rc_g, s->item_cap)); ok(dalloc(&s->ro_g, s->item_cap)); ok(dalloc(&s->item_E, s->item_cap));
  ok(dalloc(&s->hkeys, s->rec_cap)); ok(dalloc(&s->hkeys_alt, s->rec_cap));
  ok(dalloc(&s->hvals, s->rec_cap)); ok(dalloc(&s->hvals_alt, s->rec_cap)); ok(dalloc(&s->hrec, kHRecStride * s->rec_cap));
  ok(dalloc(&s->hvp_out, 3 * (Ns + 64)));
  ok(dalloc(&s->seg_flag, s->rec_cap)); ok(dalloc(&s->seg_id, s->rec_cap)); ok(dalloc(&s->seg_start, s->rec_cap));
  ok(dalloc(&s->hinv, s->rec_cap));
  {
    const int64_t pr = s->rec_cap + s->rec_cap / 32 + 2;
    ok(dalloc(&s->piece, 9 * pr));
  }
  ok(dalloc(&s->hunit, s->rec_cap + 1));
  ok(dalloc(&s->gkeys, s->gcap)); ok(dalloc(&s->gkeys_alt, s->gcap));
  ok(dalloc(&s->gvals, s->gcap)); ok(dalloc(&s->gvals_alt, s->gcap)); ok(dalloc(&s->grec, kGRecStride * s->gcap));
  ok(dalloc(&s->gseg_start, s->gcap));
  ok(dalloc(&s->edge_key, E > 0 ? E : 1)); ok(dalloc(&s->edge_id, E > 0 ? E : 1));
  ok(dalloc(&s->moll_r2, E > 0 ? E : 1));
  ok(dalloc(&s->scan_partial, 2 * (kScanBlocks + 1))); ok(dalloc(&s->sum_partial, kScanBlocks));
  ok(dalloc(&s->status, 1));
  ok(cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking));
  ok(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
  ok(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
  if (e != cudaSuccess) {
    free_scene(s);
    cudaGetLastError();
    return EIPC_ERR_NOMEM;
  }
  ok(cudaMemcpy(s->tris, tris, sizeof(int32_t) * 3 * F, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->edges, edges, sizeof(int32_t) * 2 * E, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->cage_idx, cage_idx, sizeof(int32_t) * 4 * Nv, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->w, w, sizeof(double) * 4 * Nv, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->x_kin4, xk4.data(), sizeof(double) * 4 * Nv, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->vkin, vkin.data(), Nv, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->ekin, ekin.data(), E, cudaMemcpyHostToDevice));
  ok(cudaMemcpy(s->fkin, fkin.data(), F, cudaMemcpyHostToDevice));
  {
    // edge lookup table for the deduplicated pair set: keys a * Nv + b (a < b) sorted
    std::vector<std::pair<uint64_t, int32_t>> ek((size_t)E);
    for (int64_t e2 = 0; e2 < E; ++e2) {
      int64_t a = edges[2 * e2], b = edges[2 * e2 + 1];
      if (a > b) std::swap(a, b);
      ek[(size_t)e2] = {(uint64_t)a * (uint64_t)Nv + (uint64_t)b, (int32_t)e2};
    }
    std::sort(ek.begin(), ek.end());
    std::vector<uint64_t> keys((size_t)E);
    std::vector<int32_t> ids((size_t)E);
    for (size_t q = 0; q < ek.size(); ++q) { keys[q] = ek[q].first; ids[q] = ek[q].second; }
    if (E > 0) {
      ok(cudaMemcpy(s->edge_key, keys.data(), sizeof(uint64_t) * E, cudaMemcpyHostToDevice));
      ok(cudaMemcpy(s->edge_id, ids.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice));
    }
  }
  ok(cudaMemset(s->counters, 0, sizeof(int64_t) * kCntN));
  ok(cudaMemset(s->status, 0, sizeof(DevStatus)));
  ok(cudaMemset(s->vgroup, 0, sizeof(int32_t) * Nv));
  s->n_groups = 1;
  ok(cudaMemset(s->x4, 0, sizeof(double) * 4 * Nv));
  ok(cudaMemset(s->dx4, 0, sizeof(double) * 4 * Nv));
  if (e != cudaSuccess) {
    free_scene(s);
    cudaGetLastError();
    return EIPC_ERR_CUDA;
  }
  Topo& T = s->topo;
  T.nv = Nv; T.ne = E; T.nf = F;
  T.tris = s->tris; T.edges = s->edges; T.vkin = s->vkin; T.ekin = s->ekin; T.fkin = s->fkin;
  T.vgroup = s->vgroup;
  T.bits_i = bits_for((uint64_t)(Nv > E ? Nv : E));
  T.bits_j = bits_for((uint64_t)(F > E ? F : E));
  s->bits_h = bits_for((uint64_t)Ns * (uint64_t)(Ns + 1) / 2);    // upper keys (eval.cu)
  s->bits_g = bits_for((uint64_t)Ns);
  {
    int64_t mx = Nv > E ? Nv : E;
    mx = mx > F ? mx : F;
    s->feat_bits = bits_for((uint64_t)mx);
  }
  s->rebuild_interval = 8;
  // the scene was zero-filled after construction: every launch-shape default is set here
  s->tune.eval_threads = 128; s->tune.eval_bps = 16; s->tune.eval_variant = 2; s->tune.eval_tile = 32;
  s->tune.ccd_tile = 128;
  s->tune.query_threads = 128; s->tune.query_bps = 24; s->tune.query_variant = 2; s->tune.refit_variant = 2;
  s->contact_refits = 0;
  *out = s;
  return EIPC_OK;
}

void eipc_scene_destroy(eipc_scene* scene) {
  if (!scene) return;
  cudaDeviceSynchronize();
  free_scene(scene);
}

eipc_status eipc_embed(eipc_scene* sc, const double* q, double* x, int32_t displacement, eipc_stream stream) {
  if (!sc || (!q && sc->ns > 0) || !x) return EIPC_ERR_INVALID;
  embed_launch(sc, q, x, 0, displacement, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_build_candidates(eipc_scene* sc, const double* q, const eipc_params* p, eipc_pairs* out,
                                  eipc_stream stream) {
  if (!sc || (!q && sc->ns > 0) || !params_ok(p) || !pairs_ok(out)) return EIPC_ERR_INVALID;
  pairs_launch(sc, q, *p, *out, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_friction_lag(eipc_scene* sc, const double* q_n, const eipc_pairs* pairs_n, const eipc_params* p,
                              eipc_lag* out, eipc_stream stream) {
  if (!sc || (!q_n && sc->ns > 0) || !params_ok(p) || !pairs_ok(pairs_n) || !out || !out->count ||
      out->capacity < 0 || (out->capacity > 0 && (!out->v || !out->gamma || !out->n || !out->anchor || !out->lambda)))
    return EIPC_ERR_INVALID;
  lag_launch(sc, q_n, *pairs_n, *p, *out, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_eval_contact(eipc_scene* sc, const double* q, const eipc_pairs* pairs, const eipc_lag* lag,
                              const eipc_params* p, double* E, double* g_r, eipc_bsr* H, eipc_stream stream) {
  if (!sc || (!q && sc->ns > 0) || !params_ok(p) || !pairs_ok(pairs) || !E || !g_r || !H || !H->row_ptr ||
      !H->nnzb || H->capacity < 0 || (H->capacity > 0 && (!H->col || !H->val)))
    return EIPC_ERR_INVALID;
  if (lag && (!lag->count || lag->capacity < 0 || (lag->capacity > 0 && (!lag->v || !lag->gamma || !lag->n ||
                                                                          !lag->anchor || !lag->lambda))))
    return EIPC_ERR_INVALID;
  eval_launch(sc, q, *pairs, lag, *p, E, g_r, *H, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_contact_hvp(eipc_scene* sc, const double* q, const eipc_pairs* pairs, const eipc_lag* lag,
                             const eipc_params* p, const double* v, const double* kin_dir, double* out_r,
                             double* out_kin, eipc_stream stream) {
  if (!sc || (!q && sc->ns > 0) || !params_ok(p) || !pairs_ok(pairs) || (!v && sc->ns > 0) ||
      (!out_r && sc->ns > 0))
    return EIPC_ERR_INVALID;
  if (lag && (!lag->count || lag->capacity < 0 || (lag->capacity > 0 && (!lag->v || !lag->gamma || !lag->n ||
                                                                          !lag->anchor || !lag->lambda))))
    return EIPC_ERR_INVALID;
  if (kin_dir && !(std::isfinite(kin_dir[0]) && std::isfinite(kin_dir[1]) && std::isfinite(kin_dir[2])))
    return EIPC_ERR_INVALID;
  hvp_launch(sc, q, *pairs, lag, *p, v, kin_dir, out_r, out_kin, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_bsr_spmv(int64_t nrows, const int32_t* row_ptr, const int32_t* col, const double* val,
                          const double* x, double alpha, double beta, double* y, eipc_stream stream) {
  if (nrows < 0 || (nrows > 0 && (!row_ptr || !x || !y)) || !std::isfinite(alpha) || !std::isfinite(beta))
    return EIPC_ERR_INVALID;
  bsr_spmv_launch(nrows, row_ptr, col, val, x, alpha, beta, y, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_scene_set_mollifier(eipc_scene* sc, const double* x_rest, double factor, eipc_stream stream) {
  if (!sc || !(factor >= 0.0) || !std::isfinite(factor) || (factor > 0.0 && !x_rest)) return EIPC_ERR_INVALID;
  if (factor > 0.0 && sc->ne > 0) {
    // squared rest lengths on the device, then a synchronous check that all are positive
    cudaStream_t s = (cudaStream_t)stream;
    int64_t* bad = sc->counters + kCntMollBad;
    if (cudaMemsetAsync(bad, 0, sizeof(int64_t), s) != cudaSuccess) return EIPC_ERR_CUDA;
    mollifier_rest_launch(sc, x_rest, bad, s);
    int64_t nbad = -1;
    if (cudaMemcpyAsync(&nbad, bad, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return EIPC_ERR_CUDA;
    if (nbad != 0) {
      sc->moll_factor = 0.0;
      return EIPC_ERR_INVALID;
    }
  }
  sc->moll_factor = factor;
  return EIPC_OK;
}

eipc_status eipc_candidates_read(eipc_scene* sc, int32_t* type, int32_t* i, int32_t* j, int64_t capacity,
                                 int64_t* n, eipc_stream stream) {
  if (!sc || !n || capacity < 0 || (capacity > 0 && (!type || !i || !j))) return EIPC_ERR_INVALID;
  candidates_launch(sc, type, i, j, capacity, n, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_scene_set_kinematic(eipc_scene* sc, const double* x_kin, eipc_stream stream) {
  if (!sc || !x_kin) return EIPC_ERR_INVALID;
  set_kinematic_launch(sc, x_kin, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_accd_toi(eipc_scene* sc, const double* x, const double* dx, const eipc_params* p, double* alpha,
                          int64_t* n_candidates, eipc_stream stream) {
  if (!sc || !x || !dx || !params_ok(p) || !alpha) return EIPC_ERR_INVALID;
  accd_launch(sc, x, dx, *p, alpha, n_candidates, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_status_read(eipc_scene* sc, eipc_stream stream, int32_t* flags, int64_t* needed,
                             int64_t* accd_iters) {
  if (!sc) return EIPC_ERR_INVALID;
  DevStatus h;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, sc->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return EIPC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return EIPC_ERR_CUDA;
  if (cudaMemsetAsync(sc->status, 0, sizeof(DevStatus), s) != cudaSuccess) return EIPC_ERR_CUDA;
  if (flags) *flags = h.flags;
  if (needed) {
    needed[0] = h.need_pairs; needed[1] = h.need_cand; needed[2] = h.need_rec; needed[3] = h.need_bsr;
  }
  if (accd_iters) *accd_iters = (int64_t)h.accd_iters;
  return EIPC_OK;
}

eipc_status eipc_work_counts(eipc_scene* sc, eipc_stream stream, int64_t* out, int32_t n) {
  if (!sc || n < 0 || n > EIPC_WORK_COUNTS || (n > 0 && !out)) return EIPC_ERR_INVALID;
  int64_t c[kCntN];
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c, sc->counters, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess) return EIPC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return EIPC_ERR_CUDA;
  const int64_t v[EIPC_WORK_COUNTS] = {c[kCntCand], c[kCntScreened], c[kCntSurv], c[kCntItems], c[kCntRecH],
                                       c[kCntRecG],  c[kCntSegH],     c[kCntSegG], c[kCntAccd]};
  for (int32_t k = 0; k < n; ++k) out[k] = v[k];
  return EIPC_OK;
}

eipc_status eipc_timing_enable(eipc_scene* sc, uint32_t mask) {
  if (!sc) return EIPC_ERR_INVALID;
  if (mask) sc->timers->create();
  sc->timers->mask = mask;
  return EIPC_OK;
}

eipc_status eipc_timing_read(eipc_scene* sc, double* total_ms, int64_t* launches, int32_t n) {
  if (!sc || n < 0 || (n > 0 && (!total_ms || !launches))) return EIPC_ERR_INVALID;
  for (int k = 0; k < kKNum; ++k) sc->timers->drain(k);
  for (int k = 0; k < n && k < kKNum; ++k) {
    total_ms[k] = sc->timers->total_ms[k];
    launches[k] = sc->timers->launches[k];
    sc->timers->total_ms[k] = 0.0;
    sc->timers->launches[k] = 0;
  }
  return EIPC_OK;
}

eipc_status eipc_scene_set_groups(eipc_scene* sc, const int32_t* vertex_group, int32_t n_groups) {
  if (!sc || !vertex_group || n_groups < 1 || n_groups > (1 << 24)) return EIPC_ERR_INVALID;
  for (int64_t v = 0; v < sc->nv; ++v)
    if (vertex_group[v] < 0 || vertex_group[v] >= n_groups) return EIPC_ERR_INVALID;
  // every primitive must lie in one group (a pair never spans two scenes)
  std::vector<int32_t> tr(3 * sc->nf), ed(2 * sc->ne);
  if (cudaMemcpy(tr.data(), sc->tris, sizeof(int32_t) * tr.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(ed.data(), sc->edges, sizeof(int32_t) * ed.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return EIPC_ERR_CUDA;
  for (int64_t f = 0; f < sc->nf; ++f)
    if (vertex_group[tr[3 * f]] != vertex_group[tr[3 * f + 1]] || vertex_group[tr[3 * f]] != vertex_group[tr[3 * f + 2]])
      return EIPC_ERR_INVALID;
  for (int64_t e = 0; e < sc->ne; ++e)
    if (vertex_group[ed[2 * e]] != vertex_group[ed[2 * e + 1]]) return EIPC_ERR_INVALID;
  unsigned long long* gb = nullptr;
  int64_t* gc = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&gb), sizeof(unsigned long long) * n_groups) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&gc), sizeof(int64_t) * (2 * (size_t)n_groups + 2)) != cudaSuccess) {
    if (gb) cudaFree(gb);
    cudaGetLastError();
    return EIPC_ERR_NOMEM;
  }
  if (cudaMemcpy(sc->vgroup, vertex_group, sizeof(int32_t) * sc->nv, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(gb); cudaFree(gc);
    return EIPC_ERR_CUDA;
  }
  cudaFree(sc->group_alpha_bits);
  cudaFree(sc->group_count);
  sc->group_alpha_bits = gb;
  sc->group_count = gc;
  sc->n_groups = n_groups;
  sc->tri_bvh.built = sc->edge_bvh.built = false;   // leaf records carry the group
  return EIPC_OK;
}

eipc_status eipc_group_energy(eipc_scene* sc, double* E_groups, eipc_stream stream) {
  if (!sc || !E_groups) return EIPC_ERR_INVALID;
  group_energy_launch(sc, E_groups, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_group_alpha(eipc_scene* sc, double* alpha_groups, eipc_stream stream) {
  if (!sc || !alpha_groups) return EIPC_ERR_INVALID;
  group_alpha_launch(sc, alpha_groups, (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}

eipc_status eipc_set_launch(eipc_scene* sc, int32_t kernel, int32_t threads, int32_t blocks_per_sm,
                            int32_t variant) {
  if (!sc || blocks_per_sm < 1 || blocks_per_sm > 64) return EIPC_ERR_INVALID;
  if (kernel == 0) {
    if ((threads != 64 && threads != 128) || variant < 2 || variant > 4) return EIPC_ERR_INVALID;
    sc->tune.eval_threads = threads;
    sc->tune.eval_bps = blocks_per_sm;
    sc->tune.eval_variant = variant;
    return EIPC_OK;
  }
  if (kernel == 1) {
    if ((threads != 64 && threads != 128 && threads != 256) || (variant != 2 && variant != 3)) return EIPC_ERR_INVALID;
    sc->tune.query_threads = threads;
    sc->tune.query_bps = blocks_per_sm;
    sc->tune.query_variant = variant;
    return EIPC_OK;
  }
  if (kernel == 2) {
    if (threads != 256 || variant < 0 || variant > 2) return EIPC_ERR_INVALID;
    sc->tune.refit_variant = variant;
    return EIPC_OK;
  }
  if (kernel == 3 || kernel == 4) {
    // work-queue tiles: `threads` = items a warp claims at a time (32, 64, 128 or 256)
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256) return EIPC_ERR_INVALID;
    if (kernel == 3) sc->tune.eval_tile = threads;
    else sc->tune.ccd_tile = threads;
    return EIPC_OK;
  }
  return EIPC_ERR_INVALID;
}

eipc_status eipc_set_rebuild_interval(eipc_scene* sc, int32_t n) {
  if (!sc || n < 1) return EIPC_ERR_INVALID;
  sc->rebuild_interval = n;
  sc->contact_refits = 0;
  return EIPC_OK;
}

int64_t eipc_launch_count(void) { return (int64_t)g_launches.load(); }

void eipc_set_programmatic_launch(int32_t on) { g_programmatic.store(on ? 1 : 0); }

const char* eipc_kernel_name(int32_t id) {
  static const char* names[kKNum] = {"embed", "bvh_build", "bvh_query", "narrow_phase", "pair_sort", "friction_lag",
                                     "stencil_nodes", "eval_barrier", "eval_friction", "hessian_reduce",
                                     "gradient_reduce", "energy_sum", "ccd_advance", "eval_kernels"};
  return (id >= 0 && id < kKNum) ? names[id] : "";
}

}  // extern "C"
