// LBVH build (Morton sort, Karras hierarchy, bottom-up refit) and traversal.
#include "bvh.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

// order-preserving map float -> int for atomic min / max
__device__ __forceinline__ int32_t f2ord(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int32_t i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bounds_init(int32_t* b) {
  pdl_entry();
  if (threadIdx.x < 3) b[threadIdx.x] = 0x7fffffff;
  else if (threadIdx.x < 6) b[threadIdx.x] = (int32_t)0x80000000;
}

// scene box over all vertex positions (and their swept ends)
__global__ void __launch_bounds__(kBlock) k_bounds(const double* __restrict__ x4, const double* __restrict__ dx4,
                                                   int64_t nv, int32_t* __restrict__ b) {
  pdl_entry();
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += grid_stride()) {
    V3 p = load_x(x4, (int32_t)v);
    double c[3] = {p.x, p.y, p.z};
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], __double2float_rd(c[k]));
      hi[k] = fmaxf(hi[k], __double2float_ru(c[k]));
    }
    if (dx4) {
      V3 d = load_x(dx4, (int32_t)v);
      double e[3] = {p.x + d.x, p.y + d.y, p.z + d.z};
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(lo[k], __double2float_rd(e[k]));
        hi[k] = fmaxf(hi[k], __double2float_ru(e[k]));
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) {
      atomicMin(&b[k], f2ord(lo[k]));
      atomicMax(&b[3 + k], f2ord(hi[k]));
    }
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Per-vertex FP32 boxes, rounded outward from the FP64 positions (swept over x + dx when
// dx4 is given): vbox[8v..8v+5] = lo xyz, hi xyz (rows of 8 floats), and vbox_pad the same
// grown by pad in FP64 before rounding.  Outward rounding and the pad subtraction are
// monotone, so the min / max over a primitive's vertices of these boxes is bit for bit the
// box made from the primitive's FP64 positions (FP64 min / max, padded, rounded outward):
// the hierarchy and traversal read these instead of recomputing FP64 minima per primitive.
__global__ void __launch_bounds__(kBlock) k_vertex_boxes(int64_t nv, const double* __restrict__ x4,
                                                         const double* __restrict__ dx4, double pad,
                                                         float* __restrict__ vbox, float* __restrict__ vbox_pad) {
  pdl_entry();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += grid_stride()) {
    const V3 p = load_x(x4, (int32_t)v);
    double lo[3] = {p.x, p.y, p.z}, hi[3] = {p.x, p.y, p.z};
    if (dx4) {
      const V3 d = load_x(dx4, (int32_t)v);
      const double e[3] = {p.x + d.x, p.y + d.y, p.z + d.z};
      for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], e[k]); hi[k] = fmax(hi[k], e[k]); }
    }
    float4* o = reinterpret_cast<float4*>(vbox + 8 * v);
    o[0] = make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]), __double2float_rd(lo[2]),
                       __double2float_ru(hi[0]));
    o[1] = make_float4(__double2float_ru(hi[1]), __double2float_ru(hi[2]), 0.f, 0.f);
    if (vbox_pad) {
      float4* op = reinterpret_cast<float4*>(vbox_pad + 8 * v);
      op[0] = make_float4(__double2float_rd(__dsub_rd(lo[0], pad)), __double2float_rd(__dsub_rd(lo[1], pad)),
                          __double2float_rd(__dsub_rd(lo[2], pad)), __double2float_ru(__dadd_ru(hi[0], pad)));
      op[1] = make_float4(__double2float_ru(__dadd_ru(hi[1], pad)), __double2float_ru(__dadd_ru(hi[2], pad)), 0.f, 0.f);
    }
  }
}

// box of up to three vertices from the per-vertex boxes (ids < 0 are skipped)
__device__ __forceinline__ void verts_box(const float* __restrict__ vbox, int32_t a, int32_t b, int32_t c,
                                          float lo[3], float hi[3]) {
  for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
  const int32_t v[3] = {a, b, c};
  for (int s = 0; s < 3; ++s) {
    if (v[s] < 0) continue;
    const float4 p = __ldg(reinterpret_cast<const float4*>(vbox + 8 * (int64_t)v[s]));
    const float4 q = __ldg(reinterpret_cast<const float4*>(vbox + 8 * (int64_t)v[s]) + 1);
    lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.w); hi[1] = fmaxf(hi[1], q.x); hi[2] = fmaxf(hi[2], q.y);
  }
}

// box of one primitive from the per-vertex boxes
__device__ __forceinline__ void prim_box_v(PrimKind kind, int64_t i, const Topo& T, const float* __restrict__ vbox,
                                           float lo[3], float hi[3]) {
  if (kind == kVertex) verts_box(vbox, (int32_t)i, -1, -1, lo, hi);
  else if (kind == kEdge) verts_box(vbox, T.edges[2 * i], T.edges[2 * i + 1], -1, lo, hi);
  else verts_box(vbox, T.tris[3 * i], T.tris[3 * i + 1], T.tris[3 * i + 2], lo, hi);
}

__global__ void __launch_bounds__(kBlock) k_leaves(PrimKind kind, int64_t n, Topo T, const float* __restrict__ vbox,
                                                   const int32_t* __restrict__ b,
                                                   float* __restrict__ leaf_box, uint64_t* __restrict__ keys,
                                                   uint32_t* __restrict__ vals) {
  pdl_entry();
  float blo[3], bext[3];
  for (int k = 0; k < 3; ++k) {
    blo[k] = ord2f(b[k]);
    float e = ord2f(b[3 + k]) - blo[k];
    bext[k] = e > 0.f ? e : 1.f;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += grid_stride()) {
    float lo[3], hi[3];
    prim_box_v(kind, i, T, vbox, lo, hi);
    uint32_t code = 0;
    for (int k = 0; k < 3; ++k) {
      float c = (0.5f * (lo[k] + hi[k]) - blo[k]) / bext[k];
      c = fminf(fmaxf(c, 0.f), 1.f);
      uint32_t q = (uint32_t)fminf(c * 1024.f, 1023.f);
      code |= spread10(q) << (2 - k);
    }
    for (int k = 0; k < 3; ++k) { leaf_box[6 * i + k] = lo[k]; leaf_box[6 * i + 3 + k] = hi[k]; }
    keys[i] = code;
    vals[i] = (uint32_t)i;
  }
}

__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = k[i], b = k[j];
  if (a == b) return 64 + __clzll((unsigned long long)(i ^ j));
  return __clzll((unsigned long long)(a ^ b));
}

// Karras 2012: internal node i covers a key range; its split is the highest differing bit.
__global__ void __launch_bounds__(kBlock) k_internal(const uint64_t* __restrict__ keys, int64_t n,
                                                     BvhNode* __restrict__ nodes, int32_t* __restrict__ parent,
                                                     int2* __restrict__ range) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1; i += grid_stride()) {
    int dir = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - dir);
    int64_t lmax = 2;
    while (delta(keys, n, i, i + lmax * dir) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
      if (delta(keys, n, i, i + (l + t) * dir) > dmin) l += t;
    int64_t j = i + l * dir;
    int dnode = delta(keys, n, i, j);
    int64_t s = 0;
    for (int64_t div = 2;; div *= 2) {
      int64_t t = (l + div - 1) / div;
      if (delta(keys, n, i, i + (s + t) * dir) > dnode) s += t;
      if (t == 1) break;
    }
    int64_t gamma = i + s * dir + (dir < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int32_t c0 = (lo == gamma) ? ~(int32_t)gamma : (int32_t)gamma;
    int32_t c1 = (hi == gamma + 1) ? ~(int32_t)(gamma + 1) : (int32_t)(gamma + 1);
    nodes[i].c0 = c0;
    nodes[i].c1 = c1;
    nodes[i].split = (int32_t)gamma;   // last leaf position under child 0
    range[i] = make_int2((int32_t)lo, (int32_t)hi);
    parent[c0 >= 0 ? c0 : (n - 1 + ~c0)] = (int32_t)(i << 1);
    parent[c1 >= 0 ? c1 : (n - 1 + ~c1)] = (int32_t)(i << 1) | 1;
  }
}

__device__ __forceinline__ uint8_t prim_kin(PrimKind kind, const Topo& T, int64_t p) {
  return kind == kTri ? T.fkin[p] : (kind == kEdge ? T.ekin[p] : T.vkin[p]);
}

// The per-leaf records of a build, in leaf (Morton) order for the traversal: the primitive,
// and its vertex ids with (kinematic flag | scene group << 1).  Returns the kinematic flag.
__device__ __forceinline__ int write_leaf_record(PrimKind kind, const Topo& T, int32_t prim, int64_t l,
                                                 int32_t* __restrict__ leaf_prim, int4* __restrict__ leaf_info) {
  leaf_prim[l] = prim;
  const int kin = prim_kin(kind, T, prim);
  if (kind == kTri) {
    const int32_t v0 = T.tris[3 * (int64_t)prim];
    leaf_info[l] = make_int4(v0, T.tris[3 * (int64_t)prim + 1], T.tris[3 * (int64_t)prim + 2], kin | (T.vgroup[v0] << 1));
  } else {
    const int32_t v0 = T.edges[2 * (int64_t)prim];
    leaf_info[l] = make_int4(v0, T.edges[2 * (int64_t)prim + 1], -1, kin | (T.vgroup[v0] << 1));
  }
  return kin;
}

template <bool first>
__device__ __forceinline__ void write_child(BvhNode* nd, int slot, const float lo[3], const float hi[3], int kin) {
  float* l = slot ? nd->lo1 : nd->lo0;
  float* h = slot ? nd->hi1 : nd->hi0;
  for (int k = 0; k < 3; ++k) { __stcg(&l[k], lo[k]); __stcg(&h[k], hi[k]); }
  if (first && kin) atomicOr(&nd->kin, 1 << slot);
}

// Arrival counter of the bottom-up refit with release-acquire semantics at device scope:
// the child box a thread stored before its increment is visible to the thread whose
// increment comes second, which then reads both boxes.
__device__ __forceinline__ int32_t arrive_acq_rel(int32_t* f) {
  int32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(f) : "memory");
  return old;
}

template <bool fences>
__device__ __forceinline__ int32_t arrive(int32_t* f) {
  if (fences) {
    __threadfence();
    return atomicAdd(f, 1);
  }
  return arrive_acq_rel(f);
}

// leaf boxes in leaf order, for refitting an existing hierarchy; the leaf's vertex ids
// come from its leaf record (coalesced) rather than the primitive tables
// FP32 box of one leaf from the per-vertex boxes of its leaf record's vertex ids
__device__ __forceinline__ void leaf_box_of(int4 li, const float* __restrict__ vbox, float lo[3], float hi[3]) {
  verts_box(vbox, li.x, li.y, li.z, lo, hi);
}

__global__ void __launch_bounds__(kBlock) k_leaf_boxes(int64_t n, const int4* __restrict__ leaf_info,
                                                       const float* __restrict__ vbox, float* __restrict__ leaf_box) {
  pdl_entry();
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += grid_stride()) {
    float lo[3], hi[3];
    leaf_box_of(leaf_info[l], vbox, lo, hi);
    float2* o = reinterpret_cast<float2*>(leaf_box + 6 * l);
    o[0] = make_float2(lo[0], lo[1]);
    o[1] = make_float2(lo[2], hi[0]);
    o[2] = make_float2(hi[1], hi[2]);
  }
}

// Bottom-up refit: the second child to finish a node unions both child boxes and
// carries on upward; the first one stops.  No thread ever waits on another.  On a build
// (`first`) it also writes the per-leaf records and the kinematic bits, which a refit of
// the same hierarchy leaves as they are.  Leaf boxes are indexed by primitive on a build
// (written by the Morton pass) and by leaf on a refit (k_leaf_boxes).
template <bool first, bool fences>
__global__ void __launch_bounds__(kBlock) k_refit(PrimKind kind, int64_t n, Topo T, const uint32_t* __restrict__ sorted,
                                                  const float* __restrict__ leaf_box, BvhNode* nodes,
                                                  const int32_t* __restrict__ parent, int32_t* leaf_prim,
                                                  int4* __restrict__ leaf_info, int32_t* flag) {
  pdl_entry();
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += grid_stride()) {
    int kin = 0;
    float lo[3], hi[3];
    if (first) {
      const int32_t prim = (int32_t)sorted[l];
      kin = write_leaf_record(kind, T, prim, l, leaf_prim, leaf_info);
      for (int k = 0; k < 3; ++k) { lo[k] = leaf_box[6 * prim + k]; hi[k] = leaf_box[6 * prim + 3 + k]; }
    } else {
      const float2* b = reinterpret_cast<const float2*>(leaf_box + 6 * l);
      const float2 a0 = b[0], a1 = b[1], a2 = b[2];
      lo[0] = a0.x; lo[1] = a0.y; lo[2] = a1.x; hi[0] = a1.y; hi[1] = a2.x; hi[2] = a2.y;
    }
    if (n == 1) continue;
    int32_t ps = parent[n - 1 + l];
    int32_t node = ps >> 1;
    write_child<first>(&nodes[node], ps & 1, lo, hi, kin);
    int32_t up = node ? parent[node] : 0;       // fetched before the arrival, not after it
    if (arrive<fences>(&flag[node]) == 0) continue;
    for (int64_t step = 0; step < n; ++step) {   // a root path has at most n-1 nodes
      if (fences) __threadfence();
      const BvhNode* nd = &nodes[node];
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(__ldcg(&nd->lo0[k]), __ldcg(&nd->lo1[k]));
        hi[k] = fmaxf(__ldcg(&nd->hi0[k]), __ldcg(&nd->hi1[k]));
      }
      if (first) kin = (__ldcg(&nd->kin) & 3) == 3;
      if (node == 0) break;
      ps = up;
      node = ps >> 1;
      write_child<first>(&nodes[node], ps & 1, lo, hi, kin);
      up = node ? parent[node] : 0;
      if (arrive<fences>(&flag[node]) == 0) break;
    }
  }
}

// ---------------------------------------------------------------- two-phase refit
// Every subtree covers a contiguous leaf range and its internal nodes carry indices inside
// that range.  At build time the tree is cut into treelets: subtrees of at most kTreelet
// leaves whose parent covers more.  A refit then (A) refits each treelet with one warp:
// its leaf boxes, leaf parents and node links are loaded coalesced into shared memory and
// the bottom-up union runs on shared-memory arrival counters, with no dependent global
// loads; and (B) climbs from the treelet roots (and the few leaves hanging directly off
// larger nodes) with the release-acquire counters.  Box unions are exact, so the boxes
// are those of any other refit order.

// On a build refitted by treelets (leaf_prim not null) it also writes the leaf records,
// which both refit phases read.
__global__ void __launch_bounds__(kBlock) k_treelet_lists(int64_t n, const int2* __restrict__ range,
                                                          const int32_t* __restrict__ parent, int32_t* __restrict__ tl_root,
                                                          int32_t* __restrict__ up_start, int32_t* __restrict__ count,
                                                          PrimKind kind, Topo T, const uint32_t* __restrict__ sorted,
                                                          int32_t* __restrict__ leaf_prim, int4* __restrict__ leaf_info) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * n - 1; i += grid_stride()) {
    if (i < n - 1) {                              // internal node i
      const int2 r = range[i];
      const int64_t size = (int64_t)r.y - r.x + 1;
      const int64_t psize = (i == 0) ? INT64_MAX : (int64_t)range[parent[i] >> 1].y - range[parent[i] >> 1].x + 1;
      if (size <= kTreelet && psize > kTreelet) {
        tl_root[atomicAdd(&count[0], 1)] = (int32_t)i;
        up_start[atomicAdd(&count[1], 1)] = (int32_t)i;
      }
    } else {                                      // leaf l = i - (n - 1)
      const int64_t l = i - (n - 1);
      if (leaf_prim) write_leaf_record(kind, T, (int32_t)sorted[l], l, leaf_prim, leaf_info);
      const int32_t p = parent[i] >> 1;
      if ((int64_t)range[p].y - range[p].x + 1 > kTreelet) up_start[atomicAdd(&count[1], 1)] = ~(int32_t)l;
    }
  }
}

constexpr int kTreeletWarps = kBlock / 32;

// What the two-phase refit needs of one tree; n <= 1 marks an absent tree.
struct RefitView {
  int64_t n;
  const int32_t* tl_root;
  const int32_t* up_start;
  const int32_t* count;      // [2]: treelet roots, upper starts
  const int2* range;
  const int32_t* parent;
  const int4* leaf_info;
  BvhNode* nodes;
  int32_t* flag;
};

__host__ __device__ __forceinline__ RefitView refit_view(const Bvh& t) {
  return RefitView{t.n, t.tl_root, t.up_start, t.tl_count, t.range, t.parent, t.leaf_info, t.nodes, t.refit_flag};
}

// Phase A of the refit of up to two trees in one launch: one warp per treelet, lane l
// computing leaf l's box from the positions and climbing in shared memory.  The grid also
// clears both trees' arrival counters for phase B.  On a build (`first`) it also sets each
// node's kinematic bits (bit s: every primitive under child s is kinematic), which a refit
// leaves as they are.
template <bool first>
__global__ void __launch_bounds__(kBlock) k_treelet_refit(RefitView A, RefitView B, const float* __restrict__ vbox) {
  pdl_entry();
  __shared__ float sbox[kTreeletWarps][kTreelet][2][6];
  __shared__ int scnt[kTreeletWarps][kTreelet];
  __shared__ int spar[kTreeletWarps][kTreelet];
  __shared__ int skin[kTreeletWarps][kTreelet];
  const int nA = A.n > 1 ? (int)A.n : 0, nB = B.n > 1 ? (int)B.n : 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)nA + nB; i += grid_stride()) {
    if (i < nA) A.flag[i] = 0;
    else B.flag[i - nA] = 0;
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntA = nA ? A.count[0] : 0, ntB = nB ? B.count[0] : 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntA + ntB; w += nw) {
    const bool inA = w < ntA;
    const RefitView T = inA ? A : B;
    const int64_t n = T.n;
    const int32_t root = T.tl_root[inA ? w : w - ntA];
    const int2 rg = T.range[root];
    const int lo = rg.x, m = rg.y - rg.x + 1;           // m <= kTreelet leaves, m - 1 internal nodes
    // parent links (parent << 1 | slot) of the indices lo .. hi (the treelet's internal
    // nodes are among them)
    if (lane < m && lo + lane < n - 1) spar[wib][lane] = T.parent[lo + lane];
    scnt[wib][lane] = 0;
    if (first) skin[wib][lane] = 0;
    __syncwarp();
    if (lane < m) {
      const int32_t l = lo + lane;
      float b[6];
      const int4 li = T.leaf_info[l];
      leaf_box_of(li, vbox, b, b + 3);
      int kin = li.w & 1;
      int32_t ps = T.parent[n - 1 + l];
      for (int step = 0; step < kTreelet; ++step) {  // a treelet is at most kTreelet - 1 deep
        const int32_t node = ps >> 1;
        const int off = node - lo, slot = ps & 1;
        if (off < 0 || off >= m) break;              // (a subtree's nodes lie in its leaf range)
        float* dl = slot ? T.nodes[node].lo1 : T.nodes[node].lo0;
        float* dh = slot ? T.nodes[node].hi1 : T.nodes[node].hi0;
        for (int k = 0; k < 3; ++k) { __stcg(&dl[k], b[k]); __stcg(&dh[k], b[3 + k]); }
        for (int k = 0; k < 6; ++k) sbox[wib][off][slot][k] = b[k];
        if (first && kin) atomicOr(&skin[wib][off], 1 << slot);
        __threadfence_block();
        if (atomicAdd(&scnt[wib][off], 1) == 0) break;   // the sibling finishes this node
        __threadfence_block();
        for (int k = 0; k < 3; ++k) {
          b[k] = fminf(sbox[wib][off][0][k], sbox[wib][off][1][k]);
          b[3 + k] = fmaxf(sbox[wib][off][0][3 + k], sbox[wib][off][1][3 + k]);
        }
        if (first) {                                 // both children's bits are in
          const int kb = skin[wib][off];
          T.nodes[node].kin = kb;
          kin = kb == 3;
        }
        if (node == root) break;                     // its box goes up in phase B
        ps = spar[wib][off];
      }
    }
    __syncwarp();
  }
}

// Phase B for up to two trees: one thread per upper start (a treelet root, or a leaf
// directly under a larger node, its box from the positions) climbs with release-acquire
// arrival counters; the two trees' climbs run side by side.  On a build (`first`) the
// kinematic bits climb with the boxes.
template <bool first>
__global__ void __launch_bounds__(kBlock) k_upper_refit(RefitView A, RefitView B, const float* __restrict__ vbox) {
  pdl_entry();
  const int64_t nuA = A.n > 1 ? A.count[1] : 0, nuB = B.n > 1 ? B.count[1] : 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nuA + nuB; k += grid_stride()) {
    const bool inA = k < nuA;
    const RefitView T = inA ? A : B;
    const int64_t n = T.n;
    const int32_t st = T.up_start[inA ? k : k - nuA];
    float lo[3], hi[3];
    int32_t ps;                                      // parent << 1 | slot of the climbing box
    int kin = 0;                                     // (first) every primitive below is kinematic
    if (st >= 0) {                                   // a treelet root: its box from its children
      const BvhNode* nd = &T.nodes[st];
      for (int q = 0; q < 3; ++q) {
        lo[q] = fminf(__ldcg(&nd->lo0[q]), __ldcg(&nd->lo1[q]));
        hi[q] = fmaxf(__ldcg(&nd->hi0[q]), __ldcg(&nd->hi1[q]));
      }
      if (first) kin = (__ldcg(&nd->kin) & 3) == 3;
      if (st == 0) continue;                         // the whole tree was one treelet
      ps = __ldg(T.parent + st);
    } else {                                         // a leaf under a larger node
      const int32_t l = ~st;
      const int4 li = T.leaf_info[l];
      leaf_box_of(li, vbox, lo, hi);
      if (first) kin = li.w & 1;
      ps = __ldg(T.parent + n - 1 + l);
    }
    // Per level: store this box into its slot, arrive, and (second arrival) take the union
    // with the sibling's box.  The slot comes with the parent link, and the next link is
    // fetched before the arrival, so the climb waits on the arrival and the sibling's box
    // only.
    for (int64_t step = 0; step < n; ++step) {       // a root path has at most n-1 nodes
      const int32_t node = ps >> 1, slot = ps & 1;
      BvhNode* nd = &T.nodes[node];
      float* dl = slot ? nd->lo1 : nd->lo0;
      float* dh = slot ? nd->hi1 : nd->hi0;
      for (int q = 0; q < 3; ++q) { __stcg(&dl[q], lo[q]); __stcg(&dh[q], hi[q]); }
      if (first && kin) atomicOr(&nd->kin, 1 << slot);
      const int32_t up = node ? __ldg(T.parent + node) : 0;
      if (arrive<false>(&T.flag[node]) == 0) break;
      const float* sl = slot ? nd->lo0 : nd->lo1;
      const float* sh = slot ? nd->hi0 : nd->hi1;
      for (int q = 0; q < 3; ++q) {                // operands in slot order, as in the build
        const float a = __ldcg(&sl[q]), b = __ldcg(&sh[q]);
        lo[q] = slot ? fminf(a, lo[q]) : fminf(lo[q], a);
        hi[q] = slot ? fmaxf(b, hi[q]) : fmaxf(hi[q], b);
      }
      if (first) kin = (__ldcg(&nd->kin) & 3) == 3;
      if (node == 0) break;
      ps = up;
    }
  }
}

__device__ __forceinline__ bool box_overlap(const float* lo, const float* hi, const float qlo[3], const float qhi[3]) {
  return !(lo[0] > qhi[0] || qlo[0] > hi[0] || lo[1] > qhi[1] || qlo[1] > hi[1] || lo[2] > qhi[2] ||
           qlo[2] > hi[2]);
}

__device__ __forceinline__ void emit(uint64_t key, uint64_t* cand, int64_t* n_cand, int64_t cap, DevStatus* st) {
  uint32_t mask = __activemask();
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(reinterpret_cast<unsigned long long*>(n_cand), (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  int64_t pos = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
  if (pos < cap) {
    cand[pos] = key;
  } else {
    raise_flag(st, EIPC_FLAG_CAND_OVERFLOW);
    raise_need(st, &st->need_cand, pos + 1);
  }
}

// Candidates found during one round of a warp's queries are appended to the warp's own
// slice of shared memory (a shared-memory atomic per candidate) and written out when the
// round ends: one global atomic per warp per round reserves their positions, and the
// copy is coalesced.  A round's candidates beyond the slice's capacity go straight to
// global memory through emit().  Without this, every leaf hit waited for a global
// atomic's returned position.
constexpr int kQueryWarpBuf = 256;

__device__ __forceinline__ void flush_warp_candidates(uint64_t* buf, int* count, uint64_t* cand, int64_t* n_cand,
                                                      int64_t cap, DevStatus* st, int lane) {
  __syncwarp();
  int c = *count;
  if (c > kQueryWarpBuf) c = kQueryWarpBuf;
  if (c > 0) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(n_cand), (unsigned long long)c);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int k = lane; k < c; k += 32) {
      const int64_t pos = (int64_t)base + k;
      if (pos < cap) cand[pos] = buf[k];
    }
    if (lane == 0 && (int64_t)base + c > cap) {
      raise_flag(st, EIPC_FLAG_CAND_OVERFLOW);
      raise_need(st, &st->need_cand, (int64_t)base + c);
    }
  }
  __syncwarp();
  if (lane == 0) *count = 0;
  __syncwarp();
}

// One launch for both query sets: threads [0, nv) run vertex boxes against the triangle
// tree (PT), threads [nv, nv + ne) run edge boxes against the edge tree (EE, j > i), the
// edges in that tree's Morton order so neighbouring threads take similar paths.  A warp's
// 32 lanes take rounds of 32 consecutive queries together (lanes past the end idle), so
// the warp can write out its round's candidates at the round's end.  MINB is the minimum
// number of 256-thread blocks per SM the register allocation must allow: the walk is
// latency-bound (dependent node fetches), so more resident warps hide more of it; 4 leaves
// the compiler free (48 registers), 6 caps it at 40 registers.  Dynamic shared memory:
// kQueryWarpBuf 8-byte keys per warp.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_query(Bvh tt, Bvh te, Topo T, const float* __restrict__ vbox_q,
                                                     uint64_t* cand, int64_t* n_cand, int64_t cap, DevStatus* st) {
  pdl_entry();
  extern __shared__ uint64_t qbuf[];
  __shared__ int qcount[8];
  const int64_t nq = (tt.n > 0 ? T.nv : 0) + (te.n > 0 ? T.ne : 0);
  const int64_t nv_q = tt.n > 0 ? T.nv : 0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint64_t* wbuf = qbuf + (size_t)wib * kQueryWarpBuf;
  int* wcount = qcount + wib;
  if (lane == 0) *wcount = 0;
  __syncwarp();
  const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t wbase = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); wbase < nq; wbase += wstride) {
    const int64_t qi = wbase + lane;
    if (qi < nq) {
      const bool is_pt = qi < nv_q;
      const Bvh& t = is_pt ? tt : te;
      const PrimKind qkind = is_pt ? kVertex : kEdge;
      const int64_t qpos = is_pt ? -1 : qi - nv_q;     // EE: the query's own leaf position
      const int64_t q = is_pt ? qi : (int64_t)te.leaf_prim[qpos];
      float qlo[3], qhi[3];
      prim_box_v(qkind, q, T, vbox_q, qlo, qhi);
      int32_t qa, qb;
      if (is_pt) { qa = (int32_t)q; qb = (int32_t)q; }
      else { qa = T.edges[2 * q]; qb = T.edges[2 * q + 1]; }
      const bool qkin = prim_kin(qkind, T, q);
      const int32_t qgroup = T.vgroup[qa];   // primitives of different scenes never pair
      auto put = [&](uint64_t key) {
        const int slot = atomicAdd(wcount, 1);
        if (slot < kQueryWarpBuf) wbuf[slot] = key;
        else emit(key, cand, n_cand, cap, st);
      };
      auto leaf = [&](int32_t lpos) {
        const int4 info = __ldg(t.leaf_info + lpos);
        if (is_pt) {
          if (info.x == qa || info.y == qa || info.z == qa) return;
          if ((qkin && (info.w & 1)) || (info.w >> 1) != qgroup) return;
          const int32_t p = t.leaf_prim[lpos];
          put(pair_key(0, (uint32_t)q, (uint32_t)p, T.bits_i, T.bits_j));
        } else {
          // each EE pair is found once, from the edge earlier in Morton order
          if (lpos <= qpos) return;
          if (info.x == qa || info.x == qb || info.y == qa || info.y == qb) return;
          if ((qkin && (info.w & 1)) || (info.w >> 1) != qgroup) return;
          const int32_t p = t.leaf_prim[lpos];
          const uint32_t lo = (uint32_t)(p < q ? p : q), hi = (uint32_t)(p < q ? q : p);
          put(pair_key(1, lo, hi, T.bits_i, T.bits_j));
        }
      };
      if (t.n == 1) {
        const float* b = t.leaf_box + 6 * (int64_t)t.leaf_prim[0];
        if (box_overlap(b, b + 3, qlo, qhi)) leaf(0);
      } else {
        // Depth-first walk that descends into an overlapping child directly and pushes only
        // the second child when both overlap, so a descent costs one node fetch and no stack
        // round trip; leaves are handled where they are found.  The stack holds (node, last
        // leaf position under it); EE queries skip subtrees that lie entirely at or before
        // their own leaf.
        int32_t stack[64], smax[64];
        int sp = 0;
        int32_t node = 0;
        int32_t nmax = (int32_t)(t.n - 1);
        // a tree of n leaves has n-1 internal nodes, each fetched at most once
        int64_t visits = 0;
        while (true) {
          if (++visits > t.n) {
            raise_flag(st, EIPC_FLAG_STACK_OVERFLOW);
            break;
          }
          const float4* np = reinterpret_cast<const float4*>(&t.nodes[node]);
          const float4 f0 = __ldg(np), f1 = __ldg(np + 1), f2 = __ldg(np + 2);
          const int4 f3 = __ldg(reinterpret_cast<const int4*>(np + 3));
          const float lo0[3] = {f0.x, f0.y, f0.z}, hi0[3] = {f0.w, f1.x, f1.y};
          const float lo1[3] = {f1.z, f1.w, f2.x}, hi1[3] = {f2.y, f2.z, f2.w};
          const int32_t c0 = f3.x, c1 = f3.y, kin = f3.z, split = f3.w;
          bool o0 = box_overlap(lo0, hi0, qlo, qhi) && !(qkin && (kin & 1)) && (split > qpos);
          bool o1 = box_overlap(lo1, hi1, qlo, qhi) && !(qkin && (kin & 2)) && (nmax > qpos);
          if (o0 && c0 < 0) { leaf(~c0); o0 = false; }
          if (o1 && c1 < 0) { leaf(~c1); o1 = false; }
          if (o0) {
            if (o1) {
              if (sp < 64) { stack[sp] = c1; smax[sp++] = nmax; }
              else raise_flag(st, EIPC_FLAG_STACK_OVERFLOW);
            }
            node = c0;
            nmax = split;
          } else if (o1) {
            node = c1;
          } else {
            if (sp == 0) break;
            --sp;
            node = stack[sp];
            nmax = smax[sp];
          }
        }
      }
    }
    flush_warp_candidates(wbuf, wcount, cand, n_cand, cap, st, lane);
  }
}

}  // namespace

void vertex_boxes(const Topo& topo, const double* x4, const double* dx4, double pad, float* vbox, float* vbox_pad,
                  cudaStream_t s) {
  if (topo.nv <= 0) return;
  launch(k_vertex_boxes, blocks_for(topo.nv), kBlock, 0, s, topo.nv, x4, dx4, pad, vbox, vbox_pad);
}

void bvh_build(Bvh& t, PrimKind kind, const Topo& topo, const double* x4, const double* dx4, const float* vbox,
               int32_t* bounds_ws, uint32_t* sort_hist, cudaStream_t s, int refit_variant) {
  if (t.n <= 0) return;
  zero_ranges(s, {{t.nodes, sizeof(BvhNode) * (t.n > 1 ? t.n - 1 : 1)}, {t.refit_flag, sizeof(int32_t) * t.n},
                  {t.n > 1 ? t.tl_count : nullptr, 2 * sizeof(int32_t)}});
  launch(k_bounds_init, 1, 32, 0, s, bounds_ws);
  launch(k_bounds, blocks_for(topo.nv, 4), kBlock, 0, s, x4, dx4, topo.nv, bounds_ws);
  launch(k_leaves, blocks_for(t.n), kBlock, 0, s, kind, t.n, topo, vbox, static_cast<const int32_t*>(bounds_ws),
         t.leaf_box, t.keys, t.vals);
  int which = radix_sort_u64(t.keys, t.vals, t.keys_alt, t.vals_alt, t.n_dev, t.n, 30, sort_hist, s);
  const uint64_t* sk = which ? t.keys_alt : t.keys;
  const uint32_t* sv = which ? t.vals_alt : t.vals;
  t.sorted = sv;
  if (t.n > 1) launch(k_internal, blocks_for(t.n - 1), kBlock, 0, s, sk, t.n, t.nodes, t.parent, t.range);
  if (refit_variant == 2 && t.n > 1) {
    // the treelet lists first (with the leaf records), then both refit phases with the
    // kinematic bits
    launch(k_treelet_lists, blocks_for(2 * t.n), kBlock, 0, s, t.n, static_cast<const int2*>(t.range),
           static_cast<const int32_t*>(t.parent), t.tl_root, t.up_start, t.tl_count, kind, topo, sv, t.leaf_prim,
           t.leaf_info);
    const RefitView A = refit_view(t);
    const RefitView none{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    launch(k_treelet_refit<true>, blocks_for(t.n, 8), kBlock, 0, s, A, none, vbox);
    launch(k_upper_refit<true>, blocks_for(t.n), kBlock, 0, s, A, none, vbox);
    t.built = true;
    return;
  }
  if (refit_variant == 0)
    launch(k_refit<true, true>, blocks_for(t.n), kBlock, 0, s, kind, t.n, topo, sv,
           static_cast<const float*>(t.leaf_box), t.nodes, static_cast<const int32_t*>(t.parent), t.leaf_prim,
           t.leaf_info, t.refit_flag);
  else
    launch(k_refit<true, false>, blocks_for(t.n), kBlock, 0, s, kind, t.n, topo, sv,
           static_cast<const float*>(t.leaf_box), t.nodes, static_cast<const int32_t*>(t.parent), t.leaf_prim,
           t.leaf_info, t.refit_flag);
  if (t.n > 1) {
    launch(k_treelet_lists, blocks_for(2 * t.n), kBlock, 0, s, t.n, static_cast<const int2*>(t.range),
           static_cast<const int32_t*>(t.parent), t.tl_root, t.up_start, t.tl_count, kind, topo, sv,
           static_cast<int32_t*>(nullptr), static_cast<int4*>(nullptr));
  }
  t.built = true;
}

// both phases of the treelet refit for one or two trees (b may be null)
static void treelet_refit(Bvh& a, Bvh* b, const float* vbox, cudaStream_t s) {
  RefitView A = refit_view(a);
  RefitView Bv = b ? refit_view(*b) : RefitView{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const int64_t n = a.n + (b ? b->n : 0);
  launch(k_treelet_refit<false>, blocks_for(n, 8), kBlock, 0, s, A, Bv, vbox);
  launch(k_upper_refit<false>, blocks_for(n), kBlock, 0, s, A, Bv, vbox);
}

void bvh_refit_pair(Bvh& a, PrimKind ka, Bvh& b, PrimKind kb, const Topo& topo, const float* vbox, cudaStream_t s,
                    int refit_variant) {
  if (refit_variant == 2 && a.n > 1 && b.n > 1) {
    treelet_refit(a, &b, vbox, s);
    return;
  }
  bvh_refit(a, ka, topo, vbox, s, refit_variant);
  bvh_refit(b, kb, topo, vbox, s, refit_variant);
}

void bvh_refit(Bvh& t, PrimKind kind, const Topo& topo, const float* vbox, cudaStream_t s, int refit_variant) {
  if (t.n <= 0) return;
  if (refit_variant == 2 && t.n > 1) {
    treelet_refit(t, nullptr, vbox, s);
    return;
  }
  launch(k_leaf_boxes, blocks_for(t.n), kBlock, 0, s, t.n, static_cast<const int4*>(t.leaf_info), vbox, t.leaf_box);
  zero_ranges(s, {{t.refit_flag, sizeof(int32_t) * t.n}});
  if (refit_variant == 0)
    launch(k_refit<false, true>, blocks_for(t.n), kBlock, 0, s, kind, t.n, topo, t.sorted,
           static_cast<const float*>(t.leaf_box), t.nodes, static_cast<const int32_t*>(t.parent), t.leaf_prim,
           t.leaf_info, t.refit_flag);
  else
    launch(k_refit<false, false>, blocks_for(t.n), kBlock, 0, s, kind, t.n, topo, t.sorted,
           static_cast<const float*>(t.leaf_box), t.nodes, static_cast<const int32_t*>(t.parent), t.leaf_prim,
           t.leaf_info, t.refit_flag);
}

void bvh_query(const Bvh& tri, const Bvh& edge, const Topo& topo, const float* vbox_q, uint64_t* cand,
               int64_t* n_cand, int64_t cap, DevStatus* st, cudaStream_t s, int threads, int bps, int variant) {
  const int64_t nq = (tri.n > 0 ? topo.nv : 0) + (edge.n > 0 ? topo.ne : 0);
  if (nq <= 0) return;
  const size_t smem = (size_t)(threads / 32) * kQueryWarpBuf * sizeof(uint64_t);
  if (variant == 3)
    launch(k_query<6>, blocks_for(nq, bps, threads), threads, smem, s, tri, edge, topo, vbox_q, cand, n_cand, cap, st);
  else
    launch(k_query<4>, blocks_for(nq, bps, threads), threads, smem, s, tri, edge, topo, vbox_q, cand, n_cand, cap, st);
}

}  // namespace eipc
