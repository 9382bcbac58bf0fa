// Linear BVH over the surface primitives (Karras 2012 construction on 30-bit Morton
// codes) and the traversal that produces candidate pairs for the contact set and for the
// CCD step bound.  Boxes are FP32 rounded outward from the FP64 positions, so a box test
// never rejects a pair that the exact FP64 test would keep.
#pragma once
#include "common.cuh"

namespace eipc {

// One internal node holds the boxes of both children so a traversal step is one 64-byte
// fetch.  Child ids: >= 0 internal node, < 0 leaf ~position in Morton order.
struct alignas(16) BvhNode {
  float lo0[3], hi0[3];
  float lo1[3], hi1[3];
  int32_t c0, c1;
  int32_t kin;   // bit 0 / bit 1: every primitive under child 0 / 1 is kinematic
  int32_t split; // last leaf position under child 0 (child 1 ends where its parent ends)
};

struct Bvh {
  int64_t n;             // primitives (static per scene)
  int64_t* n_dev;        // [1] device copy of n (element count for the Morton sort)
  BvhNode* nodes;        // [n-1]
  int32_t* parent;       // [2n-1]: parent << 1 | slot (0: child c0, 1: c1); internal i at i, leaf l at n-1+l
  int32_t* leaf_prim;    // [n]
  int4* leaf_info;       // [n] per leaf (Morton order): vertex ids (-1 if unused), kinematic flag
  float* leaf_box;       // [6n], by primitive id (lo xyz, hi xyz)
  int32_t* refit_flag;   // [n]
  uint64_t* keys;        // [n] Morton keys (sorted in place)
  uint32_t* vals;        // [n]
  const uint32_t* sorted; // Morton order of the last build (points into vals / vals_alt)
  bool built;            // a hierarchy exists and can be refitted
  uint64_t* keys_alt;    // [n]
  uint32_t* vals_alt;    // [n]
  int2* range;           // [n-1] leaf range [lo, hi] of each internal node
  int32_t* tl_root;      // [n] roots of the treelets (subtrees of <= kTreelet leaves under a larger parent)
  int32_t* up_start;     // [n] starts of the refit's upper climb: a treelet root (>= 0) or a leaf ~l
  int32_t* tl_count;     // [2] number of treelet roots, number of upper starts
};

// leaves per treelet of the two-phase refit (one warp per treelet)
constexpr int kTreelet = 32;

enum PrimKind { kVertex = 0, kEdge = 1, kTri = 2 };

// Static topology needed by the broad and narrow phases.
struct Topo {
  int64_t nv, ne, nf;
  const int32_t* tris;   // [nf*3]
  const int32_t* edges;  // [ne*2]
  const uint8_t* vkin;   // [nv]
  const uint8_t* ekin;   // [ne] both ends kinematic
  const uint8_t* fkin;   // [nf] all three kinematic
  const int32_t* vgroup; // [nv] independent-scene id of each vertex (0 when not batched)
  int bits_i, bits_j;    // pair key packing
};

// Pair key: type << (bi+bj) | i << bj | j, ordered like (type, i, j).
__host__ __device__ __forceinline__ uint64_t pair_key(int type, uint32_t i, uint32_t j, int bi, int bj) {
  return ((uint64_t)type << (bi + bj)) | ((uint64_t)i << bj) | (uint64_t)j;
}

// Per-vertex FP32 boxes of the positions x4 (padded), swept over x + dx when dx4 is given,
// rounded outward: vbox[8 nv] unpadded and, when vbox_pad is not null, vbox_pad[8 nv] grown
// by pad.  The leaf and query boxes below are taken from these; they are bit for bit the
// boxes computed from the positions primitive by primitive.
void vertex_boxes(const Topo& topo, const double* x4, const double* dx4, double pad, float* vbox, float* vbox_pad,
                  cudaStream_t s);

// Build the tree over primitives of `kind`: scene bounds from positions x4 (padded),
// optionally swept by dx4 (CCD), leaf boxes from the matching per-vertex boxes vbox;
// `bounds_ws` holds 6 ints of scratch.  Enqueued on stream s.
// refit_variant: 0 = arrival counters behind full device fences, 1 = release-acquire
// arrival counters, 2 = treelets of <= 32 leaves refitted by one warp each in shared memory,
// then release-acquire counters above them (all give the same boxes).  With 2 the build's
// own bottom-up pass is the treelet refit too: the treelet lists come first and write the
// leaf records, and the kinematic bits climb with the boxes.
void bvh_build(Bvh& t, PrimKind kind, const Topo& topo, const double* x4, const double* dx4, const float* vbox,
               int32_t* bounds_ws, uint32_t* sort_hist, cudaStream_t s, int refit_variant);

// Refit the hierarchy of the last bvh_build with new leaf boxes (from the per-vertex boxes
// vbox): any binary tree over the primitives with conservative boxes gives the same exact
// candidate set, so the Morton sort and hierarchy can be reused while the topology stays.
void bvh_refit(Bvh& t, PrimKind kind, const Topo& topo, const float* vbox, cudaStream_t s, int refit_variant);

// Refit of two hierarchies (the triangle and edge trees) at once: with the treelet refit
// both trees share two launches, so their latency-bound climbs overlap.  The boxes are
// those of two bvh_refit calls.  With the treelet refit, the leaf boxes are computed inside
// the refit and leaf_box is not updated (only single-leaf trees and the other refits read
// it).
void bvh_refit_pair(Bvh& a, PrimKind ka, Bvh& b, PrimKind kb, const Topo& topo, const float* vbox, cudaStream_t s,
                    int refit_variant);

// Traverse both trees in one launch: every vertex box (from vbox_q: the per-vertex boxes
// grown by the contact distance, or swept for CCD) against the triangle tree -> PT
// candidates, every edge box against the edge tree -> EE
// candidates with j > i.  Incident pairs and all-kinematic pairs are skipped; candidates
// are appended as pair keys to cand[0..cap) with the running count in *n_cand, and an
// overflow raises CAND_OVERFLOW.
void bvh_query(const Bvh& tri, const Bvh& edge, const Topo& topo, const float* vbox_q, uint64_t* cand,
               int64_t* n_cand, int64_t cap, DevStatus* st, cudaStream_t s, int threads, int bps, int variant);

}  // namespace eipc
