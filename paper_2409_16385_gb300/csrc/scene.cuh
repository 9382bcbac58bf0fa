// Scene object behind the opaque eipc_scene handle: static topology, embedding weights and
// the device workspace every compute call reuses (sized once at creation).
#pragma once
#include "bvh.cuh"
#include "common.cuh"
#include "timing.cuh"

struct eipc_scene {
  int64_t nv, nf, ne, ns;
  // topology and embedding (device)
  int32_t* tris;
  int32_t* edges;
  int32_t* cage_idx;     // [nv*4], -1 rows kinematic
  double* w;             // [nv*4]
  double* x_kin4;        // [nv*4] padded kinematic positions
  uint8_t* vkin;
  uint8_t* ekin;
  uint8_t* fkin;
  int32_t* vgroup;       // [nv] independent-scene id per vertex (all 0 unless set)
  int32_t n_groups;
  unsigned long long* group_alpha_bits;   // [n_groups] CCD bound per group (IEEE bits)
  int64_t* group_count;  // [n_groups + 1] items per group, then offsets
  int32_t* item_group;   // [item_cap] group of each evaluated item
  int32_t* fric_of_pair; // [item_cap] friction item riding on each contact pair (see eval.cu)
  int32_t* pair_of_fric; // [item_cap] contact pair found for each friction item
  uint64_t* lag_key;     // [item_cap] (type, i, j) of each item of the last lag state built here
  const int32_t* lag_src; // that lag state's v array (identifies it at evaluation)
  eipc::Topo topo;
  // positions (padded, 4 doubles per vertex)
  double* x4;
  double* dx4;
  float* x4f;            // [nv*4] FP32 copy of x4 for the narrow-phase screen
  float* vbox;           // [nv*8] per-vertex FP32 boxes of the last call (contact or swept)
  float* vbox_pad;       // [nv*8] the contact ones grown by dhat (the query boxes)
  // broad phase
  eipc::Bvh tri_bvh, edge_bvh;
  int32_t* bounds_ws;
  uint32_t* sort_hist;
  int64_t cand_cap;
  uint64_t* cand;
  uint64_t* cand2;       // candidates the FP32 screen passed on to the FP64 test
  int64_t* counters;     // [kCntN] device counters (see kCnt*)
  // narrow phase survivors
  uint64_t* skeys;
  uint64_t* skeys_alt;
  uint32_t* svals;
  uint32_t* svals_alt;
  double* sd;
  // reduction workspace
  int64_t item_cap;      // pairs + friction items per eval
  int32_t* item_nodes;   // [item_cap*16]
  int32_t* item_n;       // [item_cap]
  int64_t* rc_h;         // [item_cap] record counts, then offsets
  int64_t* ro_h;
  int64_t* rc_g;
  int64_t* ro_g;
  double* item_E;        // [item_cap]
  int64_t rec_cap;
  uint64_t* hkeys;
  uint64_t* hkeys_alt;
  uint32_t* hvals;
  uint32_t* hvals_alt;
  double* hrec;          // [rec_cap*kHRecStride] 3x3 blocks, 16-byte aligned rows
  double* hvp_out;       // [(ns+64)*3] Hessian-vector product: reduced rows, then 64 kinematic partials
  uint64_t* edge_key;    // [ne] sorted a * nv + b of every edge (a < b), for edge-id lookup
  int32_t* edge_id;      // [ne] edge id of each sorted key
  int feat_bits;         // bits per id in the feature keys of the deduplicated pair set
  double* moll_r2;       // [ne] rest squared edge lengths of the EE mollifier
  double moll_factor;    // eps_x = moll_factor |e_i|^2 |e_j|^2; 0 = mollifier off
  int64_t* seg_flag;     // [rec_cap] key of each Hessian segment (upper block), as uint64
  int64_t* seg_id;       // [rec_cap] BSR entries of each segment's block and transpose, as int32 pairs
  int64_t* seg_start;    // [rec_cap]
  uint32_t* hinv;        // [rec_cap] sorted position of each Hessian record
  double* piece;         // [9 * (rec_cap + rec_cap / 32 + 2)] partial segment sums of the Hessian records
  int64_t* hunit;        // [rec_cap + 1] first summation unit of each Hessian segment
  int64_t gcap;          // gradient records
  uint64_t* gkeys;
  uint64_t* gkeys_alt;
  uint32_t* gvals;
  uint32_t* gvals_alt;
  double* grec;          // [gcap*kGRecStride] 3-vectors, 16-byte aligned rows
  int64_t* gseg_start;
  int64_t* scan_partial; // [2 (kScanBlocks+1)] scan partials (two arrays for exclusive_scan2_i64)
  double* sum_partial;   // [kScanBlocks]
  int bits_h, bits_g;    // key widths of the reduction sorts
  int rebuild_interval;  // contact LBVH: full rebuild every this many build_candidates calls
  struct {
    int eval_threads = 128, eval_bps = 16, eval_variant = 2, eval_tile = 32;
    int ccd_tile = 128;
    int query_threads = 128, query_bps = 24, query_variant = 2;
    int refit_variant = 2;
  } tune;                // launch shapes of the tunable kernels (eipc_set_launch)
  int contact_refits;    // refits since the last full rebuild
  eipc::DevStatus* status;
  eipc::Timers* timers;   // host-side event timers (off unless enabled)
  // a second stream of the scene's device: the friction evaluation runs on it beside the
  // barrier evaluation (they write disjoint records), forked from and joined back to the
  // caller's stream with two events, which also works inside a graph capture
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join;
};

namespace eipc {
// device counters
// record row strides (doubles): 9 (3) values padded so that each row starts on 16 bytes
constexpr int kHRecStride = 10, kGRecStride = 4;

enum { kCntCand = 0, kCntSurv = 1, kCntItems = 2, kCntRecH = 3, kCntRecG = 4, kCntSegH = 5, kCntSegG = 6,
       kCntAccd = 7, kCntZero = 8, kCntEvalQueue = 16, kCntScreened = 15, kCntDedup = 17, kCntUnitsH = 18,
       kCntMollBad = 20, kCntCcdQueue = 21,
       kCntN = 24 };

// id of the edge with end vertices {a, b} from the scene's sorted edge keys a * nv + b
// (a < b), or -1 if there is none
__device__ __forceinline__ int32_t edge_id_of(int32_t a, int32_t b, int64_t nv, const uint64_t* __restrict__ ekey,
                                              const int32_t* __restrict__ eid, int64_t ne) {
  if (a > b) { const int32_t t = a; a = b; b = t; }
  const uint64_t key = (uint64_t)a * (uint64_t)nv + (uint64_t)b;
  int64_t lo = 0, hi = ne;                 // first position with ekey >= key
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ekey[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < ne && ekey[lo] == key) ? eid[lo] : -1;
}

#define EIPC_TIMED(sc, id, s, ...)        \
  do {                                    \
    (sc)->timers->start((id), (s));       \
    __VA_ARGS__;                          \
    (sc)->timers->stop((id), (s));        \
  } while (0)

void embed_launch(const eipc_scene* sc, const double* q, double* out, int out_padded, int displacement,
                  cudaStream_t s);
void pairs_launch(eipc_scene* sc, const double* q, const eipc_params& p, const eipc_pairs& out, cudaStream_t s);
void lag_launch(eipc_scene* sc, const double* q_n, const eipc_pairs& pr, const eipc_params& p, const eipc_lag& out,
                cudaStream_t s);
void eval_launch(eipc_scene* sc, const double* q, const eipc_pairs& pr, const eipc_lag* lag, const eipc_params& p,
                 double* E, double* g_r, const eipc_bsr& H, cudaStream_t s);
int bits_for(uint64_t maxval);
void group_energy_launch(eipc_scene* sc, double* E_groups, cudaStream_t s);
void hvp_launch(eipc_scene* sc, const double* q, const eipc_pairs& pr, const eipc_lag* lag, const eipc_params& p,
                const double* v, const double* kin_dir, double* out_r, double* out_kin, cudaStream_t s);
void set_kinematic_launch(eipc_scene* sc, const double* x_kin, cudaStream_t s);
void mollifier_rest_launch(eipc_scene* sc, const double* x_rest, int64_t* bad, cudaStream_t s);
void candidates_launch(eipc_scene* sc, int32_t* type, int32_t* ci, int32_t* cj, int64_t cap, int64_t* n,
                       cudaStream_t s);
void bsr_spmv_launch(int64_t nrows, const int32_t* row_ptr, const int32_t* col, const double* val, const double* x,
                     double alpha, double beta, double* y, cudaStream_t s);
void group_alpha_launch(eipc_scene* sc, double* alpha_groups, cudaStream_t s);
void accd_launch(eipc_scene* sc, const double* x, const double* dx, const eipc_params& p, double* alpha,
                 int64_t* n_candidates, cudaStream_t s);
}  // namespace eipc
