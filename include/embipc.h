/* embipc.h -- C ABI of the GB300 contact stage of Embedded IPC (arxiv 2409.16385).
 *
 * One Newton iteration's contact work, for a high-resolution collision surface embedded
 * in a coarse tetrahedral cage (Sec. III-D):
 *   eipc_embed             x = phi(q) = J q                          (Sec. III-D, Eq. 14)
 *   eipc_build_candidates  contact set B: PT / EE pairs with 0 < d < dhat (Sec. III-B)
 *   eipc_friction_lag      lagged friction state at x^n               (Sec. III-B)
 *   eipc_eval_contact      E = kappa sum b(d_k) + sum D_k, g_r = J^T grad E,
 *                          H_r = J^T (sum P+(kappa hess b_k) + sum hess D_k) J
 *                                                   (Eq. 7-8, Sec. III-C, Eq. 17)
 *   eipc_accd_toi          step bound alpha for a straight full-space motion x + t dx,
 *                          linear in the reduced step because phi is linear (Sec. III-C)
 *
 * Conventions
 *  - Every array passed to a compute call is DEVICE memory owned by the caller, and every
 *    compute call is asynchronous on the given CUDA stream; nothing synchronises and no
 *    count is read back to the host, so a sequence of calls can be captured in a CUDA
 *    graph.  eipc_scene_create takes HOST arrays and copies them to the device.
 *  - The scene owns its topology copy and a workspace sized at creation; compute calls
 *    allocate nothing.  A scene may be used from one stream at a time.
 *  - Host-detectable misuse (null pointer, negative size, capacity too small for the
 *    scene) returns a negative status synchronously and enqueues nothing.
 *  - Device-detected conditions (a pair at d <= 0, a full buffer, a non-finite input,
 *    a CCD pair that hit its iteration cap) set bits of the scene's device status word;
 *    eipc_status_read synchronises the stream and returns them.  After an overflow the
 *    outputs of that call are incomplete and the status reports the size needed.
 *  - Energies and derivatives are the unscaled contact potential; the caller multiplies
 *    by h^2 as in the incremental potential of Sec. III-B.
 */
#ifndef EMBIPC_H
#define EMBIPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t eipc_status;
typedef struct CUstream_st* eipc_stream; /* a cudaStream_t; NULL = legacy default stream */

enum {
  EIPC_OK = 0,
  EIPC_ERR_INVALID = -1,      /* bad argument (null pointer, size, capacity)            */
  EIPC_ERR_CUDA = -2,         /* a CUDA runtime call failed                             */
  EIPC_ERR_NOMEM = -3,        /* workspace allocation failed at scene creation          */
  EIPC_ERR_TOO_LARGE = -4,    /* a size exceeds a fixed maximum of the call             */
  /* device status bits (eipc_status_read) */
  EIPC_FLAG_PENETRATION = 1,  /* some pair has d <= 0: the configuration is infeasible  */
  EIPC_FLAG_PAIR_OVERFLOW = 2,/* more contact pairs than the caller's pair capacity     */
  EIPC_FLAG_CAND_OVERFLOW = 4,/* more broad-phase candidates than the scene workspace   */
  EIPC_FLAG_REC_OVERFLOW = 8, /* more reduction records than the scene workspace        */
  EIPC_FLAG_BSR_OVERFLOW = 16,/* more BSR blocks than the caller's block capacity       */
  EIPC_FLAG_NONFINITE = 32,   /* a non-finite position or displacement was read         */
  EIPC_FLAG_ACCD_CAP = 64,    /* a CCD pair reached accd_max_iter (alpha still safe)    */
  EIPC_FLAG_LAG_OVERFLOW = 128,/* more friction pairs than the lag buffer capacity      */
  EIPC_FLAG_STACK_OVERFLOW = 256,/* a BVH traversal exceeded its 64-entry stack         */
  EIPC_FLAG_BAD_INDEX = 512   /* a caller-supplied candidate names an out-of-range id   */
};

/* Contact parameters.  dhat: barrier activation distance (m); kappa: barrier stiffness;
 * mu: friction coefficient; eps_v: static-friction velocity threshold (m/s) and h: time
 * step (s), whose product eps_v*h is the f0/f1 transition; accd_s in (0,1): the CCD
 * stops advancing once a pair's distance has shrunk to accd_s times its initial value;
 * accd_max_iter: per-pair cap on CCD advancements. */
typedef struct {
  double dhat, kappa, mu, eps_v, h, accd_s;
  int32_t accd_max_iter;
  int32_t flags;            /* EIPC_PARAM_* bits, 0 for the defaults */
} eipc_params;

/* eipc_params.flags:
 *   EIPC_PARAM_NO_PROJECTION makes eipc_eval_contact return the exact (unprojected) Hessian
 *     instead of the projected-Newton one;
 *   EIPC_PARAM_DEDUP makes eipc_build_candidates return the deduplicated contact set: each
 *     pair stands for the feature pair realising its distance (face-vertex, vertex-edge,
 *     vertex-vertex, edge-edge interior), and pairs realising the same feature pair count
 *     once, as the first of them in (type, i, j) order.  The paper's set B (Sec. III-B)
 *     counts every pair; this is the IPC-style alternative. */
enum { EIPC_PARAM_NO_PROJECTION = 1, EIPC_PARAM_DEDUP = 2 };

/* Contact pair list, all device arrays owned by the caller.  Pair k is a point-triangle
 * pair (type 0: i = vertex, j = triangle) or an edge-edge pair (type 1: i < j edge ids),
 * with unsigned distance d[k].  Lists written by eipc_build_candidates are ordered by
 * (type, i, j).  *count (device) receives the number of pairs found, which may exceed
 * capacity (then only capacity entries are written and PAIR_OVERFLOW is raised). */
typedef struct {
  int64_t capacity;
  int32_t* type;
  int32_t* i;
  int32_t* j;
  double* d;
  int64_t* count;
} eipc_pairs;

/* Lagged friction state (Sec. III-B), one entry per pair active at x^n, device arrays
 * owned by the caller: v[4] the stencil's vertices, gamma[4] the closest-point weights
 * (r = sum_a gamma_a x_a is the vector between the closest points), n[3] the contact
 * normal r/|r| at x^n, anchor[3] = r at x^n and lambda = kappa |b'(d^n)| the lagged
 * normal force magnitude.  u(x) is the part of sum_a gamma_a x_a - anchor orthogonal
 * to n, and D = mu lambda f0(|u|). */
typedef struct {
  int64_t capacity;
  int32_t* v;       /* [capacity,4] */
  double* gamma;    /* [capacity,4] */
  double* n;        /* [capacity,3] */
  double* anchor;   /* [capacity,3] */
  double* lambda;   /* [capacity]   */
  int64_t* count;   /* [1]          */
} eipc_lag;

/* Reduced Hessian in 3x3-block CSR (BSR) form, full symmetric pattern, device arrays
 * owned by the caller: row_ptr[Ns+1], col[capacity], val[capacity*9] (row-major 3x3),
 * *nnzb (device) = number of blocks.  Columns are sorted within each row. */
typedef struct {
  int64_t capacity;
  int32_t* row_ptr;
  int32_t* col;
  double* val;
  int64_t* nnzb;
} eipc_bsr;

typedef struct eipc_scene eipc_scene;

/* Creates a scene from HOST arrays (copied; the caller keeps ownership):
 *   tris[F*3], edges[E*2] (a < b, unique) vertex ids in [0,Nv);
 *   cage_idx[Nv*4], w[Nv*4]: containing-tet node ids and barycentric weights of each
 *     embedded vertex (Sec. III-D); a row with cage_idx[4v] = -1 marks a kinematic vertex
 *     whose position is x_kin[3v..3v+2] and which has no reduced DoF;
 *   Ns: number of cage nodes (q has Ns*3 entries);
 *   cand_capacity: broad-phase candidate buffer entries (<= 0: 48 per primitive);
 *   rec_capacity: reduction record entries (<= 0: 2^24).  The evaluation holds up to
 *     min(cand_capacity, max(2^22, rec_capacity / 4)) items (contact + friction pairs).
 * Returns EIPC_ERR_INVALID for inconsistent sizes or out-of-range ids, EIPC_ERR_NOMEM
 * if the device workspace cannot be allocated. */
eipc_status eipc_scene_create(int64_t Nv, int64_t F, int64_t E, int64_t Ns, const int32_t* tris,
                              const int32_t* edges, const int32_t* cage_idx, const double* w,
                              const double* x_kin, int64_t cand_capacity, int64_t rec_capacity,
                              eipc_scene** out);
void eipc_scene_destroy(eipc_scene* scene);

/* x[Nv*3] = J q for q[Ns*3] (Sec. III-D, Eq. 14).  displacement != 0 maps a reduced
 * displacement instead: kinematic rows are then 0 rather than x_kin. */
eipc_status eipc_embed(eipc_scene* scene, const double* q, double* x, int32_t displacement,
                       eipc_stream stream);

/* Contact set B at x = J q (Sec. III-B): every PT and EE pair that is not incident
 * (shares no vertex), is not made only of kinematic vertices, and has 0 < d < dhat,
 * found by an LBVH broad phase and an exact FP64 distance test. */
eipc_status eipc_build_candidates(eipc_scene* scene, const double* q, const eipc_params* p,
                                  eipc_pairs* out, eipc_stream stream);

/* Lagged friction state at x^n = J q_n for the pairs of pairs_n (Sec. III-B). */
eipc_status eipc_friction_lag(eipc_scene* scene, const double* q_n, const eipc_pairs* pairs_n,
                              const eipc_params* p, eipc_lag* out, eipc_stream stream);

/* Contact potential at x = J q over the barrier pairs and (if lag != NULL and mu > 0)
 * the lagged friction pairs: E (device scalar), g_r[Ns*3] and H_r (BSR).  Each pair's
 * barrier Hessian is projected to the nearest PSD matrix before the reduction; friction
 * Hessians are PSD as written.  Reduction is deterministic (bitwise repeatable). */
eipc_status eipc_eval_contact(eipc_scene* scene, const double* q, const eipc_pairs* pairs,
                              const eipc_lag* lag, const eipc_params* p, double* E, double* g_r,
                              eipc_bsr* H_r, eipc_stream stream);

/* Step bound for the straight motion x + t dx, t in [0,1] (x, dx: [Nv*3]): over every
 * PT / EE pair (not incident, not all kinematic) whose closed swept boxes overlap,
 * conservative advancement gives a collision-free t_k; alpha = min(1, min_k t_k),
 * written to the device scalar *alpha and reduced by exact minimum.  *n_candidates
 * (device, may be NULL) receives the number of pairs advanced. */
eipc_status eipc_accd_toi(eipc_scene* scene, const double* x, const double* dx,
                          const eipc_params* p, double* alpha, int64_t* n_candidates,
                          eipc_stream stream);

/* Hessian-vector product of the contact potential (Eq. 7-8 barrier and lagged friction,
 * reduced by Eq. 17) WITHOUT the PSD projection: the exact second derivative that an
 * adjoint (implicit differentiation of a Newton step) needs.  With y = H u, where H is
 * the full-space contact Hessian at x = J q over `pairs` (and `lag`, if given and mu > 0)
 * and u is J v on the embedded vertices and kin_dir on every kinematic vertex:
 *   out_r[Ns*3]  (device) <- J^T y, i.e. H_r v plus the mixed term of the kinematic motion;
 *   out_kin[3]   (device, may be NULL) <- the sum of y over the kinematic vertices, i.e.
 *                 the derivative of the contact force on the kinematic set along v.
 * v: device [Ns*3]; kin_dir: HOST array of 3 doubles, or NULL for zero.  The reduction
 * is deterministic (sort by node, fixed-order warp sums), like eipc_eval_contact's. */
eipc_status eipc_contact_hvp(eipc_scene* scene, const double* q, const eipc_pairs* pairs, const eipc_lag* lag,
                             const eipc_params* params, const double* v, const double* kin_dir, double* out_r,
                             double* out_kin, eipc_stream stream);

/* EE mollifier, the IPC-style variant for nearly parallel edges (the paper applies none):
 * with factor > 0, an edge-edge pair (i, j) with c = |e_i x e_j|^2 below
 * eps_x = factor * rest_len2[i] * rest_len2[j] carries kappa m(c) b(d), m(c) = c (2/eps_x
 * - c/eps_x^2), in every later eval_contact, contact_hvp and friction_lag (whose lambda is
 * scaled by m at x^n); such pairs take a full 12 x 12 Hessian (PSD-projected by Jacobi for
 * eval_contact).  IPC's factor is 1e-3.  x_rest: DEVICE [Nv*3] (caller-owned, read
 * during the call only), the rest positions the edge lengths |e|^2 are taken from; the
 * library computes and keeps the squared rest length of every edge.  Returns
 * EIPC_ERR_INVALID (and leaves the mollifier off) if any edge has a zero or non-finite
 * rest length.  factor = 0 turns it off (x_rest may then be NULL).  Synchronises `stream`
 * (the length check is read back). */
eipc_status eipc_scene_set_mollifier(eipc_scene* scene, const double* x_rest, double factor, eipc_stream stream);

/* y <- alpha A x + beta y for a 3x3-block CSR matrix A with nrows block rows (the eipc_bsr
 * layout: row_ptr[nrows+1], col[nnzb], val[nnzb*9] row-major blocks), for the Krylov
 * solves of a Newton step.  x, y: device [nrows*3] (x must not alias y); beta = 0 ignores
 * y's old contents.  One warp per block row with a fixed summation order (deterministic). */
eipc_status eipc_bsr_spmv(int64_t nrows, const int32_t* row_ptr, const int32_t* col, const double* val,
                          const double* x, double alpha, double beta, double* y, eipc_stream stream);

/* New prescribed positions of the kinematic vertices: x_kin is a DEVICE array [Nv*3]
 * (rows of embedded vertices are ignored).  Asynchronous on `stream`, capturable. */
eipc_status eipc_scene_set_kinematic(eipc_scene* scene, const double* x_kin, eipc_stream stream);

/* Synchronises the stream, copies the device status word and clears it.
 * flags <- OR of EIPC_FLAG_*; needed[0..3] <- pairs, candidates, records, BSR blocks
 * required by the last overflowing call (0 if none); accd_iters <- total CCD
 * advancements since the last read.  Any pointer may be NULL. */
eipc_status eipc_status_read(eipc_scene* scene, eipc_stream stream, int32_t* flags, int64_t* needed,
                             int64_t* accd_iters);

/* Work counts of the scene's last calls, for sizing capacities and reading where the time
 * goes.  Synchronises the stream and copies n (<= EIPC_WORK_COUNTS) int64 entries to the
 * HOST array out:
 *   out[0] broad-phase candidates of the last eipc_build_candidates or eipc_accd_toi call;
 *   out[1] candidates the FP32 screen of the last eipc_build_candidates passed on to the
 *          exact FP64 test;
 *   out[2] contact pairs it kept (before deduplication);
 *   out[3] items of the last evaluation (contact pairs + friction pairs);
 *   out[4] its Hessian block records, out[5] its gradient contributions, one per item and
 *          cage node, carried in the item's diagonal block records (a friction pair whose
 *          stencil has the same four vertices as a contact pair's is evaluated with that
 *          pair, into its records, and adds none);
 *   out[6] distinct upper-triangle Hessian blocks, out[7] distinct gradient nodes;
 *   out[8] CCD candidates the last eipc_accd_toi advanced.
 * Values beyond a buffer's capacity are clamped as the kernels clamp them. */
enum { EIPC_WORK_COUNTS = 9 };
eipc_status eipc_work_counts(eipc_scene* scene, eipc_stream stream, int64_t* out, int32_t n);

/* The broad-phase candidate list of the scene's last eipc_build_candidates or
 * eipc_accd_toi call (the pairs whose FP32 boxes overlap, before any exact test), for
 * inspection and for running another implementation of the same stage on identical input
 * (the CCD bound of Sec. III-C over the same candidates).  Entry k is a PT pair (type 0:
 * vertex i[k], triangle j[k]) or an EE pair (type 1: edges i[k] < j[k]) in the list's own
 * (unsorted) order.  type, i, j: caller-owned DEVICE int32 arrays of `capacity` entries;
 * *n: DEVICE int64, set to the full count (entries beyond `capacity` are not written).
 * Asynchronous on `stream`. */
eipc_status eipc_candidates_read(eipc_scene* scene, int32_t* type, int32_t* i, int32_t* j, int64_t capacity,
                                 int64_t* n, eipc_stream stream);

/* Tracing: per-kernel CUDA-event timers.  Bit k of mask enables timer k (0 embed,
 * 1 bvh_build, 2 bvh_query, 3 narrow_phase, 4 pair_sort, 5 friction_lag, 6 stencil_nodes,
 * 7 eval_barrier, 8 eval_friction, 9 hessian_reduce, 10 gradient_reduce, 11 energy_sum,
 * 12 ccd_advance, 13 eval_kernels -- the barrier and friction evaluations together, which
 * run side by side on two streams; eipc_kernel_name(k) names them): each launch is
 * bracketed by two events on its stream.  eipc_timing_read synchronises, writes the summed milliseconds and launch
 * counts of the first n timers and resets them. */
eipc_status eipc_timing_enable(eipc_scene* scene, uint32_t mask);
eipc_status eipc_timing_read(eipc_scene* scene, double* total_ms, int64_t* launches, int32_t n);
const char* eipc_kernel_name(int32_t id);

/* eipc_build_candidates rebuilds its LBVHs (Morton sort + hierarchy) every n-th call and
 * only refits the boxes of the existing hierarchy in between (default n = 8; n = 1 rebuilds
 * every call).  The contact set is exact either way; only the traversal cost depends on how
 * well the reused hierarchy fits the current positions.  eipc_accd_toi always refits the
 * last hierarchy with swept boxes. */
eipc_status eipc_set_rebuild_interval(eipc_scene* scene, int32_t n);

/* Batched scenes.  Several independent scenes concatenated into one eipc_scene (disjoint
 * vertex and cage-node ranges) run through one set of launches per call; vertex_group[v]
 * (HOST array [Nv], values in [0, n_groups)) names the scene of each vertex.  Every
 * triangle and edge must lie inside one group (EIPC_ERR_INVALID otherwise), and pairs
 * across groups are never formed.  Each scene's g_r and H_r are the rows and columns of its
 * own cage nodes.  Its energy and step bound come from:
 *   eipc_group_energy: after eipc_eval_contact, E_groups[g] (device, [n_groups]) is group g's
 *     share of E, summed in an order fixed by the group's own pairs, so it is bitwise the
 *     value the same scene gives on its own;
 *   eipc_group_alpha: after eipc_accd_toi, alpha_groups[g] (device) is group g's step bound.
 * The scene keeps one group (all of it) until eipc_scene_set_groups is called; the call
 * synchronises (host-side validation). */
eipc_status eipc_scene_set_groups(eipc_scene* scene, const int32_t* vertex_group, int32_t n_groups);
eipc_status eipc_group_energy(eipc_scene* scene, double* E_groups, eipc_stream stream);
eipc_status eipc_group_alpha(eipc_scene* scene, double* alpha_groups, eipc_stream stream);

/* Launch shape of a tunable kernel (the autotuner's knobs).  kernel: 0 = per-pair barrier
 * evaluation, 1 = BVH traversal, 2 = BVH bottom-up refit, 3 = the evaluation's work-queue
 * tile, 4 = the CCD advancement's work-queue tile.  threads per block: 64, 128 (eval), 64,
 * 128, 256 (traversal) or 256 (refit); for kernels 3 and 4 `threads` is instead the number
 * of items a warp claims from the kernel's work queue at a time (32, 64, 128 or 256;
 * defaults 32 and 128), and the other two arguments are ignored.  blocks_per_sm: cap on the
 * grid as a multiple of the 152 SMs (1..64; ignored by the refit); variant: eval 2 = no
 * register cap, 3 = at most 170 registers (3 blocks of 128 per SM), 4 = at most 128
 * registers (4 blocks of 128 per SM); traversal 2 = no register cap, 3 = at most 40
 * registers (6 blocks of 256 per SM); refit 0 = arrival counters behind full device
 * fences, 1 = release-acquire arrival counters, 2 = treelets of up to 32 leaves refitted per
 * warp in shared memory below release-acquire counters, for the refits and for the
 * rebuilds' own bottom-up pass (default).  Results never depend on the shape. */
eipc_status eipc_set_launch(eipc_scene* scene, int32_t kernel, int32_t threads, int32_t blocks_per_sm,
                            int32_t variant);

/* Number of kernel launches the library has enqueued in this process (all scenes). */
int64_t eipc_launch_count(void);

/* Launch mode of every later kernel launch of the library, process-wide (all scenes and
 * streams).  on != 0 (the default): programmatic dependent launch -- each kernel may be
 * scheduled while its predecessor in the stream still runs and waits on the device for
 * that predecessor's completion before its first memory access, which hides the launch
 * latency between the short kernels of a step.  on == 0: plain stream order.  Results are
 * the same bits either way.  Graphs keep the mode they were captured with.  Not thread-
 * safe against launches in flight on other host threads (they see either mode). */
void eipc_set_programmatic_launch(int32_t on);

/* CCD step bound without any device allocation.  The paper has no counterpart: this
 * exists for callers that cannot call cudaMalloc -- code running under another framework's
 * device-memory allocator or pool that must own every allocation, or a control loop that
 * cannot afford the implicit device synchronisation of an allocation -- and so cannot
 * create an eipc_scene, whose workspace is allocated at creation.
 *
 * Same arithmetic as eipc_accd_toi, over a candidate list the caller supplies instead of
 * the LBVH search: for k < n_cand, pair (cand_type[k], cand_i[k], cand_j[k]) is a PT pair
 * (type 0: vertex i, triangle j) or an EE pair (type 1: edges i, j).  Candidates whose
 * closed FP64 swept boxes over [x, x + dx] do not overlap, and incident ones, are skipped,
 * so any superset of the overlapping pairs gives the same alpha.  This call has no
 * kinematic mask: a pair whose four vertices are all kinematic is advanced like any other
 * (eipc_accd_toi's search drops such pairs), so to get the scene path's alpha the caller
 * leaves them out of the list.  Inputs (device, caller-
 * owned): x[Nv*3], dx[Nv*3], tris[F*3], edges[E*2], the three candidate arrays.  Outputs
 * (device, caller-owned): *alpha; *flags (EIPC_FLAG_PENETRATION / NONFINITE / ACCD_CAP /
 * BAD_INDEX, may be NULL); *n_advanced (candidates whose boxes overlap, may be NULL).
 * Scratch: a fixed device array inside the library holding two padded copies of the
 * positions, for at most eipc_accd_static_max_vertices() = 131,072 vertices (8 MiB plus a
 * 256-byte header, resident on every device that loads the library until the process
 * exits).  Nv above that returns EIPC_ERR_TOO_LARGE before anything is enqueued.
 * The first call on a device looks up that array's device address with the device
 * current (cudaGetSymbolAddress); make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset the library's module
 * is loaded again and the array may move, so a process that resets a device must not
 * call this entry point on that device afterwards.  Every
 * call re-initialises the scratch it needs, but all calls share the one array, so calls
 * whose work overlaps on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller. */
eipc_status eipc_accd_toi_static(int64_t Nv, int64_t F, int64_t E, const double* x, const double* dx,
                                 const int32_t* tris, const int32_t* edges, int64_t n_cand,
                                 const int32_t* cand_type, const int32_t* cand_i, const int32_t* cand_j,
                                 const eipc_params* p, double* alpha, int32_t* flags, int64_t* n_advanced,
                                 eipc_stream stream);
int64_t eipc_accd_static_max_vertices(void);

/* FP64 throughput probe, a measurement utility with no counterpart in the paper: one
 * launch of eight independent DFMA chains per thread, `iters` rounds each, over
 * 4 x 152 blocks of 256 threads, on `stream`.  The caller times it (CUDA events on the same
 * stream) and divides eipc_fp64_probe_flops(iters) by the time to get the device's FP64
 * rate, the denominator of the FP64 rooflines.  sink: caller-owned DEVICE double array of
 * at least 152 * 4 * 256 entries (only entry 0 is written in practice).  iters in
 * [1, 2^30], else EIPC_ERR_INVALID.  Asynchronous. */
eipc_status eipc_fp64_probe(int64_t iters, double* sink, eipc_stream stream);
int64_t eipc_fp64_probe_flops(int64_t iters);

/* Library version string: static, NUL-terminated ASCII owned by the library (never NULL,
 * never freed by the caller); needs no GPU. */
const char* eipc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EMBIPC_H */
