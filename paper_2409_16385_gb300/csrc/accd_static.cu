// eipc_accd_toi_static: the CCD step bound over a caller-supplied candidate list, with
// its scratch memory in a fixed-size device array compiled into the library, so the call
// allocates no device memory at all.
//
// The advancement arithmetic is the same as the scene-based eipc_accd_toi (accd.cu): exact
// FP64 closed swept-box test, mean displacement removed, L = largest relative speed on
// each side, advance by (1 - s) d(t) / L until d <= s d(0), t >= 1 or max_iter advances;
// the pair's t is scaled by (1 - 2^-30) and alpha is the exact minimum over pairs.
// Incident candidates (sharing a vertex) are skipped here because the caller builds the
// list.
#include <mutex>

#include "geometry.cuh"

namespace eipc {
namespace {

constexpr int64_t kStaticMaxVertices = 1 << 17;   // 131,072 vertices
constexpr int kStaticThreads = 128;
constexpr double kStaticMargin = 1.0 - 9.313225746154785e-10;   // 1 - 2^-30

// Layout: [0, 256): alpha bits (u64) at 0, flags (i32) at 8, advanced count (u64) at 16;
// then padded x (32 B per vertex), then padded dx.
constexpr size_t kStaticHeader = 256;
constexpr size_t kStaticBytes = kStaticHeader + 2 * (size_t)kStaticMaxVertices * 32;

static __device__ __align__(256) unsigned char g_accd_scratch[kStaticBytes];

struct StaticView {
  unsigned long long* alpha_bits;
  int32_t* flags;
  unsigned long long* n_adv;
  double* x4;
  double* dx4;
};

__host__ __device__ inline StaticView view_of(unsigned char* base) {
  StaticView v;
  v.alpha_bits = reinterpret_cast<unsigned long long*>(base);
  v.flags = reinterpret_cast<int32_t*>(base + 8);
  v.n_adv = reinterpret_cast<unsigned long long*>(base + 16);
  v.x4 = reinterpret_cast<double*>(base + kStaticHeader);
  v.dx4 = reinterpret_cast<double*>(base + kStaticHeader + (size_t)kStaticMaxVertices * 32);
  return v;
}

// every call starts from alpha = 1, no flags, no advanced pairs
__global__ void k_static_init(unsigned char* base) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    StaticView v = view_of(base);
    *v.alpha_bits = (unsigned long long)__double_as_longlong(1.0);
    *v.flags = 0;
    *v.n_adv = 0ull;
  }
}

__global__ void __launch_bounds__(256) k_static_pad(const double* __restrict__ x, const double* __restrict__ dx,
                                                    int64_t nv, unsigned char* base) {
  pdl_entry();
  StaticView sv = view_of(base);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const double a = x[3 * v], b = x[3 * v + 1], c = x[3 * v + 2];
    const double e = dx[3 * v], f = dx[3 * v + 1], g = dx[3 * v + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(e) && isfinite(f) && isfinite(g)))
      atomicOr(sv.flags, EIPC_FLAG_NONFINITE);
    reinterpret_cast<double2*>(sv.x4)[2 * v] = make_double2(a, b);
    reinterpret_cast<double2*>(sv.x4)[2 * v + 1] = make_double2(c, 0.0);
    reinterpret_cast<double2*>(sv.dx4)[2 * v] = make_double2(e, f);
    reinterpret_cast<double2*>(sv.dx4)[2 * v + 1] = make_double2(g, 0.0);
  }
}

__device__ __forceinline__ double static_pair_distance(int type, const V3 p[4]) {
  const V3 o = p[0];
  if (type == 0) return sqrt(pt_distance<false>(p[0] - o, p[1] - o, p[2] - o, p[3] - o, nullptr));
  return sqrt(ee_distance<false>(p[0] - o, p[1] - o, p[2] - o, p[3] - o, nullptr));
}

__global__ void __launch_bounds__(kStaticThreads) k_static_ca(int64_t nv, int64_t nf, int64_t ne,
                                                              const int32_t* __restrict__ tris,
                                                              const int32_t* __restrict__ edges, int64_t nc,
                                                              const int32_t* __restrict__ ctype,
                                                              const int32_t* __restrict__ ci,
                                                              const int32_t* __restrict__ cj, double s, int max_iter,
                                                              unsigned char* base) {
  pdl_entry();
  StaticView sv = view_of(base);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x) {
    const int type = ctype[k];
    const int32_t i = ci[k], j = cj[k];
    const bool ids_ok = (type == 0) ? (i >= 0 && i < nv && j >= 0 && j < nf)
                                    : (type == 1 && i >= 0 && i < ne && j >= 0 && j < ne);
    if (!ids_ok) {
      atomicOr(sv.flags, EIPC_FLAG_BAD_INDEX);
      continue;
    }
    int32_t v[4];
    if (type == 0) {
      v[0] = i;
      v[1] = tris[3 * (int64_t)j]; v[2] = tris[3 * (int64_t)j + 1]; v[3] = tris[3 * (int64_t)j + 2];
    } else {
      v[0] = edges[2 * (int64_t)i]; v[1] = edges[2 * (int64_t)i + 1];
      v[2] = edges[2 * (int64_t)j]; v[3] = edges[2 * (int64_t)j + 1];
    }
    bool bad_id = false;
    for (int a = 0; a < 4; ++a) bad_id |= (v[a] < 0 || v[a] >= nv);
    if (bad_id) {
      atomicOr(sv.flags, EIPC_FLAG_BAD_INDEX);
      continue;
    }
    const int na = type == 0 ? 1 : 2;
    bool incident = false;
    for (int a = 0; a < na; ++a)
      for (int b = na; b < 4; ++b) incident |= (v[a] == v[b]);
    if (incident) continue;
    V3 X[4], D[4];
    for (int a = 0; a < 4; ++a) { X[a] = load_x(sv.x4, v[a]); D[a] = load_x(sv.dx4, v[a]); }
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
    if (!ov) continue;
    atomicAdd(sv.n_adv, 1ull);
    const V3 mean = (D[0] + D[1] + D[2] + D[3]) * 0.25;
    V3 R[4];
    double la = 0.0, lb = 0.0;
    for (int a = 0; a < 4; ++a) {
      R[a] = D[a] - mean;
      const double sp = sqrt(dot(R[a], R[a]));
      if (a < na) la = fmax(la, sp); else lb = fmax(lb, sp);
    }
    const double L = la + lb;
    double t = 1.0;
    if (L > 0.0) {
      const double d0 = static_pair_distance(type, X);
      if (!(d0 > 0.0)) {
        atomicOr(sv.flags, EIPC_FLAG_PENETRATION);
        t = 0.0;
      } else {
        double d = d0;
        int iters = 0;
        t = 0.0;
        while (true) {
          const double tn = t + (1.0 - s) * d / L;
          if (tn >= 1.0) { t = 1.0; break; }
          t = tn;
          V3 P[4];
          for (int a = 0; a < 4; ++a) P[a] = X[a] + R[a] * t;
          d = static_pair_distance(type, P);
          ++iters;
          if (d <= s * d0) break;
          if (iters >= max_iter) { atomicOr(sv.flags, EIPC_FLAG_ACCD_CAP); break; }
        }
      }
    }
    if (t < 1.0) atomicMin(sv.alpha_bits, (unsigned long long)__double_as_longlong(t * kStaticMargin));
  }
}

__global__ void k_static_out(const unsigned char* base, double* alpha, int32_t* flags, int64_t* n_adv) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    StaticView v = view_of(const_cast<unsigned char*>(base));
    *alpha = __longlong_as_double((long long)*v.alpha_bits);
    if (flags) *flags = *v.flags;
    if (n_adv) *n_adv = (int64_t)*v.n_adv;
  }
}

// Device address of g_accd_scratch, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_accd_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace eipc

extern "C" int64_t eipc_accd_static_max_vertices(void) { return eipc::kStaticMaxVertices; }

extern "C" eipc_status eipc_accd_toi_static(int64_t Nv, int64_t F, int64_t E, const double* x, const double* dx,
                                            const int32_t* tris,
                                            const int32_t* edges, int64_t n_cand, const int32_t* cand_type,
                                            const int32_t* cand_i, const int32_t* cand_j, const eipc_params* p,
                                            double* alpha, int32_t* flags, int64_t* n_advanced,
                                            eipc_stream stream) {
  using namespace eipc;
  if (Nv <= 0 || Nv > kStaticMaxVertices) return EIPC_ERR_TOO_LARGE;
  if (!x || !dx || !alpha || !p || F < 0 || E < 0 || n_cand < 0 || n_cand >= (1ll << 31)) return EIPC_ERR_INVALID;
  if (n_cand > 0 && (!tris || !edges || !cand_type || !cand_i || !cand_j)) return EIPC_ERR_INVALID;
  if (!(p->accd_s > 0.0 && p->accd_s < 1.0 && p->accd_max_iter > 0)) return EIPC_ERR_INVALID;
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return EIPC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch(k_static_init, 1, 32, 0, s, base);
  int pb = (int)((Nv + 255) / 256);
  if (pb > kSMs * 4) pb = kSMs * 4;
  launch(k_static_pad, pb, 256, 0, s, x, dx, Nv, base);
  if (n_cand > 0) {
    int cb = (int)((n_cand + kStaticThreads - 1) / kStaticThreads);
    if (cb > kSMs * 16) cb = kSMs * 16;
    launch(k_static_ca, cb, kStaticThreads, 0, s, Nv, F, E, tris, edges, n_cand, cand_type, cand_i, cand_j, p->accd_s,
           (int)p->accd_max_iter, base);
  }
  launch(k_static_out, 1, 32, 0, s, static_cast<const unsigned char*>(base), alpha, flags, n_advanced);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}
