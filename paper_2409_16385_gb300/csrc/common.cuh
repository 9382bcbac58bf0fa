// Shared device-side definitions of the embipc library: status word, small vector
// helpers and launch helpers.  Every kernel that depends on a device-side count uses a
// grid-stride loop bounded by that count, so launches never need a host read-back.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "../../include/embipc.h"

namespace eipc {

// Process-wide count of kernel launches enqueued by the library (eipc_launch_count).
inline std::atomic<long long> g_launches{0};
// Process-wide launch mode (eipc_set_programmatic_launch): 1 = programmatic dependent
// launch, 0 = plain stream order.
inline std::atomic<int> g_programmatic{1};

// Every kernel of the library is launched through here.  With programmatic stream
// serialisation a kernel may be scheduled while the kernel before it in the stream is
// still running (its CTAs occupy free slots and its launch latency overlaps the
// predecessor's tail); correctness rests on pdl_entry() below being the first statement
// of every kernel.
template <class... KArgs, class... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_programmatic.load(std::memory_order_relaxed);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// First statement of every kernel.  griddepcontrol.wait returns once the grids this one
// depends on (the previous kernel in the stream, when launched programmatically) have
// completed and their memory operations are visible; it returns at once otherwise.  Since
// every kernel waits before it can complete, completion stays transitive along the stream.
// launch_dependents then lets the next kernel's CTAs be scheduled once every CTA of this
// grid has started, so they never compete with this grid's own unscheduled CTAs.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

constexpr int kSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kBlock = 256;

// Device status word shared by all kernels of a scene.
struct DevStatus {
  int32_t flags;          // OR of EIPC_FLAG_*
  int32_t pad;
  int64_t need_pairs;     // required capacities after an overflow
  int64_t need_cand;
  int64_t need_rec;
  int64_t need_bsr;
  unsigned long long accd_iters;
};

__device__ __forceinline__ void raise_flag(DevStatus* st, int32_t f) { atomicOr(&st->flags, f); }

__device__ __forceinline__ void raise_need(DevStatus* st, int64_t* field, int64_t n) {
  atomicMax(reinterpret_cast<unsigned long long*>(field), static_cast<unsigned long long>(n));
}

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// x is stored padded: 4 doubles per vertex (x, y, z, 0), 32-byte aligned, so a vertex
// gather is two aligned 16-byte loads from one sector.
__device__ __forceinline__ V3 load_x(const double* __restrict__ x4, int32_t v) {
  const double2* p = reinterpret_cast<const double2*>(x4 + 4 * (int64_t)v);
  double2 a = __ldg(p), b = __ldg(p + 1);
  return {a.x, a.y, b.x};
}

__device__ __forceinline__ int grid_stride() { return gridDim.x * blockDim.x; }

// Number of blocks for a grid-stride loop over at most `n_max` items.
inline int blocks_for(int64_t n_max, int per_sm = 8, int block = kBlock) {
  int64_t b = (n_max + block - 1) / block;
  int64_t cap = (int64_t)kSMs * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// clamp a device-side count to a capacity (the producer flagged the overflow)
__device__ __forceinline__ int64_t clamp_count(const int64_t* count, int64_t cap) {
  int64_t n = *count;
  return n < cap ? n : cap;
}

}  // namespace eipc
