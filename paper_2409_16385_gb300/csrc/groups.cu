// Per-scene results of a batched scene: several independent scenes concatenated into one
// (disjoint vertex and cage-node ranges, one group id per vertex).  One set of launches
// serves all of them; these calls split the last evaluation's energy and the last CCD
// step bound by group.
//
// Energy: items (contact pairs, then lagged friction pairs) are stably sorted by group,
// which keeps each group's items in evaluation order; one warp per group then sums them
// in a fixed lane order and shuffle tree.  The result depends only on the group's own items,
// so a group's energy is bitwise the same whether it is evaluated alone or in a batch.
#include "scene.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

__global__ void __launch_bounds__(kBlock) k_group_keys(const int32_t* __restrict__ item_group, const int64_t* n_items,
                                                       int64_t cap, int32_t ng, uint64_t* __restrict__ keys,
                                                       uint32_t* __restrict__ vals, int64_t* __restrict__ counts) {
  pdl_entry();
  const int64_t n = clamp_count(n_items, cap);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += grid_stride()) {
    int32_t g = item_group[k];
    g = g < 0 ? 0 : (g >= ng ? ng - 1 : g);
    keys[k] = (uint64_t)g;
    vals[k] = (uint32_t)k;
    atomicAdd(reinterpret_cast<unsigned long long*>(counts + g), 1ull);
  }
}

__global__ void k_group_prefix(const int64_t* __restrict__ counts, int32_t ng, int64_t* __restrict__ offsets) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int32_t g = 0; g < ng; ++g) {
      offsets[g] = run;
      run += counts[g];
    }
    offsets[ng] = run;
  }
}

__global__ void __launch_bounds__(kBlock) k_group_sum(const uint32_t* __restrict__ sorted, const double* __restrict__ item_E,
                                                      const int64_t* __restrict__ offsets, int32_t ng,
                                                      double* __restrict__ E_groups) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nw) {
    const int64_t b = offsets[g], e = offsets[g + 1];
    double s = 0.0;
    for (int64_t r = b + lane; r < e; r += 32) s += item_E[sorted[r]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) E_groups[g] = s;
  }
}

__global__ void k_group_alpha_out(const unsigned long long* __restrict__ bits, int32_t ng, double* __restrict__ out) {
  pdl_entry();
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
    out[g] = __longlong_as_double((long long)bits[g]);
}

}  // namespace

void group_energy_launch(eipc_scene* sc, double* E_groups, cudaStream_t s) {
  const int32_t ng = sc->n_groups;
  int64_t* counts = sc->group_count;
  int64_t* offsets = sc->group_count + (ng + 1);
  zero_ranges(s, {{counts, sizeof(int64_t) * (ng + 1)}});
  const int64_t* n_items = sc->counters + kCntItems;
  launch(k_group_keys, blocks_for(sc->item_cap), kBlock, 0, s, static_cast<const int32_t*>(sc->item_group), n_items,
         sc->item_cap, ng, sc->gkeys, sc->gvals, counts);
  const int which = radix_sort_u64(sc->gkeys, sc->gvals, sc->gkeys_alt, sc->gvals_alt, n_items, sc->item_cap,
                                   bits_for((uint64_t)ng), sc->sort_hist, s);
  const uint32_t* sorted = which ? sc->gvals_alt : sc->gvals;
  launch(k_group_prefix, 1, 32, 0, s, static_cast<const int64_t*>(counts), ng, offsets);
  launch(k_group_sum, blocks_for((int64_t)ng * 32, 8), kBlock, 0, s, sorted, static_cast<const double*>(sc->item_E),
         static_cast<const int64_t*>(offsets), ng, E_groups);
}

void group_alpha_launch(eipc_scene* sc, double* alpha_groups, cudaStream_t s) {
  launch(k_group_alpha_out, blocks_for(sc->n_groups), kBlock, 0, s,
         static_cast<const unsigned long long*>(sc->group_alpha_bits), sc->n_groups, alpha_groups);
}

}  // namespace eipc
