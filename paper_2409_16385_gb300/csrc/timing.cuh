// Per-kernel CUDA-event timers.  When enabled for a kernel id, every launch of that kernel
// (or kernel group) is bracketed by two events recorded on the launching stream; reading
// the timers synchronises and returns the summed device time and launch count.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eipc {

enum KernelId {
  kKEmbed = 0,       // k_embed / k_pad
  kKBvh = 1,         // Morton codes + radix sort + hierarchy + refit (group)
  kKQuery = 2,       // BVH traversal producing candidates
  kKNarrow = 3,      // exact FP64 distance filter
  kKPairSort = 4,    // canonical sort of the pair list + emit (group)
  kKLag = 5,         // lagged friction state
  kKItems = 6,       // stencil cage nodes + record offsets (group)
  kKEvalBarrier = 7, // barrier energy, gradient, projected Hessian, records
  kKEvalFriction = 8,
  kKHReduce = 9,     // sort-and-reduce of Hessian blocks into BSR (group)
  kKGReduce = 10,    // sort-and-reduce of the reduced gradient (group)
  kKEnergy = 11,
  kKCa = 12,         // conservative advancement of CCD candidates
  kKEvalPair = 13,   // barrier and friction evaluation together (they overlap on two streams)
  kKNum = 14
};

constexpr int kTimerRing = 512;

struct Timers {
  uint32_t mask = 0;
  bool created = false;
  cudaEvent_t ev[kKNum][kTimerRing][2];
  int pending[kKNum] = {};
  double total_ms[kKNum] = {};
  int64_t launches[kKNum] = {};

  void create() {
    if (created) return;
    for (int k = 0; k < kKNum; ++k)
      for (int r = 0; r < kTimerRing; ++r) {
        cudaEventCreate(&ev[k][r][0]);
        cudaEventCreate(&ev[k][r][1]);
      }
    created = true;
  }
  void destroy() {
    if (!created) return;
    for (int k = 0; k < kKNum; ++k)
      for (int r = 0; r < kTimerRing; ++r) {
        cudaEventDestroy(ev[k][r][0]);
        cudaEventDestroy(ev[k][r][1]);
      }
    created = false;
  }
  void drain(int k) {
    if (pending[k] == 0) return;
    cudaEventSynchronize(ev[k][pending[k] - 1][1]);
    for (int r = 0; r < pending[k]; ++r) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k][r][0], ev[k][r][1]) == cudaSuccess) total_ms[k] += ms;
      ++launches[k];
    }
    pending[k] = 0;
  }
  bool on(int k) const { return created && (mask >> k) & 1u; }
  void start(int k, cudaStream_t s) {
    if (!on(k)) return;
    if (pending[k] == kTimerRing) drain(k);
    cudaEventRecord(ev[k][pending[k]][0], s);
  }
  void stop(int k, cudaStream_t s) {
    if (!on(k)) return;
    cudaEventRecord(ev[k][pending[k]][1], s);
    ++pending[k];
  }
};

}  // namespace eipc
