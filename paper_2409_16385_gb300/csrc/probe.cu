// FP64 throughput probe: the denominator of the FP64 rooflines of the evaluation and CCD
// kernels, measured on the device the library runs on instead of taken from a data sheet.
// Every thread runs `iters` rounds of eight independent DFMA chains (a <- a * m + c), so
// the FP64 pipe always has independent work and nothing else is issued in the loop; the
// chains' sum is written out so that the compiler keeps them.  FP64 flops per launch =
// blocks x threads x iters x 8 x 2.
#include "common.cuh"

namespace eipc {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int64_t iters, double m, double c, double* sink) {
  pdl_entry();
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains
  if (blockIdx.x == 0 && threadIdx.x == 0) sink[0] = s;
}

}  // namespace
}  // namespace eipc

extern "C" int64_t eipc_fp64_probe_flops(int64_t iters) {
  return (int64_t)eipc::kSMs * eipc::kProbeBlocksPerSM * eipc::kProbeThreads * iters * 16;
}

extern "C" eipc_status eipc_fp64_probe(int64_t iters, double* sink, eipc_stream stream) {
  using namespace eipc;
  if (iters < 1 || iters > (1ll << 30) || !sink) return EIPC_ERR_INVALID;
  // m slightly below 1 and c small: the chains stay finite and normal for any iters
  launch(k_fp64_probe, kSMs * kProbeBlocksPerSM, kProbeThreads, 0, (cudaStream_t)stream, iters, 0.999999999,
         1e-9, sink);
  return cudaPeekAtLastError() == cudaSuccess ? EIPC_OK : EIPC_ERR_CUDA;
}
