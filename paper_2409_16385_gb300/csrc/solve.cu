// Sparse products for the reduced Newton solve: y = alpha A x + beta y for a 3x3-block CSR
// (BSR) matrix A, the layout eipc_eval_contact returns H_r in.  One warp per block row:
// lanes take the row's blocks in a fixed stride and a fixed shuffle tree adds them, so
// the result does not depend on the launch.
#include "scene.cuh"

namespace eipc {
namespace {

__global__ void __launch_bounds__(kBlock) k_bsr_spmv(int64_t nrows, const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col, const double* __restrict__ val,
                                                     const double* __restrict__ x, double alpha, double beta,
                                                     double* __restrict__ y) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
    const int32_t b = row_ptr[r], e = row_ptr[r + 1];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int32_t k = b + lane; k < e; k += 32) {
      const double* B = val + 9 * (int64_t)k;
      const int64_t c = col[k];
      const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      a0 += B[0] * x0 + B[1] * x1 + B[2] * x2;
      a1 += B[3] * x0 + B[4] * x1 + B[5] * x2;
      a2 += B[6] * x0 + B[7] * x1 + B[8] * x2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      const double y0 = beta == 0.0 ? 0.0 : beta * y[3 * r];
      const double y1 = beta == 0.0 ? 0.0 : beta * y[3 * r + 1];
      const double y2 = beta == 0.0 ? 0.0 : beta * y[3 * r + 2];
      y[3 * r] = y0 + alpha * a0;
      y[3 * r + 1] = y1 + alpha * a1;
      y[3 * r + 2] = y2 + alpha * a2;
    }
  }
}

}  // namespace

void bsr_spmv_launch(int64_t nrows, const int32_t* row_ptr, const int32_t* col, const double* val, const double* x,
                     double alpha, double beta, double* y, cudaStream_t s) {
  if (nrows <= 0) return;
  launch(k_bsr_spmv, blocks_for(nrows * 32, 16), kBlock, 0, s, nrows, row_ptr, col, val, x, alpha, beta, y);
}

}  // namespace eipc
