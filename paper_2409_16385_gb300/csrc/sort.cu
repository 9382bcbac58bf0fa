// Stable LSD radix sort, exclusive scan and segment starts with device-resident element
// counts.
//
// Radix pass (8-bit digit): each of kSortBlocks blocks owns one contiguous chunk of the
// input.  (1) per-block digit histograms, (2) one block per digit turns its counts into
// exclusive per-block prefixes and a digit total, (3) each block scans the 256 digit totals
// for its digit bases and scatters its chunk tile by tile: warp peers
// with equal digits are found with __match_any_sync, per-warp digit counts are prefix-
// summed across the block's 8 warps, so every element lands at a position that preserves
// input order among equal digits (stability is what makes the sort-and-reduce of the
// reduced Hessian deterministic).
#include "common.cuh"
#include "sort.cuh"

namespace eipc {
namespace {

__device__ __forceinline__ void chunk_range(int64_t n, int64_t* beg, int64_t* end) {
  int64_t per = (n + kSortBlocks - 1) / kSortBlocks;
  per = (per + kSortThreads - 1) / kSortThreads * kSortThreads;
  *beg = (int64_t)blockIdx.x * per;
  int64_t e = *beg + per;
  *end = e < n ? e : n;
}

__global__ void __launch_bounds__(kSortThreads) k_hist(const uint64_t* __restrict__ keys,
                                                       const int64_t* n_dev, int64_t cap, int shift,
                                                       uint32_t* __restrict__ hist) {
  pdl_entry();
  __shared__ uint32_t h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  chunk_range(n, &beg, &end);
  // one shared-memory atomic per distinct digit of a warp's 32 elements (the record keys of
  // the reduction are heavily skewed: a few thousand distinct keys over millions)
  const uint32_t lt_mask = (1u << (threadIdx.x & 31)) - 1u;
  for (int64_t i0 = beg; i0 < end; i0 += blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const uint32_t d = i < end ? (uint32_t)((keys[i] >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 256u && (peers & lt_mask) == 0u) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * kSortBlocks + blockIdx.x] = h[d];
}

// One block per digit: exclusive prefix of that digit's counts over the blocks (in place)
// and the digit's total, stored after the 256 * kSortBlocks counters.  Thread t owns the
// consecutive counters [t * per, (t + 1) * per); a block scan of the threads' sums gives
// each its starting offset.
__global__ void __launch_bounds__(256) k_hist_digits(uint32_t* hist) {
  pdl_entry();
  constexpr int per = (kSortBlocks + 255) / 256;
  __shared__ uint32_t wsum[8];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t* row = hist + (size_t)blockIdx.x * kSortBlocks;
  uint32_t c[per];
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int b = t * per + k;
    c[k] = b < kSortBlocks ? row[b] : 0u;
    mine += c[k];
  }
  uint32_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    before += w < warp ? wsum[w] : 0u;
    all += wsum[w];
  }
  uint32_t run = before + x - mine;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int b = t * per + k;
    if (b < kSortBlocks) row[b] = run;
    run += c[k];
  }
  if (t == 0) hist[256 * kSortBlocks + blockIdx.x] = all;
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint64_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint64_t* __restrict__ kout,
                                                          uint32_t* __restrict__ vout,
                                                          const int64_t* n_dev, int64_t cap, int shift,
                                                          const uint32_t* __restrict__ offs) {
  pdl_entry();
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[W][257];
  __shared__ uint32_t total[256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  chunk_range(n, &beg, &end);
  // digit bases: exclusive scan of the 256 digit totals, plus this block's prefix
  if (t < 256) total[t] = offs[256 * kSortBlocks + t];
  __syncthreads();
  if (t < 32) {
    uint32_t run = 0;
    for (int d0 = 0; d0 < 256; d0 += 32) {
      const uint32_t c = total[d0 + t];
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (t >= o) x += y;
      }
      base[d0 + t] = run + x - c;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  __syncthreads();
  for (int d = t; d < 256; d += blockDim.x) base[d] += offs[d * kSortBlocks + blockIdx.x];
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int64_t tile = beg; tile < end; tile += kSortThreads) {
    for (int d = lane; d < 257; d += 32) wcnt[warp][d] = 0;
    __syncthreads();
    int64_t i = tile + t;
    bool valid = i < end;
    uint64_t key = valid ? kin[i] : 0;
    uint32_t val = valid ? vin[i] : 0;
    uint32_t digit = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, digit);
    uint32_t rank = __popc(peers & lt_mask);
    if (rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (t < 256) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        uint32_t c = wcnt[w][t];
        wcnt[w][t] = run;
        run += c;
      }
      total[t] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base[digit] + wcnt[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    if (t < 256) base[t] += total[t];
  }
}

// ---------------------------------------------------------------- exclusive scan
__device__ __forceinline__ void scan_range(int64_t n, int64_t* beg, int64_t* end) {
  int64_t per = (n + kScanBlocks - 1) / kScanBlocks;
  *beg = (int64_t)blockIdx.x * per;
  int64_t e = *beg + per;
  *end = e < n ? e : n;
}

__device__ int64_t block_sum_i64(int64_t v) {
  __shared__ int64_t ws[32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  int64_t r = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += ws[w];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_scan_partial(const int64_t* __restrict__ in, const int64_t* n_dev,
                                                      int64_t cap, int64_t* __restrict__ partial) {
  pdl_entry();
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t s = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) s += in[i];
  s = block_sum_i64(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// exclusive scan of the kScanBlocks partial sums by one warp (chunks of 32 with a carry)
__global__ void k_scan_partials(int64_t* partial, int64_t* total) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int b0 = 0; b0 < kScanBlocks; b0 += 32) {
    const int b = b0 + lane;
    const int64_t c = b < kScanBlocks ? partial[b] : 0;
    int64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < kScanBlocks) partial[b] = run + x - c;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) {
    partial[kScanBlocks] = run;
    if (total) *total = run;
  }
}

__global__ void __launch_bounds__(256) k_scan_apply(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                    const int64_t* n_dev, int64_t cap,
                                                    const int64_t* __restrict__ partial) {
  pdl_entry();
  __shared__ int64_t tile_sum[256];
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t run = partial[blockIdx.x];
  const int t = threadIdx.x;
  for (int64_t tile = beg; tile < end; tile += 256) {
    int64_t i = tile + t;
    int64_t v = (i < end) ? in[i] : 0;
    tile_sum[t] = v;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      int64_t u = (t >= off) ? tile_sum[t - off] : 0;
      __syncthreads();
      tile_sum[t] += u;
      __syncthreads();
    }
    if (i < end) out[i] = run + tile_sum[t] - v;
    int64_t tot = tile_sum[255];
    __syncthreads();
    run += tot;
  }
}

// ---- two exclusive scans of the same length in the launches of one: partial holds
// 2 (kScanBlocks + 1) entries, the first array's partials then the second's
__global__ void __launch_bounds__(256) k_scan2_partial(const int64_t* __restrict__ a, const int64_t* __restrict__ b,
                                                       const int64_t* n_dev, int64_t cap, int64_t* __restrict__ partial) {
  pdl_entry();
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t sa = 0, sb = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    sa += a[i];
    sb += b[i];
  }
  sa = block_sum_i64(sa);
  sb = block_sum_i64(sb);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sa;
    partial[kScanBlocks + 1 + blockIdx.x] = sb;
  }
}

// exclusive scans of both partial arrays, one warp each
__global__ void k_scan2_partials(int64_t* partial, int64_t* total_a, int64_t* total_b) {
  pdl_entry();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w > 1 || blockIdx.x != 0) return;
  int64_t* p = partial + w * (kScanBlocks + 1);
  int64_t* total = w == 0 ? total_a : total_b;
  int64_t run = 0;
  for (int b0 = 0; b0 < kScanBlocks; b0 += 32) {
    const int b = b0 + lane;
    const int64_t c = b < kScanBlocks ? p[b] : 0;
    int64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < kScanBlocks) p[b] = run + x - c;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) {
    p[kScanBlocks] = run;
    if (total) *total = run;
  }
}

// both arrays' tiles: one block-wide scan of (a, b) pairs per tile
__global__ void __launch_bounds__(256) k_scan2_apply(const int64_t* __restrict__ a, int64_t* __restrict__ out_a,
                                                     const int64_t* __restrict__ b, int64_t* __restrict__ out_b,
                                                     const int64_t* n_dev, int64_t cap,
                                                     const int64_t* __restrict__ partial) {
  pdl_entry();
  __shared__ int64_t ta[256], tb[256];
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t run_a = partial[blockIdx.x], run_b = partial[kScanBlocks + 1 + blockIdx.x];
  const int t = threadIdx.x;
  for (int64_t tile = beg; tile < end; tile += 256) {
    const int64_t i = tile + t;
    const int64_t va = (i < end) ? a[i] : 0, vb = (i < end) ? b[i] : 0;
    ta[t] = va;
    tb[t] = vb;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      const int64_t ua = (t >= off) ? ta[t - off] : 0, ub = (t >= off) ? tb[t - off] : 0;
      __syncthreads();
      ta[t] += ua;
      tb[t] += ub;
      __syncthreads();
    }
    if (i < end) {
      out_a[i] = run_a + ta[t] - va;
      out_b[i] = run_b + tb[t] - vb;
    }
    const int64_t sa = ta[255], sb = tb[255];
    __syncthreads();
    run_a += sa;
    run_b += sb;
  }
}

// ---- segment starts of a sorted key array (a segment = a run of equal keys)

__device__ __forceinline__ int64_t seg_head(const uint64_t* __restrict__ keys, int64_t i) {
  return (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// per-chunk number of segment heads (chunks of scan_range)
__global__ void __launch_bounds__(256) k_seg_heads_partial(const uint64_t* __restrict__ keys, const int64_t* n_dev,
                                                           int64_t cap, int64_t* __restrict__ partial) {
  pdl_entry();
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t c = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) c += seg_head(keys, i);
  c = block_sum_i64(c);
  if (threadIdx.x == 0) partial[blockIdx.x] = c;
}

// start[s] = position of the s-th head: each chunk ranks its heads tile by tile from its
// exclusive partial
__global__ void __launch_bounds__(256) k_seg_heads_write(const uint64_t* __restrict__ keys, const int64_t* n_dev,
                                                         int64_t cap, const int64_t* __restrict__ partial,
                                                         int64_t* __restrict__ start, const uint32_t* __restrict__ perm,
                                                         uint32_t* __restrict__ inv) {
  pdl_entry();
  __shared__ int32_t wsum[8];
  int64_t n = *n_dev;
  if (n > cap) n = cap;
  int64_t beg, end;
  scan_range(n, &beg, &end);
  int64_t run = partial[blockIdx.x];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int64_t tile = beg; tile < end; tile += 256) {
    const int64_t i = tile + t;
    if (inv && i < end) inv[perm[i]] = (uint32_t)i;
    const bool h = i < end && seg_head(keys, i);
    const unsigned m = __ballot_sync(0xffffffffu, h);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      before += w < warp ? wsum[w] : 0;
      all += wsum[w];
    }
    if (h) start[run + before + __popc(m & ((1u << lane) - 1u))] = i;
    __syncthreads();
    run += all;
  }
}

struct ZeroArgs {
  uint32_t* p[kZeroRanges];
  int64_t n[kZeroRanges];
  int count;
};

__global__ void __launch_bounds__(kBlock) k_zero_ranges(ZeroArgs z) {
  pdl_entry();
  for (int r = 0; r < z.count; ++r)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < z.n[r]; i += grid_stride()) z.p[r][i] = 0u;
}

}  // namespace

void zero_ranges(cudaStream_t s, std::initializer_list<ZeroRange> ranges) {
  ZeroArgs z{};
  int64_t most = 0;
  for (const ZeroRange& r : ranges) {
    if (r.ptr == nullptr || r.bytes == 0) continue;
    z.p[z.count] = static_cast<uint32_t*>(r.ptr);
    z.n[z.count] = (int64_t)(r.bytes / 4);
    if (z.n[z.count] > most) most = z.n[z.count];
    if (++z.count == kZeroRanges) {          // more ranges than one launch takes
      launch(k_zero_ranges, blocks_for(most, 4), kBlock, 0, s, z);
      z = ZeroArgs{};
      most = 0;
    }
  }
  if (z.count > 0) launch(k_zero_ranges, blocks_for(most, 4), kBlock, 0, s, z);
}

int radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                   const int64_t* n, int64_t cap, int bits, uint32_t* hist, cudaStream_t s, int start_bit) {
  int which = 0;
  for (int shift = start_bit; shift < start_bit + bits; shift += 8) {
    uint64_t* ki = which ? keys_alt : keys;
    uint32_t* vi = which ? vals_alt : vals;
    uint64_t* ko = which ? keys : keys_alt;
    uint32_t* vo = which ? vals : vals_alt;
    launch(k_hist, kSortBlocks, kSortThreads, 0, s, ki, n, cap, shift, hist);
    launch(k_hist_digits, 256, 256, 0, s, hist);
    launch(k_scatter, kSortBlocks, kSortThreads, 0, s, ki, vi, ko, vo, n, cap, shift, hist);
    which ^= 1;
  }
  return which;
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, const int64_t* n, int64_t cap, int64_t* total,
                        int64_t* partial, cudaStream_t s) {
  launch(k_scan_partial, kScanBlocks, 256, 0, s, in, n, cap, partial);
  launch(k_scan_partials, 1, 32, 0, s, partial, total);
  launch(k_scan_apply, kScanBlocks, 256, 0, s, in, out, n, cap, partial);
}

void exclusive_scan2_i64(const int64_t* in_a, int64_t* out_a, int64_t* total_a, const int64_t* in_b, int64_t* out_b,
                         int64_t* total_b, const int64_t* n, int64_t cap, int64_t* partial, cudaStream_t s) {
  launch(k_scan2_partial, kScanBlocks, 256, 0, s, in_a, in_b, n, cap, partial);
  launch(k_scan2_partials, 1, 64, 0, s, partial, total_a, total_b);
  launch(k_scan2_apply, kScanBlocks, 256, 0, s, in_a, out_a, in_b, out_b, n, cap, static_cast<const int64_t*>(partial));
}

void segment_starts(const uint64_t* keys, const int64_t* n, int64_t cap, int64_t* start, int64_t* n_seg,
                    int64_t* partial, cudaStream_t s, const uint32_t* perm, uint32_t* inv) {
  launch(k_seg_heads_partial, kScanBlocks, 256, 0, s, keys, n, cap, partial);
  launch(k_scan_partials, 1, 32, 0, s, partial, n_seg);
  launch(k_seg_heads_write, kScanBlocks, 256, 0, s, keys, n, cap, static_cast<const int64_t*>(partial), start, perm, inv);
}

}  // namespace eipc
