// Sorting and scan primitives whose element counts live in device memory, so that they
// can run inside a captured CUDA graph without any host read-back.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>

namespace eipc {

constexpr int kSortBlocks = 1216;  // 8 per SM; each block owns one contiguous chunk
constexpr int kSortThreads = 256;  // 8 warps, one element per thread per tile

// Scratch: 256 * kSortBlocks digit counters followed by 256 digit totals.
inline size_t sort_hist_entries() { return 256u * kSortBlocks + 256u; }

// Stable LSD radix sort of (keys[i], vals[i]), i < min(*n, cap), by the key's bits
// [start_bit, start_bit + 8 ceil(bits / 8)) in 8-bit digits: bits below start_bit are
// ignored (equal there keeps the input order), and every key must be below
// 2^(start_bit + bits) (bits above the last whole digit are ignored, bits inside it are not).
// Ping-pongs between (keys, vals) and (keys_alt, vals_alt); returns 0 if the sorted
// result ends in (keys, vals), 1 if it ends in the alternate buffers.
int radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                   const int64_t* n, int64_t cap, int bits, uint32_t* hist, cudaStream_t s, int start_bit = 0);

// out[i] = sum_{k<i} in[k] for i < min(*n, cap); *total = the full sum.
// partial needs kScanBlocks + 1 entries.
constexpr int kScanBlocks = 304;
void exclusive_scan_i64(const int64_t* in, int64_t* out, const int64_t* n, int64_t cap,
                        int64_t* total, int64_t* partial, cudaStream_t s);

// Two exclusive scans over the same count in three launches (as two exclusive_scan_i64
// calls).  partial needs 2 (kScanBlocks + 1) entries.
void exclusive_scan2_i64(const int64_t* in_a, int64_t* out_a, int64_t* total_a, const int64_t* in_b, int64_t* out_b,
                         int64_t* total_b, const int64_t* n, int64_t cap, int64_t* partial, cudaStream_t s);

// Segments of a sorted key array keys[0 .. min(*n, cap)), a segment being a run of equal
// keys: start[s] = position of segment s's first element, *n_seg = the number of segments.
// With perm (the sort's values: the original index of each sorted element), also the
// inverse permutation inv[perm[i]] = i.  partial needs kScanBlocks + 1 entries.
void segment_starts(const uint64_t* keys, const int64_t* n, int64_t cap, int64_t* start, int64_t* n_seg,
                    int64_t* partial, cudaStream_t s, const uint32_t* perm = nullptr, uint32_t* inv = nullptr);

// Zeroes up to kZeroRanges byte ranges in one launch (each range 4-byte aligned, its
// length a multiple of 4 bytes).  The library resets its counters and accumulators with
// this kernel rather than cudaMemsetAsync, so the reset stays on the programmatic-launch
// chain of the stream instead of breaking it.
constexpr int kZeroRanges = 6;
struct ZeroRange {
  void* ptr;
  size_t bytes;
};
void zero_ranges(cudaStream_t s, std::initializer_list<ZeroRange> ranges);

}  // namespace eipc
