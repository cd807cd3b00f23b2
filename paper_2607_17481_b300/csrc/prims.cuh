// Device-wide primitives: segmented scans and a stable LSD radix sort.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pn {

// Inclusive segmented sum over uint32 values: out[t] = sum of in[s..t] where s
// is the last index <= t with head[s] != 0 (or 0).  head may be null (one
// segment).  Scratch is taken with cudaMallocAsync on the stream.
cudaError_t seg_scan_u32(const uint32_t *in, const uint8_t *head, uint32_t *out, int64_t n,
                         cudaStream_t st);

// Inclusive segmented sum over (double, double) pairs, same contract.
cudaError_t seg_scan_d2(const double2 *in, const uint8_t *head, double2 *out, int64_t n,
                        cudaStream_t st);

// Exclusive (unsegmented) sum over uint32 values; *total receives the sum
// (device pointer, may be null).
cudaError_t excl_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                          cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the
// key.  Sorts in place (keys/vals), using two scratch arrays of n entries.
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t st);

}  // namespace pn
