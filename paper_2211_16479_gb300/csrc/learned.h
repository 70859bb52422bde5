// Learned-CDF partitioner (declarations shared with the pass scheduler).
#pragma once

#include <cuda_runtime.h>

#include "ctx.h"

namespace msort {

// First merge pass (0-based) whose partition uses the guided search.
int learned_first_pass(const Plan& pl, size_t n);
// Draw the key sample from the unsorted input, sort it and train the network
// on the device.  Runs on a side stream that waits for `st`; the guided
// partitions on `st` use the model once its training has finished (a device
// flag), and the ratio guess before.  keys_overwritten: the sort's first
// kernel writes `keys` (in place with an even number of passes), so `st`
// waits until the sample is taken.
template <class K>
msort_status learned_prepare(msort_ctx* ctx, const Plan& pl, const K* keys, size_t n, cudaStream_t st,
                             bool keys_overwritten);
// Partition launch that starts each co-rank search from a prediction (the
// network's in mode 1, the length ratio in mode 2) and verifies it; exact
// binary search finishes inside the verified bracket.
template <class K>
cudaError_t launch_guided_partition(msort_ctx* ctx, const Plan& pl, const K* src, size_t n, size_t L,
                                    unsigned long long* splits, cudaStream_t st);
void learned_destroy(msort_ctx* ctx);
void graphs_destroy(msort_ctx* ctx);

// Plain keys-only sort with caller-provided scratch (used for the sample).
template <class K>
size_t sort_keys_scratch(size_t n);
template <class K>
msort_status sort_keys_internal(msort_ctx* ctx, const K* in, K* out, size_t n, void* scratch, cudaStream_t st);

// Any sort with caller-provided scratch (serving loop arena).
template <class K, bool PAIRS>
msort_status sort_with_scratch(msort_ctx* ctx, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                               void* scratch, cudaStream_t st);
size_t sort_scratch_need(size_t n, int key_bytes, bool pairs);

// Grid-barrier self-test of the single launch (msort.cu).
msort_status selftest_single_timeout(msort_ctx* ctx, void* d_keys, size_t n, long long limit_cycles,
                                     cudaStream_t st);

}  // namespace msort
