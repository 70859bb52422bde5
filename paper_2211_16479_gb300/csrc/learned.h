// Learned-CDF partitioner (declarations shared with the pass scheduler).
#pragma once

#include <cuda_runtime.h>

#include "ctx.h"

namespace msort {

// First merge pass (0-based) whose partition uses the learned predictor.
int learned_first_pass(const Plan& pl, size_t n);
// Draw the key sample from the unsorted input, sort it and train the network
// on the device, all enqueued on st before the sort's tile pass.
template <class K>
msort_status learned_prepare(msort_ctx* ctx, const Plan& pl, const K* keys, size_t n, cudaStream_t st);
// Partition launch that starts each co-rank search from the network's
// prediction and verifies it (exact search remains the fallback).
template <class K>
cudaError_t launch_learned_partition(msort_ctx* ctx, const Plan& pl, const K* src, size_t n, size_t L,
                                     unsigned long long* splits, cudaStream_t st);
void learned_destroy(msort_ctx* ctx);
void graphs_destroy(msort_ctx* ctx);

}  // namespace msort
