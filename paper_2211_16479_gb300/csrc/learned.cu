// Learned-CDF partitioner: placeholder until the training kernels land.
#include "learned.h"

namespace msort {

int learned_first_pass(const Plan& pl, size_t) { return pl.passes; }

template <class K>
msort_status learned_prepare(msort_ctx*, const Plan&, const K*, size_t, cudaStream_t) {
    return fail(MSORT_ERR_UNSUPPORTED, "learned partitioning is not built yet");
}

template <class K>
cudaError_t launch_learned_partition(msort_ctx*, const Plan&, const K*, size_t, size_t, unsigned long long*,
                                     cudaStream_t) {
    return cudaErrorNotSupported;
}

template msort_status learned_prepare<uint32_t>(msort_ctx*, const Plan&, const uint32_t*, size_t, cudaStream_t);
template msort_status learned_prepare<uint64_t>(msort_ctx*, const Plan&, const uint64_t*, size_t, cudaStream_t);
template cudaError_t launch_learned_partition<uint32_t>(msort_ctx*, const Plan&, const uint32_t*, size_t, size_t,
                                                        unsigned long long*, cudaStream_t);
template cudaError_t launch_learned_partition<uint64_t>(msort_ctx*, const Plan&, const uint64_t*, size_t, size_t,
                                                        unsigned long long*, cudaStream_t);

void learned_destroy(msort_ctx*) {}


}  // namespace msort
