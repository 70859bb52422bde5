// Sort kernels and launchers for 64-bit keys.
#include "launch_impl.cuh"

namespace msort {
MSORT_INSTANTIATE(uint64_t)
}
