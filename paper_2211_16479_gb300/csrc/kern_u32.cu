// Sort kernels and launchers for 32-bit keys.
#include "launch_impl.cuh"

namespace msort {
MSORT_INSTANTIATE(uint32_t)
}
