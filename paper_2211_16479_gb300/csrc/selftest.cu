// Self-test of the failure path of the bounded device waits.
//
// Every wait in the sort's kernels (a block waiting on its mbarrier for its
// bulk copies) gives up after a cycle limit, records kStatusTimeout in the
// context's status word, waits once more (bounded) for copies of its own
// still in flight and returns; msort_ctx_sync then reports MSORT_ERR_TIMEOUT.
// This file launches the production merge block on a barrier that expects
// one arrival more than the block makes, with a short limit, so that this
// path runs without any fault, trap or unbounded wait: the block's windows
// are too short for a bulk copy (no copy is ever in flight) and its output
// is never written.  A second self-test does the same to the grid barrier
// of the single-launch sort (msort.cu, selftest_single_timeout).
#include <cuda_runtime.h>

#include "ctx.h"
#include "launch.h"
#include "learned.h"
#include "sort_kernels.cuh"

namespace msort {
namespace {

// Two runs of three keys each (zero-initialised; their values do not matter).
__device__ __align__(16) uint32_t g_selftest_keys[16];
__device__ __align__(16) uint32_t g_selftest_out[16];

constexpr int kSelftestThreads = 256;
constexpr int kSelftestIpt = 33;

__global__ void __launch_bounds__(kSelftestThreads) k_selftest_wait(unsigned int* status, long long limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);  // merge_block arrives once; the phase never completes
        fence_mbar_init();
    }
    uint32_t phase = 0;
    merge_block<uint32_t, false, kSelftestThreads, kSelftestIpt, false>(
        g_selftest_keys, 3, g_selftest_keys + 8, 3, nullptr, nullptr, g_selftest_out, nullptr, smem_raw, &bar, phase,
        status, 0, limit);
}

}  // namespace
}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_selftest_wait_timeout(msort_ctx* ctx, long long limit_cycles, void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    if (limit_cycles < 1000 || limit_cycles > kWaitLimitCycles)
        return fail(MSORT_ERR_INVALID_ARG, "limit_cycles must be in [1000, 2e9]");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const size_t sm = merge_block_smem<uint32_t, false, kSelftestThreads, kSelftestIpt>();
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_selftest_wait),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_fail(e, "self-test kernel attributes");
    k_selftest_wait<<<1, kSelftestThreads, sm, (cudaStream_t)stream>>>(ctx->d_status, limit_cycles);
    ++ctx->launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "self-test launch");
}

msort_status msort_selftest_grid_timeout(msort_ctx* ctx, void* d_keys, size_t n, long long limit_cycles,
                                         void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    if (!d_keys) return fail(MSORT_ERR_INVALID_ARG, "d_keys is NULL");
    if (limit_cycles < 1000 || limit_cycles > kWaitLimitCycles)
        return fail(MSORT_ERR_INVALID_ARG, "limit_cycles must be in [1000, 2e9]");
    return selftest_single_timeout(ctx, d_keys, n, limit_cycles, (cudaStream_t)stream);
}

}  // extern "C"
