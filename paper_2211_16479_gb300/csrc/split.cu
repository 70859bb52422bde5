// Cuts of a sorted chunk at (key, global position) splitters: the partition
// step of the one-exchange multi-GPU form of the merge sort.
//
// The paper's message-passing sort (Section "MPI Merge Sort") scatters the
// array into one subarray per process, sorts each, and merges them up a tree
// (Figs. 16-17).  The one-exchange form sorts each rank's chunk, picks p - 1
// splitters from regular samples of all chunks, and sends every element to
// the rank whose key range holds it.  Ordering elements by (key, global input
// position) makes that order total, so a splitter cuts runs of equal keys at
// an exact place and rank r receives exactly the r-th slice of the stable
// sort.  This kernel computes, for each splitter, how many elements of the
// locally sorted chunk come before it: one binary search per splitter over
// the chunk (sorted by key, equal keys in increasing position because the
// local sort is stable and carries the local index).
#include <cuda_runtime.h>

#include "ctx.h"

namespace msort {
namespace {

template <class K>
__global__ void k_split_points(const K* __restrict__ keys, const uint32_t* __restrict__ idx, size_t n,
                               unsigned long long offset, const K* __restrict__ skeys,
                               const unsigned long long* __restrict__ spos, size_t ns,
                               unsigned long long* __restrict__ cuts) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns) return;
    const K sk = skeys[t];
    const unsigned long long sp = spos[t];
    size_t lo = 0, hi = n;  // first element not ordered before (sk, sp)
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        const K k = keys[mid];
        if (k < sk || (k == sk && offset + idx[mid] < sp))
            lo = mid + 1;
        else
            hi = mid;
    }
    cuts[t] = lo;
}

}  // namespace
}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_split_points(msort_ctx* ctx, const void* d_keys, const uint32_t* d_idx, size_t n,
                                uint64_t offset, const void* d_split_keys, const uint64_t* d_split_pos,
                                size_t nsplit, uint64_t* d_cuts, msort_key_type kt, void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    if (kt != MSORT_U32 && kt != MSORT_U64)
        return fail(MSORT_ERR_UNSUPPORTED, "msort_split_points takes unsigned keys (MSORT_U32 or MSORT_U64)");
    if (nsplit == 0) return MSORT_OK;
    if (!d_split_keys || !d_split_pos || !d_cuts) return fail(MSORT_ERR_INVALID_ARG, "splitter or cut pointer is NULL");
    if (n && (!d_keys || !d_idx)) return fail(MSORT_ERR_INVALID_ARG, "key or index pointer is NULL");
    if (n > 0xFFFFFFFFull) return fail(MSORT_ERR_INVALID_ARG, "a chunk holds at most 2^32 - 1 elements");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const unsigned th = 128;
    const unsigned blocks = (unsigned)((nsplit + th - 1) / th);
    cudaStream_t st = (cudaStream_t)stream;
    if (kt == MSORT_U32)
        k_split_points<uint32_t><<<blocks, th, 0, st>>>(
            static_cast<const uint32_t*>(d_keys), d_idx, n, offset, static_cast<const uint32_t*>(d_split_keys),
            reinterpret_cast<const unsigned long long*>(d_split_pos), nsplit,
            reinterpret_cast<unsigned long long*>(d_cuts));
    else
        k_split_points<uint64_t><<<blocks, th, 0, st>>>(
            static_cast<const uint64_t*>(d_keys), d_idx, n, offset, static_cast<const uint64_t*>(d_split_keys),
            reinterpret_cast<const unsigned long long*>(d_split_pos), nsplit,
            reinterpret_cast<unsigned long long*>(d_cuts));
    ++ctx->launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "split-point launch");
}

}  // extern "C"
