// msort_sort_noalloc: the stable merge sort without any device allocation.
//
// Some callers cannot call cudaMalloc: a framework that hands out all device
// memory from its own pool and forbids allocations behind its back, a
// service that must never take the implicit device synchronisation a first
// cudaMalloc or a scratch growth can cause, or code that runs where the CUDA
// allocator must not be entered at all.  For them this entry point sorts
// with a scratch area that is part of the library image: a fixed array in
// device global memory that every GPU which loads the library holds until
// the process exits.  The caller supplies only its inputs and outputs.
//
// The scratch is shared by every call on a device and keeps whatever the
// last call left in it; the status word that kernels may set is cleared at
// the start of each call (msort_noalloc_sync reads it afterwards), the rest
// is fully rewritten before it is read.  Calls whose work overlaps on the GPU
// (different streams without ordering, or several host threads) race on the
// scratch and give wrong results: order them on one stream or serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>

#include "ctx.h"
#include "launch.h"

// The scratch area: 48 MiB per device, enough for a 32-bit keys-only sort of
// up to about 12.5 million keys (fewer for 64-bit keys or key-value sorts; the
// exact limit is msort_noalloc_max_keys()).
static constexpr size_t kNoAllocScratchBytes = size_t(48) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace msort {
namespace {

constexpr int kNoAllocTile = 8448;  // 256 threads x 33 keys; valid for every key/value type
std::mutex g_mu;

// Driver calls that identify the calling thread's current CUDA context,
// reached through the runtime (the library does not link libcuda itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
// Scratch address per CUDA context id.  The array's address belongs to the
// context that loaded the library's module: after a device reset, or under
// another context, the runtime loads the module again at a new address, so
// the cache is keyed by the context's unique id, not by the device index.
std::map<unsigned long long, unsigned char*> g_scratch_addr;

msort_status driver_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return MSORT_OK;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void *f1 = nullptr, *f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDriverEntryPointByVersion");
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return fail(MSORT_ERR_UNSUPPORTED, "the CUDA driver lacks cuCtxGetCurrent / cuCtxGetId");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    return MSORT_OK;
}

// Device address of the scratch array in the calling thread's current
// context, looked up once per context (the first call under a context does
// it; cudaGetSymbolAddress allocates nothing).  With no context current yet,
// the lookup itself makes the current device's primary context current.
msort_status scratch_on_current_device(unsigned char** out) {
    std::lock_guard<std::mutex> g(g_mu);
    msort_status s = driver_entry_points();
    if (s != MSORT_OK) return s;
    CUcontext cu = nullptr;
    if (g_ctx_get_current(&cu) != CUDA_SUCCESS) return fail(MSORT_ERR_CUDA, "cuCtxGetCurrent failed");
    void* fresh = nullptr;
    if (!cu) {
        cudaError_t e = cudaGetSymbolAddress(&fresh, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
        if (g_ctx_get_current(&cu) != CUDA_SUCCESS || !cu) return fail(MSORT_ERR_CUDA, "no current CUDA context");
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(cu, &id) != CUDA_SUCCESS) return fail(MSORT_ERR_CUDA, "cuCtxGetId failed");
    auto it = g_scratch_addr.find(id);
    if (it == g_scratch_addr.end()) {
        if (!fresh) {
            cudaError_t e = cudaGetSymbolAddress(&fresh, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
        }
        it = g_scratch_addr.emplace(id, static_cast<unsigned char*>(fresh)).first;
    }
    *out = it->second;
    return MSORT_OK;
}

struct NoAllocLayout {
    size_t status, splits, keys, vals, end;
};

template <class K, bool PAIRS>
NoAllocLayout layout_for(size_t n, size_t W) {
    NoAllocLayout l{};
    l.status = 0;
    l.splits = 256;
    l.keys = l.splits + align_up(((n + W - 1) / W + 1) * sizeof(unsigned long long), 256);
    l.vals = l.keys + align_up(n * sizeof(K), 256);
    l.end = l.vals + (PAIRS ? align_up(n * sizeof(uint32_t), 256) : 0);
    return l;
}

template <class K, bool PAIRS>
size_t max_keys() {
    size_t lo = 0, hi = kNoAllocScratchBytes;
    while (lo < hi) {  // largest n whose layout fits
        const size_t mid = (lo + hi + 1) / 2;
        if (layout_for<K, PAIRS>(mid, kNoAllocTile).end <= kNoAllocScratchBytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <class K, bool PAIRS>
msort_status noalloc_sort(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, cudaStream_t st) {
    const NoAllocLayout l = layout_for<K, PAIRS>(n, kNoAllocTile);
    if (l.end > kNoAllocScratchBytes)
        return fail(MSORT_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                               std::to_string(max_keys<K, PAIRS>()) +
                                               " elements for this key/value type");
    unsigned char* base = nullptr;
    msort_status s = scratch_on_current_device(&base);
    if (s != MSORT_OK) return s;

    Plan pl{};
    pl.tile = kNoAllocTile;
    pl.W = kNoAllocTile;
    pl.passes = 0;
    for (size_t L = (size_t)pl.tile; L < n; L *= 2) ++pl.passes;
    pl.status = reinterpret_cast<unsigned int*>(base + l.status);
    unsigned long long* splits = reinterpret_cast<unsigned long long*>(base + l.splits);
    K* tk = reinterpret_cast<K*>(base + l.keys);
    uint32_t* tv = PAIRS ? reinterpret_cast<uint32_t*>(base + l.vals) : nullptr;

    cudaError_t e = cudaMemsetAsync(pl.status, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the no-allocation status word");

    K* bk[2] = {kout, tk};
    uint32_t* bv[2] = {vout, tv};
    int cur = (pl.passes & 1) ? 1 : 0;
    e = launch_tile<K, PAIRS>(pl, kin, vin, bk[cur], bv[cur], n, st);
    if (e != cudaSuccess) return cuda_fail(e, "tile sort launch");
    for (int p = 0; p < pl.passes; ++p) {
        const size_t L = (size_t)pl.tile << p;
        e = launch_partition<K>(pl, bk[cur], n, L, splits, st);
        if (e != cudaSuccess) return cuda_fail(e, "partition launch");
        e = launch_merge<K, PAIRS>(pl, bk[cur], bk[cur ^ 1], bv[cur], bv[cur ^ 1], n, L, splits, st);
        if (e != cudaSuccess) return cuda_fail(e, "merge pass launch");
        cur ^= 1;
    }
    return MSORT_OK;
}

}  // namespace
}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_sort_noalloc(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out,
                                uint32_t* d_vals_out, size_t n, msort_key_type kt, void* stream) {
    if (kt == MSORT_I32 || kt == MSORT_I64 || kt == MSORT_F32 || kt == MSORT_F64)
        return fail(MSORT_ERR_UNSUPPORTED, "msort_sort_noalloc takes unsigned keys (signed and floating-point keys: the plain "
                                           "and host-buffer sorts)");
    if (kt != MSORT_U32 && kt != MSORT_U64) return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
    if (n == 0) return MSORT_OK;
    if (!d_keys_in || !d_keys_out) return fail(MSORT_ERR_INVALID_ARG, "key pointer is NULL");
    if ((d_vals_in == nullptr) != (d_vals_out == nullptr))
        return fail(MSORT_ERR_INVALID_ARG, "give both value pointers or none");
    const size_t ks = kt == MSORT_U32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(d_keys_in) | reinterpret_cast<uintptr_t>(d_keys_out)) % ks ||
        (d_vals_in && ((reinterpret_cast<uintptr_t>(d_vals_in) | reinterpret_cast<uintptr_t>(d_vals_out)) & 3)))
        return fail(MSORT_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    cudaStream_t st = (cudaStream_t)stream;
    if (kt == MSORT_U32)
        return d_vals_in ? noalloc_sort<uint32_t, true>(static_cast<const uint32_t*>(d_keys_in), d_vals_in,
                                                        static_cast<uint32_t*>(d_keys_out), d_vals_out, n, st)
                         : noalloc_sort<uint32_t, false>(static_cast<const uint32_t*>(d_keys_in), nullptr,
                                                         static_cast<uint32_t*>(d_keys_out), nullptr, n, st);
    return d_vals_in ? noalloc_sort<uint64_t, true>(static_cast<const uint64_t*>(d_keys_in), d_vals_in,
                                                    static_cast<uint64_t*>(d_keys_out), d_vals_out, n, st)
                     : noalloc_sort<uint64_t, false>(static_cast<const uint64_t*>(d_keys_in), nullptr,
                                                     static_cast<uint64_t*>(d_keys_out), nullptr, n, st);
}

msort_status msort_noalloc_sync(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned char* base = nullptr;
    msort_status s = scratch_on_current_device(&base);
    if (s != MSORT_OK) return s;
    unsigned int st = 0;
    e = cudaMemcpy(&st, base, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation status read");
    if (!st) return MSORT_OK;
    e = cudaMemset(base, 0, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation status clear");
    if (st & DEV_TIMEOUT) return fail(MSORT_ERR_TIMEOUT, "a kernel of msort_sort_noalloc gave up a bounded wait");
    return fail(MSORT_ERR_CUDA, "a kernel of msort_sort_noalloc recorded status " + std::to_string(st));
}

size_t msort_noalloc_max_keys(msort_key_type kt, int with_vals) {
    if (kt == MSORT_U32) return with_vals ? max_keys<uint32_t, true>() : max_keys<uint32_t, false>();
    if (kt == MSORT_U64) return with_vals ? max_keys<uint64_t, true>() : max_keys<uint64_t, false>();
    return 0;
}

}  // extern "C"
