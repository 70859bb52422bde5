// Launcher definitions (included once per key type).
#pragma once

#include <cstdio>

#include "launch.h"
#include "merge4.cuh"
#include "merge_runs.cuh"
#include "small.cuh"
#include "sort_kernels.cuh"

namespace msort {

std::string& launch_info_ref();

template <class F>
static cudaError_t prepare(F* f, size_t smem) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(f));
    char buf[200];
    std::snprintf(buf, sizeof buf, " [regs %d, max threads %d, dyn smem %zu, max dyn %d]", fa.numRegs,
                  fa.maxThreadsPerBlock, smem, fa.maxDynamicSharedSizeBytes);
    launch_info_ref() = buf;
    if (e != cudaSuccess) return e;
    if ((int)smem <= fa.maxDynamicSharedSizeBytes) return cudaSuccess;
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

static inline int tile_threads(int tile) {
    return tile == 33792 ? 1024 : (tile == 8704 || tile == 16896) ? 512 : 256;
}

template <class K, bool PAIRS>
size_t tile_smem_bytes(int tile) {
    switch (tile_threads(tile)) {
        case 1024: return tile_block_smem<K, PAIRS, 1024>(tile);
        case 512: return tile_block_smem<K, PAIRS, 512>(tile);
        default: return tile_block_smem<K, PAIRS, 256>(tile);
    }
}

// ipt = outputs per thread of the merge block (W = 256 * ipt).
template <class K, bool PAIRS>
size_t merge_smem_bytes(int W) {
    const int ipt = W / 256;
    return sizeof(K) * merge_slots(W, ipt, sizeof(K)) + (PAIRS ? 4 * merge_slots(W, ipt, 4) : 0);
}

template <class K, bool PAIRS>
bool tile_supported(int tile) {
    if (tile != 4352 && tile != 8448 && tile != 8704 && tile != 16896 && tile != 33792) return false;
    if (tile == 33792 && (PAIRS || sizeof(K) != 4)) return false;  // 32-bit keys alone
    return tile_smem_bytes<K, PAIRS>(tile) <= 227 * 1024;
}

// tile = threads * keys per thread (odd); merge blocks use 256 threads with
// the same keys per thread, so W divides 2 * tile.
#define MSORT_TILE_CFG(X) X(4352, 256, 17) X(8448, 256, 33) X(8704, 512, 17) X(16896, 512, 33) X(33792, 1024, 33)

template <class K, bool PAIRS>
cudaError_t launch_tile(const Plan& pl, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                        cudaStream_t st, int xf_in, int xf_out) {
    const size_t nblocks = (n + pl.tile - 1) / pl.tile;
    const size_t sm = tile_smem_bytes<K, PAIRS>(pl.tile);
    if (!tile_supported<K, PAIRS>(pl.tile)) return cudaErrorInvalidConfiguration;
    cudaError_t e;
#define MSORT_TILE_CASE(TILE, TH, IPT)                                         \
    if (pl.tile == TILE) {                                                     \
        auto f = (xf_in || xf_out) ? k_tile_sort<K, PAIRS, TH, IPT, true> : k_tile_sort<K, PAIRS, TH, IPT, false>; \
        if ((e = prepare(f, sm)) != cudaSuccess) return e;                     \
        f<<<(unsigned)nblocks, TH, sm, st>>>(kin, vin, kout, vout, n, pl.status, xf_in, xf_out); \
        return cudaGetLastError();                                             \
    }
    MSORT_TILE_CFG(MSORT_TILE_CASE)
#undef MSORT_TILE_CASE
    return cudaErrorInvalidConfiguration;
}

template <class K, bool PAIRS>
cudaError_t launch_merge(const Plan& pl, const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst, size_t n,
                         size_t L, const unsigned long long* splits, cudaStream_t st, size_t c0, size_t c1,
                         int xf_out) {
    const size_t nblocks = (n + pl.W - 1) / pl.W;
    if (c1 > nblocks) c1 = nblocks;
    if (c0 >= c1) return cudaSuccess;
    const size_t sm = merge_smem_bytes<K, PAIRS>(pl.W);
    cudaError_t e;
#define MSORT_MERGE_CASE(WW, TH, IPT)                                          \
    if (pl.W == WW) {                                                          \
        auto f = xf_out ? k_merge_pass<K, PAIRS, TH, IPT, true> : k_merge_pass<K, PAIRS, TH, IPT, false>; \
        if ((e = prepare(f, sm)) != cudaSuccess) return e;                     \
        f<<<(unsigned)(c1 - c0), TH, sm, st>>>(src, dst, vsrc, vdst, n, L, splits, pl.status, c0, xf_out); \
        return cudaGetLastError();                                             \
    }
    MSORT_MERGE_CASE(4352, 256, 17)
    MSORT_MERGE_CASE(8448, 256, 33)
#undef MSORT_MERGE_CASE
    return cudaErrorInvalidConfiguration;
}

template <class K>
cudaError_t launch_partition(const Plan& pl, const K* src, size_t n, size_t L, unsigned long long* splits,
                             cudaStream_t st) {
    const size_t nblocks = (n + pl.W - 1) / pl.W;
    const unsigned th = 128;
    k_partition<K><<<(unsigned)((nblocks + th - 1) / th), th, 0, st>>>(src, n, L, (size_t)pl.W, nblocks, splits);
    return cudaGetLastError();
}

// Four-way merge blocks of 256 threads: 11 outputs per thread (W = 2816,
// which divides 4 x every tile of 33 keys per thread) or 17 (W = 4352, for
// tiles of 17 keys per thread); grid step an eighth of the block.
#define MSORT_MERGE4_CFG(X) X(2816, 256, 11) X(4352, 256, 17)

template <class K>
size_t merge4_smem_bytes(int W4) {
#define MSORT_M4_SMEM(WW, TH, IPT) \
    if (W4 == WW) return merge4_smem<K, TH, IPT, 8>();
    MSORT_MERGE4_CFG(MSORT_M4_SMEM)
#undef MSORT_M4_SMEM
    return 0;
}

template <class K>
cudaError_t launch_merge4_partition(const Plan& pl, const K* src, size_t n, size_t L, unsigned long long* gco,
                                    K* gval, unsigned long long* gpos, unsigned long long* brk, cudaStream_t st) {
    const size_t G = (size_t)pl.G4;
    const size_t total = merge4_grid_points(n, L, G);
    const size_t nblocks = (n + pl.W4 - 1) / pl.W4;
    const unsigned th = 128;
    const unsigned gb = (unsigned)((total + th - 1) / th);
    k_grid4<K><<<gb, th, 0, st>>>(src, n, L, G, total, gco, gval);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pos4<K><<<gb, th, 0, st>>>(src, n, L, G, total, gco, gval, gpos);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bracket4<K><<<(unsigned)((2 * nblocks + th - 1) / th), th, 0, st>>>(n, L, G, (size_t)pl.W4, nblocks, gpos,
                                                                          gco, brk);
    return cudaGetLastError();
}

template <class K>
cudaError_t launch_merge4(const Plan& pl, const K* src, K* dst, size_t n, size_t L, const unsigned long long* brk,
                          cudaStream_t st) {
    const size_t nblocks = (n + pl.W4 - 1) / pl.W4;
    cudaError_t e;
#define MSORT_M4_CASE(WW, TH, IPT)                                             \
    if (pl.W4 == WW) {                                                         \
        auto f = k_merge4_pass<K, TH, IPT, 8>;                                 \
        const size_t sm = merge4_smem<K, TH, IPT, 8>();                        \
        if ((e = prepare(f, sm)) != cudaSuccess) return e;                     \
        f<<<(unsigned)nblocks, TH, sm, st>>>(src, dst, n, L, brk, pl.status);      \
        return cudaGetLastError();                                             \
    }
    MSORT_MERGE4_CFG(MSORT_M4_CASE)
#undef MSORT_M4_CASE
    return cudaErrorInvalidConfiguration;
}

// Merge blocks of 256 threads x 33 keys for 32-bit keys-only merges, 256 x 17
// otherwise (register pressure).
template <class K, bool PAIRS>
size_t merge_two_block() {
    return (sizeof(K) == 4 && !PAIRS) ? 256 * 33 : 256 * 17;
}

template <class K, bool PAIRS>
cudaError_t launch_merge_two(const K* A, size_t na, const K* B, size_t nb, const uint32_t* va, const uint32_t* vb,
                             K* out, uint32_t* vout, unsigned long long* splits, unsigned int* status,
                             cudaStream_t st) {
    const size_t W = merge_two_block<K, PAIRS>();
    const size_t total = na + nb;
    if (total == 0) return cudaSuccess;
    const size_t nblocks = (total + W - 1) / W;
    k_partition_two<K><<<(unsigned)((nblocks + 127) / 128), 128, 0, st>>>(A, na, B, nb, W, nblocks, splits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (W == 256 * 33) {
        auto f = k_merge_two<K, PAIRS, 256, 33>;
        const size_t sm = merge_block_smem<K, PAIRS, 256, 33>();
        if ((e = prepare(f, sm)) != cudaSuccess) return e;
        f<<<(unsigned)nblocks, 256, sm, st>>>(A, na, B, nb, va, vb, out, vout, splits, status);
    } else {
        auto f = k_merge_two<K, PAIRS, 256, 17>;
        const size_t sm = merge_block_smem<K, PAIRS, 256, 17>();
        if ((e = prepare(f, sm)) != cudaSuccess) return e;
        f<<<(unsigned)nblocks, 256, sm, st>>>(A, na, B, nb, va, vb, out, vout, splits, status);
    }
    return cudaGetLastError();
}

template <class K, bool PAIRS>
cudaError_t launch_merge_runs(const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst, const RunPairs& rp,
                              unsigned long long* splits, unsigned int* status, int xf_out, cudaStream_t st) {
    const size_t W = merge_two_block<K, PAIRS>();
    const unsigned long long nblocks = rp.c[rp.np];
    if (nblocks == 0) return cudaSuccess;
    k_partition_runs<K><<<(unsigned)((nblocks + 127) / 128), 128, 0, st>>>(src, rp, W, splits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (W == 256 * 33) {
        auto f = xf_out ? k_merge_runs<K, PAIRS, 256, 33, true> : k_merge_runs<K, PAIRS, 256, 33, false>;
        const size_t sm = merge_block_smem<K, PAIRS, 256, 33>();
        if ((e = prepare(f, sm)) != cudaSuccess) return e;
        f<<<(unsigned)nblocks, 256, sm, st>>>(src, dst, vsrc, vdst, rp, splits, status, xf_out);
    } else {
        auto f = xf_out ? k_merge_runs<K, PAIRS, 256, 17, true> : k_merge_runs<K, PAIRS, 256, 17, false>;
        const size_t sm = merge_block_smem<K, PAIRS, 256, 17>();
        if ((e = prepare(f, sm)) != cudaSuccess) return e;
        f<<<(unsigned)nblocks, 256, sm, st>>>(src, dst, vsrc, vdst, rp, splits, status, xf_out);
    }
    return cudaGetLastError();
}

// Single-launch shapes (threads x keys per thread; tile = merge block).
// 32-bit keys alone: 256 x 11, 256 x 17, 256 x 33, 512 x 11, 512 x 17,
// 512 x 33 or 1024 x 11; other key/value types: 256 x 11 and 256 x 33
// (256 x 17 for 64-bit key-value pairs, whose 33-key blocks need too many
// registers).  Small blocks keep each thread's serial merge short and spread
// a small array over many SMs, which is what bounds a sort whose data stays
// in L2.  Measured on GB300 (uniform 32-bit keys, graph replay): 256 x 17
// is fastest up to 2^19 keys, 512 x 17 at 2^20 (59.5 us against 63.6 and
// 61.4 for 256 x 17 and 256 x 33), 512 x 33 above; other types take
// 256 x 11 up to 2^18 keys and their larger block above.
template <class K, bool PAIRS>
int small_tile(size_t n) {
    if constexpr (!PAIRS && sizeof(K) == 4) {
        if (n <= (size_t(1) << 19)) return 256 * 17;
        return n <= (size_t(1) << 20) ? 512 * 17 : 512 * 33;
    }
    if (n <= (size_t(1) << 18)) return 256 * 11;
    return (PAIRS && sizeof(K) == 8) ? 256 * 17 : 256 * 33;
}

template <class K, bool PAIRS>
bool small_tile_supported(int tile) {
    if (!PAIRS && sizeof(K) == 4)
        return tile == 256 * 11 || tile == 256 * 17 || tile == 256 * 33 || tile == 512 * 11 || tile == 512 * 17 ||
               tile == 512 * 33 || tile == 1024 * 11;
    if (PAIRS && sizeof(K) == 8) return tile == 256 * 11 || tile == 256 * 17;
    return tile == 256 * 11 || tile == 256 * 33;
}

template <class K, bool PAIRS, int TH, int IPT>
static cudaError_t launch_small_shape(const Plan& pl, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
                                      K* tk, uint32_t* tv, size_t n, void* barrier, cudaStream_t st, int xf_in,
                                      int xf_out, long long wait_limit, unsigned int extra_arrivals) {
    auto f = (xf_in || xf_out) ? k_small_sort<K, PAIRS, TH, IPT, true> : k_small_sort<K, PAIRS, TH, IPT, false>;
    const size_t sm = small_sort_smem<K, PAIRS, TH, IPT>();
    cudaError_t e = prepare(f, sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0, coop = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, TH, sm)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const size_t tiles = (n + (size_t)TH * IPT - 1) / ((size_t)TH * IPT);
    const size_t cap = (size_t)sms * (size_t)per;  // blocks that can all be resident at once
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    if ((e = cudaMemsetAsync(barrier, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TH);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, kin, vin, kout, vout, tk, tv, n, pl.passes,
                              static_cast<GridBarrier*>(barrier), pl.status, xf_in, xf_out, wait_limit,
                              extra_arrivals);
}

template <class K, bool PAIRS>
cudaError_t launch_small(const Plan& pl, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, K* tk,
                         uint32_t* tv, size_t n, void* barrier, cudaStream_t st, int xf_in, int xf_out,
                         long long wait_limit, unsigned int extra_arrivals) {
#define MSORT_SMALL_CASE(TH, IPT)                                                                            \
    if (pl.tile == TH * IPT)                                                                                \
        return launch_small_shape<K, PAIRS, TH, IPT>(pl, kin, vin, kout, vout, tk, tv, n, barrier, st, xf_in, \
                                                     xf_out, wait_limit, extra_arrivals);
    MSORT_SMALL_CASE(256, 11)
    if constexpr (!PAIRS && sizeof(K) == 4) {
        MSORT_SMALL_CASE(256, 17)
        MSORT_SMALL_CASE(256, 33)
        MSORT_SMALL_CASE(512, 11)
        MSORT_SMALL_CASE(512, 17)
        MSORT_SMALL_CASE(512, 33)
        MSORT_SMALL_CASE(1024, 11)
    } else if constexpr (PAIRS && sizeof(K) == 8) {
        MSORT_SMALL_CASE(256, 17)
    } else {
        MSORT_SMALL_CASE(256, 33)
    }
#undef MSORT_SMALL_CASE
    return cudaErrorInvalidConfiguration;
}

#define MSORT_INSTANTIATE(K)                                                                                    \
    template size_t tile_smem_bytes<K, false>(int);                                                             \
    template size_t tile_smem_bytes<K, true>(int);                                                              \
    template size_t merge_smem_bytes<K, false>(int);                                                            \
    template size_t merge_smem_bytes<K, true>(int);                                                             \
    template bool tile_supported<K, false>(int);                                                                \
    template bool tile_supported<K, true>(int);                                                                 \
    template cudaError_t launch_tile<K, false>(const Plan&, const K*, const uint32_t*, K*, uint32_t*, size_t,   \
                                               cudaStream_t, int, int);                                         \
    template cudaError_t launch_tile<K, true>(const Plan&, const K*, const uint32_t*, K*, uint32_t*, size_t,    \
                                              cudaStream_t, int, int);                                          \
    template cudaError_t launch_merge<K, false>(const Plan&, const K*, K*, const uint32_t*, uint32_t*, size_t,  \
                                                size_t, const unsigned long long*, cudaStream_t, size_t, size_t, \
                                                int);                                                           \
    template cudaError_t launch_merge<K, true>(const Plan&, const K*, K*, const uint32_t*, uint32_t*, size_t,   \
                                               size_t, const unsigned long long*, cudaStream_t, size_t, size_t, \
                                               int);                                                            \
    template cudaError_t launch_partition<K>(const Plan&, const K*, size_t, size_t, unsigned long long*,        \
                                             cudaStream_t);                                                     \
    template size_t merge4_smem_bytes<K>(int);                                                                  \
    template cudaError_t launch_merge4_partition<K>(const Plan&, const K*, size_t, size_t, unsigned long long*, \
                                                    K*, unsigned long long*, unsigned long long*, cudaStream_t); \
    template cudaError_t launch_merge4<K>(const Plan&, const K*, K*, size_t, size_t, const unsigned long long*, \
                                          cudaStream_t);                                                        \
    template size_t merge_two_block<K, false>();                                                                \
    template size_t merge_two_block<K, true>();                                                                 \
    template cudaError_t launch_merge_two<K, false>(const K*, size_t, const K*, size_t, const uint32_t*,         \
                                                    const uint32_t*, K*, uint32_t*, unsigned long long*,        \
                                                    unsigned int*, cudaStream_t);                               \
    template cudaError_t launch_merge_two<K, true>(const K*, size_t, const K*, size_t, const uint32_t*,          \
                                                   const uint32_t*, K*, uint32_t*, unsigned long long*,         \
                                                   unsigned int*, cudaStream_t);                                \
    template cudaError_t launch_merge_runs<K, false>(const K*, K*, const uint32_t*, uint32_t*, const RunPairs&,  \
                                                     unsigned long long*, unsigned int*, int, cudaStream_t);     \
    template cudaError_t launch_merge_runs<K, true>(const K*, K*, const uint32_t*, uint32_t*, const RunPairs&,   \
                                                    unsigned long long*, unsigned int*, int, cudaStream_t);      \
    template int small_tile<K, false>(size_t);                                                                  \
    template int small_tile<K, true>(size_t);                                                                   \
    template bool small_tile_supported<K, false>(int);                                                          \
    template bool small_tile_supported<K, true>(int);                                                           \
    template cudaError_t launch_small<K, false>(const Plan&, const K*, const uint32_t*, K*, uint32_t*, K*,        \
                                                uint32_t*, size_t, void*, cudaStream_t, int, int, long long,     \
                                                unsigned int);                                                   \
    template cudaError_t launch_small<K, true>(const Plan&, const K*, const uint32_t*, K*, uint32_t*, K*,         \
                                               uint32_t*, size_t, void*, cudaStream_t, int, int, long long,      \
                                               unsigned int);

}  // namespace msort
