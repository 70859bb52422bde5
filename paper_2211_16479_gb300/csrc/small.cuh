// Single-launch sort for arrays that stay in L2.
//
// The method is unchanged (Section "Multiprocessing Merge Sort": sort fixed
// chunks, then Section "MPI Merge Sort", Figs. 16-17: merge runs pairwise,
// round after round), but for a few million keys every kernel of the
// multi-launch plan finishes in microseconds and the launches themselves,
// one tile sort plus a partition and a merge launch per round, dominate.
// Here one cooperative launch runs everything: the blocks sort the tiles,
// then run every merge round, with a grid barrier after the tile sort and
// after each round.  Each merge block finds the co-ranks of its first and
// last output itself, by a 32-way warp search over the (L2-resident) runs,
// so there is no partition step.
//
// Grid barrier: one arrival counter in global memory (zeroed before the
// launch) that only grows: barrier k of the launch is passed once it reaches
// k * gridDim.x.  Thread 0 of a block completes the block's bulk stores,
// fences its writes (async and generic proxy) at GPU scope, adds 1, and
// polls the counter with acquire loads under a cycle limit, after which it
// records kStatusTimeout and the block leaves the kernel (every other block
// then gives up at its own next barrier, each bounded), so a missing block
// can never hang the GPU.  The launch is cooperative, which guarantees that
// all blocks are resident at once.
#pragma once

#include "sort_kernels.cuh"

namespace msort {

struct GridBarrier {
    unsigned int count;  // arrivals since the launch
    unsigned int unused;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks of the grid reach this point before any leaves it; writes
// before it (plain or bulk-TMA) are visible after it to reads of either
// kind.  `target` = (number of this barrier in the launch) * gridDim.x.
// Returns false after a timeout (every thread of the block gets false and
// the block must return).
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned int target, unsigned int* status,
                                          long long limit) {
    __shared__ int ok;
    if (threadIdx.x == 0) tma_store_wait_all();  // the block's bulk stores (issued by thread 0) are complete
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_proxy_async_global();
        __threadfence();  // release: this block's writes, ordered before the arrival
        atomicAdd(&gb->count, 1u);
        int good = 1;
        if (ld_acquire_gpu(&gb->count) < target) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&gb->count) < target) {
                if (clock64() - t0 > limit) {
                    atomicOr(status, kStatusTimeout);
                    good = 0;
                    break;
                }
            }
        }
        fence_proxy_async_global();  // the block's later bulk loads see what the acquire made visible
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Stable co-rank (the first a in [max(0, d-|B|), min(d, |A|)] with
// B[d-1-a] < A[a]) by a 32-way search: the 32 lanes of the calling warp
// test 32 positions of the current bracket at once, and the bracket shrinks
// to the gap where the test turns true (a factor of about 33 per step;
// bracket of at most 32 positions: one last step).  Every lane of the warp
// must call it with the same arguments; every lane gets the result.
template <class K>
__device__ __forceinline__ size_t corank_warp(const K* A, size_t alen, const K* B, size_t blen, size_t d, int lane) {
    size_t lo = d > blen ? d - blen : 0;
    size_t hi = d < alen ? d : alen;  // the split is in [lo, hi]; the test holds at hi by definition
    while (lo < hi) {
        const size_t span = hi - lo;
        const bool wide = span > 32;
        const size_t p = wide ? lo + (span * (size_t)(lane + 1)) / 33 : lo + (size_t)lane;
        const bool t = p >= hi || A[p] > B[d - 1 - p];
        const unsigned int m = __ballot_sync(0xffffffffu, t);
        if (!wide) {
            lo = m ? lo + (size_t)(__ffs(m) - 1) : hi;  // no lane true: the split is hi
            break;
        }
        const size_t p31 = __shfl_sync(0xffffffffu, p, 31);
        if (m == 0) {
            lo = p31 + 1;
        } else {
            const int f = __ffs(m) - 1;
            const size_t pf = __shfl_sync(0xffffffffu, p, f);
            const size_t pb = __shfl_sync(0xffffffffu, p, f > 0 ? f - 1 : 0);
            hi = pf;
            if (f > 0) lo = pb + 1;
        }
    }
    return lo;
}

// The whole sort in one cooperative launch: tiles of T = THREADS * IPT keys,
// merge rounds with output blocks of W = T, ping-pong between (kout, vout)
// and (tk, tv) starting where the last round lands in kout.  XF: the tile
// sort applies xf_in and the last round (or, with no round, the tile sort)
// undoes xf_out.  wait_limit bounds every grid-barrier wait (production:
// kWaitLimitCycles).
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS)
k_small_sort(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, K* tk, uint32_t* tv, size_t n, int passes,
             GridBarrier* gb, unsigned int* status, int xf_in, int xf_out, long long wait_limit,
             unsigned int extra_arrivals) {
    constexpr int T = THREADS * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long split[2];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    uint32_t phase = 0;
    const unsigned int G = gridDim.x;
    K* bk[2] = {kout, tk};
    uint32_t* bv[2] = {vout, tv};
    int cur = (passes & 1) ? 1 : 0;
    const size_t nblocks = (n + T - 1) / T;

    for (size_t b = blockIdx.x; b < nblocks; b += G) {
        const size_t base = b * T;
        const int valid = (int)((n - base) < (size_t)T ? (n - base) : (size_t)T);
        if (!tile_sort_block<K, PAIRS, THREADS, IPT, XF>(kin + base, PAIRS ? vin + base : nullptr, bk[cur] + base,
                                                         PAIRS ? bv[cur] + base : nullptr, valid, smem_raw, &bar,
                                                         phase, status, xf_in, passes == 0 ? xf_out : 0))
            return;
    }
    // arrivals that end the current barrier (extra_arrivals is 0 except in the
    // self-test, where the first barrier then never completes)
    unsigned int target = extra_arrivals;
    for (int p = 0; p < passes; ++p) {
        target += G;
        if (!grid_sync(gb, target, status, wait_limit)) return;
        const size_t L = (size_t)T << p;
        const K* src = bk[cur];
        K* dst = bk[cur ^ 1];
        const uint32_t* vsrc = bv[cur];
        uint32_t* vdst = bv[cur ^ 1];
        for (size_t c = blockIdx.x; c < nblocks; c += G) {
            const size_t out0 = c * T;
            const PassGeom g = pass_geom(out0, n, L);
            const size_t d0 = out0 - g.pb;
            const size_t dend = g.alen + g.blen;
            const size_t d1 = (d0 + T < dend) ? d0 + T : dend;
            const K* A = src + g.pb;
            const K* B = A + g.alen;
            __syncthreads();  // split[] of the previous block is consumed
            if (warp == 0)
                split[0] = d0 == 0 ? 0 : corank_warp(A, g.alen, B, g.blen, d0, lane);
            else if (warp == 1)
                split[1] = d1 == dend ? g.alen : corank_warp(A, g.alen, B, g.blen, d1, lane);
            __syncthreads();
            const size_t a0 = split[0], a1 = split[1];
            const int nA = (int)(a1 - a0);
            const int nB = (int)(d1 - d0) - nA;
            const size_t oA = g.pb + a0, oB = g.pb + g.alen + (d0 - a0);
            const bool ok =
                (XF && p + 1 == passes)
                    ? merge_block<K, PAIRS, THREADS, IPT, true>(src + oA, nA, src + oB, nB,
                                                                PAIRS ? vsrc + oA : nullptr,
                                                                PAIRS ? vsrc + oB : nullptr, dst + out0,
                                                                PAIRS ? vdst + out0 : nullptr, smem_raw, &bar, phase,
                                                                status, xf_out)
                    : merge_block<K, PAIRS, THREADS, IPT, false>(src + oA, nA, src + oB, nB,
                                                                 PAIRS ? vsrc + oA : nullptr,
                                                                 PAIRS ? vsrc + oB : nullptr, dst + out0,
                                                                 PAIRS ? vdst + out0 : nullptr, smem_raw, &bar,
                                                                 phase, status, 0);
            if (!ok) return;
        }
        cur ^= 1;
    }
    if (t == 0) tma_store_wait_all();
}

template <class K, bool PAIRS, int THREADS, int IPT>
__host__ __device__ constexpr size_t small_sort_smem() {
    return tile_block_smem<K, PAIRS, THREADS>(THREADS * IPT) > merge_block_smem<K, PAIRS, THREADS, IPT>()
               ? tile_block_smem<K, PAIRS, THREADS>(THREADS * IPT)
               : merge_block_smem<K, PAIRS, THREADS, IPT>();
}

}  // namespace msort
