// One round of the pairwise merge tree over sorted runs of arbitrary
// lengths laid end to end (Section "MPI Merge Sort", "Merging the
// subarrays", Figs. 16-17: each round merges neighbouring runs until one is
// left; here the runs may have unequal lengths, as the out-of-core sort's
// slices and the sample sort's received pieces do).  Pair j merges [p[j], m[j]) with
// [m[j], p[j+1]) into the same positions of the destination; equal keys keep
// run order.  Output blocks of W never straddle two pairs: pair j owns
// blocks [c[j], c[j+1]).
#pragma once

#include "launch.h"
#include "sort_kernels.cuh"

namespace msort {

// Pair of output block `blk`: the last j with c[j] <= blk.
__device__ __forceinline__ int run_pair_of(const RunPairs& rp, unsigned long long blk) {
    int lo = 0, hi = rp.np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rp.c[mid] <= blk)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// splits[blk] = co-rank of block blk's first output inside its pair.
template <class K>
__global__ void k_partition_runs(const K* __restrict__ src, const __grid_constant__ RunPairs rp, size_t W,
                                 unsigned long long* __restrict__ splits) {
    const unsigned long long blk = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= rp.c[rp.np]) return;
    const int j = run_pair_of(rp, blk);
    const size_t pb = rp.p[j], alen = rp.m[j] - pb, blen = rp.p[j + 1] - rp.m[j];
    splits[blk] = corank_search(src + pb, alen, src + rp.m[j], blen, (size_t)(blk - rp.c[j]) * W);
}

// Block blk writes its pair's outputs [d0, min(d0 + W, pair length)).
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS)
k_merge_runs(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
             uint32_t* __restrict__ vdst, const __grid_constant__ RunPairs rp,
             const unsigned long long* __restrict__ splits, unsigned int* status, int xf_out) {
    constexpr int W = THREADS * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    const unsigned long long blk = blockIdx.x;
    const int j = run_pair_of(rp, blk);
    const size_t pb = rp.p[j], alen = rp.m[j] - pb, dend = rp.p[j + 1] - pb;
    const size_t d0 = (size_t)(blk - rp.c[j]) * W;
    const size_t d1 = d0 + W < dend ? d0 + W : dend;
    const size_t a0 = splits[blk];
    const size_t a1 = d1 == dend ? alen : (size_t)splits[blk + 1];
    const int nA = (int)(a1 - a0);
    const int nB = (int)(d1 - d0) - nA;
    const size_t oA = pb + a0, oB = pb + alen + (d0 - a0);
    uint32_t phase = 0;
    merge_block<K, PAIRS, THREADS, IPT, XF>(src + oA, nA, src + oB, nB, PAIRS ? vsrc + oA : nullptr,
                                            PAIRS ? vsrc + oB : nullptr, dst + pb + d0,
                                            PAIRS ? vdst + pb + d0 : nullptr, smem_raw, &bar, phase, status, xf_out);
}

}  // namespace msort
