// Batched segmented sort: many independent arrays sorted in one call.
//
// The paper sorts one array; its chunk-then-merge structure (Sections
// "Multiprocessing Merge Sort" and "MPI Merge Sort") applies unchanged to
// each segment [off[i], off[i+1]) of a batch.  GPU plan, all enqueued on the
// caller's stream with fixed launch shapes (so the sequence can be captured
// in a CUDA graph and replayed):
//   1. k_seg_classify: one thread per segment puts the segment's index on the
//      work list of its length bucket (atomic append; order within a bucket
//      does not affect the result because segments are independent).
//   2. One persistent launch per small bucket: blocks of the bucket's shape
//      (32 x 17 up to 1024 x 33 keys) take segments from the list with an
//      atomic counter and sort each one entirely in shared memory with the
//      tile-sort body (network + merge-path rounds).
//   3. Segments of up to four large tiles (one or two merge passes): one
//      persistent launch sorts every tile of every such segment, then each
//      merge pass is one launch of co-rank searches (a thread per output
//      block, writing the block's descriptor) and one persistent launch of
//      bulk-TMA merge blocks, all segments' blocks at once, so the whole GPU
//      runs each phase.
//   4. One persistent launch for the longer segments: a block sorts the
//      segment's tiles, then runs the segment's merge passes itself
//      (co-ranks of all its output blocks by binary search in parallel, then
//      the bulk-TMA merge body per block), ping-ponging between the keys and
//      the context scratch.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "ctx.h"
#include "launch.h"
#include "sort_kernels.cuh"

namespace msort {

constexpr int kSegMaxBuckets = 6;   // small buckets
constexpr int kSegLarge = kSegMaxBuckets;  // index of the large-segment list
constexpr int kSegMid = kSegMaxBuckets + 1;  // index of the medium-segment list (up to kMidSlots tiles)
constexpr int kSegLists = kSegMaxBuckets + 2;
// counters[q] = entries of list q; counters[kSegLists + q] = its work-fetch
// counter; then the fetch counter of the medium path's tile launch and the
// number of output blocks of each of its merge passes
constexpr int kSegFetchMidTiles = 2 * kSegLists;
constexpr int kSegMidBlocks = 2 * kSegLists + 1;  // + pass: output blocks of that medium merge pass
constexpr int kMidSlots = 4;  // tiles of a medium segment
constexpr int kMidMergeSplit = 2;  // most merge output blocks per medium tile
constexpr int kMidPasses = 2;
constexpr unsigned int kStatusBadInput = 2u;
constexpr int kSegBadFlag = 63;  // counters[63]: this call's bad-input flag

struct SegBuckets {
    int n;                       // number of small buckets in use
    int lim[kSegMaxBuckets];     // bucket b takes lengths in (lim[b-1], lim[b]]
    int mid;                     // medium bucket: lengths in (lim[n-1], mid] (kMidSlots large tiles); 0 = none
};

// Device-side classification of segments into bucket work lists.
__global__ void k_seg_classify(const unsigned long long* __restrict__ off, size_t nseg, size_t n, SegBuckets bk,
                               unsigned int* __restrict__ lists, unsigned int* __restrict__ counts,
                               unsigned int* status) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    const unsigned long long b = off[i], e = off[i + 1];
    if (e < b || e > n || (i == 0 && b != 0) || (i == nseg - 1 && e != n)) {
        atomicOr(status, kStatusBadInput);
        atomicOr(&counts[kSegBadFlag], 1u);
        return;
    }
    const unsigned long long len = e - b;
    if (len <= 1) return;
    int q = len <= (unsigned long long)bk.mid ? kSegMid : kSegLarge;
    for (int k = 0; k < bk.n; ++k)
        if (len <= (unsigned long long)bk.lim[k]) {
            q = k;
            break;
        }
    const unsigned int pos = atomicAdd(&counts[q], 1u);
    lists[(size_t)q * nseg + pos] = (unsigned int)i;
}

// Next value of fetch counter `idx` for this block (all threads get the same value).
__device__ __forceinline__ unsigned int seg_fetch(unsigned int* counters, int idx, unsigned int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(&counters[idx], 1u);
    __syncthreads();
    return *slot;
}

// Next work item of list q for this block.
__device__ __forceinline__ unsigned int seg_next(unsigned int* counters, int q, unsigned int* slot) {
    return seg_fetch(counters, kSegLists + q, slot);
}

// Odd keys per thread (conflict-free strided shared-memory access) for a
// shape holding about num/4 of a THREADS x ipt tile.
__host__ __device__ constexpr int odd_ipt(int ipt, int num) {
    return (num * ipt + 3) / 4 + ((num * ipt + 3) / 4 % 2 == 0 ? 1 : 0);
}

// Blocks of a tile-sort shape that fit on one SM by shared memory (228 KB,
// 1 KB reserved per block), threads (2048) and the block limit (32).
template <class K, bool PAIRS, int THREADS, int IPT>
__host__ __device__ constexpr int tile_blocks_per_sm() {
    const int by_smem = (int)((228u << 10) / (tile_block_smem<K, PAIRS, THREADS>(THREADS * IPT) + 1024u));
    const int by_threads = 2048 / THREADS;
    const int b = by_smem < by_threads ? by_smem : by_threads;
    return b < 32 ? b : 32;
}

// Minimum blocks per SM for the small-bucket kernel of unsigned 32-bit keys
// without values: the 17-key shapes as many as shared memory allows (32
// registers); the 33-key shapes as many as 48 registers allow, the most
// they take without spilling.  Other key types are left to the compiler.
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__host__ __device__ constexpr int small_min_blocks() {
    if (sizeof(K) != 4 || PAIRS || XF) return 0;
    if (IPT <= 17) return tile_blocks_per_sm<K, PAIRS, THREADS, IPT>();
    return 65536 / (48 * THREADS) > 0 ? 65536 / (48 * THREADS) : 1;
}

// Small bucket: every segment fits one block of THREADS x IPT keys.  A
// block's cost follows its shape, not its fill, so a segment of at most
// about three quarters of that takes the shape with three quarters of the
// keys per thread.  XF as for the medium kernels.
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS, small_min_blocks<K, PAIRS, THREADS, IPT, XF>())
k_seg_small(K* keys, uint32_t* vals, const unsigned long long* __restrict__ off, size_t nseg,
            const unsigned int* __restrict__ lists, unsigned int* counters, int q, unsigned int* status, int xf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned int slot;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (counters[kSegBadFlag]) return;  // malformed offsets: sort nothing
    uint32_t phase = 0;
    const unsigned int count = counters[q];
    for (unsigned int w = seg_next(counters, q, &slot); w < count; w = seg_next(counters, q, &slot)) {
        const unsigned int s = lists[(size_t)q * nseg + w];
        const size_t b = off[s];
        const int len = (int)(off[s + 1] - b);
        constexpr int kQ3 = odd_ipt(IPT, 3);
        static_assert(kQ3 < IPT, "a smaller shape");
        K* sk = keys + b;
        uint32_t* sv = PAIRS ? vals + b : nullptr;
        const bool ok = len <= THREADS * kQ3
                            ? tile_sort_block<K, PAIRS, THREADS, kQ3, XF>(sk, sv, sk, sv, len, smem_raw, &bar,
                                                                          phase, status, xf, xf)
                            : tile_sort_block<K, PAIRS, THREADS, IPT, XF>(sk, sv, sk, sv, len, smem_raw, &bar,
                                                                          phase, status, xf, xf);
        if (!ok) return;
    }
}

// Make this block's global writes (bulk TMA stores and plain stores) visible
// to its own later reads of either kind (plain loads and bulk TMA loads).
__device__ __forceinline__ void block_pass_barrier() {
    if (threadIdx.x == 0) tma_store_wait_all();
    fence_proxy_async_global();
    __threadfence_block();
    __syncthreads();
}

// Large segments: tiles of THREADS x IPT keys, then merge passes with merge
// blocks of the same size, all by one block per segment.
// At least two blocks per SM: left unbounded the compiler took 128
// registers, which fits only one 512-thread block per SM; the 512-thread
// keys-only variant fits in 64 (a 12-byte spill).
template <class K, bool PAIRS, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 3 : 2)
k_seg_large(K* keys, uint32_t* vals, K* tkeys, uint32_t* tvals, const unsigned long long* __restrict__ off,
            size_t nseg, const unsigned int* __restrict__ lists, unsigned int* counters, unsigned int* status,
            int xf) {
    constexpr int T = THREADS * IPT;
    constexpr int W = T;
    constexpr int kSplitChunk = THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned int slot;
    __shared__ unsigned long long splits[kSplitChunk + 1];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (counters[kSegBadFlag]) return;  // malformed offsets: sort nothing
    uint32_t phase = 0;
    const int t = threadIdx.x;
    const unsigned int count = counters[kSegLarge];
    for (unsigned int w = seg_next(counters, kSegLarge, &slot); w < count;
         w = seg_next(counters, kSegLarge, &slot)) {
        const unsigned int s = lists[(size_t)kSegLarge * nseg + w];
        const size_t base = off[s];
        const size_t len = off[s + 1] - base;
        int passes = 0;
        for (size_t L = T; L < len; L *= 2) ++passes;
        K* bk[2] = {keys + base, tkeys + base};
        uint32_t* bv[2] = {PAIRS ? vals + base : nullptr, PAIRS ? tvals + base : nullptr};
        int cur = passes & 1;
        for (size_t j = 0; j < len; j += T) {
            const int valid = (int)(len - j < (size_t)T ? len - j : (size_t)T);
            if (!tile_sort_block<K, PAIRS, THREADS, IPT, true>(keys + base + j, PAIRS ? vals + base + j : nullptr,
                                                         bk[cur] + j, PAIRS ? bv[cur] + j : nullptr, valid,
                                                         smem_raw, &bar, phase, status, xf,
                                                         passes == 0 ? xf : 0))
                return;
        }
        block_pass_barrier();
        for (int p = 0; p < passes; ++p) {
            const size_t L = (size_t)T << p;
            const K* src = bk[cur];
            K* dst = bk[cur ^ 1];
            const size_t nblocks = (len + W - 1) / W;
            for (size_t c0 = 0; c0 < nblocks; c0 += kSplitChunk) {
                const size_t cn = nblocks - c0 < (size_t)kSplitChunk ? nblocks - c0 : (size_t)kSplitChunk;
                __syncthreads();
                // the co-rank of every block start in this chunk, in parallel
                if ((size_t)t < cn) {
                    const size_t out0 = (c0 + t) * W;
                    const PassGeom g = pass_geom(out0, len, L);
                    splits[t] = corank_search(src + g.pb, g.alen, src + g.pb + g.alen, g.blen, out0 - g.pb);
                }
                if (t == 0) {
                    // split at the start of the block after the chunk (or unused)
                    const size_t out0 = (c0 + cn) * W;
                    if (c0 + cn < nblocks) {
                        const PassGeom g = pass_geom(out0, len, L);
                        splits[cn] = corank_search(src + g.pb, g.alen, src + g.pb + g.alen, g.blen, out0 - g.pb);
                    }
                }
                __syncthreads();
                for (size_t ci = 0; ci < cn; ++ci) {
                    const size_t out0 = (c0 + ci) * W;
                    const PassGeom g = pass_geom(out0, len, L);
                    const size_t d0 = out0 - g.pb;
                    const size_t dend = g.alen + g.blen;
                    const size_t d1 = (d0 + W < dend) ? d0 + W : dend;
                    const size_t a0 = splits[ci];
                    const size_t a1 = (d1 == dend) ? g.alen : (size_t)splits[ci + 1];
                    const int nA = (int)(a1 - a0);
                    const int nB = (int)(d1 - d0) - nA;
                    const size_t oA = g.pb + a0, oB = g.pb + g.alen + (d0 - a0);
                    const bool ok =
                        xf && p + 1 == passes
                            ? merge_block<K, PAIRS, THREADS, IPT, true>(
                                  src + oA, nA, src + oB, nB, PAIRS ? bv[cur] + oA : nullptr,
                                  PAIRS ? bv[cur] + oB : nullptr, dst + out0, PAIRS ? bv[cur ^ 1] + out0 : nullptr,
                                  smem_raw, &bar, phase, status, xf)
                            : merge_block<K, PAIRS, THREADS, IPT, false>(
                                  src + oA, nA, src + oB, nB, PAIRS ? bv[cur] + oA : nullptr,
                                  PAIRS ? bv[cur] + oB : nullptr, dst + out0, PAIRS ? bv[cur ^ 1] + out0 : nullptr,
                                  smem_raw, &bar, phase, status, 0);
                    if (!ok) return;
                }
            }
            block_pass_barrier();
            cur ^= 1;
        }
    }
}

// Medium segments: more than one on-chip tile, at most kMidSlots tiles of
// T = THREADS x IPT keys, so one or two merge passes.  Work item it of the
// tile phase is tile it % kMidSlots of the segment at position
// it / kMidSlots of the medium list; an item of a merge pass is output
// block it % S (W keys, S = kMidSlots x T / W) of the segment at position
// it / S.  Slots past the end of a shorter segment are skipped.  A
// segment's tiles land in the buffer its last pass does not write (keys for
// two passes, the scratch for one), and each pass ping-pongs to the other,
// so the last pass writes the keys.
__device__ __forceinline__ int mid_passes(size_t len, size_t T) { return len > 2 * T ? 2 : 1; }

// XF: whether the keys take a transform (signed or floating-point keys);
// the instance without one keeps the transform's registers out of the
// tile and merge bodies, which at 40 registers would otherwise spill.
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 3 : 2)
k_seg_mid_tiles(K* keys, uint32_t* vals, K* tkeys, uint32_t* tvals, const unsigned long long* __restrict__ off,
                size_t nseg, const unsigned int* __restrict__ lists, unsigned int* counters, unsigned int* status,
                int xf) {
    constexpr int T = THREADS * IPT;
    constexpr int kQ1 = odd_ipt(IPT, 1), kQ2 = odd_ipt(IPT, 2), kQ3 = odd_ipt(IPT, 3);
    static_assert(kQ1 < kQ2 && kQ2 < kQ3 && kQ3 < IPT, "four distinct tile shapes");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned int slot;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (counters[kSegBadFlag]) return;  // malformed offsets: sort nothing
    uint32_t phase = 0;
    const unsigned int items = counters[kSegMid] * kMidSlots;
    for (unsigned int it = seg_fetch(counters, kSegFetchMidTiles, &slot); it < items;
         it = seg_fetch(counters, kSegFetchMidTiles, &slot)) {
        const unsigned int s = lists[(size_t)kSegMid * nseg + it / kMidSlots];
        const size_t j = (size_t)(it % kMidSlots) * T;
        const size_t base = off[s], len = off[s + 1] - base;
        if (j >= len) continue;
        const int valid = (int)(len - j < (size_t)T ? len - j : (size_t)T);
        const bool odd = mid_passes(len, T) & 1;
        K* dk = (odd ? tkeys : keys) + base + j;
        uint32_t* dv = PAIRS ? (odd ? tvals : vals) + base + j : nullptr;
        // a tile's cost follows its shape, not its fill: a segment's last
        // tile takes the smallest of four shapes (about a quarter, half,
        // three quarters or all of the keys per thread) that holds it
        const K* sk = keys + base + j;
        const uint32_t* sv = PAIRS ? vals + base + j : nullptr;
        bool ok;
        if (valid <= THREADS * kQ1)
            ok = tile_sort_block<K, PAIRS, THREADS, kQ1, XF>(sk, sv, dk, dv, valid, smem_raw, &bar, phase, status, xf, 0);
        else if (valid <= THREADS * kQ2)
            ok = tile_sort_block<K, PAIRS, THREADS, kQ2, XF>(sk, sv, dk, dv, valid, smem_raw, &bar, phase, status, xf, 0);
        else if (valid <= THREADS * kQ3)
            ok = tile_sort_block<K, PAIRS, THREADS, kQ3, XF>(sk, sv, dk, dv, valid, smem_raw, &bar, phase, status, xf, 0);
        else
            ok = tile_sort_block<K, PAIRS, THREADS, IPT, XF>(sk, sv, dk, dv, valid, smem_raw, &bar, phase, status, xf, 0);
        if (!ok) return;
    }
}

// One output block of a medium merge pass, written by k_seg_mid_part and
// read by k_seg_mid_merge (48 bytes, copied to shared memory in three
// 16-byte pieces).
struct __align__(16) MidBlock {
    unsigned long long a, b, d;  // element offsets: the A and B windows (source buffer), the output (other one)
    unsigned int na, nb;         // window lengths
    unsigned int src;            // source buffer: 0 the keys, 1 the scratch
    unsigned int last;           // 1 on the segment's last merge pass
    unsigned int pad[2];
};
static_assert(sizeof(MidBlock) == 48, "three 16-byte pieces");

// Most medium merge blocks of one pass: a medium segment holds more than
// 1024 keys in every plan, so there are at most n / 1025 of them.
inline size_t mid_block_cap(size_t n, size_t nseg) {
    const size_t segs = n / 1025 < nseg ? n / 1025 : nseg;
    return (segs + 1) * kMidSlots * kMidMergeSplit;
}

// Output blocks of merge pass `pass` (a thread per segment slot): the stable
// co-ranks of the block's first and last diagonal, appended to `blocks` in
// any order (the blocks are independent).  A block's end co-rank is the next
// slot's start co-rank, so lanes take it from their neighbour and only the
// last lane of a warp searches twice.
template <class K>
__global__ void k_seg_mid_part(const K* __restrict__ keys, const K* __restrict__ tkeys,
                               const unsigned long long* __restrict__ off, size_t nseg,
                               const unsigned int* __restrict__ lists, unsigned int* counters, int pass, size_t T,
                               size_t W, MidBlock* __restrict__ blocks) {
    const size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int lane = threadIdx.x & 31u;
    const size_t slots = kMidSlots * (T / W);
    if (counters[kSegBadFlag]) return;  // the same for every thread
    bool valid = false;
    size_t a0 = 0, d0 = 0, d1 = 0, dend = 0;
    size_t base = 0, pb = 0, alen = 0, blen = 0, out0 = 0;
    int P = 0;
    const K* src = nullptr;
    if (it < (size_t)counters[kSegMid] * slots) {
        const unsigned int s = lists[(size_t)kSegMid * nseg + it / slots];
        base = off[s];
        const size_t len = off[s + 1] - base;
        P = mid_passes(len, T);
        out0 = (it % slots) * W;
        if (pass < P && out0 < len) {
            valid = true;
            src = (((P ^ pass) & 1) ? tkeys : keys) + base;  // the pass's input buffer
            const PassGeom g = pass_geom(out0, len, T << pass);
            pb = g.pb;
            alen = g.alen;
            blen = g.blen;
            d0 = out0 - pb;
            dend = alen + blen;
            d1 = d0 + W < dend ? d0 + W : dend;
            a0 = corank_search(src + pb, alen, src + pb + alen, blen, d0);
        }
    }
    // the next slot (lane + 1) starts where this block ends when the pair goes on
    const unsigned long long next = __shfl_down_sync(0xffffffffu, (unsigned long long)a0, 1);
    size_t a1 = alen;
    if (valid && d1 < dend) a1 = lane < 31 ? (size_t)next : corank_search(src + pb, alen, src + pb + alen, blen, d1);
    const unsigned int mask = __ballot_sync(0xffffffffu, valid);
    if (!mask) return;  // the same for the whole warp
    const int leader = __ffs(mask) - 1;
    unsigned int first = 0;
    if ((int)lane == leader) first = atomicAdd(&counters[kSegMidBlocks + pass], (unsigned int)__popc(mask));
    first = __shfl_sync(0xffffffffu, first, leader);
    if (!valid) return;
    MidBlock mb;
    mb.a = base + pb + a0;
    mb.b = base + pb + alen + (d0 - a0);
    mb.d = base + out0;
    mb.na = (unsigned int)(a1 - a0);
    mb.nb = (unsigned int)((d1 - d0) - (a1 - a0));
    mb.src = (unsigned int)((P ^ pass) & 1);
    mb.last = pass + 1 == P ? 1u : 0u;
    mb.pad[0] = mb.pad[1] = 0u;
    blocks[first + __popc(mask & ((1u << lane) - 1u))] = mb;
}

// 16-byte asynchronous copy from global to shared memory, completed by the
// issuing thread's cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The output blocks of merge pass `pass` (W = THREADS x IPT outputs each),
// block i to CTA i mod gridDim.x.  Thread 0 copies the next block's
// descriptor to shared memory while the current one merges, so a block's
// work starts without a chain of dependent loads.
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 3 : (sizeof(K) == 4 && !PAIRS && IPT == 33 ? 6 : 2))
k_seg_mid_merge(K* keys, uint32_t* vals, K* tkeys, uint32_t* tvals, const unsigned int* __restrict__ counters,
                int pass, const MidBlock* __restrict__ blocks, unsigned int* status, int xf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ MidBlock desc[2];
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (counters[kSegBadFlag]) return;
    uint32_t phase = 0;
    const unsigned int items = counters[kSegMidBlocks + pass];
    if (t == 0 && blockIdx.x < items) {
        for (int k = 0; k < 3; ++k)
            cp_async16(reinterpret_cast<char*>(&desc[0]) + 16 * k,
                       reinterpret_cast<const char*>(blocks + blockIdx.x) + 16 * k);
        cp_async_commit();
    }
    int cur = 0;
    for (unsigned int i = blockIdx.x; i < items; i += gridDim.x, cur ^= 1) {
        if (t == 0) cp_async_wait_all();
        __syncthreads();  // desc[cur] is in place; every thread is done with desc[cur ^ 1]
        const MidBlock d = desc[cur];
        if (t == 0 && i + gridDim.x < items) {
            for (int k = 0; k < 3; ++k)
                cp_async16(reinterpret_cast<char*>(&desc[cur ^ 1]) + 16 * k,
                           reinterpret_cast<const char*>(blocks + i + gridDim.x) + 16 * k);
            cp_async_commit();
        }
        const K* src = d.src ? tkeys : keys;
        K* dst = d.src ? keys : tkeys;
        const uint32_t* vs = PAIRS ? (d.src ? tvals : vals) : nullptr;
        uint32_t* vd = PAIRS ? (d.src ? vals : tvals) : nullptr;
        const bool ok = (XF && d.last)
                            ? merge_block<K, PAIRS, THREADS, IPT, true>(
                                  src + d.a, (int)d.na, src + d.b, (int)d.nb, PAIRS ? vs + d.a : nullptr,
                                  PAIRS ? vs + d.b : nullptr, dst + d.d, PAIRS ? vd + d.d : nullptr, smem_raw, &bar,
                                  phase, status, xf)
                            : merge_block<K, PAIRS, THREADS, IPT, false>(
                                  src + d.a, (int)d.na, src + d.b, (int)d.nb, PAIRS ? vs + d.a : nullptr,
                                  PAIRS ? vs + d.b : nullptr, dst + d.d, PAIRS ? vd + d.d : nullptr, smem_raw, &bar,
                                  phase, status, 0);
        if (!ok) return;
    }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
namespace {

template <class F>
int persistent_blocks(F* f, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(reinterpret_cast<const void*>(f), threads, smem, dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem);
    const int blocks = sms * (per > 0 ? per : 1);
    cache[key] = blocks;
    return blocks;
}

template <class F>
cudaError_t allow_smem(F* f, size_t smem) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(f));
    if (e != cudaSuccess) return e;
    if ((int)smem <= fa.maxDynamicSharedSizeBytes) return cudaSuccess;
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <class K, bool PAIRS, int TH, int IPT>
cudaError_t launch_small(K* keys, uint32_t* vals, const unsigned long long* off, size_t nseg,
                         const unsigned int* lists, unsigned int* counters, int q, unsigned int* status,
                         cudaStream_t st, int xf) {
    auto f = xf ? k_seg_small<K, PAIRS, TH, IPT, true> : k_seg_small<K, PAIRS, TH, IPT, false>;
    const size_t sm = tile_block_smem<K, PAIRS, TH>(TH * IPT);
    cudaError_t e = allow_smem(f, sm);
    if (e != cudaSuccess) return e;
    const int blocks = persistent_blocks(f, TH, sm);
    f<<<blocks, TH, sm, st>>>(keys, vals, off, nseg, lists, counters, q, status, xf);
    return cudaGetLastError();
}

template <class K, bool PAIRS, int TH, int IPT>
cudaError_t launch_large(K* keys, uint32_t* vals, K* tk, uint32_t* tv, const unsigned long long* off, size_t nseg,
                         const unsigned int* lists, unsigned int* counters, unsigned int* status,
                         cudaStream_t st, int xf) {
    auto f = k_seg_large<K, PAIRS, TH, IPT>;
    const size_t a = tile_block_smem<K, PAIRS, TH>(TH * IPT), b = merge_block_smem<K, PAIRS, TH, IPT>();
    const size_t sm = a > b ? a : b;
    cudaError_t e = allow_smem(f, sm);
    if (e != cudaSuccess) return e;
    const int blocks = persistent_blocks(f, TH, sm);
    f<<<blocks, TH, sm, st>>>(keys, vals, tk, tv, off, nseg, lists, counters, status, xf);
    return cudaGetLastError();
}

// The medium path: the tile launch, then per merge pass the co-rank launch
// and the merge launch (fixed shapes; work comes from the device-side list).
// Tiles of TH x IPT keys; merge blocks of MTH x IPT outputs.
template <class K, bool PAIRS, int TH, int IPT, int MTH, bool XF>
cudaError_t launch_mid_xf(K* keys, uint32_t* vals, K* tk, uint32_t* tv, const unsigned long long* off, size_t nseg,
                          const unsigned int* lists, unsigned int* counters, MidBlock* desc,
                          unsigned int* status, cudaStream_t st, int xf) {
    auto ft = k_seg_mid_tiles<K, PAIRS, TH, IPT, XF>;
    const size_t st_sm = tile_block_smem<K, PAIRS, TH>(TH * IPT);
    cudaError_t e = allow_smem(ft, st_sm);
    if (e != cudaSuccess) return e;
    ft<<<persistent_blocks(ft, TH, st_sm), TH, st_sm, st>>>(keys, vals, tk, tv, off, nseg, lists, counters, status,
                                                            xf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    auto fm = k_seg_mid_merge<K, PAIRS, MTH, IPT, XF>;
    const size_t m_sm = merge_block_smem<K, PAIRS, MTH, IPT>();
    if ((e = allow_smem(fm, m_sm)) != cudaSuccess) return e;
    const int mblocks = persistent_blocks(fm, MTH, m_sm);
    const size_t items = (size_t)kMidSlots * (TH / MTH) * nseg;
    for (int pass = 0; pass < kMidPasses; ++pass) {
        k_seg_mid_part<K><<<(unsigned)((items + 127) / 128), 128, 0, st>>>(
            keys, tk, off, nseg, lists, counters, pass, (size_t)(TH * IPT), (size_t)(MTH * IPT), desc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        fm<<<mblocks, MTH, m_sm, st>>>(keys, vals, tk, tv, counters, pass, desc, status, xf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template <class K, bool PAIRS, int TH, int IPT, int MTH = TH>
cudaError_t launch_mid(K* keys, uint32_t* vals, K* tk, uint32_t* tv, const unsigned long long* off, size_t nseg,
                       const unsigned int* lists, unsigned int* counters, MidBlock* desc,
                       unsigned int* status, cudaStream_t st, int xf) {
    static_assert(TH % MTH == 0 && TH / MTH <= kMidMergeSplit, "merge blocks tile a medium tile");
    return xf ? launch_mid_xf<K, PAIRS, TH, IPT, MTH, true>(keys, vals, tk, tv, off, nseg, lists, counters, desc,
                                                            status, st, xf)
              : launch_mid_xf<K, PAIRS, TH, IPT, MTH, false>(keys, vals, tk, tv, off, nseg, lists, counters, desc,
                                                             status, st, 0);
}
constexpr int kMidLaunches = 1 + 2 * kMidPasses;

// Bucket plans per key/value type: small buckets (threads x keys per thread),
// the medium bucket (up to kMidSlots large tiles) and the tile of the
// large-segment kernel.
template <class K, bool PAIRS>
struct SegPlan;

#define MSORT_SMALL_LAUNCHES(K, PAIRS)                                                                          \
    if ((e = launch_small<K, PAIRS, 32, 17>(keys, vals, off, nseg, lists, counters, 0, status, st, xf))) return e;  \
    if ((e = launch_small<K, PAIRS, 128, 17>(keys, vals, off, nseg, lists, counters, 1, status, st, xf))) return e; \
    if ((e = launch_small<K, PAIRS, 256, 33>(keys, vals, off, nseg, lists, counters, 2, status, st, xf))) return e;

// Small buckets a factor of two apart (544 ... 8448 keys; the first five
// launches, buckets 0-4).  A block's cost follows its shape, not its fill,
// and segment lengths spread evenly on a log scale fill a bucket twice as
// wide as the one below it to about 72% on average, against 54% for four
// times as wide: on 50,000 log-uniform segments 3.52 against 3.57 ms.
#define MSORT_SMALL2X_LAUNCHES(K, PAIRS)                                                                        \
    if ((e = launch_small<K, PAIRS, 32, 17>(keys, vals, off, nseg, lists, counters, 0, status, st, xf))) return e;  \
    if ((e = launch_small<K, PAIRS, 64, 17>(keys, vals, off, nseg, lists, counters, 1, status, st, xf))) return e;  \
    if ((e = launch_small<K, PAIRS, 128, 17>(keys, vals, off, nseg, lists, counters, 2, status, st, xf))) return e; \
    if ((e = launch_small<K, PAIRS, 256, 17>(keys, vals, off, nseg, lists, counters, 3, status, st, xf))) return e; \
    if ((e = launch_small<K, PAIRS, 256, 33>(keys, vals, off, nseg, lists, counters, 4, status, st, xf))) return e;

// 32-bit keys only: the largest on-chip bucket (16896 or 33792 keys) and the
// large-segment tile (8448 or 16896) are tunable (msort_tune).  Default
// 16896 / 16896: on the 50,000-segment workload 1.5% faster than a 33792-key
// bucket, and 10% faster than 8448-key large-segment tiles.
template <>
struct SegPlan<uint32_t, false> {
    static SegBuckets buckets(const msort_ctx* ctx) {
        const int mid = kMidSlots * ((ctx && ctx->seg_large_tile == 8448) ? 8448 : 16896);
        if (ctx && ctx->seg_max_small == 33792) return SegBuckets{5, {544, 2176, 8448, 16896, 33792, 0}, mid};
        return SegBuckets{6, {544, 1088, 2176, 4352, 8448, 16896}, mid};
    }
    static cudaError_t run(const msort_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* tk, uint32_t* tv,
                           const unsigned long long* off, size_t nseg, const unsigned int* lists,
                           unsigned int* counters, MidBlock* mdesc, unsigned int* status, cudaStream_t st,
                           int xf) {
        cudaError_t e;
        if (buckets(ctx).n == 6) {
            MSORT_SMALL2X_LAUNCHES(uint32_t, false)
            if ((e = launch_small<uint32_t, false, 512, 33>(keys, vals, off, nseg, lists, counters, 5, status, st,
                                                            xf)))
                return e;
        } else {  // the tuned plan with on-chip segments up to 33792 keys
            MSORT_SMALL_LAUNCHES(uint32_t, false)
            if ((e = launch_small<uint32_t, false, 512, 33>(keys, vals, off, nseg, lists, counters, 3, status, st,
                                                            xf)))
                return e;
            if ((e = launch_small<uint32_t, false, 1024, 33>(keys, vals, off, nseg, lists, counters, 4, status, st,
                                                             xf)))
                return e;
        }
        if (ctx && ctx->seg_large_tile == 8448) {
            if ((e = launch_mid<uint32_t, false, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, mdesc,
                                                          status, st, xf)))
                return e;
            return launch_large<uint32_t, false, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, status,
                                                          st, xf);
        }
        // merge blocks of half a tile: 256 x 33 at 40 registers fits six
        // blocks per SM, the shape of the plain merge pass
        if ((e = launch_mid<uint32_t, false, 512, 33, 256>(keys, vals, tk, tv, off, nseg, lists, counters, mdesc,
                                                           status, st, xf)))
            return e;
        return launch_large<uint32_t, false, 512, 33>(keys, vals, tk, tv, off, nseg, lists, counters, status, st, xf);
    }
};

template <>
struct SegPlan<uint32_t, true> {
    static SegBuckets buckets(const msort_ctx*) {
        return SegBuckets{6, {544, 1088, 2176, 4352, 8448, 16896}, kMidSlots * 8448};
    }
    static cudaError_t run(const msort_ctx*, uint32_t* keys, uint32_t* vals, uint32_t* tk, uint32_t* tv,
                           const unsigned long long* off,
                           size_t nseg, const unsigned int* lists, unsigned int* counters, MidBlock* mdesc,
                           unsigned int* status, cudaStream_t st, int xf) {
        cudaError_t e;
        MSORT_SMALL2X_LAUNCHES(uint32_t, true)
        if ((e = launch_small<uint32_t, true, 512, 33>(keys, vals, off, nseg, lists, counters, 5, status, st, xf)))
            return e;
        if ((e = launch_mid<uint32_t, true, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, mdesc, status,
                                                     st, xf)))
            return e;
        return launch_large<uint32_t, true, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, status, st, xf);
    }
};

template <>
struct SegPlan<uint64_t, false> {
    static SegBuckets buckets(const msort_ctx*) {
        return SegBuckets{6, {544, 1088, 2176, 4352, 8448, 16896}, kMidSlots * 8448};
    }
    static cudaError_t run(const msort_ctx*, uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv,
                           const unsigned long long* off,
                           size_t nseg, const unsigned int* lists, unsigned int* counters, MidBlock* mdesc,
                           unsigned int* status, cudaStream_t st, int xf) {
        cudaError_t e;
        MSORT_SMALL2X_LAUNCHES(uint64_t, false)
        if ((e = launch_small<uint64_t, false, 512, 33>(keys, vals, off, nseg, lists, counters, 5, status, st, xf)))
            return e;
        if ((e = launch_mid<uint64_t, false, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, mdesc, status,
                                                      st, xf)))
            return e;
        return launch_large<uint64_t, false, 256, 33>(keys, vals, tk, tv, off, nseg, lists, counters, status, st, xf);
    }
};

template <>
struct SegPlan<uint64_t, true> {
    static SegBuckets buckets(const msort_ctx*) {
        return SegBuckets{5, {544, 1088, 2176, 4352, 8448, 0}, kMidSlots * 4352};
    }
    static cudaError_t run(const msort_ctx*, uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv,
                           const unsigned long long* off,
                           size_t nseg, const unsigned int* lists, unsigned int* counters, MidBlock* mdesc,
                           unsigned int* status, cudaStream_t st, int xf) {
        cudaError_t e;
        MSORT_SMALL2X_LAUNCHES(uint64_t, true)
        if ((e = launch_mid<uint64_t, true, 256, 17>(keys, vals, tk, tv, off, nseg, lists, counters, mdesc, status,
                                                     st, xf)))
            return e;
        return launch_large<uint64_t, true, 256, 17>(keys, vals, tk, tv, off, nseg, lists, counters, status, st, xf);
    }
};

struct SegLayout {
    size_t keys, vals, lists, counters, mdesc, end;
};

template <class K, bool PAIRS>
SegLayout seg_layout(size_t n, size_t nseg) {
    SegLayout l{};
    l.keys = 0;
    l.vals = align_up(n * sizeof(K), 256);
    l.lists = l.vals + (PAIRS ? align_up(n * 4, 256) : 0);
    l.counters = l.lists + align_up((size_t)kSegLists * nseg * 4, 256);
    l.mdesc = l.counters + 256;
    l.end = l.mdesc + align_up(mid_block_cap(n, nseg) * sizeof(MidBlock), 256);
    return l;
}

template <class K, bool PAIRS>
msort_status seg_enqueue(msort_ctx* ctx, K* keys, uint32_t* vals, const unsigned long long* off, size_t nseg,
                         size_t n, cudaStream_t st, int xf) {
    const SegLayout l = seg_layout<K, PAIRS>(n, nseg);
    unsigned char* sp = static_cast<unsigned char*>(ctx->scratch);
    K* tk = reinterpret_cast<K*>(sp + l.keys);
    uint32_t* tv = PAIRS ? reinterpret_cast<uint32_t*>(sp + l.vals) : nullptr;
    unsigned int* lists = reinterpret_cast<unsigned int*>(sp + l.lists);
    unsigned int* counters = reinterpret_cast<unsigned int*>(sp + l.counters);
    MidBlock* mdesc = reinterpret_cast<MidBlock*>(sp + l.mdesc);
    cudaError_t e = cudaMemsetAsync(counters, 0, 256, st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing segment counters");
    prof_begin(ctx, KK_SEGMENTED, st);
    k_seg_classify<<<(unsigned)((nseg + 255) / 256), 256, 0, st>>>(off, nseg, n, SegPlan<K, PAIRS>::buckets(ctx),
                                                                   lists, counters, ctx->d_status);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = SegPlan<K, PAIRS>::run(ctx, keys, vals, tk, tv, off, nseg, lists, counters, mdesc, ctx->d_status, st,
                                   xf);
    prof_end(ctx, KK_SEGMENTED, st);
    ctx->launches += 1 + SegPlan<K, PAIRS>::buckets(ctx).n + kMidLaunches + 1;
    if (e != cudaSuccess) return cuda_fail(e, "segmented sort launch");
    return MSORT_OK;
}

struct SegGraphKey {
    const void* keys;
    const void* vals;
    const void* off;
    size_t nseg, n;
    int kt;  // key bytes, values and key transform
    const void* scratch;
    int tune_small, tune_large;
    bool operator<(const SegGraphKey& o) const {
        return std::tie(keys, vals, off, nseg, n, kt, scratch, tune_small, tune_large) <
               std::tie(o.keys, o.vals, o.off, o.nseg, o.n, o.kt, o.scratch, o.tune_small, o.tune_large);
    }
};

// At most kMaxSegGraphs graphs are kept; a new one evicts the least
// recently used after the device has finished everything in flight.
constexpr size_t kMaxSegGraphs = 64;
struct GraphCache {
    std::map<SegGraphKey, std::pair<cudaGraphExec_t, unsigned long long>> seg;  // graph, tick of last use
    unsigned long long tick = 0;
};

}  // namespace

GraphCache* graph_cache(msort_ctx* ctx) {
    if (!ctx->graphs) ctx->graphs = new GraphCache();
    return static_cast<GraphCache*>(ctx->graphs);
}

void graphs_destroy(msort_ctx* ctx) {
    if (!ctx->graphs) return;
    GraphCache* gc = static_cast<GraphCache*>(ctx->graphs);
    for (auto& kv : gc->seg) cudaGraphExecDestroy(kv.second.first);
    delete gc;
    ctx->graphs = nullptr;
}

template <class K, bool PAIRS>
msort_status seg_sort(msort_ctx* ctx, K* keys, uint32_t* vals, const unsigned long long* off, size_t nseg, size_t n,
                      const msort_options* opt, cudaStream_t st, int xf) {
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    msort_status s = ensure_scratch(ctx, seg_layout<K, PAIRS>(n, nseg).end, st);
    if (s != MSORT_OK) return s;
    const bool use_graph = opt && opt->use_graph;
    if (!use_graph || ctx->profiling) {
        s = seg_enqueue<K, PAIRS>(ctx, keys, vals, off, nseg, n, st, xf);
    } else {
        GraphCache* gc = graph_cache(ctx);
        const SegGraphKey key{keys,         vals, off, nseg, n, ((int)sizeof(K) * 2 + PAIRS) * 4 + xf, ctx->scratch,
                              ctx->seg_max_small, ctx->seg_large_tile};
        auto it = gc->seg.find(key);
        if (it == gc->seg.end()) {
            if (gc->seg.size() >= kMaxSegGraphs) {
                auto lru = gc->seg.begin();
                for (auto j = gc->seg.begin(); j != gc->seg.end(); ++j)
                    if (j->second.second < lru->second.second) lru = j;
                e = cudaDeviceSynchronize();
                if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
                cudaGraphExecDestroy(lru->second.first);
                gc->seg.erase(lru);
            }
            cudaStream_t cap;
            e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const unsigned long long before = ctx->launches;
                s = seg_enqueue<K, PAIRS>(ctx, keys, vals, off, nseg, n, cap, xf);
                ctx->launches = before;
                cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
                if (s == MSORT_OK && e2 != cudaSuccess) s = cuda_fail(e2, "cudaStreamEndCapture");
            } else {
                s = cuda_fail(e, "cudaStreamBeginCapture");
            }
            cudaStreamDestroy(cap);
            if (s != MSORT_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            it = gc->seg.emplace(key, std::make_pair(exec, 0ull)).first;
        }
        it->second.second = ++gc->tick;
        e = cudaGraphLaunch(it->second.first, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        ctx->launches += 1 + SegPlan<K, PAIRS>::buckets(ctx).n + 1;
    }
    cudaEventRecord(ctx->scratch_done, st);
    ctx->last_stream = st;
    ctx->scratch_pending = true;
    return s;
}

}  // namespace msort

using namespace msort;

extern "C" msort_status msort_segmented_sort(msort_ctx* ctx, void* d_keys, uint32_t* d_vals,
                                             const uint64_t* d_offsets, size_t nseg, size_t n, msort_key_type kt,
                                             const msort_options* opt, void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    int xf = 0;  // order-preserving key transform (see xf_forward)
    if (kt == MSORT_I32 || kt == MSORT_I64) xf = 1;
    if (kt == MSORT_F32 || kt == MSORT_F64) xf = 2;
    const bool wide = kt == MSORT_U64 || kt == MSORT_I64 || kt == MSORT_F64;
    if (!xf && kt != MSORT_U32 && kt != MSORT_U64) return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
    if (nseg == 0) return MSORT_OK;
    if (!d_offsets) return fail(MSORT_ERR_INVALID_ARG, "d_offsets is NULL");
    if (n && !d_keys) return fail(MSORT_ERR_INVALID_ARG, "d_keys is NULL");
    if (nseg > 0xFFFFFFFFull) return fail(MSORT_ERR_UNSUPPORTED, "more than 2^32 - 1 segments");
    const size_t ks = wide ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(d_keys) % ks || reinterpret_cast<uintptr_t>(d_vals) % 4 ||
        reinterpret_cast<uintptr_t>(d_offsets) % 8)
        return fail(MSORT_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned long long* off = reinterpret_cast<const unsigned long long*>(d_offsets);
    if (!wide)
        return d_vals ? seg_sort<uint32_t, true>(ctx, static_cast<uint32_t*>(d_keys), d_vals, off, nseg, n, opt, st, xf)
                      : seg_sort<uint32_t, false>(ctx, static_cast<uint32_t*>(d_keys), nullptr, off, nseg, n, opt, st,
                                                  xf);
    return d_vals ? seg_sort<uint64_t, true>(ctx, static_cast<uint64_t*>(d_keys), d_vals, off, nseg, n, opt, st, xf)
                  : seg_sort<uint64_t, false>(ctx, static_cast<uint64_t*>(d_keys), nullptr, off, nseg, n, opt, st, xf);
}
