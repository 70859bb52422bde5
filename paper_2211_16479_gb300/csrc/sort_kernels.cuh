// Device code of the merge sort: tile sort, co-rank partition, merge pass.
//
// The method (arXiv 2211.16479): sort fixed-size chunks independently
// (Section "Multiprocessing Merge Sort", Figs. 6-7), then merge sorted runs
// pairwise, one round at a time, until a single run is left (Section "MPI
// Merge Sort", Fig. 13).  merge() itself is left undefined in the paper; it
// is read here as the stable two-way merge that takes from the left run while
// left <= right.
//
// GPU mapping:
//  * Tile sort (a "chunk" of the multiprocessing design): one thread block
//    sorts T = THREADS * IPT keys.  Each thread holds IPT keys in registers;
//    a bitonic network sorts each warp's 32 * IPT keys (in-thread stages are
//    register compare-exchanges, cross-lane stages use __shfl_xor_sync), and
//    log2(THREADS / 32) shared-memory merge rounds join the warp runs.
//    Stability for key-value tiles comes from comparing (key, tile position):
//    all such items are distinct, so any sorting network yields the stable
//    order.
//  * Partition: the Merge Path co-rank (Odeh et al., cited in Section
//    "Related Research").  For merged output position d of runs A and B, the
//    split a(d) is the number of A elements among the first d outputs; with
//    ties taken from A it is the first a in [max(0, d-|B|), min(d, |A|)]
//    with B[d-1-a] < A[a], found by binary search.
//  * Merge pass (one round of the merge tree): each block produces W
//    consecutive outputs.  Its input windows A[a(d0):a(d1)) and
//    B[d0-a(d0):d1-a(d1)) are staged in shared memory with coalesced loads,
//    every thread merges IPT outputs from its own co-rank, and the block
//    writes its W outputs back with coalesced stores.
#pragma once

#include <cstddef>
#include <cstdint>

namespace msort {

// ---------------------------------------------------------------------------
// Items of a tile: the key alone, or (key, position in tile) for pairs.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ K key_max();
template <>
__device__ __forceinline__ uint32_t key_max<uint32_t>() { return 0xFFFFFFFFu; }
template <>
__device__ __forceinline__ uint64_t key_max<uint64_t>() { return ~0ull; }

struct KeyPos64 {
    uint64_t k;
    uint32_t p;
};

template <class K, bool PAIRS>
struct TileItem;

template <class K>
struct TileItem<K, false> {
    using T = K;
    static __device__ __forceinline__ T make(K k, uint32_t) { return k; }
    static __device__ __forceinline__ K key(T t) { return t; }
    static __device__ __forceinline__ uint32_t pos(T) { return 0; }
    static __device__ __forceinline__ bool less(T a, T b) { return a < b; }
    static __device__ __forceinline__ T lo(T a, T b) { return a < b ? a : b; }
    static __device__ __forceinline__ T hi(T a, T b) { return a < b ? b : a; }
    static __device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

// 32-bit key and 32-bit tile position packed as (key << 32 | pos).
template <>
struct TileItem<uint32_t, true> {
    using T = uint64_t;
    static __device__ __forceinline__ T make(uint32_t k, uint32_t p) { return ((uint64_t)k << 32) | p; }
    static __device__ __forceinline__ uint32_t key(T t) { return (uint32_t)(t >> 32); }
    static __device__ __forceinline__ uint32_t pos(T t) { return (uint32_t)t; }
    static __device__ __forceinline__ bool less(T a, T b) { return a < b; }
    static __device__ __forceinline__ T lo(T a, T b) { return a < b ? a : b; }
    static __device__ __forceinline__ T hi(T a, T b) { return a < b ? b : a; }
    static __device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

template <>
struct TileItem<uint64_t, true> {
    using T = KeyPos64;
    static __device__ __forceinline__ T make(uint64_t k, uint32_t p) { return KeyPos64{k, p}; }
    static __device__ __forceinline__ uint64_t key(T t) { return t.k; }
    static __device__ __forceinline__ uint32_t pos(T t) { return t.p; }
    static __device__ __forceinline__ bool less(T a, T b) { return a.k < b.k || (a.k == b.k && a.p < b.p); }
    static __device__ __forceinline__ T lo(T a, T b) { return less(b, a) ? b : a; }
    static __device__ __forceinline__ T hi(T a, T b) { return less(b, a) ? a : b; }
    static __device__ __forceinline__ T shfl_xor(T v, int m) {
        return KeyPos64{__shfl_xor_sync(0xffffffffu, v.k, m), __shfl_xor_sync(0xffffffffu, v.p, m)};
    }
};

// Shared-memory index with one pad element per 128-byte row, so that the
// blocked (thread-major) and striped (element-major) access patterns of a
// warp fall in distinct banks.
template <class T>
__device__ __forceinline__ int spad(int i) {
    constexpr int ROW = 128 / (int)sizeof(T) > 0 ? 128 / (int)sizeof(T) : 1;
    return i + i / ROW;
}
template <class T>
__host__ __device__ constexpr int spad_size(int n) {
    return n + n / (128 / (int)sizeof(T) > 0 ? 128 / (int)sizeof(T) : 1) + 1;
}

// ---------------------------------------------------------------------------
// Warp-level bitonic sort of 32 * IPT items, blocked layout:
// lane l holds positions l * IPT + i, i in [0, IPT).
// ---------------------------------------------------------------------------
template <class TI, int IPT>
__device__ __forceinline__ void warp_bitonic_sort(typename TI::T (&r)[IPT], int lane) {
    using Item = typename TI::T;
    static_assert((IPT & (IPT - 1)) == 0, "IPT must be a power of two");
#pragma unroll
    for (int k = 2; k <= 32 * IPT; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= IPT) {
                // Partner lives in lane ^ (j / IPT), same register.
                const int m = j / IPT;
                const bool asc = ((lane * IPT) & k) == 0;
                const bool lower = (lane & m) == 0;
                const bool keep_lo = (asc == lower);
#pragma unroll
                for (int i = 0; i < IPT; ++i) {
                    Item p = TI::shfl_xor(r[i], m);
                    r[i] = keep_lo ? TI::lo(r[i], p) : TI::hi(r[i], p);
                }
            } else {
                // Partner is register i ^ j of the same thread.
#pragma unroll
                for (int i = 0; i < IPT; ++i) {
                    if ((i & j) == 0) {
                        const bool asc = (((lane * IPT) + i) & k) == 0;
                        Item x = r[i], y = r[i | j];
                        Item l = TI::lo(x, y), h = TI::hi(x, y);
                        r[i] = asc ? l : h;
                        r[i | j] = asc ? h : l;
                    }
                }
            }
        }
    }
}

// One shared-memory merge round inside a tile: runs of length R (power of
// two) at [2gR, 2gR+R) and [2gR+R, 2gR+2R) merge into 2R; thread t produces
// outputs [t*IPT, t*IPT+IPT) into registers.
template <class TI, int IPT>
__device__ __forceinline__ void smem_merge_round(const typename TI::T* s, int R, int t,
                                                 typename TI::T (&r)[IPT]) {
    using Item = typename TI::T;
    const int p0 = t * IPT;
    const int pb = p0 & ~(2 * R - 1);
    const int diag = p0 - pb;
    int lo = diag > R ? diag - R : 0;
    int hi = diag < R ? diag : R;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!TI::less(s[spad<Item>(pb + R + diag - 1 - mid)], s[spad<Item>(pb + mid)]))
            lo = mid + 1;
        else
            hi = mid;
    }
    int ai = pb + lo, bi = pb + R + diag - lo;
    const int aend = pb + R, bend = pb + 2 * R;
    Item av = s[spad<Item>(ai < aend ? ai : aend - 1)];
    Item bv = s[spad<Item>(bi < bend ? bi : bend - 1)];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_a = (bi >= bend) || (ai < aend && !TI::less(bv, av));
        r[i] = take_a ? av : bv;
        if (take_a) {
            ++ai;
            if (ai < aend) av = s[spad<Item>(ai)];
        } else {
            ++bi;
            if (bi < bend) bv = s[spad<Item>(bi)];
        }
    }
}

template <class K>
__device__ __forceinline__ bool aligned16(const K* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// ---------------------------------------------------------------------------
// Tile sort: block b sorts kin[b*T, min((b+1)*T, n)) into kout at the same
// place.  kin may equal kout (each block reads its whole tile first).
// Dynamic shared memory: spad_size<Item>(T) items, then T uint32 values.
// ---------------------------------------------------------------------------
template <class K, bool PAIRS, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
k_tile_sort(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n) {
    using TI = TileItem<K, PAIRS>;
    using Item = typename TI::T;
    constexpr int T = THREADS * IPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Item* s = reinterpret_cast<Item*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(Item) * spad_size<Item>(T));

    const size_t base = (size_t)blockIdx.x * T;
    const int valid = (int)((n - base) < (size_t)T ? (n - base) : (size_t)T);
    const int t = threadIdx.x, lane = t & 31;
    const K* src = kin + base;

    Item r[IPT];
    constexpr int PER = 16 / (int)sizeof(K);
    if (valid == T && aligned16(src)) {
        K k[IPT];
#pragma unroll
        for (int q = 0; q < IPT / PER; ++q) {
            uint4 v = reinterpret_cast<const uint4*>(src + t * IPT)[q];
            const K* pv = reinterpret_cast<const K*>(&v);
#pragma unroll
            for (int e = 0; e < PER; ++e) k[q * PER + e] = pv[e];
        }
#pragma unroll
        for (int i = 0; i < IPT; ++i) r[i] = TI::make(k[i], (uint32_t)(t * IPT + i));
    } else {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int p = t * IPT + i;
            r[i] = TI::make(p < valid ? src[p] : key_max<K>(), (uint32_t)p);
        }
    }
    if (PAIRS) {
        for (int p = t; p < valid; p += THREADS) sv[p] = vin[base + p];
    }

    warp_bitonic_sort<TI, IPT>(r, lane);

    constexpr int R0 = 32 * IPT;
    if (T > R0) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) s[spad<Item>(t * IPT + i)] = r[i];
        __syncthreads();
        for (int R = R0; R < T; R *= 2) {
            smem_merge_round<TI, IPT>(s, R, t, r);
            if (2 * R < T) {
                __syncthreads();
#pragma unroll
                for (int i = 0; i < IPT; ++i) s[spad<Item>(t * IPT + i)] = r[i];
                __syncthreads();
            }
        }
    }
    if (PAIRS) __syncthreads();

    K* dst = kout + base;
    if (valid == T && aligned16(dst)) {
#pragma unroll
        for (int q = 0; q < IPT / PER; ++q) {
            uint4 v;
            K* pv = reinterpret_cast<K*>(&v);
#pragma unroll
            for (int e = 0; e < PER; ++e) pv[e] = TI::key(r[q * PER + e]);
            reinterpret_cast<uint4*>(dst + t * IPT)[q] = v;
        }
    } else {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int p = t * IPT + i;
            if (p < valid) dst[p] = TI::key(r[i]);
        }
    }
    if (PAIRS) {
        uint32_t* vd = vout + base;
        if (valid == T && aligned16(vd)) {
#pragma unroll
            for (int q = 0; q < IPT / 4; ++q) {
                uint4 v;
                v.x = sv[TI::pos(r[4 * q + 0])];
                v.y = sv[TI::pos(r[4 * q + 1])];
                v.z = sv[TI::pos(r[4 * q + 2])];
                v.w = sv[TI::pos(r[4 * q + 3])];
                reinterpret_cast<uint4*>(vd + t * IPT)[q] = v;
            }
        } else {
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                const int p = t * IPT + i;
                if (p < valid) vd[p] = sv[TI::pos(r[i])];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Geometry of one merge pass: runs of length L, output blocks of W (W
// divides 2L, so a block never straddles two merge pairs).
// ---------------------------------------------------------------------------
struct PassGeom {
    size_t pb;    // start of the merge pair
    size_t alen;  // |A|
    size_t blen;  // |B| (0 when the last run has no partner)
};

__device__ __forceinline__ PassGeom pass_geom(size_t out0, size_t n, size_t L) {
    PassGeom g;
    g.pb = (out0 / (2 * L)) * (2 * L);
    const size_t rest = n - g.pb;
    g.alen = rest < L ? rest : L;
    const size_t rest2 = rest - g.alen;
    g.blen = rest2 < L ? rest2 : L;
    return g;
}

// Stable co-rank by binary search over global memory.
template <class K>
__device__ __forceinline__ size_t corank_search(const K* A, size_t alen, const K* B, size_t blen, size_t d) {
    size_t lo = d > blen ? d - blen : 0;
    size_t hi = d < alen ? d : alen;
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - 1 - mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// splits[c] = a(d) at the first output of block c, relative to its pair.
template <class K>
__global__ void k_partition(const K* __restrict__ src, size_t n, size_t L, size_t W, size_t nblocks,
                            unsigned long long* __restrict__ splits) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nblocks) return;
    const size_t out0 = c * W;
    const PassGeom g = pass_geom(out0, n, L);
    const K* A = src + g.pb;
    splits[c] = corank_search(A, g.alen, A + g.alen, g.blen, out0 - g.pb);
}

// ---------------------------------------------------------------------------
// Merge pass: block c writes dst[c*W, min((c+1)*W, pair end)).
// Dynamic shared memory: spad_size<K>(W) keys, then spad_size<uint32>(W)
// values for pairs.
// ---------------------------------------------------------------------------
template <class K, bool PAIRS, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
k_merge_pass(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
             uint32_t* __restrict__ vdst, size_t n, size_t L, const unsigned long long* __restrict__ splits) {
    constexpr int W = THREADS * IPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * spad_size<K>(W));

    const int t = threadIdx.x;
    const size_t c = blockIdx.x;
    const size_t out0 = c * W;
    const PassGeom g = pass_geom(out0, n, L);
    const size_t d0 = out0 - g.pb;
    const size_t dend = g.alen + g.blen;
    const size_t d1 = (d0 + W < dend) ? d0 + W : dend;
    const size_t a0 = splits[c];
    const size_t a1 = (d1 == dend) ? g.alen : (size_t)splits[c + 1];
    const int nA = (int)(a1 - a0);
    const int total = (int)(d1 - d0);
    const K* A = src + g.pb + a0;
    const K* B = src + g.pb + g.alen + (d0 - a0);

    for (int i = t; i < total; i += THREADS) sk[spad<K>(i)] = i < nA ? A[i] : B[i - nA];
    if (PAIRS) {
        const uint32_t* VA = vsrc + g.pb + a0;
        const uint32_t* VB = vsrc + g.pb + g.alen + (d0 - a0);
        for (int i = t; i < total; i += THREADS) sv[spad<uint32_t>(i)] = i < nA ? VA[i] : VB[i - nA];
    }
    __syncthreads();

    // Co-rank of this thread's first output inside the staged window.
    const int diag = t * IPT < total ? t * IPT : total;
    const int nB = total - nA;
    int lo = diag > nB ? diag - nB : 0;
    int hi = diag < nA ? diag : nA;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sk[spad<K>(mid)] <= sk[spad<K>(nA + diag - 1 - mid)])
            lo = mid + 1;
        else
            hi = mid;
    }
    int ai = lo, bi = nA + diag - lo;
    K av = sk[spad<K>(ai < nA ? ai : 0)];
    K bv = sk[spad<K>(bi < total ? bi : 0)];
    K ok[IPT];
    uint32_t ov[PAIRS ? IPT : 1];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_a = (bi >= total) || (ai < nA && av <= bv);
        ok[i] = take_a ? av : bv;
        if (PAIRS) {
            // past the block's last output both runs are exhausted; clamp the
            // (unused) gather index into the staged window
            const int from = take_a ? ai : bi;
            ov[i] = sv[spad<uint32_t>(from < total ? from : total - 1)];
        }
        if (take_a) {
            ++ai;
            if (ai < nA) av = sk[spad<K>(ai)];
        } else {
            ++bi;
            if (bi < total) bv = sk[spad<K>(bi)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int p = t * IPT + i;
        if (p < total) {
            sk[spad<K>(p)] = ok[i];
            if (PAIRS) sv[spad<uint32_t>(p)] = ov[i];
        }
    }
    __syncthreads();
    K* D = dst + out0;
    for (int i = t; i < total; i += THREADS) D[i] = sk[spad<K>(i)];
    if (PAIRS) {
        uint32_t* VD = vdst + out0;
        for (int i = t; i < total; i += THREADS) VD[i] = sv[spad<uint32_t>(i)];
    }
}

}  // namespace msort
