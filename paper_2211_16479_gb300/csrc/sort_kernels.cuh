// Device code of the merge sort: tile sort, co-rank partition, merge pass.
//
// The method (arXiv 2211.16479): sort fixed-size chunks independently
// (Section "Multiprocessing Merge Sort", Figs. 6-7), then merge sorted runs
// pairwise, one round at a time, until a single run is left (Section "MPI
// Merge Sort", Figs. 16-17).  merge() itself is left undefined in the paper; it
// is read here as the stable two-way merge that takes from the left run while
// left <= right.
//
// GPU mapping:
//  * Tile sort (a "chunk" of the multiprocessing design): one thread block
//    sorts T = THREADS * IPT keys.  Each thread sorts IPT keys in registers
//    with a Batcher odd-even merge network, then log2(THREADS) merge-path
//    rounds in shared memory join the per-thread runs.  Key-value tiles
//    compare (key, tile position), which makes the network stable.
//  * Partition: the Merge Path co-rank (Odeh et al., cited in Section
//    "Related Research").  For merged output position d of runs A and B, the
//    split a(d) is the number of A elements among the first d outputs; with
//    ties taken from A it is the first a in [max(0, d-|B|), min(d, |A|)]
//    with B[d-1-a] < A[a], found by binary search.
//  * Merge pass (one round of the merge tree): each block produces W
//    consecutive outputs.  Its windows A[a(d0):a(d1)) and
//    B[d0-a(d0):d1-a(d1)) arrive in shared memory by 1-D bulk TMA copies;
//    each thread merges IPT outputs from its own co-rank; the block's outputs
//    leave by one bulk TMA store.
//
// IPT is odd (17 or 33): consecutive threads then start their merges at
// shared-memory words that differ by an odd stride, which spreads a warp's
// reads over the 32 banks without any index padding arithmetic.  Tiles and
// merge blocks are therefore THREADS * IPT keys (e.g. 256 * 33 = 8448); all
// run lengths are that times a power of two, so a merge block never
// straddles two merge pairs.
#pragma once

#include <cstddef>
#include <cstdint>
#include <utility>

#include "ptx.cuh"

namespace msort {

// Device status bits (a kernel that gives up a bounded wait sets one).
constexpr unsigned int kStatusTimeout = 1u;
// About one second at GB300 clocks.
constexpr long long kWaitLimitCycles = 2000000000ll;

// ---------------------------------------------------------------------------
// Order-preserving key transforms.  Signed and floating-point keys are
// sorted as unsigned words: xf 1 flips the sign bit (two's complement order
// becomes unsigned order); xf 2 maps IEEE 754 bit patterns to unsigned
// words in totalOrder (non-negative patterns get the sign bit set, negative
// ones are complemented, so larger magnitudes of negative numbers come
// first).  The tile sort applies the forward map as it reads its input and
// the last merge round applies the inverse as it writes the output.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ K xf_forward(K k, int xf) {
    constexpr K sign = K(1) << (8 * sizeof(K) - 1);
    if (xf == 1) return k ^ sign;
    if (xf == 2) return (k & sign) ? K(~k) : K(k ^ sign);
    return k;
}
template <class K>
__device__ __forceinline__ K xf_inverse(K u, int xf) {
    constexpr K sign = K(1) << (8 * sizeof(K) - 1);
    if (xf == 1) return u ^ sign;
    if (xf == 2) return (u & sign) ? K(u ^ sign) : K(~u);
    return u;
}

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
};

// ---------------------------------------------------------------------------
// In-register sort of one thread's N items: Batcher's odd-even merge sort
// network (K. E. Batcher, "Sorting networks and their applications", 1968),
// all comparators ascending.  For N not a power of two this is the network
// of the next power of two with every comparator that touches an index >= N
// removed (those positions would hold +infinity and never move).  The
// comparator list is built at compile time and applied by a fold
// expression, so every register index is a constant.
// ---------------------------------------------------------------------------
template <int N>
struct OddEvenNet {
    struct Pairs {
        unsigned short a[N * N], b[N * N];
        int count;
    };
    static constexpr Pairs build() {
        Pairs r{};
        r.count = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < N; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                            r.a[r.count] = (unsigned short)(i + j);
                            r.b[r.count] = (unsigned short)(i + j + k);
                            ++r.count;
                        }
        return r;
    }
    static constexpr Pairs net = build();
};

template <class TI, int N, int C>
__device__ __forceinline__ void net_cas(typename TI::T (&r)[N]) {
    constexpr int a = OddEvenNet<N>::net.a[C];
    constexpr int b = OddEvenNet<N>::net.b[C];
    const typename TI::T x = r[a], y = r[b];
    r[a] = TI::lo(x, y);
    r[b] = TI::hi(x, y);
}

template <class TI, int N, int... C>
__device__ __forceinline__ void net_apply(typename TI::T (&r)[N], std::integer_sequence<int, C...>) {
    (net_cas<TI, N, C>(r), ...);
}

template <class TI, int N>
__device__ __forceinline__ void thread_sort(typename TI::T (&r)[N]) {
    net_apply<TI, N>(r, std::make_integer_sequence<int, OddEvenNet<N>::net.count>{});
}

// Byte-offset shared-memory access (keeps the merge loops on 32-bit
// offsets: one add per step, no index scaling).
template <class T>
__device__ __forceinline__ T sld(const unsigned char* base, int off) {
    return *reinterpret_cast<const T*>(base + off);
}

// Store a thread's IPT sorted items (tile positions t*IPT ..) for a merge
// round whose runs have length IPT << lg.  Runs are kept in "bitonic"
// layout: the right-hand run of every merge pair (odd run index) is stored
// reversed.  With the right run reversed, a merge that walks the left run
// forwards and the right run backwards never needs a bounds check: past the
// end of either run it meets the other run's largest element, which is at
// least every element still to come (R. Sedgewick's merge without
// sentinels, "Algorithms", 2nd ed., Ch. 12).  Each merge pair is followed by
// one unused slot, so pairs start 2R + 1 words apart (an odd stride) and the
// threads of different pairs hit different banks.
template <class Item, int IPT>
__device__ __forceinline__ void store_bitonic(Item* s, int t, int lg, const Item (&r)[IPT]) {
    const int p0 = t * IPT;
    const bool rev = (t >> lg) & 1;
    const int run = IPT << lg;
    const int qb = (t >> lg) * run;
    const int start = (rev ? qb + run - 1 - (p0 - qb) : p0) + (t >> (lg + 1));
    const int step = rev ? -1 : 1;
#pragma unroll
    for (int i = 0; i < IPT; ++i) s[start + i * step] = r[i];
}

// Shared-memory items a tile sort of T items with THREADS threads needs.
__host__ __device__ constexpr int tile_slots(int T, int THREADS) { return T + THREADS / 2 + 2; }

// One shared-memory merge round inside a tile: pair g holds the run of
// length R = IPT << lg at [g(2R+1), g(2R+1) + R) (ascending) followed by its
// partner (stored descending); they merge into 2R outputs, of which thread t
// produces [t*IPT, t*IPT + IPT) into registers.  Ties go to the left run.
// One shared load per output: both run heads stay in registers and only the
// consumed side is reloaded.
template <class TI, int IPT>
__device__ __forceinline__ void smem_merge_round(const unsigned char* s, int lg, int t, typename TI::T (&r)[IPT]) {
    using Item = typename TI::T;
    constexpr int SZ = (int)sizeof(Item);
    const int R = IPT << lg;
    const int g = t >> (lg + 1);
    const int base = g * (2 * R + 1);
    const int diag = (t & ((2 << lg) - 1)) * IPT;
    const int A0 = base * SZ;
    const int BE = (base + 2 * R - 1) * SZ;  // B[k] lives at BE - k*SZ
    int lo = diag > R ? diag - R : 0;
    int hi = diag < R ? diag : R;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!TI::less(sld<Item>(s, BE - (diag - 1 - mid) * SZ), sld<Item>(s, A0 + mid * SZ)))
            lo = mid + 1;
        else
            hi = mid;
    }
    int io = A0 + lo * SZ, jo = BE - (diag - lo) * SZ;
    Item av = sld<Item>(s, io), bv = sld<Item>(s, jo);
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool tb = TI::less(bv, av);
        r[i] = tb ? bv : av;
        io += tb ? 0 : SZ;
        jo -= tb ? SZ : 0;
        if (i + 1 < IPT) {
            const Item nx = sld<Item>(s, tb ? jo : io);
            av = tb ? av : nx;
            bv = tb ? nx : bv;
        }
    }
}

template <class K>
__device__ __forceinline__ bool aligned16(const K* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// ---------------------------------------------------------------------------
// Key-value tile sort for 64-bit keys: keys and values live in separate
// shared arrays (12 bytes per element instead of 16-byte (key, position)
// items).  The per-thread network compares (key, original register index),
// which makes it stable; the merge rounds keep ties in the left run, which
// keeps them stable; so the values can ride along and no position gather is
// needed at the end.
// ---------------------------------------------------------------------------
template <class K, int N, int C>
__device__ __forceinline__ void kv_cas(K (&k)[N], uint32_t (&v)[N], int (&tag)[N]) {
    constexpr int a = OddEvenNet<N>::net.a[C];
    constexpr int b = OddEvenNet<N>::net.b[C];
    const bool sw = k[b] < k[a] || (k[b] == k[a] && tag[b] < tag[a]);
    const K ka = k[a], kb = k[b];
    const uint32_t va = v[a], vb = v[b];
    const int ta = tag[a], tb = tag[b];
    k[a] = sw ? kb : ka;
    k[b] = sw ? ka : kb;
    v[a] = sw ? vb : va;
    v[b] = sw ? va : vb;
    tag[a] = sw ? tb : ta;
    tag[b] = sw ? ta : tb;
}

template <class K, int N, int... C>
__device__ __forceinline__ void kv_net(K (&k)[N], uint32_t (&v)[N], int (&tag)[N], std::integer_sequence<int, C...>) {
    (kv_cas<K, N, C>(k, v, tag), ...);
}

// Keys in bitonic layout (see store_bitonic), values at the same slots.
template <class K, int IPT>
__device__ __forceinline__ void kv_store_bitonic(K* sk, uint32_t* sv, int t, int lg, const K (&k)[IPT],
                                                 const uint32_t (&v)[IPT]) {
    const int p0 = t * IPT;
    const bool rev = (t >> lg) & 1;
    const int run = IPT << lg;
    const int qb = (t >> lg) * run;
    const int start = (rev ? qb + run - 1 - (p0 - qb) : p0) + (t >> (lg + 1));
    const int step = rev ? -1 : 1;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        sk[start + i * step] = k[i];
        sv[start + i * step] = v[i];
    }
}

// The merge round of smem_merge_round on separate key and value arrays.
// Unlike the key-only and (key, position) rounds, equal keys here carry
// different values, so an exhausted run must not be "overrun" into its
// partner's largest element: the run bounds decide the side once a run is
// used up (A occupies [base, base + R), the reversed B [base + R, base + 2R)).
template <class K, int IPT>
__device__ __forceinline__ void kv_merge_round(const K* sk, const uint32_t* sv, int lg, int t, K (&k)[IPT],
                                               uint32_t (&v)[IPT]) {
    const int R = IPT << lg;
    const int g = t >> (lg + 1);
    const int base = g * (2 * R + 1);
    const int diag = (t & ((2 << lg) - 1)) * IPT;
    const int BE = base + 2 * R - 1;
    int lo = diag > R ? diag - R : 0;
    int hi = diag < R ? diag : R;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(sk[BE - (diag - 1 - mid)] < sk[base + mid]))
            lo = mid + 1;
        else
            hi = mid;
    }
    int io = base + lo, jo = BE - (diag - lo);
    const int mid_end = base + R;  // first slot of B; A is exhausted at it, B below it
    K av = sk[io], bv = sk[jo];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool tb = io >= mid_end || (jo >= mid_end && bv < av);
        k[i] = tb ? bv : av;
        v[i] = sv[tb ? jo : io];
        io += tb ? 0 : 1;
        jo -= tb ? 1 : 0;
        if (i + 1 < IPT) {
            const K nx = sk[tb ? jo : io];
            av = tb ? av : nx;
            bv = tb ? nx : bv;
        }
    }
}

template <class K, int THREADS, int IPT>
__device__ __forceinline__ bool tile_sort_block_kv(const K* src, const uint32_t* vin, K* dst, uint32_t* vout,
                                                   int valid, unsigned char* smem_raw, int xf_in, int xf_out) {
    constexpr int T = THREADS * IPT;
    constexpr int SLOTS = tile_slots(T, THREADS);
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * SLOTS);
    const int t = threadIdx.x;
    __syncthreads();  // the previous user of this shared memory is done
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int p = i * THREADS + t;
        const bool in = p < valid;
        sk[p] = in ? xf_forward(src[p], xf_in) : key_max<K>();
        sv[p] = in ? vin[p] : 0u;
    }
    __syncthreads();
    K k[IPT];
    uint32_t v[IPT];
    int tag[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        k[i] = sk[t * IPT + i];
        v[i] = sv[t * IPT + i];
        tag[i] = i;
    }
    kv_net<K, IPT>(k, v, tag, std::make_integer_sequence<int, OddEvenNet<IPT>::net.count>{});
    int lg = 0;
    for (int R = IPT; R < T; R *= 2, ++lg) {
        __syncthreads();
        kv_store_bitonic<K, IPT>(sk, sv, t, lg, k, v);
        __syncthreads();
        kv_merge_round<K, IPT>(sk, sv, lg, t, k, v);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        sk[t * IPT + i] = k[i];
        sv[t * IPT + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int p = i * THREADS + t;
        if (p < valid) {
            dst[p] = xf_inverse(sk[p], xf_out);
            vout[p] = sv[p];
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Tile sort of one block: sorts src[0, valid) (valid <= T = THREADS * IPT)
// into dst[0, valid); src may equal dst.  `bar` is an initialised mbarrier
// of this block and `phase` its next parity (flipped on every bulk load).
// Returns false if a bounded wait gave up (status records it).
// Shared memory: tile_slots(T, THREADS) items, then T uint32 values for
// pairs.  Steps: bulk TMA load (or coalesced loads), per-thread network,
// merge rounds in bitonic layout, bulk TMA store (or coalesced stores).
// ---------------------------------------------------------------------------
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__device__ __forceinline__ bool tile_sort_block(const K* src, const uint32_t* vin, K* dst, uint32_t* vout, int valid,
                                                unsigned char* smem_raw, uint64_t* bar, uint32_t& phase,
                                                unsigned int* status, int xf_in, int xf_out) {
    if constexpr (!XF) {  // the instance without key transforms: their code folds away
        xf_in = 0;
        xf_out = 0;
    }
    if constexpr (PAIRS && sizeof(K) == 8) {
        return tile_sort_block_kv<K, THREADS, IPT>(src, vin, dst, vout, valid, smem_raw, xf_in, xf_out);
    }
    using TI = TileItem<K, PAIRS>;
    using Item = typename TI::T;
    constexpr int T = THREADS * IPT;
    Item* s = reinterpret_cast<Item*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(Item) * tile_slots(T, THREADS));
    const int t = threadIdx.x;
    __syncthreads();  // the previous user of this shared memory is done

    // Full, aligned keys-only tiles arrive by one bulk copy.
    const bool bulk = !PAIRS && valid == T && aligned16(src);
    if (bulk) {
        if (t == 0) {
            mbar_arrive_expect_tx(bar, (uint32_t)(T * sizeof(K)));
            tma_load_1d(s, src, (uint32_t)(T * sizeof(K)), bar);
        }
        __syncthreads();
        const bool ok = mbar_wait_bounded(bar, phase, kWaitLimitCycles);
        phase ^= 1u;
        if (!ok) {
            if (t == 0) atomicOr(status, kStatusTimeout);
            mbar_wait_bounded(bar, phase ^ 1u, kWaitLimitCycles);
            return false;
        }
    } else {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int p = i * THREADS + t;
            s[p] = TI::make(p < valid ? xf_forward(src[p], xf_in) : key_max<K>(), (uint32_t)p);
        }
        if (PAIRS) {
            for (int p = t; p < valid; p += THREADS) sv[p] = vin[p];
        }
        __syncthreads();
    }

    Item r[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) r[i] = s[t * IPT + i];
    if (bulk && xf_in) {  // the bulk copy brought the raw keys (keys-only tiles)
#pragma unroll
        for (int i = 0; i < IPT; ++i) r[i] = TI::make(xf_forward(TI::key(r[i]), xf_in), TI::pos(r[i]));
    }
    thread_sort<TI, IPT>(r);

    const unsigned char* sb = smem_raw;
    int lg = 0;
    for (int R = IPT; R < T; R *= 2, ++lg) {
        __syncthreads();
        store_bitonic<Item, IPT>(s, t, lg, r);
        __syncthreads();
        smem_merge_round<TI, IPT>(sb, lg, t, r);
    }
    __syncthreads();

    if (!PAIRS) {
        K* sk = reinterpret_cast<K*>(smem_raw);
#pragma unroll
        for (int i = 0; i < IPT; ++i) sk[t * IPT + i] = xf_inverse(TI::key(r[i]), xf_out);
        if (valid == T && aligned16(dst)) {
            fence_proxy_async_smem();
            __syncthreads();
            if (t == 0) {
                tma_store_1d(dst, sk, (uint32_t)(T * sizeof(K)));
                tma_store_commit();
                tma_store_wait_read();
            }
        } else {
            __syncthreads();
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                const int p = i * THREADS + t;
                if (p < valid) dst[p] = sk[p];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < IPT; ++i) s[t * IPT + i] = r[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int p = i * THREADS + t;
            if (p < valid) {
                const Item it = s[p];
                dst[p] = xf_inverse(TI::key(it), xf_out);
                vout[p] = sv[TI::pos(it)];
            }
        }
    }
    return true;
}

template <class K, bool PAIRS, int THREADS>
__host__ __device__ constexpr size_t tile_block_smem(int T) {
    return (PAIRS && sizeof(K) == 8) ? (8u + 4u) * (size_t)tile_slots(T, THREADS)
                                     : sizeof(typename TileItem<K, PAIRS>::T) * (size_t)tile_slots(T, THREADS) +
                                           (PAIRS ? 4u * T : 0u);
}

// Tile sort kernel: block b sorts kin[b*T, min((b+1)*T, n)) in place into
// kout.  kin may equal kout (each block reads its whole tile first).  XF:
// the instance that applies / undoes key transforms (signed and float keys).
// The 64-bit key-value 256 x 17 tile is bounded to three blocks per SM (80
// registers, a 28-byte spill) instead of the two its 98 registers allow:
// on 2^27 pairs its tile sort takes 2.55 instead of 2.83 ms.  Four blocks
// (64 registers) spilled 336 bytes and gained nothing.
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS, (sizeof(K) == 8 && PAIRS && THREADS == 256 && IPT == 17) ? 3 : 0)
k_tile_sort(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n, unsigned int* status, int xf_in,
            int xf_out) {
    constexpr int T = THREADS * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    const size_t base = (size_t)blockIdx.x * T;
    const int valid = (int)((n - base) < (size_t)T ? (n - base) : (size_t)T);
    uint32_t phase = 0;
    tile_sort_block<K, PAIRS, THREADS, IPT, XF>(kin + base, PAIRS ? vin + base : nullptr, kout + base,
                                                PAIRS ? vout + base : nullptr, valid, smem_raw, &bar, phase, status,
                                                xf_in, xf_out);
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

// Stable co-rank by binary search over global memory: the first a in
// [max(0, d-|B|), min(d, |A|)] with B[d-1-a] < A[a].  (An 8-ary variant with
// seven independent probes per step measured slower on GB300: the pass's
// searches are limited by scattered-load throughput, not by the length of
// one search's dependent chain.)
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

// Placement of one input window in shared memory: its first element sits at
// element offset `off` of the region; elements [head, head + nbulk) move by a
// bulk copy (16-byte aligned on both sides), the rest by scalar loads.
struct Window {
    int off;    // element offset of window element 0 in the shared array
    int head;   // elements before the bulk part
    int nbulk;  // elements in the bulk part (multiple of 16 / element size)
    int end;    // first element offset after the window and its slack
};

template <class E>
__device__ __forceinline__ Window place_window(const E* g, int n, int region, int slack) {
    constexpr int EPC = 16 / (int)sizeof(E);
    Window w;
    int head = (int)(((16u - (reinterpret_cast<uintptr_t>(g) & 15u)) & 15u) / sizeof(E));
    if (head > n) head = n;
    w.head = head;
    w.nbulk = ((n - head) / EPC) * EPC;
    w.off = region + (EPC - head) % EPC;
    const int e = w.off + n + slack;
    w.end = (e + EPC - 1) / EPC * EPC;
    return w;
}

// Scalar part of a window: the head and tail elements (fewer than 16 bytes
// each) and `slack` copies of `fill` after the window.  Warp w0 moves the
// head and tail, warp w0 + 1 writes the fill.
template <class E>
__device__ __forceinline__ void window_scalars(const E* g, int n, const Window& w, E* s, int warp, int lane, int w0,
                                               int slack, E fill) {
    if (warp == w0) {
        if (lane < w.head) s[w.off + lane] = g[lane];
        const int t0 = w.head + w.nbulk;
        if (lane < n - t0) s[w.off + t0 + lane] = g[t0 + lane];
    } else if (warp == w0 + 1) {
        for (int i = lane; i < slack; i += 32) s[w.off + n + i] = fill;
    }
}

// Shared slots of one merge-pass region (window A, window B, slack and
// alignment), rounded to 16 elements so the next region stays 16-byte
// aligned.
__host__ __device__ constexpr int merge_slots(int W, int IPT, int esize) {
    return (W + 2 * IPT + 6 * (16 / esize) + 8 + 15) / 16 * 16;
}

// ---------------------------------------------------------------------------
// Merge of one output block: D[0, nA + nB) = stable merge of gA[0, nA) and
// gB[0, nB) (nA + nB <= W = THREADS * IPT), values alongside for pairs.
// `bar` is an initialised mbarrier of this block, `phase` its next parity.
// XF: the block undoes the key transform xf_out as it stages its output (a
// separate instance, so the common passes keep their register budget).
// Shared memory: merge_slots(W, IPT, sizeof(K)) keys, then for pairs
// merge_slots(W, IPT, 4) values.  Returns false if a bounded wait gave up
// (after wait_limit cycles; every production caller keeps the default).
// ---------------------------------------------------------------------------
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__device__ __forceinline__ bool merge_block(const K* gA, int nA, const K* gB, int nB, const uint32_t* gvA,
                                            const uint32_t* gvB, K* D, uint32_t* VD, unsigned char* smem_raw,
                                            uint64_t* bar, uint32_t& phase, unsigned int* status, int xf_out,
                                            long long wait_limit = kWaitLimitCycles) {
    constexpr int W = THREADS * IPT;
    constexpr int KS = (int)sizeof(K);
    constexpr int KSLOTS = merge_slots(W, IPT, KS);
    constexpr int VSLOTS = merge_slots(W, IPT, 4);
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + KS * KSLOTS);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int total = nA + nB;
    __syncthreads();  // the previous user of this shared memory is done

    const Window wA = place_window(gA, nA, 0, IPT);
    const Window wB = place_window(gB, nB, wA.end, IPT);
    Window vA{}, vB{};
    if (PAIRS) {
        vA = place_window(gvA, nA, 0, 0);
        vB = place_window(gvB, nB, vA.end, 0);
    }

    if (t == 0) {
        uint32_t bytes = (uint32_t)((wA.nbulk + wB.nbulk) * KS);
        if (PAIRS) bytes += (uint32_t)((vA.nbulk + vB.nbulk) * 4);
        mbar_arrive_expect_tx(bar, bytes);
        if (wA.nbulk) tma_load_1d(sk + wA.off + wA.head, gA + wA.head, (uint32_t)(wA.nbulk * KS), bar);
        if (wB.nbulk) tma_load_1d(sk + wB.off + wB.head, gB + wB.head, (uint32_t)(wB.nbulk * KS), bar);
        if (PAIRS) {
            if (vA.nbulk) tma_load_1d(sv + vA.off + vA.head, gvA + vA.head, (uint32_t)(vA.nbulk * 4), bar);
            if (vB.nbulk) tma_load_1d(sv + vB.off + vB.head, gvB + vB.head, (uint32_t)(vB.nbulk * 4), bar);
        }
    }
    window_scalars(gA, nA, wA, sk, warp, lane, 1, IPT, key_max<K>());
    window_scalars(gB, nB, wB, sk, warp, lane, 3, IPT, key_max<K>());
    if (PAIRS) {
        window_scalars(gvA, nA, vA, sv, warp, lane, 5, 0, 0u);
        window_scalars(gvB, nB, vB, sv, warp, lane, 6, 0, 0u);
    }
    __syncthreads();
    const bool ok_wait = mbar_wait_bounded(bar, phase, wait_limit);
    phase ^= 1u;
    if (!ok_wait) {
        if (t == 0) atomicOr(status, kStatusTimeout);
        mbar_wait_bounded(bar, phase ^ 1u, wait_limit);
        return false;
    }

    // Co-rank of this thread's first output inside the staged windows.
    const unsigned char* sb = smem_raw;
    const int A0 = wA.off * KS, B0 = wB.off * KS;
    const int diag = t * IPT < total ? t * IPT : total;
    int lo = diag > nB ? diag - nB : 0;
    int hi = diag < nA ? diag : nA;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sld<K>(sb, A0 + mid * KS) <= sld<K>(sb, B0 + (diag - 1 - mid) * KS))
            lo = mid + 1;
        else
            hi = mid;
    }
    int ao = A0 + lo * KS, bo = B0 + (diag - lo) * KS;
    K ok[IPT];
    uint32_t ov[PAIRS ? IPT : 1];
    if (!PAIRS) {
        // Both windows are followed by IPT copies of the largest key, so no
        // bounds checks are needed: once a run is exhausted its "next" key
        // is the maximum, and whenever that maximum is taken the remaining
        // keys of the other run are all the maximum too.
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const K av = sld<K>(sb, ao), bv = sld<K>(sb, bo);
            const bool ta = av <= bv;
            ok[i] = ta ? av : bv;
            ao += ta ? KS : 0;
            bo += ta ? 0 : KS;
        }
    } else {
        const int ae = A0 + nA * KS, be = B0 + nB * KS;
        const int vshiftA = vA.off - wA.off, vshiftB = vB.off - wB.off;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const K av = sld<K>(sb, ao), bv = sld<K>(sb, bo);
            const bool ta = ao < ae && (bo >= be || av <= bv);
            ok[i] = ta ? av : bv;
            // value slot: the same element of the window in the value region
            ov[i] = ta ? (uint32_t)(ao / KS + vshiftA) : (uint32_t)(bo / KS + vshiftB);
            ao += ta ? KS : 0;
            bo += ta ? 0 : KS;
        }
#pragma unroll
        for (int i = 0; i < IPT; ++i) ov[i] = sv[ov[i] < (uint32_t)VSLOTS ? ov[i] : 0u];
    }
    __syncthreads();

    // Outputs back to shared memory (thread t at [t*IPT, t*IPT + IPT)),
    // shifted by the destination's element offset within 16 bytes, so that
    // the outputs from D's first 16-byte boundary on sit at a 16-byte
    // boundary of shared memory too: the whole 16-byte units go out with one
    // bulk store per array, the head before the boundary and the tail by
    // plain stores.  (An aligned destination has no shift and no head.)
    const int mine = total - t * IPT;
    const int ks0 = (int)((reinterpret_cast<uintptr_t>(D) & 15) / KS);
    const int vs0 = PAIRS ? (int)((reinterpret_cast<uintptr_t>(VD) & 15) / 4) : 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        if (i < mine) {
            sk[ks0 + t * IPT + i] = XF ? xf_inverse(ok[i], xf_out) : ok[i];
            if (PAIRS) sv[vs0 + t * IPT + i] = ov[i];
        }
    }
    const int khead = ks0 ? 16 / KS - ks0 : 0;                                   // keys before the boundary
    const int kbody = total > khead ? ((total - khead) * KS / 16) * 16 / KS : 0;  // keys by bulk store
    const int vhead = vs0 ? 4 - vs0 : 0;
    const int vbody = PAIRS && total > vhead ? ((total - vhead) * 4 / 16) * 4 : 0;
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
        if (kbody) tma_store_1d(D + khead, sk + ks0 + khead, (uint32_t)(kbody * KS));
        if (PAIRS && vbody) tma_store_1d(VD + vhead, sv + vs0 + vhead, (uint32_t)(vbody * 4));
        tma_store_commit();
    }
    if (t < khead && t < total) D[t] = sk[ks0 + t];
    for (int i = khead + kbody + t; i < total; i += THREADS) D[i] = sk[ks0 + i];
    if (PAIRS) {
        if (t < vhead && t < total) VD[t] = sv[vs0 + t];
        for (int i = vhead + vbody + t; i < total; i += THREADS) VD[i] = sv[vs0 + i];
    }
    if (t == 0) tma_store_wait_read();
    return true;
}

template <class K, bool PAIRS, int THREADS, int IPT>
__host__ __device__ constexpr size_t merge_block_smem() {
    return sizeof(K) * (size_t)merge_slots(THREADS * IPT, IPT, sizeof(K)) +
           (PAIRS ? 4u * merge_slots(THREADS * IPT, IPT, 4) : 0u);
}

// Merge pass kernel: block c = c0 + blockIdx.x writes dst[c*W, min((c+1)*W,
// pair end)) (c0 lets a pass be launched in slices).
template <class K, bool PAIRS, int THREADS, int IPT, bool XF>
__global__ void __launch_bounds__(THREADS, (sizeof(K) == 4 && !PAIRS && IPT == 33) ? 6 : 0)
k_merge_pass(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
             uint32_t* __restrict__ vdst, size_t n, size_t L, const unsigned long long* __restrict__ splits,
             unsigned int* status, size_t c0, int xf_out) {
    constexpr int W = THREADS * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    const size_t c = c0 + blockIdx.x;
    const size_t out0 = c * W;
    const PassGeom g = pass_geom(out0, n, L);
    const size_t d0 = out0 - g.pb;
    const size_t dend = g.alen + g.blen;
    const size_t d1 = (d0 + W < dend) ? d0 + W : dend;
    const size_t a0 = splits[c];
    const size_t a1 = (d1 == dend) ? g.alen : (size_t)splits[c + 1];
    const int nA = (int)(a1 - a0);
    const int nB = (int)(d1 - d0) - nA;
    const size_t oA = g.pb + a0, oB = g.pb + g.alen + (d0 - a0);
    uint32_t phase = 0;
    merge_block<K, PAIRS, THREADS, IPT, XF>(src + oA, nA, src + oB, nB, PAIRS ? vsrc + oA : nullptr,
                                            PAIRS ? vsrc + oB : nullptr, dst + out0, PAIRS ? vdst + out0 : nullptr,
                                            smem_raw, &bar, phase, status, xf_out);
}

// ---------------------------------------------------------------------------
// Merge of two separate sorted arrays (one round of the paper's merge tree
// as a library call): splits over out[0, na + nb), then one merge block per
// W outputs.
// ---------------------------------------------------------------------------
template <class K>
__global__ void k_partition_two(const K* __restrict__ A, size_t na, const K* __restrict__ B, size_t nb, size_t W,
                                size_t nblocks, unsigned long long* __restrict__ splits) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nblocks) return;
    splits[c] = corank_search(A, na, B, nb, c * W);
}

template <class K, bool PAIRS, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
k_merge_two(const K* __restrict__ A, size_t na, const K* __restrict__ B, size_t nb, const uint32_t* __restrict__ va,
            const uint32_t* __restrict__ vb, K* __restrict__ out, uint32_t* __restrict__ vout,
            const unsigned long long* __restrict__ splits, unsigned int* status) {
    constexpr int W = THREADS * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    const size_t c = blockIdx.x;
    const size_t d0 = c * W, dend = na + nb;
    const size_t d1 = d0 + W < dend ? d0 + W : dend;
    const size_t a0 = splits[c];
    const size_t a1 = d1 == dend ? na : (size_t)splits[c + 1];
    const size_t b0 = d0 - a0;
    const int nA = (int)(a1 - a0);
    const int nB = (int)(d1 - d0) - nA;
    uint32_t phase = 0;
    merge_block<K, PAIRS, THREADS, IPT, false>(A + a0, nA, B + b0, nB, PAIRS ? va + a0 : nullptr,
                                               PAIRS ? vb + b0 : nullptr, out + d0, PAIRS ? vout + d0 : nullptr,
                                               smem_raw, &bar, phase, status, 0);
}

}  // namespace msort
