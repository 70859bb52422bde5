// Four-way merge pass: two rounds of the merge tree (Section "MPI Merge
// Sort", Figs. 16-17) per round trip through HBM.  Runs A, B, C, D of length L
// become one run of length 4L equal to merge(merge(A, B), merge(C, D)) with
// equal keys ordered A, B, C, D -- exactly what two stable pairwise rounds
// produce.  The merge passes of the sort run at the copy bandwidth, so
// halving their number is what shortens the sort.
//
// Exact block boundaries without nested searches.  X = merge(A, B) and
// Y = merge(C, D) exist only virtually.  Every G-th element of X and of Y (a
// grid point) gets
//   k_grid4    its co-rank in (A, B) or (C, D) and its key;
//   k_pos4     its exact position in merge(X, Y): its own index plus the
//              number of elements of the other side ordered before it (keys
//              below it from Y, keys not above it from X), found by binary
//              searches that the other side's grid bounds to G elements;
//   k_bracket4 for the first output d of every block, kx(d) = the number of
//              X grid points placed before d (and ky(d) for Y).  The block's
//              share of X then starts in ((kx-1)G, kx G] and its window is
//              cut at grid points, where the (A, B) split is known exactly.
// The merge block loads the four windows (at most W + 4G - 2 keys), merges
// A/B and C/D into shared memory (level 1), and merges the part of X and Y
// it owns into its W outputs (level 2).  Keys only: values take the
// pairwise passes.
#pragma once

#include "sort_kernels.cuh"

namespace msort {

// A kernel found block geometry that contradicts the grid (never expected).
constexpr unsigned int kStatusInternal = 4u;

struct QuadGeom {
    size_t qb;      // first element of the quad
    size_t q;       // quad index
    size_t len[4];  // |A|, |B|, |C|, |D| (the last quad may be short)
};

__device__ __forceinline__ QuadGeom quad_geom(size_t q, size_t n, size_t L) {
    QuadGeom g;
    g.q = q;
    g.qb = q * 4 * L;
    size_t rest = n - g.qb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        g.len[i] = rest < L ? rest : L;
        rest -= g.len[i];
    }
    return g;
}

// Grid layout: quad q owns entries [2Hq, 2H(q+1)) with H = 2L/G; X's grid
// points first, then Y's.  When a warp's 32 consecutive points share one
// side of one quad, lanes 0 and 31 search the whole co-rank range and the
// other lanes search only between those two results (co-ranks are monotone
// in the position), which touches far fewer memory lines than 32 full
// searches; other warps search per lane.
template <class K>
__global__ void k_grid4(const K* __restrict__ src, size_t n, size_t L, size_t G, size_t total,
                        unsigned long long* __restrict__ gco, K* __restrict__ gval) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const size_t H = 2 * L / G;
    const size_t i0 = i - lane;  // first point of the warp (blockDim is a multiple of 32)
    if (i0 >= total) return;     // whole warp out of range
    const size_t ilast = i0 + 31 < total ? i0 + 31 : total - 1;
    const bool uni = (i0 / H) == (ilast / H);
    const size_t ic = i < total ? i : total - 1;
    const size_t q = ic / (2 * H), r = ic - q * 2 * H;
    const int side = r >= H ? 1 : 0;
    const size_t k = side ? r - H : r;
    const QuadGeom g = quad_geom(q, n, L);
    const size_t lp = side ? g.len[2] : g.len[0], lq = side ? g.len[3] : g.len[1];
    const size_t len = lp + lq;
    const K* P = src + g.qb + (side ? g.len[0] + g.len[1] : 0);
    const K* Q = P + lp;
    const size_t pos = k * G < len ? k * G : len;  // clamped (points past the end write nothing)
    size_t a_full = 0;
    if (!uni || lane == 0 || lane == 31) a_full = corank_search(P, lp, Q, lq, pos);
    const size_t a0 = __shfl_sync(0xffffffffu, a_full, 0);
    const size_t a31 = __shfl_sync(0xffffffffu, a_full, 31);
    const size_t p0 = __shfl_sync(0xffffffffu, pos, 0);
    const size_t p31 = __shfl_sync(0xffffffffu, pos, 31);
    size_t a = a_full;
    if (uni && lane != 0 && lane != 31) {
        // a(pos) in [a0, a31] and b(pos) = pos - a(pos) in [p0 - a0, p31 - a31]
        size_t lo = pos > lq ? pos - lq : 0, hi = pos < lp ? pos : lp;
        const size_t b0 = p0 - a0, b31 = p31 - a31;
        if (lo < a0) lo = a0;
        if (pos > b31 && lo < pos - b31) lo = pos - b31;
        if (hi > a31) hi = a31;
        if (hi > pos - b0) hi = pos - b0;
        while (lo < hi) {
            const size_t mid = (lo + hi) >> 1;
            if (P[mid] <= Q[pos - 1 - mid])
                lo = mid + 1;
            else
                hi = mid;
        }
        a = lo;
    }
    if (i >= total || k * G >= len) return;
    const size_t b = pos - a;
    gco[i] = a;
    gval[i] = (a < lp && (b >= lq || P[a] <= Q[b])) ? P[a] : Q[b];
}

// First index in [lo, hi) of a sorted array whose key is not ordered before
// v: keys < v are before it (incl = false), or keys <= v (incl = true).
template <class K>
__device__ __forceinline__ size_t count_before(const K* a, size_t lo, size_t hi, K v, bool incl) {
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        const K w = a[mid];
        if (incl ? w <= v : w < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

template <class K>
__global__ void k_pos4(const K* __restrict__ src, size_t n, size_t L, size_t G, size_t total,
                       const unsigned long long* __restrict__ gco, const K* __restrict__ gval,
                       unsigned long long* __restrict__ gpos) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t H = 2 * L / G;
    const size_t q = i / (2 * H), r = i - q * 2 * H;
    const int side = r >= H ? 1 : 0;
    const size_t k = side ? r - H : r;
    const QuadGeom g = quad_geom(q, n, L);
    const size_t lx = g.len[0] + g.len[1];
    if (k * G >= (side ? g.len[2] + g.len[3] : lx)) return;
    const K v = gval[i];
    // The other side: an X point counts Y keys < v, a Y point X keys <= v.
    const int o = side ^ 1;
    const bool incl = side == 1;
    const K* P = src + g.qb + (o ? lx : 0);
    const size_t lp = g.len[2 * o], lq = g.len[2 * o + 1];
    const size_t no = (lp + lq + G - 1) / G;
    const size_t ob = q * 2 * H + (o ? H : 0);
    // j = other-side grid points ordered before v
    size_t lo = 0, hi = no;
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        const K w = gval[ob + mid];
        if (incl ? w <= v : w < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    const size_t j = lo;
    // Point j-1 is before v, so are its first (j-1)G + 1 elements; point j
    // is not, nor is anything after it: the counts lie between the splits.
    size_t p0 = 0, q0 = 0, p1 = lp, q1 = lq;
    if (j > 0) {
        p0 = gco[ob + j - 1];
        q0 = (j - 1) * G - p0;
    }
    if (j < no) {
        p1 = gco[ob + j];
        q1 = j * G - p1;
    }
    const size_t cp = count_before(P, p0, p1, v, incl);
    const size_t cq = count_before(P + lp, q0, q1, v, incl);
    gpos[i] = k * G + cp + cq;
}

// For block c's first output d and each side (0: X, 1: Y), one record of
// three words: k = the side's grid points placed before d, the split of the
// side's first run at grid point k - 1 (0 if k = 0; where the block's window
// starts) and at grid point k (the first run's length past the last point;
// where the previous block's window ends).  One thread per (block, side).
// (Templated on the key type only so that each key type's translation unit
// owns its copy.)
template <class K>
__global__ void k_bracket4(size_t n, size_t L, size_t G, size_t W, size_t nblocks,
                           const unsigned long long* __restrict__ gpos, const unsigned long long* __restrict__ gco,
                           unsigned long long* __restrict__ brk) {
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2 * nblocks) return;
    const size_t c = j >> 1;
    const int side = (int)(j & 1);
    const size_t out0 = c * W;
    const QuadGeom g = quad_geom(out0 / (4 * L), n, L);
    const size_t d = out0 - g.qb;
    const size_t H = 2 * L / G;
    const size_t len = side ? g.len[2] + g.len[3] : g.len[0] + g.len[1];
    const size_t first = side ? g.len[2] : g.len[0];
    const size_t base = g.q * 2 * H + (side ? H : 0);
    const size_t np = (len + G - 1) / G;
    size_t lo = 0, hi = np;
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        if (gpos[base + mid] < d)
            lo = mid + 1;
        else
            hi = mid;
    }
    brk[3 * j] = lo;
    brk[3 * j + 1] = lo ? gco[base + lo - 1] : 0;
    brk[3 * j + 2] = lo < np ? gco[base + lo] : first;
}

// Shared memory of one four-way merge block, in keys: region 1 holds the
// four input windows (each followed by QMAX + 1 sentinels, plus 16-byte
// alignment) and later the staged output; region 2 holds X and Y (each
// followed by IPT + 1 sentinels).
__host__ __device__ constexpr int merge4_qmax(int THREADS, int W, int G) {
    return ((W + 4 * G + THREADS - 1) / THREADS) | 1;
}
__host__ __device__ constexpr int merge4_r1(int THREADS, int IPT, int GDIV, int esize) {
    return (THREADS * IPT + 4 * (THREADS * IPT / GDIV) +
            4 * (merge4_qmax(THREADS, THREADS * IPT, THREADS * IPT / GDIV) + 1 + 2 * (16 / esize)) + 16 + 15) /
           16 * 16;
}
__host__ __device__ constexpr int merge4_r2(int THREADS, int IPT, int GDIV) {
    return (THREADS * IPT + 4 * (THREADS * IPT / GDIV) + 2 * (IPT + 1) + 8 + 15) / 16 * 16;
}
template <class K, int THREADS, int IPT, int GDIV>
__host__ __device__ constexpr size_t merge4_smem() {
    return sizeof(K) * (size_t)(merge4_r1(THREADS, IPT, GDIV, sizeof(K)) + merge4_r2(THREADS, IPT, GDIV));
}

// Shared-memory store at a byte offset (the merge loops keep 32-bit byte
// offsets from the shared base: one add per step, no index scaling).
template <class T>
__device__ __forceinline__ void sst(unsigned char* base, int off, T v) {
    *reinterpret_cast<T*>(base + off) = v;
}

// Outputs [diag, diag + cnt) of the stable merge of the runs at byte offsets
// a0 (na keys) and b0 (nb keys) of sb, written from byte offset o0 on; both
// runs are followed by at least cnt + 1 copies of the largest key.
template <class K>
__device__ __forceinline__ void merge_run_smem(unsigned char* sb, int a0, int na, int b0, int nb, int diag, int cnt,
                                               int o0) {
    constexpr int KS = (int)sizeof(K);
    int lo = diag > nb ? diag - nb : 0;
    int hi = diag < na ? diag : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sld<K>(sb, a0 + mid * KS) <= sld<K>(sb, b0 + (diag - 1 - mid) * KS))
            lo = mid + 1;
        else
            hi = mid;
    }
    int io = a0 + lo * KS, jo = b0 + (diag - lo) * KS, oo = o0 + diag * KS;
    K av = sld<K>(sb, io), bv = sld<K>(sb, jo);
    auto step = [&]() {
        const bool ta = av <= bv;
        sst<K>(sb, oo, ta ? av : bv);
        oo += KS;
        io += ta ? KS : 0;
        jo += ta ? 0 : KS;
        const K nv = sld<K>(sb, ta ? io : jo);
        av = ta ? nv : av;
        bv = ta ? bv : nv;
    };
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {
        step();
        step();
        step();
        step();
    }
    for (; i < cnt; ++i) step();
}

// Block geometry, computed once by thread 0 and shared.
template <class K>
struct Merge4Geo {
    const K* gw[4];  // window starts in A, B, C, D
    int nw[4];       // window lengths
    int off[4];      // window offsets in region 1
    int e0, e1;      // the block's outputs within merge(X window, Y window)
    int ok;
};

template <class K, int THREADS, int IPT, int GDIV>
__global__ void __launch_bounds__(THREADS)
k_merge4_pass(const K* __restrict__ src, K* __restrict__ dst, size_t n, size_t L,
              const unsigned long long* __restrict__ brk, unsigned int* status) {
    constexpr int W = THREADS * IPT;
    constexpr int G = W / GDIV;
    constexpr int KS = (int)sizeof(K);
    constexpr int QMAX = merge4_qmax(THREADS, W, G);
    constexpr int R1 = merge4_r1(THREADS, IPT, GDIV, KS);
    constexpr int NW = THREADS / 32;
    static_assert(W % GDIV == 0, "the grid step must divide the block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ Merge4Geo<K> geo;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    K* s1 = reinterpret_cast<K*>(smem_raw);
    K* s2 = s1 + R1;
    const size_t out0 = (size_t)blockIdx.x * W;

    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        // ---- block geometry from the grid ----
        const size_t c = blockIdx.x;
        const QuadGeom g = quad_geom(out0 / (4 * L), n, L);
        const size_t lx = g.len[0] + g.len[1], ly = g.len[2] + g.len[3];
        const size_t nx = (lx + G - 1) / G, ny = (ly + G - 1) / G;
        const size_t d0 = out0 - g.qb;
        const size_t dend = lx + ly;
        const size_t d1 = d0 + W < dend ? d0 + W : dend;
        const bool last = d1 == dend;
        const unsigned long long* r0 = brk + 6 * c;  // this block's start: X record, Y record
        const unsigned long long* r1 = r0 + 6;       // the next block's start (same quad unless last)
        const size_t kx0 = r0[0], ax0 = r0[1], ky0 = r0[3], ay0 = r0[4];
        const size_t kx1 = last ? nx : r1[0], ax1 = last ? g.len[0] : r1[2];
        const size_t ky1 = last ? ny : r1[3], ay1 = last ? g.len[2] : r1[5];
        const size_t px0 = (kx0 ? kx0 - 1 : 0) * G, py0 = (ky0 ? ky0 - 1 : 0) * G;
        const size_t px1 = kx1 * G < lx ? kx1 * G : lx, py1 = ky1 * G < ly ? ky1 * G : ly;
        const K* A = src + g.qb;
        const K* B = A + g.len[0];
        const K* C = B + g.len[1];
        const K* D = C + g.len[2];
        const K* gw[4] = {A + ax0, B + (px0 - ax0), C + ay0, D + (py0 - ay0)};
        const long long nwl[4] = {(long long)ax1 - (long long)ax0,
                                  (long long)(px1 - ax1) - (long long)(px0 - ax0),
                                  (long long)ay1 - (long long)ay0,
                                  (long long)(py1 - ay1) - (long long)(py0 - ay0)};
        const long long e0l = (long long)d0 - (long long)(px0 + py0);
        const long long e1l = (long long)d1 - (long long)(px0 + py0);
        const long long tot = nwl[0] + nwl[1] + nwl[2] + nwl[3];
        geo.ok = !(nwl[0] < 0 || nwl[1] < 0 || nwl[2] < 0 || nwl[3] < 0 || tot > W + 4 * G || e0l < 0 || e1l > tot);
        if (!geo.ok) {
            atomicOr(status, kStatusInternal);
        } else {
            // ---- four windows into region 1 by bulk copies ----
            Window w[4];
            int region = 0;
            uint32_t bytes = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                w[i] = place_window(gw[i], (int)nwl[i], region, QMAX + 1);
                region = w[i].end;
                bytes += (uint32_t)(w[i].nbulk * KS);
            }
            mbar_arrive_expect_tx(&bar, bytes);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (w[i].nbulk)
                    tma_load_1d(s1 + w[i].off + w[i].head, gw[i] + w[i].head, (uint32_t)(w[i].nbulk * KS), &bar);
                geo.gw[i] = gw[i];
                geo.nw[i] = (int)nwl[i];
                geo.off[i] = w[i].off;
            }
            geo.e0 = (int)e0l;
            geo.e1 = (int)e1l;
        }
    }
    __syncthreads();
    if (!geo.ok) return;
    int nw[4], off[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        nw[i] = geo.nw[i];
        off[i] = geo.off[i];
    }
    const int e0 = geo.e0, e1 = geo.e1;

    // Scalar parts: the elements before and after each window's bulk part
    // (fewer than 16 bytes each) and the sentinels after it.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (warp != i % NW) continue;  // warp i % NW serves window i
        const K* gwi = geo.gw[i];
        constexpr int EPC = 16 / KS;
        const int head = (int)(((16u - (reinterpret_cast<uintptr_t>(gwi) & 15u)) & 15u) / KS);
        const int h = head < nw[i] ? head : nw[i];
        const int t0 = h + ((nw[i] - h) / EPC) * EPC;
        if (lane < h) s1[off[i] + lane] = gwi[lane];
        if (lane < nw[i] - t0) s1[off[i] + t0 + lane] = gwi[t0 + lane];
        for (int j = lane; j <= QMAX; j += 32) s1[off[i] + nw[i] + j] = key_max<K>();
    }
    const int nX = nw[0] + nw[1], nY = nw[2] + nw[3];
    const int yoff = nX + IPT + 1;
    if (warp == NW - 1)
        for (int j = lane; j <= IPT; j += 32) {
            s2[nX + j] = key_max<K>();
            s2[yoff + nY + j] = key_max<K>();
        }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, kWaitLimitCycles)) {
        if (t == 0) atomicOr(status, kStatusTimeout);
        mbar_wait_bounded(&bar, 0, kWaitLimitCycles);  // copies still in flight
        return;
    }

    // ---- level 1: X window = merge(A, B), Y window = merge(C, D) ----
    constexpr int R2B = R1 * KS;  // byte offset of region 2
    {
        const int N1 = nX + nY;
        const int qn = ((N1 + THREADS - 1) / THREADS) | 1;  // odd: conflict-free stores
        const int s = t * qn;
        const int e = s + qn < N1 ? s + qn : N1;
        if (s < e && s < nX) {
            const int xe = e < nX ? e : nX;
            merge_run_smem<K>(smem_raw, off[0] * KS, nw[0], off[1] * KS, nw[1], s, xe - s, R2B);
        }
        if (s < e && e > nX) {
            const int ys = (s > nX ? s : nX) - nX;
            merge_run_smem<K>(smem_raw, off[2] * KS, nw[2], off[3] * KS, nw[3], ys, e - nX - ys, R2B + yoff * KS);
        }
    }
    __syncthreads();

    // ---- level 2: this block's outputs, staged in region 1 ----
    {
        const int X0 = R2B, Y0 = R2B + yoff * KS;
        const int diag = e0 + t * IPT;
        const int mine = e1 - diag;
        if (mine > 0) {
            int lo = diag > nY ? diag - nY : 0;
            int hi = diag < nX ? diag : nX;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sld<K>(smem_raw, X0 + mid * KS) <= sld<K>(smem_raw, Y0 + (diag - 1 - mid) * KS))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int io = X0 + lo * KS, jo = Y0 + (diag - lo) * KS, oo = t * IPT * KS;
            K av = sld<K>(smem_raw, io), bv = sld<K>(smem_raw, jo);
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                const bool ta = av <= bv;
                if (i < mine) sst<K>(smem_raw, oo + i * KS, ta ? av : bv);
                io += ta ? KS : 0;
                jo += ta ? 0 : KS;
                const K nv = sld<K>(smem_raw, ta ? io : jo);
                av = ta ? nv : av;
                bv = ta ? bv : nv;
            }
        }
    }
    const int total = e1 - e0;
    K* Dst = dst + out0;
    const bool dst_ok = aligned16(Dst);
    const int nbk = dst_ok ? (total * KS / 16) * 16 / KS : 0;
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
        if (nbk) tma_store_1d(Dst, s1, (uint32_t)(nbk * KS));
        tma_store_commit();
    }
    for (int i = nbk + t; i < total; i += THREADS) Dst[i] = s1[i];
    if (t == 0) tma_store_wait_read();
}

}  // namespace msort
