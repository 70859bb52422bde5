// Pass scheduler and C ABI of the plain merge sort.
//
// One sort = one tile-sort launch (the chunk sort of Section
// "Multiprocessing Merge Sort", Figs. 6-7) followed by P = ceil(log2(n / T))
// rounds of the pairwise merge tree (Section "MPI Merge Sort", Figs. 16-17); each
// round is a partition launch (merge-path co-ranks of every output block) and
// a merge launch.  Buffers ping-pong between the caller's output and the
// context's scratch; the tile sort writes to whichever of the two makes the
// last round land in the caller's buffer, so no final copy is needed.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "learned.h"
#include "launch.h"

namespace msort {

static thread_local std::string tl_error;

msort_status fail(msort_status s, const std::string& msg) {
    tl_error = msg;
    return s;
}

msort_status cuda_fail(cudaError_t e, const char* what) {
    tl_error = std::string(what) + ": " + cudaGetErrorString(e);
    return MSORT_ERR_CUDA;
}

// Names of the kernel kinds in NVTX ranges (profilers show each logged
// launch as a named range on the host timeline).
static const char* const kKindName[KK_COUNT] = {"msort tile sort", "msort partition", "msort merge pass",
                                                "msort segmented", "msort mlp", "msort single launch"};

void prof_begin(msort_ctx* ctx, int k, cudaStream_t st) {
    if (!ctx->profiling) return;
    nvtxRangePushA(kKindName[k]);
    auto& v = ctx->prof[k];
    size_t& u = ctx->prof_used[k];
    if (u == v.size()) {
        EventPair p;
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        v.push_back(p);
    }
    cudaEventRecord(v[u].a, st);
}

void prof_end(msort_ctx* ctx, int k, cudaStream_t st) {
    if (!ctx->profiling) return;
    cudaEventRecord(ctx->prof[k][ctx->prof_used[k]].b, st);
    ++ctx->prof_used[k];
    nvtxRangePop();
}

msort_status ensure_scratch(msort_ctx* ctx, size_t bytes, cudaStream_t st) {
    if (ctx->scratch_pending && ctx->last_stream != st) {
        cudaError_t e = cudaStreamWaitEvent(st, ctx->scratch_done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    if (bytes <= ctx->scratch_bytes) return MSORT_OK;
    if (ctx->budget && bytes + ctx->staging_bytes > ctx->budget)
        return fail(MSORT_ERR_OOM, "scratch of " + std::to_string(bytes) + " bytes exceeds the context budget of " +
                                       std::to_string(ctx->budget) + " bytes");
    // Growth is rare (first call at a new size): wait until no kernel can
    // still be using the old block, then replace it.
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    size_t want = align_up(bytes, size_t(2) << 20);
    e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MSORT_ERR_OOM, "cudaMalloc of scratch (" + std::to_string(want) + " bytes) failed");
    }
    ctx->scratch_bytes = want;
    return MSORT_OK;
}

static void scratch_release(msort_ctx* ctx, cudaStream_t st) {
    cudaEventRecord(ctx->scratch_done, st);
    ctx->last_stream = st;
    ctx->scratch_pending = true;
}

// ----------------------------------------------------------------------------
// Plans
// ----------------------------------------------------------------------------
std::string& launch_info_ref() {
    static thread_local std::string info;
    return info;
}
const std::string& last_launch_info() { return launch_info_ref(); }

// Key types: element size and the order-preserving transform that maps them
// to unsigned keys (0 unsigned, 1 signed integers, 2 IEEE floating point).
static int key_bytes(msort_key_type kt) {
    switch (kt) {
        case MSORT_U32: case MSORT_I32: case MSORT_F32: return 4;
        case MSORT_U64: case MSORT_I64: case MSORT_F64: return 8;
        default: return 0;
    }
}
static int key_xform(msort_key_type kt) {
    return (kt == MSORT_I32 || kt == MSORT_I64) ? 1 : (kt == MSORT_F32 || kt == MSORT_F64) ? 2 : 0;
}

template <class K, bool PAIRS>
static int default_tile() {
    // measured best on GB300 (msort_tune): 512 x 33 for 32-bit keys alone,
    // 256 x 17 for 64-bit key-value pairs, 512 x 17 otherwise
    if (!PAIRS && sizeof(K) == 4) return 16896;
    if (PAIRS && sizeof(K) == 8) return 4352;
    return 8704;
}

template <class K, bool PAIRS>
static bool make_plan(size_t n, const msort_options* opt, Plan* pl, std::string* why, int xform = 0) {
    Plan p{};
    p.tile = opt && opt->tile ? opt->tile : default_tile<K, PAIRS>();
    // a tile of the single launch only (options.single_launch = 1): the
    // multi-launch fields below keep the default tile; apply_single replaces them
    if (opt && opt->single_launch == 1 && opt->tile && !tile_supported<K, PAIRS>(opt->tile) &&
        small_tile_supported<K, PAIRS>(opt->tile))
        p.tile = default_tile<K, PAIRS>();
    if (!tile_supported<K, PAIRS>(p.tile)) {
        *why = "options.tile " + std::to_string(p.tile) +
               " is not available for this key/value type (4352, 8448, 8704 or 16896)";
        return false;
    }
    // merge blocks use 256 threads and the tile's keys per thread
    const int ipt = (p.tile == 4352 || p.tile == 8704) ? 17 : 33;  // W = 256 * ipt divides 2 * tile
    p.W = 256 * ipt;
    if (opt && opt->merge_block && opt->merge_block != p.W) {
        *why = "options.merge_block must be 0 or " + std::to_string(p.W) + " for tile " + std::to_string(p.tile);
        return false;
    }
    p.passes = 0;
    for (size_t L = (size_t)p.tile; L < n; L *= 2) ++p.passes;
    p.partition_mode = opt ? opt->partition_mode : 0;
    p.learned_passes = opt ? opt->learned_passes : 0;
    // Four-way passes (two merge rounds per pass over memory) are offered
    // for keys-only sorts with the exact partition.  They are not the
    // default: on GB300 the pairwise pass already runs at the copy
    // bandwidth, and the four-way pass spends more time merging twice in
    // shared memory and partitioning than it saves in HBM traffic.
    const bool four_ok = !PAIRS && p.partition_mode == 0;
    const int ways = opt && opt->merge_ways ? opt->merge_ways : 2;
    if (ways != 2 && ways != 4) {
        *why = "options.merge_ways must be 0, 2 or 4";
        return false;
    }
    if (ways == 4 && !four_ok) {
        *why = "options.merge_ways = 4 needs a keys-only sort with partition_mode 0";
        return false;
    }
    p.ways = ways;
    p.xform = xform;
    p.xform_out = xform;
    if (xform && (p.partition_mode != 0 || ways != 2)) {
        *why = "signed and floating-point keys need partition_mode 0 and pairwise merge passes";
        return false;
    }
    p.W4 = ipt == 33 ? 2816 : 4352;  // four-way block: 256 threads x 11 or 17 outputs
    p.G4 = p.W4 / 8;
    p.status = nullptr;
    *pl = p;
    return true;
}

// The single-launch plan (csrc/small.cuh): tile sort and every merge round
// in one cooperative launch.  Chosen automatically for n up to 2^22 (such an
// array stays in L2, and launch cost dominates the multi-launch plan) when
// the caller leaves the tile and merge block at 0 with partition_mode 0 and
// pairwise passes; options.single_launch = 1 asks for it up to 2^28
// elements, -1 never uses it.
constexpr size_t kSingleLaunchAuto = size_t(1) << 22;
constexpr size_t kSingleLaunchForcedMax = size_t(1) << 28;

// Options the single launch accepts: partition_mode 0, pairwise passes,
// merge_block 0, and tile 0 (or, with single_launch = 1, one of its tiles).
static bool single_eligible(const msort_options* opt) {
    return !(opt && ((opt->tile && opt->single_launch != 1) || opt->merge_block || opt->partition_mode ||
                     (opt->merge_ways && opt->merge_ways != 2)));
}

static bool single_wanted(size_t n, const msort_options* opt) {
    const int mode = opt ? opt->single_launch : 0;
    if (n == 0 || mode < 0 || !single_eligible(opt)) return false;
    return mode == 1 ? n <= kSingleLaunchForcedMax : n <= kSingleLaunchAuto;
}

template <class K, bool PAIRS>
static bool apply_single(size_t n, const msort_options* opt, Plan* pl, std::string* why) {
    const int mode = opt ? opt->single_launch : 0;
    if (mode < -1 || mode > 1) {
        *why = "options.single_launch must be -1, 0 or 1";
        return false;
    }
    if (mode == 1 && !single_eligible(opt)) {
        *why = "options.single_launch = 1 needs tile and merge_block 0, partition_mode 0 and pairwise passes";
        return false;
    }
    if (mode == 1 && n > kSingleLaunchForcedMax) {
        *why = "options.single_launch = 1 takes at most 2^28 elements";
        return false;
    }
    if (mode == 1 && opt->tile && !small_tile_supported<K, PAIRS>(opt->tile)) {
        *why = "options.tile " + std::to_string(opt->tile) + " is not a single-launch tile for this key/value type";
        return false;
    }
    if (!single_wanted(n, opt)) return true;
    const int T = (opt && opt->tile) ? opt->tile : small_tile<K, PAIRS>(n);
    pl->single = 1;
    pl->tile = T;
    pl->W = T;
    pl->passes = 0;
    for (size_t L = (size_t)T; L < n; L *= 2) ++pl->passes;
    return true;
}

// Run length of the first four-way pass (the pairwise pass, if the pass
// count is odd, goes first), and the largest four-way grid over the plan.
static size_t merge4_grid_max(size_t n, const Plan& pl) {
    size_t m = 0;
    if (pl.ways != 4) return 0;
    for (int p = pl.passes & 1; p + 1 < pl.passes; p += 2)
        m = std::max(m, merge4_grid_points(n, (size_t)pl.tile << p, (size_t)pl.G4));
    return m;
}

template <class K, bool PAIRS>
static size_t scratch_need(size_t n, const Plan& pl) {
    size_t b = align_up(n * sizeof(K), 256);
    if (PAIRS) b += align_up(n * sizeof(uint32_t), 256);
    // the single launch keeps a split table big enough for the multi-launch
    // plan it falls back to (merge blocks of at least 4352 outputs)
    const size_t Wt = pl.single ? std::min<size_t>((size_t)pl.W, 4352) : (size_t)pl.W;
    size_t nblocks = (n + Wt - 1) / Wt;
    b += align_up((nblocks + 1) * sizeof(unsigned long long), 256);
    const size_t gm = merge4_grid_max(n, pl);
    if (gm) {
        const size_t nb4 = (n + pl.W4 - 1) / pl.W4;
        b += 2 * align_up(gm * sizeof(unsigned long long), 256) + align_up(gm * sizeof(K), 256) +
             align_up(6 * (nb4 + 1) * sizeof(unsigned long long), 256);
    }
    return b;
}

// The whole sort on stream st.  kin may equal kout (in-place).  `scratch`
// holds the ping-pong buffer and the split table (scratch_need bytes);
// `log` brackets launches with the profiling events.
template <class K, bool PAIRS>
static msort_status run_sort(msort_ctx* ctx, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                             const Plan& pl, void* scratch, bool log, cudaStream_t st) {
    unsigned char* sp = static_cast<unsigned char*>(scratch);
    K* tk = reinterpret_cast<K*>(sp);
    sp += align_up(n * sizeof(K), 256);
    uint32_t* tv = nullptr;
    if (PAIRS) {
        tv = reinterpret_cast<uint32_t*>(sp);
        sp += align_up(n * sizeof(uint32_t), 256);
    }
    unsigned long long* splits = reinterpret_cast<unsigned long long*>(sp);
    sp += align_up(((n + pl.W - 1) / pl.W + 1) * sizeof(unsigned long long), 256);
    // four-way grid: co-ranks, positions, keys, block brackets
    const size_t gm = merge4_grid_max(n, pl);
    unsigned long long* gco = reinterpret_cast<unsigned long long*>(sp);
    sp += align_up(gm * sizeof(unsigned long long), 256);
    unsigned long long* gpos = reinterpret_cast<unsigned long long*>(sp);
    sp += align_up(gm * sizeof(unsigned long long), 256);
    K* gval = reinterpret_cast<K*>(sp);
    sp += align_up(gm * sizeof(K), 256);
    unsigned long long* brk = reinterpret_cast<unsigned long long*>(sp);

    if (pl.single) {
        // the split table is unused by this plan; its first 8 bytes hold the grid barrier
        if (log) prof_begin(ctx, KK_SINGLE, st);
        cudaError_t es = launch_small<K, PAIRS>(pl, kin, vin, kout, vout, tk, tv, n, splits, st, pl.xform,
                                                pl.xform_out);
        if (log) prof_end(ctx, KK_SINGLE, st);
        if (es == cudaErrorCooperativeLaunchTooLarge || es == cudaErrorNotSupported) {
            // the device refused a grid that must be resident at once (for
            // example under a limit on the SMs this process may use): sort
            // with the multi-launch plan instead (its split table fits, see
            // scratch_need)
            cudaGetLastError();
            Plan mp;
            std::string why;
            if (!make_plan<K, PAIRS>(n, nullptr, &mp, &why, pl.xform)) return fail(MSORT_ERR_INVALID_ARG, why);
            mp.status = pl.status;
            mp.xform_out = pl.xform_out;
            return run_sort<K, PAIRS>(ctx, kin, vin, kout, vout, n, mp, scratch, log, st);
        }
        ++ctx->launches;
        if (es != cudaSuccess) return cuda_fail(es, ("single-launch sort" + last_launch_info()).c_str());
        return MSORT_OK;
    }
    // Passes over memory: with four-way passes, one pairwise pass first when
    // the number of merge rounds is odd, then one pass per two rounds.
    const int four = gm ? pl.passes / 2 : 0;
    const int two = pl.passes - 2 * four;
    K* bk[2] = {kout, tk};
    uint32_t* bv[2] = {vout, tv};
    int cur = ((two + four) & 1) ? 1 : 0;
    cudaError_t e;
    if (log) prof_begin(ctx, KK_TILE, st);
    e = launch_tile<K, PAIRS>(pl, kin, vin, bk[cur], bv[cur], n, st, pl.xform, pl.passes == 0 ? pl.xform_out : 0);
    if (log) prof_end(ctx, KK_TILE, st);
    ++ctx->launches;
    if (e != cudaSuccess) return cuda_fail(e, ("tile sort launch" + last_launch_info()).c_str());
    const int first_guided = pl.partition_mode != 0 ? learned_first_pass(pl, n) : pl.passes;
    for (int p = 0; p < two; ++p) {
        const size_t L = (size_t)pl.tile << p;
        if (log) prof_begin(ctx, KK_PARTITION, st);
        if (p >= first_guided)
            e = launch_guided_partition<K>(ctx, pl, bk[cur], n, L, splits, st);
        else
            e = launch_partition<K>(pl, bk[cur], n, L, splits, st);
        if (log) prof_end(ctx, KK_PARTITION, st);
        ++ctx->launches;
        if (e != cudaSuccess) return cuda_fail(e, "partition launch");
        if (log) prof_begin(ctx, KK_MERGE, st);
        const int xf_out = (p + 1 == pl.passes) ? pl.xform_out : 0;  // the last round writes the caller's keys
        e = launch_merge<K, PAIRS>(pl, bk[cur], bk[cur ^ 1], bv[cur], bv[cur ^ 1], n, L, splits, st, 0, ~size_t(0),
                                   xf_out);
        if (log) prof_end(ctx, KK_MERGE, st);
        ++ctx->launches;
        if (e != cudaSuccess) return cuda_fail(e, ("merge pass launch" + last_launch_info()).c_str());
        cur ^= 1;
    }
    for (int p = two; p < pl.passes; p += 2) {
        const size_t L = (size_t)pl.tile << p;
        if (log) prof_begin(ctx, KK_PARTITION, st);
        e = launch_merge4_partition<K>(pl, bk[cur], n, L, gco, gval, gpos, brk, st);
        if (log) prof_end(ctx, KK_PARTITION, st);
        ctx->launches += 3;
        if (e != cudaSuccess) return cuda_fail(e, "four-way partition launch");
        if (log) prof_begin(ctx, KK_MERGE, st);
        e = launch_merge4<K>(pl, bk[cur], bk[cur ^ 1], n, L, brk, st);
        if (log) prof_end(ctx, KK_MERGE, st);
        ++ctx->launches;
        if (e != cudaSuccess) return cuda_fail(e, ("four-way merge launch" + last_launch_info()).c_str());
        cur ^= 1;
    }
    return MSORT_OK;
}

// ---------------------------------------------------------------------------
// CUDA-graph replay of plain sorts (options.use_graph): the launch sequence
// of a (buffers, size, plan) is captured once and replayed, which removes
// the per-launch host cost that dominates small sorts.
// ---------------------------------------------------------------------------
struct PlainGraphKey {
    const void *kin, *vin, *kout, *vout, *scratch;
    size_t n;
    int type, tile, W, passes, ways, xform, single;
    bool operator<(const PlainGraphKey& o) const {
        return std::tie(kin, vin, kout, vout, scratch, n, type, tile, W, passes, ways, xform, single) <
               std::tie(o.kin, o.vin, o.kout, o.vout, o.scratch, o.n, o.type, o.tile, o.W, o.passes, o.ways,
                        o.xform, o.single);
    }
};
// At most kMaxPlainGraphs graphs are kept; a new one evicts the least
// recently used after the device has finished everything in flight (so no
// evicted graph can still be running).
constexpr size_t kMaxPlainGraphs = 64;
struct PlainGraphs {
    struct Entry {
        cudaGraphExec_t exec;
        unsigned long long launches;  // kernel launches one replay stands for
        unsigned long long used;      // tick of the last replay
    };
    std::map<PlainGraphKey, Entry> exec;
    unsigned long long tick = 0;
};

void plain_graphs_destroy(msort_ctx* ctx) {
    PlainGraphs* pg = static_cast<PlainGraphs*>(ctx->plain_graphs);
    if (!pg) return;
    for (auto& kv : pg->exec) cudaGraphExecDestroy(kv.second.exec);
    delete pg;
    ctx->plain_graphs = nullptr;
}

template <class K, bool PAIRS>
static msort_status run_sort_graph(msort_ctx* ctx, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
                                   size_t n, const Plan& pl, cudaStream_t st) {
    if (!ctx->plain_graphs) ctx->plain_graphs = new PlainGraphs();
    PlainGraphs* pg = static_cast<PlainGraphs*>(ctx->plain_graphs);
    const PlainGraphKey key{kin,     vin,  kout,      vout,    ctx->scratch, n, (int)sizeof(K) * 2 + (PAIRS ? 1 : 0),
                            pl.tile, pl.W, pl.passes, pl.ways, pl.xform, pl.single};
    auto it = pg->exec.find(key);
    if (it == pg->exec.end()) {
        if (pg->exec.size() >= kMaxPlainGraphs) {
            auto lru = pg->exec.begin();
            for (auto j = pg->exec.begin(); j != pg->exec.end(); ++j)
                if (j->second.used < lru->second.used) lru = j;
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaGraphExecDestroy(lru->second.exec);
            pg->exec.erase(lru);
        }
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        cudaGraph_t graph = nullptr;
        msort_status s = MSORT_OK;
        const unsigned long long before = ctx->launches;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s = run_sort<K, PAIRS>(ctx, kin, vin, kout, vout, n, pl, ctx->scratch, false, cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (s == MSORT_OK && e2 != cudaSuccess) s = cuda_fail(e2, "cudaStreamEndCapture");
        } else {
            s = cuda_fail(e, "cudaStreamBeginCapture");
        }
        const unsigned long long nl = ctx->launches - before;
        ctx->launches = before;
        cudaStreamDestroy(cap);
        if (s != MSORT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        it = pg->exec.emplace(key, PlainGraphs::Entry{exec, nl, 0}).first;
    }
    it->second.used = ++pg->tick;
    cudaError_t e = cudaGraphLaunch(it->second.exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    ctx->launches += it->second.launches;
    return MSORT_OK;
}

// Self-test of the single launch's grid barriers (msort_selftest_grid_timeout):
// the single-launch sort of the n uint32 keys at d_keys, launched so that its
// first grid barrier expects one arrival more than the grid makes, with
// every wait limited to limit_cycles.  All blocks give up there, record the
// timeout in the context's status word and leave; the keys are left in an
// unspecified order.
msort_status selftest_single_timeout(msort_ctx* ctx, void* d_keys, size_t n, long long limit_cycles,
                                     cudaStream_t st) {
    msort_options o{};
    o.single_launch = 1;
    Plan pl;
    std::string why;
    if (!make_plan<uint32_t, false>(n, &o, &pl, &why) || !apply_single<uint32_t, false>(n, &o, &pl, &why))
        return fail(MSORT_ERR_INVALID_ARG, why);
    if (!pl.single || pl.passes < 1) return fail(MSORT_ERR_INVALID_ARG, "n must span at least two single-launch tiles");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    pl.status = ctx->d_status;
    msort_status s = ensure_scratch(ctx, scratch_need<uint32_t, false>(n, pl), st);
    if (s != MSORT_OK) return s;
    unsigned char* sp = static_cast<unsigned char*>(ctx->scratch);
    uint32_t* tk = reinterpret_cast<uint32_t*>(sp);
    void* barrier = sp + align_up(n * sizeof(uint32_t), 256);  // the split table (unused by this plan)
    uint32_t* keys = static_cast<uint32_t*>(d_keys);
    e = launch_small<uint32_t, false>(pl, keys, nullptr, keys, nullptr, tk, nullptr, n, barrier, st, 0, 0,
                                      limit_cycles, 1u);
    ++ctx->launches;
    scratch_release(ctx, st);
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, ("single-launch self-test" + last_launch_info()).c_str());
}

template <class K>
size_t sort_keys_scratch(size_t n) {
    Plan pl;
    std::string why;
    make_plan<K, false>(n, nullptr, &pl, &why);
    return scratch_need<K, false>(n, pl);
}

template <class K>
msort_status sort_keys_internal(msort_ctx* ctx, const K* in, K* out, size_t n, void* scratch, cudaStream_t st) {
    Plan pl;
    std::string why;
    if (!make_plan<K, false>(n, nullptr, &pl, &why)) return fail(MSORT_ERR_INVALID_ARG, why);
    pl.status = ctx->d_status;
    return run_sort<K, false>(ctx, in, nullptr, out, nullptr, n, pl, scratch, false, st);
}

// Any sort (keys or pairs, in or out of place) with caller-provided scratch
// of scratch_need bytes; used by the serving loop, whose scratch comes from
// its own arena.  No allocation, no host synchronisation.
template <class K, bool PAIRS>
msort_status sort_with_scratch(msort_ctx* ctx, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                               void* scratch, cudaStream_t st) {
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, nullptr, &pl, &why)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (n == 0) return MSORT_OK;
    pl.status = ctx->d_status;
    return run_sort<K, PAIRS>(ctx, kin, vin, kout, vout, n, pl, scratch, false, st);
}

size_t sort_scratch_need(size_t n, int key_bytes, bool pairs) {
    Plan pl;
    std::string why;
    if (key_bytes == 4) {
        if (pairs) return make_plan<uint32_t, true>(n, nullptr, &pl, &why) ? scratch_need<uint32_t, true>(n, pl) : 0;
        return make_plan<uint32_t, false>(n, nullptr, &pl, &why) ? scratch_need<uint32_t, false>(n, pl) : 0;
    }
    if (pairs) return make_plan<uint64_t, true>(n, nullptr, &pl, &why) ? scratch_need<uint64_t, true>(n, pl) : 0;
    return make_plan<uint64_t, false>(n, nullptr, &pl, &why) ? scratch_need<uint64_t, false>(n, pl) : 0;
}

template msort_status sort_with_scratch<uint32_t, false>(msort_ctx*, const uint32_t*, const uint32_t*, uint32_t*,
                                                         uint32_t*, size_t, void*, cudaStream_t);
template msort_status sort_with_scratch<uint32_t, true>(msort_ctx*, const uint32_t*, const uint32_t*, uint32_t*,
                                                        uint32_t*, size_t, void*, cudaStream_t);
template msort_status sort_with_scratch<uint64_t, false>(msort_ctx*, const uint64_t*, const uint32_t*, uint64_t*,
                                                         uint32_t*, size_t, void*, cudaStream_t);
template msort_status sort_with_scratch<uint64_t, true>(msort_ctx*, const uint64_t*, const uint32_t*, uint64_t*,
                                                        uint32_t*, size_t, void*, cudaStream_t);

template size_t sort_keys_scratch<uint32_t>(size_t);
template size_t sort_keys_scratch<uint64_t>(size_t);
template msort_status sort_keys_internal<uint32_t>(msort_ctx*, const uint32_t*, uint32_t*, size_t, void*,
                                                   cudaStream_t);
template msort_status sort_keys_internal<uint64_t>(msort_ctx*, const uint64_t*, uint64_t*, size_t, void*,
                                                   cudaStream_t);

// Tuned tile for (key type, values, n): the entry of the largest tuned size
// class not above log2(n) (or the smallest class), 0 if nothing was tuned.
static int tuned_choice(const std::map<std::tuple<int, int, int>, int>& table, int key_bytes, bool pairs, size_t n) {
    int best = 0, best_cls = -1, lowest = 0, lowest_cls = 1 << 30;
    int lg = 0;
    while (lg < 63 && (size_t(1) << (lg + 1)) <= n) ++lg;
    for (const auto& kv : table) {
        if (std::get<0>(kv.first) != key_bytes || std::get<1>(kv.first) != (int)pairs) continue;
        const int cls = std::get<2>(kv.first);
        if (cls <= lg && cls > best_cls) {
            best_cls = cls;
            best = kv.second;
        }
        if (cls < lowest_cls) {
            lowest_cls = cls;
            lowest = kv.second;
        }
    }
    return best ? best : lowest;
}

static int tuned_tile_for(const msort_ctx* ctx, int key_bytes, bool pairs, size_t n) {
    return tuned_choice(ctx->tuned_tile, key_bytes, pairs, n);
}

template <class K, bool PAIRS>
static msort_status sort_entry(msort_ctx* ctx, const void* kin, const uint32_t* vin, void* kout, uint32_t* vout,
                               size_t n, const msort_options* opt, cudaStream_t st, int xform) {
    msort_options tuned_opt{};
    const msort_options* caller = opt;
    const bool single = single_wanted(n, opt);  // tuned shapes do not apply to the single launch
    if (!single && (!opt || !opt->tile)) {
        const int tile = tuned_tile_for(ctx, (int)sizeof(K), PAIRS, n);
        if (tile) {
            if (opt) tuned_opt = *opt;
            tuned_opt.tile = tile;
            opt = &tuned_opt;
        }
    }
    // tuned merge fan-in where the caller left it open (the four-way pass
    // takes neither transformed keys nor the learned partition)
    if (!single && !xform && (!opt || (!opt->merge_ways && opt->partition_mode == 0))) {
        const int ways = tuned_choice(ctx->tuned_ways, (int)sizeof(K), PAIRS, n);
        if (ways) {
            if (opt && opt != &tuned_opt) tuned_opt = *opt;
            tuned_opt.merge_ways = ways;
            opt = &tuned_opt;
        }
    }
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (!apply_single<K, PAIRS>(n, caller, &pl, &why)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (n == 0) return MSORT_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    pl.status = ctx->d_status;
    msort_status s = ensure_scratch(ctx, scratch_need<K, PAIRS>(n, pl), st);
    if (s != MSORT_OK) return s;
    if (pl.partition_mode == 1 && pl.passes > 0) {
        // the tile sort writes the caller's output when the pass count is even
        s = learned_prepare<K>(ctx, pl, static_cast<const K*>(kin), n, st, kin == kout && !(pl.passes & 1));
        if (s != MSORT_OK) return s;
    }
    // Graph replay for the exact partition (the learned one prepares its
    // model on the host side per call); not while profiling, whose events
    // bracket individual launches.
    if (opt && opt->use_graph && pl.partition_mode == 0 && !ctx->profiling)
        s = run_sort_graph<K, PAIRS>(ctx, static_cast<const K*>(kin), vin, static_cast<K*>(kout), vout, n, pl, st);
    else
        s = run_sort<K, PAIRS>(ctx, static_cast<const K*>(kin), vin, static_cast<K*>(kout), vout, n, pl,
                               ctx->scratch, true, st);
    scratch_release(ctx, st);
    return s;
}

static msort_status check_common(msort_ctx* ctx, msort_key_type kt, const msort_options* opt) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    if (!key_bytes(kt)) return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
    if (opt) {
        for (int r : opt->reserved)
            if (r) return fail(MSORT_ERR_INVALID_ARG, "options.reserved must be zero");
        if (opt->partition_mode < 0 || opt->partition_mode > 3)
            return fail(MSORT_ERR_INVALID_ARG, "options.partition_mode must be 0, 1, 2 or 3");
        if (opt->learned_passes < 0) return fail(MSORT_ERR_INVALID_ARG, "options.learned_passes must be >= 0");
    }
    return MSORT_OK;
}

template <class K, bool PAIRS>
msort_status plan_info_for(size_t n, const msort_options* opt, int* tile, int* W, int* passes, int xform) {
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (!apply_single<K, PAIRS>(n, opt, &pl, &why)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (tile) *tile = pl.tile;
    if (W) *W = pl.W;
    if (passes) *passes = pl.passes;
    return MSORT_OK;
}

template <class K, bool PAIRS>
msort_status plan_passes_for(size_t n, const msort_options* opt, int* ways, int* memory_passes, int xform) {
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (!apply_single<K, PAIRS>(n, opt, &pl, &why)) return fail(MSORT_ERR_INVALID_ARG, why);
    const bool four = merge4_grid_max(n, pl) != 0;
    if (ways) *ways = four ? 4 : 2;
    if (memory_passes) *memory_passes = four ? pl.passes / 2 + (pl.passes & 1) : pl.passes;
    return MSORT_OK;
}

template <class K, bool PAIRS>
size_t scratch_bytes_for(size_t n, const msort_options* opt, int xform) {
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return 0;
    if (!apply_single<K, PAIRS>(n, opt, &pl, &why)) return 0;
    return scratch_need<K, PAIRS>(n, pl);
}

// ---------------------------------------------------------------------------
// Sorting host buffers.  The sort of n keys is the same plan as on device
// buffers; what changes is where the copies go:
//  * the host-to-device copy is issued in chunks of T * 2^m keys (about n/8)
//    on a copy stream, and each chunk's tile sort and its chunk-local merge
//    rounds (runs shorter than a chunk) start as soon as the chunk arrives;
//  * the remaining log2(chunks) rounds run over the whole array; the last
//    one is launched in slices, and each slice's device-to-host copy starts
//    on a second copy stream as soon as the slice is written;
//  * three staging slots serve consecutive calls in turn, and the work runs on the
//    context's own copy and compute streams (the caller's stream only waits
//    for the last copy), so with the asynchronous entry point one sort's
//    device-to-host copy overlaps the next sort's host-to-device copy and
//    sort (the link carries both directions at once).
// The tile sort writes to whichever buffer makes the last round land in the
// staging slot, so the shared scratch is free as soon as the compute stream
// moves on.
// ---------------------------------------------------------------------------
// Chunks of the host-to-device copy and slices of the last merge round.  A
// synchronous call has nothing else to overlap with, so it splits finely;
// back-to-back asynchronous calls overlap one another's copies anyway, and
// every chunk repeats the latency-bound partition launches of the
// chunk-local rounds, so they split coarsely (measured on GB300 at 2^28
// keys: 4/4 gives the fastest single call, 1/2 the highest throughput).
constexpr int kHostChunks = 8;  // array sizes (maximum chunks / slices)
constexpr int kHostSlices = 8;
constexpr int kSyncChunks = 4, kSyncSlices = 4;
constexpr int kAsyncChunks = 1, kAsyncSlices = 2;
constexpr int kHostSlots = 3;   // staging slots used by consecutive calls in turn

struct HostPipe {
    cudaStream_t h2d = nullptr, cs = nullptr, d2h = nullptr;
    void* slot[kHostSlots] = {};
    size_t slot_bytes[kHostSlots] = {};
    cudaEvent_t done[kHostSlots] = {};
    cudaEvent_t in_ev[kHostSlots][kHostChunks] = {};
    cudaEvent_t out_ev[kHostSlots][kHostSlices] = {};
    bool used[kHostSlots] = {};
    int next = 0;
    // out-of-core sorts: pinned host buffer of sorted runs, kept between
    // calls (pinning memory is slow)
    void* runs = nullptr;
    size_t runs_bytes = 0;
};

void host_pipe_destroy(msort_ctx* ctx);

// After a host-buffer call failed part-way: wait until nothing it enqueued
// on the context's streams can still read or write the caller's host
// buffers, so that the caller may free them once the call returns.
static void host_pipe_drain(msort_ctx* ctx) {
    HostPipe* hp = static_cast<HostPipe*>(ctx->host_pipe);
    if (!hp) return;
    cudaStreamSynchronize(hp->h2d);
    cudaStreamSynchronize(hp->cs);
    cudaStreamSynchronize(hp->d2h);
}

static msort_status host_pipe_get(msort_ctx* ctx, HostPipe** out) {
    if (ctx->host_pipe) {
        *out = static_cast<HostPipe*>(ctx->host_pipe);
        return MSORT_OK;
    }
    HostPipe* hp = new HostPipe();
    cudaError_t e = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking);
    for (int s = 0; s < kHostSlots && e == cudaSuccess; ++s) {
        e = cudaEventCreateWithFlags(&hp->done[s], cudaEventDisableTiming);
        for (int i = 0; i < kHostChunks && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&hp->in_ev[s][i], cudaEventDisableTiming);
        for (int i = 0; i < kHostSlices && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&hp->out_ev[s][i], cudaEventDisableTiming);
    }
    ctx->host_pipe = hp;
    if (e != cudaSuccess) {
        host_pipe_destroy(ctx);  // with whatever was created; the next call tries again
        return cuda_fail(e, "host-sort streams/events");
    }
    *out = hp;
    return MSORT_OK;
}

void host_pipe_destroy(msort_ctx* ctx) {
    HostPipe* hp = static_cast<HostPipe*>(ctx->host_pipe);
    if (!hp) return;
    for (int s = 0; s < kHostSlots; ++s) {
        if (hp->slot[s]) cudaFree(hp->slot[s]);
        if (hp->done[s]) cudaEventDestroy(hp->done[s]);
        for (cudaEvent_t ev : hp->in_ev[s])
            if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t ev : hp->out_ev[s])
            if (ev) cudaEventDestroy(ev);
    }
    if (hp->runs) cudaFreeHost(hp->runs);
    if (hp->h2d) cudaStreamDestroy(hp->h2d);
    if (hp->cs) cudaStreamDestroy(hp->cs);
    if (hp->d2h) cudaStreamDestroy(hp->d2h);
    delete hp;
    ctx->host_pipe = nullptr;
    ctx->staging_bytes = 0;
}

template <class K, bool PAIRS>
static msort_status host_sort(msort_ctx* ctx, const void* h_kin_v, const uint32_t* h_vin, void* h_kout_v,
                              uint32_t* h_vout, size_t n, const msort_options* opt, cudaStream_t st, int chunks,
                              int slices, int xform, bool keep_xform = false) {
    const K* h_kin = static_cast<const K*>(h_kin_v);
    K* h_kout = static_cast<K*>(h_kout_v);
    msort_options tuned_opt{};
    const bool single = single_wanted(n, opt);  // tuned shapes do not apply to the single launch
    if (!single && (!opt || !opt->tile)) {
        const int tile = tuned_tile_for(ctx, (int)sizeof(K), PAIRS, n);
        if (tile) {
            if (opt) tuned_opt = *opt;
            tuned_opt.tile = tile;
            opt = &tuned_opt;
        }
    }
    Plan pl;
    std::string why;
    if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return fail(MSORT_ERR_INVALID_ARG, why);
    if (keep_xform) pl.xform_out = 0;  // output keys stay in their transformed (unsigned) order
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    pl.status = ctx->d_status;
    HostPipe* hp = nullptr;
    msort_status s = host_pipe_get(ctx, &hp);
    if (s != MSORT_OK) return s;

    // staging slot for this call
    const int sl = hp->next;
    const size_t kbytes = align_up(n * sizeof(K), 256);
    const size_t need = kbytes + (PAIRS ? align_up(n * sizeof(uint32_t), 256) : 0);
    if (hp->slot_bytes[sl] < need) {
        const size_t others = ctx->staging_bytes - hp->slot_bytes[sl];
        if (ctx->budget && need + others + ctx->scratch_bytes > ctx->budget)
            return fail(MSORT_ERR_OOM, "host-sort staging exceeds the context budget");
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        if (hp->slot[sl]) cudaFree(hp->slot[sl]);
        hp->slot[sl] = nullptr;
        ctx->staging_bytes = others;
        hp->slot_bytes[sl] = 0;
        if (cudaMalloc(&hp->slot[sl], need) != cudaSuccess) {
            cudaGetLastError();
            return fail(MSORT_ERR_OOM, "cudaMalloc of host-sort staging failed");
        }
        hp->slot_bytes[sl] = need;
        ctx->staging_bytes = others + need;
    }
    const cudaStream_t cs = hp->cs;
    s = ensure_scratch(ctx, scratch_need<K, PAIRS>(n, pl), cs);
    if (s != MSORT_OK) return s;
    hp->next = (hp->next + 1) % kHostSlots;

    unsigned char* sbase = static_cast<unsigned char*>(hp->slot[sl]);
    K* S = reinterpret_cast<K*>(sbase);
    uint32_t* SV = PAIRS ? reinterpret_cast<uint32_t*>(sbase + kbytes) : nullptr;
    unsigned char* sp = static_cast<unsigned char*>(ctx->scratch);
    K* Tk = reinterpret_cast<K*>(sp);
    sp += align_up(n * sizeof(K), 256);
    uint32_t* Tv = nullptr;
    if (PAIRS) {
        Tv = reinterpret_cast<uint32_t*>(sp);
        sp += align_up(n * sizeof(uint32_t), 256);
    }
    unsigned long long* splits = reinterpret_cast<unsigned long long*>(sp);

    // The copies and kernels run on the context's own streams (host to
    // device, compute, device to host); `st` only waits for the last
    // device-to-host copy, so consecutive calls overlap.  A slot's
    // host-to-device copy waits for the last device-to-host copy out of it.
    if (hp->used[sl]) cudaStreamWaitEvent(hp->h2d, hp->done[sl], 0);

    // Pipelined schedule for the exact pairwise plan; the guided partition
    // and four-way passes keep one whole copy each way around the sort.
    const bool pipelined = pl.partition_mode == 0 && pl.ways == 2;
    const int P = pl.passes;
    int m = 0;  // chunk-local rounds: chunk = T << m, about n / chunks
    if (pipelined)
        while (m < P && ((size_t)pl.tile << m) * (size_t)chunks < n) ++m;
    const size_t chunk = pipelined && m < P ? (size_t)pl.tile << m : n;
    const size_t nc = (n + chunk - 1) / chunk;
    const int mloc = nc > 1 ? m : 0;

    K* bk[2] = {S, Tk};
    uint32_t* bv[2] = {SV, Tv};
    if (!pipelined) {
        if ((e = cudaMemcpyAsync(S, h_kin, n * sizeof(K), cudaMemcpyHostToDevice, hp->h2d)) != cudaSuccess ||
            (PAIRS && (e = cudaMemcpyAsync(SV, h_vin, n * 4, cudaMemcpyHostToDevice, hp->h2d)) != cudaSuccess))
            return cuda_fail(e, "host to device copy");
        cudaEventRecord(hp->in_ev[sl][0], hp->h2d);
        cudaStreamWaitEvent(cs, hp->in_ev[sl][0], 0);
        if (pl.partition_mode == 1 && P > 0) {
            s = learned_prepare<K>(ctx, pl, S, n, cs, !(P & 1));  // sorted in place
            if (s != MSORT_OK) return s;
        }
        s = run_sort<K, PAIRS>(ctx, S, SV, S, SV, n, pl, ctx->scratch, false, cs);
        if (s != MSORT_OK) return s;
        cudaEventRecord(hp->out_ev[sl][0], cs);
        cudaStreamWaitEvent(hp->d2h, hp->out_ev[sl][0], 0);
        if ((e = cudaMemcpyAsync(h_kout, S, n * sizeof(K), cudaMemcpyDeviceToHost, hp->d2h)) != cudaSuccess ||
            (PAIRS && (e = cudaMemcpyAsync(h_vout, SV, n * 4, cudaMemcpyDeviceToHost, hp->d2h)) != cudaSuccess))
            return cuda_fail(e, "device to host copy");
    } else {
        // the tile sort writes where the last of the P rounds lands in S
        const int cur0 = (P & 1) ? 1 : 0;
        for (size_t i = 0; i < nc; ++i) {
            const size_t off = i * chunk;
            const size_t ni = n - off < chunk ? n - off : chunk;
            if ((e = cudaMemcpyAsync(S + off, h_kin + off, ni * sizeof(K), cudaMemcpyHostToDevice, hp->h2d)) !=
                    cudaSuccess ||
                (PAIRS && (e = cudaMemcpyAsync(SV + off, h_vin + off, ni * 4, cudaMemcpyHostToDevice, hp->h2d)) !=
                              cudaSuccess))
                return cuda_fail(e, "host to device copy");
            cudaEventRecord(hp->in_ev[sl][i], hp->h2d);
            cudaStreamWaitEvent(cs, hp->in_ev[sl][i], 0);
            e = launch_tile<K, PAIRS>(pl, S + off, PAIRS ? SV + off : nullptr, bk[cur0] + off,
                                      PAIRS ? bv[cur0] + off : nullptr, ni, cs, pl.xform, P == 0 ? pl.xform_out : 0);
            ++ctx->launches;
            if (e != cudaSuccess) return cuda_fail(e, ("tile sort launch" + last_launch_info()).c_str());
            int cur = cur0;
            for (int p = 0; p < mloc; ++p) {
                const size_t L = (size_t)pl.tile << p;
                e = launch_partition<K>(pl, bk[cur] + off, ni, L, splits, cs);
                if (e == cudaSuccess)
                    e = launch_merge<K, PAIRS>(pl, bk[cur] + off, bk[cur ^ 1] + off, PAIRS ? bv[cur] + off : nullptr,
                                               PAIRS ? bv[cur ^ 1] + off : nullptr, ni, L, splits, cs);
                ctx->launches += 2;
                if (e != cudaSuccess) return cuda_fail(e, ("merge pass launch" + last_launch_info()).c_str());
                cur ^= 1;
            }
        }
        int cur = cur0 ^ (mloc & 1);
        const size_t nblocks = (n + pl.W - 1) / pl.W;
        for (int p = mloc; p < P; ++p) {
            const size_t L = (size_t)pl.tile << p;
            e = launch_partition<K>(pl, bk[cur], n, L, splits, cs);
            ++ctx->launches;
            if (e != cudaSuccess) return cuda_fail(e, "partition launch");
            const int ns = p + 1 == P ? slices : 1;
            for (int j = 0; j < ns; ++j) {
                const size_t c0 = nblocks * j / ns, c1 = nblocks * (j + 1) / ns;
                e = launch_merge<K, PAIRS>(pl, bk[cur], bk[cur ^ 1], bv[cur], bv[cur ^ 1], n, L, splits, cs, c0, c1,
                                           p + 1 == P ? pl.xform_out : 0);
                ++ctx->launches;
                if (e != cudaSuccess) return cuda_fail(e, ("merge pass launch" + last_launch_info()).c_str());
                if (p + 1 == P && c1 > c0) {
                    const size_t o0 = c0 * pl.W, o1 = c1 * pl.W < n ? c1 * pl.W : n;
                    cudaEventRecord(hp->out_ev[sl][j], cs);
                    cudaStreamWaitEvent(hp->d2h, hp->out_ev[sl][j], 0);
                    if ((e = cudaMemcpyAsync(h_kout + o0, S + o0, (o1 - o0) * sizeof(K), cudaMemcpyDeviceToHost,
                                             hp->d2h)) != cudaSuccess ||
                        (PAIRS && (e = cudaMemcpyAsync(h_vout + o0, SV + o0, (o1 - o0) * 4, cudaMemcpyDeviceToHost,
                                                       hp->d2h)) != cudaSuccess))
                        return cuda_fail(e, "device to host copy");
                }
            }
            cur ^= 1;
        }
        if (P == mloc) {  // no global round (P == 0): the tile sort's output in S is the result
            cudaEventRecord(hp->out_ev[sl][0], cs);
            cudaStreamWaitEvent(hp->d2h, hp->out_ev[sl][0], 0);
            if ((e = cudaMemcpyAsync(h_kout, S, n * sizeof(K), cudaMemcpyDeviceToHost, hp->d2h)) != cudaSuccess ||
                (PAIRS && (e = cudaMemcpyAsync(h_vout, SV, n * 4, cudaMemcpyDeviceToHost, hp->d2h)) != cudaSuccess))
                return cuda_fail(e, "device to host copy");
        }
    }
    // st completes only after the device-to-host copies
    cudaEventRecord(hp->done[sl], hp->d2h);
    cudaStreamWaitEvent(st, hp->done[sl], 0);
    hp->used[sl] = true;
    scratch_release(ctx, cs);
    return MSORT_OK;
}

// ---------------------------------------------------------------------------
// One round of the merge tree over sorted runs of arbitrary lengths laid end
// to end (boundaries ro, at least one run): runs 2j and 2j + 1 merge from src
// into the same positions of dst, up to kRunPairsMax pairs per launch pair;
// ro becomes the boundaries of the merged runs.  xf_out: key transform the
// round undoes as it writes.
// ---------------------------------------------------------------------------
template <class K, bool PAIRS>
static msort_status merge_runs_round(msort_ctx* ctx, const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst,
                                     std::vector<size_t>& ro, unsigned long long* splits, int xf_out,
                                     cudaStream_t st) {
    const size_t W = merge_two_block<K, PAIRS>();
    const size_t runs = ro.size() - 1;
    const size_t np = (runs + 1) / 2;
    for (size_t j0 = 0; j0 < np; j0 += kRunPairsMax) {
        RunPairs rp{};
        rp.np = (int)std::min<size_t>(kRunPairsMax, np - j0);
        for (int j = 0; j < rp.np; ++j) {
            const size_t a = 2 * (j0 + j);
            rp.p[j] = ro[a];
            rp.m[j] = ro[std::min(a + 1, runs)];
            rp.p[j + 1] = ro[std::min(a + 2, runs)];
            rp.c[j + 1] = rp.c[j] + (rp.p[j + 1] - rp.p[j] + W - 1) / W;
        }
        const cudaError_t e = launch_merge_runs<K, PAIRS>(src, dst, vsrc, vdst, rp, splits, ctx->d_status, xf_out, st);
        ctx->launches += 2;
        if (e != cudaSuccess) return cuda_fail(e, ("run merge launch" + last_launch_info()).c_str());
    }
    std::vector<size_t> next;
    for (size_t i = 0; i < runs; i += 2) next.push_back(ro[i]);
    next.push_back(ro[runs]);
    ro.swap(next);
    return MSORT_OK;
}

// Split table entries one round over `len` elements in runs may need.
template <class K, bool PAIRS>
static size_t merge_runs_splits(size_t len) {
    return len / merge_two_block<K, PAIRS>() + kRunPairsMax + 2;
}

// ---------------------------------------------------------------------------
// Host arrays larger than the device budget: an external merge sort.  The
// context's budget (msort_ctx_create) caps the device memory a sort may use;
// when the pipelined host sort of n elements would exceed it, the array is
// sorted in chunks that fit (each by the pipelined host sort, into a pinned
// host buffer of sorted runs) and the runs are merged in blocks that fit:
//  * regular samples, every sigma-th element of every run, sorted by
//    (key order, position), and every m-th of them as a block splitter bound
//    every block to at most (m + R) * sigma <= B elements (each run
//    contributes at most (its samples in the block + 1) * sigma elements);
//  * each block's slice of every run is copied to the device, merged there
//    by rounds of the pairwise merge tree over runs of unequal length (ties
//    to the earlier run, so the result is the stable merge), and copied to
//    its place in the output.  Blocks rotate through the host sort's staging slots and streams, so one
//    block's copy-in, the previous one's merge and the one before's copy-out
//    overlap.
// Splitters order equal keys by position, so runs of equal keys split too
// and the result is the stable sort of the whole array.
// ---------------------------------------------------------------------------
// Device bytes the pipelined host sort of n elements may hold (three
// staging slots and the sort scratch).
template <class K, bool PAIRS>
static size_t host_incore_bytes(size_t n, const Plan& pl) {
    const size_t slot = align_up(n * sizeof(K), 256) + (PAIRS ? align_up(n * 4, 256) : 0);
    return (size_t)kHostSlots * slot + align_up(scratch_need<K, PAIRS>(n, pl), size_t(2) << 20);  // scratch grows in 2 MiB steps
}

// Largest chunk whose in-core host sort fits the budget (0 if not even a
// few tiles fit).  The merge blocks reuse the same staging slots.
template <class K, bool PAIRS>
static size_t external_chunk(size_t budget, const msort_options* opt, int xform) {
    size_t lo = 0, hi = budget / sizeof(K) + 1;
    while (lo + 1 < hi) {
        const size_t mid = lo + (hi - lo) / 2;
        Plan pl;
        std::string why;
        const bool ok = make_plan<K, PAIRS>(mid, opt, &pl, &why, xform);
        if (ok && host_incore_bytes<K, PAIRS>(mid, pl) <= budget)
            lo = mid;
        else
            hi = mid;
    }
    return lo >= 4 * 16896 ? lo : 0;
}

// Merge blocks of an out-of-core sort (host logic): the R = ceil(n / chunk)
// sorted runs of `chunk` elements (the last ragged) lie end to end in
// tk[0, n), keys in unsigned order.  Returns cut[b * R + r] = the elements of
// run r ordered before block b, b = 0..nb, ordering by (key, global
// position); every block holds at most B elements (B >= 2R).  Splitters are
// regular samples: a block from one splitter sample to the next holding m
// samples has at most (m + R) * sigma elements (each run adds at most one
// unsampled stretch of sigma - 1), so splitters every m = (k - 1) R samples
// with sigma = B / (k R) keep blocks within B while their expected size is
// (1 - 1/k) B: k = 16 when sigma stays >= 1, else 2.
template <class K>
static std::vector<size_t> external_cuts(const K* tk, size_t n, size_t chunk, size_t B, size_t* nb_out) {
    const size_t R = (n + chunk - 1) / chunk;
    const size_t kover = 16 * R <= B ? 16 : 2;
    const size_t sigma = std::max<size_t>(1, B / (kover * R));
    const size_t every = (kover - 1) * R;
    struct Smp {
        K u;
        size_t g;
    };
    auto before = [](const Smp& a, const Smp& b) { return a.u < b.u || (a.u == b.u && a.g < b.g); };
    std::vector<Smp> smp;
    for (size_t r = 0; r < R; ++r) {
        const size_t off = r * chunk, len = std::min(chunk, n - off);
        for (size_t j = 0; j < len; j += sigma) smp.push_back(Smp{tk[off + j], off + j});
    }
    std::sort(smp.begin(), smp.end(), before);
    std::vector<Smp> spl;
    for (size_t i = every; i < smp.size(); i += every) spl.push_back(smp[i]);
    const size_t nb = spl.size() + 1;  // blocks
    std::vector<size_t> cut((nb + 1) * R);
    for (size_t r = 0; r < R; ++r) {
        const size_t off = r * chunk, len = std::min(chunk, n - off);
        cut[r] = 0;
        cut[nb * R + r] = len;
        for (size_t i = 0; i < spl.size(); ++i) {  // run-r elements ordered before splitter i
            size_t lo = 0, hi = len;
            while (lo < hi) {
                const size_t mid = lo + (hi - lo) / 2;
                if (before(Smp{tk[off + mid], off + mid}, spl[i]))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            cut[(i + 1) * R + r] = lo;
        }
    }
    *nb_out = nb;
    return cut;
}

template <class K, bool PAIRS>
static msort_status host_sort_external(msort_ctx* ctx, const K* h_kin, const uint32_t* h_vin, K* h_kout,
                                       uint32_t* h_vout, size_t n, const msort_options* opt, cudaStream_t st,
                                       int xform, size_t chunk) {
    HostPipe* hp = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        msort_status s = host_pipe_get(ctx, &hp);
        if (s != MSORT_OK) return s;
        const size_t need = n * sizeof(K) + (PAIRS ? n * 4 : 0);
        if (hp->runs_bytes < need) {
            // no copy of an earlier call (one that failed part-way included)
            // may still use the old buffer
            cudaError_t e = cudaStreamSynchronize(st);
            for (cudaStream_t q : {hp->h2d, hp->cs, hp->d2h})
                if (e == cudaSuccess) e = cudaStreamSynchronize(q);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            if (hp->runs) cudaFreeHost(hp->runs);
            hp->runs = nullptr;
            hp->runs_bytes = 0;
            if (cudaMallocHost(&hp->runs, need) != cudaSuccess) {
                cudaGetLastError();
                return fail(MSORT_ERR_OOM, "pinned host buffer for the sorted runs");
            }
            hp->runs_bytes = need;
        }
    }
    K* tk = static_cast<K*>(hp->runs);
    uint32_t* tv = PAIRS ? reinterpret_cast<uint32_t*>(tk + n) : nullptr;
    const size_t R = (n + chunk - 1) / chunk;
    // A block fills a staging slot (up to a chunk); its merge rounds
    // ping-pong between the slot and the context scratch, which phase 1
    // sized for the in-core sort of a chunk and which holds, after the
    // block's keys and values, the rounds' split table.  The largest block
    // whose share fits the scratch as it stands: larger blocks mean larger
    // slices, which the host link moves faster.
    auto scratch_for = [](size_t b) {
        return align_up(b * sizeof(K), 256) + (PAIRS ? align_up(b * 4, 256) : 0) +
               align_up(merge_runs_splits<K, PAIRS>(b) * sizeof(unsigned long long), 256);
    };
    if (2 * R > ((chunk / 2) & ~size_t(63)))
        return fail(MSORT_ERR_OOM, "the context budget is too small for this many out-of-core runs");

    // 1. sorted runs, one budget-sized chunk at a time (consecutive chunks
    //    overlap on the context's streams).  The runs keep their keys
    //    transformed (unsigned order); the last merge round undoes the
    //    transform.
    for (size_t r = 0; r < R; ++r) {
        const size_t off = r * chunk, len = std::min(chunk, n - off);
        msort_status s = host_sort<K, PAIRS>(ctx, h_kin + off, PAIRS ? h_vin + off : nullptr, tk + off,
                                             PAIRS ? tv + off : nullptr, len, opt, st, kAsyncChunks, kAsyncSlices,
                                             xform, true);
        if (s != MSORT_OK) return s;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");

    // the block size, now that phase 1 has sized the scratch
    size_t B = chunk & ~size_t(63);
    while (B > 64 && scratch_for(B) > ctx->scratch_bytes) B = (B - B / 16) & ~size_t(63);
    if (2 * R > B) return fail(MSORT_ERR_OOM, "the context budget is too small for this many out-of-core runs");

    // 2. splitters from regular samples of the runs
    size_t nb = 0;
    const std::vector<size_t> cut = external_cuts<K>(tk, n, chunk, B, &nb);

    // 3. every block: slices in, merged on the device, out, pipelined
    //    through the staging slots on the context's copy-in, compute and
    //    copy-out streams
    const size_t kb = align_up(B * sizeof(K), 256), vb = PAIRS ? align_up(B * 4, 256) : 0;
    int slots[kHostSlots], ns = 0;
    for (int i = 0; i < kHostSlots; ++i)
        if (hp->slot_bytes[i] >= kb + vb) slots[ns++] = i;
    if (!ns) return fail(MSORT_ERR_CUDA, "no staging slot holds an out-of-core block");
    K* pk = nullptr;  // the rounds' second buffer, in the scratch
    uint32_t* pv = nullptr;
    unsigned long long* splits = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        msort_status s = ensure_scratch(ctx, scratch_for(B), hp->cs);
        if (s != MSORT_OK) return s;
        unsigned char* sp = static_cast<unsigned char*>(ctx->scratch);
        pk = reinterpret_cast<K*>(sp);
        pv = PAIRS ? reinterpret_cast<uint32_t*>(sp + kb) : nullptr;
        splits = reinterpret_cast<unsigned long long*>(sp + kb + vb);
    }
    size_t out = 0, bi = 0;
    int last = -1;
    for (size_t b = 0; b < nb; ++b) {
        size_t len = 0;
        for (size_t r = 0; r < R; ++r) len += cut[(b + 1) * R + r] - cut[b * R + r];
        if (!len) continue;
        if (len > B) return fail(MSORT_ERR_CUDA, "out-of-core block larger than its bound");
        const int sl = slots[bi++ % ns];
        unsigned char* base = static_cast<unsigned char*>(hp->slot[sl]);
        K* dk[2] = {reinterpret_cast<K*>(base), pk};
        uint32_t* dv[2] = {PAIRS ? reinterpret_cast<uint32_t*>(base + kb) : nullptr, pv};
        if (hp->used[sl]) cudaStreamWaitEvent(hp->h2d, hp->done[sl], 0);  // its last block has left
        std::vector<size_t> ro(1, 0);  // boundaries of the block's non-empty slices
        for (size_t r = 0; r < R; ++r) {
            const size_t off = r * chunk, lo = cut[b * R + r], cnt = cut[(b + 1) * R + r] - lo;
            if (!cnt) continue;
            const size_t pos = ro.back();
            e = cudaMemcpyAsync(dk[0] + pos, tk + off + lo, cnt * sizeof(K), cudaMemcpyHostToDevice, hp->h2d);
            if (e == cudaSuccess && PAIRS)
                e = cudaMemcpyAsync(dv[0] + pos, tv + off + lo, cnt * 4, cudaMemcpyHostToDevice, hp->h2d);
            if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
            ro.push_back(pos + cnt);
        }
        cudaEventRecord(hp->in_ev[sl][0], hp->h2d);
        cudaStreamWaitEvent(hp->cs, hp->in_ev[sl][0], 0);
        // merge-tree rounds over the slices (at least one, which undoes the
        // key transform)
        int fin = 0;  // buffer that holds the block's result: 0 the slot, 1 the scratch
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            msort_status s;
            do {
                const bool lastr = ro.size() <= 3;
                s = merge_runs_round<K, PAIRS>(ctx, dk[fin], dk[fin ^ 1], dv[fin], dv[fin ^ 1], ro, splits,
                                               lastr ? xform : 0, hp->cs);
                if (s != MSORT_OK) return s;
                fin ^= 1;
            } while (ro.size() > 2);
            if (fin) {  // back into the slot: the next block's rounds reuse the scratch while this one is copied out
                e = cudaMemcpyAsync(dk[0], dk[1], len * sizeof(K), cudaMemcpyDeviceToDevice, hp->cs);
                if (e == cudaSuccess && PAIRS)
                    e = cudaMemcpyAsync(dv[0], dv[1], len * 4, cudaMemcpyDeviceToDevice, hp->cs);
                if (e != cudaSuccess) return cuda_fail(e, "copy of a merged block into its slot");
                fin = 0;
            }
        }
        cudaEventRecord(hp->out_ev[sl][0], hp->cs);
        cudaStreamWaitEvent(hp->d2h, hp->out_ev[sl][0], 0);
        e = cudaMemcpyAsync(h_kout + out, dk[fin], len * sizeof(K), cudaMemcpyDeviceToHost, hp->d2h);
        if (e == cudaSuccess && PAIRS)
            e = cudaMemcpyAsync(h_vout + out, dv[fin], len * 4, cudaMemcpyDeviceToHost, hp->d2h);
        if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
        cudaEventRecord(hp->done[sl], hp->d2h);
        hp->used[sl] = true;
        last = sl;
        out += len;
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        scratch_release(ctx, hp->cs);
    }
    if (last >= 0) cudaStreamWaitEvent(st, hp->done[last], 0);
    e = cudaStreamSynchronize(st);  // the caller's host output is complete on return
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return out == n ? MSORT_OK : fail(MSORT_ERR_CUDA, "out-of-core blocks did not cover the array");
}

// Host sort of n elements: in core when it fits the budget, else external.
template <class K, bool PAIRS>
static msort_status host_sort_any(msort_ctx* ctx, const void* h_kin, const uint32_t* h_vin, void* h_kout,
                                  uint32_t* h_vout, size_t n, const msort_options* opt, cudaStream_t st, int chunks,
                                  int slices, int xform, bool* synced) {
    *synced = false;
    if (ctx->budget) {
        Plan pl;
        std::string why;
        if (!make_plan<K, PAIRS>(n, opt, &pl, &why, xform)) return fail(MSORT_ERR_INVALID_ARG, why);
        if (host_incore_bytes<K, PAIRS>(n, pl) > ctx->budget) {
            const size_t chunk = external_chunk<K, PAIRS>(ctx->budget, opt, xform);
            if (!chunk) return fail(MSORT_ERR_OOM, "the context budget is too small even for out-of-core sorting");
            *synced = true;
            return host_sort_external<K, PAIRS>(ctx, static_cast<const K*>(h_kin), h_vin, static_cast<K*>(h_kout),
                                                h_vout, n, opt, st, xform, chunk);
        }
    }
    return host_sort<K, PAIRS>(ctx, h_kin, h_vin, h_kout, h_vout, n, opt, st, chunks, slices, xform);
}

// msort_merge_runs: rounds of the merge tree from d_in to out, the second
// buffer in scratch; round r writes out when rounds - 1 - r is even, so the
// last round lands in out and the input is only read.
template <class K, bool PAIRS>
static msort_status merge_runs_entry(msort_ctx* ctx, const K* in, const uint32_t* vin, std::vector<size_t> ro,
                                     K* out, uint32_t* vout, cudaStream_t st) {
    std::vector<size_t> nz(1, 0);  // drop empty runs
    for (size_t i = 1; i < ro.size(); ++i)
        if (ro[i] != nz.back()) nz.push_back(ro[i]);
    ro.swap(nz);
    const size_t n = ro.back();
    int rounds = 0;
    while (((size_t)1 << rounds) < ro.size() - 1) ++rounds;
    if (rounds == 0) rounds = 1;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const size_t kbytes = rounds > 1 ? align_up(n * sizeof(K), 256) : 0;
    const size_t vbytes = rounds > 1 && PAIRS ? align_up(n * 4, 256) : 0;
    msort_status s =
        ensure_scratch(ctx, kbytes + vbytes + merge_runs_splits<K, PAIRS>(n) * sizeof(unsigned long long), st);
    if (s != MSORT_OK) return s;
    unsigned char* sp = static_cast<unsigned char*>(ctx->scratch);
    K* tgt[2] = {out, reinterpret_cast<K*>(sp)};
    uint32_t* vtgt[2] = {vout, PAIRS ? reinterpret_cast<uint32_t*>(sp + kbytes) : nullptr};
    unsigned long long* splits = reinterpret_cast<unsigned long long*>(sp + kbytes + vbytes);
    const K* src = in;
    const uint32_t* vsrc = vin;
    for (int r = 0; r < rounds; ++r) {
        const int w = (rounds - 1 - r) & 1;
        s = merge_runs_round<K, PAIRS>(ctx, src, tgt[w], vsrc, vtgt[w], ro, splits, 0, st);
        if (s != MSORT_OK) break;
        src = tgt[w];
        vsrc = vtgt[w];
    }
    scratch_release(ctx, st);
    return s;
}

}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_ctx_create(int device, size_t budget, msort_ctx** out) {
    if (!out) return fail(MSORT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(MSORT_ERR_INVALID_ARG, "no such CUDA device");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    msort_ctx* c = new msort_ctx();
    c->device = device;
    c->budget = budget;
    if ((e = cudaEventCreateWithFlags(&c->scratch_done, cudaEventDisableTiming)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaEventCreate");
    }
    if ((e = cudaMalloc(&c->d_status, 256)) != cudaSuccess || (e = cudaMemset(c->d_status, 0, 256)) != cudaSuccess) {
        cudaEventDestroy(c->scratch_done);
        delete c;
        return cuda_fail(e, "status word");
    }
    *out = c;
    return MSORT_OK;
}

msort_status msort_ctx_destroy(msort_ctx* ctx) {
    if (!ctx) return MSORT_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    learned_destroy(ctx);
    graphs_destroy(ctx);
    if (ctx->scratch) cudaFree(ctx->scratch);
    host_pipe_destroy(ctx);
    plain_graphs_destroy(ctx);
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (auto& v : ctx->prof)
        for (auto& p : v) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    cudaEventDestroy(ctx->scratch_done);
    delete ctx;
    return MSORT_OK;
}

const char* msort_last_error(msort_ctx*) { return tl_error.c_str(); }

msort_status msort_ctx_sync(msort_ctx* ctx, void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st) {
        cudaMemset(ctx->d_status, 0, sizeof(unsigned int));
        if (st & DEV_TIMEOUT) return fail(MSORT_ERR_TIMEOUT, "a kernel gave up a bounded wait");
        if (st & DEV_INTERNAL) return fail(MSORT_ERR_CUDA, "a four-way merge block found inconsistent geometry");
        return fail(MSORT_ERR_INVALID_ARG, "a kernel rejected its input (status " + std::to_string(st) + ")");
    }
    return MSORT_OK;
}

size_t msort_scratch_bytes(size_t n, msort_key_type kt, int with_vals, const msort_options* opt) {
    const int kb = key_bytes(kt), xf = key_xform(kt);
    if (kb == 4)
        return with_vals ? scratch_bytes_for<uint32_t, true>(n, opt, xf) : scratch_bytes_for<uint32_t, false>(n, opt, xf);
    if (kb == 8)
        return with_vals ? scratch_bytes_for<uint64_t, true>(n, opt, xf) : scratch_bytes_for<uint64_t, false>(n, opt, xf);
    return 0;
}

msort_status msort_plan_passes(size_t n, msort_key_type kt, int with_vals, const msort_options* opt, int* ways,
                               int* memory_passes) {
    const int kb = key_bytes(kt), xf = key_xform(kt);
    if (kb == 4)
        return with_vals ? plan_passes_for<uint32_t, true>(n, opt, ways, memory_passes, xf)
                         : plan_passes_for<uint32_t, false>(n, opt, ways, memory_passes, xf);
    if (kb == 8)
        return with_vals ? plan_passes_for<uint64_t, true>(n, opt, ways, memory_passes, xf)
                         : plan_passes_for<uint64_t, false>(n, opt, ways, memory_passes, xf);
    return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
}

msort_status msort_plan_info(size_t n, msort_key_type kt, int with_vals, const msort_options* opt, int* tile,
                             int* merge_block, int* passes) {
    const int kb = key_bytes(kt), xf = key_xform(kt);
    if (kb == 4)
        return with_vals ? plan_info_for<uint32_t, true>(n, opt, tile, merge_block, passes, xf)
                         : plan_info_for<uint32_t, false>(n, opt, tile, merge_block, passes, xf);
    if (kb == 8)
        return with_vals ? plan_info_for<uint64_t, true>(n, opt, tile, merge_block, passes, xf)
                         : plan_info_for<uint64_t, false>(n, opt, tile, merge_block, passes, xf);
    return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
}

msort_status msort_sort_copy(msort_ctx* ctx, const void* kin, const uint32_t* vin, void* kout, uint32_t* vout,
                             size_t n, msort_key_type kt, const msort_options* opt, void* stream) {
    msort_status s = check_common(ctx, kt, opt);
    if (s != MSORT_OK) return s;
    if (n == 0) return MSORT_OK;
    if (!kin || !kout) return fail(MSORT_ERR_INVALID_ARG, "key pointer is NULL");
    if ((vin == nullptr) != (vout == nullptr)) return fail(MSORT_ERR_INVALID_ARG, "give both value pointers or none");
    const size_t ks = (size_t)key_bytes(kt);
    if ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(kout)) % ks ||
        (vin && ((reinterpret_cast<uintptr_t>(vin) | reinterpret_cast<uintptr_t>(vout)) & 3)))
        return fail(MSORT_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    cudaStream_t st = (cudaStream_t)stream;
    const int xf = key_xform(kt);
    if (ks == 4)
        return vin ? sort_entry<uint32_t, true>(ctx, kin, vin, kout, vout, n, opt, st, xf)
                   : sort_entry<uint32_t, false>(ctx, kin, nullptr, kout, nullptr, n, opt, st, xf);
    return vin ? sort_entry<uint64_t, true>(ctx, kin, vin, kout, vout, n, opt, st, xf)
               : sort_entry<uint64_t, false>(ctx, kin, nullptr, kout, nullptr, n, opt, st, xf);
}

msort_status msort_merge(msort_ctx* ctx, const void* d_a, const uint32_t* d_va, size_t na, const void* d_b,
                         const uint32_t* d_vb, size_t nb, void* d_out, uint32_t* d_vout, msort_key_type kt,
                         void* stream) {
    msort_status s = check_common(ctx, kt, nullptr);
    if (s != MSORT_OK) return s;
    if (key_xform(kt))
        return fail(MSORT_ERR_UNSUPPORTED, "msort_merge takes unsigned keys (signed and floating-point keys: "
                                           "the plain and host-buffer sorts)");
    if (na + nb == 0) return MSORT_OK;
    if ((na && !d_a) || (nb && !d_b) || !d_out) return fail(MSORT_ERR_INVALID_ARG, "key pointer is NULL");
    const bool pairs = d_vout != nullptr;
    if (pairs && ((na && !d_va) || (nb && !d_vb))) return fail(MSORT_ERR_INVALID_ARG, "value pointer is NULL");
    const size_t ks = kt == MSORT_U32 ? 4 : 8;
    const size_t W = kt == MSORT_U32 ? (pairs ? merge_two_block<uint32_t, true>() : merge_two_block<uint32_t, false>())
                                     : (pairs ? merge_two_block<uint64_t, true>() : merge_two_block<uint64_t, false>());
    const size_t nblocks = (na + nb + W - 1) / W;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    s = ensure_scratch(ctx, (nblocks + 1) * sizeof(unsigned long long), st);
    if (s != MSORT_OK) return s;
    unsigned long long* splits = static_cast<unsigned long long*>(ctx->scratch);
    cudaError_t e;
    if (kt == MSORT_U32) {
        const uint32_t* a = static_cast<const uint32_t*>(d_a);
        const uint32_t* b = static_cast<const uint32_t*>(d_b);
        uint32_t* o = static_cast<uint32_t*>(d_out);
        e = pairs ? launch_merge_two<uint32_t, true>(a, na, b, nb, d_va, d_vb, o, d_vout, splits, ctx->d_status, st)
                  : launch_merge_two<uint32_t, false>(a, na, b, nb, nullptr, nullptr, o, nullptr, splits,
                                                      ctx->d_status, st);
    } else {
        const uint64_t* a = static_cast<const uint64_t*>(d_a);
        const uint64_t* b = static_cast<const uint64_t*>(d_b);
        uint64_t* o = static_cast<uint64_t*>(d_out);
        e = pairs ? launch_merge_two<uint64_t, true>(a, na, b, nb, d_va, d_vb, o, d_vout, splits, ctx->d_status, st)
                  : launch_merge_two<uint64_t, false>(a, na, b, nb, nullptr, nullptr, o, nullptr, splits,
                                                      ctx->d_status, st);
    }
    ctx->launches += 2;
    scratch_release(ctx, st);
    if (e != cudaSuccess) return cuda_fail(e, ("merge launch" + last_launch_info()).c_str());
    (void)ks;
    return MSORT_OK;
}

size_t msort_external_plan(const void* h_runs, size_t n, msort_key_type kt, size_t chunk, size_t block_max,
                           uint64_t* h_cuts, size_t cuts_cap) {
    if (!h_runs || n == 0 || chunk == 0 || (kt != MSORT_U32 && kt != MSORT_U64)) return 0;
    const size_t R = (n + chunk - 1) / chunk;
    if (2 * R > block_max) return 0;
    size_t nb = 0;
    const std::vector<size_t> cut = kt == MSORT_U32
                                        ? external_cuts<uint32_t>(static_cast<const uint32_t*>(h_runs), n, chunk,
                                                                  block_max, &nb)
                                        : external_cuts<uint64_t>(static_cast<const uint64_t*>(h_runs), n, chunk,
                                                                  block_max, &nb);
    if (h_cuts && cuts_cap >= cut.size())
        for (size_t i = 0; i < cut.size(); ++i) h_cuts[i] = cut[i];
    return nb;
}

msort_status msort_merge_runs(msort_ctx* ctx, const void* d_keys, const uint32_t* d_vals, const uint64_t* offsets,
                              size_t nruns, void* d_out, uint32_t* d_vout, msort_key_type kt, void* stream) {
    msort_status s = check_common(ctx, kt, nullptr);
    if (s != MSORT_OK) return s;
    if (key_xform(kt))
        return fail(MSORT_ERR_UNSUPPORTED, "msort_merge_runs takes unsigned keys (signed and floating-point keys: "
                                           "the plain and host-buffer sorts)");
    if (nruns == 0) return MSORT_OK;
    if (!offsets) return fail(MSORT_ERR_INVALID_ARG, "offsets is NULL");
    if (offsets[0] != 0) return fail(MSORT_ERR_INVALID_ARG, "offsets[0] must be 0");
    std::vector<size_t> ro(nruns + 1);
    for (size_t i = 0; i <= nruns; ++i) {
        if (i && offsets[i] < offsets[i - 1]) return fail(MSORT_ERR_INVALID_ARG, "offsets must not decrease");
        ro[i] = (size_t)offsets[i];
    }
    const size_t n = ro[nruns];
    if (n == 0) return MSORT_OK;
    if (!d_keys || !d_out) return fail(MSORT_ERR_INVALID_ARG, "key pointer is NULL");
    if ((d_vals == nullptr) != (d_vout == nullptr)) return fail(MSORT_ERR_INVALID_ARG, "give both value pointers or none");
    const size_t ks = key_bytes(kt);
    const uintptr_t ki = reinterpret_cast<uintptr_t>(d_keys), ko = reinterpret_cast<uintptr_t>(d_out);
    if (ki < ko + n * ks && ko < ki + n * ks) return fail(MSORT_ERR_INVALID_ARG, "d_out overlaps d_keys");
    if (d_vals) {
        const uintptr_t vi = reinterpret_cast<uintptr_t>(d_vals), vo = reinterpret_cast<uintptr_t>(d_vout);
        if (vi < vo + n * 4 && vo < vi + n * 4) return fail(MSORT_ERR_INVALID_ARG, "d_vout overlaps d_vals");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (ks == 4)
        return d_vals ? merge_runs_entry<uint32_t, true>(ctx, static_cast<const uint32_t*>(d_keys), d_vals, ro,
                                                         static_cast<uint32_t*>(d_out), d_vout, st)
                      : merge_runs_entry<uint32_t, false>(ctx, static_cast<const uint32_t*>(d_keys), nullptr, ro,
                                                          static_cast<uint32_t*>(d_out), nullptr, st);
    return d_vals ? merge_runs_entry<uint64_t, true>(ctx, static_cast<const uint64_t*>(d_keys), d_vals, ro,
                                                     static_cast<uint64_t*>(d_out), d_vout, st)
                  : merge_runs_entry<uint64_t, false>(ctx, static_cast<const uint64_t*>(d_keys), nullptr, ro,
                                                      static_cast<uint64_t*>(d_out), nullptr, st);
}

msort_status msort_sort(msort_ctx* ctx, void* d_keys, size_t n, msort_key_type kt, const msort_options* opt,
                        void* stream) {
    return msort_sort_copy(ctx, d_keys, nullptr, d_keys, nullptr, n, kt, opt, stream);
}

msort_status msort_sort_pairs(msort_ctx* ctx, void* d_keys, uint32_t* d_vals, size_t n, msort_key_type kt,
                              const msort_options* opt, void* stream) {
    if (n && !d_vals) return fail(MSORT_ERR_INVALID_ARG, "d_vals is NULL");
    return msort_sort_copy(ctx, d_keys, d_vals, d_keys, d_vals, n, kt, opt, stream);
}

static msort_status host_sort_call(msort_ctx* ctx, const void* h_kin, const uint32_t* h_vin, void* h_kout,
                                   uint32_t* h_vout, size_t n, msort_key_type kt, const msort_options* opt,
                                   void* stream, bool wait) {
    msort_status s = check_common(ctx, kt, opt);
    if (s != MSORT_OK) return s;
    if (n == 0) return MSORT_OK;
    if (!h_kin || !h_kout) return fail(MSORT_ERR_INVALID_ARG, "host key pointer is NULL");
    if ((h_vin == nullptr) != (h_vout == nullptr)) return fail(MSORT_ERR_INVALID_ARG, "give both value pointers or none");
    cudaStream_t st = (cudaStream_t)stream;
    const int ch = wait ? kSyncChunks : kAsyncChunks, sl = wait ? kSyncSlices : kAsyncSlices;
    const int xf = key_xform(kt);
    bool synced = false;
    if (key_bytes(kt) == 4)
        s = h_vin ? host_sort_any<uint32_t, true>(ctx, h_kin, h_vin, h_kout, h_vout, n, opt, st, ch, sl, xf, &synced)
                  : host_sort_any<uint32_t, false>(ctx, h_kin, nullptr, h_kout, nullptr, n, opt, st, ch, sl, xf,
                                                   &synced);
    else
        s = h_vin ? host_sort_any<uint64_t, true>(ctx, h_kin, h_vin, h_kout, h_vout, n, opt, st, ch, sl, xf, &synced)
                  : host_sort_any<uint64_t, false>(ctx, h_kin, nullptr, h_kout, nullptr, n, opt, st, ch, sl, xf,
                                                   &synced);
    if (s != MSORT_OK) {
        host_pipe_drain(ctx);
        return s;
    }
    if (!wait || synced) return s;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return MSORT_OK;
}

msort_status msort_sort_host(msort_ctx* ctx, const void* h_kin, const uint32_t* h_vin, void* h_kout,
                             uint32_t* h_vout, size_t n, msort_key_type kt, const msort_options* opt, void* stream) {
    return host_sort_call(ctx, h_kin, h_vin, h_kout, h_vout, n, kt, opt, stream, true);
}

msort_status msort_sort_host_async(msort_ctx* ctx, const void* h_kin, const uint32_t* h_vin, void* h_kout,
                                   uint32_t* h_vout, size_t n, msort_key_type kt, const msort_options* opt,
                                   void* stream) {
    return host_sort_call(ctx, h_kin, h_vin, h_kout, h_vout, n, kt, opt, stream, false);
}

msort_status msort_ctx_set_profiling(msort_ctx* ctx, int on) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->profiling = on != 0;
    ctx->count_probes = on >= 2;
    for (auto& u : ctx->prof_used) u = 0;
    return MSORT_OK;
}

msort_status msort_ctx_kernel_log(msort_ctx* ctx, int kind, double* h_ms, size_t cap, uint64_t* launches) {
    if (!ctx || kind < 0 || kind >= KK_COUNT || !launches || (cap && !h_ms))
        return fail(MSORT_ERR_INVALID_ARG, "bad argument to msort_ctx_kernel_log");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    const size_t used = ctx->prof_used[kind];
    for (size_t i = 0; i < used; ++i) {
        const EventPair& p = ctx->prof[kind][i];
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        if (i < cap) h_ms[i] = ms;
    }
    *launches = used;
    ctx->prof_used[kind] = 0;
    return MSORT_OK;
}

msort_status msort_ctx_kernel_times(msort_ctx* ctx, int kind, uint64_t* launches, double* total_ms) {
    if (!ctx || kind < 0 || kind >= KK_COUNT || !launches || !total_ms)
        return fail(MSORT_ERR_INVALID_ARG, "bad argument to msort_ctx_kernel_times");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    double tot = 0.0;
    const size_t used = ctx->prof_used[kind];
    for (size_t i = 0; i < used; ++i) {
        const EventPair& p = ctx->prof[kind][i];
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        tot += ms;
    }
    *launches = used;
    *total_ms = tot;
    ctx->prof_used[kind] = 0;
    return MSORT_OK;
}

unsigned long long msort_ctx_launch_count(msort_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
