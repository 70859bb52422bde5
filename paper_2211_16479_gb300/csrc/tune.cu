// Autotuner: picks the tile shape (threads x keys per thread, hence tile
// size and merge-block size) of the plain sort per key type, value presence
// and size class, the merge fan-in (two-way or four-way passes) for 32-bit
// keys without values, and the bucket shapes of the segmented sort of 32-bit
// keys, by timing every candidate on this GPU.  Every candidate's output is
// compared bit for bit with the first candidate's before its time counts;
// a candidate that disagrees is rejected.  Results live in the context and
// can be written to / read from a small cache file.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace msort {
namespace {

__device__ __forceinline__ uint64_t tmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class K>
__global__ void k_fill(K* keys, uint32_t* vals, size_t n, uint64_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        keys[i] = (K)tmix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
        if (vals) vals[i] = (uint32_t)i;
    }
}

__global__ void k_count_diff(const unsigned char* a, const unsigned char* b, size_t bytes,
                             unsigned long long* diff) {
    unsigned long long local = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += (size_t)gridDim.x * blockDim.x)
        local += a[i] != b[i];
    if (local) atomicAdd(diff, local);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

bool same_bytes(const void* a, const void* b, size_t bytes, unsigned long long* d_diff) {
    cudaMemset(d_diff, 0, sizeof(unsigned long long));
    k_count_diff<<<1024, 256>>>(static_cast<const unsigned char*>(a), static_cast<const unsigned char*>(b), bytes,
                                d_diff);
    unsigned long long h = 1;
    cudaMemcpy(&h, d_diff, sizeof(h), cudaMemcpyDeviceToHost);
    return h == 0;
}

template <class F>
float time_ms(F&& fn, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fn();
    cudaEventRecord(a);
    for (int i = 0; i < reps; ++i) fn();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / reps;
}

const int kTiles[] = {4352, 8448, 8704, 16896, 33792};

}  // namespace
}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_tune(msort_ctx* ctx, const char* cache_path, int quick) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    const std::vector<int> classes = quick ? std::vector<int>{20} : std::vector<int>{16, 20, 24};
    const size_t nmax = ((size_t)1 << classes.back()) + 4097;
    DevBuf kin, vin, kout, vout, kref, vref, diff;
    if (cudaMalloc(&kin.p, nmax * 8) || cudaMalloc(&vin.p, nmax * 4) || cudaMalloc(&kout.p, nmax * 8) ||
        cudaMalloc(&vout.p, nmax * 4) || cudaMalloc(&kref.p, nmax * 8) || cudaMalloc(&vref.p, nmax * 4) ||
        cudaMalloc(&diff.p, 8)) {
        cudaGetLastError();
        return fail(MSORT_ERR_OOM, "tuning buffers");
    }
    auto* d_diff = static_cast<unsigned long long*>(diff.p);
    std::string log = "{\n  \"plain\": [\n";
    bool first_line = true;
    for (int kt = 0; kt < 2; ++kt) {
        const size_t ks = kt == 0 ? 4 : 8;
        for (int pairs = 0; pairs < 2; ++pairs) {
            for (int cls : classes) {
                const size_t n = ((size_t)1 << cls) + 4097;
                if (kt == 0)
                    k_fill<uint32_t><<<1024, 256>>>(static_cast<uint32_t*>(kin.p), static_cast<uint32_t*>(vin.p), n,
                                                    1234 + cls);
                else
                    k_fill<uint64_t><<<1024, 256>>>(static_cast<uint64_t*>(kin.p), static_cast<uint32_t*>(vin.p), n,
                                                    1234 + cls);
                int best_tile = 0, best_ways = 2;
                float best_ms = 1e30f;
                bool have_ref = false;
                std::string times;
                const bool four = kt == 0 && !pairs;  // four-way passes: 32-bit keys without values
                for (int tile : kTiles)
                for (int ways : {2, 4}) {
                    if (ways == 4 && !four) continue;
                    msort_options o{};
                    o.tile = tile;
                    o.merge_ways = ways;
                    if (msort_scratch_bytes(n, (msort_key_type)kt, pairs, &o) == 0) continue;  // not offered
                    auto run = [&] {
                        msort_sort_copy(ctx, kin.p, pairs ? static_cast<uint32_t*>(vin.p) : nullptr, kout.p,
                                        pairs ? static_cast<uint32_t*>(vout.p) : nullptr, n, (msort_key_type)kt, &o,
                                        nullptr);
                    };
                    const float ms = time_ms(run, 3);
                    if (cudaGetLastError() != cudaSuccess) continue;
                    bool ok = true;
                    if (!have_ref) {
                        cudaMemcpy(kref.p, kout.p, n * ks, cudaMemcpyDeviceToDevice);
                        if (pairs) cudaMemcpy(vref.p, vout.p, n * 4, cudaMemcpyDeviceToDevice);
                        have_ref = true;
                    } else {
                        ok = same_bytes(kref.p, kout.p, n * ks, d_diff) &&
                             (!pairs || same_bytes(vref.p, vout.p, n * 4, d_diff));
                    }
                    char buf[64];
                    std::snprintf(buf, sizeof buf, "%s\"%d%s\": %.4f", times.empty() ? "" : ", ", tile,
                                  ways == 4 ? "x4" : "", ok ? ms : -1.f);
                    times += buf;
                    if (ok && ms < best_ms) {
                        best_ms = ms;
                        best_tile = tile;
                        best_ways = ways;
                    }
                }
                if (best_tile) {
                    ctx->tuned_tile[std::make_tuple((int)ks, pairs, cls)] = best_tile;
                    if (four) ctx->tuned_ways[std::make_tuple((int)ks, pairs, cls)] = best_ways;
                }
                char line[640];
                std::snprintf(line, sizeof line,
                              "%s    {\"key_bytes\": %zu, \"values\": %d, \"log2n\": %d, \"tile\": %d, \"ways\": %d, "
                              "\"ms\": {%s}}",
                              first_line ? "" : ",\n", ks, pairs, cls, best_tile, best_ways, times.c_str());
                log += line;
                first_line = false;
            }
        }
    }
    log += "\n  ],\n";

    // Segmented sort of 32-bit keys: 4000 segments, lengths log-uniform in [1, 65536].
    {
        const size_t nseg = 4000;
        std::vector<unsigned long long> off(nseg + 1, 0);
        uint64_t x = 99;
        for (size_t i = 0; i < nseg; ++i) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            const double u = (double)(x >> 11) * (1.0 / 9007199254740992.0);
            size_t len = (size_t)std::floor(std::exp(u * std::log(65537.0)));
            len = len < 1 ? 1 : (len > 65536 ? 65536 : len);
            off[i + 1] = off[i] + len;
        }
        const size_t n = off[nseg];
        DevBuf src, work, doff, ref;
        if (cudaMalloc(&src.p, n * 4) || cudaMalloc(&work.p, n * 4) || cudaMalloc(&doff.p, (nseg + 1) * 8) ||
            cudaMalloc(&ref.p, n * 4)) {
            cudaGetLastError();
            return fail(MSORT_ERR_OOM, "tuning buffers");
        }
        cudaMemcpy(doff.p, off.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice);
        k_fill<uint32_t><<<1024, 256>>>(static_cast<uint32_t*>(src.p), nullptr, n, 77);
        const int smalls[] = {33792, 16896};
        const int larges[] = {16896, 8448};
        float best = 1e30f;
        int bs = 0, bl = 0;
        bool have_ref = false;
        std::string times;
        for (int sm : smalls)
            for (int lg : larges) {
                ctx->seg_max_small = sm;
                ctx->seg_large_tile = lg;
                auto run = [&] {
                    cudaMemcpyAsync(work.p, src.p, n * 4, cudaMemcpyDeviceToDevice, nullptr);
                    msort_segmented_sort(ctx, work.p, nullptr, static_cast<const uint64_t*>(doff.p), nseg, n,
                                         MSORT_U32, nullptr, nullptr);
                };
                const float ms = time_ms(run, 3);
                bool ok = cudaGetLastError() == cudaSuccess;
                if (ok && !have_ref) {
                    cudaMemcpy(ref.p, work.p, n * 4, cudaMemcpyDeviceToDevice);
                    have_ref = true;
                } else if (ok) {
                    ok = same_bytes(ref.p, work.p, n * 4, d_diff);
                }
                char buf[96];
                std::snprintf(buf, sizeof buf, "%s\"%d/%d\": %.4f", times.empty() ? "" : ", ", sm, lg, ok ? ms : -1.f);
                times += buf;
                if (ok && ms < best) {
                    best = ms;
                    bs = sm;
                    bl = lg;
                }
            }
        ctx->seg_max_small = bs;
        ctx->seg_large_tile = bl;
        char line[512];
        std::snprintf(line, sizeof line, "  \"segmented_u32\": {\"max_small\": %d, \"large_tile\": %d, \"ms\": {%s}}\n}\n",
                      bs, bl, times.c_str());
        log += line;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "tuning");
    if (cache_path && *cache_path) {
        FILE* f = std::fopen(cache_path, "w");
        if (!f) return fail(MSORT_ERR_INVALID_ARG, std::string("cannot write ") + cache_path);
        std::fputs(log.c_str(), f);
        std::fclose(f);
    }
    return MSORT_OK;
}

msort_status msort_tune_load(msort_ctx* ctx, const char* cache_path) {
    if (!ctx || !cache_path) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    FILE* f = std::fopen(cache_path, "r");
    if (!f) return fail(MSORT_ERR_INVALID_ARG, std::string("cannot read ") + cache_path);
    char line[1024];
    int loaded = 0;
    while (std::fgets(line, sizeof line, f)) {
        int kb = 0, v = 0, lg = 0, tile = 0, ways = 0;
        const char* p = std::strstr(line, "\"key_bytes\"");
        const int got = p ? std::sscanf(p, "\"key_bytes\": %d, \"values\": %d, \"log2n\": %d, \"tile\": %d, \"ways\": %d",
                                        &kb, &v, &lg, &tile, &ways)
                          : 0;
        if (got >= 4) {
            if (tile) {
                ctx->tuned_tile[std::make_tuple(kb, v, lg)] = tile;
                if (got == 5 && kb == 4 && v == 0 && (ways == 2 || ways == 4))
                    ctx->tuned_ways[std::make_tuple(kb, v, lg)] = ways;
                ++loaded;
            }
            continue;
        }
        p = std::strstr(line, "\"segmented_u32\"");
        int sm = 0, lt = 0;
        if (p && std::sscanf(p, "\"segmented_u32\": {\"max_small\": %d, \"large_tile\": %d", &sm, &lt) == 2) {
            ctx->seg_max_small = sm;
            ctx->seg_large_tile = lt;
            ++loaded;
        }
    }
    std::fclose(f);
    return loaded ? MSORT_OK : fail(MSORT_ERR_INVALID_ARG, "no tuning entries in the cache file");
}

msort_status msort_tune_clear(msort_ctx* ctx) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    ctx->tuned_tile.clear();
    ctx->tuned_ways.clear();
    ctx->seg_max_small = 0;
    ctx->seg_large_tile = 0;
    return MSORT_OK;
}

}  // extern "C"
