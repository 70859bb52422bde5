// Host-side context shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/msort.h"

namespace msort {

enum KernelKind { KK_TILE = 0, KK_PARTITION = 1, KK_MERGE = 2, KK_SEGMENTED = 3, KK_MLP = 4, KK_SINGLE = 5, KK_COUNT = 6 };

// Status bits a kernel may raise in the context's device status word.
enum : unsigned int { DEV_OK = 0, DEV_TIMEOUT = 1u, DEV_BAD_INPUT = 2u, DEV_INTERNAL = 4u };

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

struct Plan {
    int tile;       // keys per tile sort block
    int W;          // outputs per merge block
    int passes;     // merge passes after the tile sort
    int partition_mode;
    int learned_passes;
    int ways;   // 2: one merge round per pass; 4: two rounds per pass (four-way)
    int W4;     // outputs per four-way merge block
    int G4;     // grid step of the four-way partition
    int xform;  // key transform: 0 unsigned keys, 1 signed integers, 2 IEEE floating point
    int xform_out;  // transform the last round undoes: xform, or 0 to leave the keys transformed
    int single;     // 1: the whole sort in one cooperative launch (csrc/small.cuh)
    unsigned int* status;  // device status word of the context
};

}  // namespace msort

struct msort_ctx {
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    void* host_pipe = nullptr;  // msort_sort_host staging slots, copy streams and events (msort.cu)
    size_t staging_bytes = 0;   // device bytes those slots hold
    unsigned int* d_status = nullptr;
    cudaEvent_t scratch_done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool scratch_pending = false;
    bool profiling = false;
    bool count_probes = false;  // profiling level 2: guided partitions count their probes
    std::vector<msort::EventPair> prof[msort::KK_COUNT];
    size_t prof_used[msort::KK_COUNT] = {};
    unsigned long long launches = 0;
    std::mutex mu;
    // learned partitioner state (owned by learned.cu)
    void* learned = nullptr;
    // graph cache (owned by segmented.cu)
    void* graphs = nullptr;
    // graph cache of plain sorts (owned by msort.cu)
    void* plain_graphs = nullptr;
    // autotuned choices (msort_tune): (key bytes, values, log2 size class) -> tile
    std::map<std::tuple<int, int, int>, int> tuned_tile;
    // merge fan-in (2 or 4) of the same classes; tuned for unsigned keys only
    std::map<std::tuple<int, int, int>, int> tuned_ways;
    // segmented sort of 32-bit keys: largest on-chip bucket and large-segment tile (0 = default)
    int seg_max_small = 0;
    int seg_large_tile = 0;
};

namespace msort {

msort_status fail(msort_status s, const std::string& msg);
msort_status cuda_fail(cudaError_t e, const char* what);
// Make sure ctx->scratch holds at least `bytes`; orders the caller's stream
// after the previous scratch user.
msort_status ensure_scratch(msort_ctx* ctx, size_t bytes, cudaStream_t st);
// Profiling helpers around one launch of kind `k` on stream st.
void prof_begin(msort_ctx* ctx, int k, cudaStream_t st);
void prof_end(msort_ctx* ctx, int k, cudaStream_t st);
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace msort
