/*
 * msort -- stable GPU merge sort for sm_103a (GB300), C ABI.
 *
 * The method is the divide-and-conquer merge sort of arXiv 2211.16479
 * ("Approaches to the Parallelization of Merge Sort in Python"): sort
 * fixed-size chunks independently (Section "Multiprocessing Merge Sort",
 * Figs. 6-7, where each chunk of ceil(n/p) elements goes to one worker), then
 * merge sorted runs pairwise, round after round, until one run is left
 * (Section "MPI Merge Sort", Figs. 16-17).  Here a chunk is a tile of T keys
 * sorted by one thread block, and a round is one global merge pass over the
 * whole array, so ceil(log2(ceil(n / T))) passes follow the tile sort.  The
 * merge takes from the left run on ties (Section "Sequential Merge Sort"
 * leaves merge() undefined; this is the stable reading), so every sort here
 * is stable.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers on the context's device; h_*
 *    are host pointers (pinned memory gives the fastest copies).  The caller
 *    owns every buffer it passes; the library never frees them.
 *  - Keys are 32- or 64-bit unsigned or signed integers or IEEE floats
 *    (msort_key_type, ordered as described there).  Values are optional
 *    uint32 words that travel with their key.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it and the call returns without
 *    waiting, except where a function says it synchronises.
 *  - Return value: MSORT_OK, or an error code; msort_last_error() gives a
 *    message for the calling thread's last failure on that context.  Invalid
 *    arguments are rejected before any work is enqueued.  n == 0 and
 *    nseg == 0 are valid and do nothing.
 *  - Scratch memory (a second key/value buffer of n elements plus a small
 *    split table) belongs to the context and is reused; calls on one context
 *    are ordered by the context itself (a call on a new stream waits for the
 *    previous call's scratch use).  Use one context per thread for
 *    concurrent host threads.
 */
#ifndef MSORT_H_
#define MSORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSORT_OK = 0,
    MSORT_ERR_INVALID_ARG = 1,
    MSORT_ERR_UNSUPPORTED = 2,
    MSORT_ERR_OOM = 3,
    MSORT_ERR_CUDA = 4,
    MSORT_ERR_TIMEOUT = 5,
    MSORT_ERR_BUSY = 6
} msort_status;

/* Key types.  Unsigned keys compare as unsigned integers; signed keys as
 * two's-complement integers; floating-point keys by the IEEE 754 totalOrder
 * relation: -NaN < -inf < negative numbers < -0 < +0 < positive numbers <
 * +inf < +NaN, NaNs ordered among themselves by payload (their bit pattern),
 * so every bit pattern has one place and equal bit patterns keep their input
 * order.  Signed and floating-point keys are accepted by msort_sort,
 * msort_sort_pairs, msort_sort_copy, msort_sort_host(_async),
 * msort_segmented_sort, msort_scratch_bytes and the plan queries, with
 * partition_mode 0 and pairwise passes; msort_merge, msort_merge_runs, msort_sort_noalloc and
 * the server return MSORT_ERR_UNSUPPORTED for them.  They are sorted as unsigned keys after an order-preserving bit
 * transform that the tile sort applies as it reads the input and the last
 * merge round undoes as it writes the output (no extra pass over memory). */
typedef enum {
    MSORT_U32 = 0,
    MSORT_U64 = 1,
    MSORT_I32 = 2,
    MSORT_I64 = 3,
    MSORT_F32 = 4,
    MSORT_F64 = 5
} msort_key_type;

typedef struct msort_ctx msort_ctx;

/* Tuning knobs; a zeroed struct (or NULL) selects the defaults. */
typedef struct {
    int tile;           /* keys per tile-sort block: 0 = default (or tuned), else 4352
                           (256 x 17), 8448 (256 x 33), 8704 (512 x 17), 16896 (512 x 33)
                           or 33792 (1024 x 33, 32-bit keys without values only); 16896 is
                           not available for 64-bit key-value sorts */
    int merge_block;    /* outputs per merge block: 0, or the value the tile implies
                           (4352 for tiles of 17 keys per thread, 8448 for 33) */
    int partition_mode; /* 0 = exact merge-path binary search; 1 = learned CDF predictor
                           (window verified, exact search inside, so the result is the same;
                           the network is trained on a key sample on a second stream while the
                           sort runs, and partitions that start before its training has finished
                           use the ratio guess of mode 2 instead of waiting; at profiling level 2
                           they wait for it);
                           2 = ratio guess d*|A|/(|A|+|B|) with the same verification
                           (the learned mode without its model, for comparison);
                           3 = exact binary search in the guided kernel (diagnostics: its
                           probes are counted like modes 1 and 2) */
    int learned_passes; /* with modes 1/2: how many final passes use the guided search;
                           0 = the passes whose runs hold >= 2^22 keys */
    int use_graph;      /* 1 = replay the launch sequence from a CUDA graph captured on the first
                           call with the same buffers, size and plan (plain sorts with
                           partition_mode 0, and segmented sorts); removes the per-launch
                           host cost that dominates small sorts.  A context keeps up to 64
                           graphs of each kind; a new one evicts the least recently used,
                           after a device synchronisation */
    int merge_ways;     /* merge rounds per pass over memory: 0 = default (2); 2 = one round
                           of the pairwise merge tree per pass; 4 = two rounds per pass (four
                           runs merged at once; keys-only sorts with partition_mode 0; half
                           the HBM traffic of the merge phase but slower on GB300, where the
                           pairwise pass runs at the copy bandwidth) */
    int single_launch;  /* 0 = automatic: msort_sort, msort_sort_pairs and msort_sort_copy
                           sort arrays of up to 2^22 elements by one cooperative launch that
                           runs the tile sort and every merge round, with a grid barrier
                           between rounds (such arrays stay in L2, where launch cost
                           dominates), when tile, merge_block and partition_mode are 0 and
                           passes are pairwise; its tile (= merge block) follows n: 4352,
                           8704 or 16896 for 32-bit keys alone, 2816 then 8448 (4352 for
                           64-bit key-value pairs) otherwise.  1 = that single launch up to
                           2^28 elements (same conditions, except that tile may name one of
                           its shapes: 2816, 4352, 5632, 8448, 8704, 11264 or 16896 for 32-bit
                           keys alone, 2816 and 8448 (4352 for 64-bit pairs) otherwise).
                           -1 = never.  If the device refuses the cooperative grid, the sort
                           runs the multi-launch plan instead (same result).  The host-buffer,
                           segmented and serving paths always use the multi-launch plan */
    int reserved[1];    /* must be zero */
} msort_options;

/* Context on CUDA device `device`.  scratch_budget_bytes caps the scratch the
 * context may hold (0 = no cap); a sort that needs more fails with
 * MSORT_ERR_OOM and enqueues nothing.  The host-buffer sorts instead switch to
 * an out-of-core sort that stays within the cap (see msort_sort_host). */
msort_status msort_ctx_create(int device, size_t scratch_budget_bytes, msort_ctx** out);
/* Waits for the context's outstanding work, frees its scratch and itself. */
msort_status msort_ctx_destroy(msort_ctx* ctx);
/* Message for the calling thread's last failing call on ctx ("" if none). */
const char* msort_last_error(msort_ctx* ctx);
/* Waits for `stream`, then reports any error a kernel recorded in the
 * context's device status word (MSORT_ERR_TIMEOUT for a bounded wait that
 * gave up) and clears it. */
msort_status msort_ctx_sync(msort_ctx* ctx, void* stream);

/* Bytes of scratch a sort of n elements needs (tile sort buffer + splits);
 * 0 if the options are invalid for this key/value type. */
size_t msort_scratch_bytes(size_t n, msort_key_type kt, int with_vals, const msort_options* opt);

/* The plan a sort of n elements would use: keys per tile, outputs per merge
 * block and number of merge passes (any output pointer may be NULL). */
msort_status msort_plan_info(size_t n, msort_key_type kt, int with_vals, const msort_options* opt, int* tile,
                             int* merge_block, int* passes);

/* How the plan's merge rounds map to passes over memory: *ways = 2 (one
 * round of the merge tree per pass) or 4 (two rounds per pass, four runs
 * merged at once), *memory_passes = the merge passes that read and write
 * every element once (rounds for ways = 2; rounds / 2 plus one pairwise pass
 * when rounds is odd, for ways = 4).  Either pointer may be NULL. */
msort_status msort_plan_passes(size_t n, msort_key_type kt, int with_vals, const msort_options* opt, int* ways,
                               int* memory_passes);

/* In-place stable sort of d_keys[0:n). */
msort_status msort_sort(msort_ctx* ctx, void* d_keys, size_t n, msort_key_type kt,
                        const msort_options* opt, void* stream);

/* In-place stable sort of (d_keys, d_vals)[0:n) by key. */
msort_status msort_sort_pairs(msort_ctx* ctx, void* d_keys, uint32_t* d_vals, size_t n,
                              msort_key_type kt, const msort_options* opt, void* stream);

/* Out-of-place stable sort: d_keys_in (and d_vals_in) are only read, the
 * result goes to d_keys_out (and d_vals_out).  d_vals_in/d_vals_out are both
 * NULL for a keys-only sort.  Each output is either the same buffer as its
 * input (an in-place sort, which msort_sort and msort_sort_pairs are) or
 * does not overlap it; a partial overlap gives undefined results. */
msort_status msort_sort_copy(msort_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                             void* d_keys_out, uint32_t* d_vals_out, size_t n, msort_key_type kt,
                             const msort_options* opt, void* stream);

/* Batched segmented sort, in place: each segment [d_offsets[i],
 * d_offsets[i+1]) of d_keys (and d_vals, nullable) is sorted on its own,
 * stably.  d_offsets holds nseg + 1 nondecreasing uint64 offsets with
 * d_offsets[0] = 0 and d_offsets[nseg] = n (the total key count).  The
 * offsets are checked on the device: malformed offsets leave the keys
 * untouched and make the next msort_ctx_sync return MSORT_ERR_INVALID_ARG.
 * Segments are bucketed by length on the device and each bucket is sorted
 * by one persistent launch, so the call never synchronises; with
 * opt->use_graph the whole launch sequence is captured once per
 * (buffers, sizes) and replayed from a CUDA graph afterwards.
 * (Segmented sorting is the paper's method applied per array; the paper
 * itself sorts one array.) */
msort_status msort_segmented_sort(msort_ctx* ctx, void* d_keys, uint32_t* d_vals, const uint64_t* d_offsets,
                                  size_t nseg, size_t n, msort_key_type kt, const msort_options* opt,
                                  void* stream);

/* Stable merge of two sorted arrays: d_out[0:na+nb) = merge(d_a[0:na),
 * d_b[0:nb)), equal keys taking from d_a first (one round of the paper's
 * merge tree, Section "MPI Merge Sort", Figs. 16-17).  d_vout non-NULL merges
 * values alongside (d_va, d_vb required).  The output must not overlap the
 * inputs.  Scratch: the context's split table. */
msort_status msort_merge(msort_ctx* ctx, const void* d_a, const uint32_t* d_va, size_t na, const void* d_b,
                         const uint32_t* d_vb, size_t nb, void* d_out, uint32_t* d_vout, msort_key_type kt,
                         void* stream);

/* Stable merge of nruns sorted runs laid end to end: run i of d_keys (and
 * d_vals) is [offsets[i], offsets[i+1]), where offsets is a host array of
 * nruns + 1 non-decreasing element counts starting at 0; empty runs are
 * allowed.  The merged array (equal keys in run order, values alongside)
 * goes to d_out (and d_vout; give both value pointers or neither), which must
 * not overlap the input.  It runs ceil(log2(non-empty runs)) rounds of the
 * pairwise merge tree (Section "MPI Merge Sort", "Merging the subarrays",
 * Figs. 16-17: one round merges runs 2j and 2j + 1 for every j), each a partition and a merge launch per 32
 * pairs; a second buffer of offsets[nruns] elements comes from the
 * context's scratch.  Unsigned key types only (MSORT_ERR_UNSUPPORTED for the
 * others); MSORT_ERR_INVALID_ARG for decreasing offsets or overlapping
 * buffers.  The runs must be sorted (not checked). */
msort_status msort_merge_runs(msort_ctx* ctx, const void* d_keys, const uint32_t* d_vals, const uint64_t* offsets,
                              size_t nruns, void* d_out, uint32_t* d_vout, msort_key_type kt, void* stream);

/* Cuts of one rank's sorted chunk for the one-exchange multi-GPU sort.  The
 * paper's message-passing sort scatters the array into one subarray per
 * process and merges the sorted subarrays up a tree (Section "MPI Merge
 * Sort", Figs. 16-17); the one-exchange form instead sends every element
 * once, to the rank owning its key range, with p - 1 splitters taken from
 * regular samples of all chunks.  Elements are ordered by (key, global input
 * position), a total order, so that splitters cut runs of equal keys and
 * rank r receives exactly the r-th slice of the stable sort.
 *   d_keys[0:n)     the chunk's keys, stably sorted (unsigned, kt MSORT_U32
 *                   or MSORT_U64; others give MSORT_ERR_UNSUPPORTED)
 *   d_idx[0:n)      each sorted key's index in the unsorted chunk (the values
 *                   of a key-value sort whose values were 0..n-1), so its
 *                   global position is offset + d_idx[i]
 *   d_split_keys / d_split_pos [0:nsplit)   the splitters (key of type kt,
 *                   uint64 global position), in any order
 *   d_cuts[0:nsplit) (output, uint64) for each splitter, the number of chunk
 *                   elements ordered before it: keys below it, plus equal
 *                   keys at a smaller global position.
 * One binary search per splitter on `stream`; n <= 2^32 - 1. */
msort_status msort_split_points(msort_ctx* ctx, const void* d_keys, const uint32_t* d_idx, size_t n,
                                uint64_t offset, const void* d_split_keys, const uint64_t* d_split_pos,
                                size_t nsplit, uint64_t* d_cuts, msort_key_type kt, void* stream);

/* Merge blocks the out-of-core sort (msort_sort_host) uses, computed on the
 * host: h_runs holds n unsigned keys (kt MSORT_U32 or MSORT_U64) as
 * R = ceil(n / chunk) sorted runs of `chunk` keys laid end to end (the last
 * may be shorter).  Returns the number of blocks nb (0 for invalid
 * arguments or block_max < 2R) and, when cuts_cap >= (nb + 1) * R, fills
 * h_cuts[b * R + r] with the number of run r's keys ordered before block b
 * (b = 0..nb), ordering keys by (value, position in h_runs): block b takes
 * [h_cuts[b*R + r], h_cuts[(b+1)*R + r]) of every run r, and holds at most
 * block_max keys.  Pure host code; needs no GPU. */
size_t msort_external_plan(const void* h_runs, size_t n, msort_key_type kt, size_t chunk, size_t block_max,
                           uint64_t* h_cuts, size_t cuts_cap);

/* Host-buffer sort: copies h_keys_in (and h_vals_in, nullable) to the
 * device, sorts there, and copies the result to h_keys_out (and h_vals_out;
 * give both value pointers or neither).  Output may be the same buffer as
 * input.  Pinned host memory is fastest; pageable memory works but its
 * copies do not overlap.  With the default exact pairwise plan the copies
 * are pipelined with the sort: the host-to-device copy goes in chunks of
 * about n/4 keys whose tile sorts and chunk-local merge rounds start as
 * each chunk arrives, and the last merge round is written in slices whose
 * device-to-host copies start as each slice is done (other options copy
 * the whole array each way around the sort).  Device buffers come from the
 * context: three staging slots, used by consecutive calls in turn, each
 * growing to the largest n it served, plus the sort scratch.  Synchronises on `stream`
 * before returning.  When the call (or msort_sort_host_async) fails after
 * enqueuing work, it first waits for that work, so that on any error return
 * nothing it started still uses the host buffers.
 *
 * Out of core: when the context has a budget and the three staging slots
 * plus the scratch for n elements would exceed it, the array is sorted in
 * budget-sized chunks C whose sorted runs go to a pinned host buffer owned by
 * the context (n keys and values, kept for later calls).  With a block
 * bound B of up to C (as many elements as the context scratch holds beside
 * the merge's split table, at least C/2), every B/(16R)-th element of the R
 * runs is sampled, and every 15R-th sample in (key, position) order becomes
 * a splitter (B/(2R) and R when 16R > B), so each block between consecutive
 * splitters holds at most B elements.  Each block's slices of all runs are
 * copied to a staging slot, merged there with the scratch as the second
 * buffer (msort_merge_runs' rounds; ties in run order) and copied to their
 * place in the output,
 * consecutive blocks overlapping on the context's streams.  MSORT_ERR_OOM if
 * the budget does not fit a chunk of four 16896-key tiles.
 * This path is taken by msort_sort_host_async too, and then returns with the
 * output complete. */
msort_status msort_sort_host(msort_ctx* ctx, const void* h_keys_in, const uint32_t* h_vals_in,
                             void* h_keys_out, uint32_t* h_vals_out, size_t n, msort_key_type kt,
                             const msort_options* opt, void* stream);

/* The same, asynchronous: enqueues the copies and the sort on the
 * context's own copy and compute streams and returns; `stream` is made to
 * wait for the last device-to-host copy, so the result is in h_keys_out
 * (h_vals_out) once `stream` has completed the work enqueued so far
 * (cudaStreamSynchronize or msort_ctx_sync).  The copies do not wait for
 * earlier work on `stream` (the call reads and writes only host memory and
 * its own device buffers): the input must hold its final contents when the
 * call is made, and the host buffers must stay allocated and the input
 * unmodified until `stream` completes.  Tuned for throughput: one
 * host-to-device copy per call and the last round in two slices, since
 * consecutive calls overlap one another.  Consecutive calls take the three
 * staging slots in turn, so one call's device-to-host copy overlaps the next
 * calls' host-to-device copies and sorts; a fourth call waits (on the
 * device) for the first call's slot to be copied out. */
msort_status msort_sort_host_async(msort_ctx* ctx, const void* h_keys_in, const uint32_t* h_vals_in,
                                   void* h_keys_out, uint32_t* h_vals_out, size_t n, msort_key_type kt,
                                   const msort_options* opt, void* stream);

/* ---- serving: continuous batching of sort requests ---------------------- */

/* A server owns one GPU-side loop (a host thread), max_slots CUDA streams
 * and a device arena of mem_budget_bytes from which every admitted
 * request's scratch is carved.  Requests are admitted in FIFO order as soon
 * as a slot is free and their scratch fits in the arena; admitted requests
 * run concurrently on their slots' streams, and each completion immediately
 * frees its slot and memory for the next queued request.  The budget is a
 * hard cap: no device memory is allocated while serving.  (Serving is not
 * in the paper; each request is the paper's sort of one array.) */
typedef struct msort_server msort_server;

typedef struct {
    uint64_t completed;        /* requests finished since the last reset */
    uint64_t queued;           /* waiting for a slot or memory */
    uint64_t inflight;         /* on the GPU now */
    uint64_t max_inflight;     /* most requests on the GPU at once */
    double p50_ms, p99_ms, max_ms; /* submit-to-completion latency */
    double keys_per_s;         /* keys completed / (last completion - first submit) */
    uint64_t arena_high_water; /* most scratch bytes in use at once (<= budget) */
    uint64_t budget;           /* arena size in bytes */
} msort_server_stats;

msort_status msort_server_create(int device, size_t mem_budget_bytes, int max_slots, msort_server** out);
/* Queues an in-place stable sort of d_keys[0:n) (and d_vals, nullable); the
 * buffers must stay valid and untouched until the request is done.  Never
 * blocks.  MSORT_ERR_OOM if the request's scratch alone exceeds the budget. */
msort_status msort_server_submit(msort_server* s, void* d_keys, uint32_t* d_vals, size_t n, msort_key_type kt,
                                 uint64_t* req_id);
/* *done = 1 once the request finished (its latency in *latency_ms, nullable);
 * returns the request's own status when done. */
msort_status msort_server_poll(msort_server* s, uint64_t req_id, int* done, double* latency_ms);
/* Blocks until the request finishes or timeout_ms passes (MSORT_ERR_TIMEOUT). */
msort_status msort_server_wait(msort_server* s, uint64_t req_id, double timeout_ms, double* latency_ms);
msort_status msort_server_get_stats(msort_server* s, msort_server_stats* out);
msort_status msort_server_reset_stats(msort_server* s);
/* Finishes every queued and running request, then frees the server. */
msort_status msort_server_destroy(msort_server* s);

/* ---- sorting without device allocation -------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory: code that owns the device's memory
 * through its own pool, or a latency-critical path that cannot afford the
 * device synchronisation an allocation can cause.  It runs the same stable
 * sort as msort_sort_copy with the default plan, but takes its scratch from
 * a fixed 48 MiB array compiled into the library (held on every GPU that
 * loads the library until the process exits), and calls no allocator.
 *  - Works in the calling thread's current CUDA context (the current
 *    device's primary context if none is current).  The first call under a
 *    context looks up the array's device address there
 *    (cudaGetSymbolAddress, which allocates nothing); make that first call
 *    before any stream capture.  The address is kept per context id, so a
 *    device reset or another context gets its own lookup.
 *  - n above msort_noalloc_max_keys(kt, with_vals) is rejected with
 *    MSORT_ERR_INVALID_ARG before any work is enqueued.
 *  - All calls on a device share the one array: calls whose work overlaps
 *    on the GPU (unordered streams, concurrent host threads) race and give
 *    wrong results.  Order them on one stream.
 *  - d_keys_out may equal d_keys_in (in place); value pointers are both
 *    NULL (keys only) or both set.  Errors a kernel detects on the device
 *    (a bounded wait that gave up) go to a status word inside the array,
 *    cleared at the start of every call: msort_noalloc_sync reads it. */
msort_status msort_sort_noalloc(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out,
                                uint32_t* d_vals_out, size_t n, msort_key_type kt, void* stream);
/* Waits for `stream`, then reports what the kernels of the last
 * msort_sort_noalloc call in the current context recorded: MSORT_OK, or
 * MSORT_ERR_TIMEOUT for a bounded wait that gave up (the word is then
 * cleared).  Allocates nothing; the word is shared like the array, so call
 * it after the call it checks and before the next one is enqueued. */
msort_status msort_noalloc_sync(void* stream);
/* Largest n msort_sort_noalloc accepts for this key type (with or without
 * values). */
size_t msort_noalloc_max_keys(msort_key_type kt, int with_vals);

/* ---- failure detection ------------------------------------------------ */

/* Self-test of the bounded device waits.  The paper's only failure remark is
 * that a blocking Send/Recv waits forever when its peer has failed (Section
 * "MPI Merge Sort"); here no device wait is unbounded: a block that waits
 * for its bulk copies longer than a cycle limit (about one second in every
 * production kernel) records MSORT_ERR_TIMEOUT in the context's status word,
 * waits once more (bounded) for any copy of its own still in flight, and
 * returns.  This call enqueues on `stream` one production merge block whose
 * barrier expects one arrival more than the block makes, with the limit set
 * to limit_cycles (1000 .. 2e9 SM cycles): the block issues no copy, gives up
 * after about 2 x limit_cycles and writes no output.  The next
 * msort_ctx_sync then returns MSORT_ERR_TIMEOUT and clears the word; the
 * context stays usable.  Touches no caller memory; MSORT_ERR_INVALID_ARG for
 * a limit outside the range. */
msort_status msort_selftest_wait_timeout(msort_ctx* ctx, long long limit_cycles, void* stream);
/* The same for the grid barriers of the single-launch sort (options.single_launch):
 * enqueues that sort of the n uint32 keys at d_keys (n spanning at least two
 * of its tiles, so that there is a barrier; up to 2^28) with every barrier
 * wait limited to limit_cycles and the first barrier expecting one arrival
 * more than the grid makes.  Every block completes its stores, gives up at
 * that barrier after about limit_cycles, records MSORT_ERR_TIMEOUT and leaves;
 * no copy is in flight.  The keys are left in an unspecified order.  Uses
 * the context's scratch like a sort; MSORT_ERR_INVALID_ARG for a limit
 * outside [1000, 2e9] or too small an n. */
msort_status msort_selftest_grid_timeout(msort_ctx* ctx, void* d_keys, size_t n, long long limit_cycles,
                                         void* stream);

/* ---- autotuning ---------------------------------------------------------- */

/* Times every tile shape (tile size = threads x keys per thread, which also
 * fixes the merge block) of the plain sort for 32/64-bit keys, with and
 * without values, at n = 2^16, 2^20 and 2^24 (quick != 0: 2^20 only), each
 * with two-way and four-way merge passes for 32-bit keys without values, and
 * the segmented sort's bucket shapes for 32-bit keys; each candidate's output
 * must equal the first candidate's bit for bit or the candidate is rejected.
 * The winners are used by later calls on ctx whose options leave tile (and,
 * for the device-buffer sorts of unsigned keys with partition_mode 0,
 * merge_ways) at 0 (size class = largest tuned class not above log2(n)).  cache_path
 * (nullable) receives the results as JSON.  Allocates its own test buffers
 * and synchronises the device; meant for start-up, not for a hot loop. */
msort_status msort_tune(msort_ctx* ctx, const char* cache_path, int quick);
/* Loads results written by msort_tune into ctx. */
msort_status msort_tune_load(msort_ctx* ctx, const char* cache_path);
/* Forgets tuned choices (back to the built-in defaults). */
msort_status msort_tune_clear(msort_ctx* ctx);

/* ---- learned partitioner: model access and checks ---------------------- */

/* The network of partition_mode 1 (1 -> 32 -> 1, ReLU; 97 fp32 parameters
 * ordered w1[32], b1[32], w2[32], b2) is fitted by mean squared error to the
 * empirical CDF of a sorted key sample: target of the r-th of m samples is
 * (r + 1/2) / m.  These calls run the library's own training kernels on
 * caller data (m <= 65536), so that gradients and training can be checked
 * against a reference. */
/* d_grad[97] = gradient of the loss at d_params over d_x[0:m). */
msort_status msort_mlp_grad(msort_ctx* ctx, const float* d_x, size_t m, const float* d_params, float* d_grad,
                            void* stream);
/* `steps` safeguarded Adam steps (betas 0.9/0.999, eps 1e-8, starting rate
 * lr) on d_params in place: before each update the loss of the current
 * parameters is compared with the best so far; if it is higher, the best
 * parameters are restored, the rate halves and the Adam moments restart.
 * A final check keeps the best parameters seen.  Each step is one launch of
 * 8 blocks that add their partial sums in block order, so the result does
 * not depend on scheduling.  knot_init != 0 first sets
 * d_params to the piecewise-linear interpolant through 32 quantiles of the
 * sorted d_x. */
msort_status msort_mlp_train(msort_ctx* ctx, const float* d_x, size_t m, float* d_params, int knot_init,
                             int steps, float lr, void* stream);
/* Copies the last model trained by a partition_mode 1 sort (97 floats) and
 * its maximum error on its sample (nullable) to host memory; synchronises. */
msort_status msort_learned_model(msort_ctx* ctx, float* h_params, float* h_err);
/* Installs h_params (97 floats) and its error bound as the model of later
 * partition_mode 1 sorts on ctx, which then skip sampling and training
 * (a model trained once can serve many sorts of similar data).  Any model
 * is safe: the prediction is verified and exact search completes it, so a
 * poor model costs probes, never correctness.  h_params == NULL returns to
 * training a fresh model per sort.  Synchronises the device. */
msort_status msort_learned_set_model(msort_ctx* ctx, const float* h_params, float err);
/* One merge pass's partition, as a call (to check every co-rank the sort
 * uses): d_keys[0:n) holds sorted runs of run_length keys laid end to end
 * (the last may be shorter), merged pairwise (runs 2j and 2j + 1) into
 * output blocks of `block` keys (block divides 2 * run_length).  For every
 * output block c, d_splits[c] = the stable co-rank of its first output c *
 * block within its pair: how many of the pair's first-run keys come before
 * it (Merge Path, cited in the paper's Section "Related Research").  mode:
 * 0 the exact binary search of the plain sort, 1 the learned network's
 * guided search (needs a model: a partition_mode 1 sort trained one on ctx,
 * or msort_learned_set_model installed one; while a sort's training is
 * still running on the side stream, blocks start from the ratio guess), 2
 * the ratio-guess guided
 * search, 3 the guided kernel's plain binary search.  Every mode returns the
 * same exact co-ranks.  d_splits holds ceil(n / block) uint64 entries;
 * unsigned key types only. */
msort_status msort_partition_splits(msort_ctx* ctx, const void* d_keys, size_t n, size_t run_length,
                                    size_t block, int mode, uint64_t* d_splits, msort_key_type kt, void* stream);
/* Probes (tests of A[a] <= B[d-1-a]) and searches made by guided partition
 * launches (modes 1-3) while profiling was at level 2; resets the counts.
 * Synchronises the device. */
msort_status msort_ctx_partition_stats(msort_ctx* ctx, uint64_t* probes, uint64_t* searches);

/* ---- measurement ------------------------------------------------------ */

/* Kernel kinds for msort_ctx_kernel_times. */
enum { MSORT_KERNEL_TILE = 0, MSORT_KERNEL_PARTITION = 1, MSORT_KERNEL_MERGE = 2,
       MSORT_KERNEL_SEGMENTED = 3, MSORT_KERNEL_MLP = 4, MSORT_KERNEL_SINGLE = 5 };

/* on != 0: bracket every later launch with CUDA events on its own stream
 * (resets the event log).  Off by default; events cost a few microseconds
 * of host time per launch.  on >= 2 also makes the guided partitions
 * (partition_mode 1-3) count their probes for msort_ctx_partition_stats,
 * with one atomic per warp, which slows those launches: time them at
 * level 1. */
msort_status msort_ctx_set_profiling(msort_ctx* ctx, int on);
/* Waits for the logged events of kernel kind `kind`, returns how many
 * launches were logged and their summed device time, and clears that log. */
msort_status msort_ctx_kernel_times(msort_ctx* ctx, int kind, uint64_t* launches, double* total_ms);
/* Number of kernels this context has launched since it was created. */
unsigned long long msort_ctx_launch_count(msort_ctx* ctx);
/* Like msort_ctx_kernel_times, launch by launch: waits for the logged events
 * of kind `kind`, writes the first min(cap, launches) device times in launch
 * order to h_ms (milliseconds), sets *launches and clears that log. */
msort_status msort_ctx_kernel_log(msort_ctx* ctx, int kind, double* h_ms, size_t cap, uint64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* MSORT_H_ */
