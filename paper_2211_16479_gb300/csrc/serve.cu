// Serving loop: continuous batching of sort requests on one GPU.
//
// The paper sorts one array per run; this is the GPU-side service around
// its method.  A host thread owns the GPU side:
//   * requests enter a FIFO queue (msort_server_submit never blocks);
//   * a request is admitted when a slot (a CUDA stream) is free and its
//     scratch fits in the memory budget; scratch comes from one arena
//     allocated at creation (first fit, neighbours coalesced on release), so
//     no device allocation happens while serving and the budget is a hard
//     cap;
//   * admitted requests run concurrently on their slots' streams (their
//     kernels overlap on the device); a completion event per slot retires the
//     request, frees its slot and scratch, and the next queued requests are
//     admitted at once -- requests that arrive while others are on the GPU
//     join as soon as a slot and memory free up;
//   * latency is host wall-clock time from submit to the loop seeing the
//     completion event.
// The queue is strictly FIFO: a request that does not fit yet blocks the
// ones behind it, so none starves.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"
#include "learned.h"

namespace msort {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    void* keys;
    uint32_t* vals;
    size_t n;
    msort_key_type kt;
    size_t need;
    Clock::time_point t_submit;
};

struct Done {
    bool done = false;
    msort_status status = MSORT_OK;
    double latency_ms = 0.0;
    size_t n = 0;
};

// First-fit arena over [0, size) in 256-byte units.
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length
    size_t used = 0, high_water = 0;
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t len, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                const size_t rest = it->second - len;
                const size_t noff = it->first + len;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used += len;
                high_water = std::max(high_water, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len) {
        used -= len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    Request req{};
    size_t off = 0;
};

}  // namespace
}  // namespace msort

struct msort_server {
    msort_ctx* ctx = nullptr;
    unsigned char* arena_mem = nullptr;
    size_t budget = 0;
    msort::Arena* arena = nullptr;
    std::vector<msort::Slot> slots;
    std::deque<msort::Request> queue;
    std::map<uint64_t, msort::Done> results;
    std::mutex mu;
    std::condition_variable cv;      // wakes the loop (new request / shutdown)
    std::condition_variable cv_done; // wakes waiters (a request finished)
    std::thread loop;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    // statistics
    std::vector<double> latencies;
    size_t keys_done = 0;
    int inflight = 0, max_inflight = 0;
    msort::Clock::time_point t_first{}, t_last{};
    bool any = false;
};

namespace msort {
namespace {

msort_status launch_request(msort_server* s, Slot& sl) {
    const Request& r = sl.req;
    void* scratch = s->arena_mem + sl.off;
    msort_status st;
    if (r.kt == MSORT_U32) {
        uint32_t* k = static_cast<uint32_t*>(r.keys);
        st = r.vals ? sort_with_scratch<uint32_t, true>(s->ctx, k, r.vals, k, r.vals, r.n, scratch, sl.stream)
                    : sort_with_scratch<uint32_t, false>(s->ctx, k, nullptr, k, nullptr, r.n, scratch, sl.stream);
    } else {
        uint64_t* k = static_cast<uint64_t*>(r.keys);
        st = r.vals ? sort_with_scratch<uint64_t, true>(s->ctx, k, r.vals, k, r.vals, r.n, scratch, sl.stream)
                    : sort_with_scratch<uint64_t, false>(s->ctx, k, nullptr, k, nullptr, r.n, scratch, sl.stream);
    }
    if (st == MSORT_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = MSORT_ERR_CUDA;
    return st;
}

void finish(msort_server* s, const Request& r, msort_status st) {
    const auto now = Clock::now();
    Done& d = s->results[r.id];
    d.done = true;
    d.status = st;
    d.n = r.n;
    d.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
    if (st == MSORT_OK) {
        s->latencies.push_back(d.latency_ms);
        s->keys_done += r.n;
        s->t_last = now;
    }
}

void serve_loop(msort_server* s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        // retire finished requests
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish(s, sl.req, q == cudaSuccess ? MSORT_OK : MSORT_ERR_CUDA);
            s->arena->release(sl.off, sl.req.need);
            sl.busy = false;
            --s->inflight;
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // admit in FIFO order while a slot and memory are available
        while (!s->queue.empty()) {
            Slot* free_slot = nullptr;
            for (Slot& sl : s->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            size_t off = 0;
            if (!s->arena->alloc(s->queue.front().need, &off)) break;
            free_slot->req = s->queue.front();
            free_slot->off = off;
            s->queue.pop_front();
            const msort_status st = launch_request(s, *free_slot);
            if (st != MSORT_OK) {
                cudaStreamSynchronize(free_slot->stream);  // nothing may still use the scratch
                finish(s, free_slot->req, st);
                s->arena->release(off, free_slot->req.need);
                s->cv_done.notify_all();
                continue;
            }
            free_slot->busy = true;
            ++s->inflight;
            s->max_inflight = std::max(s->max_inflight, s->inflight);
            progressed = true;
        }
        if (s->stop && s->queue.empty() && s->inflight == 0) break;
        if (!progressed) {
            if (s->inflight == 0) {
                s->cv.wait(lk, [&] { return s->stop.load() || !s->queue.empty(); });
            } else {
                // poll the completion events without holding the lock
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
}

}  // namespace
}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_server_create(int device, size_t mem_budget_bytes, int max_slots, msort_server** out) {
    if (!out) return fail(MSORT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return fail(MSORT_ERR_INVALID_ARG, "max_slots must be in [1, 64]");
    if (mem_budget_bytes < (size_t(1) << 20)) return fail(MSORT_ERR_INVALID_ARG, "budget below 1 MiB");
    msort_ctx* ctx = nullptr;
    msort_status st = msort_ctx_create(device, 0, &ctx);
    if (st != MSORT_OK) return st;
    msort_server* s = new msort_server();
    s->ctx = ctx;
    s->budget = align_up(mem_budget_bytes, 256);
    if (cudaMalloc(&s->arena_mem, s->budget) != cudaSuccess) {
        cudaGetLastError();
        msort_ctx_destroy(ctx);
        delete s;
        return fail(MSORT_ERR_OOM, "cudaMalloc of the serving arena failed");
    }
    s->arena = new Arena(s->budget);
    s->slots.resize(max_slots);
    for (Slot& sl : s->slots) {
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    s->loop = std::thread(serve_loop, s);
    *out = s;
    return MSORT_OK;
}

msort_status msort_server_submit(msort_server* s, void* d_keys, uint32_t* d_vals, size_t n, msort_key_type kt,
                                 uint64_t* req_id) {
    if (!s || !req_id) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    if (kt == MSORT_I32 || kt == MSORT_I64 || kt == MSORT_F32 || kt == MSORT_F64)
        return fail(MSORT_ERR_UNSUPPORTED, "msort_server_submit takes unsigned keys (signed and floating-point keys: the plain "
                                           "and host-buffer sorts)");
    if (kt != MSORT_U32 && kt != MSORT_U64) return fail(MSORT_ERR_INVALID_ARG, "unknown key type");
    if (n && !d_keys) return fail(MSORT_ERR_INVALID_ARG, "d_keys is NULL");
    const size_t need = align_up(sort_scratch_need(n, kt == MSORT_U32 ? 4 : 8, d_vals != nullptr), 256);
    if (need > s->budget) return fail(MSORT_ERR_OOM, "request scratch exceeds the server's memory budget");
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return fail(MSORT_ERR_BUSY, "server is shutting down");
    Request r{s->next_id++, d_keys, d_vals, n, kt, need ? need : 256, Clock::now()};
    if (!s->any) {
        s->any = true;
        s->t_first = r.t_submit;
    }
    *req_id = r.id;
    s->results[r.id] = Done{};
    if (n < 2) {  // nothing to sort
        finish(s, r, MSORT_OK);
        s->cv_done.notify_all();
        return MSORT_OK;
    }
    s->queue.push_back(r);
    s->cv.notify_one();
    return MSORT_OK;
}

msort_status msort_server_poll(msort_server* s, uint64_t req_id, int* done, double* latency_ms) {
    if (!s || !done) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->results.find(req_id);
    if (it == s->results.end()) return fail(MSORT_ERR_INVALID_ARG, "unknown request id");
    *done = it->second.done;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    return it->second.done ? it->second.status : MSORT_OK;
}

msort_status msort_server_wait(msort_server* s, uint64_t req_id, double timeout_ms, double* latency_ms) {
    if (!s) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(req_id);
    if (it == s->results.end()) return fail(MSORT_ERR_INVALID_ARG, "unknown request id");
    const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000.0));
    if (!s->cv_done.wait_until(lk, deadline, [&] { return s->results[req_id].done; }))
        return fail(MSORT_ERR_TIMEOUT, "request not finished before the timeout");
    const Done& d = s->results[req_id];
    if (latency_ms) *latency_ms = d.latency_ms;
    return d.status;
}

msort_status msort_server_get_stats(msort_server* s, msort_server_stats* out) {
    if (!s || !out) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    std::vector<double> lat = s->latencies;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)(q * (double)(lat.size() - 1) + 0.5);
        return lat[std::min(i, lat.size() - 1)];
    };
    out->completed = lat.size();
    out->queued = s->queue.size();
    out->inflight = (uint64_t)s->inflight;
    out->max_inflight = (uint64_t)s->max_inflight;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    const double span = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    out->keys_per_s = span > 0 ? (double)s->keys_done / span : 0.0;
    out->arena_high_water = s->arena->high_water;
    out->budget = s->budget;
    return MSORT_OK;
}

msort_status msort_server_reset_stats(msort_server* s) {
    if (!s) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    s->latencies.clear();
    s->keys_done = 0;
    s->max_inflight = s->inflight;
    s->arena->high_water = s->arena->used;
    s->any = false;
    return MSORT_OK;
}

msort_status msort_server_destroy(msort_server* s) {
    if (!s) return MSORT_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->loop.joinable()) s->loop.join();
    cudaSetDevice(s->ctx->device);
    for (Slot& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
    }
    cudaFree(s->arena_mem);
    delete s->arena;
    msort_ctx_destroy(s->ctx);
    delete s;
    return MSORT_OK;
}

}  // extern "C"
