// Learned-CDF partitioner for the final merge passes.
//
// The paper has no learned component: its merge tree hands each pair of
// runs to one process (Section "MPI Merge Sort", Figs. 16-17) and only cites
// Merge Path partitioning (Section "Related Research").  Here the co-rank
// search that splits every merge pass into equal output blocks starts from
// a prediction made by a small network, F: key -> [0, 1], an estimate of the
// keys' cumulative distribution:
//
//   network   h_j = max(0, w1_j x + b1_j) (32 units), F(x) = clamp(w2 . h + b2)
//   input     x = key / 2^32 (32-bit keys) or key / 2^64 (64-bit), in fp32
//   data      2^16 keys drawn at seeded random positions of the input, sorted
//             by this library's own sort; target of the r-th smallest is
//             (r + 1/2) / 2^16
//   init      piecewise-linear interpolant through 32 sample quantiles
//   training  full-batch mean squared error, Adam (0.9, 0.999, 1e-8) from
//             lr 1e-3 with a safeguard: a step whose loss is above the best
//             so far is undone and the rate halved, so the model never ends
//             worse than its initialisation; forward / backward / update
//             kernels below reduce in a fixed order, so training is
//             reproducible
//
// Prediction for runs A, B and output position d: start from the length
// ratio a0 = d |A| / (|A| + |B|), then take two secant steps in F-space:
// the model's values at the two probed keys, scaled by each run's density
// in F-space (from the model's values at the run's first and last keys);
// each probe also narrows the bracket by its exact comparison.  The step
// is computed without cancellation: F(kb) - F(ka) unit by unit from the
// exact integer key difference, and the new position in 64-bit integers
// (in fp32, positions near 2^29 and differences of nearby outputs resolve
// only tens of elements).
// Verification: an exponential search outward from the prediction (probes
// at distance 1, 2, 4, ... until the split is bracketed; J. L. Bentley and
// A. C. Yao, "An almost optimal algorithm for unbounded searching", 1976),
// then binary search inside the bracket.  A prediction off by e costs about
// 2 log2(e) + 1 probes; the split returned is always the exact co-rank, so
// the sort's output never changes, whatever the model.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "learned.h"
#include "launch.h"
#include "sort_kernels.cuh"

namespace msort {

constexpr int kH = 32;
constexpr int kNP = 3 * kH + 1;  // w1[32], b1[32], w2[32], b2
constexpr int kSample = 1 << 16;
constexpr int kTrainSteps = 32;
constexpr int kTrainStride = 4;  // train on every 4th sorted sample (2^14 points)
constexpr float kLr = 1e-3f;

struct LearnedState {
    unsigned char* block = nullptr;
    uint64_t* sample = nullptr;
    uint64_t* sorted = nullptr;
    void* sort_scratch = nullptr;
    float* x = nullptr;
    float* params = nullptr;
    void* train = nullptr;  // TrainState of the round kernels
    float* err = nullptr;
    unsigned long long* probes = nullptr;  // [0] probes, [1] searches
    unsigned int* ready = nullptr;         // epoch of the last model whose training has finished
    unsigned int epoch = 0;                // epoch of the model the current sort trains
    cudaStream_t side = nullptr;
    cudaEvent_t input_ready = nullptr, model_ready = nullptr, sampled = nullptr;
    cudaGraphExec_t train_exec = nullptr;  // the training rounds of a sort, captured once
    bool pending = false;
    bool trained = false;
    bool frozen = false;  // a caller-installed model: skip sampling and training
    int key_bits = 32;
};

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mlp_f(const float* p, float x) {
    float y = p[3 * kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        const float h = fmaxf(fmaf(p[j], x, p[kH + j]), 0.f);
        y = fmaf(p[2 * kH + j], h, y);
    }
    return y;
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }



template <class K>
__device__ __forceinline__ float key_to_x(K k);
template <>
__device__ __forceinline__ float key_to_x<uint32_t>(uint32_t k) {
    return __uint2float_rn(k) * 2.3283064365386963e-10f;  // k / 2^32, rounded to fp32
}
template <>
__device__ __forceinline__ float key_to_x<uint64_t>(uint64_t k) {
    return __ull2float_rn(k) * 5.421010862427522e-20f;  // k / 2^64, rounded to fp32
}

// (kb - ka) in the network's input units, from the exact integer difference
template <class K>
__device__ __forceinline__ float key_diff_x(K ka, K kb);
template <>
__device__ __forceinline__ float key_diff_x<uint32_t>(uint32_t ka, uint32_t kb) {
    return (float)((long long)kb - (long long)ka) * 2.3283064365386963e-10f;
}
template <>
__device__ __forceinline__ float key_diff_x<uint64_t>(uint64_t ka, uint64_t kb) {
    const double d = kb >= ka ? (double)(kb - ka) : -(double)(ka - kb);
    return (float)(d * 5.421010862427522e-20);
}

// F(kb) - F(ka) without the cancellation of subtracting two nearby outputs:
// per hidden unit, the difference of its two ReLU values, taken from the
// exact key difference where the unit is active at both keys.
template <class K>
__device__ __forceinline__ float mlp_diff(const float* p, K ka, K kb) {
    const float xa = key_to_x<K>(ka), xb = key_to_x<K>(kb), dx = key_diff_x<K>(ka, kb);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        const float ua = fmaf(p[j], xa, p[kH + j]), ub = fmaf(p[j], xb, p[kH + j]);
        const float dh = (ua > 0.f && ub > 0.f) ? p[j] * dx : fmaxf(ub, 0.f) - fmaxf(ua, 0.f);
        s = fmaf(p[2 * kH + j], dh, s);
    }
    return s;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Sample r = key at position floor(mix(seed, r) * n / 2^64).
template <class K>
__global__ void k_sample(const K* __restrict__ keys, size_t n, uint64_t seed, K* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= kSample) return;
    const uint64_t h = mix64(seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull);
    out[r] = keys[__umul64hi(h, (uint64_t)n)];
}

// x[r] = key_to_x(sorted[r * stride]) for r < m / stride.
template <class K>
__global__ void k_keys_to_x(const K* __restrict__ sorted, int m, int stride, float* __restrict__ x) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m / stride) x[r] = key_to_x<K>(sorted[(size_t)r * stride + stride / 2]);
}

// Knot initialisation from sorted x (one block of kH threads): unit j is
// relu(x - q_j) with q_j the sample quantile at (j + 1/2) / H; output
// weights are the slope changes between consecutive knots.
__global__ void k_knot_init(const float* __restrict__ x, int m, float* __restrict__ p) {
    __shared__ float q[kH], slope[kH];
    const int j = threadIdx.x;
    const float rank_j = (j + 0.5f) / kH;
    int idx = (int)(rank_j * m);
    q[j] = x[idx < m ? idx : m - 1];
    __syncthreads();
    if (j < kH - 1) {
        const float dx = q[j + 1] - q[j];
        slope[j] = dx > 0.f ? (1.0f / kH) / dx : 0.f;
    } else {
        slope[j] = 0.f;
    }
    __syncthreads();
    p[j] = 1.f;
    p[kH + j] = -q[j];
    p[2 * kH + j] = slope[j] - (j > 0 ? slope[j - 1] : 0.f);
    if (j == 0) p[3 * kH] = 0.5f / kH;
}

// Training, one launch per round, spread over kTrainBlocks blocks.  Each
// round evaluates the loss at the current parameters and (when an update
// may follow) the full-batch gradient there: block b takes the points
// [b m / B, (b + 1) m / B) in chunks of kChunk (x and dy of a chunk in
// shared memory), sums its squared residuals by a fixed tree and its
// gradient with each warp owning four hidden units (lane-strided sums over
// the chunks, then a fixed xor-shuffle tree), and writes the 98 partial sums
// to its own row.  Few blocks: a round is bound by its fixed latency (launch,
// the L2 round trips of the reduction), not by its arithmetic, and every
// block it holds is an SM slot the concurrent sort does not get.  The last block to finish (a
// counter taken after a release fence) adds the rows in block order, so the
// totals do not depend on which blocks ran first, and applies the guard and
// the Adam update to the state the next round starts from:
//   accept (first round, or loss <= best): best = loss; save the parameters;
//     in the final round stop there, else take one Adam step;
//   reject: restore the saved parameters, halve the rate, restart the moments.
// A final round that is rejected needs one more forward evaluation (of the
// restored parameters, which is then accepted), so the host launches
// steps + 2 rounds and a round that finds the training finished returns at
// once.  grad_only: one round that writes the summed gradient to grad_out.
constexpr int kTrainBlocks = 8;
constexpr int kRoundThreads = 256;
constexpr int kUnitsPerWarp = kH / (kRoundThreads / 32);
constexpr int kChunk = 2048;
constexpr int kPartStride = 100;  // 97 gradient sums, the squared-residual sum, padding

struct TrainState {
    float saved[128], m1[128], m2[128];
    float lr, best, pw1, pw2;  // pw1 = 0.9^k, pw2 = 0.999^k for the bias corrections
    int seen, finished;
    unsigned int arrived;      // blocks of the current round done
    unsigned int pad;
    float part[kTrainBlocks][kPartStride];
};

__global__ void __launch_bounds__(kRoundThreads)
k_mlp_round(const float* __restrict__ x, int m, float* __restrict__ params, TrainState* __restrict__ ts, int first,
            int need_grad, int final_round, float lr0, float* __restrict__ grad_out) {
    __shared__ float p[kNP], xs[kChunk], dys[kChunk], red[kRoundThreads], tot[kPartStride];
    __shared__ int is_last, accept;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, b = blockIdx.x;
    if (!first && !grad_out && ts->finished) return;  // uniform: every block reads the same flag
    for (int i = tid; i < kNP; i += kRoundThreads) p[i] = params[i];
    const int r0 = (int)(((long long)b * m) / kTrainBlocks), r1 = (int)(((long long)(b + 1) * m) / kTrainBlocks);
    const int cnt = r1 - r0;
    const float inv_m = 1.f / (float)m;
    float w1[kUnitsPerWarp], b1[kUnitsPerWarp], w2[kUnitsPerWarp];
    float a0[kUnitsPerWarp], a1[kUnitsPerWarp], a2[kUnitsPerWarp];
    float ab = 0.f, e2 = 0.f;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kUnitsPerWarp; ++u) {
        const int j = warp * kUnitsPerWarp + u;
        w1[u] = p[j];
        b1[u] = p[kH + j];
        w2[u] = p[2 * kH + j];
        a0[u] = a1[u] = a2[u] = 0.f;
    }
    for (int c0 = 0; c0 < cnt; c0 += kChunk) {
        const int cc = cnt - c0 < kChunk ? cnt - c0 : kChunk;
        for (int i = tid; i < cc; i += kRoundThreads) {
            const int r = r0 + c0 + i;
            const float xr = x[r];
            const float res = mlp_f(p, xr) - (r + 0.5f) * inv_m;
            xs[i] = xr;
            dys[i] = 2.f * res * inv_m;
            e2 += res * res;
        }
        __syncthreads();
        if (need_grad) {
            for (int i = lane; i < cc; i += 32) {
                const float xr = xs[i], d = dys[i];
#pragma unroll
                for (int u = 0; u < kUnitsPerWarp; ++u) {
                    const float pre = fmaf(w1[u], xr, b1[u]);
                    const bool act = pre > 0.f;
                    const float h = act ? pre : 0.f;
                    const float gp = act ? d * w2[u] : 0.f;
                    a0[u] = fmaf(gp, xr, a0[u]);
                    a1[u] += gp;
                    a2[u] = fmaf(d, h, a2[u]);
                }
                ab += d;
            }
        }
        __syncthreads();  // the chunk buffers are reused
    }
    red[tid] = e2;
    __syncthreads();
    for (int w = kRoundThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    float* row = ts->part[b];
    if (tid == 0) row[kNP] = red[0];
    if (need_grad) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < kUnitsPerWarp; ++u) {
                a0[u] += __shfl_xor_sync(0xffffffffu, a0[u], o);
                a1[u] += __shfl_xor_sync(0xffffffffu, a1[u], o);
                a2[u] += __shfl_xor_sync(0xffffffffu, a2[u], o);
            }
            ab += __shfl_xor_sync(0xffffffffu, ab, o);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < kUnitsPerWarp; ++u) {
                const int j = warp * kUnitsPerWarp + u;
                row[j] = a0[u];
                row[kH + j] = a1[u];
                row[2 * kH + j] = a2[u];
            }
            if (warp == 0) row[3 * kH] = ab;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // release this block's row before counting it
        is_last = atomicAdd(&ts->arrived, 1u) == (unsigned)(kTrainBlocks - 1);
        if (is_last) __threadfence();  // acquire: every row is visible below
    }
    __syncthreads();
    if (!is_last) return;

    // the last block: totals in block order, then the guard and the update
    if (tid <= kNP) {
        float s = 0.f;
        for (int q = 0; q < kTrainBlocks; ++q) s += __ldcg(&ts->part[q][tid]);
        tot[tid] = s;
    }
    __syncthreads();
    if (grad_out) {
        for (int i = tid; i < kNP; i += kRoundThreads) grad_out[i] = tot[i];
        if (tid == 0) ts->arrived = 0;
        return;
    }
    if (tid == 0) {
        if (first) {
            ts->lr = lr0;
            ts->best = 0.f;
            ts->pw1 = 1.f;
            ts->pw2 = 1.f;
            ts->seen = 0;
        }
        const float loss = tot[kNP] * inv_m;
        accept = !ts->seen || loss <= ts->best;
        if (accept) {
            ts->best = loss;
            ts->seen = 1;
        } else {
            ts->lr *= 0.5f;
            ts->pw1 = 1.f;
            ts->pw2 = 1.f;
        }
    }
    __syncthreads();
    if (tid < kNP) {
        float m1 = first ? 0.f : ts->m1[tid], m2 = first ? 0.f : ts->m2[tid];
        float pi = p[tid];
        if (!accept) {
            pi = ts->saved[tid];
            m1 = 0.f;
            m2 = 0.f;
        } else {
            ts->saved[tid] = pi;
            if (!final_round) {
                const float b1c = 0.9f, b2c = 0.999f, eps = 1e-8f;
                const float c1 = 1.f - ts->pw1 * b1c, c2 = 1.f - ts->pw2 * b2c;  // 1 - beta^(k+1)
                const float gi = tot[tid];
                m1 = b1c * m1 + (1.f - b1c) * gi;
                m2 = b2c * m2 + (1.f - b2c) * gi * gi;
                pi -= ts->lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
            }
        }
        ts->m1[tid] = m1;
        ts->m2[tid] = m2;
        params[tid] = pi;  // accepted final round: pi is the saved (best) value
    }
    __syncthreads();
    if (tid == 0) {
        if (accept && !final_round) {
            ts->pw1 *= 0.9f;
            ts->pw2 *= 0.999f;
        }
        ts->finished = accept && final_round;
        ts->arrived = 0;
    }
}

// err[0] = max_r |clamp(F(x_r)) - t_r| (one block, fixed reduction).
// Also publishes the model: after err is written, *ready = epoch (release),
// which the guided partitions of the sort poll once per block.
__global__ void k_model_error(const float* __restrict__ x, int m, const float* __restrict__ params,
                              float* __restrict__ err, unsigned int* ready, unsigned int epoch) {
    constexpr int TH = 256;
    __shared__ float p[kNP];
    __shared__ float s[TH];
    for (int i = threadIdx.x; i < kNP; i += TH) p[i] = params[i];
    __syncthreads();
    float e = 0.f;
    for (int r = threadIdx.x; r < m; r += TH) e = fmaxf(e, fabsf(clamp01(mlp_f(p, x[r])) - (r + 0.5f) / m));
    s[threadIdx.x] = e;
    __syncthreads();
    for (int w = TH / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        err[0] = s[0];
        __threadfence();  // the parameters (earlier kernels of this stream) and err before the flag
        atomicExch(ready, epoch);
    }
}

// Co-rank with a guided start.  params == nullptr: ratio guess (mode 2);
// exact_only: no guess at all (plain binary search, mode 3, used to count
// its probes).  Counts probes (one probe = one test of A[a] <= B[d-1-a]).
// A model trained beside the sort is used once its training has finished:
// each block reads *ready (acquire) once and takes the model if it holds
// this sort's epoch, else starts from the ratio guess.  The split is the
// exact co-rank either way; the sort never waits for its model.  ready ==
// nullptr: the parameters are a fixed, installed model.
template <class K>
__global__ void k_partition_guided(const K* __restrict__ src, size_t n, size_t L, size_t W, size_t nblocks,
                                   unsigned long long* __restrict__ splits, const float* __restrict__ params,
                                   const unsigned int* ready, unsigned int epoch, int exact_only,
                                   unsigned long long* probes) {
    __shared__ float p[kNP];
    __shared__ float fend[2][4];  // F at A[0], A[|A|-1], B[0], B[|B|-1] of the block's first two pairs
    __shared__ int use_model;
    if (threadIdx.x == 0) {
        unsigned int v = epoch;
        if (params && ready) asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ready) : "memory");
        use_model = params != nullptr && v == epoch;
    }
    __syncthreads();
    if (use_model)  // L2 loads: the parameters were written by another stream's kernels
        for (int i = threadIdx.x; i < kNP; i += blockDim.x) p[i] = __ldcg(params + i);
    __syncthreads();
    // The searches of a block usually fall in one or two merge pairs (the
    // guided passes' runs span many output blocks): evaluate the network at
    // those pairs' run ends once, by 8 threads, instead of in every thread.
    const size_t cfirst = (size_t)blockIdx.x * blockDim.x;
    const size_t clast = (cfirst + blockDim.x < nblocks ? cfirst + blockDim.x : nblocks) - 1;
    const size_t pair0 = cfirst * W / (2 * L);
    const bool shared_ends = use_model && clast * W / (2 * L) - pair0 <= 1;  // block-uniform
    if (shared_ends) {
        if (threadIdx.x < 8) {
            const size_t pp = pair0 + (threadIdx.x >> 2);
            const int which = threadIdx.x & 3;
            if (pp * 2 * L < n) {
                const PassGeom gp = pass_geom(pp * 2 * L, n, L);
                const K* pa = src + gp.pb;
                const size_t len = which < 2 ? gp.alen : gp.blen;
                const K* run = which < 2 ? pa : pa + gp.alen;
                if (len > 0)
                    fend[threadIdx.x >> 2][which] = mlp_f(p, key_to_x<K>(run[(which & 1) ? len - 1 : 0]));
            }
        }
        __syncthreads();
    }
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int live = __ballot_sync(0xffffffffu, c < nblocks);  // lanes that search (blockDim % 32 == 0)
    if (c >= nblocks) return;
    const size_t out0 = c * W;
    const PassGeom g = pass_geom(out0, n, L);
    const K* A = src + g.pb;
    const K* B = A + g.alen;
    const size_t alen = g.alen, blen = g.blen, d = out0 - g.pb;
    size_t lo = d > blen ? d - blen : 0;
    size_t hi = d < alen ? d : alen;
    unsigned long long np = 0;
    if (lo < hi && !exact_only) {
        size_t ahat = (size_t)((double)d * (double)alen / (double)(alen + blen));
        ahat = ahat < lo ? lo : (ahat > hi ? hi : ahat);
        if (use_model) {
            // Secant steps in F-space.  A run's keys cover [F(first), F(last)]
            // (the whole CDF for random-order runs, a sliver for presorted
            // ones), so moving a by D shifts F(A[a]) by about D * sA and
            // F(B[d-1-a]) by -D * sB, sR = (F(R_last) - F(R_first)) / |R|.
            // At a probe a the two keys sit near the split, so the model's
            // error largely cancels in F(B[d-1-a]) - F(A[a]).  Every probe
            // also narrows the bracket by its exact comparison.
            float fa0, fa1, fb0, fb1;
            if (shared_ends) {
                const int q = (int)(g.pb / (2 * L) - pair0);
                fa0 = fend[q][0];
                fa1 = fend[q][1];
                fb0 = fend[q][2];
                fb1 = fend[q][3];
            } else {
                fa0 = mlp_f(p, key_to_x<K>(A[0]));
                fa1 = mlp_f(p, key_to_x<K>(A[alen - 1]));
                fb0 = mlp_f(p, key_to_x<K>(B[0]));
                fb1 = mlp_f(p, key_to_x<K>(B[blen - 1]));
            }
            np += 2;
            const float sA = fmaxf(fa1 - fa0, 1e-12f) / (float)alen;
            const float sB = fmaxf(fb1 - fb0, 1e-12f) / (float)blen;
            const float inv = 1.f / (sA + sB);
            for (int it = 0; it < 2 && lo < hi && ahat < hi; ++it) {
                const K ka = A[ahat], kb = B[d - 1 - ahat];
                ++np;
                if (ka <= kb)
                    lo = ahat + 1;
                else
                    hi = ahat;
                if (lo >= hi) break;
                const float delta = mlp_diff<K>(p, ka, kb) * inv;  // positions to move
                const long long step = (long long)rintf(fminf(fmaxf(delta, -4.0e18f), 4.0e18f));
                const long long cand = (long long)ahat + step;
                ahat = cand <= (long long)lo ? lo : (cand >= (long long)hi ? hi : (size_t)cand);
            }
        }
        // Exponential search outward from the prediction; f(a) = A[a] <=
        // B[d-1-a] is true below the split and false from it on.
        if (ahat < hi && (++np, A[ahat] <= B[d - 1 - ahat])) {
            size_t last_true = ahat, step = 1;
            for (;;) {
                const size_t probe = last_true + step;
                if (probe >= hi) {
                    lo = last_true + 1;
                    break;
                }
                ++np;
                if (A[probe] <= B[d - 1 - probe]) {
                    last_true = probe;
                    step *= 2;
                } else {
                    lo = last_true + 1;
                    hi = probe;
                    break;
                }
            }
        } else {
            size_t first_false = ahat, step = 1;  // the split is at or below ahat
            while (first_false >= lo + step) {
                const size_t probe = first_false - step;
                ++np;
                if (A[probe] <= B[d - 1 - probe]) {
                    lo = probe + 1;
                    break;
                }
                first_false = probe;
                step *= 2;
            }
            hi = first_false;
        }
    }
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        ++np;
        if (A[mid] <= B[d - 1 - mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    splits[c] = lo;
    if (probes) {  // one atomic per warp
        const unsigned int wp = __reduce_add_sync(live, (unsigned int)np);
        if ((threadIdx.x & 31) == __ffs(live) - 1) {
            atomicAdd(&probes[0], (unsigned long long)wp);
            atomicAdd(&probes[1], (unsigned long long)__popc(live));
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static LearnedState* state(msort_ctx* ctx) { return static_cast<LearnedState*>(ctx->learned); }

static msort_status ensure_state(msort_ctx* ctx) {
    if (ctx->learned) return MSORT_OK;
    LearnedState* s = new LearnedState();
    const size_t ssz = align_up(sort_keys_scratch<uint64_t>(kSample), 256);
    const size_t tsz = align_up(sizeof(TrainState), 256);
    const size_t bytes = 2 * (size_t)kSample * 8 + ssz + (size_t)kSample * 4 + tsz + 3 * 512 + 256;
    if (cudaMalloc(&s->block, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(MSORT_ERR_OOM, "cudaMalloc of the learned-partitioner state failed");
    }
    unsigned char* q = s->block;
    s->sample = reinterpret_cast<uint64_t*>(q);
    q += (size_t)kSample * 8;
    s->sorted = reinterpret_cast<uint64_t*>(q);
    q += (size_t)kSample * 8;
    s->sort_scratch = q;
    q += ssz;
    s->x = reinterpret_cast<float*>(q);
    q += (size_t)kSample * 4;
    s->train = q;
    q += tsz;
    s->params = reinterpret_cast<float*>(q);
    q += 512;
    s->err = reinterpret_cast<float*>(q);
    q += 512;
    s->probes = reinterpret_cast<unsigned long long*>(q);
    s->ready = reinterpret_cast<unsigned int*>(q + 16);
    cudaMemset(s->train, 0, sizeof(TrainState));  // the round counter starts at zero
    cudaMemset(s->probes, 0, 16 + sizeof(unsigned int));
    cudaMemset(s->err, 0, 4);
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    // highest priority: the few blocks of the sample sort and training get
    // scheduled ahead of the sort's own blocks as SMs free up
    cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, hi_prio);
    cudaEventCreateWithFlags(&s->input_ready, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&s->model_ready, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&s->sampled, cudaEventDisableTiming);
    ctx->learned = s;
    return MSORT_OK;
}

void learned_destroy(msort_ctx* ctx) {
    LearnedState* s = state(ctx);
    if (!s) return;
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->train_exec) cudaGraphExecDestroy(s->train_exec);
    if (s->input_ready) cudaEventDestroy(s->input_ready);
    if (s->model_ready) cudaEventDestroy(s->model_ready);
    if (s->sampled) cudaEventDestroy(s->sampled);
    cudaFree(s->block);
    delete s;
    ctx->learned = nullptr;
}

int learned_first_pass(const Plan& pl, size_t) {
    if (pl.learned_passes > 0) return pl.passes > pl.learned_passes ? pl.passes - pl.learned_passes : 0;
    int p = 0;
    while (p < pl.passes && ((size_t)pl.tile << p) < ((size_t)1 << 22)) ++p;
    return p;
}

// steps + 2 rounds (the last one returns at once unless the final round was
// rejected); each round's launch waits for the previous one on the stream.
static cudaError_t train_on(msort_ctx* ctx, LearnedState* s, const float* x, int m, float* params, int steps,
                            float lr, cudaStream_t st) {
    TrainState* ts = static_cast<TrainState*>(s->train);
    for (int r = 0; r <= steps + 1; ++r) {
        k_mlp_round<<<kTrainBlocks, kRoundThreads, 0, st>>>(x, m, params, ts, r == 0, r < steps, r >= steps, lr,
                                                            nullptr);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

// The training of a sort (kTrainSteps steps on the fixed sample buffers)
// replayed from a CUDA graph: one host call instead of one per round, so
// the host does not hold back the sort's own launches.  Captured on a
// stream of its own the first time.
static cudaError_t train_sample(msort_ctx* ctx, LearnedState* s, int m) {
    if (!s->train_exec) {
        cudaStream_t cs = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const unsigned long long before = ctx->launches;
            const cudaError_t le = train_on(ctx, s, s->x, m, s->params, kTrainSteps, kLr, cs);
            ctx->launches = before;
            e = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->train_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            s->train_exec = nullptr;
            return e;
        }
    }
    ctx->launches += kTrainSteps + 2;
    return cudaGraphLaunch(s->train_exec, s->side);
}

template <class K>
msort_status learned_prepare(msort_ctx* ctx, const Plan& pl, const K* keys, size_t n, cudaStream_t st,
                             bool keys_overwritten) {
    msort_status rs = ensure_state(ctx);
    if (rs != MSORT_OK) return rs;
    LearnedState* s = state(ctx);
    if (s->frozen) return MSORT_OK;
    if (++s->epoch == 0) s->epoch = 1;  // 0 is the flag's value before any model
    cudaError_t e = cudaEventRecord(s->input_ready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->input_ready, 0);
    if (e != cudaSuccess) return cuda_fail(e, "learned partitioner stream order");
    K* sample = reinterpret_cast<K*>(s->sample);
    K* sorted = reinterpret_cast<K*>(s->sorted);
    k_sample<K><<<kSample / 256, 256, 0, s->side>>>(keys, n, 0x5EEDull + n, sample);
    ++ctx->launches;
    if (keys_overwritten) {  // the sort's first kernel writes `keys`: it waits until the sample is taken
        e = cudaEventRecord(s->sampled, s->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->sampled, 0);
        if (e != cudaSuccess) return cuda_fail(e, "learned partitioner stream order");
    }
    rs = sort_keys_internal<K>(ctx, sample, sorted, kSample, s->sort_scratch, s->side);
    if (rs != MSORT_OK) return rs;
    const int mt = kSample / kTrainStride;
    k_keys_to_x<K><<<mt / 256, 256, 0, s->side>>>(sorted, kSample, kTrainStride, s->x);
    k_knot_init<<<1, kH, 0, s->side>>>(s->x, mt, s->params);
    ctx->launches += 2;
    e = train_sample(ctx, s, mt);
    if (e == cudaSuccess) {
        k_model_error<<<1, 256, 0, s->side>>>(s->x, mt, s->params, s->err, s->ready, s->epoch);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->model_ready, s->side);
    if (e != cudaSuccess) return cuda_fail(e, "learned partitioner training launch");
    s->pending = true;
    s->trained = true;
    s->key_bits = 8 * (int)sizeof(K);
    return MSORT_OK;
}

template <class K>
cudaError_t launch_guided_partition(msort_ctx* ctx, const Plan& pl, const K* src, size_t n, size_t L,
                                    unsigned long long* splits, cudaStream_t st) {
    if (ensure_state(ctx) != MSORT_OK) return cudaErrorMemoryAllocation;
    LearnedState* s = state(ctx);
    const bool model = pl.partition_mode == 1;
    const int exact_only = pl.partition_mode == 3;
    if (model && s->pending && ctx->count_probes) {
        // counting probes measures the model: wait for it instead of
        // searching from the ratio guess until it is ready
        cudaError_t e = cudaStreamWaitEvent(st, s->model_ready, 0);
        if (e != cudaSuccess) return e;
        s->pending = false;
    }
    const size_t nblocks = (n + pl.W - 1) / pl.W;
    const unsigned th = 128;
    k_partition_guided<K><<<(unsigned)((nblocks + th - 1) / th), th, 0, st>>>(
        src, n, L, (size_t)pl.W, nblocks, splits, model ? s->params : nullptr, s->frozen ? nullptr : s->ready,
        s->epoch, exact_only, ctx->count_probes ? s->probes : nullptr);
    return cudaGetLastError();
}

template msort_status learned_prepare<uint32_t>(msort_ctx*, const Plan&, const uint32_t*, size_t, cudaStream_t, bool);
template msort_status learned_prepare<uint64_t>(msort_ctx*, const Plan&, const uint64_t*, size_t, cudaStream_t, bool);
template cudaError_t launch_guided_partition<uint32_t>(msort_ctx*, const Plan&, const uint32_t*, size_t, size_t,
                                                       unsigned long long*, cudaStream_t);
template cudaError_t launch_guided_partition<uint64_t>(msort_ctx*, const Plan&, const uint64_t*, size_t, size_t,
                                                       unsigned long long*, cudaStream_t);

}  // namespace msort

using namespace msort;

extern "C" {

msort_status msort_mlp_grad(msort_ctx* ctx, const float* d_x, size_t m, const float* d_params, float* d_grad,
                            void* stream) {
    if (!ctx || !d_x || !d_params || !d_grad) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    if (m == 0 || m > (size_t)kSample) return fail(MSORT_ERR_INVALID_ARG, "m must be in [1, 65536]");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    msort_status rs = ensure_state(ctx);
    if (rs != MSORT_OK) return rs;
    LearnedState* s = state(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamSynchronize(s->side);
    k_mlp_round<<<kTrainBlocks, kRoundThreads, 0, st>>>(d_x, (int)m, const_cast<float*>(d_params),
                                                        static_cast<TrainState*>(s->train), 1, 1, 0, 0.f, d_grad);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    // the training state is shared with the side stream: its later work waits for this launch
    if (e == cudaSuccess) e = cudaEventRecord(s->input_ready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->input_ready, 0);
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "gradient launch");
}

msort_status msort_mlp_train(msort_ctx* ctx, const float* d_x, size_t m, float* d_params, int knot_init, int steps,
                             float lr, void* stream) {
    if (!ctx || !d_x || !d_params) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    if (m == 0 || m > (size_t)kSample) return fail(MSORT_ERR_INVALID_ARG, "m must be in [1, 65536]");
    if (steps < 0) return fail(MSORT_ERR_INVALID_ARG, "steps must be >= 0");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    msort_status rs = ensure_state(ctx);
    if (rs != MSORT_OK) return rs;
    LearnedState* s = state(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamSynchronize(s->side);
    if (knot_init) {
        k_knot_init<<<1, kH, 0, st>>>(d_x, (int)m, d_params);
        ++ctx->launches;
    }
    cudaError_t e = train_on(ctx, s, d_x, (int)m, d_params, steps, lr, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->input_ready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->input_ready, 0);
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "training launch");
}

msort_status msort_learned_model(msort_ctx* ctx, float* h_params, float* h_err) {
    if (!ctx || !h_params) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    LearnedState* s = state(ctx);
    if (!s || !s->trained) return fail(MSORT_ERR_INVALID_ARG, "no model trained on this context yet");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(s->side);
    cudaError_t e = cudaMemcpy(h_params, s->params, kNP * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_err) e = cudaMemcpy(h_err, s->err, sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "model read");
}

msort_status msort_learned_set_model(msort_ctx* ctx, const float* h_params, float err) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    msort_status rs = ensure_state(ctx);
    if (rs != MSORT_OK) return rs;
    LearnedState* s = state(ctx);
    cudaStreamSynchronize(s->side);
    cudaDeviceSynchronize();
    if (!h_params) {
        s->frozen = false;
        return MSORT_OK;
    }
    cudaError_t e = cudaMemcpy(s->params, h_params, kNP * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->err, &err, sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "model upload");
    s->frozen = true;
    s->trained = true;
    s->pending = false;
    return MSORT_OK;
}

msort_status msort_partition_splits(msort_ctx* ctx, const void* d_keys, size_t n, size_t run_length,
                                    size_t block, int mode, uint64_t* d_splits, msort_key_type kt, void* stream) {
    if (!ctx) return fail(MSORT_ERR_INVALID_ARG, "ctx is NULL");
    if (kt != MSORT_U32 && kt != MSORT_U64) return fail(MSORT_ERR_UNSUPPORTED, "unsigned keys only");
    if (mode < 0 || mode > 3) return fail(MSORT_ERR_INVALID_ARG, "mode must be 0, 1, 2 or 3");
    if (n == 0) return MSORT_OK;
    if (!d_keys || !d_splits) return fail(MSORT_ERR_INVALID_ARG, "NULL pointer");
    if (block == 0 || block > (size_t)1 << 30 || run_length == 0 || (2 * run_length) % block)
        return fail(MSORT_ERR_INVALID_ARG, "block must divide 2 * run_length");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (mode != 0) {
        msort_status rs = ensure_state(ctx);
        if (rs != MSORT_OK) return rs;
        if (mode == 1 && !state(ctx)->trained)
            return fail(MSORT_ERR_INVALID_ARG, "mode 1 needs a model: run a partition_mode 1 sort or install one first");
    }
    Plan pl{};
    pl.W = (int)block;
    pl.partition_mode = mode;
    pl.status = ctx->d_status;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* splits = reinterpret_cast<unsigned long long*>(d_splits);
    if (kt == MSORT_U32)
        e = mode == 0 ? launch_partition<uint32_t>(pl, static_cast<const uint32_t*>(d_keys), n, run_length, splits, st)
                      : launch_guided_partition<uint32_t>(ctx, pl, static_cast<const uint32_t*>(d_keys), n,
                                                          run_length, splits, st);
    else
        e = mode == 0 ? launch_partition<uint64_t>(pl, static_cast<const uint64_t*>(d_keys), n, run_length, splits, st)
                      : launch_guided_partition<uint64_t>(ctx, pl, static_cast<const uint64_t*>(d_keys), n,
                                                          run_length, splits, st);
    ++ctx->launches;
    return e == cudaSuccess ? MSORT_OK : cuda_fail(e, "partition launch");
}

msort_status msort_ctx_partition_stats(msort_ctx* ctx, uint64_t* probes, uint64_t* searches) {
    if (!ctx || !probes || !searches) return fail(MSORT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    msort_status rs = ensure_state(ctx);
    if (rs != MSORT_OK) return rs;
    LearnedState* s = state(ctx);
    cudaDeviceSynchronize();
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemcpy(h, s->probes, 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(s->probes, 0, 16);
    if (e != cudaSuccess) return cuda_fail(e, "partition stats");
    *probes = h[0];
    *searches = h[1];
    return MSORT_OK;
}

}  // extern "C"
