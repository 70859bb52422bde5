// Kernel launchers of the sort passes, instantiated per key type in
// kern_u32.cu / kern_u64.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "ctx.h"

namespace msort {

// Shared memory bytes of one tile-sort / merge block.
template <class K, bool PAIRS>
size_t tile_smem_bytes(int tile);
template <class K, bool PAIRS>
size_t merge_smem_bytes(int W);
// True when this (tile, key type, values) combination has a kernel.
template <class K, bool PAIRS>
bool tile_supported(int tile);

// xf_in / xf_out: key transform applied as the tile sort reads its input /
// undone as it writes its output (0 = none; see xf_forward).
template <class K, bool PAIRS>
cudaError_t launch_tile(const Plan& pl, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t n,
                        cudaStream_t st, int xf_in = 0, int xf_out = 0);
// Merge pass over blocks [c0, min(c1, blocks)) (the whole pass by default).
template <class K, bool PAIRS>
cudaError_t launch_merge(const Plan& pl, const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst, size_t n,
                         size_t L, const unsigned long long* splits, cudaStream_t st, size_t c0 = 0,
                         size_t c1 = ~size_t(0), int xf_out = 0);
template <class K>
cudaError_t launch_partition(const Plan& pl, const K* src, size_t n, size_t L, unsigned long long* splits,
                             cudaStream_t st);
// Four-way pass (two merge-tree rounds): runs of L -> runs of 4L.  The grid
// arrays hold merge4_grid_points(n, L, G) entries each; brk 6 * blocks.
inline size_t merge4_grid_points(size_t n, size_t L, size_t G) {
    return (n + 4 * L - 1) / (4 * L) * (4 * L / G);
}
template <class K>
cudaError_t launch_merge4_partition(const Plan& pl, const K* src, size_t n, size_t L, unsigned long long* gco,
                                    K* gval, unsigned long long* gpos, unsigned long long* brk, cudaStream_t st);
template <class K>
cudaError_t launch_merge4(const Plan& pl, const K* src, K* dst, size_t n, size_t L, const unsigned long long* brk,
                          cudaStream_t st);
template <class K>
size_t merge4_smem_bytes(int W4);
// Stable merge of two separate sorted arrays into out (splits: nblocks + 1).
template <class K, bool PAIRS>
cudaError_t launch_merge_two(const K* A, size_t na, const K* B, size_t nb, const uint32_t* va, const uint32_t* vb,
                             K* out, uint32_t* vout, unsigned long long* splits, unsigned int* status,
                             cudaStream_t st);
template <class K, bool PAIRS>
size_t merge_two_block();
// One merge-tree round over sorted runs of arbitrary lengths laid end to
// end: pair j merges [p[j], m[j]) with [m[j], p[j+1]) in place of both (in
// the destination buffer); its output blocks of merge_two_block() outputs
// are [c[j], c[j+1]).  Passed to the kernels by value.
constexpr int kRunPairsMax = 32;
struct RunPairs {
    int np;                                  // pairs (1..kRunPairsMax)
    unsigned long long p[kRunPairsMax + 1];  // pair starts; p[np] = end of the last pair
    unsigned long long m[kRunPairsMax];      // start of each pair's second run (= p[j+1] if none)
    unsigned long long c[kRunPairsMax + 1];  // first output block of each pair; c[np] = blocks
};
// splits: c[np] + 1 entries; xf_out: key transform the round undoes as it
// writes (see xf_inverse).
template <class K, bool PAIRS>
cudaError_t launch_merge_runs(const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst, const RunPairs& rp,
                              unsigned long long* splits, unsigned int* status, int xf_out, cudaStream_t st);
// Single-launch sort of n keys (csrc/small.cuh): tiles of pl.tile keys (the
// default shape for n is small_tile<K, PAIRS>(n)) and every merge round in
// one cooperative launch; `barrier`
// points to 8 bytes of scratch that this function zeroes on `st` first.
template <class K, bool PAIRS>
int small_tile(size_t n);
template <class K, bool PAIRS>
bool small_tile_supported(int tile);
// wait_limit: cycle limit of every grid-barrier wait; extra_arrivals: 0
// (the self-test raises it so that the first barrier never completes).
template <class K, bool PAIRS>
cudaError_t launch_small(const Plan& pl, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, K* tk,
                         uint32_t* tv, size_t n, void* barrier, cudaStream_t st, int xf_in, int xf_out,
                         long long wait_limit = 2000000000ll, unsigned int extra_arrivals = 0);
// Resource summary of the last kernel the calling thread prepared to launch.
const std::string& last_launch_info();

}  // namespace msort
