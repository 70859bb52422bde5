/*
 * CPU oracle for the merge sort -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load this file.  The GPU library never includes, links or calls it, and
 * this file includes nothing from the GPU library.
 *
 * What it computes, and where the paper defines it:
 *
 *  - oracle_sort_*: the top-down recursive merge sort of Section "Sequential
 *    Merge Sort" (the four numbered steps and Fig. 2): an input with fewer
 *    than two elements is returned as is; otherwise it is split at
 *    mid = n / 2 into left = a[0:mid) and right = a[mid:n) (Fig. 2 prints
 *    right = array[:mid], read as a typo for array[mid:]), both halves are
 *    sorted by the same procedure, and the halves are merged.  The paper
 *    never defines merge(); it is read as the textbook two-way merge that
 *    takes from the left run while left <= right, which makes the sort
 *    stable (equal keys keep their input order).
 *  - oracle_merge_*: that two-way merge on its own.
 *  - oracle_corank_*: the number of elements of A among the first d outputs
 *    of merge(A, B).  The paper only cites Merge Path partitioning (Section
 *    "Related Research"); this is its definition written out: run the merge
 *    and count.
 *  - oracle_par_sort_*: the multiprocessing design (Section "Multiprocessing
 *    Merge Sort", Figs. 6-7: chunks of ceil(n / p) elements, one worker per
 *    chunk) followed by the pairwise merge tree of Section "MPI Merge Sort"
 *    (Figs. 16-17: in each round the chunk in the upper half of the remaining
 *    workers is merged into its partner in the lower half, until one run is
 *    left), with POSIX threads as workers.  It returns the same bytes as
 *    oracle_sort_*; it exists to be timed.
 *  - oracle_segmented_sort_*: oracle_sort_* applied to each segment
 *    [off[i], off[i+1]) on its own.
 *
 * Keys are compared as unsigned integers (u32, u64), as signed integers
 * (i32, i64), or, for floating-point keys held as bit patterns (f32, f64),
 * by IEEE 754 totalOrder; values ride along with their key.
 * Memory: the sorts allocate an n-element temporary (a two-way merge needs
 * room for its output) and return -1 if malloc fails, 0 on success.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* tests rebuild this file with planted mistakes */
#endif

#define DEFINE_ORACLE(SUF, KT, LE)                                                      \
    /* merge(left, right): take from the left run while left <= right. */               \
    static void merge_##SUF(const KT* ak, const uint32_t* av, size_t na, const KT* bk,  \
                            const uint32_t* bv, size_t nb, KT* ok, uint32_t* ov) {     \
        size_t i = 0, j = 0, o = 0;                                                     \
        while (i < na && j < nb) {                                                      \
            int take_left = (ORACLE_MUTANT == 1) ? !LE(bk[j], ak[i]) : LE(ak[i], bk[j]); \
            if (take_left) {                                                            \
                ok[o] = ak[i];                                                          \
                if (ov) ov[o] = av[i];                                                  \
                ++i;                                                                    \
            } else {                                                                    \
                ok[o] = bk[j];                                                          \
                if (ov) ov[o] = bv[j];                                                  \
                ++j;                                                                    \
            }                                                                           \
            ++o;                                                                        \
        }                                                                               \
        for (; i < na; ++i, ++o) {                                                      \
            ok[o] = ak[i];                                                              \
            if (ov) ov[o] = av[i];                                                      \
        }                                                                               \
        if (ORACLE_MUTANT != 2) {                                                       \
            for (; j < nb; ++j, ++o) {                                                  \
                ok[o] = bk[j];                                                          \
                if (ov) ov[o] = bv[j];                                                  \
            }                                                                           \
        }                                                                               \
    }                                                                                   \
                                                                                        \
    /* Sort k[0:n) (and v alongside) using t[0:n) as merge space. */                    \
    static void msort_rec_##SUF(KT* k, uint32_t* v, size_t n, KT* tk, uint32_t* tv) {   \
        if (n < 2) return;                                                              \
        size_t mid = n / 2;                                                             \
        size_t rbeg = (ORACLE_MUTANT == 3) ? mid - mid / 2 : mid;                       \
        msort_rec_##SUF(k, v, mid, tk, tv);                                             \
        msort_rec_##SUF(k + rbeg, v ? v + rbeg : 0, n - rbeg, tk, tv);                  \
        merge_##SUF(k, v, mid, k + mid, v ? v + mid : 0, n - mid, tk, tv);              \
        memcpy(k, tk, n * sizeof(KT));                                                  \
        if (v) memcpy(v, tv, n * sizeof(uint32_t));                                     \
    }                                                                                   \
                                                                                        \
    int oracle_sort_##SUF(KT* keys, uint32_t* vals, size_t n) {                         \
        if (n < 2) return 0;                                                            \
        KT* tk = (KT*)malloc(n * sizeof(KT));                                           \
        uint32_t* tv = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : 0;              \
        if (!tk || (vals && !tv)) {                                                     \
            free(tk);                                                                   \
            free(tv);                                                                   \
            return -1;                                                                  \
        }                                                                               \
        msort_rec_##SUF(keys, vals, n, tk, tv);                                         \
        free(tk);                                                                       \
        free(tv);                                                                       \
        return 0;                                                                       \
    }                                                                                   \
                                                                                        \
    void oracle_merge_##SUF(const KT* ak, const uint32_t* av, size_t na, const KT* bk,  \
                            const uint32_t* bv, size_t nb, KT* ok, uint32_t* ov) {     \
        merge_##SUF(ak, av, na, bk, bv, nb, ok, ov);                                    \
    }                                                                                   \
                                                                                        \
    /* Elements of A among the first d outputs of merge(A, B), by running it. */        \
    int64_t oracle_corank_##SUF(const KT* a, size_t na, const KT* b, size_t nb,         \
                                size_t d) {                                             \
        if (d > na + nb) return -1;                                                     \
        size_t i = 0, j = 0;                                                            \
        while (i + j < d) {                                                             \
            int take_left = (j >= nb) || (i < na && LE(a[i], b[j]));                    \
            if (ORACLE_MUTANT == 4 && i < na && j < nb && a[i] == b[j]) take_left = 0;  \
            if (take_left)                                                              \
                ++i;                                                                    \
            else                                                                        \
                ++j;                                                                    \
        }                                                                               \
        return (int64_t)i;                                                              \
    }                                                                                   \
                                                                                        \
    int oracle_segmented_sort_##SUF(KT* keys, uint32_t* vals, const uint64_t* off,      \
                                    size_t nseg) {                                      \
        for (size_t s = 0; s < nseg; ++s) {                                             \
            size_t b = (size_t)off[s], e = (size_t)off[s + 1];                          \
            if (e < b) return -2;                                                       \
            if (oracle_sort_##SUF(keys + b, vals ? vals + b : 0, e - b)) return -1;     \
        }                                                                               \
        return 0;                                                                       \
    }                                                                                   \
                                                                                        \
    typedef struct {                                                                    \
        KT* k;                                                                          \
        uint32_t* v;                                                                    \
        size_t n;                                                                       \
        KT* tk;                                                                         \
        uint32_t* tv;                                                                   \
        size_t mid; /* merge jobs: left run is [0, mid) */                              \
    } job_##SUF;                                                                        \
                                                                                        \
    static void* sort_job_##SUF(void* p) {                                              \
        job_##SUF* j = (job_##SUF*)p;                                                   \
        msort_rec_##SUF(j->k, j->v, j->n, j->tk, j->tv);                                \
        return 0;                                                                       \
    }                                                                                   \
                                                                                        \
    static void* merge_job_##SUF(void* p) {                                             \
        job_##SUF* j = (job_##SUF*)p;                                                   \
        merge_##SUF(j->k, j->v, j->mid, j->k + j->mid, j->v ? j->v + j->mid : 0,        \
                    j->n - j->mid, j->tk, j->tv);                                       \
        memcpy(j->k, j->tk, j->n * sizeof(KT));                                         \
        if (j->v) memcpy(j->v, j->tv, j->n * sizeof(uint32_t));                         \
        return 0;                                                                       \
    }                                                                                   \
                                                                                        \
    int oracle_par_sort_##SUF(KT* keys, uint32_t* vals, size_t n, int workers) {        \
        if (workers < 1) workers = 1;                                                   \
        if (n < 2) return 0;                                                            \
        size_t size = (n + (size_t)workers - 1) / (size_t)workers; /* ceil(n/p) */      \
        size_t nchunk = (n + size - 1) / size;                                          \
        KT* tk = (KT*)malloc(n * sizeof(KT));                                           \
        uint32_t* tv = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : 0;              \
        job_##SUF* jobs = (job_##SUF*)calloc(nchunk, sizeof(job_##SUF));                \
        pthread_t* th = (pthread_t*)calloc(nchunk, sizeof(pthread_t));                  \
        size_t* beg = (size_t*)calloc(nchunk + 1, sizeof(size_t));                      \
        int* started = (int*)calloc(nchunk, sizeof(int));                               \
        if (!tk || (vals && !tv) || !jobs || !th || !beg || !started) {                 \
            free(tk); free(tv); free(jobs); free(th); free(beg); free(started);         \
            return -1;                                                                  \
        }                                                                               \
        for (size_t c = 0; c <= nchunk; ++c) beg[c] = c * size < n ? c * size : n;      \
        for (size_t c = 0; c < nchunk; ++c) {                                           \
            job_##SUF jb = {keys + beg[c], vals ? vals + beg[c] : 0, beg[c + 1] - beg[c], \
                            tk + beg[c], tv ? tv + beg[c] : 0, 0};                      \
            jobs[c] = jb;                                                               \
            started[c] = !pthread_create(&th[c], 0, sort_job_##SUF, &jobs[c]);          \
            if (!started[c]) sort_job_##SUF(&jobs[c]);                                  \
        }                                                                               \
        for (size_t c = 0; c < nchunk; ++c)                                             \
            if (started[c]) pthread_join(th[c], 0);                                     \
        /* Merge tree: run r absorbs run r + step while step < #runs. */                \
        for (size_t step = 1; step < nchunk; step *= 2) {                               \
            size_t nj = 0;                                                              \
            for (size_t r = 0; r + step < nchunk; r += 2 * step) {                      \
                size_t e = (r + 2 * step < nchunk) ? beg[r + 2 * step] : n;             \
                job_##SUF jb = {keys + beg[r], vals ? vals + beg[r] : 0, e - beg[r],    \
                                tk + beg[r], tv ? tv + beg[r] : 0,                      \
                                beg[r + step] - beg[r]};                                \
                jobs[nj] = jb;                                                          \
                started[nj] = !pthread_create(&th[nj], 0, merge_job_##SUF, &jobs[nj]);  \
                if (!started[nj]) merge_job_##SUF(&jobs[nj]);                           \
                ++nj;                                                                   \
            }                                                                           \
            for (size_t q = 0; q < nj; ++q)                                             \
                if (started[q]) pthread_join(th[q], 0);                                 \
        }                                                                               \
        free(tk); free(tv); free(jobs); free(th); free(beg); free(started);             \
        return 0;                                                                       \
    }

/* Key orders.  Unsigned and signed keys: the integers' own order.
 * Floating-point keys (held as their bit patterns): the totalOrder relation
 * of IEEE 754 (2008/2019, clause 5.10): a value with the sign bit set comes
 * before one without (so -0 < +0 and -NaN before everything); among
 * non-negative patterns the larger magnitude field is the larger value
 * (+inf below +NaN, NaNs by payload); among negative ones the larger
 * magnitude is the smaller value. */
#define NATIVE_LE(a, b) ((a) <= (b))
static int total_le_f32(uint32_t a, uint32_t b) {
    const int na = (a >> 31) != 0, nb = (b >> 31) != 0;
    if (na != nb) return na;
    return na ? a >= b : a <= b;
}
static int total_le_f64(uint64_t a, uint64_t b) {
    const int na = (a >> 63) != 0, nb = (b >> 63) != 0;
    if (na != nb) return na;
    return na ? a >= b : a <= b;
}

DEFINE_ORACLE(u32, uint32_t, NATIVE_LE)
DEFINE_ORACLE(u64, uint64_t, NATIVE_LE)
DEFINE_ORACLE(i32, int32_t, NATIVE_LE)
DEFINE_ORACLE(i64, int64_t, NATIVE_LE)
DEFINE_ORACLE(f32, uint32_t, total_le_f32)
DEFINE_ORACLE(f64, uint64_t, total_le_f64)

int oracle_mutant_id(void) { return ORACLE_MUTANT; }
