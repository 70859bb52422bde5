"""Pins for the CPU oracle: facts fixed by the definition of a stable sort.

The stable sort of (key, original index) pairs is unique (Section "Sequential
Merge Sort" defines merge sort; a merge that takes from the left run on ties
is stable).  Each test below checks the oracle against something other than
itself: brute-force enumeration of all permutations, counting sort over a
small alphabet, numpy's stable argsort (a library routine), the invariants
(sorted, permutation, stable), and the closed-form split conditions of a
merge.  ``test_planted_mistakes_are_caught`` rebuilds the oracle with four
plausible mistakes and checks that these pins catch every one.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _stable_by_enumeration(keys):
    n = len(keys)
    found = []
    for perm in itertools.permutations(range(n)):
        ok = True
        for a, b in zip(perm, perm[1:]):
            if keys[a] > keys[b] or (keys[a] == keys[b] and a > b):
                ok = False
                break
        if ok:
            found.append(perm)
    assert len(found) == 1, "the stable order must be unique"
    return np.asarray(found[0], dtype=np.int64)


def _check_invariants(keys_in, vals_in, keys_out, vals_out):
    assert np.all(keys_out[:-1] <= keys_out[1:]), "not sorted"
    assert sorted(np.unique(keys_in, return_counts=True)[1].tolist()) == \
        sorted(np.unique(keys_out, return_counts=True)[1].tolist())
    ui, ci = np.unique(keys_in, return_counts=True)
    uo, co = np.unique(keys_out, return_counts=True)
    assert np.array_equal(ui, uo) and np.array_equal(ci, co), "not a permutation of the keys"
    if vals_out is not None:
        # values are original indices: a permutation, each key still attached
        assert np.array_equal(np.sort(vals_out), np.arange(len(keys_in), dtype=vals_out.dtype))
        assert np.array_equal(keys_in[vals_out.astype(np.int64)], keys_out)
        same = keys_out[:-1] == keys_out[1:]
        assert np.all(vals_out[:-1][same] < vals_out[1:][same]), "not stable"


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_brute_force_permutations(oracle_lib, dtype):
    rng = np.random.default_rng(7)
    for n in range(0, 9):
        reps = 1 if n == 8 else 4
        for r in range(reps):
            alphabet = 3 if r % 2 == 0 else 1000
            keys = rng.integers(0, alphabet, size=n).astype(dtype)
            if dtype == np.uint64 and r == 3:
                keys = keys + dtype(0xFFFFFFFF00000000)  # high words matter
            perm = _stable_by_enumeration(keys.tolist())
            k, v = oracle.sort(keys, np.arange(n, dtype=np.uint32), lib=oracle_lib)
            assert np.array_equal(v.astype(np.int64), perm)
            assert np.array_equal(k, keys[perm])


def test_exhaustive_small_alphabet(oracle_lib):
    # Every key vector over {0,1,2}^n: the stable sort is the counting sort.
    for n in range(0, 9):
        for tup in itertools.product(range(3), repeat=n):
            keys = np.asarray(tup, dtype=np.uint32)
            k, v = oracle.sort(keys, np.arange(n, dtype=np.uint32), lib=oracle_lib)
            exp_v = [i for c in range(3) for i in range(n) if tup[i] == c]
            exp_k = [c for c in range(3) for i in range(n) if tup[i] == c]
            assert v.tolist() == exp_v and k.tolist() == exp_k


GEN = {
    "uniform": lambda n, s: synth.uniform_u32(n, s),
    "sorted": lambda n, s: synth.sorted_u32(n, s),
    "reverse": lambda n, s: synth.reverse_u32(n, s),
    "distinct16": lambda n, s: synth.distinct16_u32(n, s),
    "zipf": lambda n, s: synth.zipf_u32(n, s),
    "lognormal3": lambda n, s: synth.lognormal3_u32(n, s),
    "dup64": lambda n, s: synth.dup_u64(n, s)[0],
    "uniform64": lambda n, s: synth.uniform_u64(n, s),
}


@pytest.mark.parametrize("name", sorted(GEN))
def test_matches_library_stable_sort(oracle_lib, name):
    n = (1 << 18) + 37
    keys = GEN[name](n, 3)
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.sort(keys, vals, lib=oracle_lib)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(v, order.astype(np.uint32))
    assert np.array_equal(k, keys[order])
    _check_invariants(keys, vals, k, v)
    k2, _ = oracle.sort(keys, None, lib=oracle_lib)
    assert np.array_equal(k2, k)


@pytest.mark.parametrize("workers", [1, 2, 3, 5, 8, 13])
def test_parallel_variant_equals_sequential(oracle_lib, workers):
    for n in (0, 1, 2, 7, 1000, 4097, 65536 + 3):
        keys, vals = synth.dup_u64(n, 11)
        if n > 7:
            keys = keys % np.uint64(97)   # heavy duplicates across chunks
        k1, v1 = oracle.sort(keys, vals, lib=oracle_lib)
        k2, v2 = oracle.par_sort(keys, vals, workers=workers, lib=oracle_lib)
        assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def _split_ok(a, b, d, i):
    na, nb = len(a), len(b)
    j = d - i
    if not (max(0, d - nb) <= i <= min(d, na)):
        return False
    c1 = i == 0 or j == nb or a[i - 1] <= b[j]
    c2 = i == na or j == 0 or b[j - 1] < a[i]
    return c1 and c2


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_corank_closed_form_conditions(oracle_lib, dtype):
    rng = np.random.default_rng(5)
    for trial in range(120):
        na, nb = rng.integers(0, 14, size=2)
        hi = [2, 4, 50][trial % 3]
        a = np.sort(rng.integers(0, hi, size=na)).astype(dtype)
        b = np.sort(rng.integers(0, hi, size=nb)).astype(dtype)
        for d in range(na + nb + 1):
            i = oracle.corank(a, b, d, lib=oracle_lib)
            sat = [x for x in range(na + 1) if _split_ok(a, b, d, x)]
            assert sat == [i], (a, b, d, i, sat)
    with pytest.raises(ValueError):
        oracle.corank(np.zeros(2, dtype), np.zeros(2, dtype), 5, lib=oracle_lib)


def test_merge_is_stable_concatenation(oracle_lib):
    rng = np.random.default_rng(9)
    for trial in range(50):
        na, nb = rng.integers(0, 300, size=2)
        a = np.sort(rng.integers(0, 20, size=na)).astype(np.uint32)
        b = np.sort(rng.integers(0, 20, size=nb)).astype(np.uint32)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ok, ov = oracle.merge(a, b, av, bv, lib=oracle_lib)
        cat = np.concatenate([a, b])
        order = np.argsort(cat, kind="stable")
        assert np.array_equal(ok, cat[order]) and np.array_equal(ov, order.astype(np.uint32))


def test_segmented_matches_per_segment_library_sort(oracle_lib):
    lens = np.asarray([0, 1, 5, 0, 33, 1, 700, 4096, 2, 0], dtype=np.int64)
    off = synth.segment_offsets(lens)
    n = int(off[-1])
    keys = synth.uniform_u32(n, 2) % np.uint32(50)
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.segmented_sort(keys, off, vals, lib=oracle_lib)
    for s in range(len(lens)):
        b, e = int(off[s]), int(off[s + 1])
        o = np.argsort(keys[b:e], kind="stable")
        assert np.array_equal(k[b:e], keys[b:e][o])
        assert np.array_equal(v[b:e], (o + b).astype(np.uint32))


def _pins_pass(lib) -> bool:
    """Run a compact version of the pins above; False when any fails."""
    try:
        rng = np.random.default_rng(1)
        for n in range(0, 7):
            for _ in range(3):
                keys = rng.integers(0, 3, size=n).astype(np.uint32)
                perm = _stable_by_enumeration(keys.tolist())
                k, v = oracle.sort(keys, np.arange(n, dtype=np.uint32), lib=lib)
                if not np.array_equal(v.astype(np.int64), perm):
                    return False
        keys = synth.zipf_u32(5000, 1)
        k, v = oracle.sort(keys, np.arange(5000, dtype=np.uint32), lib=lib)
        _check_invariants(keys, np.arange(5000, dtype=np.uint32), k, v)
        for trial in range(40):
            na, nb = rng.integers(0, 10, size=2)
            a = np.sort(rng.integers(0, 3, size=na)).astype(np.uint32)
            b = np.sort(rng.integers(0, 3, size=nb)).astype(np.uint32)
            for d in range(na + nb + 1):
                if not _split_ok(a, b, d, oracle.corank(a, b, d, lib=lib)):
                    return False
        return True
    except AssertionError:
        return False


def test_planted_mistakes_are_caught(tmp_path):
    # mutant 1: merge takes from the right run on ties (unstable)
    # mutant 2: merge drops the tail of the right run
    # mutant 3: the right half is taken from the wrong place (cf. Fig. 2's typo)
    # mutant 4: the co-rank counts ties from the wrong run
    assert _pins_pass(oracle.load(0))
    for m in (1, 2, 3, 4):
        lib = oracle.load(m, outdir=str(tmp_path))
        assert lib.oracle_mutant_id() == m
        assert not _pins_pass(lib), f"mutant {m} slipped through the pins"


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_split_points_is_the_rank_in_the_stable_sort(oracle_lib, dtype):
    """oracle.split_points against the oracle's stable sort: a splitter equal
    to element e (its key and position) has exactly as many elements before
    it as e's index in the stably sorted array; a splitter between two
    positions falls between their ranks."""
    rng = np.random.default_rng(13)
    for trial in range(60):
        n = int(rng.integers(0, 40))
        keys = rng.integers(0, [2, 5, 1000][trial % 3], size=n).astype(dtype)
        offset = int(rng.integers(0, 1 << 40))
        pos = np.arange(n, dtype=np.uint64) + np.uint64(offset)
        _, order = oracle.sort(keys, np.arange(n, dtype=np.uint32), lib=oracle_lib)
        rank = np.empty(n, dtype=np.int64)
        rank[order] = np.arange(n)
        cuts = oracle.split_points(keys, pos, keys, pos)
        assert np.array_equal(cuts.astype(np.int64), rank)
        if n:
            # (key, position - 0.5): just before e; (key, beyond every position): after all equal keys
            two = np.uint64(2)
            below = oracle.split_points(keys, pos * two + np.uint64(1), keys, pos * two)
            assert np.array_equal(below.astype(np.int64), rank)
            after = oracle.split_points(keys, pos, keys, np.full(n, offset + n, dtype=np.uint64))
            assert np.array_equal(after.astype(np.int64), [np.count_nonzero(keys <= k) for k in keys])
