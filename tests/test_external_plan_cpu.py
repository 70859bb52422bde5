"""Host logic of the out-of-core sort (no GPU): the merge blocks it derives
from sampled (key, position) splitters over sorted runs in host memory
(msort_external_plan, the same code the sort runs).

For every input the cuts must start at 0 and end at each run's length,
never decrease, keep every block within its bound, and partition the
(key, position) order: everything before a block boundary, in any run,
precedes everything after it in any run.  Then merging each block's slices
and concatenating the blocks gives the stable sort of the whole array.
Inputs: random keys, all-equal keys (split by position alone), presorted
and reverse-sorted arrays, 64-bit keys with duplicates, many runs with the
smallest allowed bound, and a ragged last run.
"""
import numpy as np
import pytest

ms = pytest.importorskip("paper_2211_16479_gb300")


def _runs(keys, chunk):
    out = keys.copy()
    for o in range(0, len(keys), chunk):
        out[o:o + chunk] = np.sort(out[o:o + chunk], kind="stable")
    return out


def _check(runs, chunk, bound):
    cuts = ms.msort_external_plan(runs, chunk, bound).astype(np.int64)
    nruns = cuts.shape[1]
    lens = [min(chunk, len(runs) - r * chunk) for r in range(nruns)]
    assert (cuts[0] == 0).all() and list(cuts[-1]) == lens
    steps = np.diff(cuts, axis=0)
    assert (steps >= 0).all()
    sizes = steps.sum(axis=1)
    assert sizes.max() <= bound, (sizes.max(), bound)
    assert sizes.sum() == len(runs)
    for b in range(1, cuts.shape[0] - 1):
        before, after = [], []
        for r in range(nruns):
            off, c = r * chunk, int(cuts[b, r])
            if c > 0:
                before.append((int(runs[off + c - 1]), off + c - 1))
            if c < lens[r]:
                after.append((int(runs[off + c]), off + c))
        if before and after:
            assert max(before) < min(after), b
    return sizes


RNG = np.random.default_rng(2211)


@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "reverse", "few_values"])
@pytest.mark.parametrize("bound_div", [2, 7])
def test_blocks_u32(kind, bound_div):
    n, chunk = 200_003, 12_000  # 17 runs, the last one ragged
    if kind == "random":
        keys = RNG.integers(0, 2 ** 32, size=n, dtype=np.uint32)
    elif kind == "equal":
        keys = np.full(n, 7, dtype=np.uint32)
    elif kind == "sorted":
        keys = np.sort(RNG.integers(0, 2 ** 32, size=n, dtype=np.uint32))
    elif kind == "reverse":
        keys = np.sort(RNG.integers(0, 2 ** 32, size=n, dtype=np.uint32))[::-1].copy()
    else:
        keys = RNG.integers(0, 3, size=n).astype(np.uint32)
    sizes = _check(_runs(keys, chunk), chunk, chunk // bound_div)
    assert len(sizes) >= n // (chunk // bound_div)


def test_blocks_u64_duplicates():
    n, chunk = 150_001, 9_000
    keys = RNG.integers(0, 50, size=n).astype(np.uint64) << np.uint64(40)
    _check(_runs(keys, chunk), chunk, chunk // 2)


def test_many_runs_smallest_bound():
    n, chunk = 60_000, 500  # 120 runs; the bound 2R is the smallest allowed
    keys = RNG.integers(0, 1000, size=n, dtype=np.uint32)
    _check(_runs(keys, chunk), chunk, 2 * 120)


def test_rejects_bound_below_two_runs():
    keys = np.arange(10_000, dtype=np.uint32)
    with pytest.raises(ValueError):
        ms.msort_external_plan(keys, 100, 150)  # 100 runs need a bound of at least 200
