"""GPU parity of the four-way merge passes (two rounds of the merge tree per
pass over memory) against the CPU oracle, element by element.

Sizes are chosen per tile so that the number of merge rounds is odd and even
(the odd one starts with a pairwise pass), the last group of four runs is
complete, short by one to three runs, or a single partial run, and blocks end
in ragged tails.  Key patterns stress the grid positions: all keys equal
(every grid point ties), the largest key value (the one the merge uses as
padding), two values, sorted, reversed and organ-pipe inputs.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _sizes(T):
    return [T + 1, 2 * T + 5, 3 * T, 4 * T, 4 * T + 1, 5 * T + 17, 9 * T - 1, 16 * T + 3, 17 * T + T // 2,
            33 * T + 11, 64 * T + 1000]


def _pattern(name, n, seed, dtype):
    top = dtype(np.iinfo(dtype).max)
    if name == "uniform":
        k = synth.uniform_u32(n, seed) if dtype == np.uint32 else synth.uniform_u64(n, seed)
        return k.astype(dtype)
    if name == "equal":
        return np.full(n, 12345, dtype=dtype)
    if name == "max":
        return np.full(n, top, dtype=dtype)
    if name == "two":
        return np.where(synth.uniform_u32(n, seed) & np.uint32(1), top, dtype(0)).astype(dtype)
    if name == "few":
        return (synth.uniform_u32(n, seed) % np.uint32(7)).astype(dtype)
    if name == "sorted":
        return np.arange(n, dtype=dtype)
    if name == "reverse":
        return np.arange(n, 0, -1).astype(dtype)
    if name == "organ":
        h = np.arange(n, dtype=np.int64)
        return np.minimum(h, n - 1 - h).astype(dtype)
    raise ValueError(name)


PATTERNS = ["uniform", "equal", "max", "two", "few", "sorted", "reverse", "organ"]


@pytest.mark.parametrize("tile", [4352, 8448, 16896, 33792])
@pytest.mark.parametrize("pattern", PATTERNS)
def test_four_way_u32(ctx, tile, pattern):
    for i, n in enumerate(_sizes(tile)):
        keys = _pattern(pattern, n, 100 + i, np.uint32)
        exp, _ = oracle.sort(keys)
        for ways in (4, 2):
            d = to_dev(keys)
            ms.msort_sort(ctx, d, options={"tile": tile, "merge_ways": ways})
            got = to_host(d)
            assert np.array_equal(got, exp), (n, ways)


@pytest.mark.parametrize("tile", [4352, 8704])
@pytest.mark.parametrize("pattern", ["uniform", "max", "two", "few", "reverse"])
def test_four_way_u64(ctx, tile, pattern):
    for i, n in enumerate(_sizes(tile)[::2]):
        keys = _pattern(pattern, n, 200 + i, np.uint64)
        if pattern == "uniform":
            keys[::5] = np.uint64(0xFFFFFFFFFFFFFFFF)
        exp, _ = oracle.sort(keys)
        d = to_dev(keys)
        ms.msort_sort(ctx, d, options={"tile": tile, "merge_ways": 4}, key_type=ms.MSORT_U64)
        assert np.array_equal(to_host(d), exp), n


def test_four_way_distributions(ctx):
    # 2^22 + 3 keys of every benchmark distribution
    n = (1 << 22) + 3
    for j, name in enumerate(synth.DIST_NAMES):
        keys = synth.u32_distribution(name, n, 31 + j)
        exp, _ = oracle.sort(keys)
        d = to_dev(keys)
        ms.msort_sort(ctx, d, options={"merge_ways": 4})
        assert np.array_equal(to_host(d), exp), name


def test_four_way_options_rejected(ctx):
    keys = to_dev(synth.uniform_u32(100000, 5))
    vals = to_dev(np.arange(100000, dtype=np.uint32))
    with pytest.raises(ms.MsortError):
        ms.msort_sort(ctx, keys, options={"merge_ways": 3})
    with pytest.raises(ms.MsortError):
        ms.msort_sort_pairs(ctx, keys, vals, options={"merge_ways": 4})
    with pytest.raises(ms.MsortError):
        ms.msort_sort(ctx, keys, options={"merge_ways": 4, "partition_mode": 1})
    ms.msort_ctx_sync(ctx)
