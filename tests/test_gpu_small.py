"""Single-launch sort (one cooperative launch for the tile sort and every
merge round, grid barriers between rounds) against the CPU oracle.

The automatic plan takes it for arrays of up to 2^22 elements with default
options; options.single_launch = 1 forces it (up to 2^28), -1 forbids it.
Sizes cover one partial tile, exact tile multiples, ragged tails, odd round
counts, an unpaired last run, the automatic limit, and a forced size larger
than the grid (blocks loop over tiles and merge blocks).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _keys(kind, n, seed, dtype=np.uint32):
    if kind == "uniform":
        k = synth.uniform_u64(n, seed)
        return (k.astype(np.uint32) if dtype == np.uint32 else k).astype(dtype)
    if kind == "few":
        return (synth.uniform_u64(n, seed) % np.uint64(7)).astype(dtype)
    if kind == "sorted":
        return np.sort(synth.uniform_u64(n, seed)).astype(dtype)
    if kind == "reverse":
        return np.sort(synth.uniform_u64(n, seed))[::-1].astype(dtype).copy()
    return np.full(n, np.iinfo(dtype).max, dtype=dtype)  # all equal to the largest key


def _sort_and_check(ctx, keys, vals, options):
    dk = to_dev(keys)
    dv = to_dev(vals) if vals is not None else None
    ok = torch.empty_like(dk)
    ov = torch.empty_like(dv) if dv is not None else None
    ms.msort_sort_copy(ctx, dk, ok, dv, ov, options=options)
    ms.msort_ctx_sync(ctx)
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(ok), ek)
    if vals is not None:
        assert np.array_equal(to_host(ov), ev)


# default single-launch tiles: 4352 / 8704 / 16896 for 32-bit keys, 2816 / 8448 (4352 for 64-bit pairs) otherwise
SIZES = [1, 2, 4351, 4352, 4353, 8447, 8448, 8449, 16895, 16896, 16897, 3 * 16896 + 7, 5 * 8448 + 1,
         (1 << 16) + 13, 1 << 20, (1 << 20) + 12345]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype,pairs", [(np.uint32, False), (np.uint32, True), (np.uint64, False),
                                         (np.uint64, True)])
def test_single_launch_matches_oracle(ctx, n, dtype, pairs):
    kt = ms.MSORT_U32 if dtype == np.uint32 else ms.MSORT_U64
    tile, W, passes = ms.msort_plan_info(n, kt, pairs)
    _, _, p_multi = ms.msort_plan_info(n, kt, pairs, {"single_launch": -1})
    keys = _keys("few" if n % 2 else "uniform", n, n % 1000 + 3, dtype)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    before = ms.msort_ctx_launch_count(ctx)
    _sort_and_check(ctx, keys, vals, None)
    assert ms.msort_ctx_launch_count(ctx) - before == 1  # the whole sort is one launch
    assert tile == W and passes == max(0, int(np.ceil(np.log2(max(n, 1) / tile))))
    assert p_multi >= 0


@pytest.mark.parametrize("kind", ["sorted", "reverse", "equal", "few"])
def test_single_launch_structured_keys(ctx, kind):
    n = (1 << 20) + 77
    keys = _keys(kind, n, 5)
    _sort_and_check(ctx, keys, np.arange(n, dtype=np.uint32), None)
    _sort_and_check(ctx, keys, None, None)


def test_single_launch_signed_and_float_keys(ctx):
    n = 300001
    bits = synth.uniform_u64(n, 9).astype(np.uint32)
    for dtype in (np.int32, np.float32):
        keys = bits.view(dtype)
        d = to_dev(keys)
        out = torch.empty_like(d)
        ms.msort_sort_copy(ctx, d, out)
        ms.msort_ctx_sync(ctx)
        ek, _ = oracle.sort(keys)
        assert np.array_equal(to_host(out).view(np.uint32), ek.view(np.uint32)), dtype


def test_single_launch_forced_beyond_the_grid(ctx):
    # 2^24 + 3 keys: 993 tiles, more than one cooperative grid holds, so blocks loop
    n = (1 << 24) + 3
    keys = _keys("uniform", n, 11)
    _sort_and_check(ctx, keys, None, {"single_launch": 1})
    _sort_and_check(ctx, keys[: 1 << 22], np.arange(1 << 22, dtype=np.uint32), {"single_launch": 1})


def test_single_launch_in_place_and_graph_replay(ctx):
    n = (1 << 20) + 5
    keys = _keys("uniform", n, 13)
    ek, _ = oracle.sort(keys)
    d = to_dev(keys)
    out = torch.empty_like(d)
    for _ in range(3):  # captured once, then replayed
        ms.msort_sort_copy(ctx, d, out, options={"use_graph": 1})
        ms.msort_ctx_sync(ctx)
        assert np.array_equal(to_host(out), ek)
    ms.msort_sort(ctx, d)  # in place
    ms.msort_ctx_sync(ctx)
    assert np.array_equal(to_host(d), ek)


def test_single_launch_option_checks(ctx):
    n = 1 << 20
    t_auto = ms.msort_plan_info(n, ms.MSORT_U32, False)
    t_multi = ms.msort_plan_info(n, ms.MSORT_U32, False, {"single_launch": -1})
    assert t_auto[0] == 8704 and t_multi[0] == 16896  # 512 x 17 single launch vs 512 x 33 tiles
    assert ms.msort_plan_info(1 << 16, ms.MSORT_U32, False)[0] == 4352  # 256 x 17 up to 2^19 keys
    assert ms.msort_plan_info(1 << 16, ms.MSORT_U64, True)[0] == 2816  # 256 x 11 for other types
    for tile in (2816, 4352, 5632, 8704, 11264, 16896):  # every single-launch shape of 32-bit keys
        keys = _keys("uniform", 300007, tile)
        _sort_and_check(ctx, keys, None, {"single_launch": 1, "tile": tile})
    # larger than the automatic limit: the multi-launch plan unless forced
    assert ms.msort_plan_info((1 << 22) + 1, ms.MSORT_U64, False)[0] != \
        ms.msort_plan_info((1 << 22) + 1, ms.MSORT_U64, False, {"single_launch": 1})[0]
    for bad in ({"single_launch": 2}, {"single_launch": 1, "tile": 33792}, {"single_launch": 1, "merge_block": 8448},
                {"single_launch": 1, "partition_mode": 1}, {"single_launch": 1, "merge_ways": 4}):
        with pytest.raises(ms.MsortError) as e:
            ms.msort_plan_info(n, ms.MSORT_U32, False, bad)
        assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    with pytest.raises(ms.MsortError):
        ms.msort_plan_info((1 << 28) + 1, ms.MSORT_U32, False, {"single_launch": 1})


def test_concurrent_single_launches_on_several_streams():
    """Single-launch sorts issued on four streams of four contexts at once
    (their cooperative grids may run concurrently): every result is exact
    and no grid barrier reports a timeout."""
    need_gpu()
    ctxs = [ms.Context(0) for _ in range(4)]
    streams = [torch.cuda.Stream() for _ in range(4)]
    sizes = [(1 << 20) + 11, 1 << 22, (1 << 18) + 3, 3 * 8704 + 1]
    try:
        keys = [_keys("uniform", n, 40 + i) for i, n in enumerate(sizes)]
        exp = [oracle.sort(k)[0] for k in keys]
        dev = [to_dev(k) for k in keys]
        outs = [torch.empty_like(d) for d in dev]
        torch.cuda.synchronize()
        for _ in range(5):
            for c, s, d, o in zip(ctxs, streams, dev, outs):
                ms.msort_sort_copy(c.handle, d, o, stream=s)
        for c, s in zip(ctxs, streams):
            ms.msort_ctx_sync(c.handle, s)
        for o, e in zip(outs, exp):
            assert np.array_equal(to_host(o), e)
    finally:
        for c in ctxs:
            c.close()


EDGE_SIZES = [0, 31, 32, 33] + [s for k in (10, 13, 15, 17, 19, 21, 22) for s in ((1 << k), (1 << k) + 1)]


@pytest.mark.parametrize("n", EDGE_SIZES)
@pytest.mark.parametrize("dtype,pairs", [(np.uint32, False), (np.uint64, True)])
def test_single_launch_edge_sizes(ctx, n, dtype, pairs):
    """The sizes of the survey's list (0, 31, 32, 33, 2^k, 2^k + 1) with
    default options, up to the automatic limit 2^22 + 1 (the first size that
    takes the multi-launch plan)."""
    keys = _keys("uniform", n, n % 997 + 1, dtype)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    _sort_and_check(ctx, keys, vals, None)


def test_single_launch_unaligned_pairs(ctx):
    # views one element into larger buffers: the windows take scalar heads and tails
    n = 70001
    keys = _keys("few", n + 2, 4, np.uint64)
    vals = np.arange(n + 2, dtype=np.uint32)
    dk, dv = to_dev(keys), to_dev(vals)
    ok = torch.empty(n + 2, dtype=dk.dtype, device="cuda")
    ov = torch.empty(n + 2, dtype=dv.dtype, device="cuda")
    ms.msort_sort_copy(ctx, dk[1:1 + n], ok[1:1 + n], dv[1:1 + n], ov[1:1 + n])
    ms.msort_ctx_sync(ctx)
    ek, ev = oracle.sort(keys[1:1 + n], vals[1:1 + n])
    assert np.array_equal(to_host(ok)[1:1 + n], ek) and np.array_equal(to_host(ov)[1:1 + n], ev)
