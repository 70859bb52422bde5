"""GPU parity: the plain merge sort against the CPU oracle, element by element.

Keys-only and key-value sorts, 32- and 64-bit keys, every tile size, sizes
that span several tiles with ragged tails, the empty and one-element cases,
and the five 2^28 key distributions at reduced size.  Integer results must be
bit-exact; values are original indices, so stability is checked exactly.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import is_sorted_dev, multiset_hash, need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 16, 17, 18, 33, 34, 511, 4351, 4352, 4353, 8447, 8448, 8449, 3 * 8448 + 5, 16896, 16897,
         65536, 65537, 3 * 65536 + 77, (1 << 20) + 12345]
TILES = [4352, 8448, 8704, 16896, 33792]


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _keys(name, n, seed, dtype):
    if dtype == np.uint32:
        return synth.u32_distribution(name, n, seed)
    if name == "dup64":
        return synth.dup_u64(n, seed)[0]
    return synth.uniform_u64(n, seed)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("n", SIZES)
def test_keys_u32_uniform(ctx, n, tile):
    keys = synth.uniform_u32(n, 1) % np.uint32(max(1, n // 3) if n % 2 else 0xFFFFFFFF)
    d = to_dev(keys)
    ms.msort_sort(ctx, d, options={"tile": tile})
    exp, _ = oracle.sort(keys)
    assert np.array_equal(to_host(d), exp)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("n", [1, 33, 4353, 3 * 8448 + 5, 65537, (1 << 20) + 12345])
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_pairs_stable(ctx, n, tile, kt):
    if kt == "u32":
        keys = synth.uniform_u32(n, 2) % np.uint32(97)   # heavy duplicates
    else:
        keys, _ = synth.dup_u64(n, 2, distinct=211)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = to_dev(keys), to_dev(vals)
    key_type = ms.MSORT_U32 if kt == "u32" else ms.MSORT_U64
    if ms.msort_scratch_bytes(max(n, 1), key_type, True, {"tile": tile}) == 0:
        with pytest.raises(ms.MsortError):   # this tile shape is not offered for these items
            ms.msort_sort_pairs(ctx, dk, dv, options={"tile": tile})
        return
    ms.msort_sort_pairs(ctx, dk, dv, options={"tile": tile})
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(dk), ek)
    assert np.array_equal(to_host(dv), ev)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("n", [0, 5, 4352, 12345, (1 << 19) + 3])
def test_keys_u64(ctx, n, tile):
    if tile == 33792:
        with pytest.raises(ms.MsortError):
            ms.msort_sort(ctx, to_dev(synth.uniform_u64(max(n, 1), 3)), options={"tile": tile})
        return
    keys = synth.uniform_u64(n, 3)
    if n > 10:
        keys[::7] = np.uint64(0xFFFFFFFFFFFFFFFF)  # the maximum key must not be taken for padding
    d = to_dev(keys)
    ms.msort_sort(ctx, d, options={"tile": tile})
    exp, _ = oracle.sort(keys)
    assert np.array_equal(to_host(d), exp)


@pytest.mark.parametrize("name", list(synth.DIST_NAMES) + ["lognormal3"])
def test_distributions_reduced_size(ctx, name):
    n = (1 << 21) + 999
    keys = synth.u32_distribution(name, n, 4)
    d = to_dev(keys)
    ms.msort_sort(ctx, d)
    exp, _ = oracle.sort(keys)
    assert np.array_equal(to_host(d), exp)


def test_out_of_place_leaves_input(ctx):
    n = 100000
    keys = synth.zipf_u32(n, 5)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = to_dev(keys), to_dev(vals)
    ok = torch.empty_like(dk)
    ov = torch.empty_like(dv)
    ms.msort_sort_copy(ctx, dk, ok, dv, ov)
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(ok), ek) and np.array_equal(to_host(ov), ev)
    assert np.array_equal(to_host(dk), keys) and np.array_equal(to_host(dv), vals)


def test_unaligned_buffers(ctx):
    # offsets that break 16-byte alignment take the scalar load/store paths
    n = 50000
    keys = synth.uniform_u32(n + 3, 6)
    big = to_dev(keys)
    view = big[1:1 + n]
    ms.msort_sort(ctx, view)
    exp, _ = oracle.sort(keys[1:1 + n])
    out = to_host(big)
    assert np.array_equal(out[1:1 + n], exp)
    assert out[0] == keys[0] and np.array_equal(out[1 + n:], keys[1 + n:])


def test_host_buffers(ctx):
    n = 300001
    keys = synth.distinct16_u32(n, 7)
    vals = np.arange(n, dtype=np.uint32)
    hk = keys.copy()
    hv = vals.copy()
    ms.msort_sort_host(ctx, hk, hv)
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(hk, ek) and np.array_equal(hv, ev)


def test_invalid_arguments(ctx):
    d = to_dev(np.arange(10, dtype=np.uint32))
    with pytest.raises(ms.MsortError) as e:
        ms.msort_sort(ctx, d, options={"tile": 1000})
    assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    with pytest.raises(ms.MsortError):
        ms.msort_sort(ctx, d, options={"partition_mode": 7})
    with pytest.raises(ms.MsortError):
        ms.msort_sort(ctx, d, options={"merge_block": 1000})
    with pytest.raises(ms.MsortError):
        ms.msort_sort(ctx, d, options={"tile": 4096})
    with pytest.raises(ms.MsortError):
        ms.msort_sort_copy(ctx, d, d, d, None)


def test_budget_refuses_oversize(ctx):
    small = ms.Context(0, scratch_budget_bytes=1 << 16)
    try:
        d = to_dev(synth.uniform_u32(1 << 20, 1))
        with pytest.raises(ms.MsortError) as e:
            ms.msort_sort(small.handle, d)
        assert e.value.status == ms.MSORT_ERR_OOM
    finally:
        small.close()


@pytest.mark.parametrize("name", synth.DIST_NAMES)
def test_full_size_2_28(ctx, name):
    """2^28 keys, the benchmark's launch configuration; bit-exact against the
    oracle's chunked variant on every host core."""
    import os
    from synth import torch_gen
    n = 1 << 28
    d = torch_gen.u32_distribution(name, n, 1, device="cuda")
    keys = to_host(d)
    out = torch.empty_like(d)
    ms.msort_sort_copy(ctx, d, out)
    assert is_sorted_dev(out)
    assert multiset_hash(out) == multiset_hash(d)
    exp, _ = oracle.par_sort(keys, workers=len(os.sched_getaffinity(0)))
    assert np.array_equal(to_host(out), exp)


def test_full_size_pairs_2_27(ctx):
    """2^27 (uint64 key, uint32 original index) pairs with keys from 2^20
    distinct values, the key-value benchmark's launch configuration;
    bit-exact (keys and values, so stability too) against the oracle."""
    import os
    from synth import torch_gen
    n = 1 << 27
    dk, dv = torch_gen.dup_u64(n, 1, device="cuda")
    ok, ov = torch.empty_like(dk), torch.empty_like(dv)
    ms.msort_sort_copy(ctx, dk, ok, dv, ov)
    ek, ev = oracle.par_sort(to_host(dk), to_host(dv), workers=len(os.sched_getaffinity(0)))
    assert np.array_equal(to_host(ok), ek)
    assert np.array_equal(to_host(ov), ev)


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("pairs", [False, True])
def test_graph_replay(ctx, kt, pairs):
    # options.use_graph: the first call captures the launch sequence, later
    # calls on the same buffers replay it on new data
    for n in (1000, 16897, (1 << 20) + 3):
        dk = torch.empty(n, dtype=torch.uint32 if kt == "u32" else torch.uint64, device="cuda")
        dv = torch.empty(n, dtype=torch.uint32, device="cuda") if pairs else None
        ok = torch.empty_like(dk)
        ov = torch.empty_like(dv) if pairs else None
        for rep in range(3):
            keys = (synth.uniform_u32(n, 50 + rep) % np.uint32(5000)) if kt == "u32" else \
                synth.dup_u64(n, 50 + rep, distinct=5000)[0]
            vals = np.arange(n, dtype=np.uint32)
            dk.copy_(torch.from_numpy(keys))
            if pairs:
                dv.copy_(torch.from_numpy(vals))
            ms.msort_sort_copy(ctx, dk, ok, dv, ov, options={"use_graph": 1})
            ek, ev = oracle.sort(keys, vals)
            assert np.array_equal(to_host(ok), ek), (n, rep)
            if pairs:
                assert np.array_equal(to_host(ov), ev), (n, rep)
        # in place, replayed twice
        for rep in range(2):
            keys = synth.zipf_u32(n, 70 + rep).astype(np.uint32 if kt == "u32" else np.uint64)
            dk.copy_(torch.from_numpy(keys))
            ms.msort_sort(ctx, dk, options={"use_graph": 1})
            assert np.array_equal(to_host(dk), oracle.sort(keys)[0])


def test_graph_cache_evicts(ctx):
    # more distinct (buffers, size) launch sequences than a context keeps as
    # graphs (64): every result stays exact, and the evicted ones, met again,
    # are captured again
    buf = torch.empty(2000, dtype=torch.uint32, device="cuda")
    out = torch.empty_like(buf)
    for rep in range(2):
        for i in range(70):
            n = 1000 + 7 * i
            keys = synth.uniform_u32(n, 300 + 70 * rep + i)
            buf[:n].copy_(torch.from_numpy(keys))
            ms.msort_sort_copy(ctx, buf[:n], out[:n], options={"use_graph": 1})
            assert np.array_equal(to_host(out[:n]), oracle.sort(keys)[0]), (rep, n)
