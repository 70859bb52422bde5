"""msort_sort_noalloc: the sort for callers that may not allocate device memory.

Such callers (a framework that owns all device memory through its own pool,
or a latency-critical path that cannot take the synchronisation an
allocation may cause) get the same stable sort with scratch taken from a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test.  Through
the C ABI it checks the entry point against the CPU oracle and against the
regular context-based entry point (integer sort: bit-exact) on two calls in
a row, in place for both parities of the merge-pass count, exactly at the
size limit for every key/value type, that sizes beyond the limit are
rejected up front, and that a call leaves the device's free memory
unchanged.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu

TYPES = [("u32", False), ("u32", True), ("u64", False), ("u64", True)]
# merge passes after the 8448-key tile sort: 7 (odd) and 2 (even)
SIZES = [(1 << 20) + 4097, 3 * 8448 + 11]


def _inputs(kt, pairs, n, seed):
    if kt == "u32":
        keys = synth.uniform_u32(n, seed) % np.uint32(5000)
    else:
        keys, _ = synth.dup_u64(n, seed, distinct=1 << 12)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    return keys, vals


def _check_oracle(keys, vals, out_k, out_v, what):
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(out_k), ek), f"keys differ from the oracle ({what})"
    if vals is not None:
        assert np.array_equal(to_host(out_v), ev), f"values differ from the oracle ({what})"


@pytest.mark.parametrize("kt,pairs", TYPES)
def test_noalloc_matches_oracle_and_context_sort_twice(kt, pairs):
    need_gpu()
    ctx = ms.Context(0)
    try:
        for call, n in enumerate(SIZES):
            keys, vals = _inputs(kt, pairs, n, 10 + call)
            dk = to_dev(keys)
            dv = to_dev(vals) if pairs else None
            ref_k = torch.empty_like(dk)
            ref_v = torch.empty_like(dv) if pairs else None
            ms.msort_sort_copy(ctx.handle, dk, ref_k, dv, ref_v)
            out_k = torch.empty_like(dk)
            out_v = torch.empty_like(dv) if pairs else None
            ms.msort_sort_noalloc(dk, out_k, dv, out_v)
            ms.msort_noalloc_sync()
            torch.cuda.synchronize()
            assert np.array_equal(to_host(out_k), to_host(ref_k)), f"keys differ on call {call}"
            if pairs:
                assert np.array_equal(to_host(out_v), to_host(ref_v)), f"values differ on call {call}"
            _check_oracle(keys, vals, out_k, out_v, f"call {call}")
    finally:
        ctx.close()


@pytest.mark.parametrize("kt,pairs", TYPES)
@pytest.mark.parametrize("n", SIZES)
def test_noalloc_in_place(kt, pairs, n):
    need_gpu()
    keys, vals = _inputs(kt, pairs, n, 20)
    dk = to_dev(keys)
    dv = to_dev(vals) if pairs else None
    ms.msort_sort_noalloc(dk, dk, dv, dv)
    ms.msort_noalloc_sync()
    _check_oracle(keys, vals, dk, dv, "in place")


@pytest.mark.parametrize("kt,pairs", TYPES)
def test_noalloc_exactly_at_the_limit(kt, pairs):
    need_gpu()
    key_type = ms.MSORT_U32 if kt == "u32" else ms.MSORT_U64
    n = ms.msort_noalloc_max_keys(key_type, pairs)
    keys, vals = _inputs(kt, pairs, n, 30)
    dk = to_dev(keys)
    dv = to_dev(vals) if pairs else None
    out_k = torch.empty_like(dk)
    out_v = torch.empty_like(dv) if pairs else None
    ms.msort_sort_noalloc(dk, out_k, dv, out_v)
    ms.msort_noalloc_sync()
    _check_oracle(keys, vals, out_k, out_v, f"n = {n}, the limit")


def test_noalloc_leaves_free_device_memory_unchanged():
    need_gpu()
    n = SIZES[0]
    keys, vals = _inputs("u64", True, n, 40)
    dk, dv = to_dev(keys), to_dev(vals)
    out_k, out_v = torch.empty_like(dk), torch.empty_like(dv)
    ms.msort_sort_noalloc(dk, out_k, dv, out_v)  # loads the kernels' modules
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ms.msort_sort_noalloc(dk, out_k, dv, out_v)
    ms.msort_noalloc_sync()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    _check_oracle(keys, vals, out_k, out_v, "after the memory check")


def test_noalloc_rejects_oversize():
    need_gpu()
    limit = ms.msort_noalloc_max_keys(ms.MSORT_U32, False)
    assert limit > 1 << 20
    d = torch.empty(limit + 1, dtype=torch.uint32, device="cuda")
    with pytest.raises(ms.MsortError) as e:
        ms.msort_sort_noalloc(d, d)
    assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    assert "no-allocation limit" in str(e.value)
