"""msort_sort_noalloc: the sort for callers that may not allocate device memory.

Such callers (a framework that owns all device memory through its own pool,
or a latency-critical path that cannot take the synchronisation an
allocation may cause) get the same stable sort with scratch taken from a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test.  It checks,
through the C ABI, that two calls in a row give the same bytes as the
regular context-based entry point (integer sort: bit-exact), and that sizes
beyond the fixed scratch are rejected up front.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kt,pairs", [("u32", False), ("u32", True), ("u64", False), ("u64", True)])
def test_noalloc_matches_context_sort_twice(kt, pairs):
    need_gpu()
    ctx = ms.Context(0)
    try:
        for call, n in enumerate([(1 << 20) + 4097, 3 * 8448 + 11]):
            if kt == "u32":
                keys = synth.uniform_u32(n, 10 + call) % np.uint32(5000)
            else:
                keys, _ = synth.dup_u64(n, 10 + call, distinct=1 << 12)
            vals = np.arange(n, dtype=np.uint32) if pairs else None
            dk = to_dev(keys)
            dv = to_dev(vals) if pairs else None
            ref_k = torch.empty_like(dk)
            ref_v = torch.empty_like(dv) if pairs else None
            ms.msort_sort_copy(ctx.handle, dk, ref_k, dv, ref_v)
            out_k = torch.empty_like(dk)
            out_v = torch.empty_like(dv) if pairs else None
            ms.msort_sort_noalloc(dk, out_k, dv, out_v)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(out_k), to_host(ref_k)), f"keys differ on call {call}"
            if pairs:
                assert np.array_equal(to_host(out_v), to_host(ref_v)), f"values differ on call {call}"
    finally:
        ctx.close()


def test_noalloc_rejects_oversize():
    need_gpu()
    limit = ms.msort_noalloc_max_keys(ms.MSORT_U32, False)
    assert limit > 1 << 20
    d = torch.empty(limit + 1, dtype=torch.uint32, device="cuda")
    with pytest.raises(ms.MsortError) as e:
        ms.msort_sort_noalloc(d, d)
    assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    assert "no-allocation limit" in str(e.value)
