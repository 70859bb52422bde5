"""Sorts past the 32-bit index range (maximum sizes), checked by properties
that hold at any size: the output is nondecreasing and has the same multiset
as the input (order-independent 64-bit hash, summed modulo 2^64).  For keys
alone these two properties determine the result exactly.  Both checks run
in chunks on the device, so the test needs about 3.5 bytes of free device
memory per input byte (skipped otherwise)."""
import pytest

from tests.gpu_util import multiset_hash, need_gpu, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu

CHUNK = 1 << 28


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()
    torch.cuda.empty_cache()


def _as_signed_order(x):
    # unsigned order as int64: uint32 widens, uint64 flips the sign bit
    if x.dtype == torch.uint32:
        return x.to(torch.int64)
    return x.view(torch.int64) ^ torch.iinfo(torch.int64).min


def _sorted_chunked(t) -> bool:
    prev = None
    for c0 in range(0, t.numel(), CHUNK):
        x = _as_signed_order(t[c0:c0 + CHUNK])
        if x.numel() > 1 and not bool((x[1:] >= x[:-1]).all()):
            return False
        if prev is not None and int(x[0]) < prev:
            return False
        prev = int(x[-1])
    return True


def _hash_chunked(t) -> int:
    return sum(multiset_hash(t[c0:c0 + CHUNK]) for c0 in range(0, t.numel(), CHUNK)) % (1 << 64)


def _need(nbytes):
    need_gpu()
    free = torch.cuda.mem_get_info()[0]
    if free < 3.5 * nbytes + (4 << 30):
        pytest.skip(f"needs about {3.5 * nbytes / 2**30:.0f} GiB of free device memory")


def test_u32_more_than_2_32_keys(ctx):
    from synth import torch_gen
    n = (1 << 32) + 12345
    _need(n * 4)
    d = torch_gen.uniform_u32(n, 9, device="cuda")
    h_in = _hash_chunked(d)
    out = torch.empty_like(d)
    ms.msort_sort_copy(ctx, d, out)
    ms.msort_ctx_sync(ctx)
    del d
    assert _sorted_chunked(out)
    assert _hash_chunked(out) == h_in


def test_u64_more_than_2_31_keys_in_place(ctx):
    from synth import torch_gen
    n = (1 << 31) + 77
    _need(n * 8)
    d = torch_gen.uniform_u64(n, 10, device="cuda")
    m = d[1::1000].numel()
    d[0:1000 * m:1000] = d[1::1000]  # some duplicate keys
    h_in = _hash_chunked(d)
    ms.msort_sort(ctx, d)
    ms.msort_ctx_sync(ctx)
    assert _sorted_chunked(d)
    assert _hash_chunked(d) == h_in
