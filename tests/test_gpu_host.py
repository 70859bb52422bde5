"""GPU parity of the host-buffer sorts (msort_sort_host, msort_sort_host_async)
against the CPU oracle, element by element.

The pipelined schedule changes only where copies go (chunked host-to-device
copies with chunk-local rounds, the last round in slices each followed by its
device-to-host copy), so every size class of that schedule is checked: no
merge round at all, one chunk, and eight chunks with a ragged last chunk;
keys alone and key-value pairs, 32- and 64-bit keys, pinned and pageable host
memory, in place and out of place.  Back-to-back asynchronous calls check the
rotation of the three staging slots (a fourth call reuses the first slot).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _pinned(a: np.ndarray):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t


# 5000 < one tile (no merge round); 200003: one chunk; 2^22 + 777: eight chunks
SIZES = [1, 5000, 200003, (1 << 22) + 777]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_host_keys(ctx, n, kt):
    keys = synth.zipf_u32(n, 3) if kt == "u32" else synth.dup_u64(n, 3, distinct=4099)[0]
    exp, _ = oracle.sort(keys)
    hin = _pinned(keys)
    hout = _pinned(np.zeros_like(keys))
    ms.msort_sort_host(ctx, hin, out_keys=hout)
    assert np.array_equal(hout.numpy(), exp)
    assert np.array_equal(hin.numpy(), keys)  # out of place: input untouched


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_host_pairs_in_place(ctx, n, kt):
    keys = (synth.uniform_u32(n, 4) % np.uint32(1000)) if kt == "u32" else synth.dup_u64(n, 4, distinct=1000)[0]
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.sort(keys, vals)
    hk, hv = _pinned(keys), _pinned(vals)
    ms.msort_sort_host(ctx, hk, hv)
    assert np.array_equal(hk.numpy(), ek)
    assert np.array_equal(hv.numpy(), ev)


def test_host_pageable(ctx):
    n = (1 << 21) + 99
    keys = synth.reverse_u32(n, 5)
    out = np.empty_like(keys)
    ms.msort_sort_host(ctx, keys, out_keys=out)
    exp, _ = oracle.sort(keys)
    assert np.array_equal(out, exp)


@pytest.mark.parametrize("opts", [{"partition_mode": 1}, {"merge_ways": 4}, {"tile": 4352}])
def test_host_other_plans(ctx, opts):
    n = (1 << 21) + 5
    keys = synth.lognormal3_u32(n, 6)
    exp, _ = oracle.sort(keys)
    hin, hout = _pinned(keys), _pinned(np.zeros_like(keys))
    ms.msort_sort_host(ctx, hin, out_keys=hout, options=opts)
    assert np.array_equal(hout.numpy(), exp)


def test_host_async_back_to_back(ctx):
    # five calls in flight on one stream: slots 0, 1, 2, 0, 1
    n = (1 << 22) + 4097
    names = list(synth.DIST_NAMES)
    ins = [synth.u32_distribution(name, n, 40 + i) for i, name in enumerate(names)]
    hins = [_pinned(k) for k in ins]
    houts = [_pinned(np.zeros_like(k)) for k in ins]
    stream = torch.cuda.current_stream()
    for hi, ho in zip(hins, houts):
        ms.msort_sort_host_async(ctx, hi, out_keys=ho, stream=stream)
    ms.msort_ctx_sync(ctx, stream)
    for k, ho, name in zip(ins, houts, names):
        exp, _ = oracle.sort(k)
        assert np.array_equal(ho.numpy(), exp), name


def test_host_async_then_device_work(ctx):
    # work enqueued on the stream after an asynchronous host sort runs after
    # its device-to-host copy: the stream orders both
    n = 300001
    keys = synth.uniform_u32(n, 8)
    hin, hout = _pinned(keys), _pinned(np.zeros_like(keys))
    stream = torch.cuda.current_stream()
    ms.msort_sort_host_async(ctx, hin, out_keys=hout, stream=stream)
    d = torch.from_numpy(keys.copy()).cuda()
    ms.msort_sort(ctx, d, stream=stream)
    stream.synchronize()
    exp, _ = oracle.sort(keys)
    assert np.array_equal(hout.numpy(), exp)
    assert np.array_equal(d.cpu().numpy(), exp)
