"""GPU parity of the out-of-core host sort against the CPU oracle.

A context whose device budget is smaller than the in-core host sort of n
elements sorts host arrays in budget-sized chunks (sorted runs in a
pinned host buffer) and merges the runs in blocks bounded by sampled
(key, position) splitters, merging each block's slices on the device.
Checked: a couple and many runs, ragged runs, all-equal keys (runs of equal
keys are split by position), 64-bit pairs (stability through the values),
floating-point keys (kept transformed between the phases), presorted input
(blocks of one slice) and more runs than one run-merge launch takes.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


def _ctx(budget_mb):
    need_gpu()
    return ms.Context(0, scratch_budget_bytes=budget_mb << 20)


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _bits(a):
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


@pytest.mark.parametrize("n,budget_mb", [(3_000_017, 24), (12_500_003, 16)])
def test_u32_keys(n, budget_mb):
    c = _ctx(budget_mb)
    try:
        keys = synth.zipf_u32(n, 4)
        exp, _ = oracle.sort(keys)
        hin, hout = _pinned(keys), _pinned(np.zeros_like(keys))
        ms.msort_sort_host(c.handle, hin, out_keys=hout)
        assert np.array_equal(hout.numpy(), exp)
        assert np.array_equal(hin.numpy(), keys)
    finally:
        c.close()


def test_equal_keys_and_in_place():
    c = _ctx(16)
    try:
        n = 6_000_001
        keys = np.full(n, 42, dtype=np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        hk, hv = _pinned(keys), _pinned(vals)
        ms.msort_sort_host(c.handle, hk, hv)  # in place
        assert np.array_equal(hk.numpy(), keys) and np.array_equal(hv.numpy(), vals)
    finally:
        c.close()


def test_u64_pairs():
    c = _ctx(32)
    try:
        n = 5_000_011
        keys, _ = synth.dup_u64(n, 9, distinct=1 << 12)
        vals = np.arange(n, dtype=np.uint32)
        ek, ev = oracle.sort(keys, vals)
        hk, hv = _pinned(keys), _pinned(vals)
        ok, ov = _pinned(np.zeros_like(keys)), _pinned(np.zeros_like(vals))
        ms.msort_sort_host(c.handle, hk, hv, out_keys=ok, out_vals=ov)
        assert np.array_equal(ok.numpy(), ek) and np.array_equal(ov.numpy(), ev)
    finally:
        c.close()


def test_float_keys_and_async_call():
    c = _ctx(16)
    try:
        n = 4_000_003
        rng = np.random.default_rng(5)
        keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint32).view(np.float32)
        exp, _ = oracle.sort(keys)
        hin, hout = _pinned(keys), _pinned(np.zeros_like(keys))
        ms.msort_sort_host_async(c.handle, hin, out_keys=hout)
        ms.msort_ctx_sync(c.handle)
        assert np.array_equal(_bits(hout.numpy()), _bits(exp))
    finally:
        c.close()


def test_many_runs():
    # a 3 MiB budget gives chunks of about 2^16.4 keys, so 8e6 keys make about
    # 90 runs: more pairs per merge round than one run-merge launch takes
    need_gpu()
    c = ms.Context(0, scratch_budget_bytes=3 << 20)
    try:
        n = 8_000_009
        keys = synth.uniform_u32(n, 11)
        keys[::7] = keys[3]
        exp, _ = oracle.sort(keys)
        hin, hout = _pinned(keys), _pinned(np.zeros_like(keys))
        ms.msort_sort_host(c.handle, hin, out_keys=hout)
        assert np.array_equal(hout.numpy(), exp)
    finally:
        c.close()


@pytest.mark.parametrize("order", ["ascending", "descending"])
def test_presorted_float_pairs(order):
    # ascending input puts one slice in most blocks (only the copy round,
    # which undoes the key transform, runs); descending input spreads every
    # block over all runs
    c = _ctx(16)
    try:
        n = 3_500_017
        rng = np.random.default_rng(8)
        keys = np.sort(rng.standard_normal(n).astype(np.float32))
        keys[keys == 0] = 1.0
        keys[::11] = keys[5]  # duplicates: stability through the values
        keys = np.sort(keys)
        if order == "descending":
            keys = keys[::-1].copy()
        vals = np.arange(n, dtype=np.uint32)
        ek, ev = oracle.sort(keys, vals)
        hk, hv = _pinned(keys), _pinned(vals)
        ok, ov = _pinned(np.zeros_like(keys)), _pinned(np.zeros_like(vals))
        ms.msort_sort_host(c.handle, hk, hv, out_keys=ok, out_vals=ov)
        assert np.array_equal(_bits(ok.numpy()), _bits(ek)) and np.array_equal(ov.numpy(), ev)
    finally:
        c.close()


def test_full_size_2_30():
    """The out-of-core benchmark's configuration: 2^30 uniform uint32 keys in
    pinned host memory, 1 GiB device budget; bit-exact against the oracle's
    parallel sort on every host core."""
    import os
    from synth import torch_gen
    c = _ctx(1024)
    try:
        n = 1 << 30
        hin = torch_gen.uniform_u32(n, 1, device="cuda").cpu().pin_memory()
        hout = torch.empty(n, dtype=torch.uint32).pin_memory()
        ms.msort_sort_host(c.handle, hin, out_keys=hout)
        exp, _ = oracle.par_sort(hin.numpy(), workers=len(os.sched_getaffinity(0)))
        assert np.array_equal(hout.numpy(), exp)
    finally:
        c.close()


def test_budget_too_small():
    c = _ctx(1)
    try:
        keys = _pinned(synth.uniform_u32(1_000_000, 3))
        with pytest.raises(ms.MsortError) as e:
            ms.msort_sort_host(c.handle, keys)
        assert e.value.status == ms.MSORT_ERR_OOM
    finally:
        c.close()
