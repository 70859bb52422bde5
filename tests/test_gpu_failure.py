"""Failure detection on the device: a bounded wait that runs out.

The paper's only failure remark is that a blocking Send/Recv waits forever
when its peer has failed (Section "MPI Merge Sort").  Every device wait in
this library is bounded instead.  These tests make one wait run out on
purpose (a production merge block whose barrier expects one arrival more
than it gets, with a short cycle limit): nothing faults or hangs, the
context reports MSORT_ERR_TIMEOUT once, and sorts on it still work.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1000, 100000])
def test_expired_wait_reports_timeout_then_clears(limit):
    need_gpu()
    with ms.Context(0) as ctx:
        ms.msort_ctx_sync(ctx.handle)  # nothing pending
        ms.msort_selftest_wait_timeout(ctx.handle, limit)
        with pytest.raises(ms.MsortError) as e:
            ms.msort_ctx_sync(ctx.handle)
        assert e.value.status == ms.MSORT_ERR_TIMEOUT
        ms.msort_ctx_sync(ctx.handle)  # the status word was cleared
        # the context (and the device) still sort correctly
        keys = synth.uniform_u32(3 * 16896 + 5, 3)
        d = to_dev(keys)
        ms.msort_sort(ctx.handle, d)
        ms.msort_ctx_sync(ctx.handle)
        assert np.array_equal(to_host(d), oracle.sort(keys)[0])


def test_timeout_is_reported_after_later_work_on_the_stream():
    need_gpu()
    with ms.Context(0) as ctx:
        ms.msort_selftest_wait_timeout(ctx.handle, 20000)
        d = to_dev(synth.uniform_u32(1 << 16, 4))
        ms.msort_sort(ctx.handle, d)  # enqueued behind the expired wait
        with pytest.raises(ms.MsortError) as e:
            ms.msort_ctx_sync(ctx.handle)
        assert e.value.status == ms.MSORT_ERR_TIMEOUT
        ms.msort_ctx_sync(ctx.handle)


def test_selftest_rejects_limits_out_of_range():
    need_gpu()
    with ms.Context(0) as ctx:
        for bad in (0, 999, 2000000001):
            with pytest.raises(ms.MsortError) as e:
                ms.msort_selftest_wait_timeout(ctx.handle, bad)
            assert e.value.status == ms.MSORT_ERR_INVALID_ARG
        ms.msort_ctx_sync(ctx.handle)


@pytest.mark.parametrize("n", [2 * 4352, 3 * 4352 + 5, (1 << 20) + 3])
def test_grid_barrier_expiry_reports_timeout(n):
    """The single launch's grid barrier: the first barrier expects one block
    more than the grid has; every block gives up after the short limit."""
    need_gpu()
    with ms.Context(0) as ctx:
        d = to_dev(synth.uniform_u32(n, 6))
        ms.msort_selftest_grid_timeout(ctx.handle, d, 20000)
        with pytest.raises(ms.MsortError) as e:
            ms.msort_ctx_sync(ctx.handle)
        assert e.value.status == ms.MSORT_ERR_TIMEOUT
        ms.msort_ctx_sync(ctx.handle)
        keys = synth.uniform_u32(n, 7)
        d = to_dev(keys)
        ms.msort_sort(ctx.handle, d)  # the single launch itself still works
        ms.msort_ctx_sync(ctx.handle)
        assert np.array_equal(to_host(d), oracle.sort(keys)[0])


def test_grid_selftest_rejects_bad_arguments():
    need_gpu()
    with ms.Context(0) as ctx:
        d = to_dev(synth.uniform_u32(4352, 1))
        for n, limit in ((4352, 20000), (8704, 10), (8704, 2000000001)):
            with pytest.raises(ms.MsortError) as e:
                ms.msort_selftest_grid_timeout(ctx.handle, d, limit, n=n)
            assert e.value.status == ms.MSORT_ERR_INVALID_ARG
