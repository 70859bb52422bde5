"""GPU checks of the serving loop (continuous batching of sort requests).

Each request's result must be the same alone and in the mix: bit-exact
against the oracle's stable sort of that request's input, for a mix of key
types, value presence and sizes submitted at once (so they overlap on the
GPU) and from two host threads.  Admission must respect the memory budget
(arena high-water <= budget) while still running requests concurrently.
"""
import threading

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


def _request(i, rng):
    kind = i % 4
    n = int(rng.choice([0, 1, 17, 1000, 8448, 50000, 300001, 1 << 20]))
    if kind in (0, 1):
        keys = synth.uniform_u32(n, 100 + i) % np.uint32(1 + int(rng.integers(1, 10 ** 6)))
    else:
        keys, _ = synth.dup_u64(n, 100 + i, distinct=1 << 10)
    vals = np.arange(n, dtype=np.uint32) if kind in (1, 3) else None
    return keys, vals


def test_mixed_requests_exact_and_overlapping():
    need_gpu()
    rng = np.random.default_rng(0)
    reqs = [_request(i, rng) for i in range(48)]
    with ms.Server(0, mem_budget_bytes=96 << 20, max_slots=6) as srv:
        dev = []
        for keys, vals in reqs:
            dk = to_dev(keys)
            dv = to_dev(vals) if vals is not None else None
            dev.append((dk, dv, srv.submit(dk, dv)))
        for dk, dv, rid in dev:
            srv.wait(rid)
        st = srv.stats()
    for (keys, vals), (dk, dv, _) in zip(reqs, dev):
        ek, ev = oracle.sort(keys, vals)
        assert np.array_equal(to_host(dk), ek)
        if vals is not None:
            assert np.array_equal(to_host(dv), ev)
    assert st["completed"] == len(reqs)
    assert st["arena_high_water"] <= st["budget"]
    assert st["max_inflight"] >= 2, st       # requests overlapped on the GPU
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_budget_queues_instead_of_failing():
    need_gpu()
    n = 1 << 20
    need = ms.msort_scratch_bytes(n, ms.MSORT_U32, False)
    with ms.Server(0, mem_budget_bytes=2 * need + (1 << 20), max_slots=8) as srv:
        keys = [synth.uniform_u32(n, 200 + i) for i in range(10)]
        dev = [to_dev(k) for k in keys]
        ids = [srv.submit(d) for d in dev]
        for rid in ids:
            srv.wait(rid)
        st = srv.stats()
    assert st["arena_high_water"] <= st["budget"]
    assert st["max_inflight"] <= 2
    for k, d in zip(keys, dev):
        assert np.array_equal(to_host(d), oracle.sort(k)[0])


def test_oversize_request_rejected():
    need_gpu()
    with ms.Server(0, mem_budget_bytes=4 << 20, max_slots=2) as srv:
        d = torch.empty(1 << 22, dtype=torch.uint32, device="cuda")
        with pytest.raises(ms.MsortError) as e:
            srv.submit(d)
        assert e.value.status == ms.MSORT_ERR_OOM


def test_two_submitting_threads():
    need_gpu()
    rng = np.random.default_rng(1)
    reqs = [_request(i, rng) for i in range(32)]
    dev = [(to_dev(k), to_dev(v) if v is not None else None) for k, v in reqs]
    with ms.Server(0, mem_budget_bytes=256 << 20, max_slots=4) as srv:
        ids = [None] * len(reqs)

        def worker(parity):
            for i in range(parity, len(reqs), 2):
                ids[i] = srv.submit(dev[i][0], dev[i][1])

        ts = [threading.Thread(target=worker, args=(p,)) for p in (0, 1)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for rid in ids:
            srv.wait(rid)
    for (keys, vals), (dk, dv) in zip(reqs, dev):
        ek, ev = oracle.sort(keys, vals)
        assert np.array_equal(to_host(dk), ek)
        if vals is not None:
            assert np.array_equal(to_host(dv), ev)
