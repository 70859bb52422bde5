"""The autotuner: it records a verified choice per class, the cache file
round-trips, and sorts after tuning stay bit-exact against the oracle."""
import json

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


def test_tune_quick_then_sort_exact(tmp_path):
    need_gpu()
    path = str(tmp_path / "tune.json")
    with ms.Context(0) as c:
        ms.msort_tune(c.handle, path, quick=True)
        data = json.load(open(path))
        assert {(e["key_bytes"], e["values"]) for e in data["plain"]} == {(4, 0), (4, 1), (8, 0), (8, 1)}
        for e in data["plain"]:
            assert e["tile"] in (4352, 8448, 8704, 16896)
            assert all(v > 0 for v in e["ms"].values()), e   # every candidate agreed bit for bit
            # merge fan-in: two-way and four-way passes compete for 32-bit keys without values
            four = (e["key_bytes"], e["values"]) == (4, 0)
            assert any(k.endswith("x4") for k in e["ms"]) == four, e
            assert e["ways"] in ((2, 4) if four else (2,)), e
        assert data["segmented_u32"]["max_small"] in (16896, 33792)
        for n in (5, 70001, (1 << 20) + 3):
            keys = synth.zipf_u32(n, 3)
            d = to_dev(keys)
            ms.msort_sort(c.handle, d)
            assert np.array_equal(to_host(d), oracle.sort(keys)[0])
        lens = synth.segment_lengths(500, 2)
        off = synth.segment_offsets(lens)
        keys = synth.uniform_u32(int(off[-1]), 4)
        d = to_dev(keys)
        ms.msort_segmented_sort(c.handle, d, to_dev(off))
        ms.msort_ctx_sync(c.handle)
        assert np.array_equal(to_host(d), oracle.segmented_sort(keys, off)[0])
    with ms.Context(0) as c2:
        ms.msort_tune_load(c2.handle, path)
        keys = synth.uniform_u32(123457, 5)
        d = to_dev(keys)
        ms.msort_sort(c2.handle, d)
        assert np.array_equal(to_host(d), oracle.sort(keys)[0])
        # a tuned four-way fan-in must not reach keys it does not take
        f = synth.uniform_u32(70001, 6).view(np.float32)
        df = to_dev(f)
        ms.msort_sort(c2.handle, df)
        assert np.array_equal(to_host(df).view(np.uint32), oracle.sort(f)[0].view(np.uint32))


def test_tuned_four_way_fan_in_is_exact(tmp_path):
    # a cache that selects four-way passes: later default sorts use them and
    # stay bit-exact; sorts that cannot take them keep pairwise passes
    need_gpu()
    path = tmp_path / "four.json"
    path.write_text('{\n  "plain": [\n'
                    '    {"key_bytes": 4, "values": 0, "log2n": 16, "tile": 16896, "ways": 4, "ms": {}}\n'
                    '  ]\n}\n')
    with ms.Context(0) as c:
        ms.msort_tune_load(c.handle, str(path))
        for n in (70001, (1 << 20) + 3):
            keys = synth.zipf_u32(n, 8)
            d = to_dev(keys)
            ms.msort_sort(c.handle, d)
            assert np.array_equal(to_host(d), oracle.sort(keys)[0])
        keys = synth.uniform_u32(90001, 9)
        vals = np.arange(keys.size, dtype=np.uint32)
        dk, dv = to_dev(keys), to_dev(vals)
        ms.msort_sort_pairs(c.handle, dk, dv)
        ek, ev = oracle.sort(keys, vals)
        assert np.array_equal(to_host(dk), ek) and np.array_equal(to_host(dv), ev)
        i = synth.uniform_u32(90001, 10).view(np.int32)
        di = to_dev(i)
        ms.msort_sort(c.handle, di)
        assert np.array_equal(to_host(di), oracle.sort(i)[0])
