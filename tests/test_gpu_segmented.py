"""GPU parity of the batched segmented sort against the CPU oracle.

Every segment must equal the oracle's stable sort of that segment alone
(bit-exact; values are original indices, so stability is checked exactly).
Lengths straddle every bucket boundary of the device plan, including empty
and one-element segments and segments longer than the largest on-chip tile.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu

BOUNDARY_LENS = [0, 1, 2, 3, 17, 33, 543, 544, 545, 1087, 1088, 1089, 2175, 2176, 2177, 4351, 4352, 4353, 8447, 8448,
                 8449, 16895, 16896, 16897,
                 33791, 33792, 33793, 65536, 100003,
                 # medium segments (two to four large tiles of T keys; a last tile of at most half a tile takes
                 # the half shape): T = 16896 for 32-bit keys, 8448 for 32-bit pairs and 64-bit keys, 4352
                 # for 64-bit pairs; around T + T/2, 2T, 3T, 3T + T/2 and 4T
                 25600, 25601, 50688, 50689, 59392, 59393, 67584, 67585,
                 21248, 21249, 25344, 25345, 29696, 29697,
                 11008, 11009, 13056, 13057, 15360, 15361, 17408, 17409,
                 # a medium segment's last tile takes the smallest of four shapes that holds it (about a
                 # quarter, half, three quarters or all of a tile): T + q and 3T + q, q at each shape's limit
                 # (q = 4608, 8704, 12800 of T = 16896; 2304, 4352, 6400 of 8448; 1280, 2304, 3328 of 4352)
                 21504, 21505, 55296, 55297, 63488, 63489,
                 10752, 10753, 27648, 27649, 14848, 14849, 31744, 31745,
                 5632, 5633, 14336, 14337, 6656, 6657, 15360, 7680, 7681, 16384, 16385,
                 # an on-chip segment of at most three quarters of its bucket's shape takes the
                 # three-quarter shape (32, 64, 128, 256 x 13 and 256, 512 x 25 keys)
                 416, 417, 832, 833, 1664, 1665, 3328, 3329, 6400, 6401, 12800, 12801]


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _keys(kt, n, seed, alphabet):
    if kt == "u32":
        return synth.uniform_u32(n, seed) % np.uint32(alphabet)
    k, _ = synth.dup_u64(n, seed, distinct=alphabet)
    return k


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("pairs", [False, True])
def test_bucket_boundaries(ctx, kt, pairs):
    rng = np.random.default_rng(1)
    lens = np.asarray(BOUNDARY_LENS + list(rng.permutation(BOUNDARY_LENS)), dtype=np.int64)
    off = synth.segment_offsets(lens)
    n = int(off[-1])
    keys = _keys(kt, n, 2, 1000)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    dk = to_dev(keys)
    dv = to_dev(vals) if pairs else None
    doff = to_dev(off)
    ms.msort_segmented_sort(ctx, dk, doff, vals=dv)
    ms.msort_ctx_sync(ctx)
    ek, ev = oracle.segmented_sort(keys, off, vals)
    assert np.array_equal(to_host(dk), ek)
    if pairs:
        assert np.array_equal(to_host(dv), ev)


@pytest.mark.parametrize("max_small,large_tile", [(33792, 16896), (16896, 8448), (33792, 8448)])
def test_tuned_bucket_plans(tmp_path, max_small, large_tile):
    # the bucket plans the tuner can choose besides the default (16896-key
    # on-chip bucket, 16896-key large-segment tile), on the boundary lengths
    need_gpu()
    path = tmp_path / "seg.json"
    path.write_text('{\n  "segmented_u32": {"max_small": %d, "large_tile": %d, "ms": {}}\n}\n'
                    % (max_small, large_tile))
    with ms.Context(0) as c:
        ms.msort_tune_load(c.handle, str(path))
        rng = np.random.default_rng(3)
        lens = np.asarray(BOUNDARY_LENS + list(rng.permutation(BOUNDARY_LENS)), dtype=np.int64)
        off = synth.segment_offsets(lens)
        keys = _keys("u32", int(off[-1]), 4, 1000)
        dk = to_dev(keys)
        ms.msort_segmented_sort(c.handle, dk, to_dev(off))
        ms.msort_ctx_sync(c.handle)
        assert np.array_equal(to_host(dk), oracle.segmented_sort(keys, off)[0])


@pytest.mark.parametrize("use_graph", [False, True])
def test_log_uniform_batch(ctx, use_graph):
    lens = synth.segment_lengths(3000, 5)
    off = synth.segment_offsets(lens)
    n = int(off[-1])
    keys = synth.uniform_u32(n, 6)
    doff = to_dev(off)
    exp, _ = oracle.segmented_sort(keys, off)
    dk = to_dev(keys)
    for rep in range(3):   # graph: capture on the first call, replay afterwards
        dk.copy_(to_dev(keys))
        ms.msort_segmented_sort(ctx, dk, doff, options={"use_graph": int(use_graph)})
        ms.msort_ctx_sync(ctx)
        assert np.array_equal(to_host(dk), exp), f"rep {rep}"


def test_malformed_offsets_rejected_on_device(ctx):
    lens = np.asarray([5, 7, 9], dtype=np.int64)
    off = synth.segment_offsets(lens)
    off[2] = off[1] - 1          # decreasing
    n = int(lens.sum())
    keys = synth.uniform_u32(n, 7)
    dk = to_dev(keys)
    ms.msort_segmented_sort(ctx, dk, to_dev(off))
    with pytest.raises(ms.MsortError) as e:
        ms.msort_ctx_sync(ctx)
    assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    assert np.array_equal(to_host(dk), keys)
    ms.msort_ctx_sync(ctx)       # the status word was cleared


def test_empty_batch(ctx):
    d = torch.empty(0, dtype=torch.uint32, device="cuda")
    ms.msort_segmented_sort(ctx, d, to_dev(np.zeros(1, dtype=np.uint64)), nseg=0)


def test_full_workload_50000_segments(ctx):
    """The batched workload itself: 50,000 segments, lengths log-uniform in
    [1, 65536] (about 3e8 keys), uniform uint32 keys, graph replay."""
    from synth import torch_gen
    lens = synth.segment_lengths(50000, 1)
    off = synth.segment_offsets(lens)
    n = int(off[-1])
    d = torch_gen.uniform_u32(n, 1, device="cuda")
    keys = to_host(d)
    ms.msort_segmented_sort(ctx, d, to_dev(off), options={"use_graph": 1})
    ms.msort_ctx_sync(ctx)
    exp, _ = oracle.segmented_sort(keys, off)
    assert np.array_equal(to_host(d), exp)


def test_graph_cache_evicts(ctx):
    # more distinct segmented launch sequences than a context keeps as graphs
    keys_buf = torch.empty(40000, dtype=torch.uint32, device="cuda")
    for rep in range(2):
        for i in range(70):
            lens = np.full(10 + i, 37 + i, dtype=np.int64)
            off = synth.segment_offsets(lens)
            n = int(off[-1])
            keys = synth.uniform_u32(n, 500 + 70 * rep + i)
            keys_buf[:n].copy_(torch.from_numpy(keys))
            ms.msort_segmented_sort(ctx, keys_buf[:n], to_dev(off), options={"use_graph": 1})
            ms.msort_ctx_sync(ctx)
            assert np.array_equal(to_host(keys_buf[:n]), oracle.segmented_sort(keys, off)[0]), (rep, i)
