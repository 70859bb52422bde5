"""GPU parity of signed and floating-point keys against the CPU oracle.

Keys are random bit patterns, so float inputs include NaNs of both signs,
infinities, subnormals and both zeros, each of which has one place in IEEE
754 totalOrder; integer inputs include both extremes.  The segmented sort is
checked over every length bucket.  Sizes cover a single
tile (no merge round: the tile sort applies and undoes the key transform),
several tiles with a ragged tail, and many merge rounds.  Results are
compared as bit patterns; values are original indices, so stability is
checked exactly.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu

TYPES = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}
SIZES = [1, 5000, 16897, 3 * 16896 + 7, (1 << 20) + 3]


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _keys(name, n, seed):
    dt = np.dtype(TYPES[name])
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** (8 * dt.itemsize), size=n, dtype=np.uint64 if dt.itemsize == 8 else np.uint32,
                        endpoint=False)
    k = bits.view(dt).copy()
    if n > 100:
        k[::37] = k[5]  # duplicates: stability is visible through the values
        if name.startswith("i"):
            info = np.iinfo(dt)
            k[1::41], k[2::43] = info.min, info.max
        else:
            k[1::41], k[2::43], k[3::47] = -0.0, 0.0, np.inf
    return k


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", list(TYPES))
@pytest.mark.parametrize("n", SIZES)
def test_keys_and_pairs(ctx, name, n):
    keys = _keys(name, n, n)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.sort(keys, vals)
    d = _dev(keys)
    ms.msort_sort(ctx, d)
    assert np.array_equal(_bits(d.cpu().numpy()), _bits(ek))
    dk, dv = _dev(keys), _dev(vals)
    ms.msort_sort_pairs(ctx, dk, dv)
    assert np.array_equal(_bits(dk.cpu().numpy()), _bits(ek))
    assert np.array_equal(dv.cpu().numpy(), ev)


@pytest.mark.parametrize("name", list(TYPES))
def test_copy_graph_and_host(ctx, name):
    n = (1 << 21) + 11
    keys = _keys(name, n, 77)
    ek, _ = oracle.sort(keys)
    src = _dev(keys)
    out = torch.empty_like(src)
    for rep in range(2):  # capture, then replay
        ms.msort_sort_copy(ctx, src, out, options={"use_graph": 1})
        assert np.array_equal(_bits(out.cpu().numpy()), _bits(ek)), rep
    assert np.array_equal(_bits(src.cpu().numpy()), _bits(keys))
    hin = torch.from_numpy(keys.copy()).pin_memory()
    hout = torch.from_numpy(np.zeros_like(keys)).pin_memory()
    ms.msort_sort_host(ctx, hin, out_keys=hout)
    assert np.array_equal(_bits(hout.numpy()), _bits(ek))
    hout2 = torch.from_numpy(np.zeros_like(keys)).pin_memory()
    ms.msort_sort_host_async(ctx, hin, out_keys=hout2)
    ms.msort_ctx_sync(ctx)
    assert np.array_equal(_bits(hout2.numpy()), _bits(ek))


@pytest.mark.parametrize("name", list(TYPES))
@pytest.mark.parametrize("pairs", [False, True])
def test_segmented(ctx, name, pairs):
    # every bucket: tiny, small-block, one-tile and multi-tile segments
    lens = np.array([0, 1, 2, 31, 500, 544, 2000, 8448, 9000, 16896, 20000, 33792, 40000, 65536, 7], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    n = int(off[-1])
    keys = _keys(name, n, 3 + pairs)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.segmented_sort(keys, off, vals if pairs else None)
    dk = _dev(keys)
    dv = _dev(vals) if pairs else None
    ms.msort_segmented_sort(ctx, dk, _dev(off), vals=dv)
    ms.msort_ctx_sync(ctx)
    assert np.array_equal(_bits(dk.cpu().numpy()), _bits(ek))
    if pairs:
        assert np.array_equal(dv.cpu().numpy(), ev)


def test_other_entry_points_refuse(ctx):
    k = _dev(np.arange(1000, dtype=np.float32))
    with pytest.raises(ms.MsortError) as e:
        ms.msort_merge(ctx, k[:500], k[500:], torch.empty_like(k))
    assert e.value.status == ms.MSORT_ERR_UNSUPPORTED
    for opts in ({"partition_mode": 1}, {"merge_ways": 4}):
        with pytest.raises(ms.MsortError):
            ms.msort_sort(ctx, k, options=opts)
    ms.msort_ctx_sync(ctx)
