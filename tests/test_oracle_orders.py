"""Pins for the oracle's signed and floating-point key orders (CPU only).

Signed keys must sort by value (checked against numpy's stable sort, a
library routine).  Floating-point keys sort by IEEE 754 totalOrder, pinned by
(a) numpy's stable sort on finite values with no negative zero (where
totalOrder and numeric order agree), and (b) a list of special bit patterns
written out in the order the standard fixes (clause 5.10: sign first, then
magnitude, reversed for negative patterns), shuffled and sorted back.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(2211)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_signed_matches_numpy(dtype):
    info = np.iinfo(dtype)
    n = 50000
    a = RNG.integers(info.min, info.max, size=n, dtype=dtype, endpoint=True)
    a[::97] = info.min
    a[1::89] = info.max
    a[2::83] = 0
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.sort(a, vals)
    order = np.argsort(a, kind="stable")
    assert np.array_equal(k, a[order])
    assert np.array_equal(v, vals[order])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_finite_floats_match_numpy(dtype):
    n = 50000
    a = (RNG.standard_normal(n) * 10.0 ** RNG.integers(-30, 30, size=n)).astype(dtype)
    a[::50] = a[7]  # duplicates keep their input order
    a[a == 0] = 1.0  # no zeros of either sign: numeric order = totalOrder here
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.sort(a, vals)
    order = np.argsort(a, kind="stable")
    assert np.array_equal(k.view(np.uint8), a[order].view(np.uint8))
    assert np.array_equal(v, vals[order])


def _f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def _f64(bits):
    return np.array(bits, dtype=np.uint64).view(np.float64)


# Special values in IEEE 754 totalOrder, written out from the standard's rules.
F32_ORDER = [0xFFFFFFFF,  # -NaN, largest payload
             0xFFC00001,  # -NaN
             0xFFC00000,  # -quiet NaN
             0xFF800001,  # -signalling NaN
             0xFF800000,  # -inf
             0xFF7FFFFF,  # -max
             0xBF800000,  # -1
             0x80800000,  # -smallest normal
             0x80000001,  # -smallest subnormal
             0x80000000,  # -0
             0x00000000,  # +0
             0x00000001,  # +smallest subnormal
             0x00800000,  # +smallest normal
             0x3F800000,  # +1
             0x7F7FFFFF,  # +max
             0x7F800000,  # +inf
             0x7F800001,  # +signalling NaN
             0x7FC00000,  # +quiet NaN
             0x7FFFFFFF]  # +NaN, largest payload
F64_ORDER = [0xFFFFFFFFFFFFFFFF, 0xFFF8000000000000, 0xFFF0000000000001, 0xFFF0000000000000,
             0xFFEFFFFFFFFFFFFF, 0xBFF0000000000000, 0x8000000000000001, 0x8000000000000000,
             0x0000000000000000, 0x0000000000000001, 0x3FF0000000000000, 0x7FEFFFFFFFFFFFFF,
             0x7FF0000000000000, 0x7FF0000000000001, 0x7FF8000000000000, 0x7FFFFFFFFFFFFFFF]


@pytest.mark.parametrize("order,make", [(F32_ORDER, _f32), (F64_ORDER, _f64)])
def test_float_total_order_specials(order, make):
    expected = make(order)
    for rep in range(20):
        perm = RNG.permutation(len(order))
        k, _ = oracle.sort(expected[perm])
        assert np.array_equal(k.view(np.uint8), expected.view(np.uint8)), rep
    # stability among equal bit patterns: duplicates keep input order
    a = np.concatenate([expected, expected, expected])[RNG.permutation(3 * len(order))]
    vals = np.arange(len(a), dtype=np.uint32)
    k, v = oracle.sort(a, vals)
    bits = a.view(np.uint32 if a.dtype == np.float32 else np.uint64)
    out_bits = k.view(bits.dtype)
    rank = {b: i for i, b in enumerate(np.asarray(order, dtype=bits.dtype))}
    assert [rank[b] for b in out_bits] == sorted(rank[b] for b in bits)
    for b in np.unique(bits):
        pos = v[out_bits == b]
        assert np.all(np.diff(pos.astype(np.int64)) > 0)


def test_signed_zero_order():
    a = np.array([0.0, -0.0, 1.0, -0.0, 0.0, -1.0], dtype=np.float32)
    k, v = oracle.sort(a, np.arange(6, dtype=np.uint32))
    assert list(v) == [5, 1, 3, 0, 4, 2]  # -1, -0 (input order), +0 (input order), 1


@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.float32, np.float64])
def test_parallel_oracle_agrees(dtype):
    # the chunked parallel oracle (chunks + pairwise merge tree) orders
    # signed and float keys exactly as the sequential one, values included
    size = np.dtype(dtype).itemsize
    bits = RNG.integers(0, 2 ** (8 * size), size=100_003, dtype=np.uint64 if size == 8 else np.uint32)
    keys = bits.view(dtype).copy()
    keys[::7] = keys[3]
    vals = np.arange(keys.size, dtype=np.uint32)
    a, av = oracle.sort(keys, vals)
    for workers in (1, 3, 8):
        b, bv = oracle.par_sort(keys, vals, workers=workers)
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)) and np.array_equal(av, bv), workers
