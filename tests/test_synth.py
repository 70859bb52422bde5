"""The torch generators reproduce the numpy generators bit for bit (integer
recipes), and the recipes have the stated shapes.  CPU only."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from synth import torch_gen  # noqa: E402


@pytest.mark.parametrize("name", ["uniform", "sorted", "reverse", "distinct16", "zipf"])
def test_torch_matches_numpy(name):
    for n in (0, 1, 1000, 70001):
        a = synth.u32_distribution(name, n, 3)
        b = torch_gen.u32_distribution(name, n, 3, device="cpu").numpy()
        assert np.array_equal(a, b), name


def test_torch_u64_matches_numpy():
    n = 50001
    assert np.array_equal(synth.uniform_u64(n, 2), torch_gen.uniform_u64(n, 2, device="cpu").numpy())
    k1, v1 = synth.dup_u64(n, 2)
    k2, v2 = torch_gen.dup_u64(n, 2, device="cpu")
    assert np.array_equal(k1, k2.numpy()) and np.array_equal(v1, v2.numpy())


def test_lognormal_close_to_numpy():
    a = synth.lognormal3_u32(20000, 1).astype(np.int64)
    b = torch_gen.lognormal3_u32(20000, 1, device="cpu").numpy().astype(np.int64)
    assert np.mean(a == b) > 0.999


def test_recipe_shapes():
    s = synth.sorted_u32(100000, 1)
    assert np.all(s[:-1] <= s[1:])
    assert len(np.unique(synth.distinct16_u32(100000, 1))) == 16
    L = synth.segment_lengths(50000, 1)
    assert L.min() >= 1 and L.max() <= 65536
    assert 2.5e8 < L.sum() < 3.5e8
    k, v = synth.dup_u64(1 << 16, 1)
    assert len(np.unique(k)) <= 1 << 20 and np.array_equal(v, np.arange(1 << 16))
    t, sz = synth.poisson_requests(1000, 1, rate_per_s=100.0)
    assert np.all(np.diff(t) > 0) and sz.min() >= 1 << 10 and sz.max() <= 1 << 24
