"""GPU checks of the learned-CDF partitioner.

* Gradients of the library's fp32 backward kernel against the fp64 oracle
  (oracle/mlp.py), within a bound derived from fp32 rounding (see _tolerance).
* Training on the GPU lowers the loss and tracks the fp64 reference.
* Sorts with the learned partition (and the ratio-guess and counted-exact
  diagnostics modes) are bit-exact against the oracle sort, including with a
  zeroed and a random non-monotone installed model.
* The ablation: probes per co-rank search for exact binary search, ratio
  guess and the trained model, and what the model gains.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


def _tolerance(p, x, mag):
    """Per-parameter bound on |fp32 gradient - exact gradient|.

    Two sources: (1) each fp32 product and the summation of m terms in a
    fixed order (<= 1e-5 relative to the sum of |terms| for m <= 2^16, from
    the standard (m) * 2^-24 summation bound with a factor 10 margin); (2) the
    fp32 forward value y_r, whose absolute error is bounded by 33 * 2^-24 *
    (|b2| + sum_j |w2_j| (|w1_j x_r| + |b1_j|)), carried into every term
    through dL/dy_r = 2 (y_r - t_r) / m.
    """
    w1, b1, w2, b2 = mlp.unpack(p)
    x = np.asarray(x, dtype=np.float64)
    m = len(x)
    yb = 33 * 2.0 ** -24 * (abs(b2) + (np.abs(w2)[None, :] * (np.abs(w1)[None, :] * np.abs(x)[:, None]
                                                                + np.abs(b1)[None, :])).sum(1))
    ddy = 2.0 * yb / m
    pre = x[:, None] * w1[None, :] + b1[None, :]
    act = (pre > 0).astype(np.float64)
    h = np.maximum(pre, 0.0)
    H = mlp.H
    t2 = np.empty(mlp.NPARAM)
    t2[0:H] = (ddy[:, None] * np.abs(w2)[None, :] * act * np.abs(x)[:, None]).sum(0)
    t2[H:2 * H] = (ddy[:, None] * np.abs(w2)[None, :] * act).sum(0)
    t2[2 * H:3 * H] = (ddy[:, None] * h).sum(0)
    t2[3 * H] = ddy.sum()
    return 1e-5 * mag + t2 + 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_fp64_oracle(ctx, seed):
    rng = np.random.default_rng(seed)
    m = 65536
    if seed == 0:
        x = np.sort(rng.uniform(0, 1, m)).astype(np.float32)
    else:
        x = np.sort(rng.lognormal(0, 1 + seed, m) / 50.0).astype(np.float32)
    p = rng.normal(size=mlp.NPARAM).astype(np.float32)
    p[0:mlp.H] = rng.uniform(0.5, 2, mlp.H) * rng.choice([-1, 1], mlp.H)
    # keep every ReLU kink away from the samples so fp32 and fp64 agree on
    # which units are active
    pre = x[:, None].astype(np.float64) * p[None, 0:mlp.H] + p[None, mlp.H:2 * mlp.H]
    near = (np.abs(pre) < 1e-4).any(0)
    p[mlp.H:2 * mlp.H][near] += 1e-2
    dx, dp = to_dev(x), to_dev(p)
    dg = torch.empty(mlp.NPARAM, dtype=torch.float32, device="cuda")
    ms.msort_mlp_grad(ctx, dx, dp, dg)
    g_gpu = to_host(dg).astype(np.float64)
    t = (np.arange(m) + 0.5) / m
    g_ref, mag = mlp.grad(p.astype(np.float64), x.astype(np.float64), t)
    tol = _tolerance(p.astype(np.float64), x, mag)
    bad = np.abs(g_gpu - g_ref) > tol
    assert not bad.any(), list(zip(np.nonzero(bad)[0], g_gpu[bad], g_ref[bad], tol[bad]))


@pytest.mark.parametrize("m", [1, 7, 1001, 16383, 65535])
def test_gradient_uneven_point_counts(ctx, m):
    """The training rounds split the points among their blocks by
    floor(b m / B); counts that do not divide evenly (and fewer points than
    blocks) still give the fp64 gradient."""
    rng = np.random.default_rng(m)
    x = np.sort(rng.uniform(0, 1, m)).astype(np.float32)
    p = rng.normal(size=mlp.NPARAM).astype(np.float32)
    p[0:mlp.H] = rng.uniform(0.5, 2, mlp.H) * rng.choice([-1, 1], mlp.H)
    pre = x[:, None].astype(np.float64) * p[None, 0:mlp.H] + p[None, mlp.H:2 * mlp.H]
    p[mlp.H:2 * mlp.H][(np.abs(pre) < 1e-4).any(0)] += 1e-2
    dg = torch.empty(mlp.NPARAM, dtype=torch.float32, device="cuda")
    ms.msort_mlp_grad(ctx, to_dev(x), to_dev(p), dg)
    g_gpu = to_host(dg).astype(np.float64)
    t = (np.arange(m) + 0.5) / m
    g_ref, mag = mlp.grad(p.astype(np.float64), x.astype(np.float64), t)
    tol = _tolerance(p.astype(np.float64), x, mag)
    bad = np.abs(g_gpu - g_ref) > tol
    assert not bad.any(), list(zip(np.nonzero(bad)[0], g_gpu[bad], g_ref[bad], tol[bad]))


def test_training_lowers_loss_and_tracks_fp64(ctx):
    rng = np.random.default_rng(4)
    m = 1 << 14
    x = np.sort(synth.lognormal3_u32(m, 2).astype(np.float64) / 2 ** 32).astype(np.float32)
    t = (np.arange(m) + 0.5) / m
    dx = to_dev(x)
    dp = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    ms.msort_mlp_train(ctx, dx, dp, steps=0, knot_init=True)
    p0 = to_host(dp).astype(np.float64)
    ref0 = mlp.knot_init(x.astype(np.float64))
    assert np.allclose(p0, ref0, rtol=1e-4, atol=1e-4 * np.abs(ref0).max())
    ms.msort_mlp_train(ctx, dx, dp, steps=100, lr=1e-3)
    p1 = to_host(dp).astype(np.float64)
    x64 = x.astype(np.float64)
    l0, l1 = mlp.loss(p0, x64, t), mlp.loss(p1, x64, t)
    # the same safeguarded algorithm in fp64 from the same start
    pr, _ = mlp.train_guarded(p0, x64, t, steps=100, lr=1e-3)
    lr_ = mlp.loss(pr, x64, t)
    assert l1 <= l0 * (1 + 1e-4), (l0, l1)
    assert l1 <= 1.25 * lr_ + 1e-8, (l1, lr_)


def test_training_is_reproducible(ctx):
    """Each training round adds its blocks' partial sums in block order, so
    training twice on the same points gives bit-identical parameters, and
    two learned sorts of the same keys train the same model."""
    m = 1 << 14
    x = np.sort(synth.lognormal3_u32(m, 6).astype(np.float64) / 2 ** 32).astype(np.float32)
    dx = to_dev(x)
    runs = []
    for _ in range(2):
        dp = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
        ms.msort_mlp_train(ctx, dx, dp, steps=32, lr=1e-3, knot_init=True)
        runs.append(to_host(dp).view(np.uint32))
    assert np.array_equal(runs[0], runs[1])
    keys = synth.lognormal3_u32((1 << 22) + 9, 7)
    models = []
    for _ in range(2):
        d = to_dev(keys)
        ms.msort_sort(ctx, d, options={"partition_mode": 1})
        models.append(np.asarray(ms.msort_learned_model(ctx)[0], dtype=np.float32).view(np.uint32))
    assert np.array_equal(models[0], models[1])


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("dist", ["lognormal3", "uniform", "sorted", "zipf"])
def test_guided_sorts_are_exact(ctx, mode, dist):
    n = (1 << 22) + 333
    keys = synth.u32_distribution(dist, n, 8)
    d = to_dev(keys)
    ms.msort_sort(ctx, d, options={"partition_mode": mode, "learned_passes": 64})
    exp, _ = oracle.sort(keys)
    assert np.array_equal(to_host(d), exp)


@pytest.mark.parametrize("opts", [{"partition_mode": 1}, {"partition_mode": 1, "learned_passes": 64}],
                         ids=["final_passes", "all_passes"])
def test_full_size_learned_2_30(ctx, opts):
    """2^30 keys of the lognormal mixture with the learned partition, as the
    learned-partition benchmark launches it; bit-exact against the oracle
    on every host core."""
    import os
    from synth import torch_gen
    n = 1 << 30
    src = torch_gen.lognormal3_u32(n, 1, device="cuda")
    out = torch.empty_like(src)
    ms.msort_sort_copy(ctx, src, out, options=opts)
    exp, _ = oracle.par_sort(to_host(src), workers=len(os.sched_getaffinity(0)))
    assert np.array_equal(to_host(out), exp)
    del src, out
    torch.cuda.empty_cache()


def test_guided_pairs_u64_exact(ctx):
    n = (1 << 21) + 17
    keys, vals = synth.dup_u64(n, 9)
    dk, dv = to_dev(keys), to_dev(vals)
    ms.msort_sort_pairs(ctx, dk, dv, options={"partition_mode": 1, "learned_passes": 64})
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(dk), ek) and np.array_equal(to_host(dv), ev)


@pytest.mark.parametrize("model", ["zero", "random"])
def test_adversarial_models_keep_output_exact(ctx, model):
    rng = np.random.default_rng(5)
    params = np.zeros(mlp.NPARAM) if model == "zero" else rng.normal(size=mlp.NPARAM) * 5
    ms.msort_learned_set_model(ctx, params, 0.0)
    try:
        n = (1 << 21) + 5
        keys = synth.lognormal3_u32(n, 3)
        d = to_dev(keys)
        ms.msort_sort(ctx, d, options={"partition_mode": 1, "learned_passes": 64})
        exp, _ = oracle.sort(keys)
        assert np.array_equal(to_host(d), exp)
    finally:
        ms.msort_learned_set_model(ctx, None)


def _probes(ctx, d, out, mode):
    ms.msort_ctx_set_profiling(ctx, 2)  # level 2: guided partitions count their probes
    ms.msort_sort_copy(ctx, d, out, options={"partition_mode": mode, "learned_passes": 64})
    torch.cuda.synchronize()
    probes, searches = ms.msort_ctx_partition_stats(ctx)
    ms.msort_ctx_set_profiling(ctx, False)
    return probes / max(1, searches)


def test_ablation_model_cuts_probes(ctx):
    """What the trained network gains: probes per co-rank search on 2^24
    keys of the skewed lognormal mixture and of pre-sorted keys."""
    from synth import torch_gen
    n = 1 << 24
    report = {}
    for dist in ("lognormal3", "sorted"):
        d = torch_gen.u32_distribution(dist, n, 1, device="cuda")
        out = torch.empty_like(d)
        exact = _probes(ctx, d, out, 3)
        ratio = _probes(ctx, d, out, 2)
        learned = _probes(ctx, d, out, 1)
        report[dist] = (exact, ratio, learned)
    print("probes per search (exact, ratio, learned):", report)
    for dist, (exact, ratio, learned) in report.items():
        assert learned < exact, report
        # the secant steps in the model's CDF space beat the model-free
        # length-ratio start on the skewed mixture too
        assert learned < ratio, report
    # on pre-sorted runs the positional ratio guess is far off; the CDF is not
    assert report["sorted"][2] < report["sorted"][1], report


def _expected_splits(runs, L, W):
    n = len(runs)
    out = []
    for c in range((n + W - 1) // W):
        out0 = c * W
        pb = (out0 // (2 * L)) * 2 * L
        alen = min(L, n - pb)
        blen = min(L, n - pb - alen)
        out.append(oracle.corank(runs[pb:pb + alen], runs[pb + alen:pb + alen + blen], out0 - pb))
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_every_partition_is_the_exact_corank(ctx, dtype):
    """Each mode's split table for one merge pass (exact binary search, the
    learned network's guided search, the ratio guess, the counted exact
    search) against the oracle's co-rank of every output block, on runs of
    two lengths with a ragged last run; then with a zeroed and a random
    installed model."""
    n = 300007
    if dtype == np.uint32:
        keys = synth.lognormal3_u32(n, 21)
    else:
        keys, _ = synth.dup_u64(n, 21, distinct=1 << 10)
    d = to_dev(keys)
    out = torch.empty_like(d)
    ms.msort_sort_copy(ctx, d, out, options={"partition_mode": 1, "learned_passes": 64})  # trains a model
    ms.msort_ctx_sync(ctx)
    W = 8448
    rng = np.random.default_rng(3)
    models = [None, np.zeros(mlp.NPARAM), rng.normal(size=mlp.NPARAM) * 5]
    try:
        for L in (16896, 4 * 16896):
            runs = np.concatenate([oracle.sort(keys[i:i + L])[0] for i in range(0, n, L)])
            exp = _expected_splits(runs, L, W)
            druns = to_dev(runs)
            for model in models:
                if model is not None:
                    ms.msort_learned_set_model(ctx, model, 0.0)
                for mode in (0, 1, 2, 3):
                    splits = torch.full((len(exp),), -1, dtype=torch.int64, device="cuda")
                    ms.msort_partition_splits(ctx, druns, L, W, mode, splits)
                    ms.msort_ctx_sync(ctx)
                    assert np.array_equal(to_host(splits).astype(np.uint64), exp), (L, mode, model is None)
    finally:
        ms.msort_learned_set_model(ctx, None)


def test_partition_splits_argument_checks(ctx):
    d = torch.zeros(1000, dtype=torch.uint32, device="cuda")
    s = torch.zeros(10, dtype=torch.int64, device="cuda")
    for L, W, mode in ((100, 300, 0), (100, 200, 4), (0, 100, 0)):
        with pytest.raises(ms.MsortError) as e:
            ms.msort_partition_splits(ctx, d, L, W, mode, s)
        assert e.value.status == ms.MSORT_ERR_INVALID_ARG
