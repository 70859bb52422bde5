"""Pins for the fp64 reference of the learned-CDF network.

The analytic gradient is checked against central finite differences of the
loss (independent of the backward formula), the forward pass against a closed
form, the Adam update against its first-step closed form, and the knot
initialisation against the points it must interpolate.
"""
import numpy as np

from oracle import mlp


def _random_params(rng):
    p = rng.normal(size=mlp.NPARAM)
    p[0:mlp.H] = rng.uniform(0.5, 2.0, size=mlp.H) * rng.choice([-1, 1], size=mlp.H)
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=257)
    t = np.sort(rng.uniform(0, 1, size=257))
    for trial in range(5):
        p = _random_params(rng)
        g, mag = mlp.grad(p, x, t)
        h = 1e-6
        fd = np.empty_like(g)
        for k in range(mlp.NPARAM):
            e = np.zeros(mlp.NPARAM)
            e[k] = h
            fd[k] = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * h)
        # a kink of a ReLU inside [p-h, p+h] would break the difference; skip those units
        pre = x[:, None] * p[0:mlp.H][None, :] + p[mlp.H:2 * mlp.H][None, :]
        near = (np.abs(pre) < 1e-5).any(0)
        mask = np.ones(mlp.NPARAM, bool)
        mask[0:mlp.H][near] = False
        mask[mlp.H:2 * mlp.H][near] = False
        assert np.allclose(g[mask], fd[mask], rtol=1e-5, atol=1e-8)
        assert np.all(mag >= np.abs(g) - 1e-15)


def test_forward_closed_form():
    # w1 = 1, b1 = -c_j, w2 = 1 on unit 0 only: y = relu(x - c_0) + b2
    p = np.zeros(mlp.NPARAM)
    p[0:mlp.H] = 1.0
    p[mlp.H:2 * mlp.H] = -0.25
    p[2 * mlp.H] = 1.0
    p[3 * mlp.H] = 0.125
    x = np.asarray([0.0, 0.25, 0.5, 1.0])
    y, _, _ = mlp.forward(p, x)
    assert np.allclose(y, [0.125, 0.125, 0.375, 0.875])
    assert mlp.loss(p, x, np.zeros(4)) == np.mean(np.asarray([0.125, 0.125, 0.375, 0.875]) ** 2)
    assert np.allclose(mlp.cdf(p, np.asarray([2.0])), [1.0])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(1)
    p = rng.normal(size=mlp.NPARAM)
    g = rng.normal(size=mlp.NPARAM)
    p1, m1, m2 = mlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr=0.01, eps=1e-8)
    # bias-corrected moments at step 1 are g and g^2
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_knot_init_interpolates_sample_cdf():
    rng = np.random.default_rng(2)
    xs = np.sort(rng.uniform(0, 1, size=4096))
    p = mlp.knot_init(xs)
    ranks = (np.arange(mlp.H) + 0.5) / mlp.H
    q = xs[np.minimum((ranks * len(xs)).astype(np.int64), len(xs) - 1)]
    y, _, _ = mlp.forward(p, q)
    assert np.allclose(y, ranks, atol=1e-12)
    # flat below the first knot and above the last
    y2, _, _ = mlp.forward(p, np.asarray([0.0, 1.0]))
    assert np.allclose(y2, [ranks[0], ranks[-1]])


def test_training_lowers_loss():
    rng = np.random.default_rng(3)
    xs = np.sort(rng.lognormal(0, 1, size=2048))
    xs = xs / xs.max()
    t = (np.arange(len(xs)) + 0.5) / len(xs)
    p = mlp.knot_init(xs)
    l0 = mlp.loss(p, xs, t)
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    for step in range(1, 101):
        g, _ = mlp.grad(p, xs, t)
        p, m1, m2 = mlp.adam_step(p, g, m1, m2, step, lr=1e-3)
    assert mlp.loss(p, xs, t) < l0


def _skewed_sample(m=4096):
    rng = np.random.default_rng(11)
    x = np.sort(np.concatenate([rng.lognormal(-9, 1.0, m // 2), rng.lognormal(-5, 0.5, m // 2)]))
    return np.clip(x, 0, 1), (np.arange(m) + 0.5) / m


def test_guarded_training_never_ends_worse():
    # plain Adam at lr 1e-3 diverges from the knot fit on skewed keys; the
    # safeguard must undo those steps and still end at or below the start
    x, t = _skewed_sample()
    p0 = mlp.knot_init(x)
    p, hist = mlp.train_guarded(p0, x, t, steps=60, lr=1e-3)
    assert mlp.loss(p, x, t) <= hist[0]
    assert any(b > a for a, b in zip(hist, hist[1:])), "expected at least one rejected step"


def test_guarded_training_is_adam_while_loss_falls():
    rng = np.random.default_rng(12)
    x = np.sort(rng.uniform(0, 1, 2048))
    t = (np.arange(len(x)) + 0.5) / len(x)
    p0 = mlp.knot_init(x)
    steps = 5
    p, hist = mlp.train_guarded(p0, x, t, steps=steps, lr=1e-5)
    assert all(b <= a for a, b in zip(hist, hist[1:])), "loss rose; choose a smaller rate for this pin"
    q, a, b = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for k in range(1, steps + 1):
        g, _ = mlp.grad(q, x, t)
        q, a, b = mlp.adam_step(q, g, a, b, k, lr=1e-5)
    assert np.allclose(p, q, rtol=0, atol=1e-15)
