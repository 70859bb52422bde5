"""fp64 reference of the learned-CDF network -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; the network is the partition predictor
the GPU library adds for its final merge passes.  Its shape is fixed as
Linear(1 -> 32) + ReLU + Linear(32 -> 1), output clamped to [0, 1] when used
as a CDF, trained by mean squared error against the empirical CDF of a sorted
key sample and updated with Adam (Kingma and Ba, 2015, Algorithm 1).

Parameter vector (97 values, this order): w1[32], b1[32], w2[32], b2.

Everything here is plain numpy in float64, written from the definitions:

  forward   h_j = max(0, w1_j x + b1_j),  y = sum_j w2_j h_j + b2
  loss      L = (1/m) sum_i (y_i - t_i)^2
  backward  dL/dy_i = 2 (y_i - t_i) / m
            dL/dw2_j = sum_i dL/dy_i h_ij,      dL/db2 = sum_i dL/dy_i
            dL/dw1_j = sum_i dL/dy_i w2_j [w1_j x_i + b1_j > 0] x_i
            dL/db1_j = sum_i dL/dy_i w2_j [w1_j x_i + b1_j > 0]
  Adam      m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
            p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

The ReLU derivative at exactly 0 is taken as 0.
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = 3 * H + 1


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return p[0:H], p[H:2 * H], p[2 * H:3 * H], p[3 * H]


def forward(p, x):
    w1, b1, w2, b2 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    pre = x[:, None] * w1[None, :] + b1[None, :]
    h = np.maximum(pre, 0.0)
    y = h @ w2 + b2
    return y, pre, h


def loss(p, x, t) -> float:
    y, _, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, x, t):
    """Analytic gradient (97,) and, per parameter, the sum of |terms| it adds."""
    w1, b1, w2, b2 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    m = len(x)
    y, pre, h = forward(p, x)
    dy = 2.0 * (y - t) / m
    act = (pre > 0.0).astype(np.float64)
    g = np.empty(NPARAM)
    mag = np.empty(NPARAM)
    dpre = dy[:, None] * w2[None, :] * act
    g[0:H] = (dpre * x[:, None]).sum(0)
    mag[0:H] = np.abs(dpre * x[:, None]).sum(0)
    g[H:2 * H] = dpre.sum(0)
    mag[H:2 * H] = np.abs(dpre).sum(0)
    g[2 * H:3 * H] = (dy[:, None] * h).sum(0)
    mag[2 * H:3 * H] = np.abs(dy[:, None] * h).sum(0)
    g[3 * H] = dy.sum()
    mag[3 * H] = np.abs(dy).sum()
    return g, mag


def adam_step(p, g, m1, m2, step: int, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2


def train_guarded(p0, x, t, steps: int, lr: float = 1e-3):
    """Safeguarded Adam, the training algorithm of the learned partitioner:
    before each update the loss of the current parameters is compared with
    the best so far; a higher loss restores the best parameters, halves the
    rate and restarts the Adam moments (step counter back to 0).  A final
    check keeps the best parameters.  Returns (parameters, loss history)."""
    p = np.asarray(p0, dtype=np.float64).copy()
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    best, saved, k, seen = None, p.copy(), 0, False
    hist = []
    for _ in range(steps + 1):
        cur = loss(p, x, t)
        hist.append(cur)
        final = len(hist) == steps + 1
        if not seen or cur <= best:
            best, saved, seen = cur, p.copy(), True
            if not final:
                g, _ = grad(p, x, t)
                k += 1
                p, m1, m2 = adam_step(p, g, m1, m2, k, lr=lr)
        else:
            p = saved.copy()
            m1[:] = 0.0
            m2[:] = 0.0
            k = 0
            lr *= 0.5
    return p, hist


def cdf(p, x):
    """The network read as a CDF: forward pass clamped to [0, 1]."""
    y, _, _ = forward(p, x)
    return np.clip(y, 0.0, 1.0)


def knot_init(sorted_x: np.ndarray) -> np.ndarray:
    """Start from the piecewise-linear interpolant of the sample's CDF.

    Knots q_j sit at the sample quantiles (j + 0.5) / H; unit j is
    relu(x - q_j), and the output weights are the slope changes between
    consecutive knots, so the initial network passes through the points
    (q_j, (j + 0.5) / H) and is flat below q_0.  This is a deterministic,
    data-dependent initialisation; training then lowers the MSE further.
    """
    xs = np.asarray(sorted_x, dtype=np.float64)
    m = len(xs)
    ranks = (np.arange(H) + 0.5) / H
    q = xs[np.minimum((ranks * m).astype(np.int64), m - 1)]
    w1 = np.ones(H)
    b1 = -q
    slopes = np.zeros(H)
    for j in range(H - 1):
        dx = q[j + 1] - q[j]
        slopes[j] = (ranks[j + 1] - ranks[j]) / dx if dx > 0 else 0.0
    slopes[H - 1] = 0.0
    w2 = np.diff(np.concatenate([[0.0], slopes]))
    b2 = ranks[0]
    return np.concatenate([w1, b1, w2, [b2]])
