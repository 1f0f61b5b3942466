"""Pins of the learned-preconditioner oracle (oracle/mlp.py).

* Its analytic gradient equals central finite differences of its own loss
  (a dropped term, a wrong sign or a transposed weight fails this).
* With all weights zero the network output vanishes: the correction is the
  diagonal Davidson correction r / (w - D) and the loss is the closed form
  sum (r/(w - D) - t)^2 / sum t^2.
"""
import numpy as np

from oracle import mlp


def _samples(n, rng):
    d = rng.uniform(-2, 2, n)
    d[np.abs(d) < 0.05] += 0.1
    blk = (rng.random(n) < 0.1).astype(np.uint8)
    r = rng.standard_normal(n) * 1e-2
    t = rng.standard_normal(n) * 1e-2
    return d, blk, r, t


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.standard_normal(mlp.NW) * 0.1
    d, blk, r, t = _samples(500, rng)
    _, g = mlp.loss_grad(w, d, blk, r, t)
    idx = rng.choice(mlp.NW, 60, replace=False)
    idx[0] = mlp.NW - 1  # b3
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_grad(wp, d, blk, r, t)[0] - mlp.loss_grad(wm, d, blk, r, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_zero_weights_is_the_diagonal_preconditioner():
    rng = np.random.default_rng(1)
    d, blk, r, t = _samples(300, rng)
    w = np.zeros(mlp.NW)
    loss, _ = mlp.loss_grad(w, d, blk, r, t)
    assert abs(loss - np.sum((r / (-d) - t) ** 2) / np.sum(t * t)) < 1e-12
    D = rng.uniform(0, 3, 50)
    R = rng.standard_normal(50)
    assert np.abs(mlp.precondition(w, R, 0.7, D, 5) - R / (0.7 - D)).max() < 1e-12
