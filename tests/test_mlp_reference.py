"""The FP64 proposal-MLP reference: gradients pinned by central finite differences, Adam by a
hand-computed first step, and the loss by its closed form at zero weights."""
import math

import numpy as np
import pytest

from oracle import mlp


def _net(seed=0, d_in=11, hidden=7):
    rng = np.random.default_rng(seed)
    p = mlp.init(rng, d_in, hidden)
    p["b1"] = rng.normal(size=hidden) * 0.1
    p["b2"] = rng.normal(size=hidden) * 0.1
    p["b3"] = rng.normal(size=1) * 0.1
    x = rng.normal(size=(9, d_in))
    y = (rng.random(9) < 0.3).astype(np.float64)
    return p, x, y


@pytest.mark.parametrize("seed", range(4))
def test_backward_matches_finite_differences(seed):
    p, x, y = _net(seed)
    g = mlp.backward(p, x, y)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 15)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, x, y)
            flat[idx] = old - h
            lm = mlp.loss(p, x, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-6 + 1e-5 * abs(fd), (k, idx)


def test_loss_at_zero_logit_is_log2():
    """All-zero last layer: z3 = 0, so the cross-entropy is log 2 for every label."""
    p, x, y = _net(1)
    p["w3"][:] = 0.0
    p["b3"][:] = 0.0
    assert mlp.loss(p, x, y) == pytest.approx(math.log(2.0), abs=1e-15)
    assert np.allclose(mlp.score(p, x), 0.5)


def test_adam_first_step_moves_by_lr_times_sign():
    """After one bias-corrected Adam step every parameter moves by lr * g / (|g| + eps)."""
    p, x, y = _net(2)
    g = mlp.backward(p, x, y)
    before = {k: v.copy() for k, v in p.items()}
    mlp.adam(p, g, {}, lr=1e-3)
    for k in p:
        want = before[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], want, rtol=1e-9, atol=1e-15), k


def test_features_layout():
    rng = np.random.default_rng(0)
    mf, sf = rng.normal(size=(3, 4)), rng.normal(size=(5, 4))
    mxy, sxy = rng.uniform(0, 100, (3, 2)), rng.uniform(0, 100, (5, 2))
    mt, st = np.array([0, 1, 2]), np.array([3, 4, 5, 6, 7])
    x = mlp.features(mf, sf, mxy, sxy, mt, st, [1], [4], [2], 3)
    assert x.shape == (1, 11)
    assert np.allclose(x[0, :4], mf[1]) and np.allclose(x[0, 4:8], sf[4])
    assert np.allclose(x[0, 8:], [(sxy[4, 0] - mxy[1, 0]) / 100, (sxy[4, 1] - mxy[1, 1]) / 100, (7 - 3) / 3])
