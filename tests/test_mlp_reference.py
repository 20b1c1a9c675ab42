"""The FP64 proposal-MLP reference: gradients pinned by central finite differences, Adam by a
hand-computed first step, and the loss by its closed form at zero weights. The BF16-operand variant is
pinned by its rounding function (hand-worked values, ties to even, and torch's own BF16 conversion) and by
reducing to the finite-difference-pinned FP64 backward when every operand is exactly representable in
BF16, so a dropped term, sign or transposed operand in it fails."""
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


def test_bf16_rounding_hand_values():
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                    # halfway between 1 and 1 + 2^-7: ties to even
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # halfway between 1+2^-7 and 1+2^-6: to even
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7   # above halfway: up
    assert mlp.bf16(-3.0 - 2.0 ** -7) == -3.0                   # 8 significant bits: spacing 2^-6 in [2, 4)
    assert mlp.bf16(0.0) == 0.0 and mlp.bf16(-0.0) == 0.0


def test_bf16_rounding_equals_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.float32(1.0) + np.arange(-512, 512) * np.float32(2.0 ** -16)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


@pytest.mark.parametrize("seed", range(4))
def test_bf16_variant_without_rounding_is_the_fp64_backward(seed):
    """With the rounding replaced by the identity the variant is term for term the finite-difference-pinned
    FP64 forward and backward: the variant differs from them only where it rounds."""
    p, x, y = _net(seed)
    ident = lambda v: np.asarray(v, dtype=np.float64)
    loss, g, scale = mlp.backward_bf16(p, x, y, rnd=ident)
    assert loss == pytest.approx(mlp.loss(p, x, y), rel=1e-14)
    g64 = mlp.backward(p, x, y)
    for k in g64:
        assert np.allclose(g[k], g64[k], rtol=1e-13, atol=1e-16), k
        assert np.all(scale[k] >= np.abs(g[k]) * (1 - 1e-12)), k


def _exact_net(seed, d_in=11, hidden=7, B=9):
    """Weights and inputs on coarse grids (W1, W2 in halves, x in quarters of at most 1): every forward
    operand the variant rounds -- x, W1, h1 = relu(sums of 11 products), W2 -- is exactly a BF16 value."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.integers(-2, 3, size=(hidden, d_in)) / 2.0, "b1": rng.integers(-2, 3, size=hidden) / 4.0,
         "W2": rng.integers(-2, 3, size=(hidden, hidden)) / 2.0, "b2": rng.normal(size=hidden) * 0.1,
         "w3": rng.normal(size=hidden) * 0.3, "b3": rng.normal(size=1) * 0.1}
    x = rng.integers(-4, 5, size=(B, d_in)) / 4.0
    y = (rng.random(B) < 0.3).astype(np.float64)
    return p, x, y


@pytest.mark.parametrize("seed", range(4))
def test_bf16_variant_rounds_only_what_the_tensor_cores_receive(seed):
    """On operands that are BF16 values already the forward pass is exactly forward(); the backward pass
    then differs from backward() only by the rounding of dz2 and dz1 (sigmoid values): at most 2^-8
    relative per rounding on the path of each term, two on the longest path (dz2, then dz1), so within
    2^-7 of the element's scale."""
    p, x, y = _exact_net(seed)
    c = mlp.forward(p, x)
    assert np.array_equal(mlp.bf16(c["h1"]), c["h1"])          # the premise
    cb = mlp.forward_bf16(p, x)
    assert np.array_equal(cb["z3"], c["z3"])
    loss, g, scale = mlp.backward_bf16(p, x, y)
    assert loss == mlp.loss(p, x, y)
    g64 = mlp.backward(p, x, y)
    for k in ("w3", "b3", "b2"):                 # upstream of every rounded gradient factor: unchanged
        assert np.allclose(g[k], g64[k], rtol=1e-12, atol=1e-15), k
    for k in ("W2", "b1", "W1"):                 # dz2 rounded (W2, and dz1 through it), dz1 rounded (W1)
        assert np.all(np.abs(g[k] - g64[k]) <= 2.0 ** -7 * scale[k] + 1e-15), k
        assert not np.allclose(g[k], g64[k], rtol=1e-12, atol=0), k      # the rounding is applied there


def test_split_first_layer_without_rounding_is_forward():
    """The pruning pass's split of the first layer (model part, scene part with the positions folded in,
    time term) is exact algebra: with the identity as rounding it gives forward()'s logits."""
    rng = np.random.default_rng(3)
    F, n = 6, 40
    p = mlp.init(rng, 2 * F + 3, 9)
    p["b1"] = rng.normal(size=9) * 0.1
    mf, sf = rng.normal(size=(5, F)), rng.normal(size=(8, F))
    mxy, sxy = rng.uniform(0, 160, (5, 2)), rng.uniform(0, 160, (8, 2))
    mt, st = rng.integers(0, 30, 5), rng.integers(0, 60, 8)
    i, j, o = rng.integers(0, 5, n), rng.integers(0, 8, n), rng.integers(0, 20, n)
    x = mlp.features(mf, sf, mxy, sxy, mt, st, i, j, o, 3)
    ident = lambda v: np.asarray(v, dtype=np.float64)
    z = mlp.score_split_bf16(p, x, mxy[i], sxy[j], F, rnd=ident, window=3)
    assert np.allclose(z, mlp.forward(p, x)["z3"], rtol=1e-12, atol=1e-12)
    # and with BF16 rounding it stays within BF16 relative error of the same logits
    zb = mlp.score_split_bf16(p, x, mxy[i], sxy[j], F, window=3)
    assert np.max(np.abs(zb - z)) <= 0.05 * max(1.0, np.std(z))
