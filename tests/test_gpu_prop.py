"""The proposal network's CUDA kernels against the FP64 reference (oracle/mlp.py), and the pruned
matching path: keeping every candidate reproduces the exact path bit for bit, and units whose pruned
optimum is infeasible fall back to the full lists."""
import numpy as np
import pytest

from gpu_util import handles
from oracle import mlp
from paper_1505_00581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1505_00581_gb300 import build, hgm
    build.build()
    hgm.load()
    import oracle
    oracle.build()
    return torch, hgm, oracle


def _ref_params(prop):
    w, _ = prop.get()
    d = prop.unflatten(w.astype(np.float64))
    return {"W1": d["W1"], "b1": d["b1"], "W2": d["W2"], "b2": d["b2"], "w3": d["w3"], "b3": d["b3"]}


def _batch(seed, B, F):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 2 * F + 3)).astype(np.float32)
    y = (rng.random(B) < 0.25).astype(np.float32)
    return X, y


def test_forward_matches_fp64(env):
    torch, hgm, _ = env
    F = 162
    prop = hgm.Proposal(F, seed=3)
    ref = _ref_params(prop)
    rng = np.random.default_rng(1)
    ref["b1"] = rng.normal(size=128) * 0.1
    ref["b2"] = rng.normal(size=128) * 0.1
    ref["b3"] = np.array([0.3])
    w = np.concatenate([ref[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]).astype(np.float32)
    prop.set(w)
    X, y = _batch(2, 300, F)
    out = torch.empty(300, device="cuda")
    prop.forward(torch.from_numpy(X).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    z_emu = mlp.forward_bf16(ref, X.astype(np.float64))["z3"]
    # FP32-accumulated activations can land on the other side of a BF16 rounding midpoint: ~1e-4 each
    assert np.max(np.abs(got - z_emu)) <= 2e-3 * max(1.0, np.max(np.abs(z_emu)))
    z = mlp.forward(ref, X.astype(np.float64))["z3"]       # BF16 operands vs FP64: a few percent of the spread
    assert np.max(np.abs(got - z)) <= 0.05 * max(1.0, np.std(z)), (np.max(np.abs(got - z)), np.std(z))


@pytest.mark.parametrize("B", [64, 1000])
def test_gradients_match_fp64(env, B):
    """Backward kernels against oracle/mlp.py, element by element. The oracle's backward_bf16 rounds to BF16
    exactly the operands the kernels feed to the tensor cores; the kernels then differ from it only by FP32
    accumulation (at most n 2^-24 of an element's scale, n <= 1000 terms: 6e-5) and by activations they
    compute in FP32 that land on the neighbouring BF16 value near a rounding midpoint (one BF16 spacing,
    <= 2^-7 relative, per such operand; at most two roundings, dz2 then dz1, on the longest path). So every
    element lies within 2^-6 of its scale -- the same backward pass on absolute values, the size of
    everything the element sums -- and, the midpoint cases being rare, the median element within 2^-12.
    Against plain FP64 (backward) the BF16 operands move the logits by about a percent, which reaches every
    gradient through sigmoid(z3) - y: relative Frobenius error <= 1e-1."""
    torch, hgm, _ = env
    F = 162
    prop = hgm.Proposal(F, seed=5)
    ref = _ref_params(prop)
    X, y = _batch(3, B, F)
    loss, g = prop.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    gd = prop.unflatten(g.astype(np.float64))
    loss_emu, g_emu, scale = mlp.backward_bf16(ref, X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - loss_emu) <= 1e-5 * max(1.0, loss_emu)
    g64 = mlp.backward(ref, X.astype(np.float64), y.astype(np.float64))
    ratios = []
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        err = np.abs(gd[k] - g_emu[k])
        sc = scale[k] + 1e-30
        assert np.all(err <= 2.0 ** -6 * sc + 1e-12), (k, float(np.max(err / sc)))
        ratios.append((err / sc).reshape(-1))
        rel = np.linalg.norm(gd[k] - g64[k]) / max(np.linalg.norm(g64[k]), 1e-30)
        assert rel <= 1e-1, (k, rel)
    assert np.median(np.concatenate(ratios)) <= 2.0 ** -12


def test_adam_step_and_training_progress(env):
    """One step moves every weight with a clear gradient by lr in the FP64 gradient's direction;
    200 steps on a learnable toy problem lower the loss."""
    torch, hgm, _ = env
    F = 16
    prop = hgm.Proposal(F, seed=7)
    w0, _ = prop.get()
    rng = np.random.default_rng(4)
    B = 512
    fi = rng.normal(size=(B, F))
    same = rng.random(B) < 0.3
    fj = np.where(same[:, None], fi + 0.05 * rng.normal(size=(B, F)), rng.normal(size=(B, F)))
    X = np.concatenate([fi, fj, rng.normal(size=(B, 3)) * 0.1], axis=1).astype(np.float32)
    y = same.astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    ref = _ref_params(prop)
    g64 = mlp.backward(ref, X.astype(np.float64), y.astype(np.float64))
    prop.train_step(Xd, yd, 1e-3)
    torch.cuda.synchronize()
    w1, step = prop.get()
    assert step == 1
    d = prop.unflatten(w1.astype(np.float64) - w0.astype(np.float64))
    for k in ("W1", "W2", "w3"):
        g = g64[k]
        big = np.abs(g) > np.quantile(np.abs(g), 0.5)
        agree = np.mean(np.sign(d[k][big]) == -np.sign(g[big]))
        assert agree >= 0.95, (k, agree)
        assert np.allclose(np.abs(d[k][big]), 1e-3, rtol=0.05), k
    first = mlp.loss(_ref_params(prop), X.astype(np.float64), y.astype(np.float64))
    loss = torch.zeros(1, device="cuda")
    for _ in range(200):
        prop.train_step(Xd, yd, 3e-3, loss)
    torch.cuda.synchronize()
    last = mlp.loss(_ref_params(prop), X.astype(np.float64), y.astype(np.float64))
    assert last < 0.5 * first, (first, last)


def _pair(seed=21, frames=120):
    rng = np.random.default_rng(seed)
    mod = synth.make_model(rng, 30)
    sc = synth.make_scene(rng, frames, (320.0, 240.0), ("poisson", 30.0), mod.centres, [mod], [(0, 40)])
    return synth.Workload("pair", [mod], [sc], K=64, window=3)


def _run(torch, hgm, m, s, p, n, M):
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    a = torch.empty((n, M), dtype=torch.int32, device="cuda")
    hgm.match(m, s, p, e, a)
    torch.cuda.synchronize()
    return e.cpu().numpy(), a.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_keep_all_reproduces_the_unpruned_path(env, precision):
    torch, hgm, _ = env
    wl = _pair()
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    prop = hgm.Proposal(162, seed=1)
    base = hgm.default_params(K=64, window=3, precision=precision)
    first, n = hgm.offsets(m, s, base)
    e0, a0 = _run(torch, hgm, m, s, base, n, mod.n)
    pr = hgm.default_params(K=64, window=3, precision=precision, prune=prop, keep=64)
    e1, a1 = _run(torch, hgm, m, s, pr, n, mod.n)
    if precision == 0:
        assert np.array_equal(e0, e1) and np.array_equal(a0, a1)
    else:
        # precision mode re-scores all 64 kept (instead of the 8 smallest): energies can only move by
        # the BF16 error of the other 56 candidates' costs
        fin = np.isfinite(e0)
        assert np.array_equal(fin, np.isfinite(e1))
        assert np.max(np.abs(e1[fin] - e0[fin]) / e0[fin]) <= 3e-2


def test_pruning_is_a_restriction_with_fallback(env):
    """keep = 2: every pruned optimum is a real chain of the full problem (energy >= exact optimum), and
    units whose pruned problem is infeasible are re-solved on the full lists (same result as exact)."""
    torch, hgm, oracle = env
    wl = _pair(seed=9)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    prop = hgm.Proposal(162, seed=2)
    base = hgm.default_params(K=64, window=3)
    first, n = hgm.offsets(m, s, base)
    e0, a0 = _run(torch, hgm, m, s, base, n, mod.n)
    hgm.prune_counters(reset=True)
    pr = hgm.default_params(K=64, window=3, prune=prop, keep=2)
    e1, a1 = _run(torch, hgm, m, s, pr, n, mod.n)
    pruned, fb = hgm.prune_counters(reset=True)
    assert pruned == n and fb > 0
    fin = np.isfinite(e0)
    assert np.array_equal(fin, np.isfinite(e1))
    assert np.all(e1[fin] >= e0[fin] * (1 - 1e-6))
    orc = oracle.Oracle.from_workload(wl)
    for k in range(0, n, 7):
        if fin[k]:
            assert abs(orc.energy(a1[k]) - e1[k]) <= 1e-5 * e1[k]


@pytest.mark.parametrize("keep", [6, 12])
def test_pruned_lists_are_the_top_scores(env, keep):
    """The kept candidates of every list are its `keep` highest logits (ties: lower slot), in slot order:
    on a 4-point model the pruned optimum of each offset equals the brute-force minimum of Eq. 9 over the
    lists built that way in numpy from the scoring kernel's own logits (or, when those lists hold no
    feasible chain, the exact optimum of the fallback). keep 6 takes the kernel's argmax rounds, keep 12
    its threshold bisection."""
    import itertools
    torch, hgm, oracle = env
    rng = np.random.default_rng(31)
    mod = synth.make_model(rng, 4, t_span=8)
    sc = synth.make_scene(rng, 40, (320.0, 240.0), ("poisson", 30.0), mod.centres, [mod], [(0, 10)])
    wl = synth.Workload("tiny", [mod], [sc], K=64, window=3)
    m, s = handles(hgm, mod, sc, torch)
    prop = hgm.Proposal(162, seed=5)
    base = hgm.default_params(K=64, window=3)
    first, n = hgm.offsets(m, s, base)
    idx = torch.empty((n, 4, 64), dtype=torch.int32, device="cuda")
    cnt = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    hgm.candidates(m, s, base, first, n, idx, cnt)
    sco = torch.full((n, 4, 64), 7.0, dtype=torch.float32, device="cuda")
    hgm.prop_scores(prop, m, s, base, first, n, sco)
    pr = hgm.default_params(K=64, window=3, prune=prop, keep=keep)
    e1, _ = _run(torch, hgm, m, s, pr, n, 4)
    idx, cnt, sco = idx.cpu().numpy(), cnt.cpu().numpy(), sco.cpu().numpy()
    mperm, sperm = m.order(), s.order()
    orc = oracle.Oracle.from_workload(wl)
    assert orc.first_offset == first and orc.n_offsets == n
    checked = 0
    for k in range(0, n, 3):
        lists = []
        for i in range(4):
            c = int(cnt[k, i])
            top = sorted(range(c), key=lambda j: (-float(sco[k, i, j]), j))[:keep]
            lists.append([int(sperm[idx[k, i, j]]) for j in sorted(top)])
        best = np.inf
        z = np.empty(4, np.int64)
        for combo in itertools.product(*lists):
            for i in range(4):
                z[mperm[i]] = combo[i]
            best = min(best, orc.energy(z))
        if not np.isfinite(best):
            best = orc.match(first + k)[0]   # no feasible chain through the kept candidates: the fallback
        if np.isfinite(best):
            assert abs(float(e1[k]) - best) <= 1e-5 * max(1.0, best), (k, e1[k], best)
            checked += 1
        else:
            assert not np.isfinite(e1[k])
    assert checked >= 5


def _pair_features(mod, sc, m, s, first, idx, cnt, window):
    """FP64 network inputs of every candidate slot: [f_i, f'_j, dx/100, dy/100, dt/w] with i, j the caller
    indices behind the sorted indices of the candidate lists; mask of the filled slots."""
    mperm, sperm = m.order(), s.order()
    n, M, K = idx.shape
    valid = np.arange(K)[None, None, :] < cnt[:, :, None]
    i_c = np.broadcast_to(mperm[np.arange(M)][None, :, None], (n, M, K))
    j_c = sperm[np.where(valid, idx, 0)]
    o = (first + np.arange(n))[:, None, None]
    d = np.stack([(sc.xy[j_c, 0].astype(np.float64) - mod.xy[i_c, 0]) / 100.0,
                  (sc.xy[j_c, 1].astype(np.float64) - mod.xy[i_c, 1]) / 100.0,
                  (sc.t[j_c].astype(np.float64) - mod.t[i_c] - o) / float(window)], axis=-1)
    X = np.concatenate([mod.f[i_c].astype(np.float64), sc.f[j_c].astype(np.float64), d], axis=-1)
    return X[valid], valid, mod.xy[i_c][valid].astype(np.float64), sc.xy[j_c][valid].astype(np.float64)


@pytest.mark.parametrize("K,window,precision", [(64, 0, 0), (24, 3, 1)])
def test_scoring_kernel_matches_fp64(env, K, window, precision):
    """The pruning pass's logits (first layer from the per-point projections with the position terms folded
    in, layer 2 on the tensor cores) against the FP64 network on the same candidates: to 2e-3 of the logit
    range against the emulation that rounds to BF16 what the kernels round (the descriptors and W1a/W1b in
    the projections, both projections once they hold the position terms, the first layer's BF16x2 add and
    fused multiply-add, W2 and b2 in layer 2); within
    5% of the spread against plain FP64. Empty slots are
    -inf. K = 64 with w = 0: lists of about 30 candidates (many empty slots); K = 24 with w = 3: full lists,
    four lists of 32 rows (8 of them empty) in each 128-row tile."""
    torch, hgm, _ = env
    F = 162
    wl = _pair(seed=5, frames=90)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    prop = hgm.Proposal(F, seed=11)
    ref = _ref_params(prop)
    rng = np.random.default_rng(8)
    ref["b1"] = rng.normal(size=128) * 0.1
    ref["b2"] = rng.normal(size=128) * 0.1
    ref["b3"] = np.array([-0.2])
    ref["W1"][:, 2 * F:] = rng.normal(size=(128, 3)) * 0.5
    w = np.concatenate([ref[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]).astype(np.float32)
    prop.set(w)
    ref = _ref_params(prop)
    p = hgm.default_params(K=K, window=window, precision=precision)
    first, n = hgm.offsets(m, s, p)
    first, n = first + 7, min(n - 7, 9)
    idx = torch.empty((n, mod.n, K), dtype=torch.int32, device="cuda")
    cnt = torch.empty((n, mod.n), dtype=torch.int32, device="cuda")
    hgm.candidates(m, s, p, first, n, idx, cnt)
    out = torch.full((n, mod.n, K), 7.0, dtype=torch.float32, device="cuda")
    hgm.prop_scores(prop, m, s, p, first, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    X, valid, mxy, sxy = _pair_features(mod, sc, m, s, first, idx.cpu().numpy(), cnt.cpu().numpy(),
                                        max(window, 1))
    assert valid.sum() > 1000 and (window > 0 or (~valid).sum() > 1000)
    assert np.all(got[~valid] == -np.inf)
    g = got[valid]
    assert np.all(np.isfinite(g))
    z64 = mlp.forward(ref, X)["z3"]
    # P per model point and Q per scene point, each rounded once to BF16 with the position terms folded in;
    # the first layer in BF16x2 arithmetic with the time term per candidate (oracle/mlp.py: score_split_bf16)
    z_emu = mlp.score_split_bf16(ref, X, mxy, sxy, F, window=window)
    assert np.max(np.abs(g - z_emu)) <= 2e-3 * max(1.0, np.max(np.abs(z_emu))), np.max(np.abs(g - z_emu))
    assert np.max(np.abs(g - z64)) <= 0.05 * max(1.0, np.std(z64)), (np.max(np.abs(g - z64)), np.std(z64))


def test_scoring_kernel_rejects_long_lists(env):
    torch, hgm, _ = env
    wl = _pair(seed=5, frames=60)
    m, s = handles(hgm, wl.models[0], wl.scenes[0], torch)
    prop = hgm.Proposal(162, seed=1)
    p = hgm.default_params(K=65, window=3)
    out = torch.empty(16, device="cuda")
    with pytest.raises(hgm.HgmError) as err:
        hgm.prop_scores(prop, m, s, p, 0, 1, out)
    assert err.value.status == 5
