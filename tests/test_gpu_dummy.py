"""The dummy assignment (Eq. 2, reading R5) on the GPU against the FP64 oracle with the same W^d: every
offset's energy within 1e-5 relative, assignments (eps = -2) equal or of the same FP64 energy; offsets
whose lists are empty become feasible; an expensive dummy reproduces the plain path."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from gpu_util import check_offset, handles
from paper_1505_00581_gb300 import synth

pytestmark = pytest.mark.gpu
LAM = dict(lambda1=0.6, lambda2=0.2, lambda3=5.0)


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


def _check_pair(hgm, oracle, mod, sc, K, window, wd, precision=0, torch=None, T=10):
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=K, window=window, T=T, dummy_cost=wd, precision=precision)
    first, e, a = hgm.match(m, s, p)
    orc = oracle.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=K, window=window, T=T,
                        dummy_cost=wd, **LAM)
    assert first == orc.first_offset and len(e) == orc.n_offsets
    n_eps = 0
    for k in range(len(e)):
        e64, z64, _ = orc.match(first + k)
        assert np.isfinite(e64) and np.isfinite(e[k])
        tol = 1e-5 * e64 + 1e-6 if precision == 0 else 2e-2 * e64 + 1e-4
        assert abs(e[k] - e64) <= tol, (k, e[k], e64)
        if precision == 0 and not np.array_equal(a[k], z64):
            assert orc.energy(a[k]) <= e64 * (1 + 1e-5) + 1e-6, (k, orc.energy(a[k]), e64)
        n_eps += int(np.sum(a[k] == -2))
    return n_eps


@pytest.mark.parametrize("wd", [0.5, 3.0, 8.0])
def test_dummy_matches_oracle_single_pair(env, wd):
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    n_eps = _check_pair(hgm, oracle, wl.models[0], wl.scenes[0], 32, 2, wd, torch=torch)
    if wd == 0.5:
        assert n_eps > 0           # cheap dummies are taken


def test_dummy_small_random_and_empty_windows(env):
    """Sparse scenes (Poisson 0.7 points per frame, window 0): many lists are empty and only the
    dummy makes those offsets feasible."""
    torch, hgm, oracle = env
    rng = np.random.default_rng(77)
    for k in range(4):
        mod = synth.make_model(rng, int(rng.integers(5, 12)), F=16, t_span=10)
        sc = synth.make_scene(rng, 40, (60.0, 40.0), ("poisson", 0.7), mod.centres, [mod], [(0, 9)])
        _check_pair(hgm, oracle, mod, sc, 8, 0, [0.2, 1.0, 2.5, 6.0][k], T=[10, 4, 10, 0][k])


def test_dummy_precision_mode(env):
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    _check_pair(hgm, oracle, wl.models[0], wl.scenes[0], 32, 2, 3.0, precision=1, torch=torch)


def test_expensive_dummy_is_the_plain_path(env):
    torch, hgm, _ = env
    wl = synth.batched_exact(seed=43, n_models=3, n_scenes=2, frames_range=(80, 120))
    M = [hgm.Model(m.xy, m.t, m.f) for m in wl.models]
    S = [hgm.Scene(s.xy, s.t, s.f, s.n_frames) for s in wl.scenes]
    base = hgm.default_params(K=64, window=3)
    first, es, as_ = hgm.batch_layout(M, S, base)
    e0 = np.zeros(int(es[-1]), np.float32)
    a0 = np.zeros(int(as_[-1]), np.int32)
    hgm.match_batch(M, S, base, e0, a0)
    e1 = np.zeros_like(e0)
    a1 = np.zeros_like(a0)
    hgm.match_batch(M, S, hgm.default_params(K=64, window=3, dummy_cost=1e5), e1, a1)
    fin = np.isfinite(e0)
    assert fin.sum() > 100
    assert np.max(np.abs(e1[fin] - e0[fin]) / e0[fin]) <= 2e-6
    assert np.all(e1[~fin] >= 1e5 * 0.6)
    same = 0
    for q in range(len(M) * len(S)):
        Mq = wl.models[q // len(S)].n
        for k in range(int(es[q + 1] - es[q])):
            if fin[es[q] + k]:
                ka = int(as_[q]) + k * Mq
                same += np.array_equal(a0[ka:ka + Mq], a1[ka:ka + Mq])
    assert same >= 0.99 * fin.sum()


def test_dummy_rejected_with_pruning_and_blocks(env):
    torch, hgm, _ = env
    wl = synth.single_match(0)
    m, s = handles(hgm, wl.models[0], wl.scenes[0])
    prop = hgm.Proposal(162, seed=1)
    with pytest.raises(hgm.HgmError) as err:
        hgm.match(m, s, hgm.default_params(K=32, window=2, dummy_cost=1.0, prune=prop, keep=4))
    assert err.value.status == hgm.HGM_EUNSUPPORTED
    with pytest.raises(hgm.HgmError) as err:
        hgm.match_block([m], [s], hgm.default_params(dummy_cost=1.0))
    assert err.value.status == hgm.HGM_EUNSUPPORTED


def test_full_batched_workload_sampled(env):
    """The 10-model x 8-scene workload at full size with W^d = 8, in the benchmark's launch configuration
    (one batch call, device outputs): every offset finite, and a seeded sample of units plus the implants'
    own offsets against the oracle with the same W^d."""
    torch, hgm, oracle = env
    wl = synth.batched_exact()
    wd = 8.0
    ms = [hgm.Model(*(torch.from_numpy(a).cuda() for a in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    ss = [hgm.Scene(*(torch.from_numpy(a).cuda() for a in (sc.xy, sc.t, sc.f)), sc.n_frames) for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T, dummy_cost=wd)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    hgm.match_batch(ms, ss, p, e, a)
    torch.cuda.synchronize()
    e, a = e.cpu().numpy(), a.cpu().numpy()
    assert np.all(np.isfinite(e))
    assert np.all((a >= 0) | (a == -2))
    rng = np.random.default_rng(2025)
    samples = []
    for _ in range(32):
        mi = int(rng.integers(len(wl.models)))
        si = int(rng.integers(len(wl.scenes)))
        q = mi * len(wl.scenes) + si
        samples.append((mi, si, q, int(rng.integers(int(es[q + 1] - es[q])))))
    for si, sc in enumerate(wl.scenes):
        for imp in sc.implants:
            q = imp.model * len(wl.scenes) + si
            k = imp.offset - int(first[q])
            if 0 <= k < es[q + 1] - es[q]:
                samples.append((imp.model, si, q, k))
    oracles = {}
    for mi, si, q, k in samples:
        if (mi, si) not in oracles:
            oracles[(mi, si)] = oracle.Oracle.from_workload(wl, mi, si, dummy_cost=wd)

    def run(sample):
        mi, si, q, k = sample
        M = wl.models[mi].n
        orc = oracles[(mi, si)]
        e_or, z_or, _ = orc.match(int(first[q]) + k)
        row = a[as_[q] + k * M: as_[q] + (k + 1) * M]
        return check_offset(orc, int(first[q]) + k, e[es[q] + k], row, e_or=e_or, z_or=z_or)

    with ThreadPoolExecutor(max_workers=16) as ex:
        results = list(ex.map(run, samples))
    for (ok, tie, why), smp in zip(results, samples):
        assert ok, (smp, why)


def test_accounting_variant_gives_identical_results(env):
    """hgm_profile_enable(2) runs the dummy kernel's accounting variant: same energies and assignments bit
    for bit, and a positive evaluation count no larger than the dense count of (a, b, c) over the real
    candidates of every step (the walks evaluate real a against open real cells only)."""
    torch, hgm, _ = env
    wl = synth.batched_exact(seed=7, n_models=2, n_scenes=1, frames_range=(80, 80))
    ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
    ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T, dummy_cost=8.0)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    outs = []
    for mode in (0, 2):
        e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
        a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
        hgm.profile_evaluated(reset=True)
        hgm.profile_enable(mode)
        try:
            hgm.match_batch(ms, ss, p, e, a)
        finally:
            hgm.profile_enable(0)
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy(), a.cpu().numpy(), hgm.profile_evaluated(reset=True)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == 0
    ev = outs[1][2]
    dense = 0
    for mi, mod in enumerate(wl.models):
        idx = torch.empty((int(es[mi + 1] - es[mi]), mod.n, wl.K), dtype=torch.int32, device="cuda")
        cnt = torch.empty((int(es[mi + 1] - es[mi]), mod.n), dtype=torch.int32, device="cuda")
        hgm.candidates(ms[mi], ss[0], p, int(first[mi]), int(es[mi + 1] - es[mi]), idx, cnt)
        c = cnt.cpu().numpy().astype(np.int64)
        dense += int(np.sum(c[:, 2:] * c[:, 1:-1] * c[:, :-2]))
    assert 0 < ev <= dense, (ev, dense)
