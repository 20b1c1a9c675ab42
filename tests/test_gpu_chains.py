"""The "independent chains" variant on the GPU (hgm_match_chains) against the FP64 chain oracle: every
offset's mean energy within 1e-5 relative, and each chain's part of the assignment an optimal chain of
that chain's own problem."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

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


def _multi_point_case(seed, frames, per_frame, n_scene_frames, clutter, F=162):
    rng = np.random.default_rng(seed)
    t = np.repeat(np.arange(frames), per_frame)
    rng.shuffle(t)
    base = synth.make_model(rng, len(t), F=F)
    mod = synth.PointSet(base.xy, t.astype(np.int32), base.f, base.centres)
    sc = synth.make_scene(rng, n_scene_frames, (320.0, 240.0), ("poisson", clutter), mod.centres, [mod],
                          [(0, n_scene_frames // 3)])
    return mod, sc


@pytest.mark.parametrize("K,per_frame,n_chains", [(8, 2, 2), (32, 3, 3), (32, np.array([1, 2, 3, 2, 3, 1, 2, 3, 2, 1]), 3)])
def test_chains_match_the_chain_oracle(env, K, per_frame, n_chains):
    torch, hgm, oracle = env
    frames = 10
    mod, sc = _multi_point_case(3 + K, frames, per_frame, 60, 6.0)
    dev = torch.device("cuda")
    m = hgm.Model(*(torch.from_numpy(a).to(dev) for a in (mod.xy, mod.t, mod.f)))
    s = hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (sc.xy, sc.t, sc.f)), sc.n_frames)
    p = hgm.default_params(K=K, window=2)
    first, e, a = hgm.match_chains(m, s, p, n_chains)
    co = oracle.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, n_chains, K=K, window=2, T=10,
                            **LAM)
    assert first == co.first_offset and len(e) == co.n_offsets
    finite = 0
    for k in range(len(e)):
        o = first + k
        e64, _ = co.match(o)
        assert np.isfinite(e64) == np.isfinite(e[k]), o
        if not np.isfinite(e64):
            continue
        finite += 1
        assert abs(e[k] - e64) <= 1e-5 * e64 + 1e-6, (o, e[k], e64)
        for idx, orc in zip(co.members, co.chains):
            ec, _, _ = orc.match(o)
            assert orc.energy(a[k][idx]) <= ec * (1 + 1e-5) + 1e-6
        outside = np.setdiff1d(np.arange(mod.n), np.concatenate(co.members))
        assert np.all(a[k][outside] == -1)
    assert finite > 10


def test_chains_need_a_chain_of_three(env):
    torch, hgm, _ = env
    mod, sc = _multi_point_case(7, 4, 2, 30, 4.0)        # 4 frames x 2 points: chains of 4 points
    m = hgm.Model(mod.xy, mod.t, mod.f)
    s = hgm.Scene(sc.xy, sc.t, sc.f, sc.n_frames)
    p = hgm.default_params(K=8, window=2)
    hgm.match_chains(m, s, p, 2)                          # fine
    short = synth.PointSet(mod.xy[:4], np.array([0, 0, 1, 1], np.int32), mod.f[:4], mod.centres)
    m2 = hgm.Model(short.xy, short.t, short.f)
    with pytest.raises(hgm.HgmError) as err:
        hgm.match_chains(m2, s, p, 2)                     # two chains of 2 points
    assert err.value.status == hgm.HGM_EINVAL


def test_chains_batch_matches_pairs_and_oracle(env):
    """hgm_match_chains_batch over 3 models x 2 scenes: identical (bit for bit) to per-pair hgm_match_chains,
    laid out as hgm_batch_layout, and on every offset within 1e-5 of the chain oracle; device outputs; the
    split is rebuilt when n_chains changes."""
    torch, hgm, oracle = env
    dev = torch.device("cuda")
    cases = [(11, 10, 2, 50, 5.0), (12, 8, np.array([1, 2, 3, 2, 3, 1, 2, 3]), 70, 6.0), (13, 12, 3, 40, 4.0)]
    mods, scs = [], []
    for seed, frames, per_frame, nf, clutter in cases:
        mod, sc = _multi_point_case(seed, frames, per_frame, nf, clutter)
        mods.append(mod)
        scs.append(sc)
    scs = scs[:2]
    M = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in mods]
    S = [hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (s.xy, s.t, s.f)), s.n_frames) for s in scs]
    p = hgm.default_params(K=16, window=2)
    first, es, as_ = hgm.batch_layout(M, S, p)
    for n_chains in (3, 2, 3):
        e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
        a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
        hgm.match_chains_batch(M, S, p, n_chains, e, a)
        torch.cuda.synchronize()
        e, a = e.cpu().numpy(), a.cpu().numpy()
        for mi, mod in enumerate(mods):
            for si, sc in enumerate(scs):
                q = mi * len(scs) + si
                f1, e1, a1 = hgm.match_chains(M[mi], S[si], p, n_chains)
                n = int(es[q + 1] - es[q])
                assert f1 == first[q] and len(e1) == n
                np.testing.assert_array_equal(e[es[q]:es[q + 1]], e1)
                np.testing.assert_array_equal(a[as_[q]:as_[q + 1]].reshape(n, mod.n), a1)
                if n_chains != 3:
                    continue
                co = oracle.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, n_chains, K=16,
                                        window=2, T=10, **LAM)
                assert co.first_offset == f1 and co.n_offsets == n
                for k in range(n):
                    e64, _ = co.match(f1 + k)
                    assert np.isfinite(e64) == np.isfinite(e1[k]), (q, k)
                    if np.isfinite(e64):
                        assert abs(e1[k] - e64) <= 1e-5 * e64 + 1e-6, (q, k, e1[k], e64)


def check_chain_offset(co, o, e_gpu, row):
    """(ok, why) for one offset of the chains form: the mean energy within 1e-5 relative of the FP64 one,
    each chain's part of the assignment of FP64 energy within 1e-5 of that chain's optimum, and the points
    outside every chain -1. Each chain problem is solved once."""
    energies = []
    for idx, orc in zip(co.members, co.chains):
        ec, _, _ = orc.match(o)
        energies.append(ec)
        if np.isfinite(ec) and not orc.energy(np.asarray(row)[idx]) <= ec * (1 + 1e-5) + 1e-6:
            return False, f"chain {len(energies) - 1}: E64 {orc.energy(np.asarray(row)[idx])} vs {ec}"
    e64 = float(np.mean(energies)) if all(np.isfinite(energies)) else float("inf")
    if np.isfinite(e64) != np.isfinite(e_gpu):
        return False, f"feasibility: {e_gpu} vs {e64}"
    if np.isfinite(e64) and not abs(e_gpu - e64) <= 1e-5 * e64 + 1e-6:
        return False, f"energy {e_gpu} vs {e64}"
    outside = np.setdiff1d(np.arange(co.M), np.concatenate(co.members))
    if not np.all(np.asarray(row)[outside] == -1):
        return False, "a point outside every chain is assigned"
    return True, ""


def test_full_batched_workload_sampled(env):
    """The chains form on the 10-model x 8-scene workload at full size, in the benchmark's launch
    configuration (one hgm_match_chains_batch call, 3 chains, device outputs): a seeded sample of offsets
    and the implants' own offsets against the chain oracle."""
    torch, hgm, oracle = env
    wl = synth.batched_exact()
    n_chains = 3
    ms = [hgm.Model(*(torch.from_numpy(x).cuda() for x in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    ss = [hgm.Scene(*(torch.from_numpy(x).cuda() for x in (sc.xy, sc.t, sc.f)), sc.n_frames) for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    hgm.match_chains_batch(ms, ss, p, n_chains, e, a)
    torch.cuda.synchronize()
    e, a = e.cpu().numpy(), a.cpu().numpy()
    samples = chain_samples(wl, first, es)
    oracles = {}
    for mi, si, q, k in samples:
        if (mi, si) not in oracles:
            mod, sc = wl.models[mi], wl.scenes[si]
            oracles[(mi, si)] = oracle.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, n_chains,
                                                   K=wl.K, window=wl.window, T=wl.T, lambda1=wl.lambda1,
                                                   lambda2=wl.lambda2, lambda3=wl.lambda3)

    def run(sample):
        mi, si, q, k = sample
        M = wl.models[mi].n
        return check_chain_offset(oracles[(mi, si)], int(first[q]) + k, float(e[es[q] + k]),
                                  a[as_[q] + k * M: as_[q] + (k + 1) * M])

    with ThreadPoolExecutor(max_workers=16) as ex:
        results = list(ex.map(run, samples))
    for (ok, why), smp in zip(results, samples):
        assert ok, (smp, why)


def chain_samples(wl, first, es, n=24, seed=2026):
    """Seeded (model, scene, pair, offset slot) samples plus every implant's own offset."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        mi = int(rng.integers(len(wl.models)))
        si = int(rng.integers(len(wl.scenes)))
        q = mi * len(wl.scenes) + si
        out.append((mi, si, q, int(rng.integers(int(es[q + 1] - es[q])))))
    for si, sc in enumerate(wl.scenes):
        for imp in sc.implants:
            q = imp.model * len(wl.scenes) + si
            k = imp.offset - int(first[q])
            if 0 <= k < es[q + 1] - es[q]:
                out.append((imp.model, si, q, k))
    return out
