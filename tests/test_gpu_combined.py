"""The combined workload's shape (models of up to 256 points, 640x480 scenes with Poisson(80) points per
frame, implants at about 5% of the offsets) on the combined path -- BF16 unary table with FP32 re-score,
learned pruning with exact fallback, recorded as a CUDA graph -- at a reduced scale (4 models, one
4,000-frame scene). The graph replay equals the direct call bit for bit; on a seeded sample of offsets the
pruned optimum is a restriction of the exact problem: feasible exactly where the FP64 optimum is, never
below it, and a real chain whose FP64 energy matches the reported one."""
import os

import numpy as np
import pytest

from paper_1505_00581_gb300 import synth
from test_gpu_precision import _sub_oracle

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


def test_combined_sample_bf16_pruned_graph(env):
    torch, hgm, oracle = env
    wl = synth.combined(seed=3, n_models=4, n_scenes=1, frames_range=(4000, 4000))
    wl.models[0] = synth.make_model(np.random.default_rng(11), 256)   # the largest model size of the workload
    sc = wl.scenes[0]
    dev = torch.device("cuda")
    ms = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    s = hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (sc.xy, sc.t, sc.f)), sc.n_frames)
    prop = hgm.Proposal(162, seed=21)
    p = hgm.default_params(K=64, window=3, precision=1, prune=prop, keep=8)
    first, es, as_ = hgm.batch_layout(ms, [s], p)
    e0 = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a0 = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    hgm.prune_counters(reset=True)
    hgm.match_batch(ms, [s], p, e0, a0)
    torch.cuda.synchronize()
    n_units, n_fb = hgm.prune_counters(reset=True)
    assert n_units == int(es[-1]) and n_fb > 0
    e1 = torch.full_like(e0, -1.0)
    a1 = torch.full_like(a0, -1)
    plan = hgm.Plan(ms, [s], p, e1, a1)
    e1.fill_(-1.0)
    a1.fill_(-1)
    plan.run()
    plan.check()
    assert torch.equal(e0, e1) and torch.equal(a0, a1)
    plan.close()
    rng = np.random.default_rng(5)
    checked = 0
    for m in range(len(wl.models)):
        n = int(es[m + 1] - es[m])
        for k in rng.integers(0, n, size=5):
            o = int(first[m]) + int(k)
            ep = float(e0[int(es[m]) + int(k)].item())
            M = wl.models[m].n
            row = int(as_[m]) + int(k) * M
            ap = a0[row:row + M].cpu().numpy()
            orc, o_sub, keep = _sub_oracle(oracle, wl, m, o)
            e64, _, _ = orc.match(o_sub)
            assert np.isfinite(e64) == np.isfinite(ep), (m, o)
            if np.isfinite(e64):
                assert ep >= e64 * (1 - 3e-2), (m, o, ep, e64)       # a restriction (BF16 costs: 3e-2 slack)
                z_sub = np.searchsorted(keep, ap)
                assert np.all(keep[z_sub] == ap)
                assert abs(orc.energy(z_sub) - ep) <= 3e-2 * e64
                checked += 1
            del orc
    assert checked >= 16


def test_combined_full_model_set_full_length_scene(env):
    """The combined workload's full model set (100 models of 16-256 points) against one of its full-length
    scenes (the shortest of the 16, about 19k frames of Poisson(80) points at 640x480, implants at about 5%
    of the offsets), every offset of every model in one batch, in both forms the benchmark times:
    plain exact FP32 -- on seeded offsets and on implant offsets every energy within 1e-5 of the FP64 oracle
    and every assignment the oracle's or one of the same FP64 energy -- and BF16 distances + learned pruning
    (network trained as the benchmark trains it, keep 8, exact fallback) -- on the same offsets a restriction
    of the exact problem: feasible exactly where the oracle is, never more than the BF16 error below it, and
    a real chain whose FP64 energy matches the reported one."""
    from concurrent.futures import ThreadPoolExecutor

    from gpu_util import check_offset
    from paper_1505_00581_gb300 import prop_train
    torch, hgm, oracle = env
    cs = synth.CombinedScenes(seed=3)
    s_idx = int(np.argmin(cs.n_frames))
    sc = cs.scene(s_idx)
    wl = synth.Workload("combined_full_scene", cs.models, [sc], K=64, window=3)
    dev = torch.device("cuda")
    ms = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    s = hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (sc.xy, sc.t, sc.f)), sc.n_frames)
    p = hgm.default_params(K=64, window=3)
    first, es, as_ = hgm.batch_layout(ms, [s], p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    hgm.match_batch(ms, [s], p, e, a)
    torch.cuda.synchronize()
    e_ex, a_ex = e.cpu().numpy(), a.cpu().numpy()
    prop, _ = prop_train.train_default(torch, wl, steps=2000, seed=101, train_wl=cs.training_scenes(101))
    pp = hgm.default_params(K=64, window=3, precision=1, prune=prop, keep=8)
    hgm.match_batch(ms, [s], pp, e, a)
    torch.cuda.synchronize()
    e_pr, a_pr = e.cpu().numpy(), a.cpu().numpy()
    prop.close()

    rng = np.random.default_rng(17)
    picks = [(int(m), int(first[m]) + int(rng.integers(int(es[m + 1] - es[m]))))
             for m in rng.integers(0, len(wl.models), size=20)]
    for imp in sc.implants[:4]:
        picks.append((imp.model, imp.offset))

    def solve(mo):
        m, o = mo
        orc, o_sub, keep = _sub_oracle(oracle, wl, m, o)
        e64, z64, _ = orc.match(o_sub)
        return orc, o_sub, keep, e64, z64

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        solved = list(ex.map(solve, picks))
    for (m, o), (orc, o_sub, keep, e64, z64) in zip(picks, solved):
        k = o - int(first[m])
        M = wl.models[m].n
        row = slice(int(as_[m]) + k * M, int(as_[m]) + (k + 1) * M)
        # exact form: the parity rule of every exact-path test
        z_ex = a_ex[row]
        z_sub = np.searchsorted(keep, z_ex) if np.isfinite(e64) else z_ex
        if np.isfinite(e64):
            assert np.all(keep[z_sub] == z_ex), (m, o)
        ok, tie, why = check_offset(orc, o_sub, float(e_ex[int(es[m]) + k]), z_sub, e64, z64)
        assert ok, (m, o, why)
        # pruned + BF16 form: a restriction of the exact problem
        ep = float(e_pr[int(es[m]) + k])
        assert np.isfinite(e64) == np.isfinite(ep), (m, o)
        if np.isfinite(e64):
            assert ep >= e64 * (1 - 3e-2), (m, o, ep, e64)
            zp = np.searchsorted(keep, a_pr[row])
            assert np.all(keep[zp] == a_pr[row])
            assert abs(orc.energy(zp) - ep) <= 3e-2 * e64
