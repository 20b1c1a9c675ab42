"""The whole-block problem on the GPU (hgm_match_block) against the FP64 oracle's whole-block solve:
energies within 1e-5 relative, assignments equal or of the same FP64 energy (reading R6), on blocks whose
band tables live in shared memory and on larger ones that use the global-memory form."""
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


def _check(hgm, oracle, mods, scs, T=10, device=None, torch=None):
    if device is not None:
        M = [hgm.Model(*(torch.from_numpy(a).to(device) for a in (m.xy, m.t, m.f))) for m in mods]
        S = [hgm.Scene(*(torch.from_numpy(a).to(device) for a in (s.xy, s.t, s.f)), s.n_frames) for s in scs]
    else:
        M = [hgm.Model(m.xy, m.t, m.f) for m in mods]
        S = [hgm.Scene(s.xy, s.t, s.f, s.n_frames) for s in scs]
    p = hgm.default_params(K=8, window=1, T=T)
    e, a = hgm.match_block(M, S, p)
    starts = hgm.block_layout(M, len(S))
    finite = 0
    for mi, mod in enumerate(mods):
        for si, sc in enumerate(scs):
            q = mi * len(scs) + si
            orc = oracle.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=8, window=1, T=T, **LAM)
            e64, z64, _ = orc.match_block()
            z = a[starts[q]:starts[q + 1]]
            assert np.isfinite(e64) == np.isfinite(e[q]), (q, e64, e[q])
            if not np.isfinite(e64):
                assert np.all(z == -1)
                continue
            finite += 1
            assert abs(e[q] - e64) <= 1e-5 * e64 + 1e-6, (q, e[q], e64)
            if not np.array_equal(z, z64):
                assert orc.energy(z) <= e64 * (1 + 1e-5) + 1e-6, (q, orc.energy(z), e64)
    return finite


@pytest.mark.parametrize("seed", range(6))
def test_block_small_random(env, seed):
    torch, hgm, oracle = env
    rng = np.random.default_rng(900 + seed)
    mods, scs = [], []
    for k in range(2):
        mod = synth.make_model(rng, int(rng.integers(3, 12)), F=16, t_span=12)
        mods.append(mod)
    pool = np.concatenate([m.centres for m in mods])
    for k in range(2):
        scs.append(synth.make_scene(rng, int(rng.integers(8, 30)), (60.0, 40.0), ("poisson", 2.0), pool, mods,
                                    [(k % 2, 2)]))
    T = [10, 4, 0][seed % 3]
    assert _check(hgm, oracle, mods, scs, T=T) >= 1


def test_block_paper_shaped(env):
    """Models of 30 one-per-frame points against 60-frame blocks of about one point per frame."""
    torch, hgm, oracle = env
    wl = synth.paper_blocks(seed=11, n_models=4, n_blocks=3, implant_frac=1.0)
    assert _check(hgm, oracle, wl.models, wl.scenes, device=torch.device("cuda"), torch=torch) >= 1


def test_block_global_memory_form(env):
    """A block with about 40,000 band cells (more than two copies of the alpha table fit in shared
    memory) and T = 0 (no closeness limit) on a small one."""
    torch, hgm, oracle = env
    rng = np.random.default_rng(31)
    mod = synth.make_model(rng, 7, F=16, t_span=8)
    sc = synth.make_scene(rng, 40, (60.0, 40.0), 10, mod.centres, [mod], [(0, 10)])
    assert _check(hgm, oracle, [mod], [sc], T=10) == 1
    mod2 = synth.make_model(rng, 5, F=16, t_span=6)
    sc2 = synth.make_scene(rng, 60, (60.0, 40.0), 5, mod2.centres, [mod2], [(0, 20)])
    assert _check(hgm, oracle, [mod2], [sc2], T=0) == 1


def test_block_rejects_precision_and_pruning(env):
    torch, hgm, _ = env
    wl = synth.paper_blocks(seed=12, n_models=1, n_blocks=1)
    m = hgm.Model(wl.models[0].xy, wl.models[0].t, wl.models[0].f)
    s = hgm.Scene(wl.scenes[0].xy, wl.scenes[0].t, wl.scenes[0].f, wl.scenes[0].n_frames)
    with pytest.raises(hgm.HgmError) as err:
        hgm.match_block([m], [s], hgm.default_params(K=8, window=1, precision=1))
    assert err.value.status == hgm.HGM_EUNSUPPORTED
