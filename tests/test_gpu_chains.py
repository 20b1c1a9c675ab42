"""The "independent chains" variant on the GPU (hgm_match_chains) against the FP64 chain oracle: every
offset's mean energy within 1e-5 relative, and each chain's part of the assignment an optimal chain of
that chain's own problem."""
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
