"""Streaming blocks on the GPU (hgm_stream_*): a scene cut into 60-frame blocks every 30 frames, each block
matched whole against every model, against the FP64 oracle's whole-block solve of the same block, and
bit for bit against hgm_match_block on a scene handle of that block."""
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


def _long_scene(seed, n_models=3, n_frames=240, lam=1.2):
    rng = np.random.default_rng(seed)
    models = [synth.paper_model(rng, 30) for _ in range(n_models)]
    pool = np.concatenate([m.centres for m in models])
    imps = [(k % n_models, int(o)) for k, o in enumerate(range(10, n_frames - 30, 70))]
    sc = synth.make_scene(rng, n_frames, (160.0, 120.0), ("poisson", lam), pool, models, imps)
    return models, sc


def test_stream_blocks_match_oracle_and_block_call(env):
    torch, hgm, oracle = env
    mods, sc = _long_scene(5)
    M = [hgm.Model(m.xy, m.t, m.f) for m in mods]
    p = hgm.default_params()
    st = hgm.Stream(M, p, 60)
    n_blocks = finite = 0
    for s0, bxy, bt, bf, idx in hgm.stream_blocks(sc.xy, sc.t, sc.f, sc.n_frames, 60, 30):
        e, a = st.match(bxy, bt, bf)
        # the same block as a scene handle through hgm_match_block: identical bits
        S = hgm.Scene(bxy, bt, bf, 60)
        e2, a2 = hgm.match_block(M, [S], p)
        np.testing.assert_array_equal(e, e2)
        np.testing.assert_array_equal(a, a2)
        for mi, mod in enumerate(mods):
            orc = oracle.Oracle(mod.xy, mod.t, mod.f, bxy, bt, bf, 60, K=8, window=1, T=10, **LAM)
            e64, z64, _ = orc.match_block()
            z = a[st.starts[mi]:st.starts[mi + 1]]
            assert np.isfinite(e64) == np.isfinite(e[mi])
            if np.isfinite(e64):
                finite += 1
                assert abs(e[mi] - e64) <= 1e-5 * e64 + 1e-6, (s0, mi, e[mi], e64)
                if not np.array_equal(z, z64):
                    assert orc.energy(z) <= e64 * (1 + 1e-5) + 1e-6
        n_blocks += 1
    assert n_blocks == 7 and finite >= 10


def test_stream_capacity_device_inputs_and_errors(env):
    """Blocks of very different sizes within the capacity fixed at creation (the buffers are never grown),
    device inputs and outputs equal to host ones, a block above the capacity refused with the stream still
    usable afterwards, and an out-of-range frame rejected."""
    torch, hgm, oracle = env
    mods, _ = _long_scene(6, n_models=2)
    M = [hgm.Model(m.xy, m.t, m.f) for m in mods]
    p = hgm.default_params()
    st = hgm.Stream(M, p, 60, max_points=420)
    rng = np.random.default_rng(3)
    pool = np.concatenate([m.centres for m in mods])
    dev = torch.device("cuda")
    for lam in (0.5, 6.0, 1.0):      # about 30, 360 and 60 points per block
        sc = synth.make_scene(rng, 60, (160.0, 120.0), ("poisson", lam), pool, mods, [(0, 12)])
        assert sc.n <= 420
        e, a = st.match(sc.xy, sc.t, sc.f)
        ed = torch.empty(2, dtype=torch.float32, device=dev)
        ad = torch.empty(int(st.starts[-1]), dtype=torch.int32, device=dev)
        st.match(*(torch.from_numpy(x).to(dev) for x in (sc.xy, sc.t, sc.f)), energy=ed, assign=ad)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(e, ed.cpu().numpy())
        np.testing.assert_array_equal(a, ad.cpu().numpy())
        orc = oracle.Oracle(mods[0].xy, mods[0].t, mods[0].f, sc.xy, sc.t, sc.f, 60, K=8, window=1, T=10, **LAM)
        e64, _, _ = orc.match_block()
        assert abs(e[0] - e64) <= 1e-5 * e64 + 1e-6
    big = synth.make_scene(rng, 60, (160.0, 120.0), 8, pool, mods, [])       # 480 points > 420
    with pytest.raises(hgm.HgmError) as err:
        st.match(big.xy, big.t, big.f)
    assert err.value.status == hgm.HGM_EUNSUPPORTED
    e, a = st.match(sc.xy, sc.t, sc.f)            # the last block again: same result after the refusal
    orc = oracle.Oracle(mods[0].xy, mods[0].t, mods[0].f, sc.xy, sc.t, sc.f, 60, K=8, window=1, T=10, **LAM)
    assert abs(e[0] - orc.match_block()[0]) <= 1e-5 * orc.match_block()[0] + 1e-6
    bad_t = np.full(4, 60, np.int32)
    with pytest.raises(hgm.HgmError) as err:
        st.match(np.zeros((4, 2), np.float32), bad_t, np.zeros((4, mods[0].F), np.float32))
    assert err.value.status == hgm.HGM_EINVAL
    st.close()


def test_stream_empty_and_tiny_blocks(env):
    """A block without points has no feasible chain (+inf, rows of -1); a block of two points cannot hold
    a triangle either; the stream stays usable afterwards."""
    torch, hgm, oracle = env
    mods, sc = _long_scene(8, n_models=2, n_frames=60)
    M = [hgm.Model(m.xy, m.t, m.f) for m in mods]
    st = hgm.Stream(M, hgm.default_params(), 60)
    F = mods[0].F
    e, a = st.match(np.zeros((0, 2), np.float32), np.zeros(0, np.int32), np.zeros((0, F), np.float32))
    assert np.all(np.isinf(e)) and np.all(a == -1)
    e, a = st.match(sc.xy[:2], np.array([3, 5], np.int32), sc.f[:2])
    assert np.all(np.isinf(e)) and np.all(a == -1)
    e, a = st.match(sc.xy, sc.t, sc.f)
    orc = oracle.Oracle(mods[0].xy, mods[0].t, mods[0].f, sc.xy, sc.t, sc.f, 60, K=8, window=1, T=10, **LAM)
    e64, _, _ = orc.match_block()
    assert np.isfinite(e64) and abs(e[0] - e64) <= 1e-5 * e64 + 1e-6
    st.close()


def test_stream_full_size_sampled(env):
    """The streaming workload of the benchmark at full size (50 models, a one-minute scene, 60-frame blocks
    every 30 frames), in the benchmark's launch configuration; 12 seeded (block, model) results checked
    against the oracle, and the whole-scene case of Table 2 on 6 seeded models."""
    torch, hgm, oracle = env
    ws = synth.paper_stream()
    dev = torch.device("cuda")
    M = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in ws.models]
    p = hgm.default_params()
    st = hgm.Stream(M, p, 60)
    sc = ws.scenes[0]
    blocks = list(hgm.stream_blocks(sc.xy, sc.t, sc.f, sc.n_frames, 60, 30))
    res = [st.match(bxy, bt, bf) for _, bxy, bt, bf, _ in blocks]
    rng = np.random.default_rng(5)
    for _ in range(12):
        bi, mi = int(rng.integers(len(blocks))), int(rng.integers(len(M)))
        _, bxy, bt, bf, _ = blocks[bi]
        e, a = res[bi]
        mod = ws.models[mi]
        orc = oracle.Oracle(mod.xy, mod.t, mod.f, bxy, bt, bf, 60, K=8, window=1, T=10, **LAM)
        e64, z64, _ = orc.match_block()
        z = a[st.starts[mi]:st.starts[mi + 1]]
        assert np.isfinite(e64) == np.isfinite(e[mi])
        if np.isfinite(e64):
            assert abs(e[mi] - e64) <= 1e-5 * e64 + 1e-6, (bi, mi, e[mi], e64)
            if not np.array_equal(z, z64):
                assert orc.energy(z) <= e64 * (1 + 1e-5) + 1e-6
    st.close()
    ww = synth.paper_whole()
    s0 = ww.scenes[0]
    WM = [hgm.Model(m.xy, m.t, m.f) for m in ww.models]
    S = [hgm.Scene(s0.xy, s0.t, s0.f, s0.n_frames)]
    e, a = hgm.match_block(WM, S, p)
    starts = hgm.block_layout(WM, 1)
    for mi in rng.choice(len(WM), 6, replace=False):
        mod = ww.models[mi]
        orc = oracle.Oracle(mod.xy, mod.t, mod.f, s0.xy, s0.t, s0.f, s0.n_frames, K=8, window=1, T=10, **LAM)
        e64, z64, _ = orc.match_block()
        assert np.isfinite(e64) and abs(e[mi] - e64) <= 1e-5 * e64 + 1e-6, (mi, e[mi], e64)
        z = a[starts[mi]:starts[mi + 1]]
        if not np.array_equal(z, z64):
            assert orc.energy(z) <= e64 * (1 + 1e-5) + 1e-6
