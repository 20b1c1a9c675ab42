"""hgm_match_noalloc: the match entry point for callers that may not allocate device memory
while running (real-time loops that cannot take cudaMalloc's device-wide synchronisation,
frameworks that reserve all GPU memory up front). It must give hgm_match's result from its
fixed scratch array, on repeated calls, and refuse pairs whose unary table does not fit.

This file is named to be collected last; it creates its own handles, so it passes alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from gpu_util import energy_ok
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
    return torch, hgm


def _handles(hgm, torch, mod, sc):
    m = hgm.Model(*(torch.from_numpy(a).cuda() for a in (mod.xy, mod.t, mod.f)))
    s = hgm.Scene(*(torch.from_numpy(a).cuda() for a in (sc.xy, sc.t, sc.f)), sc.n_frames)
    return m, s


def _compare(torch, hgm, wl):
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = _handles(hgm, torch, mod, sc)
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T)
    first, n = hgm.offsets(m, s, p)
    e_ref = torch.empty(n, dtype=torch.float32, device="cuda")
    a_ref = torch.empty((n, mod.n), dtype=torch.int32, device="cuda")
    hgm.match(m, s, p, e_ref, a_ref)
    torch.cuda.synchronize()
    e_ref, a_ref = e_ref.cpu().numpy(), a_ref.cpu().numpy()
    for call in range(2):   # two calls in a row: the shared scratch keeps the previous call's contents
        e = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
        a = torch.full((n, mod.n), -7, dtype=torch.int32, device="cuda")
        hgm.match_noalloc(m, s, p, e, a)
        torch.cuda.synchronize()
        e, a = e.cpu().numpy(), a.cpu().numpy()
        for k in range(n):
            assert energy_ok(e[k], float(e_ref[k])), (call, k, e[k], e_ref[k])
        assert np.array_equal(a, a_ref), call


def test_noalloc_equals_match_single_match(env):
    torch, hgm = env
    _compare(torch, hgm, synth.single_match(0))


def test_noalloc_equals_match_in_several_chunks(env):
    """About 2,000 offsets at K = 64: the argmin tables exceed the scratch, so offsets run in chunks."""
    torch, hgm = env
    rng = np.random.default_rng(77)
    mod = synth.make_model(rng, 40)
    sc = synth.make_scene(rng, 2000, (320.0, 240.0), ("poisson", 30.0), mod.centres, [mod], [(0, 700)])
    _compare(torch, hgm, synth.Workload("chunks", [mod], [sc], K=64, window=3))


def test_noalloc_rejects_a_unary_table_beyond_the_scratch(env):
    torch, hgm = env
    rng = np.random.default_rng(5)
    mod = synth.make_model(rng, 64, F=8)
    sc = synth.make_scene(rng, 3000, (320.0, 240.0), 100, mod.centres, [mod], [])   # 300k points: 64x300k floats
    m, s = _handles(hgm, torch, mod, sc)
    p = hgm.default_params(K=64, window=3)
    first, n = hgm.offsets(m, s, p)
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    a = torch.empty((n, mod.n), dtype=torch.int32, device="cuda")
    with pytest.raises(hgm.HgmError) as err:
        hgm.match_noalloc(m, s, p, e, a)
    assert err.value.status == hgm.HGM_EUNSUPPORTED
    assert "scratch" in str(err.value)


@pytest.mark.parametrize("option", ["precision", "dummy_cost", "prune", "refine", "inf_lambda"])
def test_noalloc_refuses_what_it_leaves_out(env, option):
    """Parameters are checked as hgm_match checks them (an infinite lambda is invalid); the valid options this
    entry point does not implement are refused with HGM_EUNSUPPORTED instead of being ignored."""
    torch, hgm = env
    wl = synth.single_match(0)
    m, s = _handles(hgm, torch, wl.models[0], wl.scenes[0])
    over = {"precision": dict(precision=1), "dummy_cost": dict(dummy_cost=4.0),
            "refine": dict(refine=4), "inf_lambda": dict(lambda1=float("inf"))}.get(option, {})
    prop = None
    if option == "prune":
        prop = hgm.Proposal(wl.models[0].F, seed=3)
        over = dict(prune=prop)
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T, **over)
    first, n = hgm.offsets(m, s, hgm.default_params(K=wl.K, window=wl.window, T=wl.T))
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    a = torch.empty((n, wl.models[0].n), dtype=torch.int32, device="cuda")
    with pytest.raises(hgm.HgmError) as err:
        hgm.match_noalloc(m, s, p, e, a)
    want = hgm.HGM_EINVAL if option == "inf_lambda" else hgm.HGM_EUNSUPPORTED
    assert err.value.status == want, str(err.value)
    if prop is not None:
        prop.close()
