"""Plans: a batch laid out once and replayed as a CUDA graph gives the same energies and assignments, bit for
bit, as hgm_match_batch -- exact path, BF16 + pruned path with fallback units, and segmented batches."""
import numpy as np
import pytest

from gpu_util import handles
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


def _batch(torch, hgm, wl):
    ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
    ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
    return ms, ss


def _direct(torch, hgm, ms, ss, p):
    _, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    hgm.match_batch(ms, ss, p, e, a)
    torch.cuda.synchronize()
    return e.cpu().numpy(), a.cpu().numpy()


def _plan_runs(torch, hgm, ms, ss, p, reps=2):
    _, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    plan = hgm.Plan(ms, ss, p, e, a)
    torch.cuda.synchronize()
    out = [(e.cpu().numpy().copy(), a.cpu().numpy().copy())]     # sizing pass
    for _ in range(reps):
        e.fill_(-7.0)
        a.fill_(-7)
        plan.run()
        plan.check()
        out.append((e.cpu().numpy().copy(), a.cpu().numpy().copy()))
    plan.close()
    return out


def _small_workload(seed=14):
    return synth.batched_exact(seed=seed, n_models=3, n_scenes=2, frames_range=(120, 200))


def test_plan_exact_equals_match_batch(env):
    torch, hgm = env
    wl = _small_workload()
    ms, ss = _batch(torch, hgm, wl)
    p = hgm.default_params(K=wl.K, window=wl.window)
    e0, a0 = _direct(torch, hgm, ms, ss, p)
    for e, a in _plan_runs(torch, hgm, ms, ss, p):
        assert np.array_equal(e, e0) and np.array_equal(a, a0)


def test_plan_pruned_with_fallback_equals_match_batch(env):
    """keep = 2 forces fallback units; the replayed graph re-solves them on the device (no host round trip)."""
    torch, hgm = env
    wl = _small_workload(15)
    ms, ss = _batch(torch, hgm, wl)
    prop = hgm.Proposal(162, seed=3)
    p = hgm.default_params(K=wl.K, window=wl.window, precision=1, prune=prop, keep=2)
    hgm.prune_counters(reset=True)
    e0, a0 = _direct(torch, hgm, ms, ss, p)
    n0, fb0 = hgm.prune_counters(reset=True)
    assert fb0 > 0
    runs = _plan_runs(torch, hgm, ms, ss, p, reps=2)
    n1, fb1 = hgm.prune_counters(reset=True)
    assert n1 == 3 * n0 and fb1 == 3 * fb0        # sizing pass + two replays
    for e, a in runs:
        assert np.array_equal(e, e0) and np.array_equal(a, a0)


def test_plan_segmented_equals_match_batch(env):
    torch, hgm = env
    wl = _small_workload(16)
    ms, ss = _batch(torch, hgm, wl)
    p = hgm.default_params(K=wl.K, window=wl.window)
    e0, a0 = _direct(torch, hgm, ms, ss, p)
    hgm.set_workspace_budget(6 << 20)
    try:
        runs = _plan_runs(torch, hgm, ms, ss, p, reps=1)
    finally:
        hgm.set_workspace_budget(0)
    for e, a in runs:
        assert np.array_equal(e, e0) and np.array_equal(a, a0)


def test_plan_sees_new_weights(env):
    """The graph holds the proposal network's device addresses: new weights set between replays are used."""
    torch, hgm = env
    wl = _small_workload(17)
    ms, ss = _batch(torch, hgm, wl)
    prop = hgm.Proposal(162, seed=4)
    p = hgm.default_params(K=wl.K, window=wl.window, prune=prop, keep=3)
    _, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    plan = hgm.Plan(ms, ss, p, e, a)
    other = hgm.Proposal(162, seed=9)
    prop.set(other.get()[0])
    e_ref, a_ref = _direct(torch, hgm, ms, ss, p)
    plan.run()
    plan.check()
    assert np.array_equal(e.cpu().numpy(), e_ref) and np.array_equal(a.cpu().numpy(), a_ref)
    plan.close()


def test_plan_rejects_host_outputs(env):
    torch, hgm = env
    wl = _small_workload(18)
    ms, ss = _batch(torch, hgm, wl)
    p = hgm.default_params(K=wl.K, window=wl.window)
    _, es, as_ = hgm.batch_layout(ms, ss, p)
    with pytest.raises(hgm.HgmError) as err:
        hgm.Plan(ms, ss, p, np.zeros(int(es[-1]), np.float32), None)
    assert err.value.status == hgm.HGM_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_plan_dummy_assignment_equals_match_batch(env, precision):
    """The dummy-assignment recursion recorded in a graph: replays equal the direct call bit for bit."""
    torch, hgm = env
    wl = _small_workload(seed=17)
    ms, ss = _batch(torch, hgm, wl)
    p = hgm.default_params(K=64, window=3, dummy_cost=4.0, precision=precision)
    e0, a0 = _direct(torch, hgm, ms, ss, p)
    assert np.all(np.isfinite(e0)) and np.any(a0 == -2)
    for e, a in _plan_runs(torch, hgm, ms, ss, p):
        np.testing.assert_array_equal(e, e0)
        np.testing.assert_array_equal(a, a0)


def test_calls_on_two_streams_do_not_race(env):
    """Two batches with device outputs issued back to back on different streams share the library's
    workspace; the second waits for the first, so both equal their one-at-a-time results."""
    torch, hgm = env
    wl = _small_workload(seed=19)
    ms, ss = _batch(torch, hgm, wl)
    pa = hgm.default_params(K=64, window=3)
    pb = hgm.default_params(K=24, window=2)
    ea0, aa0 = _direct(torch, hgm, ms, ss, pa)
    eb0, ab0 = _direct(torch, hgm, ms, ss, pb)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for p_, st in ((pa, sa), (pb, sb)):
        _, es, as_ = hgm.batch_layout(ms, ss, p_)
        e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
        a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
        outs.append((e, a))
    for rep in range(3):
        for (e, a), p_, st in zip(outs, (pa, pb), (sa, sb)):
            e.fill_(-1.0)
            a.fill_(-7)
        torch.cuda.synchronize()
        hgm.match_batch(ms, ss, pa, outs[0][0], outs[0][1], stream=sa)
        hgm.match_batch(ms, ss, pb, outs[1][0], outs[1][1], stream=sb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[0][0].cpu().numpy(), ea0)
        np.testing.assert_array_equal(outs[0][1].cpu().numpy(), aa0)
        np.testing.assert_array_equal(outs[1][0].cpu().numpy(), eb0)
        np.testing.assert_array_equal(outs[1][1].cpu().numpy(), ab0)
