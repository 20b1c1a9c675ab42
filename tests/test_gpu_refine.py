"""The refinement of the pruned form (hgm_params.refine): per (model, scene) pair the `refine` offsets of
lowest pruned energy are solved again without pruning. Checked on a batch of 3 models x 2 scenes: those
offsets carry the unpruned results bit for bit, every other offset the pruned ones, host and device
outputs agree, refine >= the offset count reproduces the unpruned batch, and plans refuse it."""
import numpy as np
import pytest

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


def _batch(hgm, torch):
    wl = synth.batched_exact(seed=41, n_models=3, n_scenes=2, frames_range=(90, 160))
    dev = torch.device("cuda")
    M = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in wl.models]
    S = [hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (s.xy, s.t, s.f)), s.n_frames) for s in wl.scenes]
    return wl, M, S


def _run(torch, hgm, M, S, p, n_e, n_a, device=True):
    if device:
        e = torch.empty(n_e, dtype=torch.float32, device="cuda")
        a = torch.empty(n_a, dtype=torch.int32, device="cuda")
        hgm.match_batch(M, S, p, e, a)
        torch.cuda.synchronize()
        return e.cpu().numpy(), a.cpu().numpy()
    e = np.zeros(n_e, np.float32)
    a = np.zeros(n_a, np.int32)
    hgm.match_batch(M, S, p, e, a)
    return e, a


@pytest.mark.parametrize("precision", [0, 1])
def test_refined_offsets_carry_the_unpruned_results(env, precision):
    torch, hgm = env
    wl, M, S = _batch(hgm, torch)
    prop = hgm.Proposal(162, seed=4)
    base = hgm.default_params(K=64, window=3, precision=precision)
    first, es, as_ = hgm.batch_layout(M, S, base)
    n_e, n_a = int(es[-1]), int(as_[-1])
    e0, a0 = _run(torch, hgm, M, S, base, n_e, n_a)
    pp = hgm.default_params(K=64, window=3, precision=precision, prune=prop, keep=4)
    e1, a1 = _run(torch, hgm, M, S, pp, n_e, n_a)
    r = 5
    pr = hgm.default_params(K=64, window=3, precision=precision, prune=prop, keep=4, refine=r)
    hgm.refine_counter(reset=True)
    e2, a2 = _run(torch, hgm, M, S, pr, n_e, n_a)
    e3, a3 = _run(torch, hgm, M, S, pr, n_e, n_a, device=False)
    np.testing.assert_array_equal(e2, e3)
    np.testing.assert_array_equal(a2, a3)
    refined = 0
    for q in range(len(M) * len(S)):
        mi = q // len(S)
        Mq = wl.models[mi].n
        lo, hi = int(es[q]), int(es[q + 1])
        fin = [k for k in range(lo, hi) if np.isfinite(e1[k])]
        fin.sort(key=lambda k: (e1[k], k))
        chosen = set(fin[:r])
        refined += len(chosen)
        for k in range(lo, hi):
            ka = int(as_[q]) + (k - lo) * Mq
            src_e, src_a = (e0, a0) if k in chosen else (e1, a1)
            assert e2[k] == src_e[k] or (np.isnan(e2[k]) and np.isnan(src_e[k])), (q, k, e2[k], src_e[k])
            np.testing.assert_array_equal(a2[ka:ka + Mq], src_a[ka:ka + Mq])
    assert hgm.refine_counter(reset=True) == 2 * refined


def test_refine_everything_is_the_unpruned_batch(env):
    torch, hgm = env
    wl, M, S = _batch(hgm, torch)
    prop = hgm.Proposal(162, seed=6)
    base = hgm.default_params(K=64, window=3)
    first, es, as_ = hgm.batch_layout(M, S, base)
    n_e, n_a = int(es[-1]), int(as_[-1])
    e0, a0 = _run(torch, hgm, M, S, base, n_e, n_a)
    pr = hgm.default_params(K=64, window=3, prune=prop, keep=3, refine=65535)
    e2, a2 = _run(torch, hgm, M, S, pr, n_e, n_a)
    np.testing.assert_array_equal(e0, e2)
    np.testing.assert_array_equal(a0, a2)


def test_plans_refuse_refine(env):
    torch, hgm = env
    wl, M, S = _batch(hgm, torch)
    prop = hgm.Proposal(162, seed=6)
    pr = hgm.default_params(K=64, window=3, prune=prop, keep=3, refine=4)
    first, es, as_ = hgm.batch_layout(M, S, pr)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    with pytest.raises(hgm.HgmError) as err:
        hgm.Plan(M, S, pr, e, None)
    assert err.value.status == hgm.HGM_EUNSUPPORTED
