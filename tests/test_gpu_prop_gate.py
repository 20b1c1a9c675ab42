"""What the learned pruning gains, and the quality bar read at the level recognition uses.

The network (trained as the benchmark trains it: 2,000 steps of 4,096 pairs labelled by the exact recursion
on separately seeded scenes) is compared with the same cut made without it -- the window's smallest unary
costs, K = keep -- on the 10-model x 8-scene batched workload, both in the BF16 + FP32 re-score mode and
against this run's exact FP32 results.

* Per offset, at the keep the learned stage is specified with (8 of 64), the network keeps the exact
  optimum's candidate more often than the unary cut (point recall), and neither cut reaches the per-offset
  bar of 99% recall: on offsets whose windows hold only clutter the optimum is a chain among near-equal
  ones, decided by time order and geometry, not by one candidate's features. (From keep 12 on, the unary
  cut keeps it as often or more: the network's gain is in the first few places of its ranking.)
* Per (model, scene) pair -- the matching distance recognition uses is the minimum over offsets -- keep 12
  with the 32 offsets of lowest pruned energy re-solved unpruned meets the bar: recall of the exact best
  assignment >= 0.99 and mean relative gap of the pair minimum <= 1e-3, faster than the exact path.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1505_00581_gb300 import build, hgm, prop_train, synth
    build.build()
    hgm.load()
    wl = synth.batched_exact()
    dev = torch.device("cuda")
    ms = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in wl.models]
    ss = [hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (s.xy, s.t, s.f)), s.n_frames) for s in wl.scenes]
    p = hgm.default_params(K=64, window=3)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    hgm.match_batch(ms, ss, p, e, a)
    torch.cuda.synchronize()
    ref = (e.cpu().numpy(), a.cpu().numpy())
    prop, _ = prop_train.train_default(torch, wl, steps=2000, seed=101)
    M_rows, e_rows = [], []
    for mi, m in enumerate(wl.models):
        for si in range(len(wl.scenes)):
            q = mi * len(wl.scenes) + si
            M_rows.append((int(as_[q]), int(es[q + 1] - es[q]), m.n))
            e_rows.append(int(es[q]))
    yield dict(torch=torch, hgm=hgm, prop_train=prop_train, wl=wl, ms=ms, ss=ss, ref=ref, prop=prop, e=e, a=a,
               M_rows=M_rows, e_rows=e_rows, dev=dev)
    prop.close()


def _timed(env, p, out_e, out_a, reps=3):
    torch, hgm = env["torch"], env["hgm"]
    hgm.match_batch(env["ms"], env["ss"], p, out_e, out_a)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        hgm.match_batch(env["ms"], env["ss"], p, out_e, out_a)
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def _quality(env, e, a):
    return env["prop_train"].compare(*env["ref"], e.cpu().numpy(), a.cpu().numpy(), env["M_rows"], env["e_rows"])


@pytest.mark.parametrize("keep", [8])
def test_network_keeps_the_optimum_more_often_than_the_unary_cut(env, keep):
    torch, hgm = env["torch"], env["hgm"]
    pn = hgm.default_params(K=64, window=3, precision=1, prune=env["prop"], keep=keep)
    hgm.match_batch(env["ms"], env["ss"], pn, env["e"], env["a"])
    torch.cuda.synchronize()
    qn = _quality(env, env["e"], env["a"])
    pu = hgm.default_params(K=keep, window=3, precision=1)
    _, es, as_ = hgm.batch_layout(env["ms"], env["ss"], pu)
    eu = torch.empty(int(es[-1]), dtype=torch.float32, device=env["dev"])
    au = torch.empty(int(as_[-1]), dtype=torch.int32, device=env["dev"])
    hgm.match_batch(env["ms"], env["ss"], pu, eu, au)
    torch.cuda.synchronize()
    qu = _quality(env, eu, au)
    print(f"keep {keep}: network recall {qn['point_recall']:.3f} gap {qn['mean_rel_gap']:.4f} | unary cut recall "
          f"{qu['point_recall']:.3f} gap {qu['mean_rel_gap']:.4f} infeasible {qu['feasible_mismatch']}")
    assert qn["feasible_mismatch"] == 0                      # the exact fallback: never infeasible where exact is not
    assert qn["point_recall"] >= qu["point_recall"] + 0.03
    assert qn["point_recall"] < 0.99                         # the per-offset bar is not met by a top-k cut


def test_pair_level_bar_with_refinement(env):
    torch, hgm = env["torch"], env["hgm"]
    p0 = hgm.default_params(K=64, window=3)
    ms_exact = _timed(env, p0, env["e"], env["a"])
    pr = hgm.default_params(K=64, window=3, precision=1, prune=env["prop"], keep=12, refine=32)
    ms_ref = _timed(env, pr, env["e"], env["a"])
    q = _quality(env, env["e"], env["a"])["pairs"]
    print(f"exact {ms_exact:.1f} ms, keep 12 + refine 32 {ms_ref:.1f} ms; pairs {q}")
    assert q["point_recall_at_best"] >= 0.99
    assert q["mean_rel_gap"] <= 1e-3
    assert ms_ref < ms_exact
