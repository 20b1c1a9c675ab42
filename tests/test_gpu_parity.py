"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer work (unary ranking key, candidate lists, triple counts) is compared
bit for bit; energies within 1e-5 relative; assignments equal or a near-tie
(see gpu_util). Inputs are the seeded synthetic workloads of synth.py.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from golden_io import read_examples
from gpu_util import check_offset, handles
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
    import oracle
    oracle.build()
    return torch, hgm, oracle


def _run_match(torch, hgm, m, s, p, n, M):
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    a = torch.empty((n, M), dtype=torch.int32, device="cuda")
    hgm.match(m, s, p, e, a)
    torch.cuda.synchronize()
    return e.cpu().numpy(), a.cpu().numpy()


def _check_all(orc, first, e, a, offsets=None):
    offs = range(len(e)) if offsets is None else offsets
    ties = 0
    for k in offs:
        ok, tie, why = check_offset(orc, first + k, e[k], a[k])
        assert ok, f"offset {first + k}: {why}"
        ties += tie
    return ties


def _c2_pair(seed=21, n_frames=200, lam=30.0):
    rng = np.random.default_rng(seed)
    mod = synth.make_model(rng, 40)
    sc = synth.make_scene(rng, n_frames, (320.0, 240.0), ("poisson", lam), mod.centres, [mod], [(0, 60)])
    return synth.Workload("c2_pair", [mod], [sc], K=64, window=3)


# ---- kernel (a): unary table --------------------------------------------------------

@pytest.mark.parametrize("case", ["single_match", "c2_pair", "odd_F"])
def test_unary_is_the_ranking_key_bit_for_bit(env, case):
    torch, hgm, oracle = env
    if case == "single_match":
        wl = synth.single_match(0)
    elif case == "c2_pair":
        wl = _c2_pair()
    else:
        rng = np.random.default_rng(4)
        mod = synth.make_model(rng, 9, F=7)
        sc = synth.make_scene(rng, 30, (50.0, 50.0), 13, mod.centres, [mod], [(0, 5)])
        wl = synth.Workload("oddF", [mod], [sc], K=8, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    U = torch.empty((mod.n, sc.n), dtype=torch.float32, device="cuda")
    hgm.unary(m, s, 0.6, U)
    torch.cuda.synchronize()
    U = U.cpu().numpy()
    orc = oracle.Oracle.from_workload(wl)
    rng = np.random.default_rng(0)
    pairs = [(i, j) for i in range(mod.n) for j in range(sc.n)]
    if len(pairs) > 4000:
        pairs = [pairs[k] for k in rng.choice(len(pairs), 4000, replace=False)]
    for i, j in pairs:
        assert np.float32(orc.rank_key(i, j)) == U[i, j], (i, j)


# ---- candidate lists --------------------------------------------------------------------

def _check_candidates(env, wl, offsets=None):
    torch, hgm, oracle = env
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T)
    first, n = hgm.offsets(m, s, p)
    orc = oracle.Oracle.from_workload(wl)
    offs = list(range(n)) if offsets is None else offsets
    idx = torch.empty((n, mod.n, wl.K), dtype=torch.int32, device="cuda")
    cnt = torch.empty((n, mod.n), dtype=torch.int32, device="cuda")
    hgm.candidates(m, s, p, first, n, idx, cnt)
    torch.cuda.synchronize()
    idx, cnt = idx.cpu().numpy(), cnt.cpu().numpy()
    for k in offs:
        for i in range(mod.n):
            want, _ = orc.candidates_sorted(i, first + k)
            assert cnt[k, i] == len(want), (k, i)
            assert np.array_equal(idx[k, i, :cnt[k, i]], want), (k, i)
            assert np.all(idx[k, i, cnt[k, i]:] == -1)


def test_candidates_single_match_all_offsets(env):
    _check_candidates(env, synth.single_match(0))


def test_candidates_capped_windows(env):
    wl = _c2_pair()
    _check_candidates(env, wl, offsets=list(range(0, 160, 7)))


def test_candidates_equal_keys_break_ties_by_index(env):
    """Many scene points with identical descriptors: equal FP32 keys, lower index wins."""
    rng = np.random.default_rng(9)
    mod = synth.make_model(rng, 6, F=16, n_clusters=2)
    sc = synth.make_scene(rng, 20, (60.0, 60.0), 12, mod.centres, [mod], [(0, 4)], noise=0.0)
    wl = synth.Workload("ties", [mod], [sc], K=5, window=1)
    _check_candidates(env, wl)


# ---- whole path: unary -> select -> recursion -> backtrack ------------------------------------

def test_match_single_match_all_offsets(env):
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, n = hgm.offsets(m, s, p)
    e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
    orc = oracle.Oracle.from_workload(wl)
    assert (first, n) == (orc.first_offset, orc.n_offsets)
    _check_all(orc, first, e, a)
    # the implant at o = 20 is the best offset and its chain is (mostly) the implant
    k = 20 - first
    assert np.argmin(e) == k or e[k] <= np.min(e) * (1 + 1e-5)
    imp = sc.implants[0].idx
    assert np.mean(a[k] == imp) > 0.5


@pytest.mark.parametrize("name", ["example1", "example2", "example3"])
def test_hand_examples_on_gpu(env, name):
    torch, hgm, oracle = env
    ex = read_examples()[name]
    n_frames = int(ex["scene_t"].max()) + 1
    m = hgm.Model(ex["model_xy"], ex["model_t"], ex["model_f"])
    s = hgm.Scene(ex["scene_xy"], ex["scene_t"], ex["scene_f"], n_frames)
    p = hgm.default_params(K=16, window=20)
    first, n = hgm.offsets(m, s, p)
    e, a = _run_match(torch, hgm, m, s, p, n, len(ex["model_t"]))
    hits = 0
    for k in range(n):
        o = first + k
        if ex["model_t"].min() + o - 20 <= ex["scene_t"].min() and ex["model_t"].max() + o + 20 >= ex["scene_t"].max():
            assert abs(e[k] - ex["energy"]) <= 1e-5 * ex["energy"], (e[k], ex["energy"])
            assert np.array_equal(a[k], np.arange(len(ex["model_t"])))
            hits += 1
    assert hits > 0


@pytest.mark.parametrize("seed", range(24))
def test_tiny_cases_against_bruteforce(env, seed):
    torch, hgm, oracle = env
    rng = np.random.default_rng(500 + seed)
    T = [10, 3, 2, 0][seed % 4]
    wl = synth.tiny_case(seed, M=int(rng.integers(3, 7)), n_frames=int(rng.integers(6, 14)),
                         per_frame=int(rng.integers(1, 4)), K=int(rng.integers(1, 6)), window=int(rng.integers(0, 3)),
                         T=T if T > 0 else 1000)
    wl.T = T
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc)
    p = hgm.default_params(K=wl.K, window=wl.window, T=T)
    first, n = hgm.offsets(m, s, p)
    e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
    orc = oracle.Oracle.from_workload(wl)
    for k in range(n):
        e_bf, z_bf, _ = orc.bruteforce(first + k)
        ok, tie, why = check_offset(orc, first + k, e[k], a[k], e_or=e_bf, z_or=z_bf)
        assert ok, why


def test_gaps_in_the_scene_make_offsets_infeasible(env):
    """Frames without points: windows that see none give +inf and a row of -1."""
    torch, hgm, oracle = env
    rng = np.random.default_rng(3)
    mod = synth.make_model(rng, 5, F=8, t_span=6)
    sc = synth.make_scene(rng, 40, (80.0, 80.0), 3, mod.centres, [mod], [])
    keep = (sc.t % 5) != 2
    sc = synth.Scene(sc.xy[keep], sc.t[keep], sc.f[keep], None, 40, [])
    wl = synth.Workload("gaps", [mod], [sc], K=4, window=0)
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=4, window=0)
    first, n = hgm.offsets(m, s, p)
    e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
    orc = oracle.Oracle.from_workload(wl)
    _check_all(orc, first, e, a)
    assert np.any(~np.isfinite(e)) and np.any(np.isfinite(e))


def test_empty_scene(env):
    torch, hgm, oracle = env
    rng = np.random.default_rng(1)
    mod = synth.make_model(rng, 4, F=8, t_span=5)
    m = hgm.Model(mod.xy, mod.t, mod.f)
    s = hgm.Scene(np.zeros((0, 2), np.float32), np.zeros(0, np.int32), np.zeros((0, 8), np.float32), 20)
    p = hgm.default_params(K=4, window=1)
    first, n = hgm.offsets(m, s, p)
    assert n == 20 - int(mod.t.max() - mod.t.min())
    e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
    assert np.all(np.isinf(e)) and np.all(a == -1)


def test_three_point_model_and_small_caps(env):
    torch, hgm, oracle = env
    rng = np.random.default_rng(12)
    mod = synth.make_model(rng, 3, F=12, t_span=4)
    sc = synth.make_scene(rng, 25, (40.0, 40.0), 4, mod.centres, [mod], [(0, 9)])
    for K in (1, 2, 3, 32, 33, 64):
        wl = synth.Workload("m3", [mod], [sc], K=K, window=2)
        m, s = handles(hgm, mod, sc, torch)
        p = hgm.default_params(K=K, window=2)
        first, n = hgm.offsets(m, s, p)
        e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
        _check_all(oracle.Oracle.from_workload(wl), first, e, a)


def test_closeness_limits(env):
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    mod, sc = wl.models[0], wl.scenes[0]
    for T in (0, 2, 4):
        m, s = handles(hgm, mod, sc, torch)
        p = hgm.default_params(K=wl.K, window=wl.window, T=T)
        first, n = hgm.offsets(m, s, p)
        e, a = _run_match(torch, hgm, m, s, p, n, mod.n)
        _check_all(oracle.Oracle.from_workload(wl, T=T), first, e, a, offsets=range(0, n, 3))


def test_offset_window_and_host_outputs(env):
    """offset_lo/hi restrict the range; host outputs equal device outputs bit for bit."""
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, n = hgm.offsets(m, s, p)
    e_dev, a_dev = _run_match(torch, hgm, m, s, p, n, mod.n)
    p2 = hgm.default_params(K=wl.K, window=wl.window, offset_lo=first + 5, offset_hi=first + 9)
    f2, n2 = hgm.offsets(m, s, p2)
    assert (f2, n2) == (first + 5, 5)
    e_h = np.zeros(n2, np.float32)
    a_h = np.zeros((n2, mod.n), np.int32)
    hgm.match(m, s, p2, e_h, a_h)
    assert np.array_equal(e_h, e_dev[5:10])
    assert np.array_equal(a_h, a_dev[5:10])


def test_count_triples_matches_oracle(env):
    torch, hgm, oracle = env
    wl = synth.single_match(0)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, n = hgm.offsets(m, s, p)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    hgm.count_triples(m, s, p, first, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    _, _, _, nt = oracle.Oracle.from_workload(wl).match_many(threads=8)
    assert np.array_equal(got, nt)


# ---- batches --------------------------------------------------------------------------

def test_batch_equals_single_pairs(env):
    torch, hgm, oracle = env
    wl = synth.batched_exact(seed=5, n_models=3, n_scenes=2, frames_range=(60, 90))
    ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
    ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    hgm.match_batch(ms, ss, p, e, a)
    torch.cuda.synchronize()
    e, a = e.cpu().numpy(), a.cpu().numpy()
    for mi, mod in enumerate(wl.models):
        for si, sc in enumerate(wl.scenes):
            q = mi * len(wl.scenes) + si
            f1, n1 = hgm.offsets(ms[mi], ss[si], p)
            assert f1 == first[q] and n1 == es[q + 1] - es[q]
            e1, a1 = _run_match(torch, hgm, ms[mi], ss[si], p, n1, mod.n)
            assert np.array_equal(e[es[q]:es[q + 1]], e1)
            assert np.array_equal(a[as_[q]:as_[q + 1]].reshape(n1, mod.n), a1)
            orc = oracle.Oracle.from_workload(wl, mi, si)
            _check_all(orc, f1, e1, a1, offsets=range(0, n1, 9))


def test_full_batched_workload_sampled(env):
    """The 10-model x 8-scene workload at full size, in the benchmark's launch configuration
    (one batch call, device outputs), checked on a seeded sample of units."""
    torch, hgm, oracle = env
    wl = synth.batched_exact()
    ms = [hgm.Model(*(torch.from_numpy(a).cuda() for a in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    ss = [hgm.Scene(*(torch.from_numpy(a).cuda() for a in (sc.xy, sc.t, sc.f)), sc.n_frames) for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
    hgm.match_batch(ms, ss, p, e, a)
    torch.cuda.synchronize()
    e, a = e.cpu().numpy(), a.cpu().numpy()
    rng = np.random.default_rng(2024)
    samples = []
    for _ in range(32):
        mi = int(rng.integers(len(wl.models)))
        si = int(rng.integers(len(wl.scenes)))
        q = mi * len(wl.scenes) + si
        n = int(es[q + 1] - es[q])
        k = int(rng.integers(n))
        samples.append((mi, si, q, k))
    # the implants' own offsets are checked too
    for si, sc in enumerate(wl.scenes):
        for imp in sc.implants:
            q = imp.model * len(wl.scenes) + si
            k = imp.offset - int(first[q])
            if 0 <= k < es[q + 1] - es[q]:
                samples.append((imp.model, si, q, k))
    oracles = {}
    for mi, si, q, k in samples:
        if (mi, si) not in oracles:
            oracles[(mi, si)] = oracle.Oracle.from_workload(wl, mi, si)

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
    assert np.all(np.isfinite(e)) or np.any(np.isfinite(e))


def test_accounting_variant_gives_identical_results(env):
    """hgm_profile_enable(2) runs the recursion's accounting variant: same energies and assignments
    bit for bit, and a positive evaluation count no larger than the unpruned loop's."""
    torch, hgm, oracle = env
    wl = synth.batched_exact(seed=7, n_models=2, n_scenes=1, frames_range=(80, 80))
    ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
    ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    outs = []
    for mode in (0, 2):
        e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
        a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
        hgm.profile_evaluated(reset=True)
        hgm.profile_enable(mode)
        hgm.match_batch(ms, ss, p, e, a)
        hgm.profile_enable(0)
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy(), a.cpu().numpy(), hgm.profile_evaluated(reset=True)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ev = outs[1][2]
    full = 0
    for mi, m in enumerate(ms):
        q = mi
        n = int(es[q + 1] - es[q])
        buf = torch.empty(n, dtype=torch.int64, device="cuda")
        hgm.count_triples(m, ss[0], p, int(first[q]), n, buf)
        full += int(buf.sum().item())
    assert 0 < ev, ev
    assert ev < 4 * full, (ev, full)


def test_tile_variants_identical_and_autotune(env, tmp_path, monkeypatch):
    """Every recursion tile variant gives the same energies and assignments bit for bit;
    the autotuner picks one of them and records it in its JSON cache."""
    torch, hgm, oracle = env
    monkeypatch.setenv("HGM_TUNE_CACHE", str(tmp_path / "tune.json"))
    for K, wl in ((64, synth.batched_exact(seed=8, n_models=2, n_scenes=2, frames_range=(70, 90))),
                  (32, synth.single_match(3))):
        ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
        ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
        p = hgm.default_params(K=wl.K, window=wl.window)
        first, es, as_ = hgm.batch_layout(ms, ss, p)
        outs = []
        for v in range(hgm.N_VARIANTS):
            hgm.set_recurse_variant(v)
            e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
            a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
            hgm.match_batch(ms, ss, p, e, a)
            torch.cuda.synchronize()
            outs.append((e.cpu().numpy(), a.cpu().numpy()))
        for e, a in outs[1:]:
            assert np.array_equal(e, outs[0][0]) and np.array_equal(a, outs[0][1])
        best, times = hgm.autotune(ms, ss, p, sample_offsets=16)
        assert 0 <= best < hgm.N_VARIANTS and times is not None and len(times) == hgm.N_VARIANTS
        assert hgm.autotune(ms, ss, p)[0] == best      # served from the cache
    hgm.set_recurse_variant(0)


@pytest.mark.parametrize("precision,prune", [(0, False), (1, False), (0, True)])
def test_segmented_batches_equal_whole_scene_batches(env, precision, prune):
    """A small workspace budget cuts the scenes into offset segments (several unary-table groups, several
    chunks); energies and assignments are bit-identical to the unsegmented run."""
    torch, hgm, oracle = env
    wl = synth.batched_exact(seed=12, n_models=3, n_scenes=2, frames_range=(150, 260))
    ms = [handles(hgm, mod, wl.scenes[0], torch)[0] for mod in wl.models]
    ss = [handles(hgm, wl.models[0], sc, torch)[1] for sc in wl.scenes]
    prop = hgm.Proposal(162, seed=4) if prune else None
    p = hgm.default_params(K=wl.K, window=wl.window, precision=precision, prune=prop)
    first, es, as_ = hgm.batch_layout(ms, ss, p)
    outs = []
    for budget in (0, 6 << 20):
        hgm.set_workspace_budget(budget)
        e = torch.empty(int(es[-1]), dtype=torch.float32, device="cuda")
        a = torch.empty(int(as_[-1]), dtype=torch.int32, device="cuda")
        hgm.match_batch(ms, ss, p, e, a)
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy(), a.cpu().numpy()))
    hgm.set_workspace_budget(0)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("where", ["host", "pinned", "device"])
def test_inputs_from_host_pinned_or_device_give_identical_results(env, where):
    """Handles created from pageable host arrays, pinned host tensors or device tensors (descriptors permuted
    on the device in every case) give bit-identical energies and assignments."""
    torch, hgm, _ = env
    wl = synth.single_match(seed=4)
    mod, sc = wl.models[0], wl.scenes[0]
    p = hgm.default_params(K=wl.K, window=wl.window)
    m0, s0 = handles(hgm, mod, sc)
    _, e0, a0 = hgm.match(m0, s0, p)
    if where == "host":
        m, s = handles(hgm, mod, sc)
    elif where == "pinned":
        pin = lambda a: torch.from_numpy(a).pin_memory()
        m = hgm.Model(pin(mod.xy), pin(mod.t), pin(mod.f))
        s = hgm.Scene(pin(sc.xy), pin(sc.t), pin(sc.f), sc.n_frames)
    else:
        m, s = handles(hgm, mod, sc, torch)
    _, e1, a1 = hgm.match(m, s, p)
    assert np.array_equal(e0, e1) and np.array_equal(a0, a1)
    assert np.array_equal(m.order(), m0.order()) and np.array_equal(s.order(), s0.order())


@pytest.mark.parametrize("on_device", [False, True])
def test_non_finite_descriptors_are_rejected(env, on_device):
    torch, hgm, _ = env
    wl = synth.single_match(seed=5)
    mod, sc = wl.models[0], wl.scenes[0]
    mf = mod.f.copy()
    mf[2, 7] = np.nan
    sf = sc.f.copy()
    sf[sc.n // 2, 100] = np.inf
    conv = (lambda a: torch.from_numpy(a).cuda()) if on_device else (lambda a: a)
    with pytest.raises(hgm.HgmError) as err:
        hgm.Model(conv(mod.xy), conv(mod.t), conv(mf))
    assert err.value.status == hgm.HGM_EINVAL and "non-finite model descriptor" in str(err.value)
    with pytest.raises(hgm.HgmError) as err:
        hgm.Scene(conv(sc.xy), conv(sc.t), conv(sf), sc.n_frames)
    assert err.value.status == hgm.HGM_EINVAL and "non-finite scene descriptor" in str(err.value)
    # the library stays usable
    m, s = handles(hgm, mod, sc)
    first, e, a = hgm.match(m, s, hgm.default_params(K=wl.K, window=wl.window))
    assert np.isfinite(e).any()


@pytest.mark.parametrize("K", [8, 64])
def test_coincident_points_follow_the_atan2_reading(env, K):
    """Points with identical positions (zero-length edges: atan2(0, 0) = 0, reading R1) -- clutter copies on
    top of implanted points and a model with repeated positions -- give the oracle's energies on every
    offset (K = 8: the short-list kernel; K = 64: the main kernel)."""
    torch, hgm, oracle = env
    rng = np.random.default_rng(31)
    mod = synth.make_model(rng, 12, frame=(40.0, 30.0))
    mod.xy[3] = mod.xy[1]
    mod.xy[7] = mod.xy[6]
    sc = synth.make_scene(rng, 40, (40.0, 30.0), 4, mod.centres, [mod], [(0, 9)], translate=False, xy_jitter=0.0,
                          t_jitter=0.0)
    imp = sc.implants[0].idx
    extra_xy = sc.xy[imp[::2]].copy()                       # clutter exactly on implant points, same frames
    extra_t = sc.t[imp[::2]].copy()
    extra_f = sc.f[imp[::2]] + 0.5 * rng.standard_normal((len(imp[::2]), sc.F)).astype(np.float32)
    sc = synth.Scene(np.concatenate([sc.xy, extra_xy]), np.concatenate([sc.t, extra_t]),
                     np.concatenate([sc.f, extra_f]).astype(np.float32), None, sc.n_frames, sc.implants)
    wl = synth.Workload("coincident", [mod], [sc], K=K, window=1)
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=wl.K, window=wl.window)
    first, e, a = hgm.match(m, s, p)
    orc = oracle.Oracle.from_workload(wl)
    for k in range(len(e)):
        e64, z64, _ = orc.match(first + k)
        assert np.isfinite(e64) == np.isfinite(e[k])
        if np.isfinite(e64):
            assert abs(e[k] - e64) <= 1e-5 * e64 + 1e-6, (k, e[k], e64)
            assert np.array_equal(a[k], z64) or orc.energy(a[k]) <= e64 * (1 + 1e-5) + 1e-6
