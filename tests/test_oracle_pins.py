"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: hand-derived closed forms
(tests/golden/hand_examples.txt), brute-force enumeration, invariances of
the optimum (scene permutation, similarity transforms, time shift, mirror
symmetry), an independent angle computation (acos + cross-product sign),
and the exact zero of a noise-free implant.
"""
import itertools
import math

import numpy as np
import pytest

from golden_io import read_examples
from paper_1505_00581_gb300 import synth

LAM = dict(lambda1=0.6, lambda2=0.2, lambda3=5.0)


def _oracle_for(ex, oracle_mod, window=20, K=16, T=10):
    n_frames = int(ex["scene_t"].max()) + 1
    return oracle_mod.Oracle(ex["model_xy"], ex["model_t"], ex["model_f"], ex["scene_xy"], ex["scene_t"],
                             ex["scene_f"], n_frames, K=K, window=window, T=T, **LAM)


@pytest.mark.parametrize("name", ["example1", "example2", "example3"])
def test_hand_examples_energy(name, oracle_mod):
    ex = read_examples()[name]
    orc = _oracle_for(ex, oracle_mod)
    ident = np.arange(len(ex["model_t"]))
    assert orc.energy(ident) == pytest.approx(ex["energy"], rel=0, abs=1e-12)


@pytest.mark.parametrize("name", ["example1", "example2", "example3"])
def test_hand_examples_recursion(name, oracle_mod):
    """The scene points carry strictly increasing frames, so the only feasible chain is
    the identity; the recursion must reach it with the hand-derived energy at every
    offset whose windows see all scene points."""
    ex = read_examples()[name]
    orc = _oracle_for(ex, oracle_mod)
    ident = np.arange(len(ex["model_t"]))
    hits = 0
    for o in orc.offsets():
        e, z, _ = orc.match(int(o))
        lo = ex["model_t"].min() + o - 20
        hi = ex["model_t"].max() + o + 20
        if lo <= ex["scene_t"].min() and hi >= ex["scene_t"].max():
            assert e == pytest.approx(ex["energy"], abs=1e-12)
            assert np.array_equal(z, ident)
            hits += 1
    assert hits > 0


def _angle_acos(v, p, q):
    """Signed angle at v from v->p to v->q via acos of the normalised dot product and
    the sign of the cross product (a different route from directions + wrap)."""
    u = np.asarray(p, float) - np.asarray(v, float)
    w = np.asarray(q, float) - np.asarray(v, float)
    cosang = float(np.dot(u, w) / (np.linalg.norm(u) * np.linalg.norm(w)))
    ang = math.acos(max(-1.0, min(1.0, cosang)))
    cross = u[0] * w[1] - u[1] * w[0]
    return ang if cross >= 0 else -ang


def test_geometry_term_against_independent_angles(oracle_mod):
    """D^g (Eq. 6) from or_geo vs angles computed by acos/cross on random triangles."""
    rng = np.random.default_rng(7)
    for trial in range(200):
        mxy = rng.uniform(-50, 50, size=(3, 2))
        sxy = rng.uniform(-50, 50, size=(3, 2))
        orc = oracle_mod.Oracle(mxy, np.array([0, 1, 2]), np.zeros((3, 2)), sxy, np.array([0, 1, 2]),
                                np.zeros((3, 2)), 3, K=3, window=5, **LAM)
        # triangle (i, j, k) = model points (2, 1, 0); scene (a, b, c) = (2, 1, 0)
        am1 = _angle_acos(mxy[1], mxy[2], mxy[0])
        as1 = _angle_acos(sxy[1], sxy[2], sxy[0])
        am2 = _angle_acos(mxy[2], mxy[1], mxy[0])
        as2 = _angle_acos(sxy[2], sxy[1], sxy[0])

        def circ(d):
            d = abs(d) % (2 * math.pi)
            return min(d, 2 * math.pi - d)
        expect = math.hypot(circ(am1 - as1), circ(am2 - as2))
        got = orc.lib.or_geo(orc.ctx, 2, 2, 1, 0)
        assert got == pytest.approx(expect, abs=1e-9), trial


def _tiny_oracle(seed, oracle_mod, T=10, lambda2=0.2, **kw):
    rng = np.random.default_rng(1000 + seed)
    M = int(rng.integers(3, 7))
    per_frame = int(rng.integers(1, 4))
    n_frames = int(rng.integers(6, 14))
    K = int(rng.integers(2, 6))
    window = int(rng.integers(0, 3))
    wl = synth.tiny_case(seed, M=M, n_frames=n_frames, per_frame=per_frame, K=K, window=window,
                         T=T if T > 0 else 1000)
    return oracle_mod.Oracle.from_workload(wl, T=T, lambda2=lambda2, **kw)


def _count_feasible_triples(orc, o):
    """Feasible (z_i, z_{i-1}, z_{i-2}) triples over all steps, enumerated directly."""
    n = 0
    lists = [orc.candidates_sorted(i, o)[0] for i in range(orc.M)]
    st = orc._st
    for i in range(2, orc.M):
        for a, b, c in itertools.product(lists[i], lists[i - 1], lists[i - 2]):
            if len({a, b, c}) < 3:
                continue
            if not (st[c] <= st[b] <= st[a]):
                continue
            if orc.T > 0 and not (st[a] - st[c] < orc.T):
                continue
            n += 1
    return n


@pytest.mark.parametrize("seed", range(40))
def test_recursion_equals_bruteforce(seed, oracle_mod):
    """Eqs. 10-13 reach the global minimum of Eq. 9 over the candidate product (exactness)."""
    T = [10, 3, 2, 0][seed % 4]   # 0 = no closeness limit
    orc = _tiny_oracle(seed, oracle_mod, T=T)
    for o in orc.offsets():
        e_rec, z_rec, ntrip = orc.match(int(o))
        e_bf, z_bf, nties = orc.bruteforce(int(o), tol=1e-9)
        if math.isinf(e_bf):
            assert math.isinf(e_rec)
            assert np.all(z_rec == -1)
        else:
            assert e_rec == pytest.approx(e_bf, rel=1e-12, abs=1e-12)
            assert orc.energy(z_rec) == pytest.approx(e_bf, rel=1e-12, abs=1e-12)
            if nties == 1:
                assert np.array_equal(z_rec, z_bf)
        assert ntrip == _count_feasible_triples(orc, int(o))


@pytest.mark.parametrize("seed", range(10))
def test_no_geometry_reduces_to_unary_chain(seed, oracle_mod):
    """lambda2 = 0 and no closeness limit: E* = min sum of U over chains obeying only
    causality and distinctness, checked by a direct product enumeration."""
    orc = _tiny_oracle(seed, oracle_mod, T=0, lambda2=0.0)
    st = orc._st
    for o in orc.offsets():
        lists = [orc.candidates_sorted(i, int(o)) for i in range(orc.M)]
        best = math.inf
        for combo in itertools.product(*[range(len(l[0])) for l in lists]):
            z = [lists[i][0][combo[i]] for i in range(orc.M)]
            ok = all(len({z[i], z[i - 1], z[i - 2]}) == 3 and st[z[i - 2]] <= st[z[i - 1]] <= st[z[i]]
                     for i in range(2, orc.M))
            if ok:
                best = min(best, sum(lists[i][1][combo[i]] for i in range(orc.M)))
        e, _, _ = orc.match(int(o))
        if math.isinf(best):
            assert math.isinf(e)
        else:
            assert e == pytest.approx(best, rel=1e-12)


def _small_workload(seed=3):
    rng = np.random.default_rng(seed)
    mod = synth.make_model(rng, 8, F=16)
    sc = synth.make_scene(rng, 40, (160.0, 120.0), 4, mod.centres, [mod], [(0, 12)], translate=False)
    return synth.Workload("small", [mod], [sc], K=8, window=2)


def _all(orc):
    offs, e, a, _ = orc.match_many(threads=4)
    return offs, e, a


def test_scene_permutation_invariance(oracle_mod):
    wl = _small_workload()
    sc = wl.scenes[0]
    o1 = oracle_mod.Oracle.from_workload(wl)
    offs, e1, a1 = _all(o1)
    perm = np.random.default_rng(5).permutation(sc.n)
    o2 = oracle_mod.Oracle(wl.models[0].xy, wl.models[0].t, wl.models[0].f, sc.xy[perm], sc.t[perm],
                           sc.f[perm], sc.n_frames, K=wl.K, window=wl.window)
    _, e2, a2 = _all(o2)
    assert np.allclose(e1, e2, rtol=1e-12, atol=0) or np.array_equal(e1, e2)
    fin = np.isfinite(e1)
    assert fin.sum() > 0
    # caller indices map through the permutation: perm[a2] is an index of the original scene
    mapped = np.where(a2 >= 0, perm[np.maximum(a2, 0)], -1)
    assert np.array_equal(mapped[fin], a1[fin])


def test_similarity_transform_invariance(oracle_mod):
    """Rotating, scaling and translating the scene's xy leaves every optimum unchanged."""
    wl = _small_workload()
    sc, mod = wl.scenes[0], wl.models[0]
    o1 = oracle_mod.Oracle.from_workload(wl)
    _, e1, a1 = _all(o1)
    th, s, shift = 0.7, 2.5, np.array([13.0, -40.0])
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    xy2 = (sc.xy.astype(np.float64) @ R.T) * s + shift
    o2 = oracle_mod.Oracle(mod.xy, mod.t, mod.f, xy2, sc.t, sc.f, sc.n_frames, K=wl.K, window=wl.window)
    _, e2, a2 = _all(o2)
    fin = np.isfinite(e1)
    assert np.array_equal(fin, np.isfinite(e2))
    assert np.allclose(e1[fin], e2[fin], rtol=1e-10, atol=1e-10)
    assert np.array_equal(a1[fin], a2[fin])


def test_mirror_invariance(oracle_mod):
    """Mirroring model and scene together flips every signed angle: optimum unchanged."""
    wl = _small_workload()
    sc, mod = wl.scenes[0], wl.models[0]
    o1 = oracle_mod.Oracle.from_workload(wl)
    _, e1, a1 = _all(o1)
    flip = np.array([-1.0, 1.0])
    o2 = oracle_mod.Oracle(mod.xy * flip, mod.t, mod.f, sc.xy * flip, sc.t, sc.f, sc.n_frames, K=wl.K,
                           window=wl.window)
    _, e2, a2 = _all(o2)
    fin = np.isfinite(e1)
    assert np.allclose(e1[fin], e2[fin], rtol=1e-10, atol=1e-10)
    assert np.array_equal(a1[fin], a2[fin])


def test_mirror_scene_only_changes_energy(oracle_mod):
    """Signed reading: mirroring only the scene changes the optimum at the implant offset."""
    wl = _small_workload()
    sc, mod = wl.scenes[0], wl.models[0]
    o1 = oracle_mod.Oracle.from_workload(wl)
    o2 = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy * np.array([-1.0, 1.0]), sc.t, sc.f, sc.n_frames,
                           K=wl.K, window=wl.window)
    e1, _, _ = o1.match(12)
    e2, _, _ = o2.match(12)
    assert e2 > e1 + 0.1


def test_time_shift_equivariance(oracle_mod):
    """Delaying every scene frame by d shifts the offsets by d and nothing else."""
    wl = _small_workload()
    sc, mod = wl.scenes[0], wl.models[0]
    o1 = oracle_mod.Oracle.from_workload(wl)
    offs1, e1, a1 = _all(o1)
    d = 7
    o2 = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t + d, sc.f, sc.n_frames + d, K=wl.K,
                           window=wl.window)
    offs2, e2, a2 = _all(o2)
    k = np.searchsorted(offs2, offs1 + d)
    assert np.array_equal(offs2[k], offs1 + d)
    fin = np.isfinite(e1)
    assert np.array_equal(e1[fin], e2[k][fin])
    assert np.array_equal(a1[fin], a2[k][fin])


def test_noise_free_implant_has_zero_energy(oracle_mod):
    """An exact copy of the model (same xy, descriptors, frames + o) gives E* = 0 at o."""
    rng = np.random.default_rng(11)
    mod = synth.make_model(rng, 12, F=24)
    sc = synth.make_scene(rng, 50, (160.0, 120.0), 5, mod.centres, [mod], [(0, 17)], translate=False,
                          xy_jitter=0.0, t_jitter=0.0, f_noise=0.0)
    wl = synth.Workload("clean", [mod], [sc], K=64, window=1)
    orc = oracle_mod.Oracle.from_workload(wl)
    e, z, _ = orc.match(17)
    assert e == pytest.approx(0.0, abs=1e-9)
    imp = sc.implants[0].idx
    # zero-energy chains must reproduce the implant frame by frame; with several model
    # points per frame the order of equal-frame points is the only freedom
    assert orc.energy(z) == pytest.approx(0.0, abs=1e-9)
    assert np.array_equal(np.sort(sc.t[z]), np.sort(sc.t[imp]))
    # offsets within +-w of the implant still see every implant point (Delta only uses
    # frame differences), further ones cannot reach a zero-energy chain
    for o in orc.offsets():
        if abs(o - 17) > wl.window:
            assert orc.match(int(o))[0] > 1e-3
        else:
            assert orc.match(int(o))[0] == pytest.approx(0.0, abs=1e-9)


def test_candidates_window_and_cap(oracle_mod):
    """C_i(o): the K smallest FP64 distances among the window's points, in index order
    (checked where the K-th and (K+1)-th distances are well separated)."""
    wl = synth.single_match(0)
    orc = oracle_mod.Oracle.from_workload(wl)
    st, sf, mf = orc._st, orc._sf, orc._mf
    checked = 0
    for o in orc.offsets()[::3]:
        for i in range(orc.M):
            lo, hi = orc._mt[i] + o - wl.window, orc._mt[i] + o + wl.window
            inwin = np.nonzero((st >= lo) & (st <= hi))[0]
            u = 0.6 * np.sqrt(((sf[inwin] - mf[i]) ** 2).sum(axis=1))
            idx, uc = orc.candidates_sorted(i, int(o))
            if len(inwin) <= wl.K:
                assert np.array_equal(idx, inwin)
            else:
                srt = np.sort(u)
                if srt[wl.K] - srt[wl.K - 1] < 1e-4:
                    continue
                expect = np.sort(inwin[np.argsort(u, kind="stable")[:wl.K]])
                assert np.array_equal(idx, expect)
            assert np.allclose(uc, 0.6 * np.sqrt(((sf[idx] - mf[i]) ** 2).sum(axis=1)), rtol=1e-12)
            checked += 1
    assert checked > 100


def test_rank_key_is_fp32_distance(oracle_mod):
    """The FP32 ranking key equals the distance within the FP32 summation error bound."""
    wl = synth.single_match(0)
    orc = oracle_mod.Oracle.from_workload(wl)
    F = orc.F
    for i in range(orc.M):
        for j in range(0, orc.S, 37):
            u = orc.unary(i, j)
            k = orc.rank_key(i, j)
            assert abs(k - u) <= (F + 4) * 2.0 ** -24 * u + 1e-30
