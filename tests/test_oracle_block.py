"""Pins of the oracle's whole-block problem: the paper's own formulation (Sec. 2.2, Sec. 3), where every
scene node is a candidate of every model node and only causality, temporal closeness and distinctness
(Eqs. 7-8) restrict the chain.

Brute-force enumeration of all S^M assignments on tiny instances pins the recursion over the full
domain; the hand-derived examples pin its energy; scene-point permutation leaves the optimum unchanged;
a superset of scene points can only lower the minimum."""
import math

import numpy as np
import pytest

from golden_io import read_examples

LAM = dict(lambda1=0.6, lambda2=0.2, lambda3=5.0)


def _tiny(rng, M, S, n_frames, F=4):
    mt = np.sort(rng.integers(0, max(2, n_frames // 2), M)).astype(np.int32)
    st = rng.integers(0, n_frames, S).astype(np.int32)
    mxy = rng.uniform(0, 10, (M, 2))
    sxy = rng.uniform(0, 10, (S, 2))
    mf = rng.standard_normal((M, F))
    sf = rng.standard_normal((S, F))
    return mxy, mt, mf, sxy, st, sf


@pytest.mark.parametrize("seed", range(24))
def test_block_recursion_is_the_bruteforce_minimum(seed, oracle_mod):
    rng = np.random.default_rng(400 + seed)
    M = int(rng.integers(3, 6))
    S = int(rng.integers(3, 8))
    T = [10, 3, 2, 0][seed % 4]
    mxy, mt, mf, sxy, st, sf = _tiny(rng, M, S, n_frames=int(rng.integers(3, 9)))
    orc = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, int(st.max()) + 1, K=4, window=1, T=T, **LAM)
    e, z, _ = orc.match_block()
    eb, zb, ties = orc.bruteforce_block(tol=1e-9)
    if not np.isfinite(eb):
        assert not np.isfinite(e) and np.all(z == -1)
        return
    assert e == pytest.approx(eb, rel=1e-12, abs=1e-12)
    assert orc.energy(z) == pytest.approx(eb, rel=1e-12, abs=1e-12)
    if ties == 1:
        assert np.array_equal(z, zb)


@pytest.mark.parametrize("name", ["example1", "example2", "example3"])
def test_block_hand_examples(name, oracle_mod):
    """The scene holds exactly the three assigned points at strictly increasing frames, so the
    identity is the only feasible chain of the whole block: the hand-derived energy."""
    ex = read_examples()[name]
    n_frames = int(ex["scene_t"].max()) + 1
    orc = oracle_mod.Oracle(ex["model_xy"], ex["model_t"], ex["model_f"], ex["scene_xy"], ex["scene_t"],
                            ex["scene_f"], n_frames, K=4, window=1, T=10, **LAM)
    e, z, nt = orc.match_block()
    assert e == pytest.approx(ex["energy"], abs=1e-12)
    assert np.array_equal(z, np.arange(len(ex["model_t"])))
    # every increasing triple of the S = M points spans less than T frames: (M-2) * C(S, 3) visits
    M = len(ex["model_t"])
    assert nt == (M - 2) * math.comb(M, 3)


def test_block_scene_permutation_invariance(oracle_mod):
    rng = np.random.default_rng(7)
    mxy, mt, mf, sxy, st, sf = _tiny(rng, 6, 30, n_frames=14)
    o1 = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, 14, K=4, window=1, T=10, **LAM)
    e1, z1, n1 = o1.match_block()
    perm = rng.permutation(30)
    inv = np.argsort(perm)
    o2 = oracle_mod.Oracle(mxy, mt, mf, sxy[perm], st[perm], sf[perm], 14, K=4, window=1, T=10, **LAM)
    e2, z2, n2 = o2.match_block()
    assert np.isfinite(e1)
    assert e2 == pytest.approx(e1, rel=1e-12)
    assert n2 == n1
    # the permuted optimum, mapped back, is an optimum of the original problem
    assert o1.energy(np.where(z2 >= 0, perm[np.maximum(z2, 0)], -1)) == pytest.approx(e1, rel=1e-12)
    del inv


def test_block_superset_lowers_the_minimum(oracle_mod):
    rng = np.random.default_rng(9)
    mxy, mt, mf, sxy, st, sf = _tiny(rng, 7, 40, n_frames=16)
    full = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, 16, K=4, window=1, T=10, **LAM)
    sub = oracle_mod.Oracle(mxy, mt, mf, sxy[:25], st[:25], sf[:25], 16, K=4, window=1, T=10, **LAM)
    ef, _, _ = full.match_block()
    es, zs, _ = sub.match_block()
    assert np.isfinite(es)
    assert ef <= es + 1e-12
    # the subset's optimum is a feasible chain of the full problem with the same energy
    assert full.energy(zs) == pytest.approx(es, rel=1e-12)
