"""Pins of the oracle's dummy assignment (Eq. 2, reading R5): every list gets the extra candidate eps
with U = W^d; a term involving eps vanishes; a triple holding eps is feasible iff its real points are
distinct, time-ordered and closer than T.

Brute-force enumeration with eps in every list pins the recursion; closed forms pin the energy (the
all-eps chain costs M lambda1 W^d; W^d = 0 makes 0 the minimum; a hand-worked 3-point chain with one
model point absent); a W^d above any real chain's energy reproduces the problem without dummies."""
import numpy as np
import pytest

from paper_1505_00581_gb300 import synth

LAM = dict(lambda1=0.6, lambda2=0.2, lambda3=5.0)
EPS = -2


@pytest.mark.parametrize("seed", range(30))
def test_dummy_recursion_is_the_bruteforce_minimum(seed, oracle_mod):
    wl = synth.tiny_case(700 + seed, M=4 + seed % 2, n_frames=9, per_frame=2, K=3, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    wd = [0.5, 2.0, 5.0, 12.0][seed % 4]
    T = [10, 3, 2][seed % 3]
    orc = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=3, window=1, T=T,
                            dummy_cost=wd, **LAM)
    for o in orc.offsets()[:4]:
        e, z, _ = orc.match(int(o))
        eb, zb, ties = orc.bruteforce(int(o), tol=1e-9)
        assert np.isfinite(e) and np.isfinite(eb)          # the all-eps chain is always feasible
        assert e == pytest.approx(eb, rel=1e-12, abs=1e-12)
        assert orc.energy(z) == pytest.approx(eb, rel=1e-12, abs=1e-12)
        if ties == 1:
            assert np.array_equal(z, zb)


def test_all_eps_chain_energy_and_zero_cost(oracle_mod):
    wl = synth.tiny_case(5, M=6, n_frames=12, per_frame=3, K=4, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    wd = 1.7
    orc = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=4, window=1,
                            dummy_cost=wd, **LAM)
    assert orc.energy(np.full(mod.n, EPS)) == pytest.approx(mod.n * LAM["lambda1"] * wd, rel=1e-15)
    zero = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=4, window=1,
                             dummy_cost=0.0, **LAM)
    for o in zero.offsets():
        e, z, _ = zero.match(int(o))
        assert e == 0.0                                    # no chain costs less than nothing
        assert zero.energy(z) == 0.0


def test_hand_worked_missing_point(oracle_mod):
    """Model (0,0,t0), (4,0,t1), (4,3,t2) with f = (0,0), (1,0), (0,1); the scene holds only the first
    two points' matches, at frames 5 and 6 with f' = (0,0), (1,0), plus nothing near model point 3.
    With z = (p0, p1, eps): U = 0 + 0 + W^d; the one triple (3,2,1) keeps only Delta(2,1) = |1 - 1| = 0;
    E = lambda1 W^d. Any real third point would cost more, so that chain is the optimum."""
    mxy = np.array([[0, 0], [4, 0], [4, 3]], np.float32)
    mt = np.array([0, 1, 2], np.int32)
    mf = np.array([[0, 0], [1, 0], [0, 1]], np.float32)
    sxy = np.array([[10, 10], [14, 10]], np.float32)
    st = np.array([5, 6], np.int32)
    sf = np.array([[0, 0], [1, 0]], np.float32)
    wd = 0.4
    orc = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, 10, K=4, window=3, T=10, dummy_cost=wd, **LAM)
    e, z, _ = orc.match(5)
    assert e == pytest.approx(LAM["lambda1"] * wd, abs=1e-15)
    assert list(z) == [0, 1, EPS]
    # the same chain with the dummy on the middle point: the triple keeps no Delta (both touch eps),
    # U = 0 + W^d + |(0,1) - (1,0)| = W^d + sqrt(2); z = (p0, eps, p1) is feasible (p1 after p0)
    e2 = orc.energy(np.array([0, EPS, 1]))
    assert e2 == pytest.approx(LAM["lambda1"] * (wd + np.sqrt(2.0)), abs=1e-12)
    # without a dummy the offset is infeasible: model point 3 has no candidate it can take
    plain = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, 10, K=4, window=3, T=10, **LAM)
    assert plain.match(5)[0] == float("inf")


def test_expensive_dummy_is_the_plain_problem(oracle_mod):
    wl = synth.tiny_case(17, M=6, n_frames=14, per_frame=3, K=4, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    plain = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=4, window=1, **LAM)
    dear = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, K=4, window=1,
                             dummy_cost=1e6, **LAM)
    hits = 0
    for o in plain.offsets():
        e0, z0, _ = plain.match(int(o))
        e1, z1, _ = dear.match(int(o))
        if np.isfinite(e0):
            hits += 1
            assert e1 == pytest.approx(e0, rel=1e-12)
            assert np.array_equal(z0, z1)
        else:
            assert np.any(z1 == EPS) and e1 >= 1e6 * LAM["lambda1"]
    assert hits > 0


def test_eps_feasibility_rule(oracle_mod):
    """Triples with eps: real points distinct, in time order (newest first) and within T."""
    mxy = np.zeros((3, 2), np.float32)
    mt = np.array([0, 1, 2], np.int32)
    mf = np.zeros((3, 2), np.float32)
    sxy = np.array([[0, 0], [1, 0], [2, 0]], np.float32)
    st = np.array([0, 3, 20], np.int32)
    sf = np.zeros((3, 2), np.float32)
    orc = oracle_mod.Oracle(mxy, mt, mf, sxy, st, sf, 21, K=4, window=30, T=10, dummy_cost=1.0, **LAM)
    E = lambda z: orc.energy(np.array(z))
    assert np.isfinite(E([0, EPS, 1]))        # c = p0 (frame 0) before a = p1 (frame 3)
    assert not np.isfinite(E([1, EPS, 0]))    # a before c
    assert not np.isfinite(E([0, EPS, 2]))    # frames 0 and 20: 20 frames apart >= T
    assert not np.isfinite(E([0, EPS, 0]))    # the same point twice
    assert np.isfinite(E([EPS, EPS, 2]))      # a single real point
