"""Pins of the oracle's "independent chains" variant (Sec. 4, multiple points per frame, method 2).

The chain membership is checked against its definition by direct enumeration, one chain over a
one-point-per-frame model must reduce to the plain problem, and on tiny instances the chain distance must
equal the mean of the chains' brute-force minima of Eq. 9 (enumeration, not the recursion)."""
import math

import numpy as np
import pytest

from paper_1505_00581_gb300 import synth

LAM = dict(lambda1=0.6, lambda2=0.2, lambda3=5.0)


def _multi_point_model(rng, frames, per_frame, F=8, frame=(20.0, 20.0)):
    t = np.repeat(np.arange(frames), per_frame)
    rng.shuffle(t)                                   # caller order is not frame order
    M = len(t)
    xy = rng.uniform((0, 0), frame, size=(M, 2)).astype(np.float32)
    centres = rng.standard_normal((3, F))
    f = (centres[rng.integers(0, 3, M)] + 0.3 * rng.standard_normal((M, F))).astype(np.float32)
    return synth.PointSet(xy, t.astype(np.int32), f, centres)


def test_chain_membership_follows_the_definition(oracle_mod):
    rng = np.random.default_rng(1)
    mod = _multi_point_model(rng, frames=6, per_frame=np.array([1, 3, 2, 3, 1, 2]))
    sc = synth.make_scene(rng, 12, (20.0, 20.0), 3, mod.centres, [mod], [], translate=False)
    co = oracle_mod.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, 3, K=5, window=1, **LAM)
    seen = np.concatenate(co.members)
    assert len(seen) == len(set(seen.tolist()))                       # each point in at most one chain
    for k, idx in enumerate(co.members):
        assert np.all(np.diff(mod.t[idx]) > 0)                        # one point per frame, frame order
        for i in idx:                                                 # rank k among its frame, caller order
            same = np.nonzero(mod.t == mod.t[i])[0]
            assert list(same).index(i) == k
    # chains shorter than 3 are not formed: chain 2 holds the third points of frames 1 and 3 only
    assert len(co.members) == 2


def test_one_chain_of_a_single_point_model_is_the_plain_problem(oracle_mod):
    wl = synth.tiny_case(4, M=6, n_frames=12, per_frame=3, K=4, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    if len(np.unique(mod.t)) != mod.n:
        mod = synth.PointSet(mod.xy, np.arange(mod.n, dtype=np.int32), mod.f, mod.centres)
    kw = dict(K=wl.K, window=wl.window, T=wl.T, **LAM)
    co = oracle_mod.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, 1, **kw)
    orc = oracle_mod.Oracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, **kw)
    for o in orc.offsets():
        e1, z1 = co.match(int(o))
        e0, z0, _ = orc.match(int(o))
        assert (math.isinf(e0) and math.isinf(e1)) or e1 == pytest.approx(e0, rel=1e-15)
        assert np.array_equal(z1, z0)


@pytest.mark.parametrize("seed", range(8))
def test_chain_distance_is_the_mean_of_bruteforce_minima(seed, oracle_mod):
    rng = np.random.default_rng(100 + seed)
    mod = _multi_point_model(rng, frames=4, per_frame=2)              # two chains of 4 points
    sc = synth.make_scene(rng, 10, (20.0, 20.0), 2, mod.centres, [mod], [], translate=False)
    kw = dict(K=3, window=1, T=[10, 0][seed % 2], **LAM)
    co = oracle_mod.ChainOracle(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, 2, **kw)
    assert len(co.members) == 2
    for o in range(co.first_offset, co.first_offset + co.n_offsets):
        e, z = co.match(o)
        mins = []
        for idx in co.members:
            sub = oracle_mod.Oracle(mod.xy[idx], mod.t[idx], mod.f[idx], sc.xy, sc.t, sc.f, sc.n_frames, **kw)
            e_bf, _, _ = sub.bruteforce(o)
            mins.append(e_bf)
        if all(np.isfinite(mins)):
            assert e == pytest.approx(float(np.mean(mins)), rel=1e-12)
        else:
            assert math.isinf(e)
