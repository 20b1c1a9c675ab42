"""The BF16 precision mode: tensor-core unary table within the BF16 error bound, and whole-path
energies close to the FP64 optimum (the 8 smallest candidates of every list are re-scored in FP32)."""
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
    import oracle
    oracle.build()
    return torch, hgm, oracle


@pytest.mark.parametrize("case", ["single_match", "padded176", "many_rows"])
def test_bf16_unary_within_bound(env, case):
    """|U_bf^2 - U^2| <= 2^-7 (|f|^2 + |f'|^2) lambda1^2: BF16 rounding of each operand (2^-9 relative)
    plus FP32 accumulation; U^2 from FP64."""
    torch, hgm, oracle = env
    if case == "single_match":
        wl = synth.single_match(0)
    elif case == "padded176":
        rng = np.random.default_rng(2)
        mod = synth.make_model(rng, 50)
        sc = synth.make_scene(rng, 40, (640.0, 480.0), ("poisson", 60.0), mod.centres, [mod], [(0, 5)], F_pad=176)
        wl = synth.Workload("p176", [synth.pad_model(mod, 176)], [sc], K=64, window=3)
    else:
        rng = np.random.default_rng(3)
        mod = synth.make_model(rng, 300, F=40)
        sc = synth.make_scene(rng, 30, (100.0, 100.0), 13, mod.centres, [mod], [])
        wl = synth.Workload("rows", [mod], [sc], K=8, window=1)
    mod, sc = wl.models[0], wl.scenes[0]
    m, s = handles(hgm, mod, sc, torch)
    U = torch.empty((mod.n, sc.n), dtype=torch.float32, device="cuda")
    hgm.unary_bf16(m, s, 0.6, U)
    torch.cuda.synchronize()
    U = U.cpu().numpy().astype(np.float64)
    mperm, sperm = m.order(), s.order()
    mf = mod.f[mperm].astype(np.float64)
    sf = sc.f[sperm].astype(np.float64)
    d2 = ((mf[:, None, :] - sf[None, :, :]) ** 2).sum(-1)
    bound = 2.0 ** -7 * ((mf ** 2).sum(1)[:, None] + (sf ** 2).sum(1)[None, :])
    assert np.all(np.abs((U / 0.6) ** 2 - d2) <= bound + 1e-4)


def test_precision_mode_energies(env):
    torch, hgm, oracle = env
    rng = np.random.default_rng(21)
    mod = synth.make_model(rng, 40)
    sc = synth.make_scene(rng, 160, (320.0, 240.0), ("poisson", 30.0), mod.centres, [mod], [(0, 60)])
    wl = synth.Workload("c2_pair", [mod], [sc], K=64, window=3)
    m, s = handles(hgm, mod, sc, torch)
    p = hgm.default_params(K=64, window=3, precision=1)
    first, n = hgm.offsets(m, s, p)
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    a = torch.empty((n, mod.n), dtype=torch.int32, device="cuda")
    hgm.match(m, s, p, e, a)
    torch.cuda.synchronize()
    e, a = e.cpu().numpy(), a.cpu().numpy()
    orc = oracle.Oracle.from_workload(wl)
    rel = []
    for k in range(0, n, 6):
        e_or, _, _ = orc.match(first + k)
        assert np.isfinite(e_or) == np.isfinite(e[k])
        if np.isfinite(e_or):
            rel.append(abs(e[k] - e_or) / e_or)
            # the precision path's assignment is a real chain: its FP64 energy is finite
            assert np.isfinite(orc.energy(a[k]))
    rel = np.array(rel)
    assert rel.mean() <= 2e-3 and rel.max() <= 3e-2, (rel.mean(), rel.max())


def _sub_oracle(oracle, wl, m, o):
    """FP64 oracle of model m on the scene frames its offset-o windows reach, shifted to frame 0 (energies
    and candidate lists are those of the full scene: positions, time differences and the stable order of
    the points inside each frame are unchanged). Returns (oracle, offset in the sub-scene, caller indices
    of the sub-scene's points in the full scene)."""
    mod, sc = wl.models[m], wl.scenes[0]
    f0 = max(0, o + int(mod.t.min()) - wl.window)
    f1 = min(sc.n_frames - 1, o + int(mod.t.max()) + wl.window)
    keep = np.nonzero((sc.t >= f0) & (sc.t <= f1))[0]
    orc = oracle.Oracle(mod.xy, mod.t, mod.f, sc.xy[keep], sc.t[keep] - f0, sc.f[keep], f1 - f0 + 1,
                        K=wl.K, window=wl.window, lambda1=wl.lambda1, lambda2=wl.lambda2, lambda3=wl.lambda3,
                        T=wl.T)
    return orc, o - f0, keep


def test_precision_long_full_size_sampled(env):
    """The precision workload at full size (50 models of 32-128 points vs one 30,000-frame scene with
    Poisson(60) points per frame, descriptors padded to 176, K = 64, w = 3): every offset of every model in
    one batch on the BF16 + FP32 re-score path (unary tables in segment groups, units in chunks); a seeded
    sample of 48 offsets is checked against the FP64 oracle: feasibility identical, relative energy error
    mean <= 2e-3 and max <= 3e-2, and the returned assignment is a real chain whose FP64 energy is within
    the same bound of the reported one."""
    torch, hgm, oracle = env
    wl = synth.precision_long()
    sc = wl.scenes[0]
    dev = torch.device("cuda")
    ms = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (mod.xy, mod.t, mod.f))) for mod in wl.models]
    s = hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (sc.xy, sc.t, sc.f)), sc.n_frames)
    p = hgm.default_params(K=wl.K, window=wl.window, precision=1)
    first, es, as_ = hgm.batch_layout(ms, [s], p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    hgm.match_batch(ms, [s], p, e, a)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    rel, checked = [], 0
    for m in rng.choice(len(wl.models), size=12, replace=False):
        n = int(es[m + 1] - es[m])
        for k in rng.integers(0, n, size=4):
            o = int(first[m]) + int(k)
            eg = float(e[int(es[m]) + int(k)].item())
            M = wl.models[m].n
            row = int(as_[m]) + int(k) * M
            ag = a[row:row + M].cpu().numpy()
            orc, o_sub, keep = _sub_oracle(oracle, wl, int(m), o)
            e64, _, _ = orc.match(o_sub)
            assert np.isfinite(e64) == np.isfinite(eg), (m, o)
            if np.isfinite(e64):
                rel.append(abs(eg - e64) / e64)
                z_sub = np.searchsorted(keep, ag)
                assert np.all(keep[z_sub] == ag)
                e_z = orc.energy(z_sub)
                assert abs(e_z - eg) <= 3e-2 * e64
                checked += 1
            del orc
    rel = np.array(rel)
    assert checked >= 40
    assert rel.mean() <= 2e-3 and rel.max() <= 3e-2, (rel.mean(), rel.max())
