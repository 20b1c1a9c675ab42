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
