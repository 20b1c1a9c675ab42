"""Device helpers checked on their own: the recursion kernel's FP32 atan2 against FP64."""
import numpy as np
import pytest

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


def test_fast_atan2_error_bound(env):
    """|atan2_f32(y, x) - atan2(y, x)| <= 6e-7 rad over random, axis, diagonal and wide-range inputs
    (the fit's own error is 2.5e-7 rad; the rest is FP32 evaluation)."""
    torch, hgm = env
    rng = np.random.default_rng(0)
    parts = [rng.uniform(-700, 700, size=(200000, 2)),
             rng.normal(size=(100000, 2)) * 10.0 ** rng.uniform(-6, 6, size=(100000, 1)),
             np.stack([np.linspace(-5, 5, 1001), np.zeros(1001)], 1),
             np.stack([np.zeros(1001), np.linspace(-5, 5, 1001)], 1),
             np.stack([np.linspace(-5, 5, 1001), np.linspace(-5, 5, 1001)], 1),
             np.stack([np.linspace(-5, 5, 1001), -np.linspace(-5, 5, 1001)], 1)]
    yx = np.concatenate(parts).astype(np.float32)
    y = torch.from_numpy(np.ascontiguousarray(yx[:, 0])).cuda()
    x = torch.from_numpy(np.ascontiguousarray(yx[:, 1])).cuda()
    out = torch.empty_like(y)
    hgm.atan2_f32(y, x, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = np.arctan2(yx[:, 0].astype(np.float64), yx[:, 1].astype(np.float64))
    err = np.abs(got - want)
    # +pi and -pi are the same direction on the negative x axis
    err = np.minimum(err, np.abs(np.abs(err) - 2 * np.pi))
    assert err.max() <= 6e-7, err.max()


def test_fast_atan2_special_values(env):
    torch, hgm = env
    y = torch.tensor([0.0, 0.0, -0.0, 1.0, -1.0, 0.0, 3.0], device="cuda")
    x = torch.tensor([0.0, -1.0, -1.0, 0.0, 0.0, 2.0, 3.0], device="cuda")
    out = torch.empty_like(y)
    hgm.atan2_f32(y, x, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array([0.0, np.pi, -np.pi, np.pi / 2, -np.pi / 2, 0.0, np.pi / 4], np.float32)
    assert np.allclose(got, want, atol=4e-7)


@pytest.mark.parametrize("M,N,K", [(128, 128, 16), (300, 200, 176), (1000, 64, 128), (77, 250, 256)])
def test_tensor_core_gemm_matches_bf16_reference(env, M, N, K):
    """The tcgen05 operand layout and descriptors: bf16(A) @ bf16(B).T accumulated in FP32 on the
    tensor cores equals the same product computed in FP32 by torch up to summation order."""
    torch, hgm = env
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    hgm.gemm_bf16(A, B, C, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.bfloat16().float() @ B.bfloat16().float().T
    err = (C - ref).abs().max().item()
    assert err <= 1e-5 * K * 4, err
