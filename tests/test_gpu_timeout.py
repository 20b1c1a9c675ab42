"""The bounded waits of the tensor-core kernels: a wait on a barrier that nothing completes gives up after
its poll limit, records the timeout in a status word the host reads, and leaves the context usable (a
match afterwards returns the same result as before). No GPU fault is involved."""
import time

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
    return torch, hgm


def test_wait_runs_out_and_context_survives(env):
    torch, hgm = env
    wl = synth.single_match(0)
    m, s = handles(hgm, wl.models[0], wl.scenes[0], torch)
    p = hgm.default_params(K=32, window=2)
    first, e0, a0 = hgm.match(m, s, p)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    t0 = time.time()
    hgm.debug_timeout(1 << 14, status)
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert int(status.item()) == 1
    first1, e1, a1 = hgm.match(m, s, p)
    assert first1 == first
    np.testing.assert_array_equal(e0, e1)
    np.testing.assert_array_equal(a0, a1)


def test_bad_poll_counts_are_rejected(env):
    torch, hgm = env
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for polls in (0, (1 << 20) + 1):
        with pytest.raises(hgm.HgmError) as err:
            hgm.debug_timeout(polls, status)
        assert err.value.status == hgm.HGM_EINVAL
