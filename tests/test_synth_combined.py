"""The combined workload's on-demand scene generator (host only): a block of frames is the same points as
the whole scene's frames (every 64-frame chunk and every implant has its own seeded stream), blocks of one
pass restrict every pair to the offsets whose windows lie inside them, and the clutter has the stated
statistics (Poisson(80) points per frame, uniform positions over 640x480)."""
import numpy as np

from paper_1505_00581_gb300 import synth


def _small():
    return synth.CombinedScenes(seed=9, n_models=6, n_scenes=3, frames_range=(400, 700))


def test_block_equals_the_slice_of_the_whole_scene():
    cs = _small()
    for s in range(3):
        whole = cs.scene(s)
        for f0, f1 in ((0, 65), (63, 200), (130, 131), (cs.n_frames[s] - 100, cs.n_frames[s])):
            b = cs.block(s, f0, f1)
            sel = (whole.t >= f0) & (whole.t < f1)
            # clutter first in frame order, then implant points: the same points in the same order
            assert b.n == int(sel.sum())
            assert np.array_equal(b.t, whole.t[sel] - f0)
            assert np.array_equal(b.xy, whole.xy[sel]) and np.array_equal(b.f, whole.f[sel])
            assert b.n_frames == f1 - f0


def test_implants_are_jittered_copies_of_their_models():
    cs = _small()
    whole = cs.scene(1)
    assert whole.implants
    for imp in whole.implants:
        mod = cs.models[imp.model]
        assert len(imp.idx) == mod.n
        df = whole.f[imp.idx] - mod.f
        assert abs(float(df.std()) - 0.1) < 0.02          # descriptor noise N(0, 0.1)
        dt = whole.t[imp.idx].astype(int) - (mod.t.astype(int) + imp.offset)
        clipped = (whole.t[imp.idx] == 0) | (whole.t[imp.idx] == whole.n_frames - 1)
        assert np.all((np.abs(dt) <= 5) | clipped)         # frame jitter rint(N(0, 1))


def test_clutter_statistics():
    cs = synth.CombinedScenes(seed=4, n_models=3, n_scenes=1, frames_range=(3000, 3000))
    b = cs.block(0, 0, 3000)
    imp_pts = sum(len(i.idx) for i in b.implants)
    per_frame = np.bincount(b.t[:b.n - imp_pts], minlength=3000)
    assert abs(per_frame.mean() - 80.0) < 1.0 and abs(per_frame.var() - 80.0) < 8.0
    assert b.xy[:, 0].min() >= 0 and b.xy[:, 0].max() < 640 and b.xy[:, 1].max() < 480


def test_step_blocks_own_hop_offsets_each():
    cs = _small()
    wl = cs.step(hop=64, seed=2)
    assert wl.total_frames == 3 * 64
    for m in range(len(wl.models)):
        for s in range(len(wl.scenes)):
            lo, hi = wl.offset_range(m, s)
            assert (lo, hi) == (wl.window, wl.window + 63)
            mod = wl.models[m]
            # every window of every owned offset lies inside the block (no clipping at its edges)
            assert lo + int(mod.t.min()) - wl.window >= 0
            assert hi + int(mod.t.max()) + wl.window <= wl.scenes[s].n_frames - 1


def test_full_size_job_shape():
    cs = synth.CombinedScenes()
    assert len(cs.models) == 100 and len(cs.n_frames) == 16
    assert all(16 <= m.n <= 256 for m in cs.models)
    assert all(10_000 <= n <= 100_000 for n in cs.n_frames)
    # implants cover about 5% of the offsets (each is seen by 2w+1 = 7 offsets)
    cover = sum(len(i) for i in cs.implants) * 7 / cs.total_frames
    assert 0.045 < cover < 0.055
