"""The block slicing of a long scene for streaming (hgm.stream_blocks): host logic only."""
import numpy as np

from paper_1505_00581_gb300 import hgm


def test_blocks_cover_the_scene_with_overlap():
    n_frames = 250
    t = np.repeat(np.arange(n_frames), 2).astype(np.int32)
    xy = np.zeros((t.size, 2), np.float32)
    f = np.arange(t.size, dtype=np.float32)[:, None]
    blocks = list(hgm.stream_blocks(xy, t, f, n_frames, 60, 30))
    starts = [b[0] for b in blocks]
    assert starts == [0, 30, 60, 90, 120, 150, 180, 190]      # the last block ends at the scene's end
    covered = np.zeros(n_frames, int)
    for s0, bxy, bt, bf, idx in blocks:
        assert bt.min() >= 0 and bt.max() < 60
        assert np.array_equal(t[idx] - s0, bt)
        assert np.array_equal(bf[:, 0], idx.astype(np.float32))
        covered[s0:s0 + 60] += 1
    assert covered.min() >= 1 and covered[30:180].min() == 2


def test_short_scene_is_one_block():
    t = np.array([0, 3, 5], np.int32)
    blocks = list(hgm.stream_blocks(np.zeros((3, 2), np.float32), t, np.zeros((3, 4), np.float32), 10, 60, 30))
    assert len(blocks) == 1 and blocks[0][0] == 0 and len(blocks[0][4]) == 3
