"""The block slicing of a long scene for streaming (hgm.stream_blocks): host logic only."""
import numpy as np
import pytest

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


def _frames(n_frames, per=1):
    t = np.repeat(np.arange(n_frames), per).astype(np.int32)
    return np.zeros((t.size, 2), np.float32), t, np.arange(t.size, dtype=np.float32)[:, None]


def test_exact_fit_and_hop_equal_to_block():
    xy, t, f = _frames(120)
    assert [b[0] for b in hgm.stream_blocks(xy, t, f, 120, 60, 30)] == [0, 30, 60]   # 60 + 60 = 120: no extra
    blocks = list(hgm.stream_blocks(xy, t, f, 120, 60, 60))                          # no overlap
    assert [b[0] for b in blocks] == [0, 60]
    assert np.array_equal(np.concatenate([b[4] for b in blocks]), np.arange(t.size))   # every point once


def test_hop_longer_than_a_block_skips_frames():
    xy, t, f = _frames(200)
    blocks = list(hgm.stream_blocks(xy, t, f, 200, 60, 90))
    assert [b[0] for b in blocks] == [0, 90, 140]
    seen = np.zeros(200, int)
    for s0, _, bt, _, idx in blocks:
        seen[t[idx]] += 1
        assert bt.min() >= 0 and bt.max() < 60
    assert np.all(seen[60:90] == 0) and np.all(seen[:60] == 1) and np.all(seen[90:] >= 1)


def test_points_past_the_scene_and_empty_blocks():
    xy, t, f = _frames(100)
    t = t.copy()
    t[40:60] = 0                       # frames 40..59 empty
    t[-1] = 150                        # a point past the scene's last frame is in no block
    blocks = list(hgm.stream_blocks(xy, t, f, 100, 20, 20))
    assert [b[0] for b in blocks] == [0, 20, 40, 60, 80]
    assert len(blocks[2][4]) == 0      # an empty block is still yielded (its models get no match)
    assert all(len(b[4]) == 0 or b[4].max() < t.size - 1 for b in blocks)


@pytest.mark.parametrize("block,hop", [(0, 30), (60, 0), (-5, 10)])
def test_invalid_block_or_hop(block, hop):
    xy, t, f = _frames(10)
    with pytest.raises(ValueError):
        list(hgm.stream_blocks(xy, t, f, 10, block, hop))
