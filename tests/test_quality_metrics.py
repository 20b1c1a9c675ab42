"""The pruned form's quality metrics (point recall, unit match, energy gap, and the per-pair figures
recognition uses) on hand-built results whose values are worked out by hand."""
import numpy as np

from paper_1505_00581_gb300 import prop_train


def _case():
    # two (model, scene) pairs: 3 offsets of a 2-point model, then 2 offsets of a 3-point model
    e_ref = np.array([5.0, 2.0, 4.0, np.inf, 8.0], np.float32)
    a_ref = np.array([1, 2, 3, 4, 5, 6, -1, -1, -1, 7, 8, 9], np.int32)
    e = np.array([5.0, 2.5, 3.0 * 1.5, np.inf, 10.0], np.float32)
    a = np.array([1, 2, 3, 0, 5, 0, -1, -1, -1, 7, 0, 0], np.int32)
    M_rows = [(0, 3, 2), (6, 2, 3)]
    e_rows = [0, 3]
    return e_ref, a_ref, e, a, M_rows, e_rows


def test_unit_level_metrics():
    e_ref, a_ref, e, a, M_rows, e_rows = _case()
    q = prop_train.compare(e_ref, a_ref, e, a, M_rows, e_rows)
    # feasible units: pair 0 offsets 0..2 (6 points), pair 1 offset 1 (3 points); hits 2 + 1 + 1 + 1 = 5
    assert q["point_recall"] == 5 / 9
    assert q["unit_match"] == 1 / 4
    gaps = [0.0, 0.25, 0.125, 0.25]
    assert abs(q["mean_rel_gap"] - np.mean(gaps)) < 1e-7
    assert q["feasible_mismatch"] == 0


def test_pair_level_metrics():
    e_ref, a_ref, e, a, M_rows, e_rows = _case()
    p = prop_train.compare(e_ref, a_ref, e, a, M_rows, e_rows)["pairs"]
    # pair 0: exact best offset 1 (2.0), pruned best offset 1 (2.5): same offset, recall there 1 of 2,
    # gap 0.25; pair 1: exact best offset 1 (8.0), pruned 10.0 at offset 1: recall 1 of 3, gap 0.25
    assert p["pairs"] == 2
    assert p["best_offset_match"] == 1.0
    assert p["point_recall_at_best"] == 2 / 5
    assert abs(p["mean_rel_gap"] - 0.25) < 1e-7


def test_pair_level_moved_minimum():
    e_ref, a_ref, e, a, M_rows, e_rows = _case()
    e = e.copy()
    e[0] = 2.2                     # the pruned minimum of pair 0 moves to offset 0
    p = prop_train.pair_stats(e_ref, a_ref, e, a, M_rows, e_rows)
    assert p["best_offset_match"] == 0.5
    assert abs(p["mean_rel_gap"] - (0.1 + 0.25) / 2) < 1e-7
