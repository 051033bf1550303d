"""The algorithmic byte model behind the reported roofline fraction, on schedules
small enough to count by hand (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1705_04590_gb300 import roofline  # noqa: E402

TD, BU = 0, 1


def test_path_top_down_by_hand():
    # path 0-1-2-3-4 from vertex 0, every level top-down:
    # records (dir, n_f, m_f, n_next, m_next, scanned, examined)
    rec = [(TD, 1, 1, 1, 2, 0, 1), (TD, 1, 2, 1, 2, 0, 2), (TD, 1, 2, 1, 2, 0, 2),
           (TD, 1, 2, 1, 1, 0, 2), (TD, 1, 1, 0, 0, 0, 1)]
    # n = 5: one bitmap byte; parent + level: 8 bytes per vertex
    init = 8 * 5 + 1
    # per level: 16 per frontier vertex (two offsets) + 4 per edge + 12 per found vertex
    levels = (16 + 4 + 12) + 3 * (16 + 8 + 12) + (16 + 4 + 0)
    assert roofline.search_bytes(5, rec) == init + levels == 201


def test_star_switches_direction_by_hand():
    # star with centre 0 and leaves 1..4, searched from leaf 1: top-down finds the
    # centre, bottom-up lets the three other leaves find it at their first probe,
    # then one top-down level over those leaves finds nothing
    rec = [(TD, 1, 1, 1, 4, 0, 1), (BU, 1, 4, 3, 3, 3, 3), (TD, 3, 3, 0, 0, 0, 3)]
    init = 8 * 5 + 1
    td0 = 16 * 1 + 4 * 1 + 12 * 1
    q2b = 4 * 1 + 1                                   # queue -> bitmap before bottom-up
    bu1 = 16 * 3 + 4 * 3 + 3 * 1 + 8 * 3              # offsets, ids, three bitmap passes, outputs
    b2q = 1 + 4 * 3                                   # bitmap -> queue before top-down
    td2 = 16 * 3 + 4 * 3 + 0
    assert roofline.search_bytes(5, rec) == init + td0 + q2b + bu1 + b2q + td2 == 238


def test_outputs_not_requested_are_not_charged():
    rec = [(TD, 1, 1, 1, 4, 0, 1), (BU, 1, 4, 3, 3, 3, 3)]
    both = roofline.search_bytes(5, rec)
    parent_only = roofline.search_bytes(5, rec, want_level=False)
    none = roofline.search_bytes(5, rec, want_parent=False, want_level=False)
    # 4 bytes per vertex at init and 4 per found vertex (1 + 3) for each dropped output
    assert both - parent_only == 4 * 5 + 4 * 4
    assert both - none == 2 * (4 * 5 + 4 * 4)


def test_probes_charged_once_a_bitmap_outgrows_a_quarter_of_l2():
    rec = [(TD, 1, 10, 2, 6, 0, 10), (BU, 2, 6, 5, 9, 7, 11)]
    small_n = 8 * (roofline.L2_BYTES // 4)           # bitmap exactly a quarter of L2
    big_n = small_n + 8                              # one byte more
    base_small = roofline.search_bytes(small_n, rec)
    base_big = roofline.search_bytes(big_n, rec)
    # the big graph pays for its extra vertices and bitmap bytes, plus 4 bytes per probe:
    # 10 top-down edge probes and 11 bottom-up examinations
    W_small, W_big = small_n // 8, big_n // 8
    extra_size = 8 * (big_n - small_n) + (W_big - W_small) * (1 + 1 + 3)
    assert base_big - base_small == extra_size + 4 * (10 + 11)
