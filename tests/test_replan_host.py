"""Host logic of the replanning loop (Alg. 1's "move the robot" and the goal
substitution), tested on the CPU: arc-length motion along the smoothed path,
the goal candidates, and the trajectory statistics the evaluation reports."""
import numpy as np
import pytest

from paper_1903_07441_gb300 import replan


def test_advance_walks_the_polyline_by_arc_length():
    path = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 2.0]])
    p, h, d = replan._advance(path, 0.5)
    assert np.allclose(p, [0.5, 0.0]) and np.allclose(h, [1.0, 0.0]) and d == 0.5
    p, h, d = replan._advance(path, 1.0)        # exactly at the corner: still on the first segment
    assert np.allclose(p, [1.0, 0.0]) and np.allclose(h, [1.0, 0.0])
    p, h, d = replan._advance(path, 2.25)
    assert np.allclose(p, [1.0, 1.25]) and np.allclose(h, [0.0, 1.0]) and d == 2.25
    p, h, d = replan._advance(path, 10.0)       # beyond the end: the last point, the last heading
    assert np.allclose(p, [1.0, 2.0]) and np.allclose(h, [0.0, 1.0]) and d == pytest.approx(3.0)


def test_advance_skips_repeated_points_and_handles_a_single_point():
    path = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 1.0], [0.0, 1.0]])
    p, h, d = replan._advance(path, 0.3)
    assert np.allclose(p, [0.0, 0.3]) and np.allclose(h, [0.0, 1.0])
    p, h, d = replan._advance(np.array([[2.0, 3.0], [2.0, 3.0]]), 0.5)
    assert np.allclose(p, [2.0, 3.0]) and h is None and d == 0.0


def test_goal_candidates_are_free_interior_cells_nearest_first():
    occ = np.zeros((20, 20), np.uint8)
    occ[8:13, 8:13] = 1                      # the goal (10, 10) sits inside a block
    cands = replan._goal_candidates(occ, (10, 10), max_r=6, count=10)
    assert len(cands) == 10
    for x, y in cands:
        assert occ[y, x] == 0 and 1 <= x < 19 and 1 <= y < 19
    ring = [max(abs(x - 10), abs(y - 10)) for x, y in cands]
    assert ring == sorted(ring)              # square rings outwards
    assert min(ring) == 3                    # the first free ring around the block
    # a free goal is its own first candidate
    assert replan._goal_candidates(np.zeros((9, 9), np.uint8), (4, 4), count=3)[0] == (4, 4)


def test_run_result_statistics():
    r = replan.RunResult(trajectory=[(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (1.0, 1.0), (2.0, 1.0)])
    assert r.path_length() == pytest.approx(3.0)
    ang = r.turning_angles()
    assert np.allclose(ang, [90.0, 90.0])    # the zero-length move is skipped
    assert r.collision_free
    r.collision_frame = 3
    assert not r.collision_free
    assert replan.RunResult(trajectory=[(0.0, 0.0)]).path_length() == 0.0
