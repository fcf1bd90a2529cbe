"""Pins of the oracle's discontinuity margin against hand geometry (no GPU).

The margin is how far a rollout point may move before a step-cost term jumps: the closest
reference segment switching to one of another heading (Eq. (12), (14)), the c_target
indicator flipping (Eq. (13)), the yaw error reaching the wrap at +-pi, or, with the
collision-only cost, d_obj crossing zero (Eq. (16)-(17)).  The parity tests use it to
decide which samples may land on the other side of a jump in binary32, so a margin that
came out too small would widen that set; each case below has a margin known exactly from
the geometry.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_01654_gb300 import scenarios as sc


def test_interior_tie_between_two_segments():
    """A V-shaped lane (0,10) -> (10,0) -> (20,10): for P = (9, 5) both projections are interior,
    the distances are 4/sqrt2 and 6/sqrt2, and the two segments tie on the bisector x = 10, one
    metre away (both distances are linear there, so the first-order estimate is exact)."""
    ref = np.array([[0.0, 10.0], [10.0, 0.0], [20.0, 10.0]])
    d2, idx, th, m = oracle.nearest_ref(ref, 9.0, 5.0)
    assert idx == 0
    assert th == pytest.approx(-math.pi / 4, abs=1e-15)
    assert d2 == pytest.approx(8.0, rel=1e-14)
    assert m == pytest.approx(1.0, rel=1e-12)
    # moving the point along the bisector's normal changes the margin one for one
    for dx in (0.25, 0.5, 0.9):
        _, idx2, _, m2 = oracle.nearest_ref(ref, 9.0 + dx, 5.0)
        assert idx2 == 0 and m2 == pytest.approx(1.0 - dx, rel=1e-12)
    _, idx3, _, _ = oracle.nearest_ref(ref, 10.25, 5.0)
    assert idx3 == 1                                   # across the tie the other segment wins


def test_tie_with_a_segment_that_is_not_a_neighbour():
    """A U-turn (0,0) -> (10,0) -> (10,4) -> (0,4): for P = (5, 1) the way back (heading pi) is 3 m
    away and ties with the way out on y = 2 (1 m away); the middle segment (heading pi/2) is 5 m
    away and ties on x + y = 10, 4/sqrt2 m away."""
    ref = np.array([[0.0, 0.0], [10.0, 0.0], [10.0, 4.0], [0.0, 4.0]])
    d2, idx, th, m = oracle.nearest_ref(ref, 5.0, 1.0)
    assert idx == 0 and th == 0.0 and d2 == pytest.approx(1.0, rel=1e-14)
    assert m == pytest.approx(1.0, rel=1e-12)
    _, _, _, m_mid = oracle.nearest_ref(ref, 7.5, 1.9)
    # (7.5, 1.9): way back 2.1 m, middle 2.5 m, way out 1.9 m; ties at y = 2 (0.1 m) and on
    # y = 10 - x (|7.5 + 1.9 - 10| / sqrt2 = 0.6 / sqrt2 m)
    assert m_mid == pytest.approx(0.1, rel=1e-9)


def test_corner_cone_margin_is_the_distance_to_the_nearest_clamp_release():
    """Outside the bend of (0,0) -> (10,0) -> (10,10), P = (12, -3) is closest to the shared vertex
    on both segments (both projections clamped): an exact tie, decided by the lower index.  The
    tie lasts until one clamp releases: at x = 10 (2 m away) or y = 0 (3 m away)."""
    ref = np.array([[0.0, 0.0], [10.0, 0.0], [10.0, 10.0]])
    d2, idx, th, m = oracle.nearest_ref(ref, 12.0, -3.0)
    assert idx == 0 and th == 0.0
    assert d2 == pytest.approx(13.0, rel=1e-14)
    assert m == pytest.approx(2.0, rel=1e-12)
    _, _, _, m2 = oracle.nearest_ref(ref, 10.5, -3.0)
    assert m2 == pytest.approx(0.5, rel=1e-12)
    _, _, _, m3 = oracle.nearest_ref(ref, 14.0, -1.25)
    assert m3 == pytest.approx(1.25, rel=1e-12)


def test_vertex_mode_margin_is_the_distance_to_the_bisector():
    """Closest-vertex mode on (0,0) -> (4,0) -> (4,4): P = (1, 0) is 1 m from vertex 0 and 3 m from
    vertex 1 (heading pi/2); they tie on x = 2, 1 m away.  Vertex 2 is 5 m away."""
    ref = np.array([[0.0, 0.0], [4.0, 0.0], [4.0, 4.0]])
    d2, idx, th, m = oracle.nearest_ref(ref, 1.0, 0.0, mode=1)
    assert idx == 0 and th == 0.0 and d2 == 1.0
    assert m == pytest.approx(1.0, rel=1e-12)


def test_one_heading_has_no_switch():
    ref = sc.straight_lane(50, 0.5)
    _, _, _, m = oracle.nearest_ref(ref, 7.3, 0.4)
    assert m == math.inf


def _one_step_problem(v0, yaw0=0.0, target_x=10.0):
    p = sc.default_params(1, 1, 0.1)
    p.update(sigma=[0.0, 0.0], sg_enable=0)
    ref = np.array([[0.0, 0.0], [target_x, 0.0]])
    return p, np.array([0.0, 0.0, yaw0, v0]), ref


def test_target_indicator_margin():
    """One Euler step from (0,0) at 8 m/s with no noise: P_1 = (0.8, 0), target (10, 0).  The
    distances to the target are 10 and 9.2; the indicator of Eq. (13) flips when the two meet,
    which takes a move of half their difference by each point: 0.4 m.  The straight lane has one
    heading and the yaw error is 0 (margin pi to the wrap), so 0.4 is the sample's margin."""
    p, x0, ref = _one_step_problem(8.0)
    S, eps, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, np.zeros((0, 5)))
    assert m == pytest.approx(0.4, rel=1e-12)


def test_yaw_wrap_margin():
    """Heading 3 rad against a lane heading 0: the yaw error is 3 rad, pi - 3 = 0.1416 rad from the
    wrap.  At 0.1 m/s the step moves 0.01 m, so the target indicator's margin (about 0.005 m) is
    the smaller; standing still, the indicator compares equal distances (margin 0)."""
    p, x0, ref = _one_step_problem(0.1, yaw0=3.0)
    S, eps, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, np.zeros((0, 5)))
    # P_1 = (0.01 cos 3, 0.01 sin 3): distances to (10, 0) differ by about 0.0099
    p1 = np.array([0.01 * math.cos(3.0), 0.01 * math.sin(3.0)])
    mt = 0.5 * abs(np.hypot(*(p1 - [10.0, 0.0])) - 10.0)
    assert m == pytest.approx(min(mt, math.pi - 3.0), rel=1e-9)
    p, x0, ref = _one_step_problem(0.0, yaw0=3.0)
    S, eps, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, np.zeros((0, 5)))
    assert m == 0.0
    p, x0, ref = _one_step_problem(30.0, yaw0=3.12)   # 3 m in one step: the wrap (0.0216 rad) is nearer
    S, eps, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, np.zeros((0, 5)))
    assert m == pytest.approx(math.pi - 3.12, rel=1e-12)


def test_collision_only_margin_is_the_clearance():
    """With the collision-only cost, c_safe switches on where d_obj crosses 0: the margin includes
    |d_obj|.  One ego circle of radius 1 at the rear axle and an obstacle circle of radius 0.5 on
    the lane.  Standing still, the target indicator compares equal distances (margin 0); moving
    0.1 m its margin is 0.05 m, and an obstacle leaving 2 cm of clearance brings it to 0.02."""
    p, x0, ref = _one_step_problem(0.0, target_x=1000.0)
    p.update(collision_only=1, n_ego=1, ego_offset=[0.0], ego_radius=[1.0])
    circ = np.array([[3.75, 0.0, 0.5, 0.0, 0.0]])
    _, _, m_plain = oracle.rollout_cost(dict(p, collision_only=0), x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, circ)
    _, _, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, circ)
    assert m_plain == 0.0                              # standing still: the indicator compares equals
    assert m == 0.0
    x0[3] = 1.0                                        # moving 0.1 m: indicator margin 0.05
    _, _, m_plain = oracle.rollout_cost(dict(p, collision_only=0), x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, circ)
    assert m_plain == pytest.approx(0.05, rel=1e-9)
    circ[0, 0] = 0.1 + 1.5 + 0.02                      # 2 cm of clearance after the step
    _, _, m = oracle.rollout_cost(p, x0, np.zeros((1, 2)), np.zeros((1, 2)), ref, circ)
    assert m == pytest.approx(0.02, rel=1e-9)
