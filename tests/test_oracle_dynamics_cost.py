"""Pins for the oracle's dynamics (Eq. (5)) and step costs (Sec. IV-C, Eq. (12)-(18)).

Each expected value here is fixed by geometry or a closed form, not by the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import golden_constants
from paper_2308_01654_gb300 import scenarios as sc

L = 2.7


# ---------------------------------------------------------------- dynamics, Eq. (5)

def euler_path(x0, a, delta, dt, n):
    xs = [np.asarray(x0, dtype=float)]
    for _ in range(n):
        xs.append(oracle.bicycle_step(xs[-1], a, delta, dt, L))
    return np.array(xs)


def test_zero_steer_constant_speed_is_a_straight_line():
    xs = euler_path([1.0, -2.0, 0.0, 8.0], 0.0, 0.0, 0.05, 200)
    assert np.all(xs[:, 1] == -2.0) and np.all(xs[:, 2] == 0.0) and np.all(xs[:, 3] == 8.0)
    np.testing.assert_allclose(xs[:, 0], 1.0 + 8.0 * 0.05 * np.arange(201), rtol=0, atol=1e-11)


def test_zero_steer_constant_accel_closed_form():
    # Euler uses v_t at step t: x_n = x0 + dt * (n v0 + a dt n(n-1)/2), v_n = v0 + a n dt
    v0, a, dt, n = 3.0, 1.5, 0.1, 40
    xs = euler_path([0.0, 0.0, 0.0, v0], a, 0.0, dt, n)
    np.testing.assert_allclose(xs[-1, 3], v0 + a * n * dt, rtol=1e-14)
    np.testing.assert_allclose(xs[-1, 0], dt * (n * v0 + a * dt * n * (n - 1) / 2.0), rtol=1e-13)


def test_heading_direction_moves_along_yaw():
    th = 0.7
    xs = euler_path([0.0, 0.0, th, 5.0], 0.0, 0.0, 0.2, 10)
    np.testing.assert_allclose(xs[-1, :2], 10 * 0.2 * 5.0 * np.array([math.cos(th), math.sin(th)]), atol=1e-13)


@pytest.mark.parametrize("delta", [0.05, -0.2, 0.4])
def test_constant_steer_vertices_lie_on_a_circle(delta):
    v, dt, n = 8.0, 0.05, 300
    xs = euler_path([0.0, 0.0, 0.0, v], 0.0, delta, dt, n)
    dth = v * dt * math.tan(delta) / L
    # yaw advances by exactly v dt tan(delta) / L per step; positive delta turns left
    np.testing.assert_allclose(np.diff(xs[:, 2]), dth, rtol=1e-12)
    assert np.sign(xs[5, 1]) == np.sign(delta)
    # chord of length v dt turning by dth: vertices on a circle of radius v dt / (2 sin(dth/2))
    rho = v * dt / (2.0 * math.sin(abs(dth) / 2.0))
    # centre: perpendicular bisector construction from the first chord
    p0, p1 = xs[0, :2], xs[1, :2]
    mid = 0.5 * (p0 + p1)
    chord = p1 - p0
    nrm = np.array([-chord[1], chord[0]]) / np.linalg.norm(chord) * np.sign(delta)
    h = math.sqrt(rho ** 2 - (np.linalg.norm(chord) / 2) ** 2)
    centre = mid + h * nrm
    r = np.linalg.norm(xs[:, :2] - centre, axis=1)
    np.testing.assert_allclose(r, rho, rtol=1e-11)
    # and rho tends to the turning radius L / tan(delta) with relative error ~ dth^2 / 24
    R_turn = L / abs(math.tan(delta))
    assert abs(rho / R_turn - 1.0) == pytest.approx(dth ** 2 / 24.0, rel=1e-3)


# ---------------------------------------------------------------- reference search, Eq. (12)/(14)

def test_nearest_point_on_straight_lane():
    ref = sc.straight_lane(50, 0.5)
    d2, idx, th, _ = oracle.nearest_ref(ref, 7.3, 0.4)
    assert d2 == pytest.approx(0.16, abs=1e-15) and th == 0.0 and idx == 14
    # beyond the end: distance to the last vertex
    d2, idx, th, _ = oracle.nearest_ref(ref, 24.5 + 3.0, 4.0)
    assert d2 == pytest.approx(25.0, abs=1e-12) and idx == 48


def test_corner_cone_ties_go_to_the_lower_segment():
    ref = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0]])
    d2, idx, th, _ = oracle.nearest_ref(ref, 2.0, -1.0)      # outside the corner: both clamp to (1,0)
    assert d2 == 2.0 and idx == 0 and th == 0.0
    d2, idx, th, _ = oracle.nearest_ref(ref, 1.5, 0.5)       # closer to the vertical segment
    assert d2 == 0.25 and idx == 1 and th == pytest.approx(math.pi / 2)
    d2, idx, th, _ = oracle.nearest_ref(ref, 0.5, 0.2)       # above the horizontal segment
    assert d2 == pytest.approx(0.04) and idx == 0


def test_nearest_point_agrees_with_dense_sampling():
    rng = np.random.default_rng(5)
    for _ in range(30):
        n = int(rng.integers(2, 8))
        ref = np.cumsum(rng.normal(size=(n, 2)), axis=0)
        px, py = rng.normal(size=2) * 2
        d2, idx, _, _ = oracle.nearest_ref(ref, px, py)
        pts = []
        for i in range(n - 1):
            s = np.linspace(0, 1, 4001)[:, None]
            pts.append(ref[i] + s * (ref[i + 1] - ref[i]))
        pts = np.concatenate(pts)
        dd = np.min(np.sum((pts - [px, py]) ** 2, axis=1))
        seglen = np.max(np.linalg.norm(np.diff(ref, axis=0), axis=1))
        h = seglen / 4000
        assert d2 <= dd + 1e-12
        assert math.sqrt(dd) - math.sqrt(d2) <= h


def test_vertex_mode_picks_closest_vertex_and_outgoing_heading():
    ref = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    d2, idx, th, _ = oracle.nearest_ref(ref, 1.2, 0.9, mode=1)
    assert idx == 2 and d2 == pytest.approx(0.05) and th == pytest.approx(math.pi)
    d2, idx, th, _ = oracle.nearest_ref(ref, -0.3, 1.1, mode=1)   # last vertex: incoming segment
    assert idx == 3 and th == pytest.approx(math.pi)
    d2, idx, th, _ = oracle.nearest_ref(ref, 0.5, -0.1, mode=1)   # equidistant from 0 and 1 -> lower
    assert idx == 0 and th == 0.0


def test_wrap_angle():
    assert oracle.wrap_angle(0.1) == pytest.approx(0.1)
    assert oracle.wrap_angle(1.5 * math.pi) == pytest.approx(-0.5 * math.pi)
    assert oracle.wrap_angle(-1.5 * math.pi) == pytest.approx(0.5 * math.pi)
    assert oracle.wrap_angle(2 * math.pi + 0.1) == pytest.approx(0.1)
    assert oracle.wrap_angle(-7 * math.pi + 0.2) == pytest.approx(-math.pi + 0.2)


# ---------------------------------------------------------------- obstacles, Eq. (16)

def test_obstacle_distance_3_4_5():
    p = sc.default_params(1, 1, 0.1)
    p.update(n_ego=1, ego_offset=[0.0], ego_radius=[1.0])
    d = oracle.obstacle_distance(p, [0.0, 0.0, 0.0, 0.0], [[3.0, 4.0, 1.0, 0.0, 0.0]], [[3.0, 4.0]])
    assert d == pytest.approx(3.0, abs=1e-15)
    # two ego circles along a heading of pi/2: the one at (0, 2) is closest: sqrt(13) - 2
    p.update(n_ego=2, ego_offset=[0.0, 2.0], ego_radius=[1.0, 1.0])
    d = oracle.obstacle_distance(p, [0.0, 0.0, math.pi / 2, 0.0], [[3.0, 4.0, 1.0, 0.0, 0.0]], [[3.0, 4.0]])
    assert d == pytest.approx(math.sqrt(13.0) - 2.0, abs=1e-14)
    # min over several circles, and +inf with none
    d = oracle.obstacle_distance(p, [0.0, 0.0, 0.0, 0.0], [[3.0, 4.0, 1.0, 0, 0], [0.0, -3.0, 0.5, 0, 0]],
                                 [[3.0, 4.0], [0.0, -3.0]])
    assert d == pytest.approx(1.5, abs=1e-14)
    assert oracle.obstacle_distance(p, [0.0, 0.0, 0.0, 0.0], np.zeros((0, 5)), np.zeros((0, 2))) == math.inf


# ---------------------------------------------------------------- whole step cost, Eq. (12)-(18)

def one_step(p, x0, U=None, z=None, ref=None, circles=None, centres=None):
    p = dict(p, T=1)
    ref = sc.straight_lane(400, 0.5) if ref is None else ref
    circles = np.zeros((0, 5)) if circles is None else np.asarray(circles, float)
    U = np.zeros((1, 2)) if U is None else np.asarray(U, float).reshape(1, 2)
    z = np.zeros((1, 2)) if z is None else np.asarray(z, float).reshape(1, 2)
    S, eps, m = oracle.rollout_cost(p, x0, U, z, ref, circles, centres)
    return S, eps


def base_params():
    p = sc.default_params(1, 1, 0.1)
    p.update(sigma=[0.0, 0.0], n_ego=1, ego_offset=[0.0], ego_radius=[0.0])
    return p


def test_weights_are_the_papers():
    g = golden_constants()
    p = sc.default_params(1, 1, 0.1)
    for k in ("w_dist", "w_target", "w_yaw", "w_speed", "w_safe"):
        assert p[k] == g[k]
    assert sc.V_G == pytest.approx(g["v_G_kmh"] / 3.6)


def test_on_lane_at_reference_speed_costs_nothing():
    p = base_params()
    S, _ = one_step(p, [0.0, 0.0, 0.0, p["v_ref"]])
    assert S == 0.0


def test_lateral_offset_gives_c_dist():
    p = base_params()
    S, _ = one_step(p, [0.0, 0.3, 0.0, p["v_ref"]])
    assert S == pytest.approx(15.0 * 0.09, rel=1e-14)


def test_speed_error_gives_c_speed():
    p = base_params()
    S, _ = one_step(p, [0.0, 0.0, 0.0, p["v_ref"] + 2.0])
    assert S == pytest.approx(5.0 * 4.0, rel=1e-14)


def test_yaw_error_gives_c_yaw_plus_drift():
    p = base_params()
    v, th, dt = p["v_ref"], 0.1, p["dt"]
    S, _ = one_step(p, [0.0, 0.0, th, v])
    y1 = v * math.sin(th) * dt
    assert S == pytest.approx(15.0 * y1 ** 2 + 120.0 * th ** 2, rel=1e-12)


def test_moving_away_from_the_target_gives_c_target():
    p = base_params()
    # heading pi at the lane start: distance to the last vertex grows
    # (the yaw error pi - 0 sits on the wrap point; rint(1/2) = 0 keeps it at +pi, c_yaw = pi^2)
    S, _ = one_step(p, [5.0, 0.0, math.pi, p["v_ref"]])
    assert S == pytest.approx(7.0 + 120.0 * math.pi ** 2, rel=1e-14)
    # standing still: the distance to the target does not grow, so c_target = 0
    S2, _ = one_step(p, [5.0, 0.0, math.pi, 0.0])
    assert S2 == pytest.approx(120.0 * math.pi ** 2 + 5.0 * p["v_ref"] ** 2, rel=1e-12)


def test_obstacle_inside_the_safe_band_gives_c_safe():
    p = base_params()
    p.update(n_ego=1, ego_offset=[0.0], ego_radius=[1.0], d_safe_c=0.5, d_safe_0=1.0)
    v = p["v_ref"]
    x1 = v * p["dt"]
    # obstacle circle r = 1 placed 3-4-5 from the next position: d_obj = 5 - 1 - 1 = 3
    circ = [[x1 + 3.0, 4.0, 1.0, 0.0, 0.0]]
    S, _ = one_step(p, [0.0, 0.0, 0.0, v], circles=circ)
    d_safe = 0.5 * v + 1.0
    assert S == pytest.approx(25.0 * max(d_safe - 3.0, 0.0) ** 2, rel=1e-12)
    # collision-only variant: no cost while d_obj > 0 ...
    S, _ = one_step(dict(p, collision_only=1), [0.0, 0.0, 0.0, v], circles=circ)
    assert S == 0.0
    # ... and the full penalty once the circles overlap (d_obj = 5 - 3 - 3 = -1)
    circ_big = [[x1 + 3.0, 4.0, 3.0, 0.0, 0.0]]
    p3 = dict(p, collision_only=1, ego_radius=[3.0])
    S, _ = one_step(p3, [0.0, 0.0, 0.0, v], circles=circ_big)
    assert S == pytest.approx(25.0 * (d_safe + 1.0) ** 2, rel=1e-12)


def test_moving_obstacle_uses_position_at_step_t_plus_1():
    p = base_params()
    p.update(n_ego=1, ego_offset=[0.0], ego_radius=[0.0], d_safe_0=10.0)
    v = p["v_ref"]
    x1 = v * p["dt"]
    # circle starts 6 m ahead and moves back towards the car at 10 m/s: after dt it is 5 m from x1
    circ = [[x1 + 6.0, 0.0, 0.0, -10.0, 0.0]]
    S, _ = one_step(p, [0.0, 0.0, 0.0, v], circles=circ)
    assert S == pytest.approx(25.0 * (10.0 - 5.0) ** 2, rel=1e-12)
    # the same through an explicit per-step centre table
    S2, _ = one_step(p, [0.0, 0.0, 0.0, v], circles=[[0, 0, 0.0, 0, 0]], centres=np.array([[[x1 + 5.0, 0.0]]]))
    assert S2 == pytest.approx(S, rel=1e-14)


def test_control_cost_eq_8_9():
    p = base_params()
    v = p["v_ref"]
    u = np.array([0.5, 0.1])
    R = np.array([4.0, 400.0])
    p.update(R=list(R), sigma=[1.0, 0.1], gamma=2.0)        # alpha = (2-1)/(2*2) = 1/4
    z = np.array([0.2, -0.3])
    eps = np.array([1.0, 0.1]) * z
    S, ep = one_step(p, [0.0, 0.0, 0.0, v], U=u, z=z)
    np.testing.assert_allclose(ep[0], eps, rtol=1e-15)
    qu = 0.25 * eps @ (R * u) + u @ (R * eps) + 0.5 * u @ (R * u)
    # the controls also move the car: recover the state part from the sigma = 0 run
    S_state, _ = one_step(dict(p, sigma=[0.0, 0.0], R=[0.0, 0.0]), [0.0, 0.0, 0.0, v], U=u + eps)
    assert S == pytest.approx(S_state + qu, rel=1e-12)


def test_noise_check_clamps_to_the_control_box():
    p = base_params()
    p.update(sigma=[1.0, 1.0], R=[0.0, 0.0])
    u = np.array([2.5, 0.4])
    S, ep = one_step(p, [0.0, 0.0, 0.0, 5.0], U=u, z=[10.0, -10.0])
    np.testing.assert_allclose(ep[0], [3.0 - 2.5, -0.5 - 0.4], rtol=1e-15)


def test_speed_cap_limits_acceleration():
    p = base_params()
    p.update(v_max=10.0, R=[0.0, 0.0])
    x0 = [0.0, 0.0, 0.0, 9.9]
    S, _ = one_step(p, x0, U=[3.0, 0.0])
    # the car reaches exactly v_max: v1 = 10 -> c_speed = (10 - v_ref)^2
    assert S == pytest.approx(5.0 * (10.0 - p["v_ref"]) ** 2, rel=1e-12)
