"""Seeded synthetic planning problems shaped like the paper's driving workloads.

This module only *draws inputs*: an initial state, a reference polyline, obstacle
circles (with constant-velocity motion or a per-step centre table) and a
parameter dictionary.  It holds none of the planner's arithmetic (no dynamics,
no cost, no noise), so both the FP64 oracle and the CUDA path can consume the
same problem without sharing code.

Shapes follow the paper's setting (Sec. IV: a lane to follow, obstacles
approximated by circles, Fig. 3) and the five workloads this library is
measured on:

* ``single_plan``    K=1024,  T=50,  dt=0.05, straight 200-point lane, one
                     obstacle of 3 circles at x=20 m, 10 warm-started iterations.
* ``closed_loop``    K=8192,  T=100, dt=0.05, sinusoidal lane (A=3 m, 80 m
                     period, 1000 points), 8 obstacles x 3 circles, half moving
                     at constant velocity along the lane tangent.
* ``roofline``       K=65536, T=200, dt=0.025, straight 2000-point lane,
                     64 obstacles x 3 circles in a 200 m x 10 m corridor.
* ``batched``        256 uneven instances (K in 2^{10..14}, T in [30,150],
                     0..32 obstacles).
* ``serving``        512 sessions with sizes drawn like ``batched``.

Random numbers come from numpy's PCG64 seeded with ``seed*1000 + config_id``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# Table I of the paper and the cost weights of Eq. (20).
PAPER_WEIGHTS = dict(w_dist=15.0, w_target=7.0, w_yaw=120.0, w_speed=5.0, w_safe=25.0)
V_G = 30.0 / 3.6  # target speed v_G = 30 km/h (Table I)

CONFIG_IDS = {"single_plan": 1, "closed_loop": 2, "roofline": 3, "batched": 4, "serving": 5, "paper_preset": 6}


@dataclasses.dataclass
class Problem:
    """One planning problem: everything ``mppi_plan`` consumes."""

    params: Dict[str, object]
    x0: np.ndarray                 # (4,) float64: x, y, yaw, v
    ref: np.ndarray                # (n_ref, 2) float64 polyline vertices
    circles: np.ndarray            # (n_circ, 5) float64: x, y, r, vx, vy
    centres: Optional[np.ndarray] = None  # (T, n_circ, 2) float64 or None
    name: str = ""

    @property
    def K(self) -> int:
        return int(self.params["K"])

    @property
    def T(self) -> int:
        return int(self.params["T"])

    def copy(self) -> "Problem":
        return Problem(dict(self.params), self.x0.copy(), self.ref.copy(), self.circles.copy(),
                       None if self.centres is None else self.centres.copy(), self.name)


def default_params(K: int, T: int, dt: float, lam: float = 1.0,
                   sigma=(0.5, 0.05), u_min=(-3.0, -0.5), u_max=(3.0, 0.5),
                   gamma: float = 1.0) -> Dict[str, object]:
    """Parameter dictionary with the field names of ``mppi_params``.

    R defaults to lambda / sigma^2 per channel (the information-theoretic control
    weight of the MPPI derivation the paper builds on); gamma = 1 gives alpha = 0
    in the control cost of Eq. (9)-(10).
    """
    sa, sd = float(sigma[0]), float(sigma[1])
    return dict(
        K=int(K), T=int(T), dt=float(dt), wheelbase=2.7,
        sigma=[sa, sd], u_min=[float(u_min[0]), float(u_min[1])], u_max=[float(u_max[0]), float(u_max[1])],
        lam=float(lam), gamma=float(gamma),
        R=[lam / (sa * sa) if sa > 0 else 0.0, lam / (sd * sd) if sd > 0 else 0.0],
        w_terminal=0.0, v_ref=V_G, v_max=math.inf,
        d_safe_c=0.0, d_safe_0=0.5, collision_only=0,
        n_ego=3, ego_offset=[0.0, 1.35, 2.7], ego_radius=[1.1, 1.1, 1.1],
        ref_mode=0, sg_enable=1, shift=0, noise_bf16=0,
        seed=0, session=0, model=0, cost_to_go=0,
        **PAPER_WEIGHTS,
    )


def _rng(seed: int, config_id: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed * 1000 + config_id))


def straight_lane(n: int, spacing: float) -> np.ndarray:
    xs = spacing * np.arange(n, dtype=np.float64)
    return np.stack([xs, np.zeros(n)], axis=1)


def sinusoid_lane(n: int, spacing: float, amplitude: float, period: float) -> np.ndarray:
    xs = spacing * np.arange(n, dtype=np.float64)
    return np.stack([xs, amplitude * np.sin(2.0 * np.pi * xs / period)], axis=1)


def _lane_point_and_tangent(ref: np.ndarray, x: float):
    """Point on the lane polyline at abscissa x (the lanes here are graphs y(x))."""
    i = int(np.clip(np.searchsorted(ref[:, 0], x) - 1, 0, len(ref) - 2))
    a, b = ref[i], ref[i + 1]
    s = (x - a[0]) / (b[0] - a[0])
    p = a + s * (b - a)
    d = (b - a) / np.linalg.norm(b - a)
    return p, d


def obstacle_circles(rng: np.random.Generator, ref: np.ndarray, n_obs: int, x_range, lat_range,
                     r_range=(0.8, 1.2), spacing=1.5, speeds=None) -> np.ndarray:
    """n_obs car-like objects, each approximated by 3 circles along the lane tangent (Fig. 3)."""
    rows: List[List[float]] = []
    for j in range(n_obs):
        cx = rng.uniform(*x_range)
        lat = rng.uniform(*lat_range)
        r = rng.uniform(*r_range)
        p, d = _lane_point_and_tangent(ref, cx)
        nrm = np.array([-d[1], d[0]])
        centre = p + lat * nrm
        spd = 0.0 if speeds is None else float(speeds[j])
        for o in (-spacing, 0.0, spacing):
            c = centre + o * d
            rows.append([c[0], c[1], r, spd * d[0], spd * d[1]])
    return np.asarray(rows, dtype=np.float64).reshape(-1, 5)


def predicted_centres(circles: np.ndarray, T: int, dt: float) -> np.ndarray:
    """Per-step predicted centres of constant-velocity circles, table [T][n][2] for steps 1..T.

    This is the obstacle forecast handed to the planner (the paper's O^k_t of
    Eq. (17)); the planner itself only reads it.
    """
    steps = (np.arange(T, dtype=np.float64) + 1.0) * dt
    cx = circles[None, :, 0] + circles[None, :, 3] * steps[:, None]
    cy = circles[None, :, 1] + circles[None, :, 4] * steps[:, None]
    return np.stack([cx, cy], axis=2)


def single_plan(seed: int = 0) -> Problem:
    """K=1024, T=50, dt=0.05: straight lane, one static obstacle of 3 circles r=1 m at x=20 m."""
    p = default_params(1024, 50, 0.05, lam=1.0)
    p["seed"] = seed
    ref = straight_lane(200, 0.5)
    circles = np.array([[18.5, 0.0, 1.0, 0.0, 0.0],
                        [20.0, 0.0, 1.0, 0.0, 0.0],
                        [21.5, 0.0, 1.0, 0.0, 0.0]])
    return Problem(p, np.array([0.0, 0.0, 0.0, 8.0]), ref, circles, None, "single_plan")


def closed_loop(seed: int = 0) -> Problem:
    """K=8192, T=100, dt=0.05: sinusoidal lane, 8 obstacles x 3 circles, 4 of them moving."""
    rng = _rng(seed, CONFIG_IDS["closed_loop"])
    p = default_params(8192, 100, 0.05, lam=1.0)
    p["seed"] = seed
    ref = sinusoid_lane(1000, 0.5, 3.0, 80.0)
    speeds = np.concatenate([np.zeros(4), rng.uniform(0.0, 10.0, 4)])
    circles = obstacle_circles(rng, ref, 8, (20.0, 300.0), (-2.5, 2.5), speeds=speeds)
    centres = predicted_centres(circles, p["T"], p["dt"])
    return Problem(p, np.array([0.0, 0.0, math.atan2(ref[1, 1] - ref[0, 1], ref[1, 0] - ref[0, 0]), 8.0]),
                   ref, circles, centres, "closed_loop")


def roofline(seed: int = 0, bf16: bool = False) -> Problem:
    """K=65536, T=200, dt=0.025: straight 2000-point lane, 64 static obstacles x 3 circles."""
    rng = _rng(seed, CONFIG_IDS["roofline"])
    p = default_params(65536, 200, 0.025, lam=1.0)
    p["seed"] = seed
    p["noise_bf16"] = int(bf16)
    ref = straight_lane(2000, 0.1)
    circles = obstacle_circles(rng, ref, 64, (0.0, 200.0), (-5.0, 5.0))
    return Problem(p, np.array([0.0, 0.0, 0.0, 8.0]), ref, circles, None, "roofline")


def uneven_instance(rng: np.random.Generator, idx: int, seed: int = 0) -> Problem:
    """One instance of the batched/serving mix: K in 2^{10..14}, T in [30,150], 0..32 obstacles."""
    K = 1 << int(rng.integers(10, 15))
    T = int(rng.integers(30, 151))
    n_obs = int(rng.integers(0, 33))
    p = default_params(K, T, 0.05, lam=1.0)
    p["seed"] = seed
    p["session"] = idx
    if idx % 2 == 0:
        ref = straight_lane(1000, 0.5)
    else:
        ref = sinusoid_lane(1000, 0.5, 3.0, 80.0)
    v0 = float(rng.uniform(0.0, 15.0))
    circles = obstacle_circles(rng, ref, n_obs, (10.0, 300.0), (-4.0, 4.0))
    yaw0 = math.atan2(ref[1, 1] - ref[0, 1], ref[1, 0] - ref[0, 0])
    return Problem(p, np.array([0.0, float(rng.uniform(-1.0, 1.0)), yaw0, v0]), ref, circles, None,
                   f"batched[{idx}]")


def batched(seed: int = 0, n: int = 256) -> List[Problem]:
    rng = _rng(seed, CONFIG_IDS["batched"])
    return [uneven_instance(rng, i, seed) for i in range(n)]


def serving_sessions(seed: int = 0, n: int = 512) -> List[Problem]:
    rng = _rng(seed, CONFIG_IDS["serving"])
    return [uneven_instance(rng, i, seed) for i in range(n)]


def tiny(seed: int = 0, K: int = 8, T: int = 4, n_ref: int = 12, n_obs: int = 1,
         moving: bool = False) -> Problem:
    """A few samples and steps, for brute-force and invariant checks."""
    rng = _rng(seed, 90)
    p = default_params(K, T, 0.1, lam=1.0)
    p["seed"] = seed
    ref = sinusoid_lane(n_ref, 1.0, 1.0, 16.0)
    speeds = rng.uniform(0.0, 3.0, n_obs) if moving else None
    circles = obstacle_circles(rng, ref, n_obs, (2.0, float(n_ref - 2)), (-1.5, 1.5), speeds=speeds)
    return Problem(p, np.array([0.0, 0.2, 0.1, 4.0]), ref, circles, None, "tiny")


def paper_preset(seed: int = 0) -> Problem:
    """The paper's own setting (Table I) on the 5-state steering-rate model: M = 2560 samples,
    T = 16 steps of 0.25 s, lambda = 150, sigma = (0.85 m/s^2, 0.05 rad/s), |omega| <= 0.11,
    a in [-2.5, 1.1], d_safe = 1.36 v + 11, target speed 30 km/h as the speed cap.  A curved
    lane with two static objects of three circles each; state (x, y, yaw, v, delta)."""
    rng = _rng(seed, CONFIG_IDS["paper_preset"])
    p = default_params(2560, 16, 0.25, lam=150.0, sigma=(0.85, 0.05), u_min=(-2.5, -0.11), u_max=(1.1, 0.11))
    p.update(model=1, seed=seed, d_safe_c=1.36, d_safe_0=11.0, v_max=V_G)
    ref = sinusoid_lane(600, 0.5, 3.0, 80.0)
    circles = obstacle_circles(rng, ref, 2, (45.0, 90.0), (-3.0, 3.0))
    yaw0 = math.atan2(ref[1, 1] - ref[0, 1], ref[1, 0] - ref[0, 0])
    return Problem(p, np.array([0.0, 0.0, yaw0, 7.0, 0.0]), ref, circles, None, "paper_preset")


def car_circles(x: float, y: float, yaw: float = 0.0, speed: float = 0.0, length: float = 4.5,
                width: float = 1.8) -> np.ndarray:
    """A car-sized object as three circles along its length (Fig. 3), each the circle through
    the corners of a third of the car, moving at `speed` along its heading."""
    h = length / 6.0
    r = math.hypot(h, width / 2.0)
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[x + o * c, y + o * s, r, speed * c, speed * s] for o in (-2 * h, 0.0, 2 * h)])


def _primitive(seed: int, name: str) -> Problem:
    p = paper_preset(seed).params
    p["session"] = {"merge": 1, "follow": 2, "avoid": 3}[name]
    ref = straight_lane(800, 0.5)
    return p, ref


def scenario_merge(seed: int = 0) -> Problem:
    """Lane merge: the vehicle starts on a parallel lane 3.5 m to the right of the reference lane
    at 7 m/s and joins it; no objects."""
    p, ref = _primitive(seed, "merge")
    return Problem(p, np.array([0.0, -3.5, 0.0, 7.0, 0.0]), ref, np.zeros((0, 5)), None, "merge")


def scenario_follow(seed: int = 0) -> Problem:
    """Following: a car 30 m ahead in the lane drives at 4 m/s; the vehicle starts at 7 m/s.
    The speed-dependent safe distance d_safe = 1.36 v + 11 m makes it drop back."""
    p, ref = _primitive(seed, "follow")
    return Problem(p, np.array([0.0, 0.0, 0.0, 7.0, 0.0]), ref, car_circles(30.0, 0.0, 0.0, 4.0), None, "follow")


def scenario_avoid(seed: int = 0) -> Problem:
    """Object avoidance (the collision-only cost with a 0.7 m margin): a stopped car 40 m ahead
    reaches 1.0 m into the lane from the left."""
    p, ref = _primitive(seed, "avoid")
    p.update(collision_only=1, d_safe_c=0.0, d_safe_0=0.7)
    return Problem(p, np.array([0.0, 0.0, 0.0, 7.0, 0.0]), ref, car_circles(40.0, 1.9, 0.0, 0.0), None, "avoid")


def by_name(name: str, seed: int = 0) -> Problem:
    if name == "single_plan":
        return single_plan(seed)
    if name == "closed_loop":
        return closed_loop(seed)
    if name == "roofline":
        return roofline(seed)
    if name == "roofline_bf16":
        return roofline(seed, bf16=True)
    if name == "paper_preset":
        return paper_preset(seed)
    if name in ("merge", "follow", "avoid"):
        return {"merge": scenario_merge, "follow": scenario_follow, "avoid": scenario_avoid}[name](seed)
    raise KeyError(name)
