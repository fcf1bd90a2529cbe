"""Receding-horizon closed loop around the planner (the paper's Algorithm 1 outer loop).

Each cycle: plan one MPPI iteration from the current state (``mppi_plan``, warm start
shifted by the library), apply the first smoothed control u*_0 for one step to the
"true" vehicle, move the obstacles on, repeat.  The true vehicle and the obstacle
motion are the environment of the loop (a plain binary64 Euler step of the bicycle
model and constant velocities); the planning itself runs in the CUDA library.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import Planner
from .scenarios import Problem, predicted_centres


@dataclass
class LoopResult:
    states: np.ndarray            # [cycles + 1][4] true vehicle states
    controls: np.ndarray          # [cycles][2] applied controls u*_0 ((a, delta), or (a, omega) for model 1)
    plan_ms: np.ndarray           # [cycles] wall time of each mppi_plan call
    min_clearance: float          # smallest ego-circle / obstacle-circle clearance over the run (m)
    statuses: List[int] = field(default_factory=list)


def vehicle_step(x: np.ndarray, a: float, delta: float, dt: float, wheelbase: float) -> np.ndarray:
    """The environment's vehicle: one explicit Euler step of the kinematic bicycle."""
    px, py, th, v = x
    return np.array([px + v * math.cos(th) * dt, py + v * math.sin(th) * dt,
                     th + v * math.tan(delta) / wheelbase * dt, v + a * dt])


def vehicle5_step(x: np.ndarray, a: float, omega: float, dt: float, wheelbase: float) -> np.ndarray:
    """The environment's vehicle in the steering-rate form: the steering angle is a state
    driven by the applied rate."""
    return np.concatenate([vehicle_step(x[:4], a, x[4], dt, wheelbase), [x[4] + omega * dt]])


def applied_accel(p: dict, a: float, v: float) -> float:
    """The speed cap of the plans applies to the vehicle too: a <= (v_max - v) / dt."""
    vmax = float(p["v_max"])
    if math.isfinite(vmax):
        a = max(min(a, (vmax - v) / float(p["dt"])), float(p["u_min"][0]))
    return a


def clearance(p: dict, x: np.ndarray, circles: np.ndarray) -> float:
    """Smallest gap between the ego circles at state x and the obstacle circles."""
    if circles.shape[0] == 0:
        return math.inf
    best = math.inf
    for e in range(int(p["n_ego"])):
        ex = x[0] + p["ego_offset"][e] * math.cos(x[2])
        ey = x[1] + p["ego_offset"][e] * math.sin(x[2])
        d = np.hypot(circles[:, 0] - ex, circles[:, 1] - ey) - circles[:, 2] - p["ego_radius"][e]
        best = min(best, float(d.min()))
    return best


def run(prob: Problem, cycles: int = 200, device: int = 0, use_table: Optional[bool] = None,
        planner: Optional[Planner] = None) -> LoopResult:
    p = dict(prob.params, shift=1)
    dt, L = float(p["dt"]), float(p["wheelbase"])
    use_table = prob.centres is not None if use_table is None else use_table
    own = planner is None
    pl = Planner(p, device=device) if own else planner
    x = prob.x0.astype(np.float64).copy()
    circ = prob.circles.astype(np.float64).copy()
    states, controls, times, statuses = [x.copy()], [], [], []
    min_clear = clearance(p, x, circ)
    try:
        for _ in range(cycles):
            cen = predicted_centres(circ, int(p["T"]), dt) if use_table else None
            t0 = time.perf_counter()
            u, xs, info = pl.plan(x, prob.ref, circ, cen)
            times.append((time.perf_counter() - t0) * 1e3)
            statuses.append(0)
            a, d = float(u[0, 0]), float(u[0, 1])
            controls.append((a, d))
            a = applied_accel(p, a, x[3])
            x = vehicle5_step(x, a, d, dt, L) if int(p.get("model", 0)) == 1 else vehicle_step(x, a, d, dt, L)
            circ[:, 0] += circ[:, 3] * dt
            circ[:, 1] += circ[:, 4] * dt
            states.append(x.copy())
            min_clear = min(min_clear, clearance(p, x, circ))
    finally:
        if own:
            pl.close()
    return LoopResult(np.array(states), np.array(controls), np.array(times), min_clear, statuses)
