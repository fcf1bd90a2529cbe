"""Scenario primitives as closed loops on the steering-rate model with the paper's Table I
preset (needs a GB300).  The paper reports these experiments as figures only, so the checks
are qualitative gates: no collision, speed within the target speed v_G, controls within their
bounds, and the behaviour each scenario is about (joining the lane, dropping back behind a
slower car, passing a car that reaches into the lane).
"""
import math

import numpy as np
import pytest

from paper_2308_01654_gb300 import closed_loop
from paper_2308_01654_gb300 import scenarios as sc

pytestmark = pytest.mark.gpu

CYCLES = 160          # 40 s of 0.25 s cycles


def run(prob, cycles=CYCLES):
    res = closed_loop.run(prob, cycles=cycles)
    p = prob.params
    xs, us = res.states, res.controls
    assert np.isfinite(xs).all()
    assert xs[:, 3].max() <= p["v_max"] + 1e-9                       # v <= v_G (the speed cap)
    assert np.all(us[:, 0] >= p["u_min"][0] - 1e-12) and np.all(us[:, 0] <= p["u_max"][0] + 1e-12)
    assert np.all(np.abs(us[:, 1]) <= p["u_max"][1] + 1e-12)        # |omega| <= omega_max
    return res


def test_lane_merge_joins_the_reference_lane():
    res = run(sc.scenario_merge())
    y = res.states[:, 1]
    assert abs(y[-1]) < 0.1 and abs(y[0] + 3.5) < 1e-12
    assert np.abs(res.states[:, 4]).max() < 0.1                       # gentle steering
    assert y.min() > -3.6 and y.max() < 0.6                           # never moves away; overshoot (steering-rate limited) under 0.6 m


def test_following_drops_back_behind_the_slower_car():
    res = run(sc.scenario_follow())
    assert res.min_clearance > 10.0
    assert abs(res.states[-1, 3] - 4.0) < 0.1                         # settles at the lead car's speed
    assert abs(res.states[-1, 1]) < 0.1                               # stays in the lane


def test_avoidance_with_the_papers_weights_grazes_at_most():
    # With the paper's weights (w_dist = 15, w_safe = 25) the cost of leaving the lane by the
    # ~1.1 m that clears the car and its 0.7 m band is about that of touching it, so the plans
    # pass it with a few centimetres of contact, in both the band form and the collision-only
    # form; recorded here as a property of those weights.
    for collision_only in (0, 1):
        prob = sc.scenario_avoid()
        prob.params["collision_only"] = collision_only
        res = run(prob)
        assert res.min_clearance > -0.05, collision_only
        assert res.states[-1, 0] > 60.0                               # got past the car at x = 40 m
        assert abs(res.states[-1, 1]) < 0.3                           # and back in the lane


def test_avoidance_passes_without_contact_when_safety_outweighs_the_lane():
    prob = sc.scenario_avoid()
    prob.params.update(collision_only=0, w_safe=250.0)               # band form, safety weighted 10x
    res = run(prob)
    assert res.min_clearance > 0.0
    assert res.states[:, 1].min() < -0.3                              # it moved away from the car
    assert abs(res.states[-1, 1]) < 0.3                               # and came back to the lane
