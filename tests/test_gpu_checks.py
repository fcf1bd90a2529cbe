"""The bounds-checking debug build (libmppi_checks.so, -DMPPI_CHECKS) on the small parity cases.

In that build every index the rollout kernels read from the staged scene, the circle index,
the controls and the centre table is tested against its array's length, and every block's
dynamic shared memory against the scene it stages; a violation is counted and the read kept
in bounds (nothing traps).  Each case below must match the FP64 oracle and leave no violation;
the self-test shows the checks are live (its two out-of-range indices are counted).
"""
import numpy as np
import pytest

import oracle
import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import _build
from paper_2308_01654_gb300 import scenarios as sc
from parity import argmin_ok, assert_costs, assert_update

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checks_lib():
    L = mp.load_library(_build.build(checks=True))
    with mp.use_library(L):
        enabled, _ = mp.check_hits()          # also resets the counters
        assert enabled
        yield L


def plan_and_check(prob, U=None, params=None):
    p = prob.params if params is None else params
    with mp.Planner(p) as pl:
        if U is not None:
            pl.set_controls(U, 0)
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
        S = pl.get_costs()
    orc = oracle.plan(prob, U=U, params=p)
    assert_costs(S, orc.S, orc.margin)
    assert argmin_ok(info["argmin"], orc.S)
    assert_update(u, x, orc)
    assert mp.check_hits() == (True, 0)


def test_the_checks_are_live(checks_lib):
    assert mp.check_selftest() == 2
    assert mp.check_hits() == (True, 0)


@pytest.mark.parametrize("group", [0, 1, 4, 32, -2, -4, -16])
def test_single_plan(checks_lib, group):
    prob = sc.single_plan()
    prob.params.update(K=777, T=33, group=group)
    plan_and_check(prob)


@pytest.mark.parametrize("variant", ["vertex", "moving_table", "moving_velocity", "no_obstacles", "two_point_ref",
                                     "curved_lane", "paper_preset", "cost_to_go", "bf16"])
def test_variants(checks_lib, variant):
    if variant == "curved_lane":
        prob = sc.closed_loop()
        prob.params.update(K=2048)
    elif variant == "paper_preset":
        prob = sc.paper_preset()
    else:
        prob = sc.tiny(K=1500, T=25, n_ref=60, n_obs=3, moving=variant.startswith("moving"))
        prob.params["d_safe_0"] = 2.0
    if variant == "vertex":
        prob.params["ref_mode"] = 1
    elif variant == "moving_table":
        prob.centres = sc.predicted_centres(prob.circles, prob.T, prob.params["dt"])
    elif variant == "no_obstacles":
        prob.circles = np.zeros((0, 5))
    elif variant == "two_point_ref":
        prob.ref = np.array([[-5.0, 0.0], [30.0, 1.0]])
    elif variant == "cost_to_go":
        prob.params["cost_to_go"] = 1
    elif variant == "bf16":
        prob.params["noise_bf16"] = 1
    plan_and_check(prob)


def test_maximum_capacities(checks_lib):
    """Every capacity at its maximum (the staged scene nearly fills a block's shared memory)."""
    rng = np.random.default_rng(11)
    T, n_ref, n_circ = 1024, 4096, 1024
    p = sc.default_params(96, T, 0.01)
    p.update(group=-4, seed=3)
    ref = sc.sinusoid_lane(n_ref, 0.05, 1.5, 60.0)
    circles = sc.obstacle_circles(rng, ref, n_circ // 3, (5.0, 200.0), (-4.0, 4.0),
                                  speeds=rng.uniform(0.0, 4.0, n_circ // 3))
    circles = np.concatenate([circles, [[30.0, 2.5, 1.0, 0.0, 0.0]]])
    prob = sc.Problem(p, np.array([0.0, 0.0, 0.0, 8.0]), ref, circles, sc.predicted_centres(circles, T, p["dt"]),
                      "max_sizes")
    with mp.Planner(p, max_ref=n_ref, max_circ=n_circ) as pl:
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
        S = pl.get_costs()
    orc = oracle.plan(prob)
    assert_costs(S, orc.S, orc.margin)
    assert_update(u, x, orc)
    assert mp.check_hits() == (True, 0)


def test_batch_engine(checks_lib):
    rng = np.random.Generator(np.random.PCG64(3))
    probs = []
    for i in range(6):
        p = sc.uneven_instance(rng, i, seed=3)
        p.params.update(K=int(rng.choice([257, 1024, 2048])), T=int(rng.integers(5, 60)), session=100 + i)
        probs.append(p)
    probs[1].centres = sc.predicted_centres(probs[1].circles, probs[1].T, probs[1].params["dt"])
    probs[2].circles = np.zeros((0, 5))
    with mp.BatchPlanner(max_slots=8, max_batch=8, max_samples=sum(p.K for p in probs),
                         max_rollout_steps=sum(p.K * p.T for p in probs), max_T=64, max_ref=1024,
                         max_circ=128) as bp:
        plans = [mp.BatchPlan(p.params, i, p.x0, p.ref, p.circles, p.centres) for i, p in enumerate(probs)]
        reqs = bp.requests(plans)
        t = bp.submit(reqs)
        bp.wait(t)
        S = [bp.get_costs(t, i, p.K) for i, p in enumerate(probs)]
    for p, bpl, s in zip(probs, plans, S):
        orc = oracle.plan(p)
        assert_costs(s, orc.S, orc.margin)
        assert_update(bpl.u, bpl.x, orc)
    assert mp.check_hits() == (True, 0)
