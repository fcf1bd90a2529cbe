"""The batched planner (mppi_batch_*) against the single-plan path and the oracle (needs a GB300).

A plan's result must not depend on the other plans of its submission: alone and in
a mix of uneven plans it is bit-identical.  Against the single-plan path it agrees to
rounding (the softmin normaliser is summed in a different order); against the FP64
oracle it meets the usual tolerances.
"""
import numpy as np
import pytest

import oracle
import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc
from parity import argmin_ok, assert_costs, assert_update

pytestmark = pytest.mark.gpu


def mixed_problems(n=12, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for i in range(n):
        p = sc.uneven_instance(rng, i, seed=seed)
        p.params["K"] = int(rng.choice([257, 1024, 1500, 4096]))
        p.params["T"] = int(rng.integers(5, 60))
        p.params["session"] = 100 + i
        probs.append(p)
    probs[1].centres = sc.predicted_centres(probs[1].circles, probs[1].T, probs[1].params["dt"])
    probs[2].circles = np.zeros((0, 5))
    return probs


def batch_for(probs, pipelines=2, bf16=0, max_T=128):
    return mp.BatchPlanner(max_slots=64, max_batch=64, max_samples=sum(p.K for p in probs) + 8,
                           max_rollout_steps=sum(p.K * p.T for p in probs) + 8, max_T=max_T, max_ref=1024,
                           max_circ=128, noise_bf16=bf16, pipelines=pipelines)


def c4_sized_problems(seed=41):
    """Plans at the sizes of the batched workload: K up to 2^14, T up to 150, up to 32 obstacles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [(16384, 150), (8192, 121), (1024, 30), (4096, 77), (2048, 143)]
    probs = []
    for i, (K, T) in enumerate(shapes):
        p = sc.uneven_instance(rng, i, seed=seed)
        p.params.update(K=K, T=T, session=200 + i)
        probs.append(p)
    probs[1].centres = sc.predicted_centres(probs[1].circles, probs[1].T, probs[1].params["dt"])
    return probs


def oracle_check(p, bpl, S):
    """A batched plan against the FP64 oracle: every sample cost, the argmin, u* and x*."""
    orc = oracle.plan(p)
    rep = assert_costs(S, orc.S, orc.margin)
    assert argmin_ok(bpl.info.argmin, orc.S), (bpl.info.argmin, orc.info.argmin)
    assert bpl.info.n_finite == orc.info.n_finite
    assert_update(bpl.u, bpl.x, orc)
    return rep


def plans_of(probs, slots=None):
    slots = list(range(len(probs))) if slots is None else slots
    return [mp.BatchPlan(p.params, s, p.x0, p.ref, p.circles, p.centres) for p, s in zip(probs, slots)]


def test_alone_and_in_the_mix_are_bit_identical():
    probs = mixed_problems()
    with batch_for(probs) as bp:
        mix = plans_of(probs)
        bp.plan(mix)
        for i in (0, 1, 2, 5, len(probs) - 1):
            bp.set_controls(i, np.zeros((probs[i].T, 2)), 0)
            alone = plans_of([probs[i]], [i])
            bp.plan(alone)
            np.testing.assert_array_equal(alone[0].u, mix[i].u)
            np.testing.assert_array_equal(alone[0].x, mix[i].x)
            assert alone[0].info.argmin == mix[i].info.argmin
            assert alone[0].info.s_min == mix[i].info.s_min
            assert alone[0].info.eta == mix[i].info.eta


@pytest.mark.parametrize("group,block", [(1, 128), (4, 256), (-2, 128), (-4, 448), (-8, 256)])
def test_every_launch_shape_gives_the_same_plans(group, block):
    """Lane splits of the work of a step and of the steps give bit-identical costs."""
    probs = mixed_problems(n=6)
    out = {}
    for gb in ((1, 64), (group, block)):
        with batch_for(probs) as bp:
            bp.set_launch(*gb)
            plans = plans_of(probs)
            bp.plan(plans)
            out[gb] = plans
    for a, b in zip(out[(1, 64)], out[(group, block)]):
        assert a.info.s_min == b.info.s_min and a.info.argmin == b.info.argmin
        np.testing.assert_array_equal(a.u, b.u)


def test_launch_shape_validation():
    probs = mixed_problems(n=3)
    with batch_for(probs) as bp:
        for g, b in ((3, 128), (-16, 448), (1, 480), (32, 256), (2, 100)):
            with pytest.raises(mp.MppiError) as e:
                bp.set_launch(g, b)
            assert e.value.status == -1


def test_batch_agrees_with_the_single_plan_path():
    probs = mixed_problems()
    with batch_for(probs) as bp:
        plans = plans_of(probs)
        bp.plan(plans)
    for p, bpl in zip(probs, plans):
        with mp.Planner(p.params) as pl:
            u, x, info = pl.plan(p.x0, p.ref, p.circles, p.centres)
        assert bpl.info.argmin == info["argmin"] and bpl.info.n_finite == info["n_finite"]
        assert bpl.info.s_min == info["s_min"]                       # same rollout arithmetic: same costs
        np.testing.assert_allclose(bpl.u, u, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(bpl.x, x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("K", [16384, 32768])
def test_weighted_sum_step_tiles_do_not_change_the_update(K):
    """The single-plan weighted sum tiles the steps by 2 (8 k-tiles) or 4 (16 k-tiles) at T = 100,
    the batch engine always by 8: the per-step partial sums do not depend on the tiling, so the two
    updates agree to the rounding of the normaliser (summed in a different order)."""
    rng = np.random.Generator(np.random.PCG64(29))
    p = sc.uneven_instance(rng, 0, seed=29)
    p.params.update(K=K, T=100, session=7)
    with batch_for([p]) as bp:
        plans = plans_of([p])
        bp.plan(plans)
    with mp.Planner(p.params) as pl:
        u, x, info = pl.plan(p.x0, p.ref, p.circles, p.centres)
    assert plans[0].info.argmin == info["argmin"] and plans[0].info.s_min == info["s_min"]
    np.testing.assert_allclose(plans[0].u, u, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(plans[0].x, x, rtol=1e-12, atol=1e-12)


def test_batch_matches_the_oracle():
    probs = mixed_problems(n=6)
    with batch_for(probs) as bp:
        plans = plans_of(probs)
        reqs = bp.requests(plans)        # kept alive: wait() writes each request's status
        t = bp.submit(reqs)
        bp.wait(t)
        S = [bp.get_costs(t, i, p.K) for i, p in enumerate(probs)]
    for p, bpl, s in zip(probs, plans, S):
        oracle_check(p, bpl, s)


@pytest.mark.slow
@pytest.mark.parametrize("bf16", [0, 1])
def test_batch_matches_the_oracle_at_batched_workload_sizes(bf16):
    """K up to 16384 and T up to 150 in one submission, noise in binary32 or bfloat16.  The bf16
    form is compared with the oracle on the same bf16-rounded noise (the same method), and its
    error against the unrounded FP64 method is reported."""
    probs = c4_sized_problems()
    for p in probs:
        p.params["noise_bf16"] = bf16
    with batch_for(probs, bf16=bf16, max_T=160) as bp:
        plans = plans_of(probs)
        reqs = bp.requests(plans)        # kept alive: wait() writes each request's status
        t = bp.submit(reqs)
        bp.wait(t)
        S = [bp.get_costs(t, i, p.K) for i, p in enumerate(probs)]
    for p, bpl, s in zip(probs, plans, S):
        rep = oracle_check(p, bpl, s)
        line = f"K={p.K} T={p.T} n_circ={p.circles.shape[0]}: max rel S err {rep['max_rel_all']:.2e}"
        if bf16:
            full = oracle.plan(p, params=dict(p.params, noise_bf16=0))
            rel = np.abs(s - full.S) / np.maximum(np.abs(full.S), 1.0)
            line += (f"; vs the unrounded FP64 method: max rel S err {rel.max():.2e}, "
                     f"|du*| {np.abs(bpl.u - full.u_star).max():.2e}")
        print(line)


def test_batch_costs_view_errors():
    probs = mixed_problems(n=3)[:2]
    with batch_for(probs) as bp:
        plans = plans_of(probs)
        reqs = bp.requests(plans)        # kept alive: wait() writes each request's status
        t = bp.submit(reqs)
        with pytest.raises(mp.MppiError) as e:           # still in flight
            bp.get_costs(t, 0, probs[0].K)
        assert e.value.status == -6
        bp.wait(t)
        for i, K in ((0, probs[0].K + 1), (2, probs[0].K), (-1, probs[0].K)):
            with pytest.raises(mp.MppiError) as e:
                bp.get_costs(t, i, K)
            assert e.value.status == -1


def test_warm_starts_persist_in_the_slots():
    probs = mixed_problems(n=4)
    for p in probs:
        p.params["shift"] = 1
    with batch_for(probs) as bp:
        plans = plans_of(probs)
        bp.plan(plans)
        bp.plan(plans)
        for i, p in enumerate(probs):
            U, it = bp.get_controls(i, p.T)
            assert it == 2 and plans[i].info.iter == 1
    for p, bpl in zip(probs, plans):
        with mp.Planner(p.params) as pl:
            pl.plan(p.x0, p.ref, p.circles, p.centres)
            u, x, info = pl.plan(p.x0, p.ref, p.circles, p.centres)
        np.testing.assert_allclose(bpl.u, u, rtol=1e-12, atol=1e-14)


def test_two_submissions_in_flight():
    probs = mixed_problems(n=8)
    with batch_for(probs, pipelines=2) as bp:
        a, b = plans_of(probs[:4], [0, 1, 2, 3]), plans_of(probs[4:], [4, 5, 6, 7])
        ra, rb = bp.requests(a), bp.requests(b)
        ta = bp.submit(ra)
        tb = bp.submit(rb)
        with pytest.raises(mp.MppiError) as e:          # both pipelines busy
            bp.submit(bp.requests(plans_of(probs[:1], [9])))
        assert e.value.status == -6
        bp.wait(tb)
        bp.wait(ta)
        for i in range(8):
            bp.set_controls(i, np.zeros((probs[i].T, 2)), 0)
        seq = plans_of(probs)
        bp.plan(seq)
    for x, y in zip(a + b, seq):
        np.testing.assert_array_equal(x.u, y.u)


def test_autotune_leaves_the_slots_and_is_used():
    probs = mixed_problems(n=6)
    with batch_for(probs) as bp:
        U0 = np.full((probs[0].T, 2), 0.01)
        bp.set_controls(0, U0, 4)
        g, b = bp.autotune(plans_of(probs))
        assert g in (1, 2, 4, 8, 16, 32, -2, -4, -8) and b in (64, 128, 256, 448)
        U, it = bp.get_controls(0, probs[0].T)
        np.testing.assert_array_equal(U, U0)
        assert it == 4
        plans = plans_of(probs)
        bp.plan(plans)
        assert plans[0].info.iter == 4
    with mp.Planner(probs[3].params) as pl:
        u, x, info = pl.plan(probs[3].x0, probs[3].ref, probs[3].circles, probs[3].centres)
    np.testing.assert_allclose(plans[3].u, u, rtol=1e-12, atol=1e-14)


def test_batch_errors():
    probs = mixed_problems(n=3)
    with batch_for(probs) as bp:
        with pytest.raises(mp.MppiError) as e:
            bp.plan(plans_of(probs, [0, 0, 1]))         # slot used twice
        assert e.value.status == -1
        bad = probs[1].copy()
        bad.ref[2, 0] = np.nan
        with pytest.raises(mp.MppiError) as e:
            bp.plan(plans_of([probs[0], bad], [0, 1]))
        assert e.value.status == -1
        big = probs[0].copy()
        big.params["T"] = 500                            # above max_T
        with pytest.raises(mp.MppiError) as e:
            bp.plan(plans_of([big], [0]))
        assert e.value.status == -6
        # the batch is still usable
        plans = plans_of(probs)
        bp.plan(plans)
        assert all(p.info.n_finite > 0 for p in plans)
