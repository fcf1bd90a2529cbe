"""Full-size parity on the roofline workload (K=65536, T=200, 2000-point lane, 192 circles).

The CUDA path runs in the launch configuration the benchmark times; the oracle
computes every one of the 65536 sample costs (brute-force reference search,
binary64) on the host cores, so costs, argmin, u* and x* are compared in full.
The BF16-noise form is compared with the oracle's bf16-rounded noise, and its
error against the unrounded FP64 oracle is reported.
"""
import numpy as np
import pytest

import oracle
import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc
from parity import argmin_ok, assert_costs, assert_update

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("bf16", [False, True])
def test_roofline_workload_full_parity(bf16):
    prob = sc.roofline(bf16=bf16)
    with mp.Planner(prob.params) as pl:
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
        S = pl.get_costs()
        z = pl.get_noise() if bf16 else None
    orc = oracle.plan(prob)
    if bf16:
        # every one of the 26.2 million bfloat16 codes is the rounding of the exact normal
        zo = oracle.noise(prob.params, info["iter"])
        mism = int(np.count_nonzero(z.astype(np.float64) != zo))
        assert mism == 0, mism
        del z, zo
    rep = assert_costs(S, orc.S, orc.margin)
    assert argmin_ok(info["argmin"], orc.S)
    assert_update(u, x, orc)
    if bf16:
        # the stated error of the BF16 form against the unrounded FP64 method
        p64 = dict(prob.params, noise_bf16=0)
        full = oracle.plan(prob, params=p64)
        rel = np.abs(S - full.S) / np.maximum(np.abs(full.S), 1.0)
        print(f"bf16 form vs fp64 oracle: max rel S err {rel.max():.3e}, median {np.median(rel):.3e}, "
              f"|du*| {np.abs(u - full.u_star).max():.3e}, argmin {info['argmin']} vs {full.info.argmin}")
    print("roofline", "bf16" if bf16 else "fp32", rep)


@pytest.mark.parametrize("group", [0, -4])
def test_maximum_sizes_parity(group):
    """Every capacity at its maximum at once: T = MPPI_MAX_T steps, MPPI_MAX_REF reference points,
    MPPI_MAX_CIRC obstacle circles (the shared-memory scene then fills a block's 227 KB almost
    entirely), moving obstacles with a per-step centre table."""
    rng = np.random.default_rng(11)
    T, n_ref, n_circ = 1024, 4096, 1024
    p = sc.default_params(192, T, 0.01)
    p.update(group=group, seed=3)
    ref = sc.sinusoid_lane(n_ref, 0.05, 1.5, 60.0)
    circles = sc.obstacle_circles(rng, ref, n_circ // 3, (5.0, 200.0), (-4.0, 4.0),
                                  speeds=rng.uniform(0.0, 4.0, n_circ // 3))
    circles = np.concatenate([circles, [[30.0, 2.5, 1.0, 0.0, 0.0]]])
    assert circles.shape[0] == n_circ
    prob = sc.Problem(p, np.array([0.0, 0.0, 0.0, 8.0]), ref, circles, sc.predicted_centres(circles, T, p["dt"]),
                      "max_sizes")
    with mp.Planner(p, max_ref=n_ref, max_circ=n_circ) as pl:
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
        S = pl.get_costs()
    orc = oracle.plan(prob)
    # 1024 steps over 0.05 m segments pass within 1e-5 m of some segment switch in about a third of
    # the rollouts; every sample, near a jump or not, must meet the cost tolerance
    rep = assert_costs(S, orc.S, orc.margin)
    assert argmin_ok(info["argmin"], orc.S)
    assert_update(u, x, orc)
    print("maximum sizes", group, rep)
