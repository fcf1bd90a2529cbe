"""Pins for the per-step (cost-to-go) reading of the update, Eq. (11) with S(tau_{t,m}):
the weights of step t come from each sample's cost from step t on.

Expected values come from brute force on the definitions, the T = 1 reduction to the
whole-cost update, and the softmin limits.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01654_gb300 import scenarios as sc


def test_cost_from_each_step_is_the_suffix_sum_of_the_step_costs():
    prob = sc.tiny(K=4, T=9, n_ref=20, n_obs=2, moving=True)
    p = dict(prob.params, w_terminal=3.0)
    z = np.random.default_rng(0).normal(size=(prob.T, 2))
    U = np.zeros((prob.T, 2))                 # u = 0: the control cost of Eq. (8) is 0, every step cost >= 0
    S, ctg, _ = oracle.rollout_cost_ctg(p, prob.x0, U, z, prob.ref, prob.circles)
    assert ctg[0] == pytest.approx(S, rel=1e-14)          # the whole cost, summed from the other end
    assert np.all(np.diff(ctg) <= 1e-12)                  # sums of fewer non-negative terms
    # shortening the horizon to the first m steps leaves the costs of those steps unchanged, so
    # the cost of steps 0..m-1 is S(T) - ctg[m] (terminal cost off to compare the two)
    p0 = dict(p, w_terminal=0.0)
    S_full, ctg_full, _ = oracle.rollout_cost_ctg(p0, prob.x0, U, z, prob.ref, prob.circles)
    for m in (1, 4, 8):
        Sm, _, _ = oracle.rollout_cost_ctg(dict(p0, T=m), prob.x0, U[:m], z[:m], prob.ref, prob.circles)
        assert Sm == pytest.approx(S_full - ctg_full[m], rel=1e-12, abs=1e-12)


def test_one_step_reduces_to_the_whole_cost_update():
    rng = np.random.default_rng(2)
    K = 50
    S = rng.normal(size=K) * 3.0
    eps = rng.normal(size=(1, K, 2))
    dU, w, info = oracle.softmin_update(S, eps, 0.7)
    dU2, eta = oracle.softmin_update_ctg(S[None, :], eps, 0.7)
    np.testing.assert_allclose(dU2, dU, rtol=1e-14, atol=1e-15)
    assert eta[0] == pytest.approx(info.eta, rel=1e-14)


def test_each_step_is_a_softmin_over_its_own_costs():
    rng = np.random.default_rng(3)
    T, K, lam = 6, 40, 1.3
    Sctg = np.cumsum(rng.uniform(0, 2, size=(T, K))[::-1], axis=0)[::-1]      # suffix sums
    eps = rng.normal(size=(T, K, 2))
    dU, eta = oracle.softmin_update_ctg(Sctg, eps, lam)
    for t in range(T):
        w = np.exp(-(Sctg[t] - Sctg[t].min()) / lam)
        np.testing.assert_allclose(dU[t], (w[:, None] * eps[t]).sum(axis=0) / w.sum(), rtol=1e-13, atol=1e-15)
        assert eta[t] == pytest.approx(w.sum(), rel=1e-13)


def test_lambda_limits_per_step():
    rng = np.random.default_rng(4)
    T, K = 5, 30
    Sctg = rng.uniform(0, 10, size=(T, K))
    eps = rng.normal(size=(T, K, 2))
    d0, _ = oracle.softmin_update_ctg(Sctg, eps, 1e-300)
    dinf, _ = oracle.softmin_update_ctg(Sctg, eps, 1e300)
    for t in range(T):
        np.testing.assert_array_equal(d0[t], eps[t, np.argmin(Sctg[t])])        # best sample of step t
    np.testing.assert_allclose(dinf, eps.mean(axis=1), rtol=1e-12, atol=1e-15)


def test_plan_with_cost_to_go_uses_the_per_step_weights():
    prob = sc.tiny(K=64, T=10, n_ref=30, n_obs=2, moving=True)
    prob.params.update(cost_to_go=1, sg_enable=0)
    U0 = np.random.default_rng(5).normal(size=(prob.T, 2)) * [0.3, 0.03]
    r = oracle.plan(prob, U=U0, want_eps=True)
    assert r.rc == 0
    # rebuild the per-step costs sample by sample with the same noise and check the update
    z = oracle.noise(prob.params, 0)
    Sctg = np.empty((prob.T, prob.K))
    for k in range(prob.K):
        S, ctg, _ = oracle.rollout_cost_ctg(prob.params, prob.x0, U0, z[:, k], prob.ref, prob.circles)
        Sctg[:, k] = ctg
        assert S == r.S[k]
    dU, _ = oracle.softmin_update_ctg(Sctg, r.eps, prob.params["lam"])
    lo, hi = prob.params["u_min"], prob.params["u_max"]
    np.testing.assert_allclose(r.u_star, np.clip(U0 + dU, lo, hi), rtol=1e-14, atol=1e-15)
    # and it differs from the whole-cost update (the reading matters)
    prob.params["cost_to_go"] = 0
    r0 = oracle.plan(prob, U=U0)
    assert np.abs(r0.u_star - r.u_star).max() > 1e-6
