"""Pins for the oracle's update (Eq. (11)), smoothing (Eq. (19)) and whole iteration (Algorithm 1).

Expected values come from limits, invariances and closed forms of the method,
and from the Savitzky-Golay coefficients printed in the paper.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import golden_constants
from paper_2308_01654_gb300 import scenarios as sc


# ---------------------------------------------------------------- Eq. (11) softmin update

def rand_eps(T, K, seed=0):
    return np.random.default_rng(seed).normal(size=(T, K, 2))


def test_weights_normalise_and_argmin_has_weight_one():
    S = np.array([3.0, 1.0, 2.0, 1.0 + 1e-9, 5.0])
    eps = rand_eps(3, 5)
    dU, w, info = oracle.softmin_update(S, eps, lam=0.7)
    assert info.argmin == 1 and info.s_min == 1.0 and info.n_finite == 5
    assert w[1] == 1.0 and info.eta == pytest.approx(w.sum(), rel=1e-15)
    np.testing.assert_allclose(w, np.exp(-(S - 1.0) / 0.7), rtol=1e-15)
    np.testing.assert_allclose(dU, np.einsum("k,tkc->tc", w / w.sum(), eps), rtol=1e-13)


def test_ties_pick_the_lowest_index():
    S = np.array([2.0, 1.0, 1.0, 1.0])
    _, _, info = oracle.softmin_update(S, rand_eps(2, 4), 1.0)
    assert info.argmin == 1


def test_two_samples_closed_form():
    lam = 2.0
    S = np.array([0.0, lam * math.log(2.0)])          # weights 1 and 1/2
    eps = rand_eps(4, 2, seed=3)
    dU, _, info = oracle.softmin_update(S, eps, lam)
    np.testing.assert_allclose(dU, (eps[:, 0] + 0.5 * eps[:, 1]) / 1.5, rtol=1e-14)
    assert info.eta == pytest.approx(1.5, rel=1e-15)


def test_lambda_to_zero_returns_the_argmin_perturbation():
    S = np.array([4.0, 3.0, 3.5, 9.0])
    eps = rand_eps(5, 4, seed=1)
    dU, _, _ = oracle.softmin_update(S, eps, 1e-300)
    np.testing.assert_array_equal(dU, eps[:, 1])


def test_lambda_to_infinity_returns_the_mean_perturbation():
    S = np.array([4.0, 3.0, 3.5, 9.0])
    eps = rand_eps(5, 4, seed=2)
    dU, _, _ = oracle.softmin_update(S, eps, 1e300)
    np.testing.assert_allclose(dU, eps.mean(axis=1), rtol=1e-14)


def test_equal_costs_return_the_mean():
    eps = rand_eps(3, 6, seed=4)
    dU, _, _ = oracle.softmin_update(np.full(6, 17.0), eps, 0.01)
    np.testing.assert_allclose(dU, eps.mean(axis=1), rtol=1e-14)


def test_shift_invariance_of_the_softmin():
    S = np.array([4.0, 3.0, 3.5, 9.0])
    eps = rand_eps(2, 4, seed=5)
    a, _, _ = oracle.softmin_update(S, eps, 1.3)
    b, _, _ = oracle.softmin_update(S + 1000.0, eps, 1.3)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_non_finite_costs_weigh_zero():
    S = np.array([np.inf, 2.0, np.nan, 3.0])
    eps = rand_eps(2, 4, seed=6)
    dU, w, info = oracle.softmin_update(S, eps, 1.0)
    assert info.n_finite == 2 and info.argmin == 1 and w[0] == 0.0 and w[2] == 0.0
    ww = np.array([0.0, 1.0, 0.0, math.exp(-1.0)])
    np.testing.assert_allclose(dU, np.einsum("k,tkc->tc", ww / ww.sum(), eps), rtol=1e-14)
    _, _, info = oracle.softmin_update(np.full(3, np.inf), rand_eps(2, 3), 1.0)
    assert info.n_finite == 0


# ---------------------------------------------------------------- Eq. (19) Savitzky-Golay

def test_sg_impulse_response_is_the_papers_coefficients():
    g = golden_constants()
    num = np.array([g["sg_num_m2"], g["sg_num_m1"], g["sg_num_0"], g["sg_num_p1"], g["sg_num_p2"]])
    u = np.zeros(11)
    u[5] = 1.0
    out = oracle.savgol5(u)
    np.testing.assert_allclose(out[3:8], num[::-1] / g["sg_den"], rtol=1e-15)   # symmetric filter
    assert np.all(out[:3] == 0.0) and np.all(out[8:] == 0.0)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_sg_reproduces_cubics_in_the_interior(deg):
    t = np.arange(20, dtype=float)
    c = np.random.default_rng(deg).normal(size=deg + 1)
    u = np.polyval(c, t / 10.0)
    out = oracle.savgol5(u)
    np.testing.assert_allclose(out[2:-2], u[2:-2], rtol=1e-12, atol=1e-12)


def test_sg_keeps_constants_at_the_edges_and_short_sequences():
    for T in (1, 2, 3, 4, 7):
        np.testing.assert_allclose(oracle.savgol5(np.full(T, 0.37)), 0.37, rtol=1e-15)
    assert oracle.savgol5(np.array([2.0]))[0] == pytest.approx(2.0)
    # edge replicate: first output uses u0,u0,u0,u1,u2
    u = np.array([1.0, 2.0, 4.0, 8.0, 16.0, 32.0])
    out = oracle.savgol5(u)
    assert out[0] == pytest.approx((-3 * 1 + 12 * 1 + 17 * 1 + 12 * 2 - 3 * 4) / 35.0)
    assert out[-1] == pytest.approx((-3 * 8 + 12 * 16 + 17 * 32 + 12 * 32 - 3 * 32) / 35.0)


# ---------------------------------------------------------------- Algorithm 1, one iteration

def small_problem(**kw):
    prob = sc.tiny(K=64, T=12, n_ref=30, n_obs=2, moving=True)
    prob.params.update(kw)
    return prob


def test_x_star_is_the_noise_free_rollout_of_u_star():
    prob = small_problem()
    r = oracle.plan(prob)
    assert r.rc == 0
    xs = [prob.x0]
    for t in range(prob.T):
        xs.append(oracle.bicycle_step(xs[-1], r.u_star[t, 0], r.u_star[t, 1], prob.params["dt"], 2.7))
    np.testing.assert_allclose(r.x_star, np.array(xs), rtol=1e-15, atol=1e-15)


def test_zero_noise_leaves_the_controls_to_the_smoother():
    prob = small_problem(sigma=[0.0, 0.0])
    U0 = np.random.default_rng(1).normal(size=(prob.T, 2)) * [0.5, 0.05]
    r = oracle.plan(prob, U=U0)
    assert np.all(r.S == r.S[0]) and r.info.argmin == 0
    sm = np.stack([oracle.savgol5(U0[:, c]) for c in range(2)], axis=1)
    lo, hi = np.array(prob.params["u_min"]), np.array(prob.params["u_max"])
    np.testing.assert_allclose(r.u_star, np.clip(sm, lo, hi), rtol=1e-14, atol=1e-15)


def test_lambda_to_zero_plan_returns_the_best_sample():
    prob = small_problem(lam=1e-300, sg_enable=0)
    U0 = np.random.default_rng(2).normal(size=(prob.T, 2)) * [0.5, 0.05]
    r = oracle.plan(prob, U=U0, want_eps=True)
    best = np.clip(U0 + r.eps[:, r.info.argmin], prob.params["u_min"], prob.params["u_max"])
    np.testing.assert_allclose(r.u_star, best, rtol=1e-14, atol=1e-15)
    assert np.argmin(r.S) == r.info.argmin


def test_lambda_to_infinity_plan_returns_the_mean_sample():
    prob = small_problem(lam=1e300, sg_enable=0)
    r = oracle.plan(prob, want_eps=True)
    np.testing.assert_allclose(r.u_star, np.clip(r.eps.mean(axis=1), prob.params["u_min"],
                                                 prob.params["u_max"]), rtol=1e-12, atol=1e-15)


def test_shift_warm_start():
    prob = small_problem(shift=1)
    r = oracle.plan(prob)
    np.testing.assert_array_equal(r.U[:-1], r.u_star[1:])
    np.testing.assert_array_equal(r.U[-1], r.u_star[-1])
    prob0 = small_problem(shift=0)
    r0 = oracle.plan(prob0)
    np.testing.assert_array_equal(r0.U, r0.u_star)


def _rotate(prob, phi, shift=(0.0, 0.0)):
    c, s = math.cos(phi), math.sin(phi)
    Rm = np.array([[c, -s], [s, c]])
    q = prob.copy()
    q.ref = prob.ref @ Rm.T + shift
    q.x0 = prob.x0.copy()
    q.x0[:2] = Rm @ prob.x0[:2] + shift
    q.x0[2] = prob.x0[2] + phi
    q.circles = prob.circles.copy()
    q.circles[:, :2] = prob.circles[:, :2] @ Rm.T + shift
    q.circles[:, 3:5] = prob.circles[:, 3:5] @ Rm.T
    return q


@pytest.mark.parametrize("phi,shift", [(0.0, (1234.5, -987.25)), (0.9, (0.0, 0.0)), (-2.1, (50.0, 20.0))])
def test_costs_are_invariant_under_rigid_motions(phi, shift):
    prob = small_problem()
    a = oracle.plan(prob)
    b = oracle.plan(_rotate(prob, phi, shift))
    np.testing.assert_allclose(b.S, a.S, rtol=1e-9)
    np.testing.assert_allclose(b.u_star, a.u_star, rtol=1e-9, atol=1e-12)


def test_margin_flags_the_reference_yaw_switches_only():
    straight = sc.single_plan()
    straight.params.update(K=128)
    r = oracle.plan(straight)
    assert np.all(r.margin > 1e-3)   # one heading: nothing can switch
    curved = sc.tiny(K=256, T=30, n_ref=40, n_obs=0)
    r = oracle.plan(curved)
    assert np.all(r.margin >= 0) and np.min(r.margin) < 0.05


def test_all_non_finite_costs_leave_u_unchanged():
    prob = small_problem()
    prob.x0[3] = 1e200           # v^2 overflows: every sample cost is +inf
    U0 = np.full((prob.T, 2), 0.01)
    r = oracle.plan(prob, U=U0)
    assert r.rc == -4 and r.info.n_finite == 0
    np.testing.assert_array_equal(r.U, U0)


@pytest.mark.parametrize("change", [dict(K=0), dict(T=0), dict(dt=0.0), dict(lam=0.0), dict(n_ego=9),
                                    dict(sigma=[-1.0, 0.1]), dict(u_min=[1.0, -0.5], u_max=[0.0, 0.5])])
def test_invalid_arguments_are_rejected(change):
    prob = small_problem(**change)
    if prob.params["n_ego"] > 8:
        prob.params["ego_offset"] = [0.0] * 9
        prob.params["ego_radius"] = [1.0] * 9
    assert oracle.plan(prob).rc == -1


def test_non_finite_inputs_are_rejected():
    prob = small_problem()
    prob.ref[3, 1] = np.nan
    assert oracle.plan(prob).rc == -1
    prob = small_problem()
    prob.x0[0] = np.inf
    assert oracle.plan(prob).rc == -1


def test_costs_range_matches_full_plan():
    prob = small_problem()
    r = oracle.plan(prob)
    np.testing.assert_array_equal(oracle.costs_range(prob, 10, 20), r.S[10:30])
