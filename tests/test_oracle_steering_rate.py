"""Pins for the oracle's steering-rate form of Eq. (5): state (x, y, yaw, v, delta), control
(a, omega), the model the paper writes down (its Table I preset runs on it).

Each expected value is fixed by a closed form or by reduction to the 4-state form, whose own
pins are in test_oracle_dynamics_cost.py.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_01654_gb300 import scenarios as sc

L = 2.7


def path5(x0, a, omega, dt, n):
    xs = [np.asarray(x0, dtype=float)]
    for _ in range(n):
        xs.append(oracle.bicycle5_step(xs[-1], a, omega, dt, L))
    return np.array(xs)


def test_zero_rate_is_the_four_state_model_at_constant_steering():
    x0 = [1.0, 2.0, 0.3, 6.0, 0.12]
    for a in (0.0, 1.1, -2.5):
        x5 = oracle.bicycle5_step(x0, a, 0.0, 0.25, L)
        x4 = oracle.bicycle_step(x0[:4], a, x0[4], 0.25, L)
        np.testing.assert_array_equal(x5[:4], x4)
        assert x5[4] == x0[4]


def test_steering_is_the_euler_integral_of_the_rate():
    # delta_n = delta_0 + n omega dt, and the yaw uses delta at the start of each step
    d0, w, dt, n, v = -0.05, 0.11, 0.25, 16, 8.0
    xs = path5([0.0, 0.0, 0.0, v, d0], 0.0, w, dt, n)
    np.testing.assert_allclose(xs[:, 4], d0 + w * dt * np.arange(n + 1), rtol=0, atol=1e-15)
    dth = v * dt * np.tan(d0 + w * dt * np.arange(n)) / L
    np.testing.assert_allclose(np.diff(xs[:, 2]), dth, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(xs[-1, 2], dth.sum(), rtol=1e-12)


def test_straight_ahead_with_zero_steering_and_rate():
    xs = path5([0.0, -1.0, 0.0, 5.0, 0.0], 0.4, 0.0, 0.1, 50)
    assert np.all(xs[:, 1] == -1.0) and np.all(xs[:, 2] == 0.0) and np.all(xs[:, 4] == 0.0)
    np.testing.assert_allclose(xs[-1, 3], 5.0 + 0.4 * 50 * 0.1, rtol=1e-14)


def test_mirror_symmetry_in_the_rate():
    a = path5([0.0, 0.0, 0.0, 7.0, 0.02], 0.3, 0.08, 0.25, 16)
    b = path5([0.0, 0.0, 0.0, 7.0, -0.02], 0.3, -0.08, 0.25, 16)
    np.testing.assert_allclose(b[:, [0, 3]], a[:, [0, 3]], rtol=0, atol=1e-14)
    np.testing.assert_allclose(b[:, [1, 2, 4]], -a[:, [1, 2, 4]], rtol=0, atol=1e-14)


def preset(K=48, T=10, **kw):
    prob = sc.paper_preset()
    prob.params.update(K=K, T=T, **kw)
    return prob


def test_x_star_is_the_noise_free_rollout_of_u_star_with_the_steering_state():
    prob = preset()
    r = oracle.plan(prob)
    assert r.rc == 0 and r.x_star.shape == (prob.T + 1, 5)
    np.testing.assert_array_equal(r.x_star[0], prob.x0)
    xs = [prob.x0]
    for t in range(prob.T):
        a = r.u_star[t, 0]
        v = xs[-1][3]
        a = max(min(a, (prob.params["v_max"] - v) / prob.params["dt"]), prob.params["u_min"][0])   # speed cap
        xs.append(oracle.bicycle5_step(xs[-1], a, r.u_star[t, 1], prob.params["dt"], L))
    np.testing.assert_allclose(r.x_star, np.array(xs), rtol=1e-15, atol=1e-15)


def test_rates_stay_in_the_papers_bounds_and_lambda_to_zero_returns_the_best_sample():
    prob = preset(lam=1e-300, sg_enable=0)
    U0 = np.random.default_rng(3).normal(size=(prob.T, 2)) * [0.5, 0.03]
    r = oracle.plan(prob, U=U0, want_eps=True)
    best = np.clip(U0 + r.eps[:, r.info.argmin], prob.params["u_min"], prob.params["u_max"])
    np.testing.assert_allclose(r.u_star, best, rtol=1e-14, atol=1e-15)
    assert np.all(np.abs(r.u_star[:, 1]) <= 0.11) and np.all(r.u_star[:, 0] >= -2.5) and np.all(r.u_star[:, 0] <= 1.1)


def test_zero_noise_and_zero_rate_drive_along_the_initial_steering():
    prob = preset(sigma=[0.0, 0.0], sg_enable=0)
    r = oracle.plan(prob)
    np.testing.assert_array_equal(r.u_star, np.zeros((prob.T, 2)))
    np.testing.assert_array_equal(r.x_star[:, 4], np.full(prob.T + 1, prob.x0[4]))


def test_model_one_needs_five_finite_state_entries():
    prob = preset()
    prob.x0 = np.array([0.0, 0.0, 0.0, 7.0, math.nan])
    assert oracle.plan(prob).rc == -1
