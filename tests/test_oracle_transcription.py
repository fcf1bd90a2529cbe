"""Transcription cross-check of the C oracle at tiny sizes.

A second, vectorised numpy evaluation of Algorithm 1 (all samples at once) is
compared with the scalar C oracle.  It is not an independent pin of the method
(the pins are in the other oracle test files); it catches indexing and layout
slips in the C code, e.g. in the [T][K][2] noise layout or the centre table.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_01654_gb300 import scenarios as sc


def numpy_iteration(prob, U, iter_):
    p = prob.params
    K, T, dt, L = p["K"], p["T"], p["dt"], p["wheelbase"]
    z = oracle.noise(p, iter_)                      # [T][K][2]
    sig, lo, hi = np.array(p["sigma"]), np.array(p["u_min"]), np.array(p["u_max"])
    R = np.array(p["R"])
    alpha = (p["gamma"] - 1) / (2 * p["gamma"])
    ref = prob.ref
    A, B = ref[:-1], ref[1:]
    E = B - A
    l2 = np.sum(E * E, axis=1)
    head = np.arctan2(E[:, 1], E[:, 0])
    tp = ref[-1]
    x = np.tile(prob.x0, (K, 1))
    S = np.zeros(K)
    eps_all = np.zeros((T, K, 2))
    for t in range(T):
        v = np.clip(U[t] + sig * z[t], lo, hi)
        ep = v - U[t]
        eps_all[t] = ep
        xn = np.empty_like(x)
        xn[:, 0] = x[:, 0] + x[:, 3] * np.cos(x[:, 2]) * dt
        xn[:, 1] = x[:, 1] + x[:, 3] * np.sin(x[:, 2]) * dt
        xn[:, 2] = x[:, 2] + x[:, 3] * np.tan(v[:, 1]) / L * dt
        xn[:, 3] = x[:, 3] + v[:, 0] * dt
        P = xn[:, None, :2]
        tau = np.sum((P - A) * E, axis=2) / l2
        Q = np.where((tau <= 0)[..., None], A, np.where((tau >= 1)[..., None], B, A + tau[..., None] * E))
        d2 = np.sum((P - Q) ** 2, axis=2)
        seg = np.argmin(d2, axis=1)                 # first minimum = lowest index
        c_dist = d2[np.arange(K), seg]
        dy = xn[:, 2] - head[seg]
        dy = dy - 2 * math.pi * np.rint(dy / (2 * math.pi))
        c_target = (np.sum((xn[:, :2] - tp) ** 2, 1) > np.sum((x[:, :2] - tp) ** 2, 1)).astype(float)
        c_speed = (xn[:, 3] - p["v_ref"]) ** 2
        if prob.centres is not None:
            C = prob.centres[t]
        else:
            C = prob.circles[:, :2] + prob.circles[:, 3:5] * (t + 1) * dt
        dobj = np.full(K, np.inf)
        for e in range(p["n_ego"]):
            Ex = xn[:, 0] + p["ego_offset"][e] * np.cos(xn[:, 2])
            Ey = xn[:, 1] + p["ego_offset"][e] * np.sin(xn[:, 2])
            if len(C):
                d = np.sqrt((Ex[:, None] - C[None, :, 0]) ** 2 + (Ey[:, None] - C[None, :, 1]) ** 2)
                d = d - prob.circles[None, :, 2] - p["ego_radius"][e]
                dobj = np.minimum(dobj, d.min(axis=1))
        gap = p["d_safe_c"] * xn[:, 3] + p["d_safe_0"] - dobj
        c_safe = np.where(gap > 0, gap * gap, 0.0)
        qx = (p["w_dist"] * c_dist + p["w_target"] * c_target + p["w_yaw"] * dy * dy +
              p["w_speed"] * c_speed + p["w_safe"] * c_safe)
        qu = alpha * ep @ (R * U[t]) + ep @ (R * U[t]) + 0.5 * U[t] @ (R * U[t])
        S += qx + qu
        x = xn
    w = np.exp(-(S - S.min()) / p["lam"])
    dU = np.einsum("k,tkc->tc", w, eps_all) / w.sum()
    un = np.clip(U + dU, lo, hi)
    if p["sg_enable"]:
        us = np.clip(np.stack([oracle.savgol5(un[:, c]) for c in range(2)], 1), lo, hi)
    else:
        us = un
    return S, us


@pytest.mark.parametrize("moving,table", [(False, False), (True, False), (True, True)])
def test_numpy_transcription_matches_c_oracle(moving, table):
    prob = sc.tiny(K=8, T=4, n_ref=12, n_obs=2, moving=moving)
    prob.params["d_safe_0"] = 3.0                   # keep the obstacle term active
    if table:
        prob.centres = sc.predicted_centres(prob.circles, prob.T, prob.params["dt"]) + 0.01
    U = np.random.default_rng(0).normal(size=(prob.T, 2)) * [0.3, 0.03]
    r = oracle.plan(prob, U=U, iter_=3)
    S, us = numpy_iteration(prob, U, 3)
    np.testing.assert_allclose(r.S, S, rtol=1e-12)
    np.testing.assert_allclose(r.u_star, us, rtol=1e-12, atol=1e-14)
