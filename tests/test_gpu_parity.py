"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Sizes: the oracle finishes each case in seconds; the cases span several tiles
of every kernel and end in ragged tails (K not a multiple of the block or tile
sizes, T not a multiple of the step tiles).  Full-size cases of the benchmark
workload are in test_gpu_fullsize.py.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc
from parity import MAX_EXCUSED_FAIL, U_ABS_TOL, argmin_ok, assert_costs, assert_update

pytestmark = pytest.mark.gpu


def run_gpu(prob, U=None, iters=1, params=None):
    p = params if params is not None else prob.params
    with mp.Planner(p) as pl:
        if U is not None:
            pl.set_controls(U, 0)
        outs = []
        for _ in range(iters):
            u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
            outs.append((u, x, info, pl.get_costs()))
        z = pl.get_noise()
        Ud, it = pl.get_controls()
    return outs, z, Ud, it


def check_iteration(prob, gpu_out, orc, max_excused_fail=0.0):
    """Every sample cost, the argmin, and u* and x* whatever the argmin."""
    u, x, info, S = gpu_out
    rep = assert_costs(S, orc.S, orc.margin, max_excused_fail)
    assert argmin_ok(info["argmin"], orc.S), (info["argmin"], orc.info.argmin)
    assert info["n_finite"] == orc.info.n_finite
    assert_update(u, x, orc)
    return rep


# ----------------------------------------------------------------------------- noise

def test_philox_words_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [7, 0, 0, 0xFFFFFFFF]]
    for seed in (0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        got = mp.philox(seed, ctr)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        exp = np.array([oracle.philox4x32_10(c, key) for c in ctr[:512]])
        np.testing.assert_array_equal(got[:512], exp)


@pytest.mark.parametrize("K,T", [(1000, 7), (2048, 16), (3, 1), (65536, 64)])
def test_noise_matches_oracle(K, T):
    prob = sc.tiny(K=K, T=T)
    prob.params.update(seed=0xABCDEF12345, session=3)
    outs, z, _, _ = run_gpu(prob)
    zo = oracle.noise(prob.params, outs[0][2]["iter"])
    # binary32 Box-Muller (logf, sqrtf, sincospif) against binary64: the error is relative to |z|
    # (1 ulp for logf and for sincospif of an exact argument, rounding of sqrt and of the
    # product: at most ~2.98e-7 |z| to first order), also next to the zeros of cos / sin.  The
    # bfloat16 form's midpoint window relies on this bound (3.2e-7 |z|); the largest case holds
    # 8.4 million normals.
    err = np.abs(z.astype(np.float64) - zo)
    rel = err / np.abs(zo)
    assert np.all(err <= 3.2e-7 * np.abs(zo)), rel.max()
    print(f"noise K={K} T={T}: largest relative error {rel.max():.3e} ({rel.max() / 2.0 ** -24:.2f} x 2^-24)")


def test_bf16_noise_is_the_rounded_normal():
    prob = sc.tiny(K=4096, T=8)
    prob.params.update(noise_bf16=1)
    outs, z, _, _ = run_gpu(prob)
    zo = oracle.noise(prob.params, outs[0][2]["iter"])          # oracle rounds its fp64 normals to bf16
    # the kernel takes the bf16 rounding decision on the exact normal near a midpoint: bit-exact codes
    np.testing.assert_array_equal(z.astype(np.float64), zo)


# ----------------------------------------------------------------------------- one iteration

@pytest.mark.parametrize("K,T,group", [(1024, 50, 0), (1000, 37, 1), (777, 33, 4), (257, 13, 32), (1, 5, 0),
                                       (1000, 37, -2), (777, 33, -4), (3, 2, -4), (900, 45, -8), (257, 21, -16)])
def test_single_plan_parity(K, T, group):
    prob = sc.single_plan()
    prob.params.update(K=K, T=T, group=group)
    outs, _, _, _ = run_gpu(prob)
    orc = oracle.plan(prob)
    check_iteration(prob, outs[0], orc)


def test_ten_warm_started_iterations():
    """Ten iterations on one state (shift off).  Each GPU iteration starts from the
    oracle's warm start, so every iteration is compared on identical inputs; the
    free-running drift of the two chains is reported separately."""
    prob = sc.single_plan()                          # K=1024, T=50, 10 iterations
    U = np.zeros((prob.T, 2))
    with mp.Planner(prob.params) as pl:
        for i in range(10):
            pl.set_controls(U, i)
            u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
            S = pl.get_costs()
            orc = oracle.plan(prob, U=U, iter_=i)
            assert info["iter"] == i
            check_iteration(prob, (u, x, info, S), orc)
            U = orc.U
        Ug, it = pl.get_controls()
        assert it == 10
        np.testing.assert_allclose(Ug, U, rtol=0, atol=U_ABS_TOL)
    outs, _, Ud, _ = run_gpu(prob, iters=10)         # free running
    print("free-running drift of u* after 10 iterations:", np.abs(outs[-1][0] - orc.u_star).max())


def closed_loop_states(prob, n_cycles):
    """The closed loop of the paper's planner driven by the oracle: plan, apply u*_0 for
    one step to the binary64 vehicle, advance the obstacles, shift the warm start."""
    p = prob.params
    x, circ, U = prob.x0.copy(), prob.circles.copy(), np.zeros((prob.T, 2))
    out = []
    for c in range(n_cycles):
        q = prob.copy()
        q.x0, q.circles = x.copy(), circ.copy()
        q.centres = sc.predicted_centres(circ, prob.T, p["dt"])
        orc = oracle.plan(q, U=U, iter_=c)
        out.append((q, U.copy(), orc))
        x = oracle.bicycle_step(x, orc.u_star[0, 0], orc.u_star[0, 1], p["dt"], p["wheelbase"])
        circ[:, 0] += circ[:, 3] * p["dt"]
        circ[:, 1] += circ[:, 4] * p["dt"]
        U = orc.U
    return out


@pytest.mark.parametrize("K", [2048, 8192])
def test_closed_loop_cycles_with_shift(K):
    prob = sc.closed_loop()
    prob.params.update(K=K, shift=1)
    cycles = closed_loop_states(prob, 4)
    with mp.Planner(prob.params) as pl:
        for c, (q, U, orc) in enumerate(cycles):
            pl.set_controls(U, c)
            u, x, info = pl.plan(q.x0, q.ref, q.circles, q.centres)
            check_iteration(q, (u, x, info, pl.get_costs()), orc)


def test_closed_loop_full_K():
    prob = sc.closed_loop()                          # K=8192, T=100, 1000-point curved lane
    outs, _, _, _ = run_gpu(prob)
    orc = oracle.plan(prob)
    rep = check_iteration(prob, outs[0], orc)
    print("closed_loop", rep)


@pytest.mark.parametrize("scene,obstacles", [("lane", "table"), ("lane", "velocity"), ("lane", "static"),
                                             ("close", "velocity"), ("close", "table")])
def test_groups_give_identical_costs(scene, obstacles):
    """Every lane split (of the work of a step, or of the steps) gives the costs of one
    lane per sample bit for bit; T = 39 leaves a ragged last block of steps.  "close"
    puts moving obstacles inside the safety band of most rollouts."""
    if scene == "lane":
        prob = sc.closed_loop()
        prob.params.update(K=512, T=39)
    else:
        prob = sc.tiny(K=1500, T=39, n_ref=60, n_obs=3, moving=True)
        prob.params["d_safe_0"] = 2.0
    if obstacles == "table":
        prob.centres = sc.predicted_centres(prob.circles, prob.T, prob.params["dt"])
    else:
        prob.centres = None
    if obstacles == "static":
        prob.circles[:, 3:] = 0.0
    S = {}
    for g in (1, 2, 4, 8, 16, 32, -2, -4, -8, -16):
        p = dict(prob.params, group=g)
        outs, _, _, _ = run_gpu(prob, params=p)
        S[g] = outs[0][3]
    for g in (2, 4, 8, 16, 32, -2, -4, -8, -16):
        np.testing.assert_array_equal(S[g], S[1], err_msg=f"group {g}")


def _hairpin_lane():
    """Out along y = 0, a half turn of radius 1.5 m, back along y = 3: segments of the return leg
    (hundreds of indices away) lie 3 m from the outgoing leg, so the search's side walks run to
    their level-2 fallback, and rollouts between the legs pass the tie of two headings 180 deg
    apart (a few of them within 1e-4 m of it)."""
    out = np.stack([np.arange(0.0, 20.0, 0.1), np.zeros(200)], axis=1)
    a = np.linspace(-np.pi / 2, np.pi / 2, 48)[1:-1]
    turn = np.stack([20.0 + 1.5 * np.cos(a), 1.5 + 1.5 * np.sin(a)], axis=1)
    back = np.stack([np.arange(20.0, 0.0, -0.1), np.full(200, 3.0)], axis=1)
    return np.concatenate([out, turn, back])


def test_hairpin_lane_parity_and_lane_splits():
    """The exact search on a lane that comes back on itself: every sample cost against the oracle's
    brute-force search (samples within 1e-5 of a heading tie excused, at most 0.1 %), and every
    lane split bit for bit."""
    prob = sc.tiny(K=2048, T=40)                     # 16 m along the outgoing leg, short of the turn
    prob.params.update(dt=0.05, sigma=[1.0, 0.3], seed=11)
    prob.ref = _hairpin_lane()
    prob.x0 = np.array([0.0, 0.4, 0.0, 8.0])
    prob.circles = np.array([[12.0, 1.5, 0.6, 0.0, 0.0]])
    prob.centres = None
    outs, _, _, _ = run_gpu(prob)
    orc = oracle.plan(prob)
    rep = check_iteration(prob, outs[0], orc, max_excused_fail=MAX_EXCUSED_FAIL)
    print("hairpin", rep)
    for g in (2, 4, -2, -4, -8):
        o, _, _, _ = run_gpu(prob, params=dict(prob.params, group=g))
        np.testing.assert_array_equal(o[0][3], outs[0][3], err_msg=f"group {g}")


@pytest.mark.parametrize("variant", ["vertex", "collision_only", "vcap", "gamma", "terminal", "dsafe_v",
                                     "radii", "sg_off", "moving_velocity", "moving_table", "no_obstacles",
                                     "two_point_ref"])
def test_variants(variant):
    prob = sc.tiny(K=1500, T=25, n_ref=60, n_obs=3, moving=variant.startswith("moving"))
    p = prob.params
    p["d_safe_0"] = 2.0
    if variant == "vertex":
        p["ref_mode"] = 1
    elif variant == "collision_only":
        p.update(collision_only=1, ego_radius=[2.5, 2.5, 2.5])
    elif variant == "vcap":
        p["v_max"] = 4.5
    elif variant == "gamma":
        p["gamma"] = 3.0
        prob_U = np.random.default_rng(1).normal(size=(prob.T, 2)) * [0.5, 0.05]
    elif variant == "terminal":
        p["w_terminal"] = 4.0
    elif variant == "dsafe_v":
        p.update(d_safe_c=0.4, d_safe_0=1.0)
    elif variant == "radii":
        p.update(ego_radius=[1.3, 0.9, 1.1])
    elif variant == "sg_off":
        p["sg_enable"] = 0
    elif variant == "moving_table":
        prob.centres = sc.predicted_centres(prob.circles, prob.T, p["dt"])
    elif variant == "no_obstacles":
        prob.circles = np.zeros((0, 5))
    elif variant == "two_point_ref":
        prob.ref = np.array([[-5.0, 0.0], [30.0, 1.0]])
    U = prob_U if variant == "gamma" else np.random.default_rng(2).normal(size=(prob.T, 2)) * [0.3, 0.03]
    outs, _, _, _ = run_gpu(prob, U=U)
    orc = oracle.plan(prob, U=U)
    check_iteration(prob, outs[0], orc)


def test_device_entry_point_matches_host_entry_point():
    torch = pytest.importorskip("torch")
    prob = sc.single_plan()
    prob.params.update(K=2000, T=30)
    outs, _, _, _ = run_gpu(prob)
    dev = torch.device("cuda:0")
    with mp.Planner(prob.params, stream=torch.cuda.current_stream().cuda_stream) as pl:
        x0 = torch.tensor(prob.x0, dtype=torch.float64, device=dev)
        ref = torch.tensor(prob.ref, dtype=torch.float64, device=dev)
        circ = torch.tensor(prob.circles, dtype=torch.float64, device=dev)
        u = torch.empty((prob.T, 2), dtype=torch.float64, device=dev)
        x = torch.empty((prob.T + 1, 4), dtype=torch.float64, device=dev)
        info = pl.plan_device(x0, ref, circ, None, u, x, wait=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u.cpu().numpy(), outs[0][0])
        np.testing.assert_array_equal(x.cpu().numpy(), outs[0][1])
        assert info["argmin"] == outs[0][2]["argmin"]


# ----------------------------------------------------------------------------- errors and state

@pytest.mark.parametrize("where", ["ref", "x0", "circles", "centres"])
@pytest.mark.parametrize("value", [np.nan, np.inf, -np.inf])
def test_non_finite_input_is_rejected_and_state_kept(where, value):
    prob = sc.single_plan()
    prob.params.update(K=256, T=10)
    with mp.Planner(prob.params) as pl:
        U0 = np.full((10, 2), 0.01)
        pl.set_controls(U0, 5)
        args = {"x0": prob.x0.copy(), "ref": prob.ref.copy(), "circles": prob.circles.copy(),
                "centres": sc.predicted_centres(prob.circles, 10, prob.params["dt"])}
        a = args[where]
        a.flat[a.size // 2] = value
        with pytest.raises(mp.MppiError) as e:
            pl.plan(args["x0"], args["ref"], args["circles"], args["centres"])
        assert e.value.status == -1
        U, it = pl.get_controls()
        np.testing.assert_array_equal(U, U0)
        assert it == 5


def test_non_finite_device_input_is_a_no_op():
    torch = pytest.importorskip("torch")
    prob = sc.single_plan()
    prob.params.update(K=256, T=10)
    dev = torch.device("cuda:0")
    with mp.Planner(prob.params) as pl:
        x0 = torch.tensor(prob.x0, dtype=torch.float64, device=dev)
        ref = torch.tensor(prob.ref, dtype=torch.float64, device=dev)
        ref[5, 1] = float("inf")
        circ = torch.tensor(prob.circles, dtype=torch.float64, device=dev)
        u = torch.zeros((10, 2), dtype=torch.float64, device=dev)
        x = torch.zeros((11, 4), dtype=torch.float64, device=dev)
        with pytest.raises(mp.MppiError) as e:
            pl.plan_device(x0, ref, circ, None, u, x, wait=True)
        assert e.value.status == -1
        U, it = pl.get_controls()
        assert np.all(U == 0.0) and it == 0
        # the context stays usable
        u2, x2, info = pl.plan(prob.x0, prob.ref, prob.circles)
        assert info["iter"] == 0


def test_all_costs_non_finite_leaves_controls():
    prob = sc.single_plan()
    prob.params.update(K=128, T=8)
    x0 = prob.x0.copy()
    x0[3] = 1e30                                   # v^2 overflows binary32: every cost is +inf
    with mp.Planner(prob.params) as pl:
        U0 = np.full((8, 2), 0.02)
        pl.set_controls(U0, 0)
        with pytest.raises(mp.MppiError) as e:
            pl.plan(x0, prob.ref, prob.circles)
        assert e.value.status == -4
        U, it = pl.get_controls()
        np.testing.assert_array_equal(U, U0)
        assert it == 0


@pytest.mark.parametrize("case", ["signed", "all_equal"])
def test_argmin_over_signed_and_tied_costs(case):
    """S_min and its sample (Algorithm 1) over costs of both signs, and over costs that are all
    exactly equal (every sample ties: the lowest index wins).  Only the control cost is on, so
    a sample's cost is sum_t (1/2 u^T R u + (1 + alpha) u^T R eps): with a small nominal u the
    noise term gives costs of either sign; with u = 0 every cost is exactly 0."""
    prob = sc.single_plan()
    prob.params.update(K=1000, T=40, seed=17)
    for w in ("w_dist", "w_target", "w_yaw", "w_speed", "w_safe", "w_terminal"):
        prob.params[w] = 0.0
    with mp.Planner(prob.params) as pl:
        if case == "signed":
            pl.set_controls(np.column_stack([np.full(40, 0.05), np.zeros(40)]), 0)
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
        S = pl.get_costs()
    if case == "signed":
        assert (S < 0).sum() > 50 and (S > 0).sum() > 50
    else:
        assert np.all(S == 0.0)
    assert info["n_finite"] == int(np.isfinite(S).sum()) == 1000
    assert info["s_min"] == S.min()
    assert info["argmin"] == int(np.flatnonzero(S == S.min())[0])
    if case == "all_equal":
        assert info["argmin"] == 0


def test_capacity_is_enforced():
    prob = sc.single_plan()
    prob.params.update(K=64, T=8)
    with mp.Planner(prob.params, max_ref=100, max_circ=2) as pl:
        with pytest.raises(mp.MppiError) as e:
            pl.plan(prob.x0, prob.ref, prob.circles)       # 200 vertices > 100
        assert e.value.status == -6
        with pytest.raises(mp.MppiError) as e:
            pl.plan(prob.x0, prob.ref[:50], prob.circles)  # 3 circles > 2
        assert e.value.status == -6
        with pytest.raises(mp.MppiError) as e:
            pl.plan(prob.x0, prob.ref[:1], prob.circles[:1])
        assert e.value.status == -1


def test_checkpoint_resume_reproduces_the_stream():
    prob = sc.single_plan()
    prob.params.update(K=512, T=20)
    with mp.Planner(prob.params) as a:
        a.plan(prob.x0, prob.ref, prob.circles)
        U, it = a.get_controls()
        u1, x1, i1 = a.plan(prob.x0, prob.ref, prob.circles)
    with mp.Planner(prob.params) as b:
        b.set_controls(U, it)
        u2, x2, i2 = b.plan(prob.x0, prob.ref, prob.circles)
    np.testing.assert_array_equal(u1, u2)
    assert i1["iter"] == i2["iter"] == 1


def test_rollout_stats_are_consistent_and_leave_state():
    prob = sc.roofline()
    prob.params.update(K=4096, T=40)
    with mp.Planner(prob.params) as pl:
        U0 = np.full((40, 2), 0.01)
        pl.set_controls(U0, 3)
        st = pl.rollout_stats(prob.x0, prob.ref, prob.circles)
        U, it = pl.get_controls()
        np.testing.assert_array_equal(U, U0)
        assert it == 3
        # straight lane: one box of the chunks before the scanned chunk and one of those after it
        # (fewer at the ends of the lane); a side whose box passes adds its neighbour chunk box
        # and the box beyond it; the fallback ranges never open
        assert 1.0 <= st["range_boxes"] <= 4.0 and 0.0 <= st["chunk_boxes"] <= 2.0
        assert 1 <= st["segments"] <= prob.ref.shape[0]
        # the broad phase tests one circle per lane per 32 circles of the indexed range, at most
        # every circle; on this lane of 200 m the range around a warp is a few circles
        assert 0.0 < st["circles_tested"] <= math.ceil(prob.circles.shape[0] / 32)
        assert st["in_band"] <= st["candidates"]
        # the plan after the stats run still matches the oracle
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
        orc = oracle.plan(prob, U=U0, iter_=3)
        check_iteration(prob, (u, x, info, pl.get_costs()), orc)


# ----------------------------------------------------------------------------- steering-rate model

def test_paper_preset_steering_rate_model_parity():
    """Table I setting on the 5-state model (state carries delta, control (a, omega))."""
    prob = sc.paper_preset()                          # K=2560, T=16, dt=0.25, lambda=150
    outs, _, _, _ = run_gpu(prob)
    orc = oracle.plan(prob)
    assert outs[0][1].shape == (prob.T + 1, 5)
    rep = check_iteration(prob, outs[0], orc)
    print("paper_preset", rep)


def test_paper_preset_three_iterations_teacher_forced():
    prob = sc.paper_preset()
    prob.params.update(shift=1)
    U = np.zeros((prob.T, 2))
    with mp.Planner(prob.params) as pl:
        for i in range(3):
            pl.set_controls(U, i)
            u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
            orc = oracle.plan(prob, U=U, iter_=i)
            check_iteration(prob, (u, x, info, pl.get_costs()), orc)
            U = orc.U


def test_steering_rate_groups_give_identical_costs():
    prob = sc.paper_preset()
    prob.params.update(K=700, T=23)
    prob.x0 = np.array([0.0, 0.3, 0.05, 6.0, -0.04])
    S = {}
    for g in (1, 2, 8, -2, -4, -8, -16):
        outs, _, _, _ = run_gpu(prob, params=dict(prob.params, group=g))
        S[g] = outs[0][3]
    for g in S:
        np.testing.assert_array_equal(S[g], S[1], err_msg=f"group {g}")


def test_steering_rate_with_speed_cap_off_and_device_entry_point():
    torch = pytest.importorskip("torch")
    prob = sc.paper_preset()
    prob.params.update(K=1000, T=30, v_max=math.inf)
    outs, _, _, _ = run_gpu(prob)
    orc = oracle.plan(prob)
    check_iteration(prob, outs[0], orc)
    dev = torch.device("cuda:0")
    with mp.Planner(prob.params, stream=torch.cuda.current_stream().cuda_stream) as pl:
        u = torch.empty((prob.T, 2), dtype=torch.float64, device=dev)
        x = torch.empty((prob.T + 1, 5), dtype=torch.float64, device=dev)
        pl.plan_device(torch.tensor(prob.x0, dtype=torch.float64, device=dev),
                       torch.tensor(prob.ref, dtype=torch.float64, device=dev),
                       torch.tensor(prob.circles, dtype=torch.float64, device=dev), None, u, x, wait=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(x.cpu().numpy(), outs[0][1])


def test_batch_engine_rejects_the_steering_rate_model():
    prob = sc.paper_preset()
    with mp.BatchPlanner(max_slots=2, max_batch=2, max_samples=4096, max_rollout_steps=100000, max_T=32,
                         max_ref=1024, max_circ=16) as bp:
        with pytest.raises(mp.MppiError) as e:
            bp.plan([mp.BatchPlan(prob.params, 0, prob.x0[:4], prob.ref, prob.circles, None)])
        assert e.value.status == -1


# ----------------------------------------------------------------------------- cost-to-go form

@pytest.mark.parametrize("scene", ["curved_lane", "close_obstacles", "paper_preset"])
def test_cost_to_go_update_parity(scene):
    """Eq. (11) read per step: each step's weights from the cost still to come."""
    if scene == "curved_lane":
        prob = sc.closed_loop()
        prob.params.update(K=2048, T=60)
    elif scene == "close_obstacles":
        prob = sc.tiny(K=1500, T=25, n_ref=60, n_obs=3, moving=True)
        prob.params["d_safe_0"] = 2.0
    else:
        prob = sc.paper_preset()
    prob.params["cost_to_go"] = 1
    U = np.random.default_rng(7).normal(size=(prob.T, 2)) * [0.3, 0.02]
    U = np.clip(U, prob.params["u_min"], prob.params["u_max"])
    outs, _, _, _ = run_gpu(prob, U=U)
    orc = oracle.plan(prob, U=U)
    rep = check_iteration(prob, outs[0], orc)
    print("cost_to_go", scene, rep)


def test_cost_to_go_same_update_for_every_lane_split():
    prob = sc.closed_loop()
    prob.params.update(K=512, T=39, cost_to_go=1)
    u = {}
    for g in (1, 4, 32, -2, -8):
        outs, _, _, _ = run_gpu(prob, params=dict(prob.params, group=g))
        u[g] = outs[0][0]
    for g in u:
        np.testing.assert_array_equal(u[g], u[1], err_msg=f"group {g}")


def test_cost_to_go_reading_changes_the_update():
    prob = sc.closed_loop()
    prob.params.update(K=2048, T=60)
    a, _, _, _ = run_gpu(prob)
    b, _, _, _ = run_gpu(prob, params=dict(prob.params, cost_to_go=1))
    np.testing.assert_array_equal(a[0][3], b[0][3])                   # same sample costs
    assert np.abs(a[0][0] - b[0][0]).max() > 1e-6                     # different update


# ----------------------------------------------------------------------------- failure path

@pytest.mark.parametrize("flag,status", [(mp.FLAG_TIMEOUT, -5), (mp.FLAG_NONFINITE_INPUT, -1)])
@pytest.mark.parametrize("entry", ["host", "device"])
def test_injected_device_flag_ends_the_iteration_and_keeps_the_state(flag, status, entry):
    """The status a kernel raises when a bounded wait runs out (or it sees non-finite input),
    written into the device record between the rollout and the update from the host: the
    iteration ends with that status, the warm start and the iteration counter stay, and the next
    iteration runs normally.  No kernel faults or waits on anything."""
    torch = pytest.importorskip("torch")
    prob = sc.single_plan()
    prob.params.update(K=512, T=20)
    U0 = np.random.default_rng(4).normal(size=(20, 2)) * [0.2, 0.02]
    with mp.Planner(prob.params, stream=torch.cuda.current_stream().cuda_stream) as pl:
        for rep in range(2):                         # also after the host-buffer graph is captured
            pl.set_controls(U0, 3)
            pl.plan(prob.x0, prob.ref, prob.circles)
            pl.plan(prob.x0, prob.ref, prob.circles)
        pl.set_controls(U0, 3)
        pl.debug_inject_flags(flag)
        with pytest.raises(mp.MppiError) as e:
            if entry == "host":
                pl.plan(prob.x0, prob.ref, prob.circles)
            else:
                dev = torch.device("cuda:0")
                t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
                u = torch.empty((20, 2), dtype=torch.float64, device=dev)
                x = torch.empty((21, 4), dtype=torch.float64, device=dev)
                pl.plan_device(t(prob.x0), t(prob.ref), t(prob.circles), None, u, x, wait=True)
        assert e.value.status == status
        U, it = pl.get_controls()
        np.testing.assert_array_equal(U, U0)
        assert it == 3
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)     # the context stays usable
        assert info["iter"] == 3
        orc = oracle.plan(prob, U=U0, iter_=3)
        check_iteration(prob, (u, x, info, pl.get_costs()), orc)
    with mp.Planner(prob.params) as pl:
        with pytest.raises(mp.MppiError) as e:
            pl.debug_inject_flags(8)
        assert e.value.status == -1


# ----------------------------------------------------------------------------- specialised step

@pytest.mark.parametrize("scene", ["straight_static", "moving", "curved"])
@pytest.mark.parametrize("group", [1, 2, 4, -2, -4, -8, 8])
def test_specialised_step_gives_the_general_bits(scene, group):
    """The rollout's specialised step (static circles, three equal ego circles, constant band, no
    speed cap, one lane heading) against the general step on the same plan: a speed cap of 1e30
    never binds (the perturbed acceleration is already clamped into the control box) but makes the
    host launch the general kernel.  Moving circles or a curved lane send the specialised kernel's
    blocks down the general branch at run time.  The costs and u* are the same bits."""
    if scene == "curved":
        prob = sc.closed_loop()
        prob.params.update(K=3000, T=45)
        prob.centres = None                      # circles moving by velocity, no table: host-simple
        prob.circles[:, 3:] = 0.0                # static, but the lane has many headings
    elif scene == "moving":
        prob = sc.tiny(K=2500, T=40, n_ref=60, n_obs=3, moving=True)
        prob.params["d_safe_0"] = 2.0
    else:
        prob = sc.roofline()
        prob.params.update(K=4096, T=60)
    prob.params["group"] = group
    a, _, _, _ = run_gpu(prob)
    b, _, _, _ = run_gpu(prob, params=dict(prob.params, v_max=1e30))
    np.testing.assert_array_equal(a[0][3], b[0][3])
    np.testing.assert_array_equal(a[0][0], b[0][0])
    np.testing.assert_allclose(a[0][1], b[0][1], rtol=0, atol=1e-9)     # x*: the capped speed is a serial sum
    assert a[0][2]["argmin"] == b[0][2]["argmin"]
