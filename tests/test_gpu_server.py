"""The continuous-batching server (mppi_server_*) (needs a GB300).

Each result must be the same whether its request ran alone or mixed with others in
micro-batches: requests of one session run in arrival order against the session's
device-resident warm start, and a plan's arithmetic does not depend on its batch.
"""
import numpy as np
import pytest

import oracle
import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc
from parity import S_REL_TOL, argmin_ok, assert_update

pytestmark = pytest.mark.gpu


def sessions(n=10, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        p = sc.uneven_instance(rng, i, seed=seed)
        p.params["K"] = int(rng.choice([512, 1024, 3000]))
        p.params["T"] = int(rng.integers(8, 50))
        p.params["shift"] = 1
        out.append(p)
    return out


def trace(probs, n_req=30, seed=1):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        s = int(rng.integers(0, len(probs)))
        p = probs[s]
        circ = p.circles.copy()
        if circ.shape[0]:
            circ[:, :2] += rng.normal(scale=0.3, size=(circ.shape[0], 2))      # obstacles redrawn per request
        reqs.append((s, np.ascontiguousarray(circ)))
    return reqs


def server_for(probs, **kw):
    cfg = dict(max_sessions=len(probs), max_batch=64, max_samples=200000, max_rollout_steps=8_000_000,
               max_T=64, max_ref=1024, max_circ=128, pipelines=3, hbm_budget_bytes=1 << 30)
    cfg.update(kw)
    return mp.Server(**cfg)


def run(srv, probs, reqs, params, alone):
    ids = {}
    results = {}
    for j, (s, circ) in enumerate(reqs):
        p = probs[s]
        rid = srv.enqueue(params[s], s, p.x0, p.ref, circ if circ.shape[0] else None)
        ids[rid] = j
        if alone:
            got = []
            while not got:
                got = srv.poll(16, wait_ms=1000, with_outputs=True)
            for r in got:
                results[ids[r["request_id"]]] = r
    while len(results) < len(reqs):
        for r in srv.poll(64, wait_ms=1000, with_outputs=True):
            results[ids[r["request_id"]]] = r
    return [results[j] for j in range(len(reqs))]


def test_results_are_the_same_alone_and_in_the_mix():
    probs = sessions()
    reqs = trace(probs)
    params = [mp.make_params(p.params) for p in probs]
    with server_for(probs) as srv:
        alone = run(srv, probs, reqs, params, alone=True)
        for s, p in enumerate(probs):
            srv.set_controls(s, np.zeros((p.T, 2)), 0)
        mix = run(srv, probs, reqs, params, alone=False)
        stats = srv.pending()
    assert stats["batches"] < 2 * len(reqs)           # the mixed run did batch requests together
    for a, b in zip(alone, mix):
        assert a["status"] == 0 and b["status"] == 0
        np.testing.assert_array_equal(a["u"], b["u"])
        np.testing.assert_array_equal(a["x"], b["x"])
        assert a["info"] == b["info"]


def test_server_agrees_with_the_single_plan_path():
    probs = sessions(n=4)
    reqs = [(0, probs[0].circles), (1, probs[1].circles), (0, probs[0].circles), (3, probs[3].circles)]
    params = [mp.make_params(p.params) for p in probs]
    with server_for(probs) as srv:
        res = run(srv, probs, reqs, params, alone=False)
    ctx = {s: mp.Planner(probs[s].params) for s in (0, 1, 3)}
    try:
        for (s, circ), r in zip(reqs, res):
            p = probs[s]
            u, x, info = ctx[s].plan(p.x0, p.ref, circ if circ.shape[0] else None)
            assert r["info"]["argmin"] == info["argmin"] and r["info"]["iter"] == info["iter"]
            np.testing.assert_allclose(r["u"], u, rtol=1e-12, atol=1e-14)
    finally:
        for c in ctx.values():
            c.close()


def test_hbm_budget_limits_what_is_in_flight():
    probs = sessions(n=6)
    params = [mp.make_params(p.params) for p in probs]
    # room for the largest request (noise, costs and weights, and up to ~250 KB for its scene with
    # the search's vertex boxes and its centre table) but not for all six
    biggest = max(p.K * p.T * 8 + p.K * 12 for p in probs)
    budget = biggest + 250_000
    assert sum(p.K * p.T * 8 for p in probs) > budget
    reqs = [(s, probs[s].circles) for s in range(6)]
    with server_for(probs, hbm_budget_bytes=budget) as srv:
        res = run(srv, probs, reqs, params, alone=False)
        st = srv.pending()
    assert all(r["status"] == 0 for r in res)
    assert st["batches"] >= 2                         # the budget split the six requests


def test_request_above_capacity_is_refused():
    probs = sessions(n=2)
    params = [mp.make_params(p.params) for p in probs]
    with server_for(probs, hbm_budget_bytes=10_000) as srv:
        with pytest.raises(mp.MppiError) as e:
            srv.enqueue(params[0], 0, probs[0].x0, probs[0].ref, probs[0].circles if probs[0].circles.shape[0] else None)
        assert e.value.status == -6
        with pytest.raises(mp.MppiError) as e:
            srv.enqueue(params[0], 5, probs[0].x0, probs[0].ref, None)      # session out of range
        assert e.value.status == -1


def test_served_results_match_the_oracle():
    """Each served result against the FP64 oracle (Eq. (11) and Algorithm 1 per request) on the
    same inputs, warm start and iteration counter.  Three rounds of one request per session, mixed
    into micro-batches by the server; before each round every session's device warm start is set
    to the oracle's (teacher forcing), so each result is compared on identical inputs."""
    probs = sessions(n=6, seed=11)
    params = [mp.make_params(p.params) for p in probs]
    rng = np.random.default_rng(3)
    U = [np.zeros((p.T, 2)) for p in probs]
    with server_for(probs) as srv:
        for rnd in range(3):
            for s, p in enumerate(probs):
                srv.set_controls(s, U[s], rnd)
            reqs = []
            for s, p in enumerate(probs):
                circ = p.circles.copy()
                if circ.shape[0]:
                    circ[:, :2] += rng.normal(scale=0.3, size=(circ.shape[0], 2))
                reqs.append((s, np.ascontiguousarray(circ)))
            res = run(srv, probs, reqs, params, alone=False)
            for (s, circ), r in zip(reqs, res):
                q = probs[s].copy()
                q.circles = circ
                orc = oracle.plan(q, U=U[s], iter_=rnd)
                assert r["status"] == 0 and r["info"]["iter"] == rnd
                assert argmin_ok(r["info"]["argmin"], orc.S), (r["info"]["argmin"], orc.info.argmin)
                assert r["info"]["n_finite"] == orc.info.n_finite
                assert abs(r["info"]["s_min"] - orc.info.s_min) <= S_REL_TOL * max(abs(orc.info.s_min), 1.0)
                assert_update(r["u"], r["x"], orc)
                U[s] = orc.U


def test_a_session_keeps_its_order_when_its_older_request_does_not_fit():
    """Session 0 queues a large request and then a small one while another session's large
    request holds most of the HBM budget: the small one fits and the large one does not, yet the
    small one must not overtake it (its warm start is the large one's output)."""
    probs = sessions(n=2)
    params = {}
    for name, K, T in (("big", 65536, 48), ("small", 512, 8)):
        q = dict(probs[0].params, K=K, T=T)
        params[name] = mp.make_params(q)
    scene = 200_000                                   # generous bound on a scene and its centre table
    big = 65536 * 48 * 8 + 65536 * 12 + scene
    small = 512 * 8 * 8 + 512 * 12 + scene
    budget = big + small + scene                      # room for one large and one small request
    p0, p1 = probs[0], probs[1]
    with server_for(probs, hbm_budget_bytes=budget, max_samples=200_000, max_rollout_steps=8_000_000) as srv:
        srv.enqueue(params["big"], 1, p1.x0, p1.ref, None)               # holds the budget for a while
        r_big = srv.enqueue(params["big"], 0, p0.x0, p0.ref, None)
        r_small = srv.enqueue(params["small"], 0, p0.x0, p0.ref, None)
        got = []
        while len(got) < 3:
            got += srv.poll(8, wait_ms=1000)
    by_id = {r["request_id"]: (i, r) for i, r in enumerate(got)}
    i_big, rb = by_id[r_big]
    i_small, rs = by_id[r_small]
    assert rb["status"] == 0 and rs["status"] == 0
    assert rb["info"]["iter"] == 0 and rs["info"]["iter"] == 1       # session 0's counter: arrival order
    assert i_big < i_small                                            # completed first


def test_poll_reports_rows_too_short_for_a_result():
    probs = sessions(n=1)
    p = probs[0]
    params = mp.make_params(p.params)
    with server_for(probs) as srv:
        srv.enqueue(params, 0, p.x0, p.ref, None)
        out = (mp.MppiResult * 4)()
        n = mp.C.c_int32()
        short = max(1, p.T - 1)
        U = np.zeros((4, short, 2))
        X = np.zeros((4, short + 1, 4))
        got = 0
        for _ in range(50):
            rc = mp.lib().mppi_server_poll(srv._h, mp.C.cast(out, mp._VP), 4, mp._dp(U), mp._dp(X), short, 200,
                                           mp.C.byref(n))
            assert rc == 0
            if n.value:
                got = n.value
                break
        assert got == 1
        assert out[0].status == -6 and out[0].T == p.T
        assert np.all(U == 0.0) and np.all(X == 0.0)


def test_watchdog_abandons_a_late_micro_batch_and_the_server_recovers():
    """A host-side watchdog far shorter than any micro-batch: every request completes with
    MPPI_ERR_TIMEOUT, nothing faults or waits on the device, and with the watchdog off again the
    server plans normally (its sessions were held until the abandoned work had ended)."""
    probs = sessions(n=4)
    params = [mp.make_params(p.params) for p in probs]
    reqs = [(s, probs[s].circles) for s in range(4)]
    with server_for(probs, watchdog_ms=1e-3) as srv:
        res = run(srv, probs, reqs, params, alone=False)
        assert all(r["status"] == -5 for r in res)
        assert srv.timeouts() == len(reqs)
        srv.set_watchdog(0.0)
        res2 = run(srv, probs, reqs, params, alone=False)
        assert all(r["status"] == 0 for r in res2)
        assert srv.timeouts() == len(reqs)
        st = srv.pending()
        assert st["queued"] == 0 and st["in_flight"] == 0


def test_session_table_snapshot_and_restore(tmp_path):
    """Every session's warm start and counter written to a file and read into a new server: the
    next request of each session gives the same result in both servers."""
    probs = sessions(n=5)
    params = [mp.make_params(p.params) for p in probs]
    reqs = [(s, probs[s].circles) for s in range(5)]
    path = str(tmp_path / "sessions.bin")
    with server_for(probs) as a:
        run(a, probs, reqs, params, alone=False)                  # warm starts move on (shift on)
        run(a, probs, reqs, params, alone=False)
        a.snapshot(path)
        nxt_a = run(a, probs, reqs, params, alone=False)
    with server_for(probs) as b:
        b.restore(path)
        nxt_b = run(b, probs, reqs, params, alone=False)
        with pytest.raises(mp.MppiError) as e:
            with server_for(probs, max_T=32) as c:               # another size: refused
                c.restore(path)
        assert e.value.status == -1
    for ra, rb in zip(nxt_a, nxt_b):
        assert ra["status"] == rb["status"] == 0
        assert ra["info"]["iter"] == rb["info"]["iter"] == 2
        np.testing.assert_array_equal(ra["u"], rb["u"])
        np.testing.assert_array_equal(ra["x"], rb["x"])
