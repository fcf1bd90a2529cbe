"""The allocation-free argmin entry point against the argmin of mppi_plan (needs a GB300).

mppi_argmin_noalloc serves callers that cannot allocate GPU memory while planning
(a control cycle that must not stall on cudaMalloc, or code limited to memory
reserved at start-up).  It keeps its scratch in a fixed array inside the library,
so two calls in a row share that scratch: the second call must still be right.
This file is collected last so that a failure here does not hide the others.
"""
import ctypes

import numpy as np
import pytest

import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc

pytestmark = pytest.mark.gpu


def _argmin_noalloc(torch, S_host, stream):
    dev = torch.device("cuda", 0)
    d_S = torch.tensor(S_host, dtype=torch.float64, device=dev)
    d_min = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    d_arg = torch.full((1,), -7, dtype=torch.int32, device=dev)
    d_n = torch.full((1,), -7, dtype=torch.int32, device=dev)
    rc = mp.lib().mppi_argmin_noalloc(ctypes.c_void_p(d_S.data_ptr()), int(d_S.numel()),
                                      ctypes.c_void_p(d_min.data_ptr()), ctypes.c_void_p(d_arg.data_ptr()),
                                      ctypes.c_void_p(d_n.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, mp.lib().mppi_status_string(rc)
    torch.cuda.synchronize()
    return float(d_min.item()), int(d_arg.item()), int(d_n.item())


def test_noalloc_argmin_matches_the_planner_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    prob = sc.single_plan()
    prob.params.update(K=70001, T=12)                 # several blocks and a ragged tail
    stream = torch.cuda.current_stream().cuda_stream
    with mp.Planner(prob.params) as pl:
        for _ in range(2):                            # consecutive calls share the scratch
            u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)
            S = pl.get_costs()
            s_min, arg, n_fin = _argmin_noalloc(torch, S, stream)
            assert arg == info["argmin"]
            assert s_min == info["s_min"]
            assert n_fin == info["n_finite"]


def test_noalloc_argmin_handles_ties_and_non_finite_costs():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    S = rng.uniform(10.0, 20.0, 300000)
    S[[5, 77, 299999]] = 1.5                          # a three-way tie: lowest index wins
    S[rng.integers(0, S.size, 1000)] = np.inf
    S[rng.integers(0, S.size, 1000)] = np.nan
    S[[5, 77, 299999]] = 1.5
    for _ in range(2):
        s_min, arg, n_fin = _argmin_noalloc(torch, S, stream)
        assert (s_min, arg, n_fin) == (1.5, 5, int(np.isfinite(S).sum()))
    s_min, arg, n_fin = _argmin_noalloc(torch, np.full(1000, np.inf), stream)
    assert arg == -1 and n_fin == 0


def test_noalloc_argmin_rejects_sizes_above_its_capacity():
    torch = pytest.importorskip("torch")
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    rc = mp.lib().mppi_argmin_noalloc(p, (1 << 28) + 1, p, p, p, None)   # rejected before any launch
    assert rc == -6
    rc = mp.lib().mppi_argmin_noalloc(p, 0, p, p, p, None)
    assert rc == -1
