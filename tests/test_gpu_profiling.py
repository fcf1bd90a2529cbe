"""Per-kernel timing modes of the planner: events around every kernel, or around the rollout
only.  Tracing never changes the results."""
import math

import numpy as np
import pytest

import paper_2308_01654_gb300 as mp
from paper_2308_01654_gb300 import scenarios as sc

pytestmark = pytest.mark.gpu


def test_profiling_modes_time_the_kernels_and_leave_results_unchanged():
    prob = sc.by_name("single_plan")
    out = {}
    for mode in (0, 1, 2):
        with mp.Planner(prob.params) as pl:
            if mode:
                pl.set_profiling(mode)
            u, x, info = pl.plan(prob.x0, prob.ref, prob.circles, prob.centres)
            out[mode] = (u, x)
            if mode == 1:
                kt = pl.kernel_times()
                assert set(kt) == set(mp.KERNELS)
                # prep and noise are one launch and the rollout ends with the argmin: those two
                # stages hold no kernel of their own (fp32 noise)
                assert all(kt[k] > 0.0 for k in ("prep", "rollout", "weights", "wsum", "finalize"))
                assert kt["noise"] >= 0.0 and kt["argmin"] >= 0.0
            elif mode == 2:
                kt = pl.kernel_times()
                assert kt["rollout"] > 0.0
                assert all(math.isnan(v) for k, v in kt.items() if k != "rollout")
            else:
                with pytest.raises(mp.MppiError):
                    pl.kernel_times()
    for mode in (1, 2):
        np.testing.assert_array_equal(out[mode][0], out[0][0])
        np.testing.assert_array_equal(out[mode][1], out[0][1])


def test_profiling_mode_out_of_range_is_refused():
    prob = sc.by_name("single_plan")
    with mp.Planner(prob.params) as pl:
        assert mp.lib().mppi_set_profiling(pl._h, 3) == -1
        assert mp.lib().mppi_set_profiling(pl._h, -1) == -1
