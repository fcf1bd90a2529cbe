"""The C-ABI library builds, loads and exports every entry point include/mppi.h declares.

These run without a GPU: no compute call is made except ones that must fail
cleanly (argument validation happens before any CUDA call; creating a planner
without a device reports MPPI_ERR_CUDA).
"""
import ctypes
import os
import re
import subprocess

import numpy as np

import pytest

import paper_2308_01654_gb300 as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mppi_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("mppi_create", "mppi_plan", "mppi_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    path = mp._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(mppi_\w+)", out))
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name)


def test_binding_covers_every_declared_symbol():
    assert declared_functions() == set(mp.SIGNATURES)


def test_struct_layouts_match_the_header():
    # sizes follow from the field lists of include/mppi.h on an LP64 ABI
    assert ctypes.sizeof(mp.MppiInfo) == 32
    assert ctypes.sizeof(mp.MppiParams) == (4 * 2 + 8 * 2 + 8 * 6 + 8 * 4 + 8 * 6 + 8 * 2 + 8 * 2 + 4 * 2 + 8 * 16
                                            + 4 * 4 + 8 + 4 * 5 + 4)


def test_default_params_are_the_papers_weights():
    p = mp.default_params(1024, 50, 0.05)
    assert (p.w_dist, p.w_target, p.w_yaw, p.w_speed, p.w_safe) == (15.0, 7.0, 120.0, 5.0, 25.0)
    assert p.R[0] == pytest.approx(p.lam / p.sigma[0] ** 2) and p.R[1] == pytest.approx(p.lam / p.sigma[1] ** 2)


def test_status_strings():
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert mp.lib().mppi_status_string(s).decode().startswith(mp.STATUS[s])


@pytest.mark.parametrize("bad", [dict(K=0), dict(T=0), dict(T=5000), dict(dt=0.0), dict(lam=-1.0),
                                 dict(n_ego=9), dict(sigma=[-0.1, 0.1]), dict(group=3), dict(group=-3), dict(group=-32),
                                 dict(block=100), dict(block=928), dict(block=1024)])
def test_invalid_params_are_rejected_before_any_cuda_call(bad):
    from paper_2308_01654_gb300 import scenarios
    p = scenarios.default_params(64, 10, 0.05)
    p.update(bad)
    if p["n_ego"] > 8:
        p["ego_offset"] = [0.0] * 9
        p["ego_radius"] = [1.0] * 9
    with pytest.raises(mp.MppiError) as e:
        mp.Planner(p)
    assert e.value.status == -1


def test_no_cpu_fallback_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2308_01654_gb300 import scenarios
    with pytest.raises(mp.MppiError) as e:
        mp.Planner(scenarios.default_params(64, 10, 0.05))
    assert e.value.status == -3


def test_array_addresses_passed_to_the_library():
    """The binding passes arrays as void* addresses taken through the buffer protocol (read-only
    and empty arrays through ndarray.ctypes): the address must be the array's data pointer."""
    a = np.arange(12, dtype=np.float64).reshape(6, 2)
    ro = np.arange(5, dtype=np.float64)
    ro.setflags(write=False)
    for arr in (a, ro, np.empty((0, 5)), np.zeros(7, dtype=np.float32), np.zeros(3, dtype=np.uint32), a[2:]):
        assert mp._dp(arr) == arr.ctypes.data
    assert mp._dp(None) is None
    # the request record's pointer fields take the same addresses
    r = mp.MppiRequest()
    r.x0, r.ref_xy = mp._dp(a), mp._dp(ro)
    assert r.x0 == a.ctypes.data and r.ref_xy == ro.ctypes.data
