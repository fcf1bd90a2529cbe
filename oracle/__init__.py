"""ctypes wrapper around the FP64 CPU oracle (``mppi_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports it.

``build()`` compiles ``mppi_oracle.c`` with gcc (``-O2 -fopenmp``, no ``-ffast-math``
so IEEE double semantics hold) into ``oracle/_build/libmppi_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_HDR = os.path.join(_HERE, "mppi_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmppi_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_EGO = 8


class OrcParams(C.Structure):
    _fields_ = [
        ("K", C.c_int32), ("T", C.c_int32),
        ("dt", C.c_double), ("wheelbase", C.c_double),
        ("sigma", C.c_double * 2), ("u_min", C.c_double * 2), ("u_max", C.c_double * 2),
        ("lam", C.c_double), ("gamma", C.c_double), ("R", C.c_double * 2),
        ("w_dist", C.c_double), ("w_target", C.c_double), ("w_yaw", C.c_double),
        ("w_speed", C.c_double), ("w_safe", C.c_double), ("w_terminal", C.c_double),
        ("v_ref", C.c_double), ("v_max", C.c_double),
        ("d_safe_c", C.c_double), ("d_safe_0", C.c_double),
        ("collision_only", C.c_int32),
        ("n_ego", C.c_int32),
        ("ego_offset", C.c_double * MAX_EGO), ("ego_radius", C.c_double * MAX_EGO),
        ("ref_mode", C.c_int32),
        ("sg_enable", C.c_int32), ("shift", C.c_int32), ("noise_bf16", C.c_int32),
        ("seed", C.c_uint64),
        ("session", C.c_uint32),
        ("model", C.c_int32),
        ("cost_to_go", C.c_int32),
    ]


class OrcInfo(C.Structure):
    _fields_ = [("argmin", C.c_int32), ("n_finite", C.c_int32), ("s_min", C.c_double), ("eta", C.c_double)]


def _stale() -> bool:
    if not os.path.exists(_LIB_PATH):
        return True
    t = os.path.getmtime(_LIB_PATH)
    return any(os.path.getmtime(f) > t for f in (_SRC, _HDR))


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP) if it is missing or stale."""
    with _lock:
        if force or _stale():
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        dp = C.POINTER(C.c_double)
        u32p = C.POINTER(C.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_uniform24.argtypes = [C.c_uint32]
        L.orc_uniform24.restype = C.c_double
        L.orc_box_muller.argtypes = [C.c_double, C.c_double, dp, dp]
        L.orc_round_bf16.argtypes = [C.c_double]
        L.orc_round_bf16.restype = C.c_double
        L.orc_noise.argtypes = [C.POINTER(OrcParams), C.c_uint32, dp]
        L.orc_bicycle_step.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.orc_bicycle5_step.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.orc_softmin_update_ctg.argtypes = [C.c_int32, C.c_int32, dp, dp, C.c_double, dp, dp]
        L.orc_softmin_update_ctg.restype = C.c_int32
        L.orc_rollout_cost_ctg.argtypes = [C.POINTER(OrcParams), dp, dp, dp, dp, C.c_int32, dp, C.c_int32,
                                           dp, dp, dp, dp]
        L.orc_rollout_cost_ctg.restype = C.c_double
        L.orc_nearest_ref.argtypes = [dp, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.POINTER(C.c_int32), dp, dp]
        L.orc_nearest_ref.restype = C.c_double
        L.orc_wrap_angle.argtypes = [C.c_double]
        L.orc_wrap_angle.restype = C.c_double
        L.orc_obstacle_distance.argtypes = [C.POINTER(OrcParams), dp, dp, dp, C.c_int32]
        L.orc_obstacle_distance.restype = C.c_double
        L.orc_rollout_cost.argtypes = [C.POINTER(OrcParams), dp, dp, dp, dp, C.c_int32, dp, C.c_int32,
                                       dp, dp, dp]
        L.orc_rollout_cost.restype = C.c_double
        L.orc_softmin_update.argtypes = [C.c_int32, C.c_int32, dp, dp, C.c_double, dp,
                                         C.POINTER(OrcInfo), dp]
        L.orc_softmin_update.restype = C.c_int32
        L.orc_savgol5.argtypes = [C.c_int32, dp, C.c_int32, dp]
        L.orc_rollout_states.argtypes = [C.POINTER(OrcParams), dp, dp, dp]
        L.orc_plan.argtypes = [C.POINTER(OrcParams), C.c_uint32, dp, dp, C.c_int32, dp, C.c_int32, dp,
                               dp, dp, dp, dp, dp, dp, C.POINTER(OrcInfo)]
        L.orc_plan.restype = C.c_int
        L.orc_costs_range.argtypes = [C.POINTER(OrcParams), C.c_uint32, dp, dp, dp, C.c_int32, dp,
                                      C.c_int32, dp, C.c_int32, C.c_int32, dp]
        L.orc_costs_range.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_params(p: Dict[str, object]) -> OrcParams:
    """Fill the oracle's parameter struct from a scenario parameter dictionary."""
    s = OrcParams()
    s.K, s.T = int(p["K"]), int(p["T"])
    s.dt, s.wheelbase = float(p["dt"]), float(p["wheelbase"])
    for name in ("sigma", "u_min", "u_max", "R"):
        v = p[name]
        arr = getattr(s, name)
        arr[0], arr[1] = float(v[0]), float(v[1])
    s.lam, s.gamma = float(p["lam"]), float(p["gamma"])
    for name in ("w_dist", "w_target", "w_yaw", "w_speed", "w_safe", "w_terminal", "v_ref", "v_max",
                 "d_safe_c", "d_safe_0"):
        setattr(s, name, float(p[name]))
    s.collision_only = int(p["collision_only"])
    n_ego = int(p["n_ego"])
    s.n_ego = n_ego                       # values above MAX_EGO are rejected by the oracle itself
    for e in range(min(max(n_ego, 0), MAX_EGO)):
        s.ego_offset[e] = float(p["ego_offset"][e])
        s.ego_radius[e] = float(p["ego_radius"][e])
    s.ref_mode = int(p["ref_mode"])
    s.sg_enable, s.shift, s.noise_bf16 = int(p["sg_enable"]), int(p["shift"]), int(p["noise_bf16"])
    s.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    s.session = int(p["session"]) & 0xFFFFFFFF
    s.model = int(p.get("model", 0))
    s.cost_to_go = int(p.get("cost_to_go", 0))
    return s


# ---------------------------------------------------------------------------
# thin numpy front-ends
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform24(word: int) -> float:
    return lib().orc_uniform24(int(word) & 0xFFFFFFFF)


def box_muller(u0: float, u1: float):
    a, b = C.c_double(), C.c_double()
    lib().orc_box_muller(u0, u1, C.byref(a), C.byref(b))
    return a.value, b.value


def round_bf16(z: float) -> float:
    return lib().orc_round_bf16(float(z))


def noise(p: Dict[str, object], iter_: int) -> np.ndarray:
    """Unit normals z[T][K][2] of one iteration."""
    s = make_params(p)
    z = np.empty((s.T, s.K, 2), dtype=np.float64)
    lib().orc_noise(C.byref(s), int(iter_) & 0xFFFFFFFF, _dp(z))
    return z


def bicycle_step(x, a: float, delta: float, dt: float, wheelbase: float) -> np.ndarray:
    xi = _f64(x)
    out = np.empty(4)
    lib().orc_bicycle_step(_dp(xi), a, delta, dt, wheelbase, _dp(out))
    return out


def bicycle5_step(x, a: float, omega: float, dt: float, wheelbase: float) -> np.ndarray:
    """The steering-rate form: state (x, y, yaw, v, delta), control (a, omega)."""
    xi = _f64(x)
    out = np.empty(5)
    lib().orc_bicycle5_step(_dp(xi), a, omega, dt, wheelbase, _dp(out))
    return out


def nx_of(p) -> int:
    """State entries of the parameter set's model: 4, or 5 for the steering-rate form."""
    return 5 if int(p.get("model", 0)) == 1 else 4


def nearest_ref(ref, px: float, py: float, mode: int = 0):
    r = _f64(ref)
    idx = C.c_int32()
    th, m = C.c_double(), C.c_double()
    d2 = lib().orc_nearest_ref(_dp(r), r.shape[0], mode, px, py, C.byref(idx), C.byref(th), C.byref(m))
    return d2, idx.value, th.value, m.value


def wrap_angle(d: float) -> float:
    return lib().orc_wrap_angle(float(d))


def obstacle_distance(p, x, circles, centres_xy) -> float:
    s = make_params(p)
    c = _f64(circles).reshape(-1, 5)
    cxy = _f64(centres_xy).reshape(-1, 2)
    return lib().orc_obstacle_distance(C.byref(s), _dp(_f64(x)), _dp(c), _dp(cxy), c.shape[0])


def rollout_cost(p, x0, U, z_k, ref, circles, centres=None):
    """S of one sample with its unit normals z_k[T][2]; returns (S, eps'[T][2], margin)."""
    s = make_params(p)
    c = _f64(circles).reshape(-1, 5)
    eps = np.empty((s.T, 2))
    m = C.c_double()
    r = _f64(ref)
    S = lib().orc_rollout_cost(C.byref(s), _dp(_f64(x0)), _dp(_f64(U)), _dp(_f64(z_k)), _dp(r), r.shape[0],
                               _dp(c), c.shape[0], _dp(None if centres is None else _f64(centres)),
                               _dp(eps), C.pointer(m))
    return S, eps, m.value


def softmin_update(S, eps, lam: float):
    """Eq. (11) on given costs S[K] and clamped perturbations eps'[T][K][2]."""
    S = _f64(S)
    eps = _f64(eps)
    T, K = eps.shape[0], eps.shape[1]
    dU = np.empty((T, 2))
    w = np.empty(K)
    info = OrcInfo()
    lib().orc_softmin_update(K, T, _dp(S), _dp(eps), lam, _dp(dU), C.byref(info), _dp(w))
    return dU, w, info


def softmin_update_ctg(Sctg, eps, lam: float):
    """Eq. (11) read per step: Sctg[T][K] costs from step t on, eps'[T][K][2]; returns (dU, eta_t)."""
    Sctg = _f64(Sctg)
    eps = _f64(eps)
    T, K = Sctg.shape
    dU = np.empty((T, 2))
    eta = np.empty(T)
    lib().orc_softmin_update_ctg(K, T, _dp(Sctg), _dp(eps), lam, _dp(dU), _dp(eta))
    return dU, eta


def rollout_cost_ctg(p, x0, U, z_k, ref, circles, centres=None):
    """S of one sample and its cost from every step on: (S, ctg[T], eps'[T][2])."""
    s = make_params(p)
    c = _f64(circles).reshape(-1, 5)
    eps = np.empty((s.T, 2))
    ctg = np.empty(s.T)
    m = C.c_double()
    r = _f64(ref)
    S = lib().orc_rollout_cost_ctg(C.byref(s), _dp(_f64(x0)), _dp(_f64(U)), _dp(_f64(z_k)), _dp(r), r.shape[0],
                                   _dp(c), c.shape[0], _dp(None if centres is None else _f64(centres)),
                                   _dp(eps), C.pointer(m), _dp(ctg))
    return S, ctg, eps


def savgol5(u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    lib().orc_savgol5(u.shape[0], _dp(u), 1, _dp(out))
    return out


def rollout_states(p, x0, u) -> np.ndarray:
    s = make_params(p)
    xs = np.empty((s.T + 1, nx_of(p)))
    lib().orc_rollout_states(C.byref(s), _dp(_f64(x0)), _dp(_f64(u)), _dp(xs))
    return xs


class PlanResult:
    def __init__(self, rc, U, u_star, x_star, S, margin, eps, info):
        self.rc, self.U, self.u_star, self.x_star = rc, U, u_star, x_star
        self.S, self.margin, self.eps, self.info = S, margin, eps, info


def plan(prob, U=None, iter_: int = 0, want_eps: bool = False, params=None) -> PlanResult:
    """One MPPI iteration of the oracle on a scenarios.Problem; U (warm start) is copied."""
    p = params if params is not None else prob.params
    s = make_params(p)
    K, T = s.K, s.T
    Uw = np.zeros((T, 2)) if U is None else _f64(U).copy()
    u_star = np.zeros((T, 2))
    x_star = np.zeros((T + 1, nx_of(p)))
    S = np.empty(K)
    margin = np.empty(K)
    eps = np.empty((T, K, 2)) if want_eps else None
    info = OrcInfo()
    ref = _f64(prob.ref)
    circ = _f64(prob.circles).reshape(-1, 5)
    cen = None if prob.centres is None else _f64(prob.centres)
    rc = lib().orc_plan(C.byref(s), int(iter_) & 0xFFFFFFFF, _dp(_f64(prob.x0)), _dp(ref), ref.shape[0],
                        _dp(circ), circ.shape[0], _dp(cen), _dp(Uw), _dp(u_star), _dp(x_star), _dp(S),
                        _dp(margin), _dp(eps), C.byref(info))
    return PlanResult(rc, Uw, u_star, x_star, S, margin, eps, info)


def costs_range(prob, k0: int, count: int, U=None, iter_: int = 0) -> np.ndarray:
    """Sample costs S[k0:k0+count] only (the bounded CPU baseline)."""
    s = make_params(prob.params)
    Uw = np.zeros((s.T, 2)) if U is None else _f64(U)
    out = np.empty(count)
    ref = _f64(prob.ref)
    circ = _f64(prob.circles).reshape(-1, 5)
    cen = None if prob.centres is None else _f64(prob.centres)
    rc = lib().orc_costs_range(C.byref(s), int(iter_) & 0xFFFFFFFF, _dp(_f64(prob.x0)), _dp(Uw), _dp(ref),
                               ref.shape[0], _dp(circ), circ.shape[0], _dp(cen), k0, count, _dp(out))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's sample loops (timing only; results do not depend on it)."""
    lib().orc_set_num_threads(int(n))


INF = math.inf
