"""GB300-native MPPI motion planner (arXiv 2308.01654): Python binding of ``libmppi.so``.

The binding only marshals arguments to the C ABI declared in ``include/mppi.h``;
every step of the iteration runs in the library's CUDA kernels.  There is no CPU
fallback: if the library cannot be built or loaded, or no GPU is present, the
calls raise.

Typical use::

    from paper_2308_01654_gb300 import Planner, scenarios
    prob = scenarios.single_plan()
    with Planner(prob.params) as pl:
        u, x, info = pl.plan(prob.x0, prob.ref, prob.circles)

``plan_device`` takes torch CUDA tensors (float64) and queues the iteration on the
planner's stream without host copies.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, Optional, Tuple

import numpy as np

from . import _build

MAX_EGO = 8
MAX_T = 1024
MAX_REF = 4096
MAX_CIRC = 1024

FLAG_NONFINITE_INPUT = 1
FLAG_TIMEOUT = 2

STATUS = {0: "MPPI_OK", -1: "MPPI_ERR_ARG", -2: "MPPI_ERR_OOM", -3: "MPPI_ERR_CUDA", -4: "MPPI_ERR_NUMERIC",
          -5: "MPPI_ERR_TIMEOUT", -6: "MPPI_ERR_CAPACITY"}


class MppiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MppiParams(C.Structure):
    _fields_ = [
        ("K", C.c_int32), ("T", C.c_int32), ("dt", C.c_double), ("wheelbase", C.c_double),
        ("sigma", C.c_double * 2), ("u_min", C.c_double * 2), ("u_max", C.c_double * 2),
        ("lam", C.c_double), ("gamma", C.c_double), ("R", C.c_double * 2),
        ("w_dist", C.c_double), ("w_target", C.c_double), ("w_yaw", C.c_double), ("w_speed", C.c_double),
        ("w_safe", C.c_double), ("w_terminal", C.c_double),
        ("v_ref", C.c_double), ("v_max", C.c_double),
        ("d_safe_c", C.c_double), ("d_safe_0", C.c_double),
        ("collision_only", C.c_int32), ("n_ego", C.c_int32),
        ("ego_offset", C.c_double * MAX_EGO), ("ego_radius", C.c_double * MAX_EGO),
        ("ref_mode", C.c_int32), ("sg_enable", C.c_int32), ("shift", C.c_int32), ("noise_bf16", C.c_int32),
        ("seed", C.c_uint64), ("session", C.c_uint32), ("group", C.c_int32), ("block", C.c_int32),
        ("model", C.c_int32), ("cost_to_go", C.c_int32),
    ]


class MppiInfo(C.Structure):
    _fields_ = [("argmin", C.c_int32), ("n_finite", C.c_int32), ("s_min", C.c_double), ("eta", C.c_double),
                ("iter", C.c_uint64)]

    def as_dict(self) -> Dict[str, object]:
        return dict(argmin=self.argmin, n_finite=self.n_finite, s_min=self.s_min, eta=self.eta, iter=self.iter)


_lib = None

# every entry point of include/mppi.h with its ctypes signature
_VP = C.c_void_p
SIGNATURES = {
    "mppi_default_params": (C.c_int, [C.POINTER(MppiParams), C.c_int32, C.c_int32, C.c_double]),
    "mppi_create": (C.c_int, [C.POINTER(MppiParams), C.c_int, _VP, C.c_int32, C.c_int32, C.POINTER(_VP)]),
    "mppi_destroy": (C.c_int, [_VP]),
    "mppi_set_stream": (C.c_int, [_VP, _VP]),
    "mppi_plan": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP, _VP, _VP, C.POINTER(MppiInfo)]),
    "mppi_plan_device": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP, _VP, _VP, C.POINTER(MppiInfo)]),
    "mppi_sync": (C.c_int, [_VP, C.POINTER(MppiInfo)]),
    "mppi_rollout_stats": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP, C.POINTER(C.c_uint64)]),
    "mppi_autotune": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP, C.c_char_p,
                                C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mppi_set_controls": (C.c_int, [_VP, _VP, C.c_uint64]),
    "mppi_get_controls": (C.c_int, [_VP, _VP, C.POINTER(C.c_uint64)]),
    "mppi_get_costs": (C.c_int, [_VP, _VP]),
    "mppi_get_noise": (C.c_int, [_VP, _VP]),
    "mppi_philox": (C.c_int, [C.c_uint64, _VP, C.c_int32, _VP]),
    "mppi_set_profiling": (C.c_int, [_VP, C.c_int32]),
    "mppi_kernel_times": (C.c_int, [_VP, _VP, C.c_int32]),
    "mppi_argmin_noalloc": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, _VP]),
    "mppi_debug_inject_flags": (C.c_int, [_VP, C.c_int32]),
    "mppi_debug_check_hits": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]),
    "mppi_debug_check_selftest": (C.c_int, [C.c_int, C.POINTER(C.c_uint64)]),
    "mppi_slice_costs": (C.c_int, [_VP, C.c_int64, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mppi_slice_sums": (C.c_int, [_VP, C.c_double, C.POINTER(C.c_double), _VP]),
    "mppi_slice_finalize": (C.c_int, [_VP, C.c_double, _VP, C.c_int32, C.c_double, C.c_int32, _VP, _VP,
                                      C.POINTER(MppiInfo)]),
    "mppi_batch_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int32, C.c_int32, C.c_int, C.POINTER(_VP)]),
    "mppi_batch_destroy": (C.c_int, [_VP]),
    "mppi_batch_submit": (C.c_int, [_VP, _VP, C.c_int32, C.POINTER(C.c_int32)]),
    "mppi_batch_wait": (C.c_int, [_VP, C.c_int32]),
    "mppi_batch_plan": (C.c_int, [_VP, _VP, C.c_int32]),
    "mppi_batch_autotune": (C.c_int, [_VP, _VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mppi_box_to_circles": (C.c_int32, [C.c_double] * 7 + [C.c_int32, _VP, C.c_int32]),
    "mppi_batch_set_launch": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "mppi_batch_set_controls": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, C.c_uint64]),
    "mppi_batch_get_controls": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, C.POINTER(C.c_uint64)]),
    "mppi_batch_get_costs": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, C.c_int32]),
    "mppi_batch_last_error": (C.c_char_p, [_VP]),
    "mppi_server_create": (C.c_int, [_VP, C.POINTER(_VP)]),
    "mppi_server_destroy": (C.c_int, [_VP]),
    "mppi_server_autotune": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, _VP, C.c_int32, C.c_int32,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mppi_server_enqueue": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP,
                                      C.POINTER(C.c_uint64)]),
    "mppi_server_poll": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "mppi_server_pending": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_uint64),
                                      C.POINTER(C.c_uint64)]),
    "mppi_server_set_controls": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, C.c_uint64]),
    "mppi_server_set_watchdog": (C.c_int, [_VP, C.c_double]),
    "mppi_server_timeouts": (C.c_int, [_VP, C.POINTER(C.c_uint64)]),
    "mppi_server_snapshot": (C.c_int, [_VP, C.c_char_p]),
    "mppi_server_restore": (C.c_int, [_VP, C.c_char_p]),
    "mppi_server_last_error": (C.c_char_p, [_VP]),
    "mppi_status_string": (C.c_char_p, [C.c_int]),
    "mppi_last_error": (C.c_char_p, [_VP]),
}


def library_path() -> str:
    return _build.LIB


def load_library(path: str):
    """Load a build of the library at `path` with every entry point's signature."""
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    """Build (if needed) and load libmppi.so; raises if that is impossible."""
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


class use_library:
    """Context manager: route the binding to another build of the library (e.g. the
    bounds-checking debug build, _build.build(checks=True)) and back."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _lib
        self.old = _lib
        _lib = self.L
        return self.L

    def __exit__(self, *exc):
        global _lib
        _lib = self.old


def check_hits():
    """(enabled, violations since the last call) of the bounds-checking debug build."""
    en, hits = C.c_int32(), C.c_uint64()
    _check(lib().mppi_debug_check_hits(C.byref(en), C.byref(hits)))
    return bool(en.value), int(hits.value)


def check_selftest(device: int = 0) -> int:
    hits = C.c_uint64()
    _check(lib().mppi_debug_check_selftest(int(device), C.byref(hits)))
    return int(hits.value)


def _check(rc: int, ctx=None):
    if rc != 0:
        msg = lib().mppi_last_error(ctx)
        raise MppiError(rc, msg.decode() if msg else "")


def make_params(p: Dict[str, object]) -> MppiParams:
    """Fill the C parameter struct from a parameter dictionary (scenarios.default_params keys)."""
    s = MppiParams()
    s.K, s.T = int(p["K"]), int(p["T"])
    s.dt, s.wheelbase = float(p["dt"]), float(p["wheelbase"])
    for name in ("sigma", "u_min", "u_max", "R"):
        arr = getattr(s, name)
        arr[0], arr[1] = float(p[name][0]), float(p[name][1])
    s.lam, s.gamma = float(p["lam"]), float(p["gamma"])
    for name in ("w_dist", "w_target", "w_yaw", "w_speed", "w_safe", "w_terminal", "v_ref", "v_max",
                 "d_safe_c", "d_safe_0"):
        setattr(s, name, float(p[name]))
    s.collision_only = int(p["collision_only"])
    s.n_ego = int(p["n_ego"])
    for e in range(min(max(s.n_ego, 0), MAX_EGO)):
        s.ego_offset[e] = float(p["ego_offset"][e])
        s.ego_radius[e] = float(p["ego_radius"][e])
    s.ref_mode, s.sg_enable, s.shift = int(p["ref_mode"]), int(p["sg_enable"]), int(p["shift"])
    s.noise_bf16 = int(p["noise_bf16"])
    s.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    s.session = int(p["session"]) & 0xFFFFFFFF
    s.group = int(p.get("group", 0))
    s.block = int(p.get("block", 0))
    s.model = int(p.get("model", 0))
    s.cost_to_go = int(p.get("cost_to_go", 0))
    return s


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: Optional[np.ndarray]):
    """Address of an array's data for a void* parameter (None stays NULL).  Through the buffer
    protocol when the array is writable (a few times cheaper than ndarray.ctypes, which is most
    of the binding's cost per call), else through ndarray.ctypes (read-only or empty arrays)."""
    if a is None:
        return None
    try:
        return C.addressof(C.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.ctypes.data


class Planner:
    """One planner context (device buffers, stream, warm start) on one GPU."""

    def __init__(self, params: Dict[str, object], device: int = 0, stream: Optional[int] = None,
                 max_ref: int = 0, max_circ: int = 0):
        self.params = dict(params)
        self.K, self.T = int(params["K"]), int(params["T"])
        self.nx = 5 if int(params.get("model", 0)) == 1 else 4      # state entries
        self._p = make_params(params)
        h = _VP()
        rc = lib().mppi_create(C.byref(self._p), int(device), _VP(stream) if stream else None, int(max_ref),
                               int(max_circ), C.byref(h))
        _check(rc)
        self._h = h

    # context management ------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream: Optional[int]):
        _check(lib().mppi_set_stream(self._h, _VP(stream) if stream else None), self._h)

    # the iteration -----------------------------------------------------------
    def plan(self, x0, ref, circles=None, centres=None) -> Tuple[np.ndarray, np.ndarray, Dict[str, object]]:
        """One MPPI iteration from host arrays; returns (u*[T][2], x*[T+1][nx], info)."""
        x0 = _f64(x0)
        ref = _f64(ref).reshape(-1, 2)
        circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        cen = None if centres is None else _f64(centres)
        u = np.empty((self.T, 2))
        x = np.empty((self.T + 1, self.nx))
        info = MppiInfo()
        rc = lib().mppi_plan(self._h, _dp(x0), _dp(ref), ref.shape[0], _dp(circ) if circ.shape[0] else None,
                             circ.shape[0], _dp(cen), _dp(u), _dp(x), C.byref(info))
        _check(rc, self._h)
        return u, x, info.as_dict()

    def plan_device(self, x0, ref, circles, centres, u_out, x_out, wait: bool = False):
        """One iteration on torch CUDA float64 tensors, queued on the planner's stream."""
        info = MppiInfo() if wait else None
        ptr = (lambda t: None if t is None else _VP(t.data_ptr()))
        n_circ = 0 if circles is None else int(circles.shape[0])
        rc = lib().mppi_plan_device(self._h, ptr(x0), ptr(ref), int(ref.shape[0]), ptr(circles) if n_circ else None,
                                    n_circ, ptr(centres), ptr(u_out), ptr(x_out),
                                    C.byref(info) if wait else None)
        _check(rc, self._h)
        return info.as_dict() if wait else None

    def autotune(self, x0, ref, circles=None, centres=None, cache_path: Optional[str] = None):
        """Pick the rollout kernel's (group, block) for these inputs; returns the choice."""
        x0 = _f64(x0)
        ref = _f64(ref).reshape(-1, 2)
        circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        cen = None if centres is None else _f64(centres)
        g, b = C.c_int32(), C.c_int32()
        rc = lib().mppi_autotune(self._h, _dp(x0), _dp(ref), ref.shape[0], _dp(circ) if circ.shape[0] else None,
                                 circ.shape[0], _dp(cen), cache_path.encode() if cache_path else None,
                                 C.byref(g), C.byref(b))
        _check(rc, self._h)
        return g.value, b.value

    STAT_NAMES = ("range_boxes", "chunk_boxes", "segments", "refinements", "circles_tested", "candidates",
                  "in_band")

    def rollout_stats(self, x0, ref, circles=None, centres=None) -> Dict[str, float]:
        """Work counters of the pruned searches, per rollout-step."""
        x0 = _f64(x0)
        ref = _f64(ref).reshape(-1, 2)
        circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        cen = None if centres is None else _f64(centres)
        out = (C.c_uint64 * len(self.STAT_NAMES))()
        rc = lib().mppi_rollout_stats(self._h, _dp(x0), _dp(ref), ref.shape[0], _dp(circ) if circ.shape[0] else None,
                                      circ.shape[0], _dp(cen), out)
        _check(rc, self._h)
        steps = float(self.K) * float(self.T)
        return {n: out[i] / steps for i, n in enumerate(self.STAT_NAMES)}

    def sync(self) -> Dict[str, object]:
        info = MppiInfo()
        _check(lib().mppi_sync(self._h, C.byref(info)), self._h)
        return info.as_dict()

    # warm start and debug views ------------------------------------------------
    def set_controls(self, U, iter_: int = 0):
        U = _f64(U).reshape(self.T, 2)
        _check(lib().mppi_set_controls(self._h, _dp(U), int(iter_)), self._h)

    def get_controls(self):
        U = np.empty((self.T, 2))
        it = C.c_uint64()
        _check(lib().mppi_get_controls(self._h, _dp(U), C.byref(it)), self._h)
        return U, it.value

    def get_costs(self) -> np.ndarray:
        S = np.empty(self.K)
        _check(lib().mppi_get_costs(self._h, _dp(S)), self._h)
        return S

    def get_noise(self) -> np.ndarray:
        z = np.empty((self.T, self.K, 2), dtype=np.float32)
        _check(lib().mppi_get_noise(self._h, _dp(z)), self._h)
        return z

    def debug_inject_flags(self, flags: int):
        """Debug: the next iteration raises these device status flags between its rollout and
        its update (FLAG_TIMEOUT = 2, FLAG_NONFINITE_INPUT = 1)."""
        _check(lib().mppi_debug_inject_flags(self._h, int(flags)), self._h)

    # K-partitioned iteration (this context holds samples k_offset .. k_offset + K - 1) -----
    def slice_costs(self, k_offset: int, x0, ref, circles=None, centres=None):
        """Noise, rollouts and costs of this slice; returns (s_min, global argmin, n_finite)."""
        x0 = _f64(x0)
        ref = _f64(ref).reshape(-1, 2)
        circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        cen = None if centres is None else _f64(centres)
        s, a, n = C.c_double(), C.c_int32(), C.c_int32()
        rc = lib().mppi_slice_costs(self._h, int(k_offset), _dp(x0), _dp(ref), ref.shape[0],
                                    _dp(circ) if circ.shape[0] else None, circ.shape[0], _dp(cen), C.byref(s),
                                    C.byref(a), C.byref(n))
        _check(rc, self._h)
        return s.value, a.value, n.value

    def slice_sums(self, s_min: float):
        """The slice's softmin normaliser and weighted noise sums against the global minimum."""
        eta = C.c_double()
        du = np.empty((self.T, 2))
        _check(lib().mppi_slice_sums(self._h, float(s_min), C.byref(eta), _dp(du)), self._h)
        return eta.value, du

    def slice_finalize(self, eta: float, du, n_finite: int, s_min: float, argmin: int):
        """The update from the totals over all slices; returns (u*, x*, info) like plan()."""
        du = _f64(du).reshape(self.T, 2)
        u = np.empty((self.T, 2))
        x = np.empty((self.T + 1, self.nx))
        info = MppiInfo()
        rc = lib().mppi_slice_finalize(self._h, float(eta), _dp(du), int(n_finite), float(s_min), int(argmin),
                                       _dp(u), _dp(x), C.byref(info))
        _check(rc, self._h)
        return u, x, info.as_dict()


KERNELS = ("prep", "noise", "rollout", "argmin", "weights", "wsum", "finalize")


def _kernel_times(self) -> Dict[str, float]:
    """Per-kernel durations (ms) of the last iteration; needs set_profiling(True)."""
    ms = (C.c_float * len(KERNELS))()
    _check(lib().mppi_kernel_times(self._h, ms, len(KERNELS)), self._h)
    return dict(zip(KERNELS, [float(v) for v in ms]))


def _set_profiling(self, on=True):
    """True / 1: events around every kernel; 2: around the rollout only (the others stay chained)."""
    mode = 2 if on == 2 else (1 if on else 0)
    _check(lib().mppi_set_profiling(self._h, mode), self._h)


Planner.kernel_times = _kernel_times
Planner.set_profiling = _set_profiling


def box_to_circles(x: float, y: float, yaw: float, length: float, width: float, vx: float = 0.0,
                   vy: float = 0.0, n: int = 0) -> np.ndarray:
    """Circles (rows x, y, r, vx, vy) covering an oriented rectangular object (mppi_box_to_circles)."""
    ok = width > 0 and length > 0 and np.isfinite(length / width)
    cap = n if n > 0 else (max(1, int(np.ceil(length / width))) if ok else 1)
    out = np.zeros((cap, 5), dtype=np.float64)
    rc = lib().mppi_box_to_circles(float(x), float(y), float(yaw), float(length), float(width), float(vx),
                                   float(vy), int(n), _dp(out), cap)
    if rc < 0:
        raise MppiError(rc, "mppi_box_to_circles")
    return out[:rc]


def philox(seed: int, ctr) -> np.ndarray:
    """Raw Philox4x32-10 words computed on the GPU for counters ctr[n][4]."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    out = np.empty_like(c)
    rc = lib().mppi_philox(int(seed) & 0xFFFFFFFFFFFFFFFF, _dp(c), c.shape[0], _dp(out))
    _check(rc)
    return out


def default_params(K: int, T: int, dt: float) -> MppiParams:
    p = MppiParams()
    _check(lib().mppi_default_params(C.byref(p), K, T, dt))
    return p


INF = math.inf


class MppiRequest(C.Structure):
    _fields_ = [("params", C.POINTER(MppiParams)), ("slot", C.c_int32),
                ("x0", _VP), ("ref_xy", _VP), ("n_ref", C.c_int32), ("circ", _VP), ("n_circ", C.c_int32),
                ("centres", _VP), ("u_out", _VP), ("x_out", _VP), ("info", C.POINTER(MppiInfo)),
                ("status", C.c_int32)]


class BatchPlan:
    """One plan of a batch submission: inputs, warm-start slot and output buffers (kept alive)."""

    def __init__(self, params: Dict[str, object], slot: int, x0, ref, circles=None, centres=None):
        self.params = dict(params)
        self.slot = int(slot)
        self.T = int(params["T"])
        self.cparams = make_params(params)
        self.x0 = _f64(x0)
        self.ref = _f64(ref).reshape(-1, 2)
        self.circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        self.centres = None if centres is None else _f64(centres)
        self.u = np.zeros((self.T, 2))
        self.x = np.zeros((self.T + 1, 4))
        self.info = MppiInfo()

    def fill(self, r: MppiRequest):
        r.params = C.pointer(self.cparams)
        r.slot = self.slot
        r.x0, r.ref_xy, r.n_ref = _dp(self.x0), _dp(self.ref), self.ref.shape[0]
        r.circ, r.n_circ = (_dp(self.circ) if self.circ.shape[0] else None), self.circ.shape[0]
        r.centres = _dp(self.centres)
        r.u_out, r.x_out = _dp(self.u), _dp(self.x)
        r.info = C.pointer(self.info)
        r.status = 0


class BatchPlanner:
    """Many independent plans per launch (mppi_batch_*): device warm-start slots, pipelines of
    graph-captured kernel sequences, one persistent rollout kernel across all plans."""

    def __init__(self, max_slots: int, max_batch: int, max_samples: int, max_rollout_steps: int, max_T: int,
                 max_ref: int, max_circ: int, noise_bf16: int = 0, pipelines: int = 2, device: int = 0):
        h = _VP()
        rc = lib().mppi_batch_create(max_slots, max_batch, max_samples, max_rollout_steps, max_T, max_ref, max_circ,
                                     noise_bf16, pipelines, device, C.byref(h))
        self._check(rc, None)
        self._h = h

    def _check(self, rc, h):
        if rc != 0:
            msg = lib().mppi_batch_last_error(h)
            raise MppiError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def requests(plans):
        arr = (MppiRequest * len(plans))()
        for r, p in zip(arr, plans):
            p.fill(r)
        return arr

    def submit(self, reqs) -> int:
        t = C.c_int32()
        self._check(lib().mppi_batch_submit(self._h, C.cast(reqs, _VP), len(reqs), C.byref(t)), self._h)
        return t.value

    def wait(self, ticket: int, check: bool = True) -> int:
        rc = lib().mppi_batch_wait(self._h, ticket)
        if check:
            self._check(rc, self._h)
        return rc

    def plan(self, plans, reqs=None):
        """One iteration of every plan; outputs land in each BatchPlan's u, x, info."""
        reqs = self.requests(plans) if reqs is None else reqs
        self._check(lib().mppi_batch_plan(self._h, C.cast(reqs, _VP), len(reqs)), self._h)
        return reqs

    def get_costs(self, ticket: int, i: int, K: int) -> np.ndarray:
        """Sample costs of plan i of the last submission completed on pipeline `ticket`."""
        S = np.empty(int(K))
        self._check(lib().mppi_batch_get_costs(self._h, int(ticket), int(i), _dp(S), int(K)), self._h)
        return S

    def autotune(self, plans):
        reqs = self.requests(plans)
        g, b = C.c_int32(), C.c_int32()
        self._check(lib().mppi_batch_autotune(self._h, C.cast(reqs, _VP), len(reqs), C.byref(g), C.byref(b)), self._h)
        return g.value, b.value

    def set_launch(self, group: int, block: int):
        """Fix the rollout launch shape (group < 0: lanes split the steps)."""
        self._check(lib().mppi_batch_set_launch(self._h, int(group), int(block)), self._h)

    def set_controls(self, slot: int, U, iter_: int = 0):
        U = _f64(U).reshape(-1, 2)
        self._check(lib().mppi_batch_set_controls(self._h, slot, _dp(U), U.shape[0], int(iter_)), self._h)

    def get_controls(self, slot: int, T: int):
        U = np.empty((T, 2))
        it = C.c_uint64()
        self._check(lib().mppi_batch_get_controls(self._h, slot, _dp(U), T, C.byref(it)), self._h)
        return U, it.value


class MppiServerConfig(C.Structure):
    _fields_ = [("max_sessions", C.c_int32), ("max_batch", C.c_int32), ("max_samples", C.c_int64),
                ("max_rollout_steps", C.c_int64), ("max_T", C.c_int32), ("max_ref", C.c_int32),
                ("max_circ", C.c_int32), ("pipelines", C.c_int32), ("noise_bf16", C.c_int32), ("device", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("max_wait_us", C.c_double), ("watchdog_ms", C.c_double)]


class MppiResult(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("session", C.c_int32), ("status", C.c_int32), ("T", C.c_int32),
                ("latency_us", C.c_double), ("queue_us", C.c_double), ("info", MppiInfo)]


class Server:
    """Continuous-batching planning server (mppi_server_*): enqueue from any thread, poll results."""

    def __init__(self, max_sessions: int, max_batch: int, max_samples: int, max_rollout_steps: int, max_T: int,
                 max_ref: int, max_circ: int, pipelines: int = 3, hbm_budget_bytes: int = 8 << 30,
                 noise_bf16: int = 0, max_wait_us: float = 0.0, device: int = 0, watchdog_ms: float = 0.0):
        self.cfg = MppiServerConfig(max_sessions, max_batch, max_samples, max_rollout_steps, max_T, max_ref,
                                    max_circ, pipelines, noise_bf16, device, hbm_budget_bytes, max_wait_us,
                                    watchdog_ms)
        self.max_T = max_T
        h = _VP()
        self._check(lib().mppi_server_create(C.byref(self.cfg), C.byref(h)), None)
        self._h = h

    def _check(self, rc, h):
        if rc != 0:
            msg = lib().mppi_server_last_error(h)
            raise MppiError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            lib().mppi_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, params: MppiParams, x0, ref, circles, n_plans: int):
        x0, ref = _f64(x0), _f64(ref).reshape(-1, 2)
        circ = _f64(np.zeros((0, 5)) if circles is None else circles).reshape(-1, 5)
        g, b = C.c_int32(), C.c_int32()
        self._check(lib().mppi_server_autotune(self._h, C.byref(params), _dp(x0), _dp(ref), ref.shape[0],
                                               _dp(circ) if circ.shape[0] else None, circ.shape[0], n_plans,
                                               C.byref(g), C.byref(b)), self._h)
        return g.value, b.value

    def enqueue(self, params: MppiParams, session: int, x0, ref, circles=None, centres=None) -> int:
        """params: an MppiParams built once per session (make_params); arrays: float64 C-contiguous."""
        rid = C.c_uint64()
        n_circ = 0 if circles is None else circles.shape[0]
        rc = lib().mppi_server_enqueue(self._h, C.byref(params), session, _dp(x0), _dp(ref), ref.shape[0],
                                       _dp(circles) if n_circ else None, n_circ, _dp(centres), C.byref(rid))
        self._check(rc, self._h)
        return rid.value

    def poll(self, max_results: int = 1024, wait_ms: int = 0, with_outputs: bool = False):
        out = (MppiResult * max_results)()
        n = C.c_int32()
        U = X = None
        if with_outputs:
            U = np.zeros((max_results, self.max_T, 2))
            X = np.zeros((max_results, self.max_T + 1, 4))
        self._check(lib().mppi_server_poll(self._h, C.cast(out, _VP), max_results, _dp(U), _dp(X), self.max_T,
                                           wait_ms, C.byref(n)), self._h)
        res = []
        for i in range(n.value):
            r = out[i]
            d = dict(request_id=r.request_id, session=r.session, status=r.status, T=r.T,
                     latency_us=r.latency_us, queue_us=r.queue_us, info=r.info.as_dict())
            if with_outputs:
                d["u"] = U[i, :r.T].copy()
                d["x"] = X[i, :r.T + 1].copy()
            res.append(d)
        return res

    def pending(self):
        q, f = C.c_int32(), C.c_int32()
        b, p = C.c_uint64(), C.c_uint64()
        self._check(lib().mppi_server_pending(self._h, C.byref(q), C.byref(f), C.byref(b), C.byref(p)), self._h)
        return dict(queued=q.value, in_flight=f.value, batches=b.value, plans=p.value)

    def set_controls(self, session: int, U, iter_: int = 0):
        U = _f64(U).reshape(-1, 2)
        self._check(lib().mppi_server_set_controls(self._h, session, _dp(U), U.shape[0], int(iter_)), self._h)

    def set_watchdog(self, watchdog_ms: float):
        """Abandon micro-batches still running watchdog_ms after submission (0: off)."""
        self._check(lib().mppi_server_set_watchdog(self._h, float(watchdog_ms)), self._h)

    def timeouts(self) -> int:
        n = C.c_uint64()
        self._check(lib().mppi_server_timeouts(self._h, C.byref(n)), self._h)
        return n.value

    def snapshot(self, path: str):
        """Write every session's warm start and iteration counter to a file (idle server)."""
        self._check(lib().mppi_server_snapshot(self._h, os.fsencode(path)), self._h)

    def restore(self, path: str):
        """Read a session table written by snapshot() into this (idle, same-sized) server."""
        self._check(lib().mppi_server_restore(self._h, os.fsencode(path)), self._h)
