"""GB300 RPY matvec (u = D F with the Rotne-Prager-Yamakawa tensor) by an
adaptive plane-wave FMM over the four Laplace potentials of the RPYFMM
decomposition.

This module is a thin ctypes binding of the C ABI in include/rpyfmm.h: every
function has the C name, marshals torch tensors / numpy arrays into pointers
and sizes, and raises RpyError on a non-zero status.  All computation happens
in librpyfmm.so (CUDA, sm_103a); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "RpyError", "RpyStats", "BuildParams", "load", "rpy_tree_build", "rpy_forest_build",
    "rpy_tree_update_positions", "rpy_matvec", "rpy_forest_matvec", "rpy_matvec_parts",
    "rpy_matvec_oneshot", "rpy_matvec_host", "rpy_laplace_far", "rpy_tree_export", "rpy_tree_stats",
    "rpy_tree_sync", "rpy_tree_footprint", "rpy_tree_free", "rpy_strerror", "rpy_last_cuda_error", "rpy_tree_work",
    "rpy_version", "rpy_debug_table", "rpy_tree_set_profiling", "rpy_tree_stage_times", "rpy_launch_count",
    "rpy_alu_peak", "rpy_bounding_cube_noalloc", "rpy_direct_sampled", "rpy_autotune", "rpy_lanczos_sqrt",
    "rpy_bd_step", "rpy_evaluate", "rpy_matvec_batched", "rpy_tree_matvec_host", "rpy_debug_wait_timeout", "STAGES", "FIELDS", "RPY_FP64", "RPY_FP32", "RPY_PART_NEAR", "RPY_PART_FAR",
    "RPY_PART_ALL", "RPY_FLAG_NO_GRAPH", "RPY_FLAG_FRAME_PASSES",
    "RPY_FLAG_EVAL_PER_POTENTIAL", "RPY_FLAG_BOX_ORIGIN", "RPY_FLAG_CUBE_ORIGIN", "RPY_FLAG_CARTESIAN",
    "EXPORTED_SYMBOLS",
]

RPY_FP64, RPY_FP32 = 0, 1
RPY_PART_NEAR, RPY_PART_FAR, RPY_PART_ALL = 1, 2, 3
RPY_FLAG_NO_GRAPH, RPY_FLAG_FRAME_PASSES, RPY_FLAG_EVAL_PER_POTENTIAL = 1, 2, 4
RPY_FLAG_BOX_ORIGIN, RPY_FLAG_CUBE_ORIGIN, RPY_FLAG_CARTESIAN = 8, 16, 32
FIELDS = {
    "perm": (1, np.int32), "keys": (2, np.uint64), "box_level": (3, np.int32), "box_range": (4, np.int32),
    "box_parent": (5, np.int32), "box_center": (6, np.float64), "box_leaf": (7, np.int32),
    "box_sys": (8, np.int32), "box_side": (9, np.float64), "leaves": (10, np.int32), "u_off": (11, np.int32),
    "u_idx": (12, np.int32), "w_off": (13, np.int32), "w_idx": (14, np.int32), "x_off": (15, np.int32),
    "x_idx": (16, np.int32), "v_off": (17, np.int32), "v_idx": (18, np.int32), "cube": (19, np.float64),
    "d_off": (20, np.int32), "d_idx": (21, np.int32),
}
EXPORTED_SYMBOLS = [
    "rpy_tree_build", "rpy_forest_build", "rpy_tree_update_positions", "rpy_matvec", "rpy_forest_matvec",
    "rpy_matvec_parts", "rpy_matvec_oneshot", "rpy_matvec_host", "rpy_laplace_far", "rpy_tree_export",
    "rpy_tree_stats", "rpy_tree_sync", "rpy_tree_footprint", "rpy_tree_free", "rpy_strerror",
    "rpy_last_cuda_error", "rpy_version", "rpy_debug_table", "rpy_tree_set_profiling", "rpy_tree_stage_times",
    "rpy_launch_count", "rpy_alu_peak", "rpy_bounding_cube_noalloc", "rpy_server_create", "rpy_server_add_system",
    "rpy_server_submit", "rpy_server_wait", "rpy_server_cancel", "rpy_server_drain", "rpy_server_stats_get",
    "rpy_server_destroy", "rpy_server_wait_times", "rpy_direct_sampled", "rpy_autotune", "rpy_lanczos_sqrt", "rpy_bd_step", "rpy_evaluate",
    "rpy_matvec_batched", "rpy_tree_work", "rpy_tree_matvec_host", "rpy_debug_wait_timeout",
]
STAGES = ["gather", "p2p", "p2m", "m2m", "m2x", "x2x", "x2l", "p2l", "l2l", "eval", "combine"]


class RpyError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = load()
        msg = lib.rpy_strerror(status).decode()
        cu = lib.rpy_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} (status {status}){' [' + cu + ']' if cu else ''}")
        self.status = status


class BuildParams(ctypes.Structure):
    _fields_ = [("digits", ctypes.c_int), ("precision", ctypes.c_int), ("leaf_cap", ctypes.c_int),
                ("order_p", ctypes.c_int), ("max_level", ctypes.c_int), ("flags", ctypes.c_int),
                ("direct_w", ctypes.c_int), ("direct_x", ctypes.c_int), ("quad", ctypes.c_int)]


class RpyStats(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int64), ("n_systems", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("depth", ctypes.c_int32), ("order_p", ctypes.c_int32),
                ("exp_nodes", ctypes.c_int32), ("exp_terms", ctypes.c_int32), ("leaf_cap", ctypes.c_int32),
                ("digits", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_leaf_count", ctypes.c_int32),
                ("leaves_over_cap", ctypes.c_int32), ("u_pairs", ctypes.c_int64), ("n_ulist", ctypes.c_int64),
                ("n_wlist", ctypes.c_int64), ("n_xlist", ctypes.c_int64), ("n_vpairs", ctypes.c_int64),
                ("n_dlist", ctypes.c_int64), ("d_pairs", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_double), ("quad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AutotuneParams(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("timed_reps", ctypes.c_int), ("margin", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class AutotuneTrial(ctypes.Structure):
    _fields_ = [("leaf_cap", ctypes.c_int), ("order_p", ctypes.c_int), ("direct_w", ctypes.c_int),
                ("direct_x", ctypes.c_int), ("quad", ctypes.c_int), ("status", ctypes.c_int),
                ("est_rel_l2", ctypes.c_double),
                ("matvec_ms", ctypes.c_double)]


class AutotuneResult(ctypes.Structure):
    _fields_ = [("best", BuildParams), ("est_rel_l2", ctypes.c_double), ("matvec_ms", ctypes.c_double),
                ("goal", ctypes.c_double), ("tune_ms", ctypes.c_double), ("n_trials", ctypes.c_int),
                ("trials", AutotuneTrial * 48), ("verify_rel_l2", ctypes.c_double), ("n_verify", ctypes.c_int),
                ("verify_ok", ctypes.c_int)]


class ServerParams(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int), ("device", ctypes.c_int)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("h2d_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("matvec_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("evictions", ctypes.c_int64), ("rebuilds", ctypes.c_int64),
                ("beads_done", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("peak_resident_bytes", ctypes.c_int64), ("resident_systems", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("busy_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load librpyfmm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"librpyfmm.so not found at {path}; run paper_1711_02976_gb300._build.build()")
        lib = ctypes.CDLL(path)
        vp, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "rpy_tree_build": [vp, i64, d, i, i, i, vp, ctypes.POINTER(vp)],
            "rpy_forest_build": [vp, vp, i, vp, ctypes.POINTER(BuildParams), vp, ctypes.POINTER(vp)],
            "rpy_tree_update_positions": [vp, vp, vp],
            "rpy_matvec": [vp, vp, d, vp, vp],
            "rpy_forest_matvec": [vp, vp, vp, vp, vp],
            "rpy_matvec_parts": [vp, vp, d, vp, i, vp],
            "rpy_matvec_oneshot": [vp, i64, d, vp, d, i, vp, vp],
            "rpy_matvec_host": [vp, i64, d, vp, d, i, i, vp, vp],
            "rpy_laplace_far": [vp, vp, vp, vp],
            "rpy_tree_export": [vp, i, vp, i64, ctypes.POINTER(i64)],
            "rpy_tree_stats": [vp, ctypes.POINTER(RpyStats)],
            "rpy_tree_sync": [vp],
            "rpy_tree_footprint": [i64, i, i, i, ctypes.POINTER(i64)],
            "rpy_tree_free": [vp],
            "rpy_strerror": [i],
            "rpy_last_cuda_error": [],
            "rpy_version": [],
            "rpy_debug_table": [i, i, i, vp, i64, ctypes.POINTER(i64)],
            "rpy_tree_set_profiling": [vp, i],
            "rpy_tree_stage_times": [vp, vp, i],
            "rpy_tree_work": [vp, vp, vp, i],
            "rpy_debug_wait_timeout": [d, vp],
            "rpy_tree_matvec_host": [vp, vp, vp, vp, vp, vp],
            "rpy_launch_count": [],
            "rpy_alu_peak": [i, ctypes.POINTER(d), vp],
            "rpy_bounding_cube_noalloc": [vp, i64, vp, vp],
            "rpy_direct_sampled": [vp, vp, i, vp, vp, vp, vp, i64, vp, vp],
            "rpy_autotune": [vp, vp, i, vp, vp, vp, i, i, ctypes.POINTER(AutotuneParams),
                             ctypes.POINTER(AutotuneResult), vp],
            "rpy_lanczos_sqrt": [vp, vp, vp, i, d, vp, ctypes.POINTER(i), ctypes.POINTER(d), vp],
            "rpy_evaluate": [vp, vp, i64, vp, i64, d, d, ctypes.POINTER(BuildParams), vp, vp],
            "rpy_matvec_batched": [vp, i, vp, vp, vp, vp],
            "rpy_bd_step": [vp, vp, vp, vp, vp, vp, d, i, d, vp, ctypes.POINTER(i), vp],
            "rpy_server_create": [ctypes.POINTER(ServerParams), ctypes.POINTER(vp)],
            "rpy_server_add_system": [vp, vp, i64, d, ctypes.POINTER(BuildParams), ctypes.POINTER(i)],
            "rpy_server_submit": [vp, i, vp, vp, d, vp, ctypes.POINTER(i64)],
            "rpy_server_wait": [vp, i64, i, ctypes.POINTER(d)],
            "rpy_server_wait_times": [vp, i64, i, ctypes.POINTER(d), ctypes.POINTER(RequestTimes)],
            "rpy_server_cancel": [vp, i64],
            "rpy_server_drain": [vp],
            "rpy_server_stats_get": [vp, ctypes.POINTER(ServerStats)],
            "rpy_server_destroy": [vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.rpy_tree_free.restype = None
        lib.rpy_server_destroy.restype = None
        lib.rpy_launch_count.restype = ctypes.c_int64
        lib.rpy_strerror.restype = ctypes.c_char_p
        lib.rpy_last_cuda_error.restype = ctypes.c_char_p
        _lib = lib
        return _lib


def _check(status: int, what: str):
    if status != 0:
        raise RpyError(status, what)


def _ptr(x) -> int:
    """Device or host address of a torch tensor / numpy array (must be contiguous float64 etc.)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    return int(x)


def _dev_f64(x, name):
    if hasattr(x, "is_cuda"):
        if not x.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        import torch
        if x.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
    return _ptr(x)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Tree:
    """Owning wrapper of an rpy_tree handle (freed on close / garbage collection)."""

    def __init__(self, handle: int, n: int, nsys: int):
        self.handle = handle
        self.n = n
        self.nsys = nsys

    def close(self):
        if self.handle:
            load().rpy_tree_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _h(tree):
    return ctypes.c_void_p(tree.handle if isinstance(tree, Tree) else tree)


def rpy_tree_build(pos, n, a, digits, leaf_cap=0, precision=RPY_FP64, stream=None) -> Tree:
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.rpy_tree_build(_dev_f64(pos, "pos"), int(n), float(a), int(digits), int(leaf_cap), int(precision),
                              _stream(stream), ctypes.byref(out)), "rpy_tree_build")
    return Tree(out.value, int(n), 1)


def rpy_forest_build(pos, sys_offsets, a, digits, leaf_cap=0, precision=RPY_FP64, order_p=0, max_level=0,
                     direct_w=0, direct_x=0, flags=0, quad=0, stream=None) -> Tree:
    lib = load()
    off = np.ascontiguousarray(sys_offsets, dtype=np.int64)
    av = np.ascontiguousarray(a, dtype=np.float64)
    prm = BuildParams(int(digits), int(precision), int(leaf_cap), int(order_p), int(max_level), int(flags),
                      int(direct_w), int(direct_x), int(quad))
    out = ctypes.c_void_p()
    _check(lib.rpy_forest_build(_dev_f64(pos, "pos"), off.ctypes.data, int(av.size), av.ctypes.data,
                                ctypes.byref(prm), _stream(stream), ctypes.byref(out)), "rpy_forest_build")
    return Tree(out.value, int(off[-1]), int(av.size))


def rpy_direct_sampled(pos, sys_offsets, a, f, kT_over_eta, targets, stream=None) -> np.ndarray:
    """FP64 direct RPY sum at the given targets (caller indices); returns (nt, 3) numpy."""
    off = np.ascontiguousarray(sys_offsets, dtype=np.int64)
    av = np.ascontiguousarray(a, dtype=np.float64)
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(kT_over_eta, dtype=np.float64), av.shape))
    tg = np.ascontiguousarray(targets, dtype=np.int64)
    u = np.zeros((tg.size, 3), dtype=np.float64)
    _check(load().rpy_direct_sampled(_dev_f64(pos, "pos"), off.ctypes.data, int(av.size), av.ctypes.data,
                                     _dev_f64(f, "f"), sv.ctypes.data, tg.ctypes.data, int(tg.size), u.ctypes.data,
                                     _stream(stream)), "rpy_direct_sampled")
    return u


def rpy_autotune(pos, sys_offsets, a, f, kT_over_eta, digits, precision=RPY_FP64, n_samples=0, timed_reps=0,
                 margin=0.0, seed=0, stream=None) -> dict:
    """Search leaf capacity, order and direct-substitution thresholds; returns a dict with the
    chosen build parameters ("best"), the sampled error and time there, and every trial."""
    off = np.ascontiguousarray(sys_offsets, dtype=np.int64)
    av = np.ascontiguousarray(a, dtype=np.float64)
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(kT_over_eta, dtype=np.float64), av.shape))
    prm = AutotuneParams(int(n_samples), int(timed_reps), float(margin), int(seed))
    res = AutotuneResult()
    _check(load().rpy_autotune(_dev_f64(pos, "pos"), off.ctypes.data, int(av.size), av.ctypes.data,
                               _dev_f64(f, "f"), sv.ctypes.data, int(digits), int(precision), ctypes.byref(prm),
                               ctypes.byref(res), _stream(stream)), "rpy_autotune")
    b = res.best
    return {
        "best": {k: getattr(b, k) for k, _ in BuildParams._fields_},
        "est_rel_l2": res.est_rel_l2, "matvec_ms": res.matvec_ms, "goal": res.goal, "tune_ms": res.tune_ms,
        "verify_rel_l2": res.verify_rel_l2, "n_verify": res.n_verify, "verify_ok": bool(res.verify_ok),
        "trials": [{k: getattr(res.trials[i], k) for k, _ in AutotuneTrial._fields_} for i in range(res.n_trials)],
    }


def rpy_evaluate(src_pos, src_f, tgt_pos, a, kT_over_eta, digits, u_tgt, precision=RPY_FP64, leaf_cap=0, order_p=0,
                 quad=0, stream=None):
    """Velocities at target points from source beads (device tensors; u_tgt written)."""
    ns, nt = int(src_pos.shape[0]), int(tgt_pos.shape[0])
    prm = BuildParams(int(digits), int(precision), int(leaf_cap), int(order_p), 0, 0, 0, 0, int(quad))
    _check(load().rpy_evaluate(_dev_f64(src_pos, "src_pos"), _dev_f64(src_f, "src_f"), ns, _dev_f64(tgt_pos, "tgt_pos"),
                               nt, float(a), float(kT_over_eta), ctypes.byref(prm), _dev_f64(u_tgt, "u_tgt"),
                               _stream(stream)), "rpy_evaluate")


def rpy_matvec_batched(trees, fs, kT_over_eta, us, stream=None):
    """Matvecs of several trees on one stream (device tensors f_k, u_k)."""
    k = len(trees)
    th = (ctypes.c_void_p * k)(*[t.handle if isinstance(t, Tree) else t for t in trees])
    fp = (ctypes.c_void_p * k)(*[_dev_f64(f, "f") for f in fs])
    up = (ctypes.c_void_p * k)(*[_dev_f64(u, "u") for u in us])
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(kT_over_eta, dtype=np.float64), (k,)))
    _check(load().rpy_matvec_batched(th, k, fp, sv.ctypes.data, up, _stream(stream)), "rpy_matvec_batched")


def rpy_lanczos_sqrt(tree, z, kT_over_eta, y, m_max=60, tol=1e-8, stream=None):
    """y = D^{1/2} z by Lanczos on the tree's D (device tensors, N x 3); returns (steps, last relative change)."""
    nsys = tree.nsys if isinstance(tree, Tree) else 1
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(kT_over_eta, dtype=np.float64), (nsys,)))
    it, ch = ctypes.c_int(), ctypes.c_double()
    _check(load().rpy_lanczos_sqrt(_h(tree), _dev_f64(z, "z"), sv.ctypes.data, int(m_max), float(tol),
                                   _dev_f64(y, "y"), ctypes.byref(it), ctypes.byref(ch), _stream(stream)),
           "rpy_lanczos_sqrt")
    return it.value, ch.value


def rpy_bd_step(tree, pos, f, xi, kT, eta, dt, m_max=60, tol=1e-8, disp=None, stream=None) -> int:
    """One Ermak-McCammon step on device tensors (pos updated in place, tree rebuilt); returns Lanczos steps."""
    nsys = tree.nsys if isinstance(tree, Tree) else 1
    kt = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64), (nsys,)))
    et = np.ascontiguousarray(np.broadcast_to(np.asarray(eta, dtype=np.float64), (nsys,)))
    it = ctypes.c_int()
    _check(load().rpy_bd_step(_h(tree), _dev_f64(pos, "pos"), _dev_f64(f, "f"), _dev_f64(xi, "xi"), kt.ctypes.data,
                              et.ctypes.data, float(dt), int(m_max), float(tol),
                              _dev_f64(disp, "disp") if disp is not None else None, ctypes.byref(it),
                              _stream(stream)), "rpy_bd_step")
    return it.value


def rpy_tree_update_positions(tree, pos, stream=None):
    _check(load().rpy_tree_update_positions(_h(tree), _dev_f64(pos, "pos"), _stream(stream)),
           "rpy_tree_update_positions")


def rpy_matvec(tree, f, kT_over_eta, u, stream=None):
    _check(load().rpy_matvec(_h(tree), _dev_f64(f, "f"), float(kT_over_eta), _dev_f64(u, "u"), _stream(stream)),
           "rpy_matvec")


def rpy_forest_matvec(tree, f, kT_over_eta, u, stream=None):
    s = np.ascontiguousarray(kT_over_eta, dtype=np.float64)
    _check(load().rpy_forest_matvec(_h(tree), _dev_f64(f, "f"), s.ctypes.data, _dev_f64(u, "u"), _stream(stream)),
           "rpy_forest_matvec")


def rpy_matvec_parts(tree, f, kT_over_eta, u, parts, stream=None):
    _check(load().rpy_matvec_parts(_h(tree), _dev_f64(f, "f"), float(kT_over_eta), _dev_f64(u, "u"), int(parts),
                                   _stream(stream)), "rpy_matvec_parts")


def rpy_matvec_oneshot(pos, n, a, f, kT_over_eta, digits, u, stream=None):
    _check(load().rpy_matvec_oneshot(_dev_f64(pos, "pos"), int(n), float(a), _dev_f64(f, "f"), float(kT_over_eta),
                                     int(digits), _dev_f64(u, "u"), _stream(stream)), "rpy_matvec_oneshot")


def rpy_matvec_host(pos, a, f, kT_over_eta, digits, u, precision=RPY_FP64, stream=None):
    """Host arrays in and out (numpy float64, N x 3, C-contiguous; u is written in place)."""
    for name, arr in (("pos", pos), ("f", f), ("u", u)):
        if not isinstance(arr, np.ndarray) or arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be a C-contiguous float64 numpy array")
    n = pos.shape[0]
    _check(load().rpy_matvec_host(_ptr(pos), int(n), float(a), _ptr(f), float(kT_over_eta), int(digits),
                                  int(precision), _ptr(u), _stream(stream)), "rpy_matvec_host")


def rpy_tree_matvec_host(tree, pos, f, kT_over_eta, u, stream=None):
    """Resident-tree matvec with host numpy arrays (N x 3 float64, C-contiguous; pos may be
    None to keep the positions): rebuild for pos, copy f, u = D f, copy u back (synchronous)."""
    nsys = tree.nsys if isinstance(tree, Tree) else 1
    for name, arr in (("pos", pos), ("f", f), ("u", u)):
        if arr is None and name == "pos":
            continue
        if not isinstance(arr, np.ndarray) or arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be a C-contiguous float64 numpy array")
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(kT_over_eta, dtype=np.float64), (nsys,)))
    _check(load().rpy_tree_matvec_host(_h(tree), _ptr(pos) if pos is not None else None, _ptr(f), sv.ctypes.data,
                                       _ptr(u), _stream(stream)), "rpy_tree_matvec_host")


def rpy_laplace_far(tree, q, out, stream=None):
    _check(load().rpy_laplace_far(_h(tree), _dev_f64(q, "q"), _dev_f64(out, "out"), _stream(stream)),
           "rpy_laplace_far")


def rpy_tree_export(tree, field: str) -> np.ndarray:
    lib = load()
    code, dt = FIELDS[field]
    nbytes = ctypes.c_int64()
    _check(lib.rpy_tree_export(_h(tree), code, None, 0, ctypes.byref(nbytes)), "rpy_tree_export")
    out = np.zeros(nbytes.value // np.dtype(dt).itemsize, dtype=dt)
    _check(lib.rpy_tree_export(_h(tree), code, out.ctypes.data, nbytes.value, ctypes.byref(nbytes)),
           "rpy_tree_export")
    if field in ("box_range",):
        out = out.reshape(-1, 2)
    elif field == "box_center":
        out = out.reshape(-1, 3)
    elif field == "cube":
        out = out.reshape(-1, 4)
    return out


def rpy_tree_stats(tree) -> dict:
    st = RpyStats()
    _check(load().rpy_tree_stats(_h(tree), ctypes.byref(st)), "rpy_tree_stats")
    return st.as_dict()


def rpy_tree_sync(tree):
    _check(load().rpy_tree_sync(_h(tree)), "rpy_tree_sync")


def rpy_tree_footprint(n, digits, precision=RPY_FP64, leaf_cap=0) -> int:
    b = ctypes.c_int64()
    _check(load().rpy_tree_footprint(int(n), int(digits), int(precision), int(leaf_cap), ctypes.byref(b)),
           "rpy_tree_footprint")
    return b.value


def rpy_tree_free(tree):
    if isinstance(tree, Tree):
        tree.close()
    else:
        load().rpy_tree_free(ctypes.c_void_p(tree))


def rpy_strerror(status: int) -> str:
    return load().rpy_strerror(int(status)).decode()


def rpy_last_cuda_error() -> str:
    return load().rpy_last_cuda_error().decode()


def rpy_version() -> int:
    return load().rpy_version()


def rpy_debug_table(p: int, digits: int, which: int) -> np.ndarray:
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.rpy_debug_table(int(p), int(digits), int(which), None, 0, ctypes.byref(cnt)), "rpy_debug_table")
    out = np.zeros(cnt.value)
    _check(lib.rpy_debug_table(int(p), int(digits), int(which), out.ctypes.data, cnt.value, ctypes.byref(cnt)),
           "rpy_debug_table")
    return out


def rpy_tree_set_profiling(tree, enable=True):
    _check(load().rpy_tree_set_profiling(_h(tree), int(bool(enable))), "rpy_tree_set_profiling")


def rpy_tree_stage_times(tree) -> dict:
    ms = np.zeros(len(STAGES))
    _check(load().rpy_tree_stage_times(_h(tree), ms.ctypes.data, len(STAGES)), "rpy_tree_stage_times")
    return dict(zip(STAGES, ms.tolist()))


def rpy_tree_work(tree) -> dict:
    """Algorithmic FLOPs and DRAM bytes of one matvec per stage: {stage: (flops, bytes)}."""
    fl = np.zeros(len(STAGES))
    by = np.zeros(len(STAGES))
    _check(load().rpy_tree_work(_h(tree), fl.ctypes.data, by.ctypes.data, len(STAGES)), "rpy_tree_work")
    return {k: (float(a), float(b)) for k, a, b in zip(STAGES, fl, by)}


def rpy_debug_wait_timeout(limit_ms, stream=None) -> int:
    """Bounded-wait self-test: returns the status (RPY_ERR_TIMEOUT, -5, is the expected one)."""
    return load().rpy_debug_wait_timeout(float(limit_ms), _stream(stream))


def rpy_launch_count() -> int:
    return int(load().rpy_launch_count())


def rpy_alu_peak(precision=RPY_FP64, stream=None) -> float:
    v = ctypes.c_double()
    _check(load().rpy_alu_peak(int(precision), ctypes.byref(v), _stream(stream)), "rpy_alu_peak")
    return v.value


def rpy_bounding_cube_noalloc(pos, n, cube, stream=None):
    """Bounding cube (centre x, y, z, side) of n device positions into the
    device array cube (4 doubles), with no device allocation in the library."""
    _check(load().rpy_bounding_cube_noalloc(_dev_f64(pos, "pos"), int(n), _dev_f64(cube, "cube"), _stream(stream)),
           "rpy_bounding_cube_noalloc")


# ---------------------------------------------------------------- serving

def rpy_server_create(device_budget_bytes=0, slots=0, device=-1) -> int:
    h = ctypes.c_void_p()
    prm = ServerParams(int(device_budget_bytes), int(slots), int(device))
    _check(load().rpy_server_create(ctypes.byref(prm), ctypes.byref(h)), "rpy_server_create")
    return h.value


def rpy_server_add_system(server, pos, a, digits, precision=RPY_FP64, leaf_cap=0, order_p=0) -> int:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    prm = BuildParams(int(digits), int(precision), int(leaf_cap), int(order_p), 0, 0, 0, 0)
    sid = ctypes.c_int()
    _check(load().rpy_server_add_system(ctypes.c_void_p(server), pos.ctypes.data, pos.shape[0], float(a),
                                        ctypes.byref(prm), ctypes.byref(sid)), "rpy_server_add_system")
    return sid.value


def rpy_server_submit(server, system_id, pos, f, kT_over_eta, u) -> int:
    """pos: host (N, 3) float64 or None; f: host (N, 3); u: host (N, 3) written on completion
    (the caller keeps u alive until rpy_server_wait returns)."""
    if pos is not None:
        pos = np.ascontiguousarray(pos, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    if not (isinstance(u, np.ndarray) and u.dtype == np.float64 and u.flags["C_CONTIGUOUS"]):
        raise ValueError("u must be a C-contiguous float64 numpy array")
    rid = ctypes.c_int64()
    _check(load().rpy_server_submit(ctypes.c_void_p(server), int(system_id), pos.ctypes.data if pos is not None else None,
                                    f.ctypes.data, float(kT_over_eta), u.ctypes.data, ctypes.byref(rid)),
           "rpy_server_submit")
    return rid.value


def rpy_server_wait(server, request_id, timeout_ms=-1):
    """Returns (status, latency_ms); status 0 on success (errors are returned, not raised)."""
    lat = ctypes.c_double()
    st = load().rpy_server_wait(ctypes.c_void_p(server), int(request_id), int(timeout_ms), ctypes.byref(lat))
    return st, lat.value


def rpy_server_wait_times(server, request_id, timeout_ms=-1):
    """Returns (status, latency_ms, {queue_ms, run_ms, h2d_ms, build_ms, matvec_ms, d2h_ms})."""
    lat = ctypes.c_double()
    tm = RequestTimes()
    st = load().rpy_server_wait_times(ctypes.c_void_p(server), int(request_id), int(timeout_ms), ctypes.byref(lat),
                                      ctypes.byref(tm))
    return st, lat.value, {k: getattr(tm, k) for k, _ in RequestTimes._fields_}


def rpy_server_cancel(server, request_id) -> int:
    return load().rpy_server_cancel(ctypes.c_void_p(server), int(request_id))


def rpy_server_drain(server):
    _check(load().rpy_server_drain(ctypes.c_void_p(server)), "rpy_server_drain")


def rpy_server_stats_get(server) -> dict:
    st = ServerStats()
    _check(load().rpy_server_stats_get(ctypes.c_void_p(server), ctypes.byref(st)), "rpy_server_stats_get")
    return st.as_dict()


def rpy_server_destroy(server):
    load().rpy_server_destroy(ctypes.c_void_p(server))
