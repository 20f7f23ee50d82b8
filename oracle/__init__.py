"""CPU FP64 oracle for the RPY matvec (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1711_02976_gb300/`` never imports it, and it imports nothing from
there: the two share no code.

Functions (each follows the passage named in ``rpy_oracle.c``):
    rpy_direct(pos, f, a, s, targets=None, threads=None)   Sec. 1, the RPY tensor
    laplace_direct(src, q, tgt)                            Sec. 2, L_k with grad, Hessian
    rpy_far_split(pos_src, f, pos_tgt, a, s, origin, dipole_sign=-1)   Eq. (2.8)
    morton_keys(pos) -> (keys, cube)                       tree key (Sec. 4.2 refinement)
    stable_sort(keys) -> perm
    rel_l2(u, uref)                                        error measure
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpy_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librpy_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d = ctypes.c_double
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_rpy_direct.argtypes = [p, p, i64, d, d, p, i64, p, ctypes.c_int]
            lib.oracle_laplace_direct.argtypes = [p, p, i64, ctypes.c_int, p, i64, p, ctypes.c_int]
            lib.oracle_rpy_far_split.argtypes = [p, p, i64, p, i64, d, d, p, d, p, ctypes.c_int]
            lib.oracle_morton_keys.argtypes = [p, i64, p, p]
            lib.oracle_stable_sort.argtypes = [p, i64, p]
            for fn in (lib.oracle_rpy_direct, lib.oracle_laplace_direct, lib.oracle_rpy_far_split,
                       lib.oracle_morton_keys, lib.oracle_stable_sort):
                fn.restype = None
            _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


def _c(x, dtype=np.float64):
    return np.ascontiguousarray(x, dtype=dtype)


def _ptr(x):
    return x.ctypes.data_as(ctypes.c_void_p)


def rpy_direct(pos, f, a, s, targets=None, threads=None):
    """u_i = sum_j D_ij F_j for i in targets (all beads if None); returns (nt, 3)."""
    lib = _load()
    pos = _c(pos).reshape(-1, 3)
    f = _c(f).reshape(-1, 3)
    n = pos.shape[0]
    if targets is None:
        nt = n
        tp = None
    else:
        targets = _c(targets, np.int64).ravel()
        nt = targets.shape[0]
        tp = _ptr(targets)
    u = np.zeros((nt, 3))
    lib.oracle_rpy_direct(_ptr(pos), _ptr(f), n, float(a), float(s), tp, nt, _ptr(u),
                          int(threads or default_threads()))
    return u


def laplace_direct(src, q, tgt, threads=None):
    """Potential, gradient and Hessian of sum_j q_j/|x - y_j| at each target.

    q: (ns,) or (ns, nq).  Returns (phi (nt,nq), grad (nt,nq,3), hess (nt,nq,3,3))."""
    lib = _load()
    src = _c(src).reshape(-1, 3)
    q = _c(q)
    if q.ndim == 1:
        q = q[:, None]
    q = _c(q)
    nq = q.shape[1]
    tgt = _c(tgt).reshape(-1, 3)
    nt = tgt.shape[0]
    out = np.zeros((nt, nq, 13))
    lib.oracle_laplace_direct(_ptr(src), _ptr(q), src.shape[0], nq, _ptr(tgt), nt, _ptr(out),
                              int(threads or default_threads()))
    return out[..., 0], out[..., 1:4], out[..., 4:13].reshape(nt, nq, 3, 3)


def rpy_far_split(pos_src, f, pos_tgt, a, s, origin=(0.0, 0.0, 0.0), dipole_sign=-1.0, threads=None):
    """Far-field velocity from the four Laplace potentials, Eq. (2.8)."""
    lib = _load()
    ps = _c(pos_src).reshape(-1, 3)
    f = _c(f).reshape(-1, 3)
    pt = _c(pos_tgt).reshape(-1, 3)
    org = _c(origin).ravel()
    u = np.zeros((pt.shape[0], 3))
    lib.oracle_rpy_far_split(_ptr(ps), _ptr(f), ps.shape[0], _ptr(pt), pt.shape[0], float(a), float(s),
                             _ptr(org), float(dipole_sign), _ptr(u), int(threads or default_threads()))
    return u


def morton_keys(pos):
    """63-bit Morton keys and the bounding cube (centre x, y, z, side)."""
    lib = _load()
    pos = _c(pos).reshape(-1, 3)
    keys = np.zeros(pos.shape[0], dtype=np.uint64)
    cube = np.zeros(4)
    lib.oracle_morton_keys(_ptr(pos), pos.shape[0], _ptr(keys), _ptr(cube))
    return keys, cube


def stable_sort(keys):
    """Permutation that sorts keys stably (ties keep index order)."""
    lib = _load()
    keys = _c(keys, np.uint64).ravel()
    perm = np.zeros(keys.shape[0], dtype=np.int64)
    lib.oracle_stable_sort(_ptr(keys), keys.shape[0], _ptr(perm))
    return perm


def rel_l2(u, uref):
    """sqrt(sum |u - uref|^2 / sum |uref|^2) over all components."""
    u = np.asarray(u, dtype=np.float64)
    uref = np.asarray(uref, dtype=np.float64)
    den = float(np.sum(uref * uref))
    if den == 0.0:
        return float(np.sqrt(np.sum((u - uref) ** 2)))
    return float(np.sqrt(np.sum((u - uref) ** 2) / den))
