"""ctypes wrapper around the FP64 CPU oracle (``stokes_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it; the product path never does.  It imports
nothing from the CUDA package.

Every function takes plain NumPy arrays in the layout of the C file: nodes and
normals (N, 2), weights and curvature (N,), densities (rows of each kind in
node order).  See ``stokes_oracle.c`` for what is summed (Eq. (S), Eq. (D),
Eq. (Dnr), Eq. (utotrep), the Nystrom diagonal of Sec. 2.3 and the Kress self
rule of Sec. 3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "stokes_oracle.c")
LIB = os.path.join(HERE, "libstokes_oracle.so")

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction, OpenMP over targets)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.ora_sum.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp, dp,
                                    ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double,
                                    ctypes.c_int, ip, dp, ctypes.c_int]
            lib.ora_sum_free.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp,
                                         ctypes.c_double, ctypes.c_double, dp, dp,
                                         ctypes.c_int, dp, dp, ctypes.c_int]
            lib.ora_kress_weights.argtypes = [ctypes.c_int, dp]
            lib.ora_stokeslet_tensor.argtypes = [ctypes.c_double] * 5 + [dp]
            lib.ora_stresslet_tensor.argtypes = [ctypes.c_double] * 6 + [dp]
            lib.ora_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleError(RuntimeError):
    pass


def _geom_args(geom):
    off, p_off = _i(geom.curve_offset)
    kind, p_kind = _i(geom.curve_kind)
    x, p_x = _d(geom.nodes.reshape(-1, 2) if geom.n_nodes else np.zeros((1, 2)))
    w, p_w = _d(geom.weights if geom.n_nodes else np.zeros(1))
    n, p_n = _d(geom.normals if geom.n_nodes else np.zeros((1, 2)))
    keep = (off, kind, x, w, n)
    return keep, (p_off, p_kind, p_x, p_w, p_n)


def sum_nodes(geom, slp_density, dlp_density, jump: float = 0.0, select=None, threads: int = 0,
              period=None, mu=None):
    """Velocity at the geometry's nodes (or at node indices ``select``), shape (T, 2)."""
    lib = _load()
    keep, (p_off, p_kind, p_x, p_w, p_n) = _geom_args(geom)
    kap, p_k = _d(geom.curvature if geom.n_nodes else np.zeros(1))
    s, p_s = _d(np.asarray(slp_density).reshape(-1, 2) if np.size(slp_density) else np.zeros((1, 2)))
    t, p_t = _d(np.asarray(dlp_density).reshape(-1, 2) if np.size(dlp_density) else np.zeros((1, 2)))
    if select is None:
        nsel, p_sel, sel = 0, None, None
        nt = geom.n_nodes
    else:
        sel, p_sel = _i(select)
        nsel = nt = int(sel.shape[0])
    out = np.zeros((max(nt, 1), 2))
    _, p_out = _d(out)
    p_out = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.ora_sum(geom.n_nodes, len(geom.curves), p_off, p_kind, p_x, p_w, p_n, p_k,
                     geom.period if period is None else period, geom.mu if mu is None else mu,
                     p_s, p_t, jump, nsel, p_sel, p_out, threads)
    if st:
        raise OracleError("ora_sum status %d" % st)
    return out[:nt]


def sum_free(geom, slp_density, dlp_density, targets, threads: int = 0, period=None, mu=None):
    """Velocity at free points ``targets`` (T, 2): plain trapezoid rule, no self terms."""
    lib = _load()
    keep, (p_off, p_kind, p_x, p_w, p_n) = _geom_args(geom)
    s, p_s = _d(np.asarray(slp_density).reshape(-1, 2) if np.size(slp_density) else np.zeros((1, 2)))
    t, p_t = _d(np.asarray(dlp_density).reshape(-1, 2) if np.size(dlp_density) else np.zeros((1, 2)))
    tg, p_tg = _d(np.asarray(targets).reshape(-1, 2))
    nt = tg.shape[0]
    out = np.zeros((max(nt, 1), 2))
    p_out = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.ora_sum_free(geom.n_nodes, len(geom.curves), p_off, p_kind, p_x, p_w, p_n,
                          geom.period if period is None else period, geom.mu if mu is None else mu,
                          p_s, p_t, nt, p_tg, p_out, threads)
    if st:
        raise OracleError("ora_sum_free status %d" % st)
    return out[:nt]


def kress_weights(n: int) -> np.ndarray:
    lib = _load()
    R = np.zeros(n)
    st = lib.ora_kress_weights(n, R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st:
        raise OracleError("ora_kress_weights status %d" % st)
    return R


def stokeslet(x, y, mu=1.0) -> np.ndarray:
    lib = _load()
    S = np.zeros(4)
    lib.ora_stokeslet_tensor(x[0], x[1], y[0], y[1], mu, S.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return S.reshape(2, 2)


def stresslet(x, y, n) -> np.ndarray:
    lib = _load()
    D = np.zeros(4)
    lib.ora_stresslet_tensor(x[0], x[1], y[0], y[1], n[0], n[1],
                             D.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return D.reshape(2, 2)


def max_threads() -> int:
    return int(_load().ora_max_threads())
