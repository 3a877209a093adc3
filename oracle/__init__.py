"""FP64 CPU oracle for exact DTW (the alignment ParDTW computes, Sec. II-D / Sec. V).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``.  The product path never
imports it.  It shares no code with the CUDA library; the C source is
``dtw_oracle.c`` next to this file and is compiled with gcc (``build()``).

Every function here documents the passage it follows; see ``dtw_oracle.c``
for the recurrence, the step set {(1,1),(1,2),(2,1)} with weights {2,3,3}
(Sec. V) and the readings of points the paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_INVALID, ERR_UNREACHABLE, ERR_NOMEM, ERR_CAPACITY = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``dtw_oracle.c`` into ``liboracle.so`` with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint8)
        ci = ctypes.c_int
        lib.oracle_reachable.argtypes = [ci, ci]
        lib.oracle_inv_norms.argtypes = [fp, ci, ci, dp]
        lib.oracle_cost_matrix.argtypes = [fp, ci, fp, ci, ci, dp]
        lib.oracle_dtw_matrix.argtypes = [dp, ci, ci, dp, up, ip, ci, ctypes.POINTER(ci), dp]
        lib.oracle_dtw.argtypes = [fp, ci, fp, ci, ci, ip, ci, ctypes.POINTER(ci), dp]
        lib.oracle_dtw_unit.argtypes = [fp, ci, fp, ci, ci, ip, ci, ctypes.POINTER(ci), dp]
        lib.oracle_path_cost.argtypes = [fp, ci, fp, ci, ci, ip, ci, dp]
        _lib = lib
    return _lib


def _f32(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("features must be L x D")
    return X


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _check(rc: int, what: str):
    if rc == ERR_UNREACHABLE:
        raise OracleError(f"{what}: end cell unreachable with steps (1,1),(1,2),(2,1)")
    if rc != OK:
        raise OracleError(f"{what}: error {rc}")


def reachable(La: int, Lb: int) -> bool:
    """(La-1, Lb-1) reachable from (0, 0) with steps (1,1), (1,2), (2,1)."""
    return bool(_load().oracle_reachable(int(La), int(Lb)))


def inv_norms(X) -> np.ndarray:
    """1/||x|| per frame in FP64; 0 for a zero frame (cosine cost, Sec. IV)."""
    X = _f32(X)
    r = np.empty(X.shape[0], dtype=np.float64)
    _check(_load().oracle_inv_norms(_ptr(X, ctypes.c_float), X.shape[0], X.shape[1],
                                    _ptr(r, ctypes.c_double)), "inv_norms")
    return r


def cost_matrix(A, B) -> np.ndarray:
    """C[i, j] = 1 - (a_i . b_j) r_a[i] r_b[j] in FP64 (cosine distance, Sec. IV)."""
    A, B = _f32(A), _f32(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("feature dimensions differ")
    C = np.empty((A.shape[0], B.shape[0]), dtype=np.float64)
    _check(_load().oracle_cost_matrix(_ptr(A, ctypes.c_float), A.shape[0],
                                      _ptr(B, ctypes.c_float), B.shape[0], A.shape[1],
                                      _ptr(C, ctypes.c_double)), "cost_matrix")
    return C


def dtw_matrix(C, *, full: bool = False):
    """Exact DTW over a given cost matrix (Sec. V steps and weights).

    Returns ``(path, total)``; with ``full=True`` returns
    ``(path, total, Dcum, codes)`` where ``Dcum`` is the La x Lb cumulative
    cost and ``codes`` the step codes (0 (1,1), 1 (1,2), 2 (2,1), 3 none).
    ``path`` is an (n, 2) int32 array of (i, j), ascending from (0, 0).
    """
    C = np.ascontiguousarray(C, dtype=np.float64)
    La, Lb = C.shape
    cap = min(La, Lb)
    path = np.empty((cap, 2), dtype=np.int32)
    n = ctypes.c_int(0)
    tot = ctypes.c_double(0.0)
    Dcum = np.empty((La, Lb), dtype=np.float64) if full else None
    codes = np.empty((La, Lb), dtype=np.uint8) if full else None
    rc = _load().oracle_dtw_matrix(
        _ptr(C, ctypes.c_double), La, Lb,
        _ptr(Dcum, ctypes.c_double) if full else None,
        _ptr(codes, ctypes.c_uint8) if full else None,
        _ptr(path, ctypes.c_int32), cap, ctypes.byref(n), ctypes.byref(tot))
    _check(rc, "dtw_matrix")
    path = path[: n.value].copy()
    if full:
        return path, tot.value, Dcum, codes
    return path, tot.value


def dtw(A, B) -> Tuple[np.ndarray, float]:
    """Exact DTW of feature sequences A (La x D) and B (Lb x D) under the cosine cost.

    The cost is formed on the fly row by row; memory is three rows of D plus
    2 bits per cell of step codes (Sec. II-D, Sec. VI-D).
    """
    A, B = _f32(A), _f32(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("feature dimensions differ")
    La, Lb = A.shape[0], B.shape[0]
    cap = min(La, Lb)
    path = np.empty((cap, 2), dtype=np.int32)
    n = ctypes.c_int(0)
    tot = ctypes.c_double(0.0)
    rc = _load().oracle_dtw(_ptr(A, ctypes.c_float), La, _ptr(B, ctypes.c_float), Lb,
                            A.shape[1], _ptr(path, ctypes.c_int32), cap, ctypes.byref(n),
                            ctypes.byref(tot))
    _check(rc, "dtw")
    return path[: n.value].copy(), tot.value


def path_cost(A, B, path) -> float:
    """FP64 cost of a given path: C[0,0] + sum of w_step * C[destination] (Sec. V weights)."""
    A, B = _f32(A), _f32(B)
    path = np.ascontiguousarray(path, dtype=np.int32)
    tot = ctypes.c_double(0.0)
    rc = _load().oracle_path_cost(_ptr(A, ctypes.c_float), A.shape[0], _ptr(B, ctypes.c_float),
                                  B.shape[0], A.shape[1], _ptr(path, ctypes.c_int32),
                                  path.shape[0], ctypes.byref(tot))
    _check(rc, "path_cost")
    return tot.value


def path_cost_matrix(C, path) -> float:
    """FP64 cost of a given path over a given cost matrix: C[0,0] plus, per
    step, its weight (2 for (1,1), 3 for (1,2) and (2,1), Sec. V) times the
    cost of the step's destination cell.  Raises on a step outside the set."""
    C = np.asarray(C, dtype=np.float64)
    p = np.asarray(path, dtype=np.int64)
    return path_cost_matrix_values(C[p[:, 0], p[:, 1]], p)


def dtw_unit(A, B) -> Tuple[np.ndarray, float]:
    """Exact DTW with C[i, j] = 1 - a_i . b_j for frames taken as they are
    (the cosine cost of Sec. IV when the frames are unit vectors; nothing is
    renormalised).  For features normalised and then rounded to a narrower
    type, whose norms are no longer exactly 1.  Cost on the fly, as ``dtw``."""
    A, B = _f32(A), _f32(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("feature dimensions differ")
    La, Lb = A.shape[0], B.shape[0]
    cap = min(La, Lb)
    path = np.empty((cap, 2), dtype=np.int32)
    n = ctypes.c_int(0)
    tot = ctypes.c_double(0.0)
    rc = _load().oracle_dtw_unit(_ptr(A, ctypes.c_float), La, _ptr(B, ctypes.c_float), Lb,
                                 A.shape[1], _ptr(path, ctypes.c_int32), cap, ctypes.byref(n),
                                 ctypes.byref(tot))
    _check(rc, "dtw_unit")
    return path[: n.value].copy(), tot.value


def path_cost_unit(A, B, path) -> float:
    """FP64 cost of a given path under C[i, j] = 1 - a_i . b_j (frames taken
    as they are, as ``dtw_unit``), with the Sec. V weights."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    p = np.asarray(path, dtype=np.int64)
    c = 1.0 - np.einsum("kd,kd->k", A[p[:, 0]], B[p[:, 1]])
    return path_cost_matrix_values(c, p)


def path_cost_matrix_values(c, p) -> float:
    """C[0,0] + sum of w_step * C[destination] given the path's cell costs
    ``c`` (one per path cell) and the path ``p``."""
    d = np.diff(p, axis=0)
    w = np.full(d.shape[0], np.nan)
    w[(d[:, 0] == 1) & (d[:, 1] == 1)] = 2.0
    w[((d[:, 0] == 1) & (d[:, 1] == 2)) | ((d[:, 0] == 2) & (d[:, 1] == 1))] = 3.0
    if np.isnan(w).any():
        raise OracleError("path cost: step outside {(1,1),(1,2),(2,1)}")
    return float(c[0] + np.sum(w * c[1:]))
