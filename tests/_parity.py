"""The acceptance rule for a GPU alignment against the FP64 oracle.

The exact method returns DTW's optimal path (Sec. II-D, Sec. V).  The GPU
computes in FP32 and the oracle in FP64, so:

  * the GPU's FP32 total must lie within 1e-5 relative of the oracle's FP64
    total;
  * the GPU path must equal the oracle's index for index, or -- where FP32
    rounding resolves a near-tie the other way -- its cost recomputed in FP64
    must lie within 1e-6 relative of the oracle's optimum.

Absolute floors apply only to totals near zero, |t_oracle| < NEAR_ZERO = 1
(identical or constant-cost sequences, where every cell cost is rounding noise
around 0 and a relative bound means nothing).  There the FP32 cell cost
1 - sum_d a_d b_d carries an absolute error of order D * 2^-24 <= 1e-6 for
unit frames, and a path weighs (La-1)+(Lb-1) cell costs, so the total may be
off by up to 2e-6 * (La + Lb) and a near-tie path's FP64 cost by up to
1e-7 * (La + Lb) (one rounding per weighted term, 2^-24 * 3 per cell, summed
over the path).

Every comparison is recorded (relative errors of the total and of the path
cost); when PARDTW_PARITY_LOG names a file, the session writes the largest
ones there (tests/conftest.py).
"""
from __future__ import annotations

import numpy as np

import oracle
from tests._pins import check_path_valid

NEAR_ZERO = 1.0
TOTAL_REL = 1e-5
PATH_REL = 1e-6

# name -> dict of the worst errors seen under that name
RECORD: dict = {}


def total_tol(to: float, La: int, Lb: int) -> float:
    if abs(to) >= NEAR_ZERO:
        return TOTAL_REL * abs(to)
    return max(TOTAL_REL * abs(to), 2e-6 * (La + Lb))


def path_tol(to: float, La: int, Lb: int) -> float:
    if abs(to) >= NEAR_ZERO:
        return PATH_REL * abs(to)
    return PATH_REL * abs(to) + 1e-7 * (La + Lb)


def record(name: str, La: int, Lb: int, total: float, to: float, tg: float | None,
           identical: bool) -> None:
    rel_t = abs(total - to) / abs(to) if to != 0 else abs(total - to)
    rel_p = 0.0 if tg is None else (abs(tg - to) / abs(to) if to != 0 else abs(tg - to))
    r = RECORD.setdefault(name, {"cases": 0, "max_total_rel": 0.0, "max_path_rel": 0.0,
                                 "paths_identical": 0, "largest": None,
                                 "near_zero_cases": 0, "max_total_abs_near_zero": 0.0})
    r["cases"] += 1
    r["paths_identical"] += int(identical)
    if abs(to) < NEAR_ZERO:
        # judged by the absolute floor: relative errors mean nothing here
        r["near_zero_cases"] += 1
        r["max_total_abs_near_zero"] = max(r["max_total_abs_near_zero"], abs(total - to))
    else:
        r["max_total_rel"] = max(r["max_total_rel"], rel_t)
    r["max_path_rel"] = max(r["max_path_rel"], rel_p)
    if r["largest"] is None or La * Lb > r["largest"][0] * r["largest"][1]:
        r["largest"] = (La, Lb, float(to), rel_t, rel_p)


def check_against(name: str, La: int, Lb: int, p: np.ndarray, total: float, po: np.ndarray,
                  to: float, path_cost) -> None:
    """The rule above, given the oracle's result (po, to) and a function that
    costs a path in FP64 (used only when the paths differ)."""
    check_path_valid(p, La, Lb)
    assert abs(total - to) <= total_tol(to, La, Lb), (name, total, to)
    identical = p.shape == po.shape and np.array_equal(p, po)
    tg = None
    if not identical:
        tg = float(path_cost(p))
        assert abs(tg - to) <= path_tol(to, La, Lb), (name, tg, to)
    record(name, La, Lb, total, to, tg, identical)


def as_numpy_path(path) -> np.ndarray:
    return path.cpu().numpy() if hasattr(path, "cpu") else np.asarray(path)


def assert_parity(A, B, path, total, name: str = "exact", ref=None):
    """GPU (path, total) for features A, B against oracle.dtw(A, B).  ``ref``
    may pass a precomputed oracle result (po, to)."""
    La, Lb = A.shape[0], B.shape[0]
    p = as_numpy_path(path)
    po, to = oracle.dtw(A, B) if ref is None else ref
    check_against(name, La, Lb, p, float(total), po, to,
                  lambda q: oracle.path_cost(A, B, q))
    return po, to

