"""Independent checks used to pin the oracle and to judge GPU results.

Nothing here calls the oracle or the CUDA library: brute-force path
enumeration, path validity, and the golden-file reader are written from the
definition of DTW with steps (1,1), (1,2), (2,1) and weights 2, 3, 3 (Sec. V).
"""
from __future__ import annotations

import os
from fractions import Fraction
from typing import Iterator, List, Sequence, Tuple

import numpy as np

STEPS = ((1, 1), (1, 2), (2, 1))  # code 0, 1, 2
WEIGHTS = (2, 3, 3)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def all_paths(La: int, Lb: int) -> Iterator[Tuple[int, ...]]:
    """Every step-code sequence leading from (0,0) to (La-1, Lb-1)."""
    ti, tj = La - 1, Lb - 1

    def rec(i, j, acc):
        if i == ti and j == tj:
            yield tuple(acc)
            return
        for code, (di, dj) in enumerate(STEPS):
            ni, nj = i + di, j + dj
            if ni <= ti and nj <= tj:
                acc.append(code)
                yield from rec(ni, nj, acc)
                acc.pop()

    yield from rec(0, 0, [])


def codes_to_path(codes: Sequence[int]) -> np.ndarray:
    p = [(0, 0)]
    for c in codes:
        di, dj = STEPS[c]
        p.append((p[-1][0] + di, p[-1][1] + dj))
    return np.array(p, dtype=np.int64)


def path_weighted_cost(C, codes: Sequence[int], exact: bool = False):
    """C[0,0] + sum of w_step * C[destination].  ``exact`` uses Fractions."""
    conv = Fraction if exact else float
    i = j = 0
    t = conv(C[0][0]) if not exact else Fraction(C[0][0])
    for c in codes:
        di, dj = STEPS[c]
        i, j = i + di, j + dj
        t += WEIGHTS[c] * (Fraction(C[i][j]) if exact else float(C[i][j]))
    return t


def brute_force(C, exact: bool = False):
    """Minimum over all monotone paths and the list of minimising code sequences."""
    La, Lb = len(C), len(C[0])
    best = None
    arg: List[Tuple[int, ...]] = []
    for codes in all_paths(La, Lb):
        t = path_weighted_cost(C, codes, exact)
        if best is None or t < best:
            best, arg = t, [codes]
        elif t == best:
            arg.append(codes)
    return best, arg


def tie_order_path(argmins: List[Tuple[int, ...]]) -> Tuple[int, ...]:
    """Among optimal paths, the one a backtrace with tie order (1,1)<(1,2)<(2,1) returns.

    Walking back from the end, each cell takes the first code (in that order)
    whose predecessor lies on an optimal path; that is the optimal path whose
    code sequence, read from the end, is lexicographically smallest.
    """
    return min(argmins, key=lambda c: tuple(reversed(c)))


def path_codes(path: np.ndarray) -> List[int]:
    """Step codes of a path given as (i, j) rows; raises on an invalid step."""
    out = []
    for k in range(1, len(path)):
        d = (int(path[k][0] - path[k - 1][0]), int(path[k][1] - path[k - 1][1]))
        out.append(STEPS.index(d))
    return out


def check_path_valid(path: np.ndarray, La: int, Lb: int) -> None:
    """Endpoints, step set, monotonicity and length bounds of a DTW path."""
    path = np.asarray(path)
    assert path.ndim == 2 and path.shape[1] == 2
    assert tuple(path[0]) == (0, 0), f"path starts at {tuple(path[0])}"
    assert tuple(path[-1]) == (La - 1, Lb - 1), f"path ends at {tuple(path[-1])}"
    path_codes(path)  # every step in the set
    n = len(path)
    lo = -(-max(La - 1, Lb - 1) // 2) + 1
    assert lo <= n <= min(La, Lb), (n, lo, min(La, Lb))


def constant_cost_path(La: int, Lb: int) -> np.ndarray:
    """Closed form of the tie-order path when every path ties (constant cost).

    With i = La-1 <= j = Lb-1: (j-i) steps (1,2) from the start, then (2i-j)
    steps (1,1); symmetric with (2,1) when i > j.
    """
    i, j = La - 1, Lb - 1
    if i <= j:
        codes = [1] * (j - i) + [0] * (2 * i - j)
    else:
        codes = [2] * (i - j) + [0] * (2 * j - i)
    return codes_to_path(codes)


def load_golden(name: str):
    """Read a hand-derived fixture (format in tests/golden/README.txt)."""
    toks = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                toks.append(line.split())
    d = {}
    k = 0
    while k < len(toks):
        t = toks[k]
        key = t[0]
        if key == "kind":
            d["kind"] = t[1]
        elif key == "shape":
            d["shape"] = tuple(int(x) for x in t[1:])
        elif key == "rows":
            La = d["shape"][0]
            d["C"] = np.array([[float(x) for x in toks[k + 1 + r]] for r in range(La)])
            k += La
        elif key in ("A", "B"):
            n = d["shape"][0] if key == "A" else d["shape"][1]
            d[key] = np.array([[float(x) for x in toks[k + 1 + r]] for r in range(n)],
                              dtype=np.float32)
            k += n
        elif key == "total":
            d["total"] = float(t[1])
        elif key == "path":
            v = [int(x) for x in t[1:]]
            d["path"] = np.array(v, dtype=np.int64).reshape(-1, 2)
        k += 1
    return d
