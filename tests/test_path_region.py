"""The region of cells a DTW path can visit (CPU).

The parallel backtrace maps only row i's columns lo(i) .. hi(i): with the
steps (1,1), (1,2), (2,1) of Sec. V (slopes 1/2 to 2) these are the cells
reachable from (0, 0) that can still reach (La-1, Lb-1).  Here the bounds
are checked against brute-force reachability on every shape up to 24 x 24:
no cell of any path lies outside them, and lo, hi never decrease with i (a
band's cells then lie between lo(first row) and hi(last row))."""
import numpy as np
import pytest

STEPS = ((1, 1), (1, 2), (2, 1))


def lo(i, La, Lb):
    return max((i + 1) // 2, Lb - 1 - 2 * (La - 1 - i))


def hi(i, La, Lb):
    return min(2 * i, Lb - 1 - (La - i) // 2)


def on_some_path(La, Lb):
    fwd = np.zeros((La, Lb), bool)
    fwd[0, 0] = True
    for i in range(La):
        for j in range(Lb):
            if not fwd[i, j]:
                fwd[i, j] = any(i >= di and j >= dj and fwd[i - di, j - dj] for di, dj in STEPS)
    bwd = np.zeros((La, Lb), bool)
    bwd[La - 1, Lb - 1] = True
    for i in range(La - 1, -1, -1):
        for j in range(Lb - 1, -1, -1):
            if not bwd[i, j]:
                bwd[i, j] = any(i + di < La and j + dj < Lb and bwd[i + di, j + dj]
                                for di, dj in STEPS)
    return fwd & bwd


@pytest.mark.parametrize("La", range(1, 25))
def test_path_cells_lie_within_bounds(La):
    for Lb in range(1, 25):
        if not (Lb - 1 <= 2 * (La - 1) and La - 1 <= 2 * (Lb - 1)):
            continue  # no path at all
        F = on_some_path(La, Lb)
        for i in range(La):
            cols = np.nonzero(F[i])[0]
            if cols.size:
                assert lo(i, La, Lb) <= cols.min() and cols.max() <= hi(i, La, Lb), (La, Lb, i)
        los = [lo(i, La, Lb) for i in range(La)]
        his = [hi(i, La, Lb) for i in range(La)]
        assert all(a <= b for a, b in zip(los, los[1:]))
        assert all(a <= b for a, b in zip(his, his[1:]))


def test_bounds_are_tight_on_a_square():
    # on a square the region is the rhombus between the slopes 1/2 and 2: the
    # bounds are attained (every column between them lies on some path)
    L = 19
    F = on_some_path(L, L)
    for i in range(L):
        cols = np.nonzero(F[i])[0]
        assert cols.min() == lo(i, L, L) and cols.max() == hi(i, L, L)
