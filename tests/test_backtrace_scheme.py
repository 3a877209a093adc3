"""The parallel backtrace scheme, restated on the CPU, gives the oracle's path
over the oracle's step codes, and the serial walk's path over random step
codes (CPU).

The CUDA backtrace (band map, two- and four-band maps, chain of crossings,
band walks)
is checked against the oracle on the GPU.  This test checks the scheme
itself, independently of its kernels, on many shapes and band counts: bands
of `BAND` rows; in every band, row by row over the columns a path can reach
(lo(r0) .. hi(r1-1)), the entry of each cell = the entry of its step's
predecessor, or the predecessor itself (2 * column + last-row bit) when that
lies in the band above; the crossings from the end cell up, four bands per
lookup through the composed map of every fourth band from the top, then two
per lookup through the map of every other band; the walks, each from
its band's crossing (or one lookup away) down to where the path leaves the
band, which must be the cell its first cell's entry names."""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import synth

BAND = 128
ORIGIN, NOPATH = -1, -2
STEP = {0: (1, 1), 1: (1, 2), 2: (2, 1)}


def lo(i, La, Lb):
    return max((i + 1) // 2, Lb - 1 - 2 * (La - 1 - i), 0)


def hi(i, La, Lb):
    return min(2 * i, Lb - 1 - (La - i) // 2)


def band_map(code, b):
    """Exits (entries of the band's last two rows) and the entries of the last row."""
    La, Lb = code.shape
    r0, r1 = b * BAND, min((b + 1) * BAND, La)
    xs, ys = lo(r0, La, Lb), hi(r1 - 1, La, Lb) + 1
    rows = {}
    for i in range(r0, r1):
        e = np.full(Lb, NOPATH, dtype=np.int64)
        for j in range(xs, ys):
            if i == 0 and j == 0:
                e[j] = ORIGIN
                continue
            c = int(code[i, j])
            if c == 3:
                continue
            di, dj = STEP[c]
            pi, pj = i - di, j - dj
            if pi < r0:
                e[j] = 2 * pj + (1 if pi == r0 - 1 else 0)
            elif xs <= pj < ys:
                e[j] = rows[pi][pj]
        rows[i] = e
    last2 = rows[r1 - 2] if r1 - 2 >= r0 else np.full(Lb, NOPATH, dtype=np.int64)
    return np.stack([last2, rows[r1 - 1]], axis=1), rows[r1 - 1]


def entry_cell(e, x):
    return ((x * BAND - 1) if (e & 1) else (x * BAND - 2), e >> 1)


def pick(ex, ci, last):
    return int(ex[1] if ci == last else ex[0])


def scheme_path(code):
    La, Lb = code.shape
    nb = -(-La // BAND)
    maps = [band_map(code, b) for b in range(nb)]
    exits = [m[0] for m in maps]
    end_entry = int(maps[-1][1][Lb - 1])
    last_row = [min((b + 1) * BAND, La) - 1 for b in range(nb)]
    # the two-band map of bands nb-2, nb-4, ... (>= 2)
    ex2 = {}
    for b in range(nb - 2, 1, -2):
        comp = np.full((Lb, 2), NOPATH, dtype=np.int64)
        for j in range(Lb):
            for r in range(2):
                e = int(exits[b][j, r])
                if e < 0:
                    continue
                ci, cj = entry_cell(e, b)
                if 0 <= cj < Lb:
                    comp[j, r] = pick(exits[b - 1][cj], ci, b * BAND - 1)
        ex2[b] = comp
    # the four-band map of bands nb-2, nb-6, ... (>= 4): the two-band map of b
    # names a cell in band b-2's last rows, whose two-band map goes on to b-4
    ex4 = {}
    for b in range(nb - 2, 3, -4):
        comp = np.full((Lb, 2), NOPATH, dtype=np.int64)
        for j in range(Lb):
            for r in range(2):
                e = int(ex2[b][j, r])
                if e < 0:
                    continue
                ci, cj = entry_cell(e, b - 1)
                if 0 <= cj < Lb:
                    comp[j, r] = pick(ex2[b - 2][cj], ci, (b - 1) * BAND - 1)
        ex4[b] = comp
    # the chain
    cross = {nb - 1: (La - 1, Lb - 1)}
    e, b = end_entry, nb - 1
    if b >= 1:
        cross[b - 1] = entry_cell(e, b)
        b -= 1
    while b >= 4:
        ci, cj = cross[b]
        cross[b - 2] = entry_cell(pick(ex2[b][cj], ci, last_row[b]), b - 1)
        cross[b - 4] = entry_cell(pick(ex4[b][cj], ci, last_row[b]), b - 3)
        b -= 4
    while b >= 2:
        ci, cj = cross[b]
        e = pick(ex2[b][cj], ci, last_row[b])
        cross[b - 2] = entry_cell(e, b - 1)
        b -= 2
    if b == 1:
        ci, cj = cross[1]
        cross[0] = entry_cell(pick(exits[1][cj], ci, last_row[1]), 1)
    ci, cj = cross[0]
    assert (pick(exits[0][cj], ci, last_row[0]) if nb >= 2 else end_entry) == ORIGIN
    # the walks
    pieces = []
    for b in range(nb):
        if b not in cross:  # one lookup from the crossing below
            c1 = cross[b + 1]
            cross[b] = entry_cell(pick(exits[b + 1][c1[1]], c1[0], last_row[b + 1]), b + 1)
        i, j = cross[b]
        target = None
        if b > 0:
            e = end_entry if b == nb - 1 else pick(exits[b][j], i, last_row[b])
            target = entry_cell(e, b)
        piece = []
        while i >= b * BAND:
            piece.append((i, j))
            if i == 0 and j == 0:
                break
            di, dj = STEP[int(code[i, j])]
            i, j = i - di, j - dj
        if b > 0:
            assert (i, j) == target, (b, (i, j), target)
        pieces.append(piece[::-1])
    return np.array([c for p in pieces for c in p], dtype=np.int32)


SHAPES = [(1, 1), (2, 3), (127, 129), (128, 128), (129, 200), (256, 300), (300, 256),
          (383, 500), (511, 600), (640, 520), (700, 900), (1030, 900), (1300, 1500)]


@pytest.mark.parametrize("La,Lb", SHAPES)
def test_scheme_gives_the_oracle_path(La, Lb):
    if La <= 3 or Lb <= 3:
        rng = np.random.default_rng(La + Lb)
        A = rng.random((La, 4)).astype(np.float32) + 0.1
        B = rng.random((Lb, 4)).astype(np.float32) + 0.1
    else:
        wp = synth.warped_pair(synth.rng_for(71, La + Lb), La, Lb, 12, knots=6, tmin=0.5,
                               tmax=2.0)
        A, B = wp.A, wp.B
    C = oracle.cost_matrix(A, B)
    path, _, _, code = oracle.dtw_matrix(C, full=True)
    np.testing.assert_array_equal(scheme_path(code), path)


def test_scheme_on_exact_ties():
    # one-hot frames: costs 0 or 1, many optimal paths; the scheme follows
    # the same step codes, so it must give the oracle's (tie-ordered) path
    rng = np.random.default_rng(3)
    A = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 700)]
    B = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 650)]
    C = oracle.cost_matrix(A, B)
    path, _, _, code = oracle.dtw_matrix(C, full=True)
    np.testing.assert_array_equal(scheme_path(code), path)


def random_codes(rng, La, Lb):
    """Step codes chosen at random among the steps whose predecessor is
    reachable from (0, 0), so that every backward walk ends at the origin;
    paths from neighbouring cells then part often (unlike DTW's, which merge),
    which exercises the row choice at every crossing."""
    code = np.full((La, Lb), 3, dtype=np.int8)
    for i in range(La):
        for j in range(Lb):
            ok = [c for c, (di, dj) in STEP.items()
                  if i - di >= 0 and j - dj >= 0 and (j - dj) <= 2 * (i - di)
                  and (i - di) <= 2 * (j - dj) and not (i - di == 0 and j - dj > 0)]
            if (i, j) != (0, 0) and ok:
                code[i, j] = ok[rng.integers(len(ok))]
    return code


def serial_walk(code):
    i, j = code.shape[0] - 1, code.shape[1] - 1
    out = [(i, j)]
    while (i, j) != (0, 0):
        di, dj = STEP[int(code[i, j])]
        i, j = i - di, j - dj
        out.append((i, j))
    return np.array(out[::-1], dtype=np.int32)


@pytest.mark.parametrize("La,Lb", [(300, 280), (520, 640), (777, 700), (1100, 1000)])
def test_scheme_on_random_step_codes(La, Lb):
    code = random_codes(np.random.default_rng(La * 3 + Lb), La, Lb)
    np.testing.assert_array_equal(scheme_path(code), serial_walk(code))
