"""Pins of the WSDTW oracle (oracle/wsdtw.py, Sec. II-C) against what the
definition fixes: brute force over every subsequence path and every choice of
fragment end frames on small inputs, the closed form for a query aligned to
itself, and invariants of the result.  CPU only."""
import itertools

import numpy as np
import pytest

from oracle import cost_matrix
from oracle import wsdtw as ws
from paper_2607_15478_gb300 import synth

STEPS = ((1, 1), (1, 2), (2, 1))
WEIGHTS = (1.0, 1.0, 2.0)


def brute_subseq(C):
    """min over every path from any (0, j0) to (n-1, j) of C[0, j0] + sum of
    w_step * C[destination], for every end column j (inf if none)."""
    n, Lb = C.shape
    best = np.full(Lb, np.inf)

    def rec(i, j, acc):
        if i == n - 1:
            best[j] = min(best[j], acc)
        for (di, dj), w in zip(STEPS, WEIGHTS):
            ni, nj = i + di, j + dj
            if ni < n and nj < Lb:
                rec(ni, nj, acc + w * C[ni, nj])

    for j0 in range(Lb):
        rec(0, j0, C[0, j0])
    return best


@pytest.mark.parametrize("n,Lb", [(1, 4), (2, 3), (3, 5), (4, 6), (5, 7), (6, 6)])
@pytest.mark.parametrize("kind", ["int", "real"])
def test_subseq_dtw_is_the_minimum_over_all_paths(n, Lb, kind):
    rng = np.random.default_rng(n * 10 + Lb)
    C = rng.integers(0, 5, size=(n, Lb)).astype(float) if kind == "int" else rng.random((n, Lb))
    D, code = ws.subseq_dtw(C)
    ref = brute_subseq(C)
    if kind == "int":
        np.testing.assert_array_equal(D[-1], ref)
    else:
        np.testing.assert_allclose(D[-1], ref, rtol=0, atol=1e-12)
    # the backtrace from every reachable end realises its score
    for j in range(Lb):
        if np.isfinite(D[-1, j]):
            p = ws.subseq_backtrace(code, j)
            assert p[0, 0] == 0 and tuple(p[-1]) == (n - 1, j)
            tot = C[p[0, 0], p[0, 1]]
            for (i0, j0), (i1, j1) in zip(p[:-1], p[1:]):
                w = WEIGHTS[STEPS.index((i1 - i0, j1 - j0))]
                tot += w * C[i1, j1]
            assert tot == pytest.approx(D[-1, j], abs=1e-12)


def test_subseq_tie_order_prefers_the_diagonal_then_12():
    # all costs equal: every candidate ties; the (1,1) step must be taken
    # wherever it exists, then (1,2)
    C = np.ones((4, 8))
    D, code = ws.subseq_dtw(C)
    diag_ok = np.isfinite(D[:-1, :-1])  # the (1,1) predecessor exists
    assert (code[1:, 1:][diag_ok] == 0).all()
    assert (code[1:, 0] == 3).all()  # column 0 below row 0 is unreachable
    assert code[2, 1] == 2 and D[2, 1] == 3.0  # only (2,1) from (0, 0) reaches (2, 1)
    # (1,1) unavailable only in column 0; a cheaper (1,2) wins where strictly smaller
    C = np.array([[0, 5, 0, 5], [5, 5, 1, 9]], float)
    D, code = ws.subseq_dtw(C)
    # cell (1,2): (1,1) from (0,1): 5 + 1 = 6; (1,2) from (0,0): 0 + 1 = 1 -> code 1
    assert code[1, 2] == 1 and D[1, 2] == 1.0


def brute_segment(Cseg, deltas):
    N, Lb = Cseg.shape
    best, arg = np.inf, None
    for e in itertools.product(range(Lb), repeat=N):
        if any(e[k] - e[k - 1] < deltas[k] for k in range(1, N)):
            continue
        t = sum(Cseg[k, e[k]] for k in range(N))
        if t < best:
            best, arg = t, e
    return best, arg


@pytest.mark.parametrize("N,Lb", [(1, 5), (2, 6), (3, 7), (3, 9)])
def test_segment_dp_is_the_minimum_over_all_end_choices(N, Lb):
    rng = np.random.default_rng(N * 100 + Lb)
    Cseg = rng.random((N, Lb))
    deltas = [0] + [int(rng.integers(1, 3)) for _ in range(N - 1)]
    Dseg, ends, total = ws.segment_dp(Cseg, deltas)
    b, e = brute_segment(Cseg, deltas)
    assert total == pytest.approx(b, abs=1e-12)
    assert sum(Cseg[k, ends[k]] for k in range(N)) == pytest.approx(total, abs=1e-12)
    assert all(ends[k] - ends[k - 1] >= deltas[k] for k in range(1, N))
    assert tuple(ends) == e  # unique optimum for random real costs


def test_segment_ties_take_the_earliest_end():
    Cseg = np.array([[1.0, 0.0, 0.0, 0.0, 0.0]])
    _, ends, total = ws.segment_dp(Cseg, [0])
    assert total == 0.0 and ends[0] == 1


def test_fragments_cover_the_query():
    for La, N in [(10, 3), (1000, 16), (7, 7), (5, 1)]:
        fr = ws.fragments(La, N)
        assert fr[0][0] == 0 and sum(n for _, n in fr) == La
        assert all(fr[k][0] + fr[k][1] == fr[k + 1][0] for k in range(N - 1))
        assert max(n for _, n in fr) - min(n for _, n in fr) <= 1


@pytest.mark.parametrize("La,N", [(64, 4), (200, 8), (150, 1)])
def test_query_aligned_to_itself_is_the_diagonal(La, N):
    rng = np.random.default_rng(La + N)
    A = synth.chroma_frames(rng, La).astype(np.float32)
    r = ws.wsdtw(A, A, N)
    np.testing.assert_array_equal(r.path, np.stack([np.arange(La)] * 2, axis=1))
    assert abs(r.total) <= 1e-12 * La
    np.testing.assert_array_equal(r.ends, [r0 + n - 1 for r0, n in r.frags])


@pytest.mark.parametrize("seed", [0, 1])
def test_invariants_on_warped_pairs(seed):
    wp = synth.warped_pair(synth.rng_for(80, seed), 300, 360, 12, knots=8, tmin=0.7, tmax=1.4)
    N = 6
    r = ws.wsdtw(wp.A, wp.B, N)
    C = cost_matrix(wp.A, wp.B)
    deltas = [n // 2 for _, n in r.frags]
    pos = 0
    total = 0.0
    for k, (r0, n) in enumerate(r.frags):
        # the fragment's path: rows r0 .. r0+n-1 once each or skipped by (2,1), ends at e_k
        p = r.path[pos:]
        m = np.searchsorted(p[:, 0], r0 + n - 1, side="right")
        p = p[:m]
        pos += m
        assert p[0, 0] == r0 and p[-1, 0] == r0 + n - 1 and p[-1, 1] == r.ends[k]
        s = C[p[0, 0], p[0, 1]]
        for (i0, j0), (i1, j1) in zip(p[:-1], p[1:]):
            s += WEIGHTS[STEPS.index((i1 - i0, j1 - j0))] * C[i1, j1]
        assert s == pytest.approx(r.Cseg[k, r.ends[k]], abs=1e-9)
        total += s
        if k:
            assert r.ends[k] - r.ends[k - 1] >= deltas[k]
    assert pos == r.path.shape[0]
    assert total == pytest.approx(r.total, abs=1e-9)
    # planted warp (sanity): the path stays near the generator's warp
    tau = wp.tau
    dev = [abs(tau[j] - i) for i, j in r.path]
    assert np.median(dev) < 3.0
