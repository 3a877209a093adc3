"""Pins for the FP64 oracle: brute force, closed forms, invariants, library routines.

Each test ties the oracle to something other than itself, so that a dropped
term, a wrong weight, a swapped step or a wrong tie order fails at least one.
"""
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2607_15478_gb300 import synth
from tests._pins import (STEPS, all_paths, brute_force, check_path_valid, codes_to_path,
                         constant_cost_path, load_golden, path_codes, path_weighted_cost,
                         tie_order_path)


# ---- cost (cosine distance, Sec. IV) ------------------------------------------------

def test_cost_matches_scipy_cosine():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((17, 12)).astype(np.float32)
    B = np.abs(rng.standard_normal((23, 12))).astype(np.float32)
    ref = cdist(A.astype(np.float64), B.astype(np.float64), metric="cosine")
    np.testing.assert_allclose(oracle.cost_matrix(A, B), ref, rtol=0, atol=1e-13)


def test_cost_special_values():
    A = np.array([[1, 0, 0], [0, 2, 0], [3, 4, 0], [0, 0, 0]], np.float32)
    B = np.array([[1, 0, 0], [-1, 0, 0], [0, 0, 5], [0, 0, 0]], np.float32)
    C = oracle.cost_matrix(A, B)
    assert C[0, 0] == 0.0           # parallel
    assert C[0, 1] == 2.0           # opposite
    assert C[1, 2] == 1.0           # orthogonal
    assert abs(C[2, 0] - (1 - 3 / 5)) < 1e-15
    assert np.all(C[3] == 1.0) and np.all(C[:, 3] == 1.0)   # zero frame: r = 0
    r = oracle.inv_norms(A)
    np.testing.assert_allclose(r[:3], [1.0, 0.5, 0.2], rtol=1e-15)
    assert r[3] == 0.0


# ---- the recurrence against brute-force enumeration --------------------------------

SMALL_SHAPES = [(a, b) for a in range(1, 7) for b in range(1, 7) if oracle.reachable(a, b)]


def test_reachability_matches_enumeration():
    for a in range(1, 8):
        for b in range(1, 8):
            has_path = next(iter(all_paths(a, b)), None) is not None
            assert oracle.reachable(a, b) == has_path, (a, b)


@pytest.mark.parametrize("La,Lb", SMALL_SHAPES)
def test_brute_force_random_costs(La, Lb):
    rng = np.random.default_rng(100 * La + Lb)
    for _ in range(5):
        C = rng.uniform(0.0, 2.0, size=(La, Lb))
        best, arg = brute_force(C)
        path, total = oracle.dtw_matrix(C)
        assert abs(total - best) <= 1e-12 * max(1.0, abs(best))
        check_path_valid(path, La, Lb)
        assert abs(path_weighted_cost(C, path_codes(path)) - best) <= 1e-12 * max(1.0, best)


@pytest.mark.parametrize("La,Lb", SMALL_SHAPES)
def test_brute_force_integer_costs_and_tie_order(La, Lb):
    rng = np.random.default_rng(7 * La + 13 * Lb)
    for _ in range(8):
        C = rng.integers(0, 3, size=(La, Lb)).astype(np.float64)
        best, arg = brute_force(C, exact=True)
        path, total = oracle.dtw_matrix(C)
        assert total == float(best)
        want = codes_to_path(tie_order_path(arg))
        np.testing.assert_array_equal(path, want)


def test_brute_force_mid_sized():
    # a few larger shapes still small enough to enumerate
    rng = np.random.default_rng(5)
    for La, Lb in [(8, 9), (9, 7), (7, 12), (10, 10)]:
        C = rng.integers(0, 4, size=(La, Lb)).astype(np.float64)
        best, arg = brute_force(C, exact=True)
        path, total = oracle.dtw_matrix(C)
        assert total == float(best)
        np.testing.assert_array_equal(path, codes_to_path(tie_order_path(arg)))


def test_full_matrices_satisfy_recurrence():
    # Every reachable cell of D is the min of its three weighted predecessors,
    # and its code names a minimiser (checked independently of run order).
    rng = np.random.default_rng(9)
    C = rng.uniform(0, 1, size=(9, 11))
    _, _, Dc, codes = oracle.dtw_matrix(C, full=True)
    inf = np.inf
    for i in range(9):
        for j in range(11):
            if i == 0 and j == 0:
                assert Dc[0, 0] == C[0, 0]
                continue
            cands = []
            for code, ((di, dj), w) in enumerate(zip(STEPS, (2, 3, 3))):
                pi, pj = i - di, j - dj
                v = Dc[pi, pj] + w * C[i, j] if pi >= 0 and pj >= 0 else inf
                cands.append(v)
            m = min(cands)
            if m == inf:
                assert Dc[i, j] == inf and codes[i, j] == 3
            else:
                assert abs(Dc[i, j] - m) <= 1e-14 * m
                assert abs(cands[codes[i, j]] - m) <= 1e-14 * m


# ---- closed forms -------------------------------------------------------------------

@pytest.mark.parametrize("La,Lb", [(1, 1), (2, 2), (2, 3), (3, 2), (5, 9), (9, 5), (40, 70),
                                   (70, 40), (64, 127), (127, 64), (100, 100)])
def test_constant_cost_closed_form(La, Lb):
    # every path weighs (La-1)+(Lb-1) (Sec. V), so total = c * (1 + (La-1) + (Lb-1))
    c = 0.75
    path, total = oracle.dtw_matrix(np.full((La, Lb), c))
    assert total == c * (1 + (La - 1) + (Lb - 1))
    np.testing.assert_array_equal(path, constant_cost_path(La, Lb))


def test_constant_cost_from_features():
    # identical frames in A and B -> cosine cost 0 everywhere; every path ties
    A = np.tile(np.array([[0.3, 0.4, 1.2]], np.float32), (33, 1))
    B = np.tile(np.array([[0.3, 0.4, 1.2]], np.float32), (50, 1))
    path, total = oracle.dtw(A, B)
    assert abs(total) < 1e-13
    np.testing.assert_array_equal(path, constant_cost_path(33, 50))


@pytest.mark.parametrize("L", [1, 2, 7, 300])
def test_identical_sequences_give_diagonal(L):
    A = synth.chroma_frames(synth.rng_for(90, L), L).astype(np.float32)
    path, total = oracle.dtw(A, A)
    np.testing.assert_array_equal(path, np.stack([np.arange(L)] * 2, axis=1))
    assert abs(total) <= 1e-12 * max(L, 1)


# ---- invariants on synthetic pairs --------------------------------------------------

@pytest.mark.parametrize("La,Lb,seed", [(60, 75, 0), (75, 60, 1), (200, 250, 2), (128, 96, 3)])
def test_invariants_on_warped_pairs(La, Lb, seed):
    wp = synth.warped_pair(synth.rng_for(91, seed), La, Lb, 12, knots=4)
    path, total = oracle.dtw(wp.A, wp.B)
    check_path_valid(path, La, Lb)
    # total equals the weighted sum of costs along the path, recomputed
    assert abs(oracle.path_cost(wp.A, wp.B, path) - total) <= 1e-12 * total
    # on-the-fly cost and explicit cost matrix give the same alignment
    p2, t2 = oracle.dtw_matrix(oracle.cost_matrix(wp.A, wp.B))
    np.testing.assert_array_equal(path, p2)
    assert t2 == total


def test_no_cheaper_path_by_local_detours():
    # replacing any two consecutive steps (1,1)(1,2) <-> (1,2)(1,1) etc. never lowers the cost
    wp = synth.warped_pair(synth.rng_for(92, 0), 120, 140, 12, knots=4)
    C = oracle.cost_matrix(wp.A, wp.B)
    path, total = oracle.dtw(wp.A, wp.B)
    codes = path_codes(path)
    for k in range(len(codes) - 1):
        if codes[k] != codes[k + 1]:
            alt = list(codes)
            alt[k], alt[k + 1] = alt[k + 1], alt[k]
            assert path_weighted_cost(C, alt) >= total - 1e-12 * total


def test_planted_warp_is_recovered():
    # sanity, not parity: the exact path follows the generator's warp closely
    wp = synth.config_pair(0)
    path, _ = oracle.dtw(wp.A, wp.B)
    dev = np.abs(path[:, 0] - wp.tau[path[:, 1]])
    assert np.median(dev) <= 1.0 and np.mean(dev) < 3.0


def test_unreachable_is_an_error():
    for La, Lb in [(1, 2), (2, 1), (2, 4), (5, 10), (10, 5)]:
        with pytest.raises(oracle.OracleError):
            oracle.dtw_matrix(np.ones((La, Lb)))


# ---- hand-derived golden fixtures ---------------------------------------------------

@pytest.mark.parametrize("name", sorted(f for f in os.listdir(os.path.join(
    os.path.dirname(__file__), "golden")) if f.endswith(".txt") and f != "README.txt"))
def test_golden(name):
    g = load_golden(name)
    if g["kind"] == "cost":
        path, total = oracle.dtw_matrix(g["C"])
    else:
        path, total = oracle.dtw(g["A"], g["B"])
    assert total == g["total"]
    np.testing.assert_array_equal(path, g["path"])


def test_path_cost_matrix_against_enumeration_and_features():
    # the matrix path cost equals the hand-written weighted sum of _pins for
    # every path of small shapes, and the on-the-fly path cost of the features
    rng = np.random.default_rng(17)
    for La, Lb in [(3, 4), (5, 5), (6, 4)]:
        C = rng.uniform(0.0, 2.0, size=(La, Lb))
        for codes in all_paths(La, Lb):
            p = codes_to_path(codes)
            assert abs(oracle.path_cost_matrix(C, p) - path_weighted_cost(C, codes)) <= 1e-12
    wp = synth.warped_pair(synth.rng_for(92, 0), 80, 95, 12, knots=4)
    path, total = oracle.dtw(wp.A, wp.B)
    C = oracle.cost_matrix(wp.A, wp.B)
    assert abs(oracle.path_cost_matrix(C, path) - oracle.path_cost(wp.A, wp.B, path)) <= 1e-12 * total
    with pytest.raises(oracle.OracleError):
        oracle.path_cost_matrix(C, np.array([[0, 0], [0, 1]]))


def test_dtw_unit_against_matrix_and_normalised_frames():
    # frames taken as they are: the same as dtw_matrix over 1 - A B^T formed by
    # a plain float64 matrix product, and the same as dtw for frames whose
    # norm is exactly 1 (one-hot and 0.5-valued frames in 4 dimensions)
    rng = np.random.default_rng(23)
    A = rng.standard_normal((70, 16)).astype(np.float32)
    B = rng.standard_normal((85, 16)).astype(np.float32)
    p1, t1 = oracle.dtw_unit(A, B)
    p2, t2 = oracle.dtw_matrix(1.0 - A.astype(np.float64) @ B.astype(np.float64).T)
    np.testing.assert_array_equal(p1, p2)
    assert abs(t1 - t2) <= 1e-12 * abs(t2)
    assert abs(oracle.path_cost_unit(A, B, p1) - t1) <= 1e-12 * abs(t1)
    E = np.eye(4, dtype=np.float32)
    A = np.concatenate([E[rng.integers(0, 4, 40)], np.full((5, 4), 0.5, np.float32)])
    B = np.concatenate([E[rng.integers(0, 4, 50)], np.full((7, 4), 0.5, np.float32)])
    pu, tu = oracle.dtw_unit(A, B)
    pd, td = oracle.dtw(A, B)
    np.testing.assert_array_equal(pu, pd)
    assert tu == td
    # unnormalised frames differ from the cosine cost (a dropped norm shows)
    A2 = 2.0 * A
    assert oracle.dtw_unit(A2, B)[1] != td
