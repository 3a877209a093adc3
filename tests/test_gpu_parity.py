"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Acceptance (tests/_parity.py): the GPU path is a valid DTW path; its FP32
total lies within 1e-5 relative of the oracle's FP64 total; the path equals
the oracle's index for index, or -- where FP32 rounding resolves a near-tie
differently -- its FP64-recomputed cost lies within 1e-6 relative of the
optimum.  Absolute floors apply only to totals below 1 (identical or
constant-cost sequences).  Where every cost is a small integer (one-hot
features) the FP32 arithmetic is exact, and paths and totals must match
exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import synth
from tests._parity import assert_parity
from tests._pins import check_path_valid, constant_cost_path

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aligner():
    from paper_2607_15478_gb300 import build, pardtw
    build.build()
    a = pardtw.Aligner(0)
    yield a
    a.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


SHAPES = [(1, 1), (2, 2), (2, 3), (3, 2), (5, 9), (31, 33), (32, 32), (33, 31), (33, 64),
          (64, 33), (100, 150), (127, 129), (128, 128), (129, 130), (130, 257), (257, 300),
          (300, 257), (500, 400), (513, 1000), (1000, 513), (700, 900), (255, 500),
          (256, 300), (257, 400), (384, 200), (1025, 900)]


@pytest.mark.parametrize("La,Lb", SHAPES)
def test_parity_small_shapes(aligner, La, Lb):
    wp = synth.warped_pair(synth.rng_for(50, La * 1000 + Lb), La, Lb, 12, knots=4,
                           tmin=0.5, tmax=2.0)
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, path, total)


@pytest.mark.parametrize("D", [1, 3, 4, 7, 12, 13, 16, 20, 32, 33, 64, 100, 128])
def test_parity_feature_dims(aligner, D):
    La, Lb = 200, 230
    rng = synth.rng_for(51, D)
    wp = synth.warped_pair(rng, La, Lb, D, kind="gaussian" if D > 12 else "chroma", knots=4)
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, path, total)


@pytest.mark.parametrize("La,Lb,K", [(40, 50, 3), (129, 170, 4), (300, 260, 2), (700, 999, 5)])
def test_exact_ties_onehot(aligner, La, Lb, K):
    # one-hot frames: cosine cost is exactly 0 or 1, FP32 arithmetic is exact,
    # many paths tie; the tie order must give the oracle's path exactly
    rng = np.random.default_rng(La + Lb)
    A = np.eye(K, dtype=np.float32)[rng.integers(0, K, La)]
    B = np.eye(K, dtype=np.float32)[rng.integers(0, K, Lb)]
    path, total = aligner.align(dev(A), dev(B))
    po, to = oracle.dtw(A, B)
    assert total == to
    np.testing.assert_array_equal(path.cpu().numpy(), po)


@pytest.mark.parametrize("La,Lb", [(1, 1), (3, 4), (40, 70), (70, 40), (300, 599), (599, 300),
                                   (1000, 1000)])
def test_all_paths_tie(aligner, La, Lb):
    # frames whose FP32 normalisation is exact (norm 1), so every cost is
    # exactly 0 on both sides and every path ties; the tie order decides
    A = np.full((La, 4), 0.5, np.float32)
    B = np.full((Lb, 4), 0.5, np.float32)
    path, total = aligner.align(dev(A), dev(B))
    np.testing.assert_array_equal(path.cpu().numpy(), constant_cost_path(La, Lb))
    assert total == 0.0


def test_near_constant_cost(aligner):
    # identical frames with an inexact FP32 norm: costs are rounding noise
    # around 0, so any path is acceptable within the FP32 resolution
    A = np.tile(np.array([[0.25, 0.5, 1.0, 0.0]], np.float32), (600, 1))
    B = A[:1].repeat(700, axis=0)
    path, total = aligner.align(dev(A), dev(B))
    assert_parity(A, B, path, total)


def test_identical_sequences_diagonal(aligner):
    A = synth.chroma_frames(synth.rng_for(52, 0), 777).astype(np.float32)
    path, total = aligner.align(dev(A), dev(A))
    np.testing.assert_array_equal(path.cpu().numpy(), np.stack([np.arange(777)] * 2, 1))
    assert_parity(A, A, path, total, name="identical")


def test_zero_frames(aligner):
    wp = synth.warped_pair(synth.rng_for(53, 0), 90, 100, 12, knots=3)
    A, B = wp.A.copy(), wp.B.copy()
    A[::7] = 0.0
    B[::5] = 0.0
    path, total = aligner.align(dev(A), dev(B))
    assert_parity(A, B, path, total)


def test_parity_config0_full(aligner):
    wp = synth.config_pair(0)
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, path, total, name="pair1000x1200")


def test_parity_config1_full(aligner):
    # the benchmark workload, in the launch configuration bench.py times
    wp = synth.config_pair(1)
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, path, total, name="pair20000x25000")


def test_cost_shift_keeps_path(aligner):
    wp = synth.config_pair(1, La=3000, Lb=3700)
    p0, t0 = aligner.align(dev(wp.A), dev(wp.B))
    p1, t1 = aligner.align(dev(wp.A), dev(wp.B), cost_shift=0.05)
    po, to = assert_parity(wp.A, wp.B, p1, t1)
    assert abs(t1 - to) <= abs(t0 - to) + 1e-5 * to


def test_deterministic(aligner):
    wp = synth.config_pair(1, La=2000, Lb=2500)
    A, B = dev(wp.A), dev(wp.B)
    p0, t0 = aligner.align(A, B)
    for _ in range(3):
        p1, t1 = aligner.align(A, B)
        assert t1 == t0
        assert torch.equal(p0, p1)


def test_host_buffers_roundtrip(aligner):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.config_pair(0, La=400, Lb=480)
    A = torch.from_numpy(wp.A).pin_memory()
    B = torch.from_numpy(wp.B).pin_memory()
    cap = 400
    path = torch.zeros((cap, 2), dtype=torch.int32).pin_memory()
    plen = torch.zeros(1, dtype=torch.int32)
    tot = torch.zeros(1, dtype=torch.float32)
    pardtw.dtw_align(aligner.h, A, B, path, plen, tot)
    n = int(plen[0])
    assert_parity(wp.A, wp.B, path[:n].numpy(), float(tot[0]))


def cost_tolerance(D):
    # FP32 against the FP64 matrix, u = 2^-24: the sums of squares (D FMAs)
    # and the reciprocal square root leave each normalised feature within
    # (D/2 + 2) u relative, which moves the dot product (|a^ . b^| <= 1) by at
    # most (D + 4) u; the D FMAs from 1 round partial sums of magnitude <= 2,
    # at most 2 D u more
    return (3 * D + 8) * 2.0 ** -24


# k_cost's tiles are 16 rows x 256 columns, 4 x 4 cells a thread: ragged row
# and column tiles, rows of a length that is not a multiple of 4 (4-byte
# stores) and of one that is (16-byte stores), every padded feature width
# (4, 8, 12, 16 with b^ in registers; 64, 128 loaded per tile)
COST_CASES = [(1, 1, 3), (150, 170, 12), (37, 517, 4), (45, 520, 12), (70, 300, 8),
              (90, 263, 16), (260, 1030, 33), (300, 777, 100), (64, 256, 128)]


@pytest.mark.parametrize("La,Lb,D", COST_CASES)
def test_cost_matrix(aligner, La, Lb, D):
    rng = synth.rng_for(55, La * 7 + Lb * 3 + D)
    A = rng.standard_normal((La, D)).astype(np.float32)
    B = rng.standard_normal((Lb, D)).astype(np.float32)
    A[La // 2] = 0.0  # a zero frame costs 1 against anything
    B[Lb // 3] = 0.0
    C = aligner.cost(dev(A), dev(B)).cpu().numpy()
    Co = oracle.cost_matrix(A, B)
    assert np.max(np.abs(C - Co)) <= cost_tolerance(D)
    assert np.all(C[La // 2] == 1.0) and np.all(C[:, Lb // 3] == 1.0)


def test_cost_matrix_host_buffers_and_many_row_tiles(aligner):
    from paper_2607_15478_gb300 import pardtw
    # host inputs and output (staged through the workspace) give the same bits
    rng = synth.rng_for(56, 0)
    A = rng.standard_normal((45, 12)).astype(np.float32)
    B = rng.standard_normal((521, 12)).astype(np.float32)
    Ch = torch.empty((45, 521), dtype=torch.float32)
    pardtw.dtw_cost(aligner.h, torch.from_numpy(A), torch.from_numpy(B), Ch)
    Cd = aligner.cost(dev(A), dev(B)).cpu()
    assert torch.equal(Ch, Cd)
    # ~66000 tiles of 16 rows for one column of blocks (the grid holds about
    # 8192 blocks, so each takes ~8 tiles), the last one ragged
    La = 65535 * 16 + 4000
    A = rng.standard_normal((La, 4)).astype(np.float32)
    B = rng.standard_normal((9, 4)).astype(np.float32)
    C = aligner.cost(dev(A), dev(B)).cpu().numpy()
    assert np.max(np.abs(C - oracle.cost_matrix(A, B))) <= cost_tolerance(4)


def _fma_f32(w, c, t):
    """float32(w * c + t) with one rounding: w * c (a float32 times 2 or 3) is
    exact in FP64, and the FP64 sum is checked to be exact (TwoSum), so the
    rounding to float32 is the only one."""
    p, t = w * float(c), float(t)
    s = p + t
    bb = s - p
    assert (p - (s - bb)) + (t - bb) == 0.0
    return np.float32(s)


@pytest.mark.parametrize("La,Lb", [(600, 700), (700, 600)])
def test_cost_matrix_is_the_dp_cost(aligner, La, Lb):
    # the explicit matrix holds the DP's own costs bit for bit: the aligner's
    # FP32 total equals D(0,0) = C(0,0), D = fma(w, C, D) along its path over
    # dtw_cost's matrix (both sweep directions)
    wp = synth.config_pair(0, La=La, Lb=Lb)
    C = aligner.cost(dev(wp.A), dev(wp.B)).cpu().numpy()
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    p = path.cpu().numpy() if hasattr(path, "cpu") else np.asarray(path)
    t = np.float32(C[0, 0])
    for (i0, j0), (i1, j1) in zip(p[:-1], p[1:]):
        t = _fma_f32(2.0 if (i1 - i0, j1 - j0) == (1, 1) else 3.0, C[i1, j1], t)
    assert float(t) == float(total)


def test_unreachable_and_invalid(aligner):
    from paper_2607_15478_gb300 import pardtw
    A = dev(np.ones((3, 4), np.float32))
    B = dev(np.ones((10, 4), np.float32))
    with pytest.raises(pardtw.PardtwError) as e:
        aligner.align(A, B)
    assert e.value.status == pardtw.DTW_ERR_UNREACHABLE
    path = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.dtw_align(aligner.h, A, dev(np.ones((4, 4), np.float32)), path, plen)
    assert e.value.status == pardtw.DTW_ERR_INVALID


def test_timeout_is_reported_and_handle_survives(aligner):
    # the first strip group never publishes its bottom border; the group below
    # waits for ~20 ms, records DTW_ERR_TIMEOUT and every CTA leaves
    from paper_2607_15478_gb300 import pardtw
    wp = synth.config_pair(0, La=600, Lb=700)
    with pytest.raises(pardtw.PardtwError) as e:
        aligner.align(dev(wp.A), dev(wp.B), wait_limit_us=20000, debug_skip_publish=0)
    assert e.value.status == pardtw.DTW_ERR_TIMEOUT
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, path, total)


def test_align_many_matches_single(aligner):
    pairs = synth.config_batch(2, n_pairs=6, La_range=(100, 900))
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    # one unreachable pair in the middle must not stop the others
    As.insert(3, dev(np.ones((3, 12), np.float32)))
    Bs.insert(3, dev(np.ones((20, 12), np.float32)))
    paths, costs, st = aligner.align_many(As, Bs)
    assert st[3] == 2 and paths[3] is None
    k = 0
    for idx in range(len(As)):
        if idx == 3:
            continue
        p = pairs[k]
        k += 1
        assert st[idx] == 0
        assert_parity(p.A, p.B, paths[idx], float(costs[idx]))


# (rows per lane, schedule, strips per CTA): one row per lane; the fused
# multi-row kernel; the cost/DP warp pairs with two and four strips per CTA
DECOMPOSITIONS = [(1, 0, 0), (2, 1, 0), (4, 1, 0), (2, 2, 2), (3, 2, 2), (4, 2, 2), (2, 2, 4),
                  (3, 2, 4)]


@pytest.mark.parametrize("La,Lb", [(61, 70), (62, 100), (63, 64), (92, 120), (93, 93),
                                   (94, 150), (124, 150), (125, 200), (186, 250), (187, 190),
                                   (247, 300), (248, 250), (249, 400), (371, 400), (372, 380),
                                   (373, 500), (744, 800), (745, 900),
                                   (500, 620), (1000, 1200), (3001, 2500)])
def test_rows_per_lane_decompositions_agree(aligner, La, Lb):
    # the row decomposition and the division of labour between warps only
    # change who computes what: every cell is computed with the same FP32
    # operations, so paths and totals must be bit-identical across
    # decompositions, and match the oracle
    wp = synth.warped_pair(synth.rng_for(55, La + Lb), La, Lb, 12, knots=4, tmin=0.5, tmax=2.0)
    A, B = dev(wp.A), dev(wp.B)
    ref = None
    for R, sched, ns in DECOMPOSITIONS:
        path, total = aligner.align(A, B, rows_per_lane=R, dp_schedule=sched,
                                    strips_per_cta=ns)
        if ref is None:
            ref = (path.cpu().numpy(), total)
            assert_parity(wp.A, wp.B, path, total)
        else:
            np.testing.assert_array_equal(path.cpu().numpy(), ref[0],
                                          err_msg=f"R={R} s={sched} ns={ns}")
            assert total == ref[1], (R, sched, ns)


@pytest.mark.parametrize("D", [4, 8, 16, 32])
def test_decompositions_agree_feature_dims(aligner, D):
    wp = synth.warped_pair(synth.rng_for(56, D), 400, 450, D, knots=4, tmin=0.5, tmax=2.0)
    A, B = dev(wp.A), dev(wp.B)
    ref = None
    for R, sched, ns in DECOMPOSITIONS:
        if R == 4 and D > 16:
            continue
        path, total = aligner.align(A, B, rows_per_lane=R, dp_schedule=sched,
                                    strips_per_cta=ns)
        if ref is None:
            ref = (path.cpu().numpy(), total)
            assert_parity(wp.A, wp.B, path, total)
        else:
            np.testing.assert_array_equal(path.cpu().numpy(), ref[0], err_msg=f"R={R} s={sched}")
            assert total == ref[1], (R, sched)


@pytest.mark.parametrize("R,sched,ns", DECOMPOSITIONS)
def test_exact_ties_every_decomposition(aligner, R, sched, ns):
    rng = np.random.default_rng(77)
    A = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 700)]
    B = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 900)]
    path, total = aligner.align(dev(A), dev(B), rows_per_lane=R, dp_schedule=sched,
                                strips_per_cta=ns)
    po, to = oracle.dtw(A, B)
    assert total == to
    np.testing.assert_array_equal(path.cpu().numpy(), po)


def test_aligner_on_its_own_stream(aligner):
    # a handle bound to a side stream: the convenience calls order that stream
    # after the inputs and torch's stream after the outputs
    from paper_2607_15478_gb300 import pardtw
    wp = synth.config_pair(0)
    side = torch.cuda.Stream()
    with pardtw.Aligner(0, side) as al2:
        for _ in range(3):
            A, B = dev(wp.A), dev(wp.B)
            path, total = al2.align(A, B)
            assert_parity(wp.A, wp.B, path, total)


@pytest.mark.parametrize("La,Lb", [(300, 400), (400, 300), (500, 500), (94, 186), (1000, 1999),
                                   (2001, 1500), (187, 250)])
def test_transposed_sweep_is_bit_identical(aligner, La, Lb):
    # the pair swept with B's frames as rows (the kernel's (1,2) and (2,1)
    # candidates swapped, the tie order mapped back) gives the same cells,
    # hence the same path and total, as the direct sweep -- for random
    # frames and for exact ties (one-hot frames: every cost is 0 or 1)
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(58, La + Lb), La, Lb, 12, knots=4, tmin=0.5, tmax=2.0)
    rng = np.random.default_rng(La * 7 + Lb)
    ties = (np.eye(3, dtype=np.float32)[rng.integers(0, 3, La)],
            np.eye(3, dtype=np.float32)[rng.integers(0, 3, Lb)])
    for A, B in ((wp.A, wp.B), ties):
        res = []
        for t in (pardtw.TRANSPOSE_NEVER, pardtw.TRANSPOSE_ALWAYS, pardtw.TRANSPOSE_AUTO):
            path, total = aligner.align(dev(A), dev(B), transpose=t)
            res.append((path.cpu().numpy(), total))
        for p, tot in res[1:]:
            np.testing.assert_array_equal(p, res[0][0])
            assert tot == res[0][1]
        assert_parity(A, B, res[0][0], res[0][1])


@pytest.mark.parametrize("La,Lb", [(700, 900), (900, 700)])
def test_transposed_sweep_bf16_and_four_strips(aligner, La, Lb):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(59, La), La, Lb, 64, kind="gaussian", knots=4,
                           tmin=0.6, tmax=1.6, sigma=0.1)
    for opts in ({"cost_precision": 1}, {"strips_per_cta": 4}):
        A = wp.A if "cost_precision" in opts else wp.A[:, :12]
        B = wp.B if "cost_precision" in opts else wp.B[:, :12]
        p0, t0 = aligner.align(dev(A), dev(B), transpose=pardtw.TRANSPOSE_NEVER, **opts)
        p1, t1 = aligner.align(dev(A), dev(B), transpose=pardtw.TRANSPOSE_ALWAYS, **opts)
        np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
        assert t1 == t0


# Pairs whose strip groups outnumber the CTAs resident at once (two strips of
# 93 rows per CTA and one CTA per SM at D = 16; 152 SMs): the DP kernel maps
# the backtrace's bands itself, on the CTAs that find no strip group left, as
# the strips of each band complete.  The path must be bit-identical to that
# of a sweep whose band map runs as a separate kernel, and match the oracle.
def test_band_map_inside_dp_kernel(aligner):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(60, 30000), 30000, 16000, 16, knots=64, tmin=1.3,
                           tmax=2.2)
    A, B = dev(wp.A), dev(wp.B)
    p0, t0 = aligner.align(A, B, transpose=pardtw.TRANSPOSE_NEVER)  # 162 groups
    p1, t1 = aligner.align(A, B, rows_per_lane=1)  # one row per lane, separate band map
    np.testing.assert_array_equal(p0.cpu().numpy(), p1.cpu().numpy())
    assert t0 == t1
    assert_parity(wp.A, wp.B, p0, t0, name="multi-wave")


@pytest.mark.parametrize("case", ["transposed", "two_ctas_per_sm", "d32"])
def test_band_map_inside_dp_kernel_variants(aligner, case):
    # the first sweep has more strip groups than resident CTAs (band map in
    # the DP kernel), the second runs its band map as a separate kernel
    from paper_2607_15478_gb300 import pardtw
    if case == "transposed":  # swept with B's 30000 frames as rows: 162 groups
        wp = synth.warped_pair(synth.rng_for(61, 16000), 16000, 30000, 16, knots=64, tmin=0.45,
                               tmax=0.77)
        first = {"transpose": pardtw.TRANSPOSE_ALWAYS}
        second = {"transpose": pardtw.TRANSPOSE_NEVER}
    elif case == "two_ctas_per_sm":  # D = 12: two CTAs per SM, 307 groups
        wp = synth.warped_pair(synth.rng_for(63, 57000), 57000, 30000, 12, knots=64, tmin=1.3,
                               tmax=2.2)
        first = {"transpose": pardtw.TRANSPOSE_NEVER}
        second = {"rows_per_lane": 1}
    else:  # D = 32: 162 groups
        wp = synth.warped_pair(synth.rng_for(62, 30000), 30000, 16000, 32, kind="gaussian",
                               knots=64, tmin=1.3, tmax=2.2, sigma=0.1)
        first = {"transpose": pardtw.TRANSPOSE_NEVER}
        second = {"rows_per_lane": 1}
    A, B = dev(wp.A), dev(wp.B)
    p0, t0 = aligner.align(A, B, **first)
    p1, t1 = aligner.align(A, B, **second)
    p0 = p0.cpu().numpy()
    check_path_valid(p0, wp.A.shape[0], wp.B.shape[0])
    np.testing.assert_array_equal(p0, p1.cpu().numpy())
    assert t0 == t1
    assert_parity(wp.A, wp.B, p0, t0, name="multi-wave")


# D = 64, 128 with the FP32 cost: the warp pairs with two cost warps per
# strip (the strip's rows of A^ in shared memory, 4 of the 8 columns of a
# sub-chunk each) keep one FMA per feature in feature order, so every cell
# equals that of the one-row-per-lane kernel bit for bit, in either sweep
# direction and with or without thread-block clusters.
@pytest.mark.parametrize("La,Lb,D", [(300, 360, 64), (700, 900, 128), (2000, 1700, 100),
                                     (3100, 3600, 128)])
def test_wide_features_equal_one_row_per_lane(aligner, La, Lb, D):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(57, La + D), La, Lb, D, kind="gaussian", knots=8,
                           tmin=0.6, tmax=1.6, sigma=0.1)
    A, B = dev(wp.A), dev(wp.B)
    p_ref, t_ref = aligner.align(A, B, rows_per_lane=1)
    p_ref = p_ref.cpu().numpy()
    for tr in (pardtw.TRANSPOSE_NEVER, pardtw.TRANSPOSE_ALWAYS):
        for cl in (pardtw.CLUSTERS_AUTO, pardtw.CLUSTERS_NEVER):
            p, t = aligner.align(A, B, transpose=tr, clusters=cl)
            np.testing.assert_array_equal(p.cpu().numpy(), p_ref, err_msg=f"tr={tr} cl={cl}")
            assert t == t_ref, (tr, cl)
    assert_parity(wp.A, wp.B, p_ref, t_ref, name="wide-fp32")


def test_wide_features_multi_wave(aligner):
    # 30000 rows swept directly at D = 64: 162 strip groups, more than one
    # wave of CTAs (persistent clusters take several tickets each)
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(58, 30000), 30000, 16000, 64, kind="gaussian",
                           knots=64, tmin=1.3, tmax=2.2, sigma=0.1)
    A, B = dev(wp.A), dev(wp.B)
    p0, t0 = aligner.align(A, B, transpose=pardtw.TRANSPOSE_NEVER)
    p1, t1 = aligner.align(A, B, transpose=pardtw.TRANSPOSE_NEVER, clusters=pardtw.CLUSTERS_NEVER)
    p2, t2 = aligner.align(A, B, rows_per_lane=1)
    np.testing.assert_array_equal(p0.cpu().numpy(), p1.cpu().numpy())
    np.testing.assert_array_equal(p0.cpu().numpy(), p2.cpu().numpy())
    assert t0 == t1 == t2
    assert_parity(wp.A, wp.B, p0, t0, name="wide-fp32-multi-wave")


def test_large_square_pair(aligner):
    # a 300000 x 300000 pair (9e10 cells, a 40.9 GB workspace: 0.45 bytes per
    # cell), far beyond what the oracle can align: the path must be a valid
    # DTW path and the FP32 total must equal the FP64 cost of that path up
    # to FP32 accumulation over its ~4.5e5 steps (1e-4 relative; the cost
    # shift keeps the partial sums small)
    from paper_2607_15478_gb300 import pardtw
    L = 300000
    assert pardtw.workspace_size(L, L, 12) < 42e9
    wp = synth.config_pair(1, La=L, Lb=L)
    path, total = aligner.align(dev(wp.A), dev(wp.B), cost_shift=0.05)
    p = path.cpu().numpy()
    check_path_valid(p, L, L)
    tg = oracle.path_cost(wp.A, wp.B, p)
    assert abs(total - tg) <= 1e-4 * abs(tg), (total, tg)
