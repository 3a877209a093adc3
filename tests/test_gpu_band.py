"""Banded exact alignment (dtw_align_banded): the band comes from the exact
alignment of the sequences averaged over `downsample` frames, the exact DP
runs inside it (strip column ranges in the warp-pair kernel, band-restricted
entry maps in the backtrace), and a path at a side of the band falls back to
the full exact DP.  Same arithmetic as dtw_align inside the band, so whenever
the exact path lies inside it the result is bit-identical to dtw_align.

Every result that claims to be exact (no fallback needed, or the fallback
taken) is judged against the FP64 oracle under the rule of tests/_parity.py;
bit-identity with dtw_align is checked on top of that."""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import synth
from tests._parity import assert_parity, path_tol, total_tol
from tests._pins import check_path_valid

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


SIZES = [(300, 360), (1000, 1200), (2500, 2000), (4000, 5000), (7000, 8000)]
_ORACLE = {}


def oracle_of(key, A, B):
    """oracle.dtw(A, B), computed once per input pair of this module."""
    if key not in _ORACLE:
        _ORACLE[key] = oracle.dtw(A, B)
    return _ORACLE[key]


@pytest.mark.parametrize("La,Lb", SIZES)
def test_wide_band_equals_exact(aligner, La, Lb):
    wp = synth.warped_pair(synth.rng_for(60, La), La, Lb, 12, knots=16, tmin=0.7, tmax=1.4)
    A, B = dev(wp.A), dev(wp.B)
    path, total, fb = aligner.align_banded(A, B, downsample=8, halfwidth=4 * max(La, Lb))
    assert not fb
    assert_parity(wp.A, wp.B, path, total, name="band",
                  ref=oracle_of(("wide", La, Lb), wp.A, wp.B))
    exact, te = aligner.align(A, B)
    np.testing.assert_array_equal(path.cpu().numpy(), exact.cpu().numpy())
    assert total == te


@pytest.mark.parametrize("La,Lb", SIZES)
@pytest.mark.parametrize("w", [48, 128])
def test_band_finds_exact_path(aligner, La, Lb, w):
    wp = synth.warped_pair(synth.rng_for(61, La), La, Lb, 12, knots=16, tmin=0.7, tmax=1.4)
    A, B = dev(wp.A), dev(wp.B)
    path, total, fb = aligner.align_banded(A, B, downsample=8, halfwidth=w)
    assert_parity(wp.A, wp.B, path, total, name="band",
                  ref=oracle_of(("narrow", La, Lb), wp.A, wp.B))
    if La >= 1000:
        assert not fb  # the warped pairs' paths lie well inside such a band
    exact, te = aligner.align(A, B)
    np.testing.assert_array_equal(path.cpu().numpy(), exact.cpu().numpy())
    assert total == te


def test_narrow_band_falls_back_to_exact(aligner):
    # random frames at a coarse scale of 16 with no margin: the coarse path is
    # a poor guide, the banded path meets the band's side and the full exact
    # DP takes over (the band, rounded out to whole strips and 8-column blocks,
    # is never narrower than a strip's slope)
    fell = 0
    for seed in range(4):
        rng = np.random.default_rng(200 + seed)
        A = synth.chroma_frames(rng, 1500).astype(np.float32)
        B = synth.chroma_frames(rng, 1800).astype(np.float32)
        path, total, fb = aligner.align_banded(dev(A), dev(B), downsample=16, halfwidth=0)
        if fb:
            fell += 1
            assert_parity(A, B, path, total, name="band-fallback")
        else:
            assert_band_optimum_not_below_exact(A, B, path, total)
    assert fell >= 1


def assert_band_optimum_not_below_exact(A, B, path, total):
    """A band that cut the exact path off and whose path kept off its sides:
    the result is the optimum inside the band, a valid path whose FP64 cost
    is never below the exact optimum, and whose FP32 total is that cost."""
    La, Lb = A.shape[0], B.shape[0]
    p = path.cpu().numpy()
    check_path_valid(p, La, Lb)
    po, to = oracle.dtw(A, B)
    tg = oracle.path_cost(A, B, p)
    assert tg >= to - path_tol(to, La, Lb)
    assert abs(total - tg) <= total_tol(tg, La, Lb)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_band_on_unstructured_pairs_is_valid(aligner, seed):
    # random frames: the coarse path says little; the result is either the
    # fallback (exact) or the optimum inside the band, never below the exact one
    rng = np.random.default_rng(100 + seed)
    La, Lb = 1500, 1700
    A = synth.chroma_frames(rng, La).astype(np.float32)
    B = synth.chroma_frames(rng, Lb).astype(np.float32)
    path, total, fb = aligner.align_banded(dev(A), dev(B), downsample=8, halfwidth=64)
    if fb:
        assert_parity(A, B, path, total, name="band-fallback")
    else:
        assert_band_optimum_not_below_exact(A, B, path, total)


def test_band_matches_oracle(aligner):
    wp = synth.config_pair(0)
    path, total, fb = aligner.align_banded(dev(wp.A), dev(wp.B), downsample=8, halfwidth=64)
    assert not fb
    assert_parity(wp.A, wp.B, path, total, name="band")


def test_band_multi_wave_matches_oracle(aligner):
    # the learned-band workload's recipe (tempo 0.6-1.6, 256 knots per 1e5
    # frames) on a 30000 x 36000 pair: the band is swept with B's 36000 frames
    # as rows, 387 strips of 93 rows in 194 groups of two, more groups than one
    # wave of CTAs, so groups start as CTAs free up along the band
    La, Lb = 30000, 36000
    wp = synth.warped_pair(synth.rng_for(64, La), La, Lb, 12, knots=77, tmin=0.6, tmax=1.6)
    path, total, fb = aligner.align_banded(dev(wp.A), dev(wp.B), downsample=8, halfwidth=128)
    assert not fb
    assert_parity(wp.A, wp.B, path, total, name="band-multi-wave")


def test_band_fallback_at_multi_wave_size(aligner):
    # unstructured frames at the same size with no margin: the band path meets
    # a side, and the fallback (the full exact DP, several waves) is exact
    for seed in range(3):
        rng = np.random.default_rng(300 + seed)
        A = synth.chroma_frames(rng, 30000).astype(np.float32)
        B = synth.chroma_frames(rng, 33000).astype(np.float32)
        path, total, fb = aligner.align_banded(dev(A), dev(B), downsample=16, halfwidth=0)
        if fb:
            assert_parity(A, B, path, total, name="band-fallback-multi-wave")
            return
    pytest.fail("no fallback on three unstructured 30000 x 33000 pairs")



@pytest.mark.parametrize("D,precision", [(33, 0), (64, 0), (128, 0), (12, 1), (128, 1)])
def test_band_unsupported_features(aligner, D, precision):
    # the banded DP runs in the narrow warp-pair kernel only: D > 32 or the
    # BF16 cost is refused with DTW_ERR_UNSUPPORTED, and the handle still
    # aligns the next pair
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(66, D), 400, 500, D, kind="gaussian", knots=8,
                           tmin=0.7, tmax=1.4, sigma=0.1)
    with pytest.raises(pardtw.PardtwError) as e:
        aligner.align_banded(dev(wp.A), dev(wp.B), downsample=8, halfwidth=64,
                             cost_precision=precision)
    assert e.value.status == pardtw.DTW_ERR_UNSUPPORTED
    path, total = aligner.align(dev(wp.A), dev(wp.B))
    check_path_valid(path.cpu().numpy(), 400, 500)
