"""Banded exact alignment (dtw_align_banded): the band comes from the exact
alignment of the sequences averaged over `downsample` frames, the exact DP
runs inside it (strip column ranges in the warp-pair kernel, band-restricted
entry maps in the backtrace), and a path at a side of the band falls back to
the full exact DP.  Same arithmetic as dtw_align inside the band, so whenever
the exact path lies inside it the result is bit-identical to dtw_align."""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import synth
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


@pytest.mark.parametrize("La,Lb", SIZES)
def test_wide_band_equals_exact(aligner, La, Lb):
    wp = synth.warped_pair(synth.rng_for(60, La), La, Lb, 12, knots=16, tmin=0.7, tmax=1.4)
    A, B = dev(wp.A), dev(wp.B)
    exact, te = aligner.align(A, B)
    path, total, fb = aligner.align_banded(A, B, downsample=8, halfwidth=4 * max(La, Lb))
    assert not fb
    np.testing.assert_array_equal(path.cpu().numpy(), exact.cpu().numpy())
    assert total == te


@pytest.mark.parametrize("La,Lb", SIZES)
@pytest.mark.parametrize("w", [48, 128])
def test_band_finds_exact_path(aligner, La, Lb, w):
    wp = synth.warped_pair(synth.rng_for(61, La), La, Lb, 12, knots=16, tmin=0.7, tmax=1.4)
    A, B = dev(wp.A), dev(wp.B)
    exact, te = aligner.align(A, B)
    path, total, fb = aligner.align_banded(A, B, downsample=8, halfwidth=w)
    np.testing.assert_array_equal(path.cpu().numpy(), exact.cpu().numpy())
    assert total == te
    if La >= 1000:
        assert not fb  # the warped pairs' paths lie well inside such a band


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
        exact, te = aligner.align(dev(A), dev(B))
        path, total, fb = aligner.align_banded(dev(A), dev(B), downsample=16, halfwidth=0)
        if fb:
            fell += 1
            np.testing.assert_array_equal(path.cpu().numpy(), exact.cpu().numpy())
            assert total == te
        else:
            check_path_valid(path.cpu().numpy(), 1500, 1800)
            assert total >= te
    assert fell >= 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_band_on_unstructured_pairs_is_valid(aligner, seed):
    # random frames: the coarse path says little; the result is either the
    # fallback (exact) or the optimum inside the band, never below the exact one
    rng = np.random.default_rng(100 + seed)
    La, Lb = 1500, 1700
    A = synth.chroma_frames(rng, La).astype(np.float32)
    B = synth.chroma_frames(rng, Lb).astype(np.float32)
    path, total, fb = aligner.align_banded(dev(A), dev(B), downsample=8, halfwidth=64)
    p = path.cpu().numpy()
    check_path_valid(p, La, Lb)
    po, to = oracle.dtw(A, B)
    tg = oracle.path_cost(A, B, p)
    assert tg >= to - 1e-6 * abs(to) - 1e-7 * (La + Lb)
    if fb:
        assert abs(total - to) <= max(1e-5 * abs(to), 2e-6 * (La + Lb))


def test_band_matches_oracle(aligner):
    wp = synth.config_pair(0)
    path, total, fb = aligner.align_banded(dev(wp.A), dev(wp.B), downsample=8, halfwidth=64)
    p = path.cpu().numpy()
    check_path_valid(p, wp.A.shape[0], wp.B.shape[0])
    po, to = oracle.dtw(wp.A, wp.B)
    assert abs(total - to) <= max(1e-5 * abs(to), 2e-6 * (wp.A.shape[0] + wp.B.shape[0]))
