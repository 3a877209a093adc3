"""The warp-pair DP of one pair in thread-block clusters (dtw_options.clusters).

By default a single pair's DP runs in clusters of up to 8 CTAs whose strip
groups hand their border to the next CTA through distributed shared memory
(the last DP warp of a CTA stores into ring 0 of the next CTA and arrives on
its barrier); only the first CTA of a cluster reads a global border.  Only
where the border travels changes: every cell is computed with the same FP32
operations, so paths and totals must be bit-identical to the same sweep
without clusters, and match the FP64 oracle (tests/_parity.py).  Covered:
pairs of one, two and many strip groups, group counts that do not fill the
last cluster, the transposed sweep, the BF16 cost, banded sweeps (several
waves of clusters along a band), and a bounded wait that expires on a
cluster link.
"""
import numpy as np
import pytest

from paper_2607_15478_gb300 import synth
from tests._parity import assert_parity

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


def both(aligner, A, B, **opts):
    from paper_2607_15478_gb300 import pardtw
    p0, t0 = aligner.align(A, B, clusters=pardtw.CLUSTERS_NEVER, **opts)
    p1, t1 = aligner.align(A, B, clusters=pardtw.CLUSTERS_AUTO, **opts)
    np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
    assert t1 == t0
    return p1, t1


# rows swept / 186 = strip groups: 1, 2, 3, 5, 7 (one cluster of 8, its
# ranks past the last group idle), 9 (two clusters of 8, the second with one
# group), 17 (three of 8), 108 (14 of 8) and 135 (23 of 6: 17 clusters of 8
# do not fit at once)
@pytest.mark.parametrize("La,Lb", [(150, 160), (300, 350), (500, 620), (900, 1000), (1300, 1400),
                                   (1700, 1500), (3100, 3500), (20000, 16000), (25000, 20000)])
def test_clusters_bit_identical_and_oracle(aligner, La, Lb):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(110, La), La, Lb, 12, knots=16, tmin=0.5, tmax=2.0)
    p, t = both(aligner, dev(wp.A), dev(wp.B), transpose=pardtw.TRANSPOSE_NEVER)
    assert_parity(wp.A, wp.B, p, t, name="clusters")


@pytest.mark.parametrize("La,Lb", [(900, 1100), (20000, 25000)])
def test_clusters_transposed(aligner, La, Lb):
    from paper_2607_15478_gb300 import pardtw
    wp = synth.config_pair(1, La=La, Lb=Lb)
    p, t = both(aligner, dev(wp.A), dev(wp.B), transpose=pardtw.TRANSPOSE_ALWAYS)
    if La * Lb <= 1e6:
        assert_parity(wp.A, wp.B, p, t, name="clusters")


def test_clusters_exact_ties(aligner):
    # one-hot frames: every cost is 0 or 1 and FP32 is exact, so the tie
    # order alone decides; the oracle's path must come out exactly
    import oracle
    rng = np.random.default_rng(111)
    A = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 2300)]
    B = np.eye(3, dtype=np.float32)[rng.integers(0, 3, 2000)]
    for tr in (1, 2):
        p, t = both(aligner, dev(A), dev(B), transpose=tr)
        po, to = oracle.dtw(A, B)
        assert t == to
        np.testing.assert_array_equal(p.cpu().numpy(), po)


def test_clusters_bf16(aligner):
    wp = synth.warped_pair(synth.rng_for(112, 0), 3000, 3400, 128, kind="gaussian", knots=8,
                           tmin=0.7, tmax=1.4, sigma=0.1)
    for tr in (1, 2):
        both(aligner, dev(wp.A), dev(wp.B), cost_precision=1, transpose=tr)


@pytest.mark.parametrize("La,Lb,w", [(4000, 5000, 48), (30000, 36000, 128)])
def test_clusters_band(aligner, La, Lb, w):
    # a band's chain of strips runs through persistent clusters, several
    # tickets per cluster along the band
    from paper_2607_15478_gb300 import pardtw
    wp = synth.warped_pair(synth.rng_for(113, La), La, Lb, 12, knots=max(8, La // 400),
                           tmin=0.6, tmax=1.6)
    A, B = dev(wp.A), dev(wp.B)
    p0, t0, f0 = aligner.align_banded(A, B, downsample=8, halfwidth=w,
                                      clusters=pardtw.CLUSTERS_NEVER)
    p1, t1, f1 = aligner.align_banded(A, B, downsample=8, halfwidth=w)
    assert f0 == f1 and not f1
    np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
    assert t1 == t0
    assert_parity(wp.A, wp.B, p1, t1, name="clusters-band")


def test_cluster_link_timeout_and_recovery(aligner):
    # group 0 never publishes: group 1, in the same cluster, waits on its
    # distributed-shared-memory ring until the 20 ms limit, the call reports
    # DTW_ERR_TIMEOUT, every CTA of every cluster leaves, and the handle
    # aligns the next pair correctly
    from paper_2607_15478_gb300 import pardtw
    wp = synth.config_pair(0, La=1500, Lb=1700)
    with pytest.raises(pardtw.PardtwError) as e:
        aligner.align(dev(wp.A), dev(wp.B), wait_limit_us=20000, debug_skip_publish=0,
                      transpose=pardtw.TRANSPOSE_NEVER)
    assert e.value.status == pardtw.DTW_ERR_TIMEOUT
    p, t = both(aligner, dev(wp.A), dev(wp.B))
    assert_parity(wp.A, wp.B, p, t, name="clusters")
