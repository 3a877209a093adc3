"""WSDTW on the GPU (dtw_wsdtw, Sec. II-C) against the FP64 oracle
(oracle/wsdtw.py): the segment costs C_seg element by element, the fragment
end frames, the path and the total.

Acceptance (FP32 against FP64): C_seg within 1e-5 relative plus 1e-6 per
fragment row (the FP32 rounding of a sum of up to 2 len costs), the same +inf
entries, the same end frames; the path equal to the oracle's, or (where FP32
decided a near-tie differently) of the same FP64 cost within that tolerance."""
import numpy as np
import pytest

from oracle import cost_matrix
from oracle import wsdtw as ws
from paper_2607_15478_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS = ((1, 1), (1, 2), (2, 1))
WEIGHTS = (1.0, 1.0, 2.0)


@pytest.fixture(scope="module")
def aligner():
    from paper_2607_15478_gb300 import build, pardtw
    build.build()
    a = pardtw.Aligner(0)
    yield a
    a.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def fragment_costs(C, path, frags):
    """FP64 subsequence cost of each fragment's part of a WSDTW path."""
    out, pos = [], 0
    for r0, n in frags:
        m = pos + np.searchsorted(path[pos:, 0], r0 + n - 1, side="right")
        p = path[pos:m]
        assert p[0, 0] == r0 and p[-1, 0] == r0 + n - 1
        s = C[p[0, 0], p[0, 1]]
        for (i0, j0), (i1, j1) in zip(p[:-1], p[1:]):
            s += WEIGHTS[STEPS.index((i1 - i0, j1 - j0))] * C[i1, j1]
        out.append(s)
        pos = m
    assert pos == path.shape[0]
    return out


CASES = [(300, 360, 4, 12), (1000, 1200, 8, 12), (2000, 2500, 16, 12), (93, 120, 1, 12),
         (500, 400, 5, 12), (1001, 1300, 7, 12), (40, 60, 20, 12), (1000, 1200, 1, 12),
         (700, 800, 6, 4), (600, 650, 3, 32), (187, 300, 2, 12)]


@pytest.mark.parametrize("La,Lb,N,D", CASES)
def test_wsdtw_matches_oracle(aligner, La, Lb, N, D):
    wp = synth.warped_pair(synth.rng_for(90, La + N), La, Lb, D, knots=8, tmin=0.6, tmax=1.6)
    path, ends, total = aligner.wsdtw(dev(wp.A), dev(wp.B), N)
    cseg = aligner.wsdtw_cseg(N, Lb).cpu().numpy().astype(np.float64)
    r = ws.wsdtw(wp.A, wp.B, N)
    lens = np.array([n for _, n in r.frags], dtype=np.float64)[:, None]
    fin = np.isfinite(r.Cseg)
    np.testing.assert_array_equal(np.isfinite(cseg), fin)
    err = np.abs(cseg[fin] - r.Cseg[fin])
    tol = (1e-5 * np.abs(r.Cseg) + 1e-6 * lens * np.ones_like(r.Cseg))[fin]
    assert (err <= tol).all(), float((err - tol).max())
    np.testing.assert_array_equal(ends.cpu().numpy(), r.ends)
    assert abs(total - r.total) <= 1e-5 * abs(r.total) + 1e-6 * La
    p = path.cpu().numpy()
    if not (p.shape == r.path.shape and np.array_equal(p, r.path)):
        C = cost_matrix(wp.A, wp.B)
        got = fragment_costs(C, p, r.frags)
        ref = fragment_costs(C, r.path, r.frags)
        for k, (g, o) in enumerate(zip(got, ref)):
            assert abs(g - o) <= 1e-6 * abs(o) + 1e-7 * r.frags[k][1], (k, g, o)
    else:
        np.testing.assert_array_equal(p, r.path)


@pytest.mark.parametrize("La,N", [(400, 4), (1000, 10)])
def test_wsdtw_of_a_query_with_itself_is_the_diagonal(aligner, La, N):
    rng = np.random.default_rng(La)
    A = synth.chroma_frames(rng, La).astype(np.float32)
    path, ends, total = aligner.wsdtw(dev(A), dev(A), N)
    np.testing.assert_array_equal(path.cpu().numpy(), np.stack([np.arange(La)] * 2, axis=1))
    frs = ws.fragments(La, N)
    np.testing.assert_array_equal(ends.cpu().numpy(), [r0 + n - 1 for r0, n in frs])
    assert abs(total) <= 2 * La * 2 ** -22


def test_wsdtw_reference_too_short_is_unreachable(aligner):
    from paper_2607_15478_gb300 import pardtw
    rng = np.random.default_rng(5)
    A = synth.chroma_frames(rng, 1000).astype(np.float32)
    B = synth.chroma_frames(rng, 200).astype(np.float32)
    with pytest.raises(pardtw.PardtwError) as e:
        aligner.wsdtw(dev(A), dev(B), 10)
    assert e.value.status == pardtw.DTW_ERR_UNREACHABLE
    # the handle keeps working
    path, ends, total = aligner.wsdtw(dev(A[:300]), dev(B), 2)
    assert path.shape[0] > 0


def test_wsdtw_argument_errors(aligner):
    from paper_2607_15478_gb300 import pardtw
    A = dev(np.ones((10, 12)))
    B = dev(np.ones((10, 12)))
    path = torch.empty((9, 2), dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.dtw_wsdtw(aligner.h, A, B, 2, path, plen)  # cap < La
    assert e.value.status == pardtw.DTW_ERR_INVALID
    path = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(pardtw.PardtwError):
        pardtw.dtw_wsdtw(aligner.h, A, B, 11, path, plen)  # more fragments than rows


def test_wsdtw_long_reference_two_launch_scan(aligner):
    # more 1024-column tiles (313) than CTAs of the one-launch segment DP that
    # are resident at once (two per SM): the scan runs as two launches per
    # fragment instead; same values, ends and total as the oracle
    rng = np.random.default_rng(7)
    B = synth.chroma_frames(rng, 320000).astype(np.float32)
    A = (B[150000:150060] + 0.01 * rng.standard_normal((60, B.shape[1]))).astype(np.float32)
    path, ends, total = aligner.wsdtw(dev(A), dev(B), 3)
    r = ws.wsdtw(A, B, 3)
    np.testing.assert_array_equal(ends.cpu().numpy(), r.ends)
    assert abs(total - r.total) <= 1e-5 * abs(r.total) + 1e-6 * 60
    cseg = aligner.wsdtw_cseg(3, B.shape[0]).cpu().numpy().astype(np.float64)
    fin = np.isfinite(r.Cseg)
    np.testing.assert_array_equal(np.isfinite(cseg), fin)
    assert (np.abs(cseg[fin] - r.Cseg[fin]) <= 1e-5 * np.abs(r.Cseg[fin]) + 2e-5).all()
