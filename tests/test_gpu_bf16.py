"""BF16 cost (dtw_options.cost_precision = DTW_COST_BF16): the features are
normalised in FP32, rounded to bf16, and the dot products run on the tensor
cores with FP32 accumulation; the DP stays FP32.

Parity: the oracle applied to the cost matrix of the bf16-rounded features
(1 - a~ . b~ in FP64, a~ and b~ the normalised features rounded to bf16 exactly
as the library rounds them) must agree with the GPU under the FP32 acceptance
rule of test_gpu_parity (the remaining difference is FP32 accumulation).
Against the exact FP64 oracle the error is measured and bounded: total cost
and mean path deviation."""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import synth
from tests._parity import check_against
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


def normalise_fp32(X):
    """Rows scaled by 1 / sqrt(sum of squares), the sum accumulated in FP32 one
    fused multiply-add per feature in feature order, as the library does."""
    X = np.asarray(X, dtype=np.float32)
    ss = np.zeros(X.shape[0], dtype=np.float32)
    for d in range(X.shape[1]):
        v = X[:, d].astype(np.float64)
        ss = (v * v + ss.astype(np.float64)).astype(np.float32)
    r = np.where(ss > 0, np.float32(1.0) / np.sqrt(ss), np.float32(0.0)).astype(np.float32)
    return (X * r[:, None]).astype(np.float32)


def round_bf16(x):
    """float32 -> bf16 (round to nearest, ties to even) -> float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def bf16_frames(X):
    """The frames the tensor cores see: normalised in FP32, rounded to bf16."""
    return round_bf16(normalise_fp32(X))


def mean_deviation(p, q, La):
    """Mean over rows i of |jbar_p(i) - jbar_q(i)|, jbar = mean column matched to
    row i, linearly interpolated over rows a (2,1) step skips."""
    def jbar(path):
        s = np.zeros(La)
        n = np.zeros(La)
        for i, j in path:
            s[i] += j
            n[i] += 1
        rows = np.flatnonzero(n)
        return np.interp(np.arange(La), rows, s[rows] / n[rows])
    return float(np.mean(np.abs(jbar(p) - jbar(q))))


CASES = [(300, 360, 128), (1000, 1200, 128), (2000, 2400, 128), (700, 650, 64), (500, 600, 12)]


def assert_bf16_parity(A, B, path, total, name):
    a, b = bf16_frames(A), bf16_frames(B)
    po, to = oracle.dtw_unit(a, b)
    check_against(name, A.shape[0], B.shape[0], path.cpu().numpy(), float(total), po, to,
                  lambda q: oracle.path_cost_unit(a, b, q))


@pytest.mark.parametrize("La,Lb,D", CASES)
def test_bf16_matches_oracle_on_bf16_features(aligner, La, Lb, D):
    wp = synth.warped_pair(synth.rng_for(3, La + D), La, Lb, D, kind="gaussian", knots=8,
                           tmin=0.7, tmax=1.4, sigma=0.1)
    path, total = aligner.align(dev(wp.A), dev(wp.B), cost_precision=1)
    assert_bf16_parity(wp.A, wp.B, path, total, "bf16-features")


def test_bf16_multi_wave_matches_oracle(aligner):
    # 30000 rows swept directly: 162 strip groups of 2 x 93 rows, more than the
    # CTAs resident at once, so the persistent grid runs several waves with
    # the tensor-core cost warps (and the band map inside the DP kernel)
    from paper_2607_15478_gb300 import pardtw
    La, Lb, D = 30000, 16000, 64
    wp = synth.warped_pair(synth.rng_for(5, La), La, Lb, D, kind="gaussian", knots=64,
                           tmin=1.3, tmax=2.2, sigma=0.1)
    path, total = aligner.align(dev(wp.A), dev(wp.B), cost_precision=1,
                                transpose=pardtw.TRANSPOSE_NEVER)
    assert_bf16_parity(wp.A, wp.B, path, total, "bf16-features-multi-wave")


@pytest.mark.parametrize("La,Lb,D", CASES[:3])
def test_bf16_error_against_exact(aligner, La, Lb, D):
    wp = synth.warped_pair(synth.rng_for(3, La + D), La, Lb, D, kind="gaussian", knots=8,
                           tmin=0.7, tmax=1.4, sigma=0.1)
    path, total = aligner.align(dev(wp.A), dev(wp.B), cost_precision=1)
    p = path.cpu().numpy()
    po, to = oracle.dtw(wp.A, wp.B)
    rel = abs(total - to) / abs(to)
    assert rel <= 2e-3, rel
    # the bf16 path, costed exactly, is within 0.2% of the optimum
    tg = oracle.path_cost(wp.A, wp.B, p)
    assert (tg - to) / abs(to) <= 2e-3, (tg, to)
    assert mean_deviation(p, po, La) <= 1.0


def test_bf16_identical_sequences_diagonal(aligner):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((400, 128)).astype(np.float32)
    path, total = aligner.align(dev(A), dev(A), cost_precision=1)
    p = path.cpu().numpy()
    np.testing.assert_array_equal(p, np.stack([np.arange(400)] * 2, axis=1))
    assert abs(total) <= 400 * 2 * 2 ** -7
