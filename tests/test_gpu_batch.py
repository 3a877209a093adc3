"""Batched alignment (dtw_align_many with device buffers): one normalisation
launch, one persistent DP launch over a (pair, strip group) work queue and one
batched backtrace for all pairs.  The kernels and their arithmetic are those of
the single-pair path, so every pair must equal its own dtw_align result bit
for bit, and match the FP64 oracle under the acceptance rule of
test_gpu_parity.  A device-side failure stays with its pair."""
import numpy as np
import pytest

import oracle
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


def uneven_pairs(seed, n, lo, hi, D=12):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        La = int(rng.integers(lo, hi + 1))
        Lb = int(round(La * rng.uniform(0.8, 1.25)))
        out.append(synth.warped_pair(synth.rng_for(seed, k), La, Lb, D, knots=8, tmin=0.7,
                                     tmax=1.4))
    return out


def assert_oracle(A, B, path, total):
    assert_parity(A, B, path, total, name="batch")


@pytest.mark.parametrize("R", [3, 2, 4])
def test_batch_equals_single_and_oracle(aligner, R):
    pairs = uneven_pairs(80 + R, 24, 30, 1500)
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    paths, costs, st = aligner.align_many(As, Bs, rows_per_lane=R)
    assert (st == 0).all(), st
    for k, p in enumerate(pairs):
        single, total = aligner.align(As[k], Bs[k], rows_per_lane=R)
        np.testing.assert_array_equal(paths[k].cpu().numpy(), single.cpu().numpy())
        assert float(costs[k]) == total
        assert_oracle(p.A, p.B, paths[k], float(costs[k]))


def test_batch_of_one_and_tiny_pairs(aligner):
    shapes = [(1, 1), (2, 3), (3, 2), (5, 9), (92, 94), (93, 93), (186, 187), (187, 300)]
    pairs = [synth.warped_pair(synth.rng_for(90, k), La, Lb, 12, knots=2, tmin=0.5, tmax=2.0)
             for k, (La, Lb) in enumerate(shapes)]
    for sub in ([pairs[0]], pairs):
        paths, costs, st = aligner.align_many([dev(p.A) for p in sub], [dev(p.B) for p in sub])
        assert (st == 0).all(), st
        for k, p in enumerate(sub):
            assert_oracle(p.A, p.B, paths[k], float(costs[k]))


@pytest.mark.parametrize("ns", [2, 4])
def test_batch_failure_stays_with_its_pair(aligner, ns):
    # group 0 of every pair never publishes its border: pairs with more than
    # one strip group (La > ns x 93 rows at 3 rows per lane) time out after
    # ~20 ms, single-group pairs are unaffected, and the handle keeps working
    from paper_2607_15478_gb300 import pardtw
    pairs = uneven_pairs(91, 12, 60, 900)
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    paths, costs, st = aligner.align_many(As, Bs, wait_limit_us=20000, debug_skip_publish=0,
                                          strips_per_cta=ns)
    assert any(p.A.shape[0] > ns * 93 for p in pairs)
    assert any(p.A.shape[0] <= ns * 93 for p in pairs)
    for k, p in enumerate(pairs):
        if p.A.shape[0] > ns * 93:
            assert st[k] == pardtw.DTW_ERR_TIMEOUT, (k, st[k])
        else:
            assert st[k] == 0
            assert_oracle(p.A, p.B, paths[k], float(costs[k]))
    paths, costs, st = aligner.align_many(As, Bs)
    assert (st == 0).all()
    for k, p in enumerate(pairs):
        assert_oracle(p.A, p.B, paths[k], float(costs[k]))


def test_batch_config2_shapes_equal_single(aligner):
    # the batching workload's length mix (La ~ U[500, 8000]) on 12 pairs:
    # bit-identical to one alignment after another
    pairs = synth.config_batch(2, n_pairs=12)
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    paths, costs, st = aligner.align_many(As, Bs)
    assert (st == 0).all()
    for k in range(len(pairs)):
        single, total = aligner.align(As[k], Bs[k])
        np.testing.assert_array_equal(paths[k].cpu().numpy(), single.cpu().numpy())
        assert float(costs[k]) == total


def test_planned_batch_equals_align_many_and_replays(aligner):
    # the graph-captured, autotuned plan: the same result as dtw_align_many
    # bit for bit, every replay identical, and a replay after the inputs
    # changed in place aligns the new inputs (fresh border tags, reset queue)
    pairs = uneven_pairs(95, 20, 40, 1800)
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    ref_paths, ref_costs, st = aligner.align_many(As, Bs)
    assert (st == 0).all()
    plan = aligner.plan_batch(As, Bs, autotune=True)
    R, NS, tuned = plan.info()
    assert R in (2, 3, 4) and NS in (2, 4) and tuned[(3 if NS == 4 else 0) + R - 2] > 0
    assert sum(t > 0 for t in tuned) == 5  # R 2, 3, 4 at two strips; R 2, 3 at four
    for rep in range(3):
        if rep:
            plan.run()
        paths, costs, lens = plan.results()
        for k in range(len(pairs)):
            np.testing.assert_array_equal(paths[k].cpu().numpy(), ref_paths[k].cpu().numpy())
        np.testing.assert_array_equal(costs, ref_costs)
    # new contents, same shapes: B of every pair replaced by another warp of A
    new = [synth.warped_pair(synth.rng_for(96, k), p.A.shape[0], p.B.shape[0], 12, knots=4,
                             tmin=0.7, tmax=1.4) for k, p in enumerate(pairs)]
    for k, q in enumerate(new):
        As[k].copy_(dev(q.A))
        Bs[k].copy_(dev(q.B))
    plan.run()
    paths, costs, lens = plan.results()
    for k, q in enumerate(new):
        assert_oracle(q.A, q.B, paths[k], float(costs[k]))
    ref2, c2, _ = aligner.align_many(As, Bs)
    np.testing.assert_array_equal(costs, c2)
    plan.close()


def test_planned_batch_without_autotune(aligner):
    pairs = uneven_pairs(97, 5, 100, 600)
    As = [dev(p.A) for p in pairs]
    Bs = [dev(p.B) for p in pairs]
    plan = aligner.plan_batch(As, Bs, autotune=False)
    R, NS, tuned = plan.info()
    # no autotuning: the default schedule only (3 rows per lane, four strips per CTA)
    assert R == 3 and NS == 4 and tuned[4] > 0
    assert all(t == -1.0 for k, t in enumerate(tuned) if k != 4)
    paths, costs, lens = plan.results()
    for k, p in enumerate(pairs):
        assert_oracle(p.A, p.B, paths[k], float(costs[k]))
    plan.close()
