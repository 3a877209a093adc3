"""The seeded synthetic inputs (CPU): the recipes the workloads and the tests
use are deterministic, have the documented shapes and distributions, and the
warps they plant are monotone with local tempos inside their bounds."""
import numpy as np
import pytest

from paper_2607_15478_gb300 import synth


def test_same_seed_same_pair():
    a = synth.config_pair(1, La=3000, Lb=3600)
    b = synth.config_pair(1, La=3000, Lb=3600)
    np.testing.assert_array_equal(a.A, b.A)
    np.testing.assert_array_equal(a.B, b.B)
    c = synth.config_pair(1, pair=1, La=3000, Lb=3600)
    assert not np.array_equal(a.A, c.A)


def test_bench_pair_shapes_and_dtype():
    wp = synth.config_pair(1)
    assert wp.A.shape == (20000, 12) and wp.B.shape == (25000, 12)
    assert wp.A.dtype == np.float32 and wp.A.flags.c_contiguous and wp.B.flags.c_contiguous


@pytest.mark.parametrize("kind,D", [("chroma", 12), ("gaussian", 128)])
def test_frames_are_unit_rows(kind, D):
    wp = synth.warped_pair(synth.rng_for(9, D), 500, 600, D, kind=kind)
    for X in (wp.A, wp.B):
        np.testing.assert_allclose(np.linalg.norm(X.astype(np.float64), axis=1), 1.0, atol=1e-6)
    if kind == "chroma":  # Dirichlet frames and clipped noisy copies: non-negative
        assert (wp.A >= 0).all() and (wp.B >= 0).all()


@pytest.mark.parametrize("La,Lb,knots,tmin,tmax", [(1000, 1200, 8, 0.7, 1.4),
                                                   (20000, 25000, 64, 0.7, 1.4),
                                                   (5000, 6000, 256, 0.6, 1.6)])
def test_planted_warp_is_monotone_within_tempo_bounds(La, Lb, knots, tmin, tmax):
    tau = synth.monotone_warp(synth.rng_for(8, La), La, Lb, knots, tmin, tmax)
    assert tau[0] == 0.0 and abs(tau[-1] - (La - 1)) < 1e-9
    d = np.diff(tau)
    assert (d >= tmin - 1e-9).all() and (d <= tmax + 1e-9).all()


def test_warp_rejects_an_impossible_mean_tempo():
    with pytest.raises(ValueError):
        synth.monotone_warp(synth.rng_for(8), 1000, 200, 8, 0.7, 1.4)


def test_batch_recipe():
    pairs = synth.config_batch(2, n_pairs=12)
    again = synth.config_batch(2, n_pairs=12)
    for p, q in zip(pairs, again):
        np.testing.assert_array_equal(p.B, q.B)
        La, Lb = p.A.shape[0], p.B.shape[0]
        assert 500 <= La <= 8000
        assert 0.7 <= (La - 1) / (Lb - 1) <= 1.4


def test_learned_band_pair_lengths():
    wp = synth.config_pair(4, La=5000, Lb=6000)
    assert wp.A.shape == (5000, 12) and wp.B.shape == (6000, 12)
    full = synth.CONFIGS[4]
    rng = synth.rng_for(4, 0)
    Lb = int(rng.integers(full["Lb_lo"], full["Lb_hi"] + 1))
    assert 100000 <= Lb <= 130000
