"""Seeded synthetic workloads for exact DTW / ParDTW.

This module only draws inputs. It holds none of the alignment arithmetic, so
both the CUDA path and the FP64 oracle can be fed from it without sharing any
of the method's code.

The paper evaluates on chroma features (12 dims, 23 ms hop, cosine cost;
Sec. IV) from the Chopin Mazurka recordings and measures runtime on random
feature sequences of length L (Sec. IV, Sec. VI-B, VI-C).  Neither the audio
nor the annotations are available here, so the workloads below stand in for
them:

* ``chroma_frames``: i.i.d. Dirichlet(0.3) frames, L2-normalised.  Real
  chroma is non-negative and peaky; a small Dirichlet concentration gives
  the same sparse, non-negative look.  I.i.d. frames lack the temporal
  smoothness of music.
* ``gaussian_frames``: N(0,1) frames, L2-normalised (embedding-like, D=128).
* ``warped_pair``: B is A resampled by a random monotone piecewise-linear
  time warp plus Gaussian noise, so the alignment has a known ground truth.

Seeds follow ``seed = 1000 * config + pair`` with numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

__all__ = [
    "rng_for",
    "chroma_frames",
    "gaussian_frames",
    "monotone_warp",
    "warp_sequence",
    "warped_pair",
    "WarpedPair",
    "config_pair",
    "config_batch",
    "band_training_pair",
    "CONFIGS",
]


def rng_for(config: int, pair: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with ``1000 * config + pair``."""
    return np.random.Generator(np.random.PCG64(1000 * int(config) + int(pair)))


def _l2_rows(X: np.ndarray) -> np.ndarray:
    n = np.linalg.norm(X, axis=1, keepdims=True)
    n[n == 0] = 1.0
    return X / n


def chroma_frames(rng: np.random.Generator, L: int, D: int = 12, alpha: float = 0.3) -> np.ndarray:
    """``L`` i.i.d. Dirichlet(alpha) frames of dimension ``D``, L2-normalised (float64)."""
    X = rng.dirichlet(np.full(D, alpha), size=L)
    return _l2_rows(X)


def gaussian_frames(rng: np.random.Generator, L: int, D: int = 128) -> np.ndarray:
    """``L`` i.i.d. N(0, I) frames of dimension ``D``, L2-normalised (float64)."""
    return _l2_rows(rng.standard_normal((L, D)))


def monotone_warp(rng: np.random.Generator, La: int, Lb: int, knots: int,
                  tmin: float, tmax: float) -> np.ndarray:
    """Random monotone piecewise-linear map tau: B index -> A position.

    ``tau(0) = 0``, ``tau(Lb-1) = La-1``.  ``knots`` segments; inner knot
    positions are sorted uniform draws on [0, Lb-1]; each segment's slope
    (local tempo, A frames per B frame) is drawn from U[tmin, tmax].  The
    slopes are then moved, by one affine map toward the bound on the side
    that needs it, so that their length-weighted mean is exactly
    (La-1)/(Lb-1); every slope stays inside [tmin, tmax].  (Rescaling all
    slopes by one factor and redrawing until they fit never terminates in
    practice once there are 64 or more segments.)
    """
    if Lb < 2:
        return np.zeros(Lb)
    target = (La - 1) / (Lb - 1)
    if not (tmin <= target <= tmax):
        raise ValueError(f"mean tempo {target:.4f} outside [{tmin}, {tmax}]")
    inner = np.sort(rng.uniform(0.0, Lb - 1, size=knots - 1))
    x = np.concatenate([[0.0], inner, [float(Lb - 1)]])
    seg = np.diff(x)
    s = rng.uniform(tmin, tmax, size=knots)
    m = float(np.dot(s, seg) / seg.sum())
    if m > target:
        s = tmin + (s - tmin) * ((target - tmin) / (m - tmin))
    elif m < target:
        s = tmax - (tmax - s) * ((tmax - target) / (tmax - m))
    y = np.concatenate([[0.0], np.cumsum(s * seg)])
    y *= (La - 1) / y[-1]  # remove the last rounding drift
    tau = np.interp(np.arange(Lb, dtype=np.float64), x, y)
    return np.clip(tau, 0.0, La - 1)


def warp_sequence(A: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Linear interpolation of the rows of ``A`` at fractional positions ``tau``."""
    La = A.shape[0]
    lo = np.floor(tau).astype(np.int64)
    lo = np.clip(lo, 0, La - 1)
    hi = np.minimum(lo + 1, La - 1)
    f = (tau - lo)[:, None]
    return (1.0 - f) * A[lo] + f * A[hi]


@dataclass
class WarpedPair:
    A: np.ndarray      # La x D float32, C-contiguous
    B: np.ndarray      # Lb x D float32, C-contiguous
    tau: np.ndarray    # Lb float64: ground-truth A position of each B frame


def warped_pair(rng: np.random.Generator, La: int, Lb: int, D: int = 12, *,
                kind: str = "chroma", knots: int = 8, tmin: float = 0.7,
                tmax: float = 1.4, sigma: float = 0.05) -> WarpedPair:
    """A synthetic pair: A random, B = A warped by ``monotone_warp`` plus noise.

    ``kind="chroma"``: Dirichlet(0.3) frames; noisy B frames clipped at 0.
    ``kind="gaussian"``: N(0,1) frames; no clipping.  Both are renormalised.
    """
    if kind == "chroma":
        A = chroma_frames(rng, La, D)
    elif kind == "gaussian":
        A = gaussian_frames(rng, La, D)
    else:
        raise ValueError(kind)
    tau = monotone_warp(rng, La, Lb, knots, tmin, tmax)
    B = warp_sequence(A, tau) + rng.normal(0.0, sigma, size=(Lb, D))
    if kind == "chroma":
        B = np.maximum(B, 0.0)
    B = _l2_rows(B)
    return WarpedPair(np.ascontiguousarray(A, dtype=np.float32),
                      np.ascontiguousarray(B, dtype=np.float32), tau)


# Workloads.  Index = config number used in seeds.
CONFIGS = {
    0: dict(name="pair-1000x12-vs-1200x12", La=1000, Lb=1200, D=12, kind="chroma",
            knots=8, tmin=0.7, tmax=1.4, sigma=0.05),
    1: dict(name="pair-20000x12-vs-25000x12", La=20000, Lb=25000, D=12, kind="chroma",
            knots=64, tmin=0.7, tmax=1.4, sigma=0.05),
    2: dict(name="batch-256-pairs-La-U500-8000", n_pairs=256, La_lo=500, La_hi=8000,
            ratio_lo=0.8, ratio_hi=1.25, D=12, kind="chroma", knots=8, tmin=0.7,
            tmax=1.4, sigma=0.05),
    3: dict(name="pair-40000x128-vs-48000x128", La=40000, Lb=48000, D=128, kind="gaussian",
            knots=64, tmin=0.7, tmax=1.4, sigma=0.1),
    4: dict(name="pair-100000x12-vs-U100000-130000x12", La=100000, Lb_lo=100000,
            Lb_hi=130000, D=12, kind="chroma", knots=256, tmin=0.6, tmax=1.6, sigma=0.05),
}


def config_pair(config: int, pair: int = 0, *, La: int | None = None,
                Lb: int | None = None) -> WarpedPair:
    """The seeded pair of a single-pair workload (configs 0, 1, 3, 4).

    ``La``/``Lb`` override the lengths (same recipe, smaller sizes for tests).
    """
    c = CONFIGS[config]
    rng = rng_for(config, pair)
    if config == 4 and Lb is None:
        Lb = int(rng.integers(c["Lb_lo"], c["Lb_hi"] + 1))
    La = c["La"] if La is None else La
    Lb = c["Lb"] if Lb is None else Lb
    return warped_pair(rng, La, Lb, c["D"], kind=c["kind"], knots=c["knots"],
                       tmin=c["tmin"], tmax=c["tmax"], sigma=c["sigma"])


def config_batch(config: int = 2, n_pairs: int | None = None,
                 La_range: Tuple[int, int] | None = None) -> List[WarpedPair]:
    """The seeded pairs of the batched workload (config 2): pair p uses seed 2000 + p."""
    c = CONFIGS[config]
    n = c["n_pairs"] if n_pairs is None else n_pairs
    lo, hi = (c["La_lo"], c["La_hi"]) if La_range is None else La_range
    out = []
    for p in range(n):
        rng = rng_for(config, p)
        La = int(rng.integers(lo, hi + 1))
        while True:
            Lb = int(round(La * rng.uniform(c["ratio_lo"], c["ratio_hi"])))
            if c["tmin"] <= (La - 1) / max(Lb - 1, 1) <= c["tmax"]:
                break
        out.append(warped_pair(rng, La, Lb, c["D"], kind=c["kind"], knots=c["knots"],
                               tmin=c["tmin"], tmax=c["tmax"], sigma=c["sigma"]))
    return out


def band_training_pair(k: int, La: int | None = None) -> WarpedPair:
    """Pair ``k`` of the band encoder's training set: the recipe of the long
    learned-band workload (config 4: chroma-like, tempo in [0.6, 1.6],
    noise 0.05) at La ~ U[5000, 20000], Lb = round(La * U[1.0, 1.3]), with the
    knot density of that workload (256 knots per 100000 frames, at least 8).
    Seeds 1000 * 4 + 1000 + k, disjoint from the workload's own pair."""
    c = CONFIGS[4]
    rng = rng_for(4, 1000 + k)
    if La is None:
        La = int(rng.integers(5000, 20001))
    Lb = int(round(La * rng.uniform(1.0, 1.3)))
    knots = max(8, int(round(256 * La / 100000)))
    return warped_pair(rng, La, Lb, c["D"], kind=c["kind"], knots=knots, tmin=c["tmin"],
                       tmax=c["tmax"], sigma=c["sigma"])
