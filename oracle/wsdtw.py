"""FP64 CPU oracle for weakly-ordered Segmental DTW (WSDTW, Sec. II-C).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by
``tests/`` and the CPU legs of ``bench.py``; the product path never imports
it.  It shares no code with the CUDA library; the cosine cost comes from this
package's own ``cost_matrix`` (FP64).

The five steps of Sec. II-C, in the paper's order and notation:

1. Break A (the query, La frames) into N fragments of nearly equal length:
   fragment k holds rows floor(k La / N) .. floor((k+1) La / N) - 1.
2. Subsequence DTW of every fragment against all of B (the reference):
   transitions (query, reference) (1,1), (1,2), (2,1) with multiplicative
   weights 1, 1, 2; the path may start at any frame of B (D_k[0][j] =
   C_k[0][j]) and end at any frame of B.
3. C_seg[k][j] = D_k[last row][j], the best subsequence path score of
   fragment k ending at frame j of B.
4. Segment-level DP with transitions (0, 1) (a skip, weight 0) and
   (1, delta_k) (a match):
       D_seg[k][j] = min(D_seg[k][j-1], D_seg[k-1][j - delta_k] + C_seg[k][j]),
   delta_k the shortest match of fragment k (half its length, Sec. II-C);
   its backtrace gives the end frame e_k of every fragment, e_k >= e_{k-1} +
   delta_k.
5. Backtrace of every fragment from (last row, e_k) to its first row; the
   WSDTW alignment is the concatenation of the fragment paths.

Readings of points the paper leaves open:
* Row 0 of a fragment: D_k[0][j] = C_k[0][j] (unweighted start, any j);
  no path enters a fragment below its first row (a (2,1) step from row -1
  does not exist).
* delta_k = floor(len_k / 2) for the fragment the match enters (the paper
  writes L_A / (2N) for equal fragments).
* D_seg[0][j] = min(D_seg[0][j-1], C_seg[0][j]) (the first fragment has no
  predecessor); D_seg[k][j] = +inf where j - delta_k < 0.
* Ties: in the frame-level DP, candidates in the order (1,1), (1,2), (2,1),
  a later one only when strictly smaller (as in the DTW of Sec. V); in the
  segment DP a match replaces the skip only when strictly smaller, so every
  fragment ends at the earliest of equally good frames.
* The result is the minimal D_seg[N-1][Lb-1]; +inf (B too short for the
  fragments) is an error.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from . import cost_matrix

INF = np.inf
W11, W12, W21 = 1.0, 1.0, 2.0   # (query, reference) steps (1,1), (1,2), (2,1)


def fragments(La: int, N: int) -> List[Tuple[int, int]]:
    """(first row, length) of the N fragments of a query of La frames (step 1)."""
    if not (1 <= N <= La):
        raise ValueError("need 1 <= N <= La")
    b = [(k * La) // N for k in range(N + 1)]
    return [(b[k], b[k + 1] - b[k]) for k in range(N)]


def subseq_dtw(C: np.ndarray):
    """Step 2 on one fragment's cost matrix C (len x Lb, FP64): cumulative
    cost D and step codes (0 (1,1), 1 (1,2), 2 (2,1), 3 start)."""
    C = np.asarray(C, dtype=np.float64)
    n, Lb = C.shape
    D = np.full((n, Lb), INF)
    code = np.full((n, Lb), 3, dtype=np.int8)
    D[0] = C[0]
    for i in range(1, n):
        c0 = np.full(Lb, INF)
        c1 = np.full(Lb, INF)
        c2 = np.full(Lb, INF)
        c0[1:] = D[i - 1, :-1] + W11 * C[i, 1:]
        c1[2:] = D[i - 1, :-2] + W12 * C[i, 2:]
        if i >= 2:
            c2[1:] = D[i - 2, :-1] + W21 * C[i, 1:]
        m = c0.copy()
        k = np.zeros(Lb, dtype=np.int8)
        s = c1 < m
        m[s], k[s] = c1[s], 1
        s = c2 < m
        m[s], k[s] = c2[s], 2
        D[i] = m
        code[i] = np.where(np.isfinite(m), k, 3)
    return D, code


def subseq_backtrace(code: np.ndarray, j_end: int) -> np.ndarray:
    """Step 5 on one fragment: the path from (last row, j_end) back to row 0,
    returned ascending as (row in the fragment, j) pairs."""
    i, j = code.shape[0] - 1, int(j_end)
    out = [(i, j)]
    steps = ((1, 1), (1, 2), (2, 1))
    while i > 0:
        c = int(code[i, j])
        if c == 3:
            raise ValueError("backtrace left the reachable cells")
        di, dj = steps[c]
        i, j = i - di, j - dj
        out.append((i, j))
    return np.array(out[::-1], dtype=np.int32)


def segment_dp(Cseg: np.ndarray, deltas) -> Tuple[np.ndarray, np.ndarray, float]:
    """Step 4: D_seg, the end frames e_k and the total D_seg[N-1][Lb-1]."""
    Cseg = np.asarray(Cseg, dtype=np.float64)
    N, Lb = Cseg.shape
    Dseg = np.full((N, Lb), INF)
    arg = np.full((N, Lb), -1, dtype=np.int64)
    for k in range(N):
        best, at = INF, -1
        for j in range(Lb):
            if k == 0:
                match = Cseg[0, j]
            else:
                jp = j - deltas[k]
                match = Dseg[k - 1, jp] + Cseg[k, j] if jp >= 0 else INF
            if match < best:
                best, at = match, j
            Dseg[k, j], arg[k, j] = best, at
    total = float(Dseg[N - 1, Lb - 1])
    if not np.isfinite(total):
        raise ValueError("B is too short for the fragments")
    ends = np.zeros(N, dtype=np.int64)
    ends[N - 1] = arg[N - 1, Lb - 1]
    for k in range(N - 1, 0, -1):
        ends[k - 1] = arg[k - 1, ends[k] - deltas[k]]
    return Dseg, ends, total


@dataclass
class WsdtwResult:
    path: np.ndarray      # (n, 2) int32, (row of A, frame of B), fragment by fragment
    ends: np.ndarray      # end frame of B of every fragment
    total: float          # D_seg[N-1][Lb-1]
    Cseg: np.ndarray      # N x Lb subsequence path scores
    frags: list           # (first row, length) per fragment


def wsdtw(A, B, N: int) -> WsdtwResult:
    """WSDTW of query A against reference B with N fragments (Sec. II-C)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    La, Lb = A.shape[0], B.shape[0]
    frs = fragments(La, N)
    Cseg = np.empty((N, Lb))
    codes = []
    for k, (r0, n) in enumerate(frs):
        D, code = subseq_dtw(cost_matrix(A[r0:r0 + n], B))
        Cseg[k] = D[-1]
        codes.append(code)
    deltas = [n // 2 for _, n in frs]
    _, ends, total = segment_dp(Cseg, deltas)
    parts = []
    for k, (r0, n) in enumerate(frs):
        p = subseq_backtrace(codes[k], ends[k])
        p[:, 0] += r0
        parts.append(p)
    return WsdtwResult(np.concatenate(parts), ends, total, Cseg, frs)
