"""FP64 CPU oracle for the coarse-to-fine search of the exact GCV minimiser.

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

Eq. (eq:mugcv) takes mu* as the minimiser of G over mu; the paper evaluates G
on a grid and gives no search.  This restates, step by step, the search the
library offers beside the full grid scan:

  K <= 32 or K > 1921: every grid value.
  Otherwise three levels, with s1 = ceil((K - 1) / 15) and
  s2 = min(s1, max(4, ceil(s1 / 8))):
    level 0: the grid values 0, s1, 2 s1, ... and K - 1 (at most 16);
    level 1: the incumbent k1 +- s2 m for m = 1 .. ceil(s1 / s2) - 1;
    level 2: the incumbent k2 +- m for m = 1 .. s2 - 1;
  where the incumbent after a level is the first minimiser (smallest G, then
  smallest index; NaN never wins) of all values evaluated so far, and the
  indices of a level are clamped into [0, K - 1].  At K = 256: s1 = 17, s2 = 4,
  16 + 8 + 6 = 30 evaluations.

If G is unimodal over the grid (non-increasing, then non-decreasing) the
result is the grid's first minimiser: the minimiser lies strictly between the
neighbours of the level-0 incumbent (s1 apart), level 1 samples that interval
every s2 values up to a gap of at most s2 before the known neighbours, and
level 2 the last gap.

parity: pinned by tests/test_exact_search_oracle.py (random unimodal curves
against brute force, the exact GCV curves of small problems against their full
scan, planted mistakes in the schedule rejected).
"""
from __future__ import annotations

import math

import numpy as np


def strides(K: int):
    """(s1, s2) of the three levels (K in 33 .. 1921)."""
    s1 = -(-(K - 1) // 15)
    s2 = min(s1, max(4, -(-s1 // 8)))
    return s1, s2


def searched(K: int) -> bool:
    """Whether a grid of K values is searched by levels (else scanned in full)."""
    return 32 < K <= 1921


def level_indices(level: int, K: int, incumbent: int | None = None) -> list:
    """Grid indices a level evaluates (a searched K)."""
    s1, s2 = strides(K)
    if level == 0:
        idx = list(range(0, K, s1))
        if idx[-1] != K - 1:
            idx.append(K - 1)
        return idx
    if level == 1:
        offs = [s2 * m for m in range(1, -(-s1 // s2))]
    else:
        offs = list(range(1, s2))
    out = []
    for o in offs:
        out += [min(max(incumbent - o, 0), K - 1), min(max(incumbent + o, 0), K - 1)]
    return out


def _better(v, k, best_v, best_k) -> bool:
    key = math.inf if (v is None or np.isnan(v)) else v
    return key < best_v or (key == best_v and k < best_k)


def exact_search(G_at, K: int):
    """The search over a grid of K values; G_at(k) gives G at grid index k.

    Returns (index of mu*, {index: G} of every value evaluated)."""
    seen = {}
    if not searched(K):
        for k in range(K):
            seen[k] = G_at(k)
        best_v, best_k = math.inf, None
        for k in range(K):
            if _better(seen[k], k, best_v, best_k if best_k is not None else K):
                best_v, best_k = (math.inf if np.isnan(seen[k]) else seen[k]), k
        return (best_k if best_k is not None else 0), seen
    best_v, best_k = math.inf, K
    incumbent = None
    for level in range(3):
        for k in level_indices(level, K, incumbent):
            if k not in seen:
                seen[k] = G_at(k)
            if _better(seen[k], k, best_v, best_k):
                best_v, best_k = (math.inf if np.isnan(seen[k]) else seen[k]), k
        incumbent = best_k if best_k < K else 0
    return incumbent, seen
