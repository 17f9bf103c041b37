"""FP64 CPU oracle for the continuous refinement of mu* (reading R15).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

Eq. (eq:mugcv) defines mu* as the minimiser of the GCV functional G over all
mu > 0; the grid argmin k only approximates it.  The refinement searches
log10 mu inside the bracket of the grid neighbours of k, with the grid value
itself as the incumbent:

    lo, mid, hi = log10 mu_{max(k-1, 0)}, log10 mu_k, log10 mu_{min(k+1, K-1)}
    every round: nine points, four equal steps from lo to mid and four from
      mid to hi (point 4 is the incumbent, evaluated at the incumbent's own mu);
      j = the first minimiser of G over the nine points;
      lo, mid, hi = x_{max(j-1, 0)}, x_j, x_{min(j+1, 8)}
    after ROUNDS rounds mu* is the last round's minimiser.

Each round shrinks the bracket about four times (the two steps around the
minimiser), so five rounds leave about 1/1000 of the two grid steps.  Each
evaluation point is a value of the plan's precision (the method evaluates G
at that value); the oracle rounds its own points the same way and evaluates G
in FP64 from the definition (hobc_oracle.gcv_curve).

parity status: pinned by tests/test_refine_oracle.py (the closed-form
minimiser of a two-entry spectrum, never worse than the grid value, bracket
containment, the K = 1 case).
"""
from __future__ import annotations

import numpy as np

from oracle import hobc_oracle as O

POINTS = 9
ROUNDS = 5


def round_points(lo: float, mid: float, hi: float) -> np.ndarray:
    """log10 of the nine evaluation points of one round."""
    x = np.empty(POINTS)
    half = POINTS // 2
    for j in range(POINTS):
        if j <= half:
            x[j] = lo + (mid - lo) * j / half
        else:
            x[j] = mid + (hi - mid) * (j - half) / half
    return x


def first_argmin(G: np.ndarray) -> int:
    """Lowest index of the smallest value; NaN never wins (all NaN -> the incumbent)."""
    key = np.where(np.isnan(G), np.inf, G)
    if np.all(np.isinf(key)) and np.all(np.isnan(G)):
        return POINTS // 2
    return int(np.argmin(key))


def refine(ghat, d, s, mus, k: int, rounds: int = ROUNDS, point_dtype=np.float64):
    """mu* and G(mu*) by the bracket refinement around grid index k.

    ghat, d, s: full spectra (any shape), mus: the grid (increasing), k: its
    argmin.  point_dtype: the precision the evaluation points are stored in
    (float32 for an FP32 plan).  Returns (mu, G, history) with history the
    (points, G values, chosen index) of every round.
    """
    mus = np.asarray(mus, dtype=np.float64)
    K = len(mus)
    lg = np.log10(mus)
    lo, mid, hi = lg[max(k - 1, 0)], lg[k], lg[min(k + 1, K - 1)]
    mid_mu = float(np.asarray(mus[k], dtype=point_dtype))
    history = []
    mu_best, G_best = mid_mu, np.nan
    for _ in range(rounds):
        x = round_points(lo, mid, hi)
        pts = 10.0 ** x
        pts[POINTS // 2] = mid_mu
        pts = pts.astype(point_dtype).astype(np.float64)
        G = O.gcv_curve(ghat, d, s, pts)
        j = first_argmin(G)
        history.append((pts, G, j))
        lo, mid, hi = x[max(j - 1, 0)], x[j], x[min(j + 1, POINTS - 1)]
        mid_mu = pts[j]
        mu_best, G_best = pts[j], G[j]
    return mu_best, G_best, history


def two_entry_minimiser(e1: float, e2: float, A: float) -> float:
    """Closed-form minimiser of G for the spectrum of two entries with
    a = 0 (energy e1) and a = A (energy e2), unit weights, e2 > e1:

      G(mu) = (e1 (A + mu)^2 + e2 mu^2) / (A + 2 mu)^2   (after multiplying
      numerator and denominator by mu^2 (A + mu)^2); dG/dmu = 0 gives
      mu (e2 - e1) = e1 A.
    """
    return e1 * A / (e2 - e1)
