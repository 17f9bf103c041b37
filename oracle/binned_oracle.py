"""FP64 CPU oracle for the binned choice of mu (not part of the paper).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

The GCV functional of Eq. (eq:gcv2) depends on a spectral entry only through
a = |d|^2 / |s|^2 and |ghat|^2 (entries with s = 0 contribute nothing):
    G(mu) = sum e_i / (a_i + mu)^2 / (sum w_i / (a_i + mu))^2
(after dividing numerator and denominator by mu^2).  The binned choice groups
the entries by a into NB bins between 10^LO and 10^HI (equal widths in log10 a,
values outside go to the end bins), keeps per bin the count W, the energy
E = sum |ghat|^2 and the sum A of a, and evaluates
    G_bin(mu) = sum_b E_b / (abar_b + mu)^2 / (sum_b W_b / (abar_b + mu))^2,
abar_b = A_b / W_b, on the grid.  Its argmin k_hat only places a bracket: the
exact G is then evaluated on the min(9, K) grid values around k_hat; mu* is the
bracket's minimiser unless that sits on a bracket edge that is not an end of
the grid, in which case the full grid is scanned.

Error bound: inside the range, a and abar share a bin, so (a + mu)/(abar + mu)
lies in [1/r, r] with r = 10^((HI - LO)/NB); hence each sum is within a factor
r (denominator) or r^2 (numerator) and G_bin / G lies in [r^-4, r^4].

parity status: pinned by tests/test_binned_oracle.py (exact agreement with
the grid scan when every bin holds a single value of a, the bound above on
random spectra, edge placement, the bracket rule on closed-form curves).
"""
from __future__ import annotations

import numpy as np

NB = 128
LO = -12.0
HI = 4.0


def bin_edges(nb: int = NB, lo: float = LO, hi: float = HI) -> np.ndarray:
    """The nb + 1 edges 10^(lo + b (hi - lo) / nb), b = 0..nb."""
    return 10.0 ** (lo + np.arange(nb + 1) * (hi - lo) / nb)


def a_values(d: np.ndarray, s: np.ndarray):
    """(mask of entries with s != 0, a = |d|^2 / |s|^2 on them)."""
    m = np.abs(s) > 0
    return m, np.abs(d[m]) ** 2 / np.abs(s[m]) ** 2


def bin_of(a: np.ndarray, nb: int = NB, lo: float = LO, hi: float = HI) -> np.ndarray:
    """Bin of each a: the number of interior edges <= a (0 .. nb - 1)."""
    return np.searchsorted(bin_edges(nb, lo, hi)[1:-1], a, side="right")


def histogram(ghat: np.ndarray, d: np.ndarray, s: np.ndarray, nb: int = NB, lo: float = LO, hi: float = HI):
    """Per-bin count W, energy E = sum |ghat|^2 and sum A of a (full spectra of
    any shape)."""
    m, a = a_values(d.ravel(), s.ravel())
    e = np.abs(ghat.ravel()[m]) ** 2
    b = bin_of(a, nb, lo, hi)
    W = np.bincount(b, minlength=nb).astype(float)
    E = np.bincount(b, weights=e, minlength=nb)
    A = np.bincount(b, weights=a, minlength=nb)
    return W, E, A


def binned_curve(W: np.ndarray, E: np.ndarray, A: np.ndarray, mus: np.ndarray) -> np.ndarray:
    """G_bin(mu) on the grid from the bin sums (empty bins skipped)."""
    k = W > 0
    abar = A[k] / W[k]
    out = np.empty(len(mus))
    for j, mu in enumerate(mus):
        num = np.sum(E[k] / (abar + mu) ** 2)
        den = np.sum(W[k] / (abar + mu))
        out[j] = num / den ** 2
    return out


def first_argmin(G: np.ndarray) -> int:
    """Index of the smallest value, lowest on ties; NaN never wins."""
    return int(np.argmin(np.where(np.isnan(G), np.inf, G)))


def binned_choice(G_at, Gbin: np.ndarray, grid: np.ndarray, width: int = 9):
    """(grid index of mu*, fell back?, k_hat).  G_at(mus) is the exact GCV."""
    K = len(grid)
    k_hat = first_argmin(Gbin)
    span = min(width, K)
    k0 = max(0, min(k_hat - span // 2, K - span))
    am = first_argmin(G_at(grid[k0:k0 + span]))
    kmin = k0 + am
    edge = (am == 0 and kmin > 0) or (am == span - 1 and kmin < K - 1)
    if edge:
        return first_argmin(G_at(grid)), True, k_hat
    return kmin, False, k_hat
