"""Pins of the refinement oracle (oracle/refine_oracle.py) against closed forms
and brute force, independent of the oracle's own search."""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from oracle import refine_oracle as R


def _two_entry(e1, e2, A):
    ghat = np.sqrt(np.array([e1, e2]))
    d = np.array([0.0, np.sqrt(A)])
    s = np.ones(2)
    return ghat, d, s


def test_two_entry_closed_form_matches_the_functional():
    """The closed-form minimiser is a stationary point of G as the oracle defines it."""
    e1, e2, A = 0.3, 1.7, 2e-3
    ghat, d, s = _two_entry(e1, e2, A)
    mu = R.two_entry_minimiser(e1, e2, A)
    eps = 1e-6 * mu
    G = O.gcv_curve(ghat, d, s, np.array([mu - eps, mu, mu + eps]))
    assert G[1] < G[0] and G[1] < G[2]
    # G(mu) by the reduced formula of the docstring
    Gr = (e1 * (A + mu) ** 2 + e2 * mu ** 2) / (A + 2 * mu) ** 2
    assert abs(G[1] - Gr) <= 1e-12 * Gr


@pytest.mark.parametrize("e1,e2,A", [(0.3, 1.7, 2e-3), (1.0, 1.05, 1e-5), (0.01, 5.0, 0.3), (2.0, 9.0, 7e-7)])
@pytest.mark.parametrize("K", [17, 64])
def test_refinement_reaches_the_closed_form_minimiser(e1, e2, A, K):
    ghat, d, s = _two_entry(e1, e2, A)
    mus = 10.0 ** np.linspace(-8, 1, K)
    mu_star = R.two_entry_minimiser(e1, e2, A)
    k = O.gcv_argmin(O.gcv_curve(ghat, d, s, mus))
    mu, G, hist = R.refine(ghat, d, s, mus, k)
    h = np.log10(mus[1]) - np.log10(mus[0])
    # within one final step of the minimiser: h / 4^ROUNDS
    assert abs(np.log10(mu) - np.log10(mu_star)) <= h / 4 ** R.ROUNDS * (1 + 1e-9)
    assert G <= O.gcv_curve(ghat, d, s, mus).min()
    assert len(hist) == R.ROUNDS


def test_rounds_shrink_the_bracket_and_keep_the_incumbent():
    rng = np.random.default_rng(3)
    ghat = rng.standard_normal(400)
    d = np.exp(-rng.uniform(0, 12, 400))
    s = np.ones(400)
    mus = 10.0 ** np.linspace(-8, 0, 33)
    k = O.gcv_argmin(O.gcv_curve(ghat, d, s, mus))
    mu, G, hist = R.refine(ghat, d, s, mus, k)
    widths = [np.log10(p[-1]) - np.log10(p[0]) for p, _, _ in hist]
    for a, b in zip(widths, widths[1:]):
        assert b <= a / 2 + 1e-12
    for (p0, G0, j0), (p1, G1, j1) in zip(hist, hist[1:]):
        assert p1[R.POINTS // 2] == p0[j0]               # the incumbent is re-evaluated
        assert G1.min() <= G0[j0] * (1 + 1e-14)          # never worse than the incumbent


@pytest.mark.parametrize("seed", range(6))
def test_refinement_matches_brute_force_inside_the_bracket(seed):
    """G at the refined mu is within the final resolution of the minimum of G
    over 20001 log-spaced points of the bracket (brute force)."""
    rng = np.random.default_rng(seed)
    n = 300
    ghat = rng.standard_normal(n) * np.exp(-rng.uniform(0, 4, n))
    d = np.exp(-rng.uniform(0, 10, n))
    s = np.where(rng.random(n) < 0.5, 1.0, rng.uniform(0.1, 2, n))
    mus = 10.0 ** np.linspace(-8, 0, 41)
    Gg = O.gcv_curve(ghat, d, s, mus)
    k = O.gcv_argmin(Gg)
    mu, G, _ = R.refine(ghat, d, s, mus, k)
    lo, hi = mus[max(k - 1, 0)], mus[min(k + 1, len(mus) - 1)]
    assert lo <= mu <= hi
    fine = 10.0 ** np.linspace(np.log10(lo), np.log10(hi), 20001)
    Gb = O.gcv_curve(ghat, d, s, fine)
    assert G <= Gg[k]
    # the brute-force step is 1/10000 of the bracket, finer than the search's
    # 1/2048; G is flat to second order at an interior minimum
    assert G <= Gb.min() * (1 + 1e-6)


def test_single_grid_value_and_float32_points():
    ghat, d, s = _two_entry(0.3, 1.7, 2e-3)
    mu, G, hist = R.refine(ghat, d, s, np.array([1e-3]), 0)
    assert mu == 1e-3 or mu == float(np.float64(1e-3))
    mus = 10.0 ** np.linspace(-6, 0, 25)
    k = O.gcv_argmin(O.gcv_curve(ghat, d, s, mus))
    mu32, _, hist32 = R.refine(ghat, d, s, mus, k, point_dtype=np.float32)
    for p, _, _ in hist32:
        assert np.all(p.astype(np.float32).astype(np.float64) == p)
    assert mu32 == float(np.float32(mu32))


def test_nan_never_wins():
    G = np.array([np.nan, 3.0, 2.0, np.nan, 2.0, 5, 6, 7, 8])
    assert R.first_argmin(G) == 2
    assert R.first_argmin(np.full(9, np.nan)) == R.POINTS // 2


def test_first_round_spans_the_grid_neighbours_in_equal_steps():
    """Round 0 evaluates mu_{k-1} and mu_{k+1} at its ends and mu_k itself in
    the middle, four equal log10 steps on each side."""
    ghat, d, s = _two_entry(0.3, 1.7, 2e-3)
    mus = 10.0 ** np.array([-7.0, -5.5, -4.0, -3.2, -2.0, -1.0])
    k = 3
    _, _, hist = R.refine(ghat, d, s, mus, k)
    p = hist[0][0]
    assert p[R.POINTS // 2] == mus[k]
    assert np.allclose(np.log10(p[[0, -1]]), np.log10(mus[[k - 1, k + 1]]), rtol=0, atol=1e-13)
    x = np.log10(p)
    assert np.allclose(np.diff(x[:5]), (np.log10(mus[k]) - np.log10(mus[k - 1])) / 4, rtol=0, atol=1e-12)
    assert np.allclose(np.diff(x[4:]), (np.log10(mus[k + 1]) - np.log10(mus[k])) / 4, rtol=0, atol=1e-12)
