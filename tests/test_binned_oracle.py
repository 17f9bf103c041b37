"""Pins for the binned choice of mu (oracle/binned_oracle.py): agreement with
the plain grid scan (oracle/hobc_oracle.gcv_curve) when every bin holds one
value of a, the bin-width bound on random spectra, edge placement, and the
bracket rule on closed-form curves."""
import numpy as np

from oracle import binned_oracle as Bn
from oracle import hobc_oracle as O


def test_single_value_per_bin_reproduces_the_grid_scan():
    """One value of a per bin (repeated entries allowed): abar = a, so G_bin = G."""
    rng = np.random.default_rng(0)
    la = -11.0 + 0.0625 + 0.5 * np.arange(28)         # bin centres 0.5 decades apart: distinct bins
    a = np.repeat(10.0 ** la, 3)                      # three entries per value
    s = rng.uniform(0.5, 2.0, a.size)
    d = np.sqrt(a) * s * np.exp(1j * rng.uniform(0, 2 * np.pi, a.size))
    ghat = rng.standard_normal(a.size) + 1j * rng.standard_normal(a.size)
    mus = 10.0 ** np.linspace(-8, 0, 40)
    W, E, A = Bn.histogram(ghat, d, s)
    assert W.sum() == a.size and np.count_nonzero(W) == 28
    assert np.allclose(Bn.binned_curve(W, E, A, mus), O.gcv_curve(ghat, d, s, mus), rtol=1e-12, atol=0)


def test_entries_with_zero_smoothing_are_dropped():
    a = np.array([1e-3, 1e-1, 10.0])
    s = np.array([1.0, 0.0, 1.0])
    W, E, A = Bn.histogram(np.ones(3), np.sqrt(a), s)
    assert W.sum() == 2 and np.isclose(A.sum(), 1e-3 + 10.0)


def test_bin_width_bound_on_random_spectra():
    """G_bin / G lies in [r^-4, r^4], r = 10^((HI - LO)/NB), for a inside the range."""
    r = 10.0 ** ((Bn.HI - Bn.LO) / Bn.NB)
    rng = np.random.default_rng(1)
    mus = 10.0 ** np.linspace(-8, 0, 33)
    for trial in range(20):
        n = 500
        a = 10.0 ** rng.uniform(Bn.LO + 0.01, Bn.HI - 0.01, n)
        s = rng.uniform(0.2, 3.0, n)
        d = np.sqrt(a) * s
        ghat = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
        G = O.gcv_curve(ghat, d, s, mus)
        Gb = Bn.binned_curve(*Bn.histogram(ghat, d, s), mus)
        q = Gb / G
        assert np.all(q <= r ** 4 * (1 + 1e-12)) and np.all(q >= r ** -4 * (1 - 1e-12)), trial
    # and the bound is not vacuous: with coarse bins the ratio does move
    W, E, A = Bn.histogram(ghat, d, s, nb=4)
    assert np.max(np.abs(Bn.binned_curve(W, E, A, mus) / G - 1)) > 1e-3


def test_edges_and_clamping():
    e = Bn.bin_edges()
    assert len(e) == Bn.NB + 1 and np.isclose(e[0], 1e-12) and np.isclose(e[-1], 1e4)
    a = np.array([0.0, 1e-30, e[1] * (1 - 1e-12), e[1], e[5], e[-2], 1e4, 1e30])
    # 0, 1e-30 and just below edge 1 -> bin 0; edge 1 -> bin 1; edge 5 -> bin 5;
    # the last interior edge and anything above it -> the last bin
    assert list(Bn.bin_of(a)) == [0, 0, 0, 1, 5, Bn.NB - 1, Bn.NB - 1, Bn.NB - 1]


def _bowl(c):
    return lambda mus: (np.log10(np.asarray(mus, dtype=float)) - c) ** 2 + 1.0


def test_bracket_rule_cases():
    grid = 10.0 ** np.linspace(-8, 0, 81)               # 0.1 decades apart
    G = _bowl(-4.0)                                    # minimum at index 40
    Gbin_at = lambda k: np.abs(np.arange(81) - k).astype(float)   # binned curve with its minimum at k
    assert Bn.binned_choice(G, Gbin_at(40), grid) == (40, False, 40)
    assert Bn.binned_choice(G, Gbin_at(43), grid) == (40, False, 43)   # inside the bracket
    assert Bn.binned_choice(G, Gbin_at(60), grid) == (40, True, 60)    # minimum at the bracket edge
    assert Bn.binned_choice(G, Gbin_at(0), grid) == (40, True, 0)
    Gs = _bowl(-8.0)                                   # minimum at the grid's first value
    assert Bn.binned_choice(Gs, Gbin_at(2), grid) == (0, False, 2)     # edge that is the grid end: kept
    nan = np.full(81, np.nan)
    assert Bn.binned_choice(G, nan, grid)[2] == 0      # NaN never wins: k_hat falls to 0
    small = 10.0 ** np.linspace(-2, 0, 5)              # K = 5 < 9: the bracket is the grid
    assert Bn.binned_choice(_bowl(-1.0), np.zeros(5), small) == (2, False, 0)
