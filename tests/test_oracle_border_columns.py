"""Pins for the border columns of the oracle's T_X (the polynomials p, q, L1, L2, Q1, Q2).

The transform-free pins cannot see these columns: A_X is the same for every choice
of border polynomials that spans the preserved space.  G of Eq. (eq:gcv2) and the
spectrum ghat do depend on them, so they are pinned here against what the paper's
definitions fix on their own:

  * a hand-worked fixture at n = 8 (tests/golden/border_columns_n8.txt), derived in
    its header from Eq. (eq:ART), (eq:points), (eq:ints), (eq:pointn), (eq:intn) and
    readings R6, R16, R17;
  * at any n, the shape each definition states: q~ = (b - x)^2 is a quadratic in the
    sample index with a double root at the last sample (Sec. 3.1, 3.2: b is the last
    grid point), p is linear with a root there (Eq. (eq:ART)), L1 has simple roots at
    the last two samples and L2 a simple and a double one (reading R6), Q1 and Q2 have
    roots of order 2 and 4 at the last sample (readings R16, R17);
  * unit 2-norm and the right columns being the flips of the left ones.

The columns are read from the oracle's assembled T_X, so a mistake in any helper
that feeds it shows here.  CPU only.
"""
import os

import numpy as np
import pytest

from oracle import hobc_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
DOUBLE_BORDER = ("S3", "C4", "F4")


def _golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "border_columns_n8.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                rows[(line[0], line[1])] = np.array([float(v) for v in line[2:]])
    return rows


def _left_columns(fam, n):
    """Left border columns (first, second) and right ones (last, second last) of T_X."""
    T = O.transform_matrix(fam, n)
    if fam in DOUBLE_BORDER:
        return [T[:, 0], T[:, 1]], [T[:, n - 1], T[:, n - 2]]
    return [T[:, 0]], [T[:, n - 1]]


def _unit(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3", "C4", "F4"])
def test_border_columns_equal_the_hand_worked_fixture(fam):
    gold = _golden()
    left, right = _left_columns(fam, 8)
    names = ["left1", "left2"][:len(left)]
    for col, rcol, name in zip(left, right, names):
        want = _unit(gold[(fam, name)])
        assert np.abs(col - want).max() < 1e-14, (fam, name)
        assert np.abs(rcol - want[::-1]).max() < 1e-14, (fam, name)    # J times the left column


def _poly_fit_residual(v, deg):
    """Largest residual of the least-squares fit of v by a polynomial of degree deg in
    the sample index, relative to max |v| (0 up to rounding iff v is such a polynomial)."""
    k = np.arange(len(v), dtype=np.float64) / len(v)
    V = np.vander(k, deg + 1)
    c, *_ = np.linalg.lstsq(V, v, rcond=None)
    return np.abs(V @ c - v).max() / np.abs(v).max()


def _root_order_at_end(v, deg):
    """Order of the root at the last sample of v, read as a polynomial of degree deg in
    u = (index of the last sample) - (sample index): the number of vanishing
    low-order coefficients in u, each to 1e-9 of the largest."""
    u = (len(v) - 1 - np.arange(len(v), dtype=np.float64)) / len(v)
    c = np.polynomial.polynomial.polyfit(u, v, deg)
    big = np.abs(c).max()
    order = 0
    for ci in c:
        if abs(ci) > 1e-9 * big:
            break
        order += 1
    return order


@pytest.mark.parametrize("n", [8, 12, 33, 256])
@pytest.mark.parametrize("fam", ["S", "C", "F"])
def test_single_border_column_shape(fam, n):
    """p: linear, root at the last sample (Eq. (eq:ART)); q: quadratic with a double
    root at the last sample, because b = x_{n-1} in Eq. (eq:ints) and (eq:intn)."""
    (col,), (rcol,) = _left_columns(fam, n)
    deg = 1 if fam == "S" else 2
    assert abs(np.linalg.norm(col) - 1.0) < 1e-14
    assert np.abs(rcol - col[::-1]).max() < 1e-15
    assert np.abs(col.imag).max() == 0 if np.iscomplexobj(col) else True
    col = col.real
    assert _poly_fit_residual(col, deg) < 1e-10
    assert _poly_fit_residual(col, deg - 1) > 1e-3          # exactly that degree
    assert _root_order_at_end(col, deg) == deg
    assert np.all(col[:-1] > 0)                             # no other root on the grid


@pytest.mark.parametrize("n", [8, 12, 33, 256])
@pytest.mark.parametrize("fam", DOUBLE_BORDER)
def test_double_border_column_shapes(fam, n):
    """S3 (reading R6): L1 = (x_{N+1}-x)(x_{N+2}-x) has simple roots at the last two
    samples, L2 = L1 (x_{N+2}-x) one simple and one double root; C4, F4 (readings R16,
    R17): Q1 = (b-x)^2, Q2 = (b-x)^4 with b the last sample."""
    (c1, c2), (r1, r2) = _left_columns(fam, n)
    c1, c2 = np.real(c1), np.real(c2)
    for c, r in ((c1, r1), (c2, r2)):
        assert abs(np.linalg.norm(c) - 1.0) < 1e-14
        assert np.abs(np.real(r) - c[::-1]).max() < 1e-15
    if fam == "S3":
        assert _poly_fit_residual(c1, 2) < 1e-10 and _poly_fit_residual(c1, 1) > 1e-3
        assert _poly_fit_residual(c2, 3) < 1e-10 and _poly_fit_residual(c2, 2) > 1e-3
        assert abs(c1[-1]) < 1e-15 and abs(c1[-2]) < 1e-15 and np.all(c1[:-2] > 0)
        assert abs(c2[-1]) < 1e-15 and abs(c2[-2]) < 1e-15 and np.all(c2[:-2] > 0)
        # the double root of L2 is at the last sample: L2 / L1 is linear with a root there
        ratio = c2[:-2] / c1[:-2]
        k = np.arange(n - 2, dtype=np.float64)
        slope, icpt = np.polyfit(k, ratio, 1)
        assert np.abs(slope * k + icpt - ratio).max() < 1e-10 * ratio.max()
        assert abs((slope * (n - 1) + icpt) / ratio.max()) < 1e-10
    else:
        assert _poly_fit_residual(c1, 2) < 1e-10 and _poly_fit_residual(c1, 1) > 1e-3
        assert _poly_fit_residual(c2, 4) < 1e-10 and _poly_fit_residual(c2, 3) > 1e-3
        assert _root_order_at_end(c1, 2) == 2 and _root_order_at_end(c2, 4) == 4
        assert np.all(c1[:-1] > 0) and np.all(c2[:-1] > 0)
        # Q2 is the square of Q1 up to scale
        assert np.abs(_unit(c1 ** 2) - c2).max() < 1e-13


def test_pins_catch_planted_border_polynomials(monkeypatch):
    """Plant plausible wrong border polynomials in the oracle (each still of the right
    degree and still vanishing at b) and check that a pin above rejects every one."""

    def rejected(fam, n=8):
        try:
            test_border_columns_equal_the_hand_worked_fixture(fam)
        except AssertionError:
            pass
        else:
            return False
        try:
            if fam in DOUBLE_BORDER:
                test_double_border_column_shapes(fam, 12)
            else:
                test_single_border_column_shape(fam, 12)
        except AssertionError:
            return True
        return False

    orig_border = O.border_vector

    def wrong_q(f, m):                       # (x - a + 0.3)(b - x): quadratic, one root at b
        if f == "S":
            return orig_border(f, m)
        x, a, b = O.extended_grid(f, m)
        v = (x - a + 0.3) * (b - x)
        return v / np.linalg.norm(v)
    monkeypatch.setattr(O, "border_vector", wrong_q)
    assert rejected("C") and rejected("F")
    monkeypatch.setattr(O, "border_vector", orig_border)

    def wrong_p(f, m):                       # p on [0, pi] with its root at the wrong end
        if f != "S":
            return orig_border(f, m)
        v = np.arange(m, dtype=np.float64) + 1.0
        return v / np.linalg.norm(v)
    monkeypatch.setattr(O, "border_vector", wrong_p)
    assert rejected("S")
    monkeypatch.setattr(O, "border_vector", orig_border)

    orig_cubic = O.cubic_border_columns

    def wrong_cubic(m):                      # L1 with its roots at x_N, x_{N+2}
        N = m - 4
        x = np.arange(-1, N + 3) * np.pi / (N + 1)
        xa, xb = N * np.pi / (N + 1), (N + 2) * np.pi / (N + 1)
        L1 = (xa - x) * (xb - x)
        L2 = L1 * (xb - x)
        return L1 / np.linalg.norm(L1), L2 / np.linalg.norm(L2)
    monkeypatch.setattr(O, "cubic_border_columns", wrong_cubic)
    assert rejected("S3")
    monkeypatch.setattr(O, "cubic_border_columns", orig_cubic)

    orig_quartic = O.quartic_border_columns

    def wrong_quartic(m, grid=None):         # Q1 = (x - a + 0.3)(b - x), Q2 = Q1^2
        x, a, b = (grid or O.quartic_grid)(m)
        Q1 = (x - a + 0.3) * (b - x)
        Q2 = Q1 ** 2
        return Q1 / np.linalg.norm(Q1), Q2 / np.linalg.norm(Q2)
    monkeypatch.setattr(O, "quartic_border_columns", wrong_quartic)
    assert rejected("C4") and rejected("F4")
    monkeypatch.setattr(O, "quartic_border_columns", orig_quartic)

    # the unplanted oracle passes both pins
    for fam in ("S", "C", "F", "S3", "C4", "F4"):
        assert not rejected(fam)
