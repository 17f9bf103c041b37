"""The truncation bound of the GCV curve by bin expansion, checked in FP64 on
the CPU (no GPU, no library call).

G(mu) of Eq. (eq:gcv2) is num(mu) / den(mu)^2 with num = sum e/(a+mu)^2 and
den = sum w/(a+mu), a = |d|^2/|s|^2.  The expansion (hobc_plan_set_gcv_mode,
include/hobc.h) groups the entries into 256 bins uniform in log a over
[1e-3 mu_min, 1e3 mu_max), one key below and one above, and replaces each
term by its power series in the entry's coordinate inside its key, cut after
the 7th power:
  inner bin of centre c:  1/(a+mu)^k = (c+mu)^-k (1 + rho u)^-k,
                          u = a/c - 1, rho = c/(c+mu)
  below (a < a_lo):       1/(a+mu)^k = mu^-k (1 + (a_lo/mu) u)^-k,  u = a/a_lo
  above (a >= a_hi):      1/(a+mu)^k = a^-k (1 + (mu/a_hi) u)^-k,   u = a_hi/a
so a key contributes through the moments sum e u^p and sum w u^p, p <= 7.
With U = sqrt(r) - 1 the bins' half-ratio, |rho u| <= U, and the remainder of
(1+y)^-2 after p = 7 is at most 9 U^8/(1-U)^2 relative (that of (1+y)^-1 is
smaller): the bound the library reports, 3.27e-9 for the grid [1e-8, 1].

Here the series is evaluated in FP64 from its definition above, term by
term against the exact sums: on random spectra reaching every key, and on
entries placed at bin edges where |u| = U (the worst case).  Dropping the
p = 7 term breaks the bound on the edge entries, so the check sees the
order of the cut."""
import numpy as np
import pytest

BINS = 256


def geometry(mu_lo, mu_hi):
    decades = np.log10(mu_hi / mu_lo) + 6.0
    r = 10.0 ** (decades / BINS)
    a_lo = 1e-3 * mu_lo
    return r, a_lo, a_lo * r ** BINS


def bound(mu_lo, mu_hi):
    r, _, _ = geometry(mu_lo, mu_hi)
    U = np.sqrt(r) - 1.0
    return max(9.0 * U ** 8 / (1.0 - U) ** 2, 9.0 * 1e-3 ** 8)


def exact_sums(a, e, w, mus):
    s = a[None, :] + mus[:, None]
    return (e[None, :] / s ** 2).sum(axis=1), (w[None, :] / s).sum(axis=1)


def expansion_sums(a, e, w, mus, mu_lo, mu_hi, P=8):
    """num and den at every mu from per-key moments (P terms of each series)."""
    r, a_lo, a_hi = geometry(mu_lo, mu_hi)
    small, large = a < a_lo, a >= a_hi
    inner = ~(small | large)
    b = np.clip(np.floor(np.log(np.where(inner, a, a_lo) / a_lo) / np.log(r)).astype(int), 0, BINS - 1)
    lower = a_lo * r ** b.astype(float)
    b = np.where(inner & (a < lower), b - 1, b)                       # the log may be one bin off
    b = np.where(inner & (a >= a_lo * r ** (b + 1.0)), b + 1, b)
    centre = a_lo * r ** (b + 0.5)
    key = np.where(small, 0, np.where(large, BINS + 1, 1 + b))
    u = np.where(small, a / a_lo, np.where(large, a_hi / a, a / centre - 1.0))
    ee = np.where(large, e / a ** 2, e)
    ww = np.where(large, w / a, w)
    p = np.arange(P)
    E = np.zeros((BINS + 2, P))
    W = np.zeros((BINS + 2, P))
    np.add.at(E, key, ee[:, None] * u[:, None] ** p)
    np.add.at(W, key, ww[:, None] * u[:, None] ** p)
    centres = a_lo * r ** (np.arange(BINS) + 0.5)
    num = np.zeros(len(mus))
    den = np.zeros(len(mus))
    for j, mu in enumerate(mus):
        x = np.concatenate([[-a_lo / mu], -centres / (centres + mu), [-mu / a_hi]])
        sn = np.concatenate([[mu ** -2.0], (centres + mu) ** -2.0, [1.0]])
        sd = np.concatenate([[1.0 / mu], 1.0 / (centres + mu), [1.0]])
        xp = x[:, None] ** p
        num[j] = (sn * ((p + 1) * E * xp).sum(axis=1)).sum()
        den[j] = (sd * (W * xp).sum(axis=1)).sum()
    return num, den


def rel(x, y):
    return np.abs(x - y) / np.abs(y)


def test_bound_for_the_default_grid():
    # the value hobc_gcv_expansion_bound reports for 256 values in [1e-8, 1]
    # (3.2749e-9 with its 1e-6 margin on U)
    assert 3.2e-9 < bound(1e-8, 1.0) < 3.3e-9


@pytest.mark.parametrize("seed,mu_lo,mu_hi", [(0, 1e-8, 1.0), (1, 1e-6, 1e-2), (2, 1e-10, 10.0)])
def test_random_spectra_reaching_every_key_stay_within_the_bound(seed, mu_lo, mu_hi):
    rng = np.random.default_rng(seed)
    n = 40000
    a = 10.0 ** rng.uniform(np.log10(mu_lo) - 8, np.log10(mu_hi) + 8, n)
    e = rng.exponential(1.0, n) * 10.0 ** rng.uniform(-3, 3, n)
    w = rng.choice([1.0, 2.0], n)
    mus = np.geomspace(mu_lo, mu_hi, 64)
    num, den = expansion_sums(a, e, w, mus, mu_lo, mu_hi)
    num0, den0 = exact_sums(a, e, w, mus)
    B = bound(mu_lo, mu_hi)
    r, a_lo, a_hi = geometry(mu_lo, mu_hi)
    assert (a < a_lo).any() and (a >= a_hi).any()
    assert rel(num, num0).max() <= B
    assert rel(den, den0).max() <= B
    G, G0 = num / den ** 2, num0 / den0 ** 2
    assert rel(G, G0).max() <= 3 * B          # num's error plus twice den's


def test_bin_edges_are_the_worst_case_and_the_cut_order_shows():
    """Entries at the lower edge of inner bins (u = 1/sqrt(r) - 1 < 0) and just
    below the upper edge (u -> sqrt(r) - 1), at the smallest mu (rho near 1):
    the error sits within a factor of a few of the bound, and with the p = 7
    term dropped it passes the bound."""
    mu_lo, mu_hi = 1e-8, 1.0
    r, a_lo, _ = geometry(mu_lo, mu_hi)
    B = bound(mu_lo, mu_hi)
    mus = np.array([mu_lo])
    worst = 0.0
    for b in (200, 230, 250):                     # centres far above mu: rho = c/(c+mu) near 1
        for a in (a_lo * r ** b, a_lo * r ** (b + 1) * (1 - 1e-12)):
            aa, e, w = np.array([a]), np.array([1.0]), np.array([1.0])
            num, den = expansion_sums(aa, e, w, mus, mu_lo, mu_hi)
            num0, den0 = exact_sums(aa, e, w, mus)
            err = max(rel(num, num0).max(), rel(den, den0).max())
            assert err <= B
            worst = max(worst, err)
            num7, _ = expansion_sums(aa, e, w, mus, mu_lo, mu_hi, P=7)
            assert rel(num7, num0).max() > B       # one term fewer: the bound fails
    assert worst > B / 10                         # the bound is within a factor 10 of the worst case
