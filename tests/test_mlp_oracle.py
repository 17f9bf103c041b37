"""Pins for the learned-mu oracle (oracle/mlp_oracle.py): gradients against
central finite differences, GELU against its closed form at known points, a
one-parameter closed-form loss, AdamW's first step, and radial features of
constant spectra."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _small(rng):
    p = M.init_params(rng, n_in=6, n_hidden=5)
    X = rng.standard_normal((7, 6))
    t = rng.standard_normal(7)
    return p, X, t


def test_gelu_closed_form_points():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # Phi(1) = 0.841344746..., so GELU(1) = 0.841344746
    assert abs(M.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    z = np.linspace(-4, 4, 41)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "w3", "b3"])
def test_gradients_match_central_differences(name):
    rng = np.random.default_rng(4)
    p, X, t = _small(rng)
    _, g = M.loss_and_grads(p, X, t)
    num = np.zeros_like(p[name])
    it = np.nditer(p[name], flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = p[name][i]
        p[name][i] = old + 1e-6
        lp, _ = M.loss_and_grads(p, X, t)
        p[name][i] = old - 1e-6
        lm, _ = M.loss_and_grads(p, X, t)
        p[name][i] = old
        num[i] = (lp - lm) / 2e-6
    assert np.allclose(g[name], num, rtol=1e-6, atol=1e-9)


def test_linear_output_layer_closed_form():
    """With W1 = W2 = 0 the hidden layers are GELU(b): y = w3.GELU(GELU(b1)-shaped) + b3,
    and d loss/d b3 = 2 mean(y - t)."""
    rng = np.random.default_rng(1)
    p, X, t = _small(rng)
    p["W1"][:] = 0
    p["W2"][:] = 0
    y, _ = M.forward(p, X)
    h2 = M.gelu(p["W2"] @ M.gelu(p["b1"]) + p["b2"])
    assert np.allclose(y, h2 @ p["w3"] + p["b3"][0])
    _, g = M.loss_and_grads(p, X, t)
    assert np.isclose(g["b3"][0], 2 * np.mean(y - t))


def test_adamw_first_step_is_signed_lr():
    """After one step from zero moments, Adam moves each weight by lr*sign(g) (plus decay)."""
    rng = np.random.default_rng(2)
    p, X, t = _small(rng)
    _, g = M.loss_and_grads(p, X, t)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    before = {k: x.copy() for k, x in p.items()}
    M.adamw_step(p, g, m, v, 1, lr=1e-3, eps=0.0, wd=0.0)
    for k in p:
        nz = g[k] != 0
        assert np.allclose((before[k] - p[k])[nz], 1e-3 * np.sign(g[k][nz]))


def test_features_of_constant_spectra():
    """|ghat|^2 = 4 and |d|^2 = 1 everywhere give log10(4) and 0 in every non-empty bin."""
    n0, n1 = 20, 24
    f = M.features("C", np.full((n0, n1), 2.0), np.ones((n0, n1)))
    b = M.radial_bins("C", n0, n1).ravel()
    full = np.bincount(b, minlength=M.NBINS) > 0
    assert np.allclose(f[:M.NBINS][full], np.log10(4.0))
    assert np.allclose(f[M.NBINS:][full], 0.0, atol=1e-12)
    assert np.allclose(f[:M.NBINS][~full], -30.0)
    # border columns sit at frequency 0: bin 0 holds the four corner products
    assert b.reshape(n0, n1)[0, 0] == 0 and b.reshape(n0, n1)[-1, -1] == 0


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
@pytest.mark.parametrize("n", [8, 13, 66])
def test_angle_fraction_matches_eigen_angles(fam, n):
    """a/q * pi is the oracle's angle grid (folded into [0, pi] for F)."""
    from oracle import hobc_oracle as O
    a, q = M.angle_fraction(fam, n)
    th = O.eigen_angles(fam, n)
    if fam == "F":
        th = np.minimum(th, 2 * np.pi - th)
    assert np.allclose(a / q * np.pi, th, rtol=0, atol=1e-14)
    assert a.dtype.kind == "i" and np.all((a >= 0) & (a <= q))


def test_exact_bins_on_and_off_edges():
    """floor(64 rho) in exact arithmetic: f0 = f1 = 1/2 lands exactly on edge 32;
    elsewhere the exact bins equal a float computation except within rounding
    distance of an edge."""
    b = M.radial_bins("C", 10, 10)          # q = 8: t = 5 gives a = 4, f = 1/2
    assert b[5, 5] == 32 and b[0, 0] == 0 and b[9, 9] == 0
    assert b[8, 8] == 56                     # f0 = f1 = 7/8: 64 rho = 56 exactly
    assert b[2, 8] == 40 and b[8, 2] == 40   # f = 1/8, 7/8: rho^2 = 50/128, 64 rho = 40
    for fam, n0, n1 in [("C", 34, 50), ("F", 66, 40), ("S", 21, 30), ("S3", 30, 19)]:
        from oracle import hobc_oracle as O
        f0 = O.eigen_angles(fam, n0) / np.pi
        f1 = O.eigen_angles(fam, n1) / np.pi
        f0, f1 = np.minimum(f0, 2 - f0), np.minimum(f1, 2 - f1)
        r = 64 * np.sqrt((f0[:, None] ** 2 + f1[None, :] ** 2) / 2)
        fl = np.minimum(63, np.floor(r)).astype(int)
        ex = M.radial_bins(fam, n0, n1)
        far = np.abs(r - np.round(r)) > 1e-9
        assert np.array_equal(ex[far], fl[far])
        assert np.all(np.abs(ex - fl) <= 1)


def test_bf16_round():
    one = np.float32(1.0)
    ulp = 2.0 ** -7                          # bfloat16 spacing at 1
    assert M.bf16_round(1.0) == 1.0
    assert M.bf16_round(1.0 + ulp) == 1.0 + ulp
    assert M.bf16_round(1.0 + ulp / 2) == 1.0                 # tie -> even
    assert M.bf16_round(1.0 + 3 * ulp / 2) == 1.0 + 2 * ulp   # tie -> even
    assert M.bf16_round(1.0 + 0.6 * ulp) == 1.0 + ulp
    assert M.bf16_round(-3.0) == -3.0 and M.bf16_round(0.0) == 0.0
    x = np.random.default_rng(0).standard_normal(1000)
    r = M.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * (1 + 1e-6))
    del one


def _bowl(c):
    """G(mu) = (log10 mu - c)^2 + 1: a GCV-like curve with its minimum at 10^c."""
    return lambda mus: (np.log10(np.asarray(mus, dtype=float)) - c) ** 2 + 1.0


def test_learned_choice_cases():
    grid = 10.0 ** np.linspace(-8, 0, 81)    # spacing 0.1 in log10
    c = -4.0                                  # on the grid (index 40)
    G = _bowl(c)
    mu, fb = M.learned_choice(G, grid, c)
    assert not fb and np.isclose(mu, 1e-4)
    mu, fb = M.learned_choice(G, grid, c + 0.2)   # G = 1.04 <= 1.05 * 1
    assert not fb and np.isclose(mu, 10 ** (c + 0.2))
    mu, fb = M.learned_choice(G, grid, c + 0.3)   # G = 1.09 > 1.05, minimum inside
    assert fb and np.isclose(mu, 1e-4)
    mu, fb = M.learned_choice(G, grid, c + 3.0)   # minimum far outside the bracket
    assert fb and np.isclose(mu, 1e-4)
    mu, fb = M.learned_choice(G, grid, np.nan)    # NaN -> grid start, minimum outside
    assert fb and np.isclose(mu, 1e-4)
    Gend = _bowl(0.0)                             # minimum at the grid's last value
    mu, fb = M.learned_choice(Gend, grid, 5.0)    # clamped to 1: edge is the grid end
    assert not fb and np.isclose(mu, 1.0)
    mu, fb = M.learned_choice(G, grid, c + 0.7)   # 7 steps off: inside the +-8 bracket, G = 1.49
    assert fb and np.isclose(mu, 1e-4)
    mu, fb = M.learned_choice(G, grid, c + 0.7, width=9)   # a 9-wide bracket: minimum on its edge
    assert fb and np.isclose(mu, 1e-4)
    small = 10.0 ** np.linspace(-2, 0, 5)         # K = 5 < 17: the bracket is the grid
    mu, fb = M.learned_choice(_bowl(-1.0), small, -1.0)
    assert not fb and np.isclose(mu, 0.1)


def test_hist_features_of_hand_placed_spectra():
    """Histogram features from their definition: entries whose a = |d|^2/|s|^2 sits
    at the centre of known bins of width 0.25 decade in log10 a over [1e-12, 1e4)."""
    nb = 64
    centres = -12.0 + 0.25 * (np.arange(nb) + 0.5)          # log10 a of each bin's centre
    # three entries in bin 10, one in bin 40, two below the range (end bin 0)
    la = np.array([centres[10]] * 3 + [centres[40]] + [-15.0, -13.0])
    a = 10.0 ** la
    d = np.sqrt(a)                    # s = 1 (L = I), so a = |d|^2
    s = np.ones_like(d)
    g = np.array([1.0, 1.0, 2.0, 4.0, 0.5, 0.5])
    x = M.hist_features(g, d, s, nb)
    E = np.zeros(nb)
    W = np.zeros(nb)
    E[10], W[10] = 1 + 1 + 4, 3
    E[40], W[40] = 16, 1
    E[0], W[0] = 0.25 + 0.25, 2
    assert np.allclose(x[:nb], np.log10(E / E.sum() + 1e-12), atol=1e-12)
    assert np.allclose(x[nb:], np.log10(W / W.sum() + 1e-12), atol=1e-12)
    # entries with s = 0 are left out; the features do not change with a common scale of ghat
    x2 = M.hist_features(np.append(g, 100.0) * 3.0, np.append(d, 0.7), np.append(s, 0.0), nb)
    assert np.allclose(x2, x, atol=1e-12)


def test_hist_feature_bins_are_every_other_binned_choice_bin():
    """The 64 feature bins merge pairs of the binned choice's 128 bins exactly."""
    from oracle import binned_oracle as Bo
    rng = np.random.default_rng(3)
    a = 10.0 ** rng.uniform(-13, 5, 2000)
    b64 = Bo.bin_of(a, 64)
    b128 = Bo.bin_of(a, 128)
    assert np.array_equal(b64, b128 // 2)


def test_bf16_matmul_rounds_both_operands():
    """The tensor-core precision model: operands rounded to bfloat16, exact sums.
    Equal to the exact product on bfloat16-representable inputs, not otherwise,
    and the rounding of each operand is what moves it (a rounded-A-only product
    differs too)."""
    rng = np.random.default_rng(4)
    A = M.bf16_round(rng.standard_normal((5, 7)))
    B = M.bf16_round(rng.standard_normal((7, 3)))
    assert np.array_equal(M.bf16_matmul(A, B), A @ B)
    A2 = A + 1e-3 * rng.standard_normal(A.shape)
    B2 = B + 1e-3 * rng.standard_normal(B.shape)
    exact = A2 @ B2
    got = M.bf16_matmul(A2, B2)
    assert not np.allclose(got, exact, rtol=1e-6, atol=0)
    assert np.allclose(got, exact, rtol=0, atol=2 * 2.0 ** -8 * (np.abs(A2) @ np.abs(B2)).max())
    assert not np.array_equal(got, M.bf16_round(A2) @ B2)
