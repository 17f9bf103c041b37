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
