"""FP64 CPU oracle for the learned-mu extension (not part of the paper).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

The extension predicts log10(mu) of the GCV choice from two radial spectra
and falls back to the full GCV scan when the prediction is poor.  Everything
below is written from its plain definition:

  features (per problem, 2 x B bins): spectral entry (t0, t1) has normalised
    frequency f_a = theta_a / pi on each axis (the angle grid of the family,
    border columns at 0), folded into [0, 1] as min(f, 2 - f) for the Fourier
    family, and radius rho = sqrt((f0^2 + f1^2) / 2);
    bin b = min(B-1, floor(B rho)).  Feature b is log10 of the mean |ghat|^2
    over the entries of bin b, feature B + b the same for |d|^2 (1e-30 is
    added before the log; an empty bin gives log10(1e-30)).
  histogram features (per problem, 2 x B bins; the GCV functional's own
    statistics): entries with s != 0 grouped by a = |d|^2 / |s|^2 into B bins of
    equal width in log10 a over [1e-12, 1e4) (values outside go to the end
    bins; the edges of the binned choice's 2B bins, every other one); feature b
    is log10(E_b / E + 1e-12) with E_b = sum |ghat|^2 over bin b and E over all
    bins, feature B + b the same for the entry counts W_b.  G of Eq. (eq:gcv2)
    is a function of the (a, |ghat|^2) pairs alone, so these shares carry what
    the GCV choice depends on, to the resolution of the bins.
  network: x (128) -> GELU(W1 x + b1) (256) -> GELU(W2 h1 + b2) (256) -> w3 . h2 + b3,
    GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2; inputs are standardised
    with per-feature mean and scale stored with the weights.  The GPU uses the
    weight matrices in bfloat16 (a parity check rounds them with bf16_round)
    and runs the matrix products of the two hidden layers, of the weight
    gradients and of the back-propagated gradient on tensor cores with both
    operands rounded to bfloat16 and FP32 sums: forward and loss_and_grads take
    that product as mm=bf16_matmul (default: the exact product).
  choice: learned_choice, the bracket test that keeps or rejects the prediction.
  loss: mean squared error of the prediction against the label.
  optimiser: AdamW (decoupled weight decay, bias-corrected moments).

parity status: pinned by tests/test_mlp_oracle.py (finite differences, a
closed-form single-layer case, the features of a constant spectrum, histogram
features of spectra with hand-placed values of a).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import hobc_oracle as O

NBINS = 64


def angle_fraction(family: str, n: int):
    """theta_t / pi of every column t as exact integers a_t / q, folded into
    [0, 1] for the Fourier family (min(f, 2 - f)); border columns give 0."""
    t = np.arange(n, dtype=np.int64)
    if family == "S":
        q = n - 1
        a = t.copy()
        a[-1] = 0
    elif family == "C":
        q = n - 2
        a = t - 1
        a[[0, -1]] = 0
    elif family == "F":
        q = n - 2
        a = 2 * (t - 1)
        a[[0, -1]] = 0
        a = np.minimum(a, 2 * q - a)
    elif family == "S3":
        q = n - 3
        a = t - 1
        a[[0, 1, n - 2, n - 1]] = 0
    else:
        raise ValueError(family)
    return a, q


def radial_bins(family: str, n0: int, n1: int, nbins: int = NBINS) -> np.ndarray:
    """Bin index floor(nbins * rho) of every spectral entry (t0, t1), clamped to
    nbins - 1, with rho^2 = (f0^2 + f1^2) / 2 and f = a / q from angle_fraction.

    The floor is taken in exact arithmetic: many entries sit exactly on a bin
    edge (f0 = f1 = 1/2, say), where a rounded rho would fall either way.
    nbins^2 rho^2 = X / Y with X = nbins^2 (a0^2 q1^2 + a1^2 q0^2), Y = 2 q0^2 q1^2,
    and floor(sqrt(X / Y)) = isqrt(X // Y).
    """
    a0, q0 = angle_fraction(family, n0)
    a1, q1 = angle_fraction(family, n1)
    X = nbins * nbins * (a0[:, None] ** 2 * q1 * q1 + a1[None, :] ** 2 * q0 * q0)
    Y = 2 * q0 * q0 * q1 * q1
    v = X // Y                                     # exact, at most nbins^2
    b = np.floor(np.sqrt(v.astype(np.float64))).astype(int)   # exact for v <= 2^52
    return np.minimum(nbins - 1, b)


def features(family: str, ghat: np.ndarray, d: np.ndarray, nbins: int = NBINS) -> np.ndarray:
    """The 2 x nbins radial log-spectra of one 2D problem (full spectra)."""
    b = radial_bins(family, ghat.shape[0], ghat.shape[1], nbins).ravel()
    cnt = np.bincount(b, minlength=nbins).astype(float)
    sg = np.bincount(b, weights=np.abs(ghat.ravel()) ** 2, minlength=nbins)
    sd = np.bincount(b, weights=np.abs(d.ravel()) ** 2, minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        mg = np.where(cnt > 0, sg / np.maximum(cnt, 1), 0.0)
        md = np.where(cnt > 0, sd / np.maximum(cnt, 1), 0.0)
    return np.concatenate([np.log10(mg + 1e-30), np.log10(md + 1e-30)])


def hist_features(ghat: np.ndarray, d: np.ndarray, s: np.ndarray, nbins: int = NBINS) -> np.ndarray:
    """The 2 x nbins histogram features of one problem (full spectra, any shape)."""
    from . import binned_oracle as Bo
    W, E, _ = Bo.histogram(ghat, d, s, nb=nbins)
    return np.concatenate([np.log10(E / E.sum() + 1e-12), np.log10(W / W.sum() + 1e-12)])


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32: bfloat16 keeps
    the top 16 bits of the IEEE float32 pattern.  Finite inputs only."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_matmul(A, B):
    """A @ B with both operands rounded to bfloat16 first (sums exact in FP64)."""
    return bf16_round(A) @ bf16_round(B)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(rng: np.random.Generator, n_in=2 * NBINS, n_hidden=256):
    """Scaled-normal initial weights (a plain He-style choice)."""
    return {
        "W1": rng.standard_normal((n_hidden, n_in)) * np.sqrt(2.0 / n_in),
        "b1": np.zeros(n_hidden),
        "W2": rng.standard_normal((n_hidden, n_hidden)) * np.sqrt(2.0 / n_hidden),
        "b2": np.zeros(n_hidden),
        "w3": rng.standard_normal(n_hidden) * np.sqrt(1.0 / n_hidden),
        "b3": np.zeros(1),
    }


def forward(p, X, mm=np.matmul):
    """Prediction for a batch X [B, n_in] (already standardised); returns (y, cache).
    mm: the product of the hidden layers."""
    z1 = mm(X, p["W1"].T) + p["b1"]
    h1 = gelu(z1)
    z2 = mm(h1, p["W2"].T) + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(p, X, t, mm=np.matmul):
    """Mean squared error and its gradient with respect to every parameter.
    mm: the product of the hidden layers, the weight gradients and dz1."""
    y, (X, z1, h1, z2, h2) = forward(p, X, mm)
    B = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * gelu_grad(z2)
    g["W2"] = mm(dz2.T, h1)
    g["b2"] = dz2.sum(axis=0)
    dz1 = mm(dz2, p["W2"]) * gelu_grad(z1)
    g["W1"] = mm(dz1.T, X)
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def learned_choice(G_at, grid: np.ndarray, y: float, width: int = 17, tol: float = 1.05):
    """mu* of the learned path for one problem and whether it fell back.

    G_at(mus) returns the GCV functional at an array of mu values.
    mu_hat = 10^y with y clamped to the grid's log10 range (NaN -> grid start);
    the bracket is the min(width, K) consecutive grid values around the grid
    value nearest to mu_hat in log10 (first on ties), shifted inside the grid.
    mu_hat is kept unless G(mu_hat) > tol * (bracket minimum of G) (or is NaN)
    or the bracket minimum (first index) is on an edge of the bracket that is
    not an end of the grid; then mu* is the full-grid GCV argmin (first index).
    """
    K = len(grid)
    lg = np.log10(grid)
    l = lg[0] if np.isnan(y) else min(max(float(y), lg[0]), lg[-1])
    mu_hat = 10.0 ** l
    kn = int(np.argmin(np.abs(lg - l)))
    span = min(width, K)
    k0 = max(0, min(kn - span // 2, K - span))
    Gb = G_at(np.concatenate([[mu_hat], grid[k0:k0 + span]]))
    inner = np.where(np.isnan(Gb[1:]), np.inf, Gb[1:])
    am = int(np.argmin(inner))
    mn = inner[am]
    kmin = k0 + am
    edge = (am == 0 and kmin > 0) or (am == span - 1 and kmin < K - 1)
    worse = not (Gb[0] <= tol * mn)
    if edge or worse:
        Gf = G_at(grid)
        Gf = np.where(np.isnan(Gf), np.inf, Gf)
        return float(grid[int(np.argmin(Gf))]), True
    return float(mu_hat), False


def adamw_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW update in place (step counts from 1)."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        p[k] = p[k] - lr * (mh / (np.sqrt(vh) + eps) + wd * p[k])
