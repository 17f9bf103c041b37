"""Helpers shared by the parity tests: seeded inputs, the oracle's answers, and
conversion of the oracle's full spectra to the library's stored layout
(include/hobc.h, "Spectrum layout")."""
from __future__ import annotations

import numpy as np

from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth

FAM_LETTER = {"sine": "S", "cosine": "C", "fourier": "F", "sine3": "S3", "reflective": "R", "periodic": "PH",
              "cosine4": "C4", "fourier4": "F4"}
EPS32 = 2.0 ** -24


def stored_t(fam: str, n: int, half: bool) -> np.ndarray:
    """Spectral index t of every stored entry along an axis."""
    if fam == "F" and half:
        H = (n - 2) // 2 + 1
        return np.concatenate([np.arange(H + 1), [n - 1]])
    if fam == "F4" and half:
        H = (n - 4) // 2 + 1
        return np.concatenate([np.arange(H + 2), [n - 2, n - 1]])
    if fam == "P" and half:
        return np.arange(n // 2 + 1)
    return np.arange(n)


def to_layout(fam: str, full: np.ndarray) -> np.ndarray:
    """Oracle spectrum (1D [n] or 2D [n0, n1], t-indexed) -> stored layout
    (1D [W]; 2D [W1, n0], i.e. [c][t0])."""
    if full.ndim == 1:
        return full[stored_t(fam, full.shape[0], True)]
    n0, n1 = full.shape
    return full[:, stored_t(fam, n1, True)].T.copy()


def psf_for(fam: str, ndim: int, taps):
    """A PSF of the right symmetry for the family (nonsymmetric for the Fourier
    families F, F4 and the periodic family P)."""
    if fam in ("F4", "P"):
        fam = "F"
    if ndim == 1:
        if fam == "F":
            h = synth.gaussian_psf_1d(1.2, taps) * np.linspace(0.6, 1.4, taps)
            return h / h.sum()
        return synth.gaussian_psf_1d(1.3, taps)
    p0, p1 = taps
    if fam == "F":
        assert p0 == p1
        return synth.gaussian_psf_2d_rotated(1.6, 0.9, 30.0, p0, 0.6, -0.4)
    h = np.outer(synth.gaussian_psf_1d(1.4, p0), synth.gaussian_psf_1d(1.1, p1))
    return h / h.sum()


def problems(ndim: int, n, h: np.ndarray, batch: int, seed: int, eta: float = 0.01):
    if ndim == 1:
        return synth.problem_1d(seed, n[0], h, eta, count=batch)
    return synth.problem_2d(seed, n[0], n[1], h, eta, count=batch)


def oracle_steps(fam: str, ndim: int, h: np.ndarray, g: np.ndarray, L: str, mus: np.ndarray):
    """Oracle answer for one problem: full spectrum, eigenvalues, smoothing, G, argmin."""
    if ndim == 1:
        n = g.shape[0]
        ghat = O.analysis_1d(fam, g)
        d = O.eigenvalues_1d(fam, h, n)
        s = O.smoothing_1d(fam, n, L)
    else:
        n0, n1 = g.shape
        ghat = O.analysis_2d(fam, g)
        d = O.eigenvalues_2d(fam, h, n0, n1)
        s = O.smoothing_2d(fam, n0, n1, L)
    G = O.gcv_curve(ghat, d, s, mus)
    return ghat, d, s, G, O.gcv_argmin(G)


def oracle_filtered(fam: str, ndim: int, ghat, d, s, mu):
    c = O.filter_factors(d, s, mu) * ghat
    return (O.synthesis_1d(fam, c) if ndim == 1 else O.synthesis_2d(fam, c)).real


def amplification(d: np.ndarray, s: np.ndarray, mu: float) -> float:
    """max_i |d_i| / (|d_i|^2 + mu |s_i|^2): how much the filter can magnify an
    absolute error in the spectrum (1/(2 sqrt(mu)) at most when L = I)."""
    a = np.abs(d)
    return float(np.max(a / (a * a + mu * np.abs(s) ** 2)))


# ----------------------------------------------------------------------------
# Forward-error bounds for FP32 (reading R13).  A product y = T x evaluated in
# working precision eps by an FFT of length M satisfies, componentwise and up to
# a small constant, |dy| <= eps * log2(M) * (|T| |x|); the bound below uses the
# largest entry of |T| |x| (|T0| |X| |T1|^T in 2D), which captures the
# cancellation between the trigonometric part and the border polynomials.
# ----------------------------------------------------------------------------

def abs_apply(fam: str, X: np.ndarray, inverse: bool = False) -> np.ndarray:
    """|T| |X| (1D) or |T0| |X| |T1|^T (2D) with T = T_X (or T_X^{-1})."""
    def mat(n):
        T = O.transform_matrix(fam, n)
        return np.abs(np.linalg.inv(T) if inverse else T)
    A = np.abs(X)
    if X.ndim == 1:
        return mat(X.shape[0]) @ A
    return mat(X.shape[0]) @ A @ mat(X.shape[1]).T


def abs_norm(fam: str, shape, inverse: bool = False) -> float:
    """Infinity norm of |T| (product over axes in 2D)."""
    out = 1.0
    for n in shape:
        T = O.transform_matrix(fam, n)
        out *= np.abs(np.linalg.inv(T) if inverse else T).sum(axis=1).max()
    return float(out)


def log2_fft(fam: str, shape) -> float:
    """log2 of the largest power-of-two FFT the kernels use for these lengths."""
    out = 0.0
    for n in shape:
        N = n - 4 if fam in ("S3", "C4", "F4") else n if fam == "P" else n - 2
        L = 2 * (N + 1) if fam in ("S", "S3") else N
        M = L if (L >= 8 and L & (L - 1) == 0) else max(8, 1 << int(np.ceil(np.log2(2 * L - 1))))
        out = max(out, np.log2(M))
    return out


def sigma(fam: str, shape, inverse: bool = False) -> float:
    """Largest singular value of the 1D/2D transform T_X (or of T_X^{-1}):
    the product over axes of ||T_axis||_2 (||T_axis^{-1}||_2)."""
    out = 1.0
    for n in shape:
        sv = np.linalg.svd(O.transform_matrix(fam, n), compute_uv=False)
        out *= (1.0 / sv.min()) if inverse else sv.max()
    return float(out)
