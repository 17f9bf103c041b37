"""FP64 CPU oracle for the exact GCV functional of Eq. (eq:gcv).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

The paper's GCV (Eq. (eq:gcv)) has the numerator ||g - A f_mu||; with
A = T_X D T_X^{-1} and the reblurred filter of Eq. (eq:freg),
g - A f_mu = T_X (I - Phi_mu) T_X^{-1} g.  The paper then drops T_X
(Eq. (eq:gcv2)), which is exact only when T_X is unitary.  Here T_X stays:

    G_ex(mu) = ||T_X (sigma * ghat)||^2 / (sum sigma)^2,
    sigma_i = |s_i|^2 / (|d_i|^2 + mu |s_i|^2) = (1 - phi_i) / mu,

the same normalisation as the approximate functional (numerator and
denominator divided by mu^2); T_X is applied as the dense matrix of each axis
(synthesis_1d / synthesis_2d).  The denominator is the trace of I - A R_mu,
which the spectral form gives exactly (pin P6).

parity status: pinned by tests/test_exact_gcv_oracle.py (equal to the dense
normal-equations functional in 1D for every family and in 2D on small
fields of view; equal to the approximate functional when T_X is orthogonal).
"""
from __future__ import annotations

import numpy as np

from oracle import hobc_oracle as O


def gcv_exact_curve(family: str, ghat: np.ndarray, d: np.ndarray, s: np.ndarray, mus) -> np.ndarray:
    """G_ex(mu) for every mu of the grid; ghat, d, s full spectra (1D or 2D)."""
    a2 = np.abs(d) ** 2
    s2 = np.abs(s) ** 2
    out = np.empty(len(mus))
    for k, mu in enumerate(mus):
        sig = s2 / (a2 + mu * s2)
        rho = sig * ghat
        y = O.synthesis_1d(family, rho) if ghat.ndim == 1 else O.synthesis_2d(family, rho)
        out[k] = np.sum(np.abs(y) ** 2) / np.sum(sig) ** 2
    return out
