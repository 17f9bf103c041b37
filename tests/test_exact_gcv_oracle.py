"""Pins of the exact-GCV oracle (oracle/exact_gcv_oracle.py): the spectral form
||T_X sigma ghat||^2 / (sum sigma)^2 against the dense normal equations of
Eq. (eq:gcv) (||g - A f||^2 / trace(I - A R)^2 with dense solves), and the
orthogonal case where it must equal the approximate functional."""
import numpy as np
import pytest

from oracle import exact_gcv_oracle as X
from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth
import parity_utils as P

MUS = synth.mu_grid(9, 1e-5, 1.0)


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
def test_1d_equals_dense_normal_equations(fam, L):
    n = 24
    h = P.psf_for(fam, 1, 5)
    g, _ = synth.problem_1d(2, n, h, 0.01)
    g = g[0]
    ghat = O.analysis_1d(fam, g)
    d = O.eigenvalues_1d(fam, h, n)
    s = O.smoothing_1d(fam, n, L)
    Gx = X.gcv_exact_curve(fam, ghat, d, s, MUS)
    Gd = O.gcv_exact_1d(fam, h, g, L, MUS)
    assert np.allclose(Gx, Gd, rtol=1e-8, atol=0)


def _dense_2d(fam, h, g, L, mus):
    n0, n1 = g.shape
    T = np.kron(O.transform_matrix(fam, n0), O.transform_matrix(fam, n1))
    Ti = np.linalg.inv(T)
    A = O.blur_matrix_2d_spectral(fam, h, n0, n1)
    Ar = O.blur_matrix_2d_spectral(fam, h[::-1, ::-1], n0, n1)
    s = O.smoothing_2d(fam, n0, n1, L).ravel()
    Lm = T @ np.diag(s) @ Ti
    gv = g.ravel()
    out = []
    for mu in mus:
        R = np.linalg.solve(Ar @ A + mu * (Lm @ Lm), Ar)
        r = gv - A @ (R @ gv)
        tr = np.trace(np.eye(len(gv)) - A @ R)
        out.append(np.linalg.norm(r) ** 2 / abs(tr) ** 2)
    return np.array(out)


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
def test_2d_equals_dense_normal_equations(fam, L):
    n0, n1 = 9, 11
    h = P.psf_for(fam, 2, (3, 3))
    g, _ = synth.problem_2d(4, n0, n1, h, 0.01)
    g = g[0]
    ghat = O.analysis_2d(fam, g)
    d = O.eigenvalues_2d(fam, h, n0, n1)
    s = O.smoothing_2d(fam, n0, n1, L)
    Gx = X.gcv_exact_curve(fam, ghat, d, s, MUS)
    Gd = _dense_2d(fam, h, g, L, MUS)
    assert np.allclose(Gx, Gd, rtol=1e-7, atol=0)


@pytest.mark.parametrize("fam", ["R", "PH"])
def test_orthogonal_transform_gives_the_approximate_functional(fam):
    n0, n1 = 16, 20
    h = np.outer(synth.gaussian_psf_1d(1.2, 5), synth.gaussian_psf_1d(0.9, 5))
    g, _ = synth.problem_2d(1, n0, n1, h, 0.01)
    g = g[0]
    ghat = O.analysis_2d(fam, g)
    d = O.eigenvalues_2d(fam, h, n0, n1)
    s = O.smoothing_2d(fam, n0, n1, "I")
    assert np.allclose(X.gcv_exact_curve(fam, ghat, d, s, MUS), O.gcv_curve(ghat, d, s, MUS), rtol=1e-12)


def test_exact_and_approximate_differ_for_high_order_conditions():
    """T_C is not orthogonal: the two functionals differ (the correction is not negligible)."""
    n0, n1 = 24, 24
    h = np.outer(synth.gaussian_psf_1d(2.0, 9), synth.gaussian_psf_1d(2.0, 9))
    g, _ = synth.problem_2d(6, n0, n1, h, 0.001)
    g = g[0]
    ghat = O.analysis_2d("C", g)
    d = O.eigenvalues_2d("C", h, n0, n1)
    s = O.smoothing_2d("C", n0, n1, "I")
    mus = synth.mu_grid(33, 1e-8, 1.0)
    Gx = X.gcv_exact_curve("C", ghat, d, s, mus)
    Ga = O.gcv_curve(ghat, d, s, mus)
    assert np.max(np.abs(Gx / Ga - 1)) > 1e-3
