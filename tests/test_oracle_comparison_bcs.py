"""Pins for the classical comparison conditions (Sec. 2, Eq. (eq:permat),
(eq:refm)) in the forms the dense engine uses: reflective conditions with the
orthonormal DCT-II, periodic conditions with the real Hartley matrix (symmetric
PSFs).  Each is checked against the matrix built directly from its boundary
rule, and the Hartley form of G against the complex-DFT form."""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth


@pytest.mark.parametrize("n", [7, 12, 33])
def test_hartley_matrix_is_orthonormal_and_symmetric(n):
    H = O.hartley_matrix(n)
    assert np.allclose(H @ H, np.eye(n), atol=1e-13) and np.allclose(H, H.T)


@pytest.mark.parametrize("n", [9, 16, 31])
@pytest.mark.parametrize("rule,fam", [("periodic", "PH"), ("reflective", "R")])
def test_spectral_form_equals_boundary_rule_matrix(n, rule, fam):
    h = synth.gaussian_psf_1d(1.4, 7)                      # symmetric
    A = O.bc_matrix(h, n, rule)
    assert np.allclose(O.blur_matrix_spectral(fam, h, n), A, atol=1e-13)
    # and the Laplacian of the same rule: s = 2 - 2 cos(theta) on the family's grid
    lap = np.array([-1.0, 2.0, -1.0])
    L = O.bc_matrix(lap, n, rule)
    T = O.transform_matrix(fam, n)
    assert np.allclose(T @ np.diag(O.laplacian_angles_1d(fam, n)) @ np.linalg.inv(T), L, atol=1e-12)


def test_hartley_fails_for_a_nonsymmetric_psf():
    """Planted mistake: the Hartley basis does not diagonalise a nonsymmetric circulant."""
    h = synth.gaussian_psf_1d(1.2, 5) * np.linspace(0.6, 1.4, 5)
    h /= h.sum()
    assert not np.allclose(O.blur_matrix_spectral("PH", h, 16), O.bc_matrix(h, 16, "periodic"), atol=1e-6)


def test_gcv_is_the_same_in_the_hartley_and_dft_bases():
    rng = np.random.default_rng(2)
    n0, n1 = 12, 10
    h = np.outer(synth.gaussian_psf_1d(1.1, 5), synth.gaussian_psf_1d(1.6, 5))
    g = rng.standard_normal((n0, n1))
    mus = synth.mu_grid(20)
    Gs = []
    for fam in ("PH", "P"):
        ghat = O.analysis_2d(fam, g)
        d = O.eigenvalues_2d(fam, h, n0, n1)
        s = O.smoothing_2d(fam, n0, n1, "lap")
        Gs.append(O.gcv_curve(ghat, d, s, mus))
    assert np.allclose(Gs[0], Gs[1], rtol=1e-10)
    # and the deblurred image is the same
    fs = []
    for fam in ("PH", "P"):
        f, _, _, _ = O.deblur_2d(fam, h, g, "lap", mus)
        fs.append(f)
    assert np.allclose(fs[0], fs[1], atol=1e-10)


@pytest.mark.parametrize("n", [9, 16, 31])
def test_periodic_dft_form_equals_the_circulant_for_a_nonsymmetric_psf(n):
    """The periodic family in the DFT basis ('P', the form the FFT path runs): for a
    nonsymmetric PSF, F^H diag(z(-theta)) F is the circulant of the periodic rule
    (Sec. 2.1, Eq. (eq:permat)); the eigenvalues at +theta (a sign slip) are not, nor
    is the Hartley form."""
    h = synth.gaussian_psf_1d(1.2, 7) * np.linspace(0.5, 1.5, 7)
    h /= h.sum()
    A = O.bc_matrix(h, n, "periodic")
    assert np.allclose(O.blur_matrix_spectral("P", h, n), A, atol=1e-13)
    T = O.transform_matrix("P", n)
    wrong = T @ np.diag(O.symbol(h, O.eigen_angles("P", n))) @ np.linalg.inv(T)
    assert not np.allclose(wrong, A, atol=1e-6)
    assert np.allclose(wrong, O.bc_matrix(h[::-1], n, "periodic"), atol=1e-13)


def test_periodic_dft_form_2d_nonsymmetric():
    h = synth.gaussian_psf_2d_rotated(1.6, 0.9, 30.0, 5, 0.6, -0.4)
    n0, n1 = 8, 9
    A = O.bc_matrix_2d(h, n0, n1, "periodic")
    assert np.allclose(O.blur_matrix_2d_spectral("P", h, n0, n1), A, atol=1e-12)
    # the Laplacian of the periodic rule has eigenvalues s(t0) + s(t1) in the same basis
    lap = np.zeros((3, 3))
    lap[1, :] += [-1.0, 2.0, -1.0]
    lap[:, 1] += [-1.0, 2.0, -1.0]
    T = np.kron(O.transform_matrix("P", n0), O.transform_matrix("P", n1))
    s = O.smoothing_2d("P", n0, n1, "lap").ravel()
    assert np.allclose(T @ np.diag(s) @ np.linalg.inv(T), O.bc_matrix_2d(lap, n0, n1, "periodic"), atol=1e-12)
