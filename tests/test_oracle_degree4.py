"""Pins for the degree-4 cosine family of the oracle ('C4', reading R16: the
construction of Sec. 3.1 with two border columns per side).  The transform is
ill-conditioned (cond(T) grows like n^3.5: 7e4 at n = 32), so every tolerance
below is the FP64 unit roundoff times cond(T) times a small factor.  CPU only.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth

EPS = 2.0 ** -53
H_SYM = synth.gaussian_psf_1d(1.3, 5)


def _cond(n):
    return np.linalg.cond(O.transform_matrix("C4", n))


def test_interior_block_is_the_dct_and_border_rows_reflect():
    """Rows 2..n-3 of the interior columns are the orthonormal DCT-II of order n-4
    (SciPy); rows 0, 1 repeat rows 3, 2 and rows n-2, n-1 repeat rows n-3, n-4
    (half-sample reflection, reading R16); the border columns are unit vectors
    and the right ones are the flipped left ones."""
    n = 15
    N = n - 4
    T = O.transform_matrix("C4", n)
    D = scipy.fft.dct(np.eye(N), type=2, norm="ortho", axis=0)
    assert np.allclose(T[2:N + 2, 2:N + 2], D.T, atol=1e-14)
    assert np.allclose(T[0, 2:N + 2], T[3, 2:N + 2], atol=1e-14)
    assert np.allclose(T[1, 2:N + 2], T[2, 2:N + 2], atol=1e-14)
    assert np.allclose(T[n - 2, 2:N + 2], T[n - 3, 2:N + 2], atol=1e-14)
    assert np.allclose(T[n - 1, 2:N + 2], T[n - 4, 2:N + 2], atol=1e-14)
    for c in (0, 1, n - 2, n - 1):
        assert abs(np.linalg.norm(T[:, c]) - 1.0) < 1e-14
    assert np.allclose(T[:, n - 1], T[::-1, 0]) and np.allclose(T[:, n - 2], T[::-1, 1])


@pytest.mark.parametrize("n", [9, 13, 24])
def test_matrix_equals_transform_free_construction(n):
    """T diag(z(-theta)) T^{-1} equals the matrix built without any transform from the
    reflective BC of order n-4 on the extended interior and the preservation of the
    quartics (monomials on the integer grid, unlike Q1, Q2)."""
    As = O.blur_matrix_spectral("C4", H_SYM, n)
    Ab = O.blur_matrix_bcfree("C4", H_SYM, n)
    assert np.abs(As - Ab).max() < 64 * EPS * _cond(n)


def test_quartics_preserved_and_quintics_not():
    """Sampled polynomials of degree <= 4 are eigenvectors with eigenvalue z(0) = 1;
    degree 5 is not preserved (the pin has teeth)."""
    n = 20
    A = O.blur_matrix_spectral("C4", H_SYM, n)
    t = np.linspace(-0.7, 1.9, n)
    tol = 64 * EPS * _cond(n) * 10
    for k in range(5):
        assert np.abs(A @ t ** k - t ** k).max() < tol * max(1.0, np.abs(t ** k).max())
    assert np.abs(A @ t ** 5 - t ** 5).max() > 1e-4


def test_spectrum_equals_dense_eigendecomposition():
    """eig(A_X) is the multiset of d (four border values z(0) = 1 and the reflective
    eigenvalues of order n-4); T T^{-1} = I."""
    n = 12
    A = O.blur_matrix_spectral("C4", H_SYM, n)
    ev = np.sort(np.linalg.eigvals(A).real)
    d = O.eigenvalues_1d("C4", H_SYM, n).real
    assert np.allclose(ev, np.sort(d), atol=1e-7)
    assert np.allclose(d[[0, 1, n - 2, n - 1]], 1.0)
    R = O.bc_matrix(H_SYM, n - 4, "reflective")
    assert np.allclose(np.sort(np.linalg.eigvalsh(R)), np.sort(d[2:n - 2]), atol=1e-12)
    T = O.transform_matrix("C4", n)
    assert np.allclose(T @ np.linalg.inv(T), np.eye(n), atol=64 * EPS * _cond(n))


def test_laplacian_null_space_is_the_quartics():
    """L = T diag(2 - 2 cos theta) T^{-1} annihilates the quartics and acts on the
    extended interior as the second difference with the reflective BC."""
    n = 14
    T = O.transform_matrix("C4", n)
    Ls = T @ np.diag(O.laplacian_angles_1d("C4", n)) @ np.linalg.inv(T)
    t = np.arange(n, dtype=float) / n
    tol = 64 * EPS * _cond(n) * 10
    for k in range(5):
        assert np.abs(Ls @ t ** k).max() < tol
    assert np.abs(Ls @ t ** 5).max() > 1e-6
    E = O.extension_matrix("C4", n)
    LN = O.bc_matrix(np.array([-1.0, 2.0, -1.0]), n - 4, "reflective")
    assert np.abs(Ls @ E - E @ LN).max() < tol


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("mu", [1e-6, 1e-2, 3.0])
def test_spectral_filter_equals_reblurred_normal_equations(L, mu):
    """Eq. (eq:freg) with the degree-4 transform = dense solve of (A'A + mu L'L) f = A'g."""
    n = 13
    g = np.random.default_rng(7).standard_normal(n)
    d = O.eigenvalues_1d("C4", H_SYM, n)
    s = O.smoothing_1d("C4", n, L)
    fs = O.synthesis_1d("C4", O.filter_factors(d, s, mu) * O.analysis_1d("C4", g)).real
    fn = O.tikhonov_normal_equations_1d("C4", H_SYM, g, L, mu)
    c = _cond(n)
    assert np.abs(fs - fn).max() < 64 * EPS * c * c * max(1.0, np.abs(fn).max())


def test_gcv_trace_identity():
    """trace(I - A R_mu) = sum (1 - Phi_i)."""
    n = 12
    A = O.blur_matrix_spectral("C4", H_SYM, n)
    d = O.eigenvalues_1d("C4", H_SYM, n)
    s = O.smoothing_1d("C4", n, "lap")
    Lm = O.blur_matrix_spectral("C4", np.array([-1.0, 2.0, -1.0]), n)
    mu = 0.03
    R = np.linalg.solve(A @ A + mu * Lm @ Lm, A)           # symmetric PSF: A' = A
    phi = np.abs(d) ** 2 / (np.abs(d) ** 2 + mu * s ** 2)
    assert abs(np.trace(np.eye(n) - A @ R) - np.sum(1 - phi)) < 64 * EPS * _cond(n) ** 2


@pytest.mark.parametrize("L", ["I", "lap"])
def test_gcv_brute_force_tiny(L):
    """Brute force on n = 10: per mu, the dense solve, ||T^{-1}(g - A f)||^2 / trace(I - AR)^2;
    equals the G of the spectral sums, same argmin."""
    n = 10
    rng = np.random.default_rng(11)
    g = np.cumsum(rng.standard_normal(n)) + 0.3 * rng.standard_normal(n)
    mus = synth.mu_grid(17, 1e-5, 10.0)
    A = O.blur_matrix_spectral("C4", H_SYM, n)
    Lm = np.eye(n) if L == "I" else O.blur_matrix_spectral("C4", np.array([-1.0, 2.0, -1.0]), n)
    T = O.transform_matrix("C4", n)
    brute = []
    for mu in mus:
        R = np.linalg.solve(A @ A + mu * Lm @ Lm, A)
        r = g - A @ (R @ g)
        brute.append(np.linalg.norm(np.linalg.solve(T, r)) ** 2 / abs(np.trace(np.eye(n) - A @ R)) ** 2)
    brute = np.array(brute)
    _, G, k, _ = O.deblur_1d("C4", H_SYM, g, L, mus)
    assert np.allclose(G, brute, rtol=64 * EPS * _cond(n) ** 2)
    assert k == int(np.argmin(brute))


def test_2d_interior_is_reflective_and_biquartics_preserved():
    """The 2D matrix (tensor transform, 2D eigenvalues) acts on the extended interior as
    the 2D reflective-BC matrix of the 2D PSF and preserves tensor products of quartics."""
    n0, n1 = 10, 11
    h = synth.gaussian_psf_2d_separable(1.0, 5)
    A2 = O.blur_matrix_2d_spectral("C4", h, n0, n1)
    E0, E1 = O.extension_matrix("C4", n0), O.extension_matrix("C4", n1)
    E = np.kron(E0, E1)
    tol = 64 * EPS * _cond(n0) * _cond(n1)
    assert np.abs(A2 @ E - E @ O.bc_matrix_2d(h, n0 - 4, n1 - 4, "reflective")).max() < tol
    t0 = np.arange(n0)[:, None] / 3.0
    t1 = np.arange(n1)[None, :] / 4.0
    u = sum(t0 ** a for a in range(5)) * sum((-0.7 * t1) ** a for a in range(5))
    assert np.abs(A2 @ u.ravel() - u.ravel()).max() < tol * np.abs(u).max()


@pytest.mark.parametrize("L", ["I", "lap"])
def test_2d_separable_mode_equals_dense_normal_equations(L):
    n0, n1 = 8, 9
    h = synth.gaussian_psf_2d_separable(0.8, 3)
    g = np.random.default_rng(2).standard_normal((n0, n1))
    mu = 0.02
    A = O.blur_matrix_2d_spectral("C4", h, n0, n1)
    lap5 = np.array([[0, -1.0, 0], [-1.0, 4.0, -1.0], [0, -1.0, 0]])
    Lm = np.eye(n0 * n1) if L == "I" else O.blur_matrix_2d_spectral("C4", lap5, n0, n1)
    # reblurring (Sec. 4.1): A' is the matrix of the rotated PSF, which is A for a symmetric PSF
    fn = np.linalg.solve(A @ A + mu * Lm @ Lm, A @ g.ravel()).real.reshape(n0, n1)
    d = O.eigenvalues_2d("C4", h, n0, n1)
    s = O.smoothing_2d("C4", n0, n1, L)
    fs = O.synthesis_2d("C4", O.filter_factors(d, s, mu) * O.analysis_2d("C4", g)).real
    c = _cond(n0) * _cond(n1)
    assert np.abs(fs - fn).max() < 64 * EPS * c * c * max(1.0, np.abs(fn).max())


def test_pins_catch_a_wrong_second_border_column(monkeypatch):
    """A cubic instead of a quartic second border column breaks the preservation of
    the quartics and the transform-free equality."""
    def cubic(n):
        x, a, b = O.quartic_grid(n)
        Q1, Q2 = (b - x) ** 2, (b - x) ** 3
        return Q1 / np.linalg.norm(Q1), Q2 / np.linalg.norm(Q2)
    monkeypatch.setattr(O, "quartic_border_columns", cubic)
    n = 13
    A = O.blur_matrix_spectral("C4", H_SYM, n)
    t = np.linspace(-0.7, 1.9, n)
    assert np.abs(A @ t ** 4 - t ** 4).max() > 1e-4
    assert np.abs(A - O.blur_matrix_bcfree("C4", H_SYM, n)).max() > 1e-6


# ----------------------------------------------- degree 4, Fourier basis (R17)

H_NONSYM = np.array([0.05, 0.3, 0.4, 0.15, 0.1])


def _condF(n):
    return np.linalg.cond(O.transform_matrix("F4", n))


def test_fourier4_interior_block_is_the_dft_and_border_rows_wrap():
    """Rows 2..n-3 of the interior columns are F^H of order n-4 (unitary DFT); rows 0, 1
    repeat rows n-4, n-3 and rows n-2, n-1 repeat rows 2, 3 (periodic wrap, R17)."""
    n = 14
    N = n - 4
    T = O.transform_matrix("F4", n)
    assert np.allclose(T[2:N + 2, 2:N + 2], O.dft_matrix(N).conj().T, atol=1e-14)
    assert np.allclose(T[0, 2:N + 2], T[n - 4, 2:N + 2], atol=1e-13)
    assert np.allclose(T[1, 2:N + 2], T[n - 3, 2:N + 2], atol=1e-13)
    assert np.allclose(T[n - 2, 2:N + 2], T[2, 2:N + 2], atol=1e-13)
    assert np.allclose(T[n - 1, 2:N + 2], T[3, 2:N + 2], atol=1e-13)


@pytest.mark.parametrize("n", [9, 13, 24])
def test_fourier4_matrix_equals_transform_free_construction(n):
    """T diag(z(-theta)) T^{-1} for a nonsymmetric PSF equals the transform-free matrix
    from the periodic rule of order n-4 on the extended interior and quartic
    preservation; it is real."""
    As = O.blur_matrix_spectral("F4", H_NONSYM, n)
    assert np.abs(As - O.blur_matrix_bcfree("F4", H_NONSYM, n)).max() < 64 * EPS * _condF(n)
    assert np.abs(As.imag).max() < 64 * EPS * _condF(n)


def test_fourier4_literal_symbol_is_the_mirrored_model():
    """Reading R3 holds for degree 4 too: z(+theta) gives the model of the mirrored PSF."""
    n = 13
    T = O.transform_matrix("F4", n)
    lit = T @ np.diag(O.symbol(H_NONSYM, O.eigen_angles("F4", n))) @ np.linalg.inv(T)
    assert np.abs(lit - O.blur_matrix_bcfree("F4", H_NONSYM, n)).max() > 1e-2
    assert np.abs(lit - O.blur_matrix_bcfree("F4", H_NONSYM[::-1], n)).max() < 64 * EPS * _condF(n)


def test_fourier4_quartics_preserved_and_quintics_not():
    n = 20
    A = O.blur_matrix_spectral("F4", H_NONSYM, n)
    t = np.linspace(-0.7, 1.9, n)
    tol = 64 * EPS * _condF(n) * 10
    for k in range(5):
        assert np.abs(A @ t ** k - t ** k).max() < tol * max(1.0, np.abs(t ** k).max())
    assert np.abs(A @ t ** 5 - t ** 5).max() > 1e-4


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("mu", [1e-6, 1e-2, 3.0])
def test_fourier4_filter_equals_reblurred_normal_equations(L, mu):
    """Eq. (eq:freg) = dense solve of (A'A + mu L'L) f = A'g with A' the matrix of the
    rotated PSF (Sec. 4.1)."""
    n = 13
    g = np.random.default_rng(7).standard_normal(n)
    d = O.eigenvalues_1d("F4", H_NONSYM, n)
    s = O.smoothing_1d("F4", n, L)
    fs = O.synthesis_1d("F4", O.filter_factors(d, s, mu) * O.analysis_1d("F4", g)).real
    fn = O.tikhonov_normal_equations_1d("F4", H_NONSYM, g, L, mu)
    c = _condF(n)
    assert np.abs(fs - fn).max() < 64 * EPS * c * c * max(1.0, np.abs(fn).max())


@pytest.mark.parametrize("L", ["I", "lap"])
def test_fourier4_2d_separable_mode_equals_dense_normal_equations(L):
    n0, n1 = 9, 10
    h = synth.gaussian_psf_2d_rotated(1.0, 0.6, 30, 3, 0.2, -0.1)
    g = np.random.default_rng(2).standard_normal((n0, n1))
    mu = 0.02
    A = O.blur_matrix_2d_spectral("F4", h, n0, n1)
    Ar = O.blur_matrix_2d_spectral("F4", h[::-1, ::-1], n0, n1)
    lap5 = np.array([[0, -1.0, 0], [-1.0, 4.0, -1.0], [0, -1.0, 0]])
    Lm = np.eye(n0 * n1) if L == "I" else O.blur_matrix_2d_spectral("F4", lap5, n0, n1)
    fn = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar @ g.ravel()).real.reshape(n0, n1)
    d = O.eigenvalues_2d("F4", h, n0, n1)
    s = O.smoothing_2d("F4", n0, n1, L)
    fs = O.synthesis_2d("F4", O.filter_factors(d, s, mu) * O.analysis_2d("F4", g)).real
    c = _condF(n0) * _condF(n1)
    assert np.abs(fs - fn).max() < 64 * EPS * c * c * max(1.0, np.abs(fn).max())


def test_pins_catch_planted_mistakes_in_grids_and_angles(monkeypatch):
    """A Fourier grid of the wrong step, a shifted cosine angle grid and a swapped wrap
    row each break the transform-free equality the pins above rely on."""
    n = 13
    tol = 1e-6
    # the degree-4 Fourier grid with the step of order n-3 (a shift of the whole grid
    # would only rephase the columns, which leaves A unchanged)
    good = O.fourier4_grid

    def shifted(m):
        x = (np.arange(m) - 2) * 2 * np.pi / (m - 3)
        return x, x[0], x[-1]
    monkeypatch.setattr(O, "fourier4_grid", shifted)
    assert np.abs(O.blur_matrix_spectral("F4", H_NONSYM, n) - O.blur_matrix_bcfree("F4", H_NONSYM, n)).max() > tol
    monkeypatch.setattr(O, "fourier4_grid", good)
    # the interior angles of the cosine family off by one frequency
    angles = O.eigen_angles

    def off_by_one(fam, m):
        th = angles(fam, m)
        if fam == "C4":
            th = th.copy()
            th[2:m - 2] = (np.arange(2, m - 2) - 1) * np.pi / (m - 4)
        return th
    monkeypatch.setattr(O, "eigen_angles", off_by_one)
    assert np.abs(O.blur_matrix_spectral("C4", H_SYM, n) - O.blur_matrix_bcfree("C4", H_SYM, n)).max() > tol
    monkeypatch.setattr(O, "eigen_angles", angles)
    # the wrap rows of the Fourier extension swapped
    ext = O.extension_matrix

    def swapped(fam, m):
        E = ext(fam, m)
        if fam == "F4":
            E = E.copy()
            E[[0, 1]] = E[[1, 0]]
        return E
    monkeypatch.setattr(O, "extension_matrix", swapped)
    assert np.abs(O.blur_matrix_spectral("F4", H_NONSYM, n) - O.blur_matrix_bcfree("F4", H_NONSYM, n)).max() > tol


@pytest.mark.parametrize("L", ["I", "lap"])
def test_fourier4_gcv_brute_force_tiny(L):
    """n = 10, nonsymmetric PSF: per mu the dense solve with A' the rotated-PSF matrix,
    ||T^{-1}(g - A f)||^2 / trace(I - A R)^2, equals the G of the spectral sums."""
    n = 10
    rng = np.random.default_rng(13)
    g = np.cumsum(rng.standard_normal(n)) + 0.3 * rng.standard_normal(n)
    mus = synth.mu_grid(17, 1e-5, 10.0)
    A = O.blur_matrix_spectral("F4", H_NONSYM, n)
    Ar = O.blur_matrix_spectral("F4", H_NONSYM[::-1], n)
    Lm = np.eye(n) if L == "I" else O.blur_matrix_spectral("F4", np.array([-1.0, 2.0, -1.0]), n)
    T = O.transform_matrix("F4", n)
    brute = []
    for mu in mus:
        R = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar)
        r = g - A @ (R @ g)
        brute.append(np.linalg.norm(np.linalg.solve(T, r)) ** 2 / abs(np.trace(np.eye(n) - A @ R)) ** 2)
    brute = np.array(brute)
    _, G, k, _ = O.deblur_1d("F4", H_NONSYM, g, L, mus)
    assert np.allclose(G, brute, rtol=64 * EPS * _condF(n) ** 2)
    assert k == int(np.argmin(brute))


def test_fourier4_2d_interior_is_periodic_and_biquartics_preserved():
    n0, n1 = 10, 11
    h = synth.gaussian_psf_2d_rotated(1.2, 0.7, 30, 5, 0.4, -0.3)
    A2 = O.blur_matrix_2d_spectral("F4", h, n0, n1)
    E0, E1 = O.extension_matrix("F4", n0), O.extension_matrix("F4", n1)
    E = np.kron(E0, E1)
    tol = 64 * EPS * _condF(n0) * _condF(n1)
    assert np.abs(A2 @ E - E @ O.bc_matrix_2d(h, n0 - 4, n1 - 4, "periodic")).max() < tol
    t0 = np.arange(n0)[:, None] / 3.0
    t1 = np.arange(n1)[None, :] / 4.0
    u = sum(t0 ** a for a in range(5)) * sum((-0.7 * t1) ** a for a in range(5))
    assert np.abs(A2 @ u.ravel() - u.ravel()).max() < tol * np.abs(u).max()
