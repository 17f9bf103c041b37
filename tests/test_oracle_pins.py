"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself -- a transform-free construction from the paper's boundary rules, a
textbook identity, a library transform, a closed form, an invariant the paper
states, or brute force on a tiny input.  CPU only.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth

H_SYM = synth.gaussian_psf_1d(1.3, 5)
H_NONSYM = np.array([0.05, 0.3, 0.4, 0.15, 0.1])
H_SYM7 = synth.gaussian_psf_1d(2.0, 7)


def _h(fam):
    return H_NONSYM if fam in ("F", "P") else H_SYM


# ---------------------------------------------------------------- transforms


@pytest.mark.parametrize("n", [5, 10, 33, 256])
def test_p_normalisation_reading_R2(n):
    """||p|| = 1 (stated after Eq. (eq:ART)); the printed factor squared equals the
    unnormalised norm^2 n(2n-1)/(6(n-1)), so the normalising factor is its reciprocal."""
    p = O.border_vector("S", n)
    assert abs(np.linalg.norm(p) - 1.0) < 1e-14
    raw = 1.0 - np.arange(n) / (n - 1)
    assert abs(np.sum(raw ** 2) - n * (2 * n - 1) / (6 * (n - 1))) < 1e-10 * n
    assert np.allclose(p * np.sqrt(n * (2 * n - 1) / (6 * (n - 1))), raw)


@pytest.mark.parametrize("N", [1, 2, 7, 16, 31])
def test_trig_matrices_match_library_transforms(N):
    """Q, C and F equal scipy's orthonormal DST-I, DCT-II and DFT."""
    x = np.random.default_rng(N).standard_normal(N)
    assert np.allclose(O.dst1_matrix(N) @ x, scipy.fft.dst(x, type=1, norm="ortho"), atol=1e-13)
    assert np.allclose(O.dct2_matrix(N) @ x, scipy.fft.dct(x, type=2, norm="ortho"), atol=1e-13)
    assert np.allclose(O.dft_matrix(N) @ x, scipy.fft.fft(x, norm="ortho"), atol=1e-13)


@pytest.mark.parametrize("fam", ["C", "F"])
def test_border_rows_extend_by_continuity(fam):
    """c_a, c_b are the trigonometric columns sampled at the extra grid points a, b:
    for C they repeat interior rows 1 and N, for F rows N and 1 (Sec. 3.1, 3.2)."""
    n = 12
    T = O.transform_matrix(fam, n)
    if fam == "C":
        assert np.allclose(T[0, 1:-1], T[1, 1:-1]) and np.allclose(T[-1, 1:-1], T[-2, 1:-1])
        j = np.arange(n - 2)
        assert np.allclose(T[-1, 1:-1], (-1.0) ** j * T[0, 1:-1])   # c_b = (-1)^{j-1} c_a
    else:
        assert np.allclose(T[0, 1:-1], T[-2, 1:-1]) and np.allclose(T[-1, 1:-1], T[1, 1:-1])
        assert np.allclose(T[-1, 1:-1], 1.0 / np.sqrt(n - 2))
    q = O.border_vector(fam, n)
    assert abs(q[-1]) < 1e-15 and abs(np.linalg.norm(q) - 1) < 1e-14


# ------------------------------------------------------- classical BCs (P2)


@pytest.mark.parametrize("n", [7, 12])
def test_periodic_is_circulant_diagonalised_by_F(n):
    """Explicit periodic-BC matrix = F^H diag(d) F (Eq. (eq:permat)) and the ratio rule."""
    A = O.bc_matrix(H_NONSYM, n, "periodic")
    assert np.abs(A - O.blur_matrix_spectral("P", H_NONSYM, n)).max() < 1e-13
    F = O.dft_matrix(n)
    e1 = np.eye(n)[:, 0]
    ratio = (F @ (A @ e1)) / (F @ e1)
    assert np.allclose(ratio, O.eigenvalues_1d("P", H_NONSYM, n), atol=1e-13)


@pytest.mark.parametrize("n", [7, 12])
def test_reflective_diagonalised_by_C(n):
    """Explicit reflective-BC matrix (symmetric PSF) = C^T diag(d) C (Eq. (eq:refm))."""
    A = O.bc_matrix(H_SYM, n, "reflective")
    assert np.abs(A - O.blur_matrix_spectral("R", H_SYM, n)).max() < 1e-13
    C = O.dct2_matrix(n)
    e1 = np.eye(n)[:, 0]
    assert np.allclose((C @ (A @ e1)) / (C @ e1), O.eigenvalues_1d("R", H_SYM, n), atol=1e-13)


# ----------------------------------------- antireflective and high order (P1)


@pytest.mark.parametrize("n,h", [(7, H_SYM), (12, H_SYM), (13, H_SYM7), (40, H_SYM7)])
def test_antireflective_spectral_equals_extension_rule(n, h):
    """T diag(z(y)) T^{-1} (Eq. (eq:jcf)) = matrix of the antireflective rule (Sec. 2.2)."""
    A = O.bc_matrix(h, n, "antireflective")
    assert np.abs(O.blur_matrix_spectral("S", h, n) - A).max() < 1e-12


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
@pytest.mark.parametrize("n", [9, 13, 24])
def test_high_order_matrix_equals_transform_free_construction(fam, n):
    """T_X diag(d) T_X^{-1} (Eq. (eq:Ac), (eq:Af); reading R6 for S3) equals the matrix
    built with no transform from the classical BC on the interior block and
    polynomial preservation."""
    h = _h(fam)
    As = O.blur_matrix_spectral(fam, h, n)
    assert np.abs(As - O.blur_matrix_bcfree(fam, h, n)).max() < 1e-12
    assert np.abs(As.imag).max() < 1e-12          # a real PSF gives a real matrix


def test_sign_reading_R3_literal_symbol_is_the_mirrored_model():
    """With g_i = sum h_j f_{i-j}, only z(-theta) reproduces the periodic interior;
    the printed z(+theta) reproduces the model of the mirrored PSF."""
    n = 12
    T = O.transform_matrix("F", n)
    lit = T @ np.diag(O.symbol(H_NONSYM, O.eigen_angles("F", n))) @ np.linalg.inv(T)
    assert np.abs(lit - O.blur_matrix_bcfree("F", H_NONSYM, n)).max() > 1e-2
    assert np.abs(lit - O.blur_matrix_bcfree("F", H_NONSYM[::-1], n)).max() < 1e-12


def test_grid_reading_R4_printed_grid_breaks_the_algebra():
    """The printed A_F grid (i-2) 2 pi/n does not give the periodic interior; (i-2) 2 pi/(n-2) does."""
    n = 12
    T = O.transform_matrix("F", n)
    th = (np.arange(1, n + 1) - 2) * 2 * np.pi / n
    th[0] = th[-1] = 0
    bad = T @ np.diag(O.symbol(H_NONSYM, -th)) @ np.linalg.inv(T)
    assert np.abs(bad - O.blur_matrix_bcfree("F", H_NONSYM, n)).max() > 1e-2


# ---------------------------------------------------- invariants (P3, P4)


@pytest.mark.parametrize("fam,deg", [("S", 1), ("C", 2), ("F", 2), ("S3", 3)])
def test_polynomials_are_preserved(fam, deg):
    """Sampled polynomials of degree <= deg are eigenvectors with eigenvalue z(0) = 1."""
    n = 20
    A = O.blur_matrix_spectral(fam, _h(fam), n)
    t = np.linspace(-0.7, 1.9, n)
    for k in range(deg + 1):
        assert np.abs(A @ t ** k - t ** k).max() < 1e-11
    # the next degree is not preserved (the pin has teeth)
    assert np.abs(A @ t ** (deg + 1) - t ** (deg + 1)).max() > 1e-4


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
def test_spectrum_equals_dense_eigendecomposition(fam):
    """eig(A_X) is the multiset of d; T_X T_X^{-1} = I."""
    n = 16
    A = O.blur_matrix_spectral(fam, _h(fam), n)
    ev = np.sort_complex(np.round(np.linalg.eigvals(A), 9))
    d = np.sort_complex(np.round(O.eigenvalues_1d(fam, _h(fam), n), 9))
    assert np.allclose(ev, d, atol=1e-8)
    T = O.transform_matrix(fam, n)
    assert np.allclose(T @ np.linalg.inv(T), np.eye(n), atol=1e-12)


# ------------------------------------------------------------ Laplacian


@pytest.mark.parametrize("n", [6, 11])
def test_antireflective_laplacian_is_eq_L(n):
    """L_A = T diag(s(y)) T^{-1} is the tridiagonal matrix of Eq. (eq:L) with zero end rows."""
    L = np.zeros((n, n))
    for i in range(1, n - 1):
        L[i, i - 1:i + 2] = [-1.0, 2.0, -1.0]
    T = O.transform_matrix("S", n)
    Ls = T @ np.diag(O.laplacian_angles_1d("S", n)) @ np.linalg.inv(T)
    assert np.abs(Ls - L).max() < 1e-12


@pytest.mark.parametrize("fam,rule,deg", [("C", "reflective", 2), ("F", "periodic", 2), ("S3", "odd", 3)])
def test_high_order_laplacian(fam, rule, deg):
    """L_X annihilates the preserved polynomials (Null(L) = preserved space) and acts
    on the extended interior as the second difference with the classical BC."""
    n = 14
    T = O.transform_matrix(fam, n)
    Ls = T @ np.diag(O.laplacian_angles_1d(fam, n)) @ np.linalg.inv(T)
    t = np.arange(n, dtype=float)
    for k in range(deg + 1):
        assert np.abs(Ls @ t ** k).max() < 1e-8
    E = O.extension_matrix(fam, n)
    LN = O.bc_matrix(np.array([-1.0, 2.0, -1.0]), E.shape[1], rule)
    assert np.abs(Ls @ E - E @ LN).max() < 1e-12


# ------------------------------------------------- reblurring and filter


@pytest.mark.parametrize("fam", ["C", "F"])
def test_rotated_psf_gives_conjugate_eigenvalues(fam):
    """A' = A_X(conj z): rotating the PSF by 180 degrees conjugates d (Sec. 4.1)."""
    n = 15
    h = _h(fam)
    assert np.allclose(O.eigenvalues_1d(fam, h[::-1], n), np.conj(O.eigenvalues_1d(fam, h, n)))


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("mu", [1e-6, 1e-2, 3.0])
def test_spectral_filter_equals_reblurred_normal_equations(fam, L, mu):
    """Eq. (eq:freg) = dense solve of (A'A + mu L'L) f = A'g (Eq. (eq:nerebl))."""
    n = 14
    h = _h(fam)
    g = np.random.default_rng(7).standard_normal(n)
    d = O.eigenvalues_1d(fam, h, n)
    s = O.smoothing_1d(fam, n, L)
    fs = O.synthesis_1d(fam, O.filter_factors(d, s, mu) * O.analysis_1d(fam, g)).real
    fn = O.tikhonov_normal_equations_1d(fam, h, g, L, mu)
    assert np.abs(fs - fn).max() < 1e-8 * max(1.0, np.abs(fn).max())


# ------------------------------------------------------------- GCV (P6, P7)


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
def test_gcv_trace_identity(fam):
    """trace(I - A R_mu) = sum (1 - Phi_i) exactly."""
    n = 12
    h = _h(fam)
    A = O.blur_matrix_spectral(fam, h, n)
    Ar = O.blur_matrix_spectral(fam, h[::-1], n)
    d = O.eigenvalues_1d(fam, h, n)
    s = O.smoothing_1d(fam, n, "lap")
    Lm = O.blur_matrix_spectral(fam, np.array([-1.0, 2.0, -1.0]), n)
    mu = 0.03
    R = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar)
    phi = np.abs(d) ** 2 / (np.abs(d) ** 2 + mu * s ** 2)
    assert abs(np.trace(np.eye(n) - A @ R) - np.sum(1 - phi)) < 1e-10


def test_gcv_exact_equals_spectral_for_periodic():
    """For the unitary (periodic) case Eq. (eq:gcv) and Eq. (eq:gcv2) coincide."""
    n = 16
    g = np.random.default_rng(3).standard_normal(n)
    mus = synth.mu_grid(9, 1e-6, 1.0)
    ghat = O.dft_matrix(n) @ g
    d = O.eigenvalues_1d("P", H_NONSYM, n)
    Gs = O.gcv_curve(ghat, d, np.ones(n), mus)
    Ge = O.gcv_exact_1d("P", H_NONSYM, g, "I", mus)
    assert np.allclose(Gs, Ge, rtol=1e-10)


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
@pytest.mark.parametrize("L", ["I", "lap"])
def test_gcv_brute_force_tiny(fam, L):
    """Brute force on n = 10: for each mu, solve the dense normal equations, form
    ||T^{-1}(g - A f)||^2 / trace(I - A R)^2; equals G from the spectral sums, same argmin."""
    n = 10
    h = _h(fam)
    rng = np.random.default_rng(11)
    g = np.cumsum(rng.standard_normal(n)) + 0.3 * rng.standard_normal(n)
    mus = synth.mu_grid(17, 1e-5, 10.0)
    A = O.blur_matrix_spectral(fam, h, n)
    Ar = O.blur_matrix_spectral(fam, h[::-1], n)
    Lm = np.eye(n) if L == "I" else O.blur_matrix_spectral(fam, np.array([-1.0, 2.0, -1.0]), n)
    T = O.transform_matrix(fam, n)
    brute = []
    for mu in mus:
        R = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar)
        r = g - A @ (R @ g)
        brute.append(np.linalg.norm(np.linalg.solve(T, r)) ** 2 / abs(np.trace(np.eye(n) - A @ R)) ** 2)
    brute = np.array(brute)
    _, G, k, _ = O.deblur_1d(fam, h, g, L, mus)
    assert np.allclose(G, brute, rtol=1e-8)
    assert k == int(np.argmin(brute))


def test_identity_psf_closed_form():
    """h = delta: d = 1, so with L = I, f = g/(1+mu) and G(mu) = sum|ghat|^2/n^2 for every mu."""
    n = 20
    g = np.random.default_rng(5).standard_normal(n)
    mus = synth.mu_grid(8)
    for fam in "SCF":
        f, G, k, ghat = O.deblur_1d(fam, np.array([1.0]), g, "I", mus)
        assert np.allclose(G, np.sum(np.abs(ghat) ** 2) / n ** 2, rtol=1e-12)
        assert np.allclose(f, g / (1 + mus[k]), atol=1e-12)


def test_zero_signal():
    mus = synth.mu_grid(5)
    f, G, k, _ = O.deblur_1d("C", H_SYM, np.zeros(16), "lap", mus)
    assert k == 0 and np.all(G == 0) and np.all(f == 0)


# ------------------------------------------------------------------- 2D


def test_symbol2_brute_force():
    h = synth.gaussian_psf_2d_rotated(1.1, 0.6, 30, 5, 0.3, -0.2)
    t0, t1 = np.array([0.0, 0.4, 2.0]), np.array([0.0, -1.1])
    ref = np.zeros((3, 2), dtype=complex)
    for a in range(3):
        for b in range(2):
            for j0 in range(-2, 3):
                for j1 in range(-2, 3):
                    ref[a, b] += h[j0 + 2, j1 + 2] * np.exp(1j * (j0 * t0[a] + j1 * t1[b]))
    assert np.allclose(O.symbol2(h, t0, t1), ref, atol=1e-14)


@pytest.mark.parametrize("fam,rule", [("F", "periodic"), ("C", "reflective"), ("S", "odd"), ("S3", "odd")])
def test_2d_interior_is_classical_bc_and_biquadratics_preserved(fam, rule):
    """2D A_X (Sec. 6, tensor transform + 2D eigenvalues) acts on the extended interior
    as the 2D classical-BC matrix of the 2D PSF, and preserves tensor products of
    preserved 1D polynomials with eigenvalue 1."""
    n0, n1 = 10, 11
    h = (synth.gaussian_psf_2d_rotated(1.2, 0.7, 30, 5, 0.4, -0.3) if fam == "F"
         else synth.gaussian_psf_2d_separable(1.0, 5))
    A2 = O.blur_matrix_2d_spectral(fam, h, n0, n1)
    E0, E1 = O.extension_matrix(fam, n0), O.extension_matrix(fam, n1)
    E = np.kron(E0, E1)
    assert np.abs(A2 @ E - E @ O.bc_matrix_2d(h, E0.shape[1], E1.shape[1], rule)).max() < 1e-12
    t0 = np.arange(n0)[:, None] / 3.0
    t1 = np.arange(n1)[None, :] / 4.0
    deg = {"S": 1, "C": 2, "F": 2, "S3": 3}[fam]
    u = sum(t0 ** a for a in range(deg + 1)) * sum((-0.7 * t1) ** a for a in range(deg + 1))
    assert np.abs(A2 @ u.ravel() - u.ravel()).max() < 1e-10


@pytest.mark.parametrize("fam", ["S", "C", "F", "S3"])
@pytest.mark.parametrize("L", ["I", "lap"])
def test_2d_separable_mode_equals_dense_normal_equations(fam, L):
    """The separable dense 2D method equals the dense (n0 n1)^2 reblurred normal equations."""
    n0, n1 = 8, 9
    h = (synth.gaussian_psf_2d_rotated(1.0, 0.6, 30, 3, 0.2, -0.1) if fam == "F"
         else synth.gaussian_psf_2d_separable(0.8, 3))
    g = np.random.default_rng(2).standard_normal((n0, n1))
    mu = 0.02
    A = O.blur_matrix_2d_spectral(fam, h, n0, n1)
    Ar = O.blur_matrix_2d_spectral(fam, h[::-1, ::-1], n0, n1)
    lap5 = np.array([[0, -1.0, 0], [-1.0, 4.0, -1.0], [0, -1.0, 0]])
    Lm = np.eye(n0 * n1) if L == "I" else O.blur_matrix_2d_spectral(fam, lap5, n0, n1)
    fn = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar @ g.ravel()).real.reshape(n0, n1)
    d = O.eigenvalues_2d(fam, h, n0, n1)
    s = O.smoothing_2d(fam, n0, n1, L)
    fs = O.synthesis_2d(fam, O.filter_factors(d, s, mu) * O.analysis_2d(fam, g)).real
    assert np.abs(fs - fn).max() < 1e-9


# ------------------------------------------ the pins catch planted mistakes


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant typical mistakes in the oracle (on the CPU) and check that the
    transform-free pin rejects each one."""
    n = 12

    def fails(fam, h):
        return np.abs(O.blur_matrix_spectral(fam, h, n) - O.blur_matrix_bcfree(fam, h, n)).max() > 1e-6

    orig_angles = O.eigen_angles
    orig_border = O.border_vector
    orig_T = O.transform_matrix

    monkeypatch.setattr(O, "eigen_angles", lambda f, m: -orig_angles(f, m))        # sign flip
    assert fails("F", H_NONSYM)
    monkeypatch.setattr(O, "eigen_angles", lambda f, m: np.roll(orig_angles(f, m), 1))  # index shift
    assert fails("C", H_SYM)
    monkeypatch.setattr(O, "eigen_angles", orig_angles)

    def cubic_q(f, m):                                                             # wrong exponent
        x, a, b = O.extended_grid(f, m)
        return (b - x) ** 3 / np.linalg.norm((b - x) ** 3)
    monkeypatch.setattr(O, "border_vector", cubic_q)
    assert fails("C", H_SYM)
    monkeypatch.setattr(O, "border_vector", orig_border)

    def drop_ca(f, m):
        T = orig_T(f, m).copy()
        T[0, 1:-1] = 0                                                             # c_a dropped
        return T
    monkeypatch.setattr(O, "transform_matrix", drop_ca)
    assert fails("F", H_NONSYM)
    monkeypatch.setattr(O, "transform_matrix", lambda f, m: orig_T(f, m).T)        # transposed
    assert fails("C", H_SYM)
