"""FP64 CPU oracle for spectral Tikhonov deblurring under high-order boundary
conditions with GCV (Donatelli, "Fast transforms for high order boundary
conditions", arXiv:0906.2704).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg may import this module.  The product
path (the CUDA library and its Python binding) never imports, links or calls
it, and it shares no code, table or constant generator with that path.

Everything here is plain and slow on purpose: every transform is a dense matrix
assembled entrywise from the paper's formulas, every inverse is a dense LU solve
(``numpy.linalg.solve``), and the blurring matrices are also built
*transform-free* from the boundary-extension rules so that the spectral
definitions can be checked against something other than themselves.

Families (per axis):
  'S'  antireflective BC, degree 1 (Sec. 2.2, Eq. (eq:ART), Eq. (eq:jcf))
  'C'  quadratic-preserving, cosine basis, symmetric PSF (Sec. 3.1, Eq. (eq:Tc), (eq:Ac))
  'F'  quadratic-preserving, Fourier basis, any PSF (Sec. 3.2, Eq. (eq:Tf), (eq:Af))
  'S3' cubic-preserving, sine basis, symmetric PSF: degree 3, which the paper
      only names (Sec. 1 "quadratic or cubic", Sec. 7); built as reading R6 below.
  'C4' quartic-preserving, cosine basis, symmetric PSF: degree 4, the cosine
      family with two border columns per side (Sec. 7 names higher orders);
      built as reading R16 below.
  'F4' quartic-preserving, Fourier basis, any PSF: degree 4, the construction of
      Sec. 3.2 with two border columns per side (reading R17 below).
Comparison (classical) families, used by the pins:
  'P'  periodic (Sec. 2.1, Eq. (eq:permat));  'R' reflective (Sec. 2.1, Eq. (eq:refm))

Readings where the paper is silent, garbled or inconsistent:
  R2  p in Eq. (eq:ART) is normalised to unit 2-norm (the printed factor is the
      reciprocal of the one that makes ||p|| = 1, which Sec. 2.2 asserts).
  R3  convolution convention g_i = sum_j h_j f_{i-j} (Eq. (eq:mod_cont)); the
      eigenvalue attached to a basis column of frequency theta is z(-theta).
  R4  the A_F grid is x_i = (i-2) 2 pi/(n-2) (the text says "circulant of order n-2").
  R8  2D Laplacian = Kronecker sum, s(t0, t1) = s(t0) + s(t1) (5-point stencil).
  R10 argmin ties -> lowest index (smallest mu).
  R6  degree 3 ('S3'): DST-I of order N = n-4 on x_i = i pi/(N+1), i = -1..N+2,
      extended oddly (rows i = 0, N+1 are zero, rows i = -1, N+2 are minus rows 1, N);
      border columns L1 = (x_{N+1}-x)(x_{N+2}-x), L2 = L1 (x_{N+2}-x) and their flips,
      each of unit norm, with eigenvalue z(0); together they span the cubics.
  R16 degree 4 ('C4'): the construction of Sec. 3.1 with two border columns per
      side: DCT-II of order N = n-4 on the grid x_i = (2i-3) pi/(2N), i = 0..n-1
      (x_2..x_{n-3} the DCT-II samples, two points added at each end by
      continuity, so rows 0, 1 repeat rows 3, 2 and rows n-2, n-1 repeat rows
      n-3, n-4: half-sample reflection), interval [a, b] = [x_0, x_{n-1}];
      border columns Q1 = (b-x)^2 and Q2 = (b-x)^4 and their flips (x-a)^2,
      (x-a)^4, each of unit norm, with eigenvalue z(0); with the cosine of
      frequency 0 they span the quartics.  Interior eigenvalues are those of the
      reflective matrix of order n-4 (angles (t-2) pi/N).
  R17 degree 4, Fourier basis ('F4'): the construction of Sec. 3.2 with two
      border columns per side: DFT of order N = n-4 on x_i = (i-2) 2 pi/N,
      i = 0..n-1 (x_2..x_{n-3} the DFT samples; two points added at each end by
      continuity, a periodic wrap: rows 0, 1 repeat rows n-4, n-3 and rows n-2,
      n-1 repeat rows 2, 3), interval [a, b] = [x_0, x_{n-1}], border columns
      (b-x)^2, (b-x)^4 and their flips, unit norm, eigenvalue z(0); interior
      eigenvalues z(-theta) of the circulant of order n-4 (angles (t-2) 2 pi/N).
  GCV with complex spectra uses |sigma_i ghat_i|^2 (Eq. (eq:gcv2) is written for
      real data).

Spectrum index convention (shared with the GPU path's documentation, not its
code): index t of a length-n spectrum is column t of T_X; t = 0 is the left
border vector (p or q), t = 1..N the trigonometric columns in the natural order
of X, t = n-1 the right border vector (Jp or Jq).

Parity status of each function is given in its docstring; every function below
is pinned by tests/test_oracle_pins.py unless it says "parity unpinned".
"""
from __future__ import annotations

import numpy as np

FAMILIES = ("S", "C", "F")

# --------------------------------------------------------------------------
# Symbol of the PSF -- Sec. 2, Eq. (eq:symbol)
# --------------------------------------------------------------------------


def symbol(h: np.ndarray, t: np.ndarray) -> np.ndarray:
    """z(t) = sum_{j=-m}^{m} h_j exp(i j t)  (Eq. (eq:symbol)); h[j+m] = h_j."""
    h = np.asarray(h, dtype=np.float64)
    m = (len(h) - 1) // 2
    j = np.arange(-m, m + 1)
    return np.exp(1j * np.outer(np.atleast_1d(t), j)) @ h


def symbol2(h: np.ndarray, t0: np.ndarray, t1: np.ndarray) -> np.ndarray:
    """2D symbol z(t0, t1) = sum h_{j0 j1} exp(i (j0 t0 + j1 t1)) on the grid t0 x t1.

    Sec. 6 (tensor-product setting).  h[j0+m0, j1+m1] = h_{j0 j1}; axis 0 = rows.
    The double sum is written as two matrix products E0 h E1^T.
    """
    h = np.asarray(h, dtype=np.float64)
    m0, m1 = (h.shape[0] - 1) // 2, (h.shape[1] - 1) // 2
    e0 = np.exp(1j * np.outer(np.atleast_1d(t0), np.arange(-m0, m0 + 1)))
    e1 = np.exp(1j * np.outer(np.atleast_1d(t1), np.arange(-m1, m1 + 1)))
    return e0 @ h @ e1.T


# --------------------------------------------------------------------------
# Trigonometric matrices, entrywise from their printed definitions
# --------------------------------------------------------------------------


def dst1_matrix(N: int) -> np.ndarray:
    """Q of order N: sqrt(2/(N+1)) sin(i j pi/(N+1)), i,j = 1..N (Sec. 2.2, with n-1 = N+1)."""
    i = np.arange(1, N + 1)
    return np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, i) * np.pi / (N + 1))


def dct2_matrix(N: int) -> np.ndarray:
    """C of order N: sqrt((2-delta_{i1})/N) cos((i-1)(2j-1) pi/(2N)) (Sec. 2.1 / Sec. 3)."""
    i = np.arange(1, N + 1)[:, None]
    j = np.arange(1, N + 1)[None, :]
    scale = np.sqrt((2.0 - (i == 1)) / N)
    return scale * np.cos((i - 1) * (2 * j - 1) * np.pi / (2 * N))


def dft_matrix(N: int) -> np.ndarray:
    """F of order N: exp(-i 2 pi (i-1)(j-1)/N)/sqrt(N) (Sec. 2.1 / Sec. 3)."""
    k = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(k, k) / N) / np.sqrt(N)


def hartley_matrix(n: int) -> np.ndarray:
    """H[k, j] = (cos(2 pi k j / n) + sin(2 pi k j / n)) / sqrt(n)."""
    k = np.arange(n)
    a = 2.0 * np.pi * np.outer(k, k) / n
    return (np.cos(a) + np.sin(a)) / np.sqrt(n)


def flip(n: int) -> np.ndarray:
    """Flip matrix J, J_{i, n+1-i} = 1."""
    return np.eye(n)[::-1]


# --------------------------------------------------------------------------
# Border vectors and grids
# --------------------------------------------------------------------------


def border_vector(family: str, n: int) -> np.ndarray:
    """The left border column of T_X (length n).

    'S': p_i proportional to 1 - (i-1)/(n-1), scaled to ||p||_2 = 1 (Eq. (eq:ART), reading R2).
    'C': q = qt/||qt||, qt_{i+1} = (b - x_i)^2 on the grid of Eq. (eq:points),
         interval Eq. (eq:ints)  (Sec. 3.1).
    'F': the same on the grid of Eq. (eq:pointn), interval Eq. (eq:intn) (Sec. 3.2).
    """
    if family == "S":
        i = np.arange(1, n + 1)
        p = 1.0 - (i - 1) / (n - 1)
        return p / np.linalg.norm(p)
    x, a, b = extended_grid(family, n)
    qt = (b - x) ** 2
    return qt / np.linalg.norm(qt)


def cubic_border_columns(n: int):
    """L1, L2 of the degree-3 transform (reading R6), unit 2-norm, on the grid
    x_i = i pi/(N+1), i = -1..N+2 (array index i+1), N = n-4."""
    N = n - 4
    x = np.arange(-1, N + 3) * np.pi / (N + 1)
    xa, xb = np.pi, (N + 2) * np.pi / (N + 1)          # x_{N+1}, x_{N+2}
    L1 = (xa - x) * (xb - x)
    L2 = L1 * (xb - x)
    return L1 / np.linalg.norm(L1), L2 / np.linalg.norm(L2)


def quartic_grid(n: int):
    """Grid x_0..x_{n-1} and interval [a, b] of the degree-4 transform (reading R16):
    x_i = (2i - 3) pi / (2N), N = n - 4."""
    N = n - 4
    x = (2 * np.arange(n) - 3) * np.pi / (2 * N)
    return x, x[0], x[-1]


def fourier4_grid(n: int):
    """Grid x_0..x_{n-1} and interval [a, b] of the degree-4 Fourier transform
    (reading R17): x_i = (i - 2) 2 pi / N, N = n - 4."""
    N = n - 4
    x = (np.arange(n) - 2) * 2 * np.pi / N
    return x, x[0], x[-1]


def quartic_border_columns(n: int, grid=None):
    """Q1 = (b-x)^2, Q2 = (b-x)^4 of the degree-4 transforms (readings R16, R17), unit
    2-norm, on the cosine grid (default) or the grid ``grid(n)`` returns."""
    x, a, b = (grid or quartic_grid)(n)
    Q1 = (b - x) ** 2
    Q2 = (b - x) ** 4
    return Q1 / np.linalg.norm(Q1), Q2 / np.linalg.norm(Q2)


def extended_grid(family: str, n: int):
    """Grid x_0..x_{n-1} and interval [a, b] of the basis functions (Sec. 3, remark)."""
    N = n - 2
    i = np.arange(0, n)
    if family == "C":
        x = (2 * i - 1) * np.pi / (2 * n - 4)            # Eq. (eq:points)
        a, b = -np.pi / (2 * n - 4), (2 * n - 3) * np.pi / (2 * n - 4)   # Eq. (eq:ints)
    elif family == "F":
        x = (i - 1) * 2 * np.pi / N                      # Eq. (eq:pointn)
        a, b = -2 * np.pi / N, 2 * np.pi                 # Eq. (eq:intn)
    elif family == "S":
        x = i * np.pi / (n - 1)                          # remark before Sec. 3.1
        a, b = 0.0, np.pi
    else:
        raise ValueError(family)
    return x, a, b


def eigen_angles(family: str, n: int) -> np.ndarray:
    """Angle theta_t attached to column t of the transform (length n).

    'S': y_i = (i-1) pi/(n-1), i = 1..n-1, y_n = 0        (Eq. (eq:jcf))
    'C': x_1 = x_n = 0, x_i = (i-2) pi/(n-2)              (Eq. (eq:Ac))
    'F': x_1 = x_n = 0, x_i = (i-2) 2 pi/(n-2)            (Eq. (eq:Af), reading R4)
    'S3': border columns 1, 2, n-1, n at 0, the others (i-2) pi/(n-3)   (reading R6)
    'C4': border columns 1, 2, n-1, n at 0, the others (i-3) pi/(n-4)   (reading R16)
    'P': x_i = 2 (i-1) pi/n                               (Eq. (eq:permat))
    'PH': as 'P' (periodic conditions in the Hartley basis)
    'R': x_i = (i-1) pi/n                                 (Eq. (eq:refm))
    """
    i = np.arange(1, n + 1, dtype=np.float64)
    if family == "S":
        th = (i - 1) * np.pi / (n - 1)
        th[-1] = 0.0
    elif family == "C":
        th = (i - 2) * np.pi / (n - 2)
        th[0] = th[-1] = 0.0
    elif family == "F":
        th = (i - 2) * 2 * np.pi / (n - 2)
        th[0] = th[-1] = 0.0
    elif family == "S3":                                 # reading R6
        th = (i - 2) * np.pi / (n - 3)
        th[[0, 1, n - 2, n - 1]] = 0.0
    elif family == "C4":                                 # reading R16
        th = (i - 3) * np.pi / (n - 4)
        th[[0, 1, n - 2, n - 1]] = 0.0
    elif family == "F4":                                 # reading R17
        th = (i - 3) * 2 * np.pi / (n - 4)
        th[[0, 1, n - 2, n - 1]] = 0.0
    elif family in ("P", "PH"):
        th = 2 * (i - 1) * np.pi / n
    elif family == "R":
        th = (i - 1) * np.pi / n
    else:
        raise ValueError(family)
    return th


# --------------------------------------------------------------------------
# The transforms T_X (synthesis) -- assembled entrywise
# --------------------------------------------------------------------------


def transform_matrix(family: str, n: int) -> np.ndarray:
    """Dense T_X of order n.

    'S': Eq. (eq:ART)  T = [p | 0; Q; 0 | Jp]
    'C': Eq. (eq:Tc)   T_C = [q | c_a^T; C^T; c_b^T | Jq]
    'F': Eq. (eq:Tf)   T_F = [q | c_a^T; F^H; c_b^T | Jq]
    'P': F^H (Eq. (eq:permat)),  'R': C^T (Eq. (eq:refm)) -- classical cases.
    'PH': the Hartley matrix H (real, orthonormal, H = H^{-1}): for a symmetric
          PSF the circulant of the periodic conditions has real eigenvalues with
          z(theta_k) = z(theta_{n-k}), so H diagonalises it as F^H does.
    """
    if family == "P":
        return dft_matrix(n).conj().T
    if family == "PH":
        return hartley_matrix(n)
    if family == "R":
        return dct2_matrix(n).T
    if family == "F4":                                   # reading R17
        N = n - 4
        Q1, Q2 = quartic_border_columns(n, fourier4_grid)
        x, a, b = fourier4_grid(n)
        j = np.arange(N)
        T = np.zeros((n, n), dtype=np.complex128)
        T[:, 0], T[:, 1] = Q1, Q2
        T[:, n - 2], T[:, n - 1] = Q2[::-1], Q1[::-1]
        T[:, 2:N + 2] = np.exp(1j * np.outer(x, j)) / np.sqrt(N)   # the columns of F^H, extended
        return T
    if family == "C4":                                   # reading R16
        N = n - 4
        Q1, Q2 = quartic_border_columns(n)
        x, a, b = quartic_grid(n)
        j = np.arange(N)
        scale = np.sqrt((2.0 - (j == 0)) / N)
        T = np.zeros((n, n))
        T[:, 0], T[:, 1] = Q1, Q2
        T[:, n - 2], T[:, n - 1] = Q2[::-1], Q1[::-1]
        T[:, 2:N + 2] = scale[None, :] * np.cos(np.outer(x, j))   # cos(j x) on the extended grid
        return T
    if family == "S3":                                   # reading R6
        N = n - 4
        L1, L2 = cubic_border_columns(n)
        Q = dst1_matrix(N)
        T = np.zeros((n, n))
        T[:, 0], T[:, 1] = L1, L2
        T[:, n - 2], T[:, n - 1] = L2[::-1], L1[::-1]
        T[2:N + 2, 2:N + 2] = Q
        T[0, 2:N + 2] = -Q[0, :]                          # sin at x_{-1} = -sin at x_1
        T[n - 1, 2:N + 2] = -Q[N - 1, :]                  # sin at x_{N+2} = -sin at x_N
        return T
    N = n - 2
    v = border_vector(family, n)
    J = flip(n)
    dtype = np.complex128 if family == "F" else np.float64
    T = np.zeros((n, n), dtype=dtype)
    T[:, 0] = v
    T[:, n - 1] = J @ v
    if family == "S":
        T[1:n - 1, 1:n - 1] = dst1_matrix(N)
    elif family == "C":
        x, a, b = extended_grid("C", n)
        j = np.arange(1, N + 1)
        scale = np.sqrt((2.0 - (j == 1)) / N)
        T[1:n - 1, 1:n - 1] = dct2_matrix(N).T
        T[0, 1:n - 1] = scale * np.cos((j - 1) * a)      # c_a
        T[n - 1, 1:n - 1] = scale * np.cos((j - 1) * b)  # c_b
    elif family == "F":
        x, a, b = extended_grid("F", n)
        j = np.arange(1, N + 1)
        T[1:n - 1, 1:n - 1] = dft_matrix(N).conj().T
        T[0, 1:n - 1] = np.exp(1j * (j - 1) * a) / np.sqrt(N)   # c_a
        T[n - 1, 1:n - 1] = np.exp(1j * (j - 1) * b) / np.sqrt(N)  # c_b
    else:
        raise ValueError(family)
    return T


# --------------------------------------------------------------------------
# Eigenvalues of A_X and of the smoothing operator
# --------------------------------------------------------------------------


def eigenvalues_1d(family: str, h: np.ndarray, n: int) -> np.ndarray:
    """d_t = z(-theta_t) (readings R3, R4) for every column t of T_X."""
    return symbol(h, -eigen_angles(family, n))


def eigenvalues_2d(family: str, h: np.ndarray, n0: int, n1: int) -> np.ndarray:
    """d[t0, t1] = z(-theta_t0, -theta_t1) on the tensor grid (Sec. 6, 3-step algorithm).

    With a border index on one axis the angle there is 0, so the value is the
    1D symbol of the PSF summed along that axis -- the "edge" eigenvalues of
    step 2; interior indices are step 3.
    """
    return symbol2(h, -eigen_angles(family, n0), -eigen_angles(family, n1))


def laplacian_angles_1d(family: str, n: int) -> np.ndarray:
    """s(theta) = 2 - 2 cos(theta) on the family's grid (Sec. 4, after Eq. (eq:L))."""
    return 2.0 - 2.0 * np.cos(eigen_angles(family, n))


def smoothing_1d(family: str, n: int, L: str) -> np.ndarray:
    """Eigenvalues s of L = I ('I') or of the Laplacian L_X ('lap')."""
    if L == "I":
        return np.ones(n)
    return laplacian_angles_1d(family, n)


def smoothing_2d(family: str, n0: int, n1: int, L: str) -> np.ndarray:
    """L = I -> 1; Laplacian -> s(t0) + s(t1) (Kronecker sum, reading R8)."""
    if L == "I":
        return np.ones((n0, n1))
    return laplacian_angles_1d(family, n0)[:, None] + laplacian_angles_1d(family, n1)[None, :]


# --------------------------------------------------------------------------
# Blurring matrices
# --------------------------------------------------------------------------


def blur_matrix_spectral(family: str, h: np.ndarray, n: int) -> np.ndarray:
    """A_X(z) = T_X diag(d) T_X^{-1}  (Eq. (eq:jcf), (eq:Ac), (eq:Af); (eq:permat), (eq:refm))."""
    T = transform_matrix(family, n)
    d = eigenvalues_1d(family, h, n)
    return T @ np.diag(d) @ np.linalg.inv(T)


def bc_matrix(h: np.ndarray, n: int, rule: str) -> np.ndarray:
    """Transform-free blurring matrix: g_i = sum_j h_j f_{i-j} with f extended outside 1..n.

    rule: 'periodic'      f_{1-j} = f_{n+1-j},    f_{n+j} = f_j          (Sec. 2.1)
          'reflective'    f_{1-j} = f_j,          f_{n+j} = f_{n+1-j}    (Sec. 2.1)
          'antireflective' f_{1-j} = 2 f_1 - f_{j+1}, f_{n+j} = 2 f_n - f_{n-j} (Sec. 2.2)
          'odd'           f_0 = f_{n+1} = 0, f_{-j} = -f_j, f_{n+1+j} = -f_{n+1-j}
                          (the sine / tau extension of the trigonometric block of T)
          'zero'          f = 0 outside the field of view
    Requires 2m+1 <= n so that one reflection suffices.
    """
    h = np.asarray(h, dtype=np.float64)
    m = (len(h) - 1) // 2
    A = np.zeros((n, n))
    for i in range(1, n + 1):
        for j in range(-m, m + 1):
            hj = h[j + m]
            k = i - j
            if 1 <= k <= n:
                A[i - 1, k - 1] += hj
                continue
            if rule == "zero":
                continue
            if rule == "periodic":
                A[i - 1, (k - 1) % n] += hj
            elif rule == "reflective":
                kk = 1 - k if k < 1 else 2 * n + 1 - k
                A[i - 1, kk - 1] += hj
            elif rule == "antireflective":
                if k < 1:      # f_k = 2 f_1 - f_{2-k}
                    A[i - 1, 0] += 2 * hj
                    A[i - 1, 2 - k - 1] -= hj
                else:          # f_k = 2 f_n - f_{2n-k}
                    A[i - 1, n - 1] += 2 * hj
                    A[i - 1, 2 * n - k - 1] -= hj
            elif rule == "odd":
                if k == 0 or k == n + 1:
                    continue
                kk = -k if k < 0 else 2 * (n + 1) - k
                A[i - 1, kk - 1] -= hj
            else:
                raise ValueError(rule)
    return A


def extension_matrix(family: str, n: int) -> np.ndarray:
    """n x N matrix E that extends the N-point trigonometric block of T_X by one
    sample at each end "by continuity" (Sec. 3, remark before Sec. 3.1).

    'C': rows 1 and n copy interior rows 1 and N (half-sample reflection).
    'F': rows 1 and n copy interior rows N and 1 (periodic wrap).
    'S': rows 1 and n are zero (the sine vanishes at x_0 and x_{n-1}).
    """
    if family == "S3":                                   # odd extension by two samples
        N = n - 4
        E = np.zeros((n, N))
        E[2:N + 2, :] = np.eye(N)
        E[0, 0] = -1.0
        E[n - 1, N - 1] = -1.0
        return E
    if family == "F4":                                   # periodic wrap by two samples
        N = n - 4
        E = np.zeros((n, N))
        E[2:N + 2, :] = np.eye(N)
        E[0, N - 2] = E[1, N - 1] = 1.0
        E[n - 2, 0] = E[n - 1, 1] = 1.0
        return E
    if family == "C4":                                   # half-sample reflection by two samples
        N = n - 4
        E = np.zeros((n, N))
        E[2:N + 2, :] = np.eye(N)
        E[0, 1] = E[1, 0] = 1.0
        E[n - 2, N - 1] = E[n - 1, N - 2] = 1.0
        return E
    N = n - 2
    E = np.zeros((n, N))
    E[1:n - 1, :] = np.eye(N)
    if family == "C":
        E[0, 0] = 1.0
        E[n - 1, N - 1] = 1.0
    elif family == "F":
        E[0, N - 1] = 1.0
        E[n - 1, 0] = 1.0
    elif family != "S":
        raise ValueError(family)
    return E


def blur_matrix_bcfree(family: str, h: np.ndarray, n: int) -> np.ndarray:
    """A_X rebuilt with no transform at all, from two requirements the paper states:

    (i) on the extended trigonometric block, A_X acts as the order-(n-2) matrix of
        the classical BC that the block diagonalises (reflective for 'C',
        periodic for 'F', the odd/tau extension for 'S'): A_X E = E A_N;
    (ii) sampled polynomials of the preserved degree (quadratics for 'C', 'F';
        linear for 'S'; cubics for 'S3'; quartics for 'C4') are eigenvectors with
        eigenvalue z(0) (Sec. 3.1, 3.2, Remark 2; readings R6, R16).
    The polynomials are sampled as monomials on the integer grid, deliberately
    unlike the paper's q and p.  A_X = [z0 P_L | E A_N | z0 P_R] B^{-1} with
    B = [P_L | E | P_R].
    """
    E = extension_matrix(family, n)
    N = E.shape[1]
    rule = {"C": "reflective", "F": "periodic", "S": "odd", "S3": "odd", "C4": "reflective",
            "F4": "periodic"}[family]
    AN = bc_matrix(h, N, rule)
    z0 = float(np.sum(h))
    t = np.arange(n, dtype=np.float64) / n
    if family == "S":
        P = [np.ones(n), t]                     # span{1, x} = linear functions
    elif family == "S3":
        P = [np.ones(n), t, t * t, t ** 3]      # cubics
    elif family in ("C4", "F4"):
        P = [t, t * t, t ** 3, t ** 4]          # with the constant in range(E): quartics
    else:
        P = [t * t, t]                          # with the constant in range(E): quadratics
    B = np.column_stack(P + [E])
    AB = np.column_stack([z0 * v for v in P] + [E @ AN])
    return AB @ np.linalg.inv(B)


# --------------------------------------------------------------------------
# The method in 1D: reblurred Tikhonov (Sec. 4.1) and GCV (Sec. 4.2)
# --------------------------------------------------------------------------


def analysis_1d(family: str, g: np.ndarray) -> np.ndarray:
    """ghat = T_X^{-1} g by dense LU (Eq. (eq:freg)); g may be (n,) or (n, k)."""
    T = transform_matrix(family, g.shape[0])
    return np.linalg.solve(T, g)


def synthesis_1d(family: str, c: np.ndarray) -> np.ndarray:
    """y = T_X c (dense product)."""
    return transform_matrix(family, c.shape[0]) @ c


def filter_factors(d: np.ndarray, s: np.ndarray, mu: float) -> np.ndarray:
    """Phi D^{-1} = conj(d) / (|d|^2 + mu |s|^2)   (Eq. (eq:freg))."""
    return np.conj(d) / (np.abs(d) ** 2 + mu * np.abs(s) ** 2)


def gcv_sums(ghat: np.ndarray, d: np.ndarray, s: np.ndarray, mus: np.ndarray):
    """Numerator and denominator of Eq. (eq:gcv2)/(eq:mugcv) for every mu:

    sigma_i = |s_i|^2 / (|d_i|^2 + mu |s_i|^2),
    num(mu) = sum_i |sigma_i ghat_i|^2,  den(mu) = sum_i sigma_i.
    Arrays of any shape (all spectral indices are summed).
    """
    a2 = np.abs(d.ravel()) ** 2
    s2 = np.abs(s.ravel()) ** 2
    e2 = np.abs(ghat.ravel()) ** 2
    num = np.empty(len(mus))
    den = np.empty(len(mus))
    for k, mu in enumerate(mus):
        sig = s2 / (a2 + mu * s2)
        num[k] = np.sum(sig * sig * e2)
        den[k] = np.sum(sig)
    return num, den


def gcv_curve(ghat, d, s, mus) -> np.ndarray:
    """G(mu) = num/den^2 for every mu of the grid (Eq. (eq:mugcv))."""
    num, den = gcv_sums(ghat, d, s, mus)
    return num / den ** 2


def gcv_argmin(G: np.ndarray) -> int:
    """Index of the smallest G; ties -> lowest index (reading R10)."""
    return int(np.argmin(G))


def tikhonov_normal_equations_1d(family: str, h: np.ndarray, g: np.ndarray,
                                 L: str, mu: float) -> np.ndarray:
    """f_reg from the reblurred normal equations (A' A + mu L' L) f = A' g
    (Eq. (eq:nerebl)), all matrices dense and multiplied out, solved by LU.

    A' is the matrix of the same boundary model for the PSF rotated by 180
    degrees (Sec. 4.1); L is the same model's Laplacian (Eq. (eq:L) and its
    C/F analogues), or I.
    """
    n = g.shape[0]
    A = blur_matrix_spectral(family, h, n)
    Ar = blur_matrix_spectral(family, np.asarray(h)[::-1], n)
    if L == "I":
        Lm = np.eye(n)
    else:
        Lm = blur_matrix_spectral(family, np.array([-1.0, 2.0, -1.0]), n)
    M = Ar @ A + mu * (Lm @ Lm)   # L is its own 180-degree rotation
    f = np.linalg.solve(M, Ar @ g)
    return f.real if np.isrealobj(g) else f


def deblur_1d(family: str, h: np.ndarray, g: np.ndarray, L: str, mus: np.ndarray):
    """The whole 1D method on one signal.

    ghat = T_X^{-1} g (dense LU); G(mu) for every mu (Eq. (eq:mugcv));
    mu* = grid argmin; f = T_X diag(conj(d)/(|d|^2 + mu* |s|^2)) ghat (Eq. (eq:freg)).
    Returns (f, G, index of mu*, ghat).
    """
    n = g.shape[0]
    ghat = analysis_1d(family, g)
    d = eigenvalues_1d(family, h, n)
    s = smoothing_1d(family, n, L)
    G = gcv_curve(ghat, d, s, mus)
    k = gcv_argmin(G)
    f = synthesis_1d(family, filter_factors(d, s, mus[k]) * ghat)
    return f.real, G, k, ghat


def gcv_exact_1d(family: str, h: np.ndarray, g: np.ndarray, L: str,
                 mus: np.ndarray) -> np.ndarray:
    """The exact GCV functional of Eq. (eq:gcv), from dense matrices:
    ||g - A f_mu||^2 / trace(I - A R_mu)^2 with R_mu = (A'A + mu L'L)^{-1} A'.
    """
    n = g.shape[0]
    A = blur_matrix_spectral(family, h, n)
    Ar = blur_matrix_spectral(family, np.asarray(h)[::-1], n)
    Lm = np.eye(n) if L == "I" else blur_matrix_spectral(family, np.array([-1.0, 2.0, -1.0]), n)
    out = np.empty(len(mus))
    for k, mu in enumerate(mus):
        R = np.linalg.solve(Ar @ A + mu * (Lm @ Lm), Ar)
        r = g - A @ (R @ g)
        tr = np.trace(np.eye(n) - A @ R)
        out[k] = np.linalg.norm(r) ** 2 / abs(tr) ** 2
    return out


# --------------------------------------------------------------------------
# The method in 2D: tensor-product transform (Sec. 6), separable dense mode
# --------------------------------------------------------------------------


def analysis_2d(family: str, g: np.ndarray) -> np.ndarray:
    """Ghat = (T0^{-1} (x) T1^{-1}) g: T1^{-1} on every row, then T0^{-1} on every column.

    Each 1D inverse is a dense LU solve with the dense T of that axis.
    """
    n0, n1 = g.shape
    T0 = transform_matrix(family, n0)
    T1 = transform_matrix(family, n1)
    rows = np.linalg.solve(T1, g.T).T           # T1^{-1} applied to each row
    return np.linalg.solve(T0, rows)            # T0^{-1} applied to each column


def synthesis_2d(family: str, c: np.ndarray) -> np.ndarray:
    """y = (T0 (x) T1) c = T0 c T1^T."""
    n0, n1 = c.shape
    return transform_matrix(family, n0) @ c @ transform_matrix(family, n1).T


def deblur_2d(family: str, h: np.ndarray, g: np.ndarray, L: str, mus: np.ndarray):
    """The whole 2D method on one image (separable dense mode).

    Returns (f, G, index of mu*, Ghat).
    """
    n0, n1 = g.shape
    ghat = analysis_2d(family, g)
    d = eigenvalues_2d(family, h, n0, n1)
    s = smoothing_2d(family, n0, n1, L)
    G = gcv_curve(ghat, d, s, mus)
    k = gcv_argmin(G)
    f = synthesis_2d(family, filter_factors(d, s, mus[k]) * ghat)
    return f.real, G, k, ghat


def blur_matrix_2d_spectral(family: str, h: np.ndarray, n0: int, n1: int) -> np.ndarray:
    """Dense (n0 n1) x (n0 n1) matrix (T0 (x) T1) diag(d) (T0 (x) T1)^{-1}, row-major vec.

    Small sizes only; used to pin the separable mode.
    """
    T = np.kron(transform_matrix(family, n0), transform_matrix(family, n1))
    d = eigenvalues_2d(family, h, n0, n1).ravel()
    return T @ np.diag(d) @ np.linalg.inv(T)


def bc_matrix_2d(h: np.ndarray, n0: int, n1: int, rule: str) -> np.ndarray:
    """2D transform-free blurring matrix: g[i0,i1] = sum h[j0,j1] f[i0-j0, i1-j1] with the
    1D extension ``rule`` applied independently on each axis (row-major vec)."""
    h = np.asarray(h, dtype=np.float64)
    m0, m1 = (h.shape[0] - 1) // 2, (h.shape[1] - 1) // 2
    A = np.zeros((n0 * n1, n0 * n1))
    for j0 in range(-m0, m0 + 1):
        for j1 in range(-m1, m1 + 1):
            # a single tap is a shift on each axis; the 2D shift is their Kronecker product
            s0 = bc_matrix(_tap(j0, m0), n0, rule)
            s1 = bc_matrix(_tap(j1, m1), n1, rule)
            A += h[j0 + m0, j1 + m1] * np.kron(s0, s1)
    return A


def _tap(j: int, m: int) -> np.ndarray:
    e = np.zeros(2 * m + 1)
    e[j + m] = 1.0
    return e


def rre(f_true: np.ndarray, f: np.ndarray) -> float:
    """Relative restoration error ||f - f_reg|| / ||f||  (Sec. 5)."""
    return float(np.linalg.norm(f_true - f) / np.linalg.norm(f_true))
