"""FP64 CPU oracle for the method on 3D arrays (Sec. 6, the multidimensional
case): the transform is the tensor product T_X^{(3)} = T_{X,n0} (x) T_{X,n1}
(x) T_{X,n2}, the eigenvalues are the 3D symbol on the tensor grid, and the
Laplacian is the Kronecker sum (reading R8 on three axes).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU leg,
never by the product path; it shares no code with the CUDA kernels.

Every axis is applied as the dense 1D matrix of hobc_oracle (solves for the
inverse).  parity status: pinned by tests/test_volume_oracle.py (transform
against the explicit Kronecker product; the spectral blur against the
transform-free matrix of the boundary rules on three axes; preserved
polynomials; the spectral filter against the dense reblurred normal
equations).
"""
from __future__ import annotations

import numpy as np

from oracle import hobc_oracle as O


def symbol3(h: np.ndarray, t0, t1, t2) -> np.ndarray:
    """z(t0, t1, t2) = sum h_{j0 j1 j2} exp(i (j0 t0 + j1 t1 + j2 t2)) on the grid
    t0 x t1 x t2 (Eq. (eq:symbol) on three axes); h[j0+m0, j1+m1, j2+m2] = h_{j0 j1 j2}."""
    h = np.asarray(h, dtype=np.float64)
    es = []
    for t, p in zip((t0, t1, t2), h.shape):
        m = (p - 1) // 2
        es.append(np.exp(1j * np.outer(np.atleast_1d(t), np.arange(-m, m + 1))))
    return np.einsum("aj,bk,cl,jkl->abc", es[0], es[1], es[2], h)


def eigenvalues_3d(family: str, h: np.ndarray, n0: int, n1: int, n2: int) -> np.ndarray:
    """d[t0, t1, t2] = z(-theta_t0, -theta_t1, -theta_t2) (readings R3, R4 on each axis)."""
    return symbol3(h, -O.eigen_angles(family, n0), -O.eigen_angles(family, n1), -O.eigen_angles(family, n2))


def smoothing_3d(family: str, n0: int, n1: int, n2: int, L: str) -> np.ndarray:
    """L = I -> 1; Laplacian -> s(t0) + s(t1) + s(t2) (Kronecker sum)."""
    if L == "I":
        return np.ones((n0, n1, n2))
    s = [O.laplacian_angles_1d(family, n) for n in (n0, n1, n2)]
    return s[0][:, None, None] + s[1][None, :, None] + s[2][None, None, :]


def _along(M: np.ndarray, x: np.ndarray, axis: int, solve: bool) -> np.ndarray:
    """Apply M (or M^{-1} by a dense solve) along one axis of a 3D array."""
    y = np.moveaxis(x, axis, 0)
    shp = y.shape
    y = y.reshape(shp[0], -1)
    y = np.linalg.solve(M, y) if solve else M @ y
    return np.moveaxis(y.reshape(shp), 0, axis)


def analysis_3d(family: str, g: np.ndarray) -> np.ndarray:
    """ghat = (T0 (x) T1 (x) T2)^{-1} g: a dense solve with T_a along every axis."""
    out = np.asarray(g, dtype=np.complex128 if family == "F" else np.float64)
    for ax in (2, 1, 0):
        out = _along(O.transform_matrix(family, out.shape[ax]), out, ax, True)
    return out


def synthesis_3d(family: str, c: np.ndarray) -> np.ndarray:
    """y = (T0 (x) T1 (x) T2) c."""
    out = np.asarray(c)
    for ax in (0, 1, 2):
        out = _along(O.transform_matrix(family, out.shape[ax]), out, ax, False)
    return out


def deblur_3d(family: str, h: np.ndarray, g: np.ndarray, L: str, mus: np.ndarray):
    """The whole method on one 3D array: returns (f, G, index of mu*, ghat)."""
    n0, n1, n2 = g.shape
    ghat = analysis_3d(family, g)
    d = eigenvalues_3d(family, h, n0, n1, n2)
    s = smoothing_3d(family, n0, n1, n2, L)
    G = O.gcv_curve(ghat, d, s, mus)
    k = O.gcv_argmin(G)
    f = synthesis_3d(family, O.filter_factors(d, s, mus[k]) * ghat)
    return f.real, G, k, ghat
