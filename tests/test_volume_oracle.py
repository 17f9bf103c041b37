"""Pins of the 3D oracle (oracle/volume_oracle.py), independent of its own
arithmetic: the Kronecker product of the 1D transforms, the transform-free
3D blurring matrix of the classical rule on the extended interior, preserved
tensor-product polynomials, and the dense reblurred normal equations."""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from oracle import volume_oracle as V
from paper_0906_2704_gb300 import synth

FAMS = ["S", "C", "F", "S3"]


def _psf3(fam, p=3, seed=0):
    rng = np.random.default_rng(seed)
    if fam == "F":                                  # nonsymmetric
        h = rng.uniform(0.2, 1.0, (p, p, p))
    else:                                           # symmetric on every axis
        a = synth.gaussian_psf_1d(0.9, p)
        b = synth.gaussian_psf_1d(0.7, p)
        c = synth.gaussian_psf_1d(1.1, p)
        h = np.einsum("i,j,k->ijk", a, b, c) * (1 + 0.3 * np.einsum("i,j,k->ijk", a[::-1] * a, b, c))
        h = (h + h[::-1] + h[:, ::-1] + h[:, :, ::-1] + h[::-1, ::-1] + h[::-1, :, ::-1]
             + h[:, ::-1, ::-1] + h[::-1, ::-1, ::-1])
    return h / h.sum()


def _dense(fam, h, n):
    T = np.kron(np.kron(O.transform_matrix(fam, n[0]), O.transform_matrix(fam, n[1])), O.transform_matrix(fam, n[2]))
    d = V.eigenvalues_3d(fam, h, *n).ravel()
    return T, T @ np.diag(d) @ np.linalg.inv(T)


def test_symbol3_brute_force():
    h = _psf3("F", 3, 1)
    t = [np.array([0.0, 0.5]), np.array([-1.2]), np.array([0.3, 2.2, 0.0])]
    ref = np.zeros((2, 1, 3), dtype=complex)
    for a in range(2):
        for b in range(1):
            for c in range(3):
                for j0 in range(-1, 2):
                    for j1 in range(-1, 2):
                        for j2 in range(-1, 2):
                            ref[a, b, c] += h[j0 + 1, j1 + 1, j2 + 1] * np.exp(
                                1j * (j0 * t[0][a] + j1 * t[1][b] + j2 * t[2][c]))
    assert np.allclose(V.symbol3(h, *t), ref, atol=1e-14)


@pytest.mark.parametrize("fam", FAMS)
def test_transforms_are_the_kronecker_product(fam):
    n = (6, 7, 9) if fam != "S3" else (8, 9, 10)
    g = np.random.default_rng(3).standard_normal(n)
    T = np.kron(np.kron(O.transform_matrix(fam, n[0]), O.transform_matrix(fam, n[1])), O.transform_matrix(fam, n[2]))
    gh = V.analysis_3d(fam, g)
    assert np.allclose(T @ gh.ravel(), g.ravel(), atol=1e-10)
    assert np.allclose(V.synthesis_3d(fam, gh).real, g, atol=1e-10)


@pytest.mark.parametrize("fam,rule", [("F", "periodic"), ("C", "reflective"), ("S", "odd"), ("S3", "odd")])
def test_interior_is_the_classical_3d_rule_and_polynomials_are_preserved(fam, rule):
    """A_X^(3) = T (diag d) T^{-1} acts on the extended interior as the transform-free
    3D matrix of the classical rule (a sum over taps of Kronecker products of 1D
    shifts), and preserves tensor products of preserved 1D polynomials."""
    n = (6, 7, 8) if fam != "S3" else (8, 8, 9)
    h = _psf3(fam)
    T, A = _dense(fam, h, n)
    tol = max(1e-12, 1e-16 * np.linalg.cond(T))          # degree 3's T is badly conditioned (reading R6)
    Es = [O.extension_matrix(fam, m) for m in n]
    E = np.kron(np.kron(Es[0], Es[1]), Es[2])
    Ns = [e.shape[1] for e in Es]
    B = np.zeros((np.prod(Ns), np.prod(Ns)))
    for j0 in range(3):
        for j1 in range(3):
            for j2 in range(3):
                tap = [np.eye(3)[j] for j in (j0, j1, j2)]
                sh = [O.bc_matrix(tap[a], Ns[a], rule) for a in range(3)]
                B += h[j0, j1, j2] * np.kron(np.kron(sh[0], sh[1]), sh[2])
    assert np.abs(A @ E - E @ B).max() < tol
    deg = {"S": 1, "C": 2, "F": 2, "S3": 3}[fam]
    t0 = np.arange(n[0])[:, None, None] / 3.0
    t1 = np.arange(n[1])[None, :, None] / 4.0
    t2 = np.arange(n[2])[None, None, :] / 5.0
    u = (sum(t0 ** a for a in range(deg + 1)) * sum((-0.7 * t1) ** a for a in range(deg + 1))
         * sum((0.4 * t2) ** a for a in range(deg + 1)))
    assert np.abs(A @ u.ravel() - u.ravel()).max() < max(1e-9, 100 * tol)
    # the next degree on one axis is not preserved (the pin has teeth)
    w = (t0 ** (deg + 1)) * np.ones((1, n[1], n[2]))
    assert np.abs(A @ w.ravel() - w.ravel()).max() > 1e-4


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("L", ["I", "lap"])
def test_filter_equals_dense_normal_equations(fam, L):
    n = (5, 6, 7) if fam != "S3" else (8, 8, 8)
    h = _psf3(fam, 3, 2)
    g = np.random.default_rng(4).standard_normal(n)
    mu = 0.03
    T, A = _dense(fam, h, n)
    Ar = _dense(fam, h[::-1, ::-1, ::-1], n)[1]
    lap7 = np.zeros((3, 3, 3))
    lap7[1, 1, 1] = 6.0
    for ax in range(3):
        idx = [1, 1, 1]
        for v in (0, 2):
            idx[ax] = v
            lap7[tuple(idx)] = -1.0
    Lm = np.eye(np.prod(n)) if L == "I" else _dense(fam, lap7, n)[1]
    fn = np.linalg.solve(Ar @ A + mu * Lm @ Lm, Ar @ g.ravel()).real.reshape(n)
    d = V.eigenvalues_3d(fam, h, *n)
    s = V.smoothing_3d(fam, *n, L)
    fs = V.synthesis_3d(fam, O.filter_factors(d, s, mu) * V.analysis_3d(fam, g)).real
    tol = max(1e-8, 1e-15 * np.linalg.cond(T))
    assert np.abs(fs - fn).max() < tol * max(1.0, np.abs(fn).max())
