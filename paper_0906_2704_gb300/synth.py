"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds the *data model* only (Sec. 1, Eq. (eq:mod_cont): a true signal
blurred by a shift-invariant PSF, plus Gaussian noise).  It contains none of the
method's arithmetic: no boundary condition, no transform, no eigenvalue, no
Tikhonov filter and no GCV.  Both the CUDA path and the FP64 oracle receive the
arrays produced here as plain inputs.

Data model (stated once, used everywhere):
  * The true object lives on an *extended* grid: the field of view (n samples per
    axis) plus m samples on each side, m = PSF half-width.
  * The observation is the valid part of the discrete convolution
    g_i = sum_j h_j f_{i-j}, i in the field of view -- the rectangle-rule
    discretisation of Eq. (eq:mod_cont).  It is *not* generated with any of the
    boundary models under test, so every model has a genuine boundary error.
  * Noise: e ~ N(0, I), rescaled so that ||e|| = eta * ||g_clean||.

Workload recipes (sizes and distributions of the paper's experiments; the
paper's own signals and images exist only as figures, so these stand in):
  * ``signal_1d``  -- piecewise quadratic with 3 random breakpoints plus
    sin(2*pi*x*U[1,4]), the 1D experiments of Sec. 5.
  * ``image_2d``   -- 20 random polynomials of degree <= 2 on random rectangles
    plus a linear ramp, the image experiments of Sec. 6.1.
  * ``gaussian_psf_1d``, ``gaussian_psf_2d_separable``,
    ``gaussian_psf_2d_rotated`` -- Gaussian blurs (symmetric and nonsymmetric).
  * ``disk_psf`` -- out-of-focus blur (a uniform disk), as in the image
    experiments of Sec. 6.1; symmetric in each axis.
  * ``learned_set`` -- the training / inference problems of the learned choice
    of mu: images as above, disk PSFs of radius U[1.5, 5], noise level
    log-uniform in [1e-3, 3e-2].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_psf_1d",
    "gaussian_psf_2d_separable",
    "gaussian_psf_2d_rotated",
    "signal_1d",
    "image_2d",
    "blur_valid_1d",
    "blur_valid_2d",
    "add_noise",
    "mu_grid",
    "problem_1d",
    "problem_2d",
    "batch_uneven",
    "disk_psf",
    "learned_set",
]


def gaussian_psf_1d(sigma: float, taps: int) -> np.ndarray:
    """Symmetric Gaussian mask h_{-m..m} (taps = 2m+1), normalised to sum 1."""
    if taps % 2 != 1:
        raise ValueError("PSF length must be odd")
    m = taps // 2
    j = np.arange(-m, m + 1, dtype=np.float64)
    h = np.exp(-0.5 * (j / sigma) ** 2)
    return h / h.sum()


def gaussian_psf_2d_separable(sigma: float, taps: int) -> np.ndarray:
    """Outer product of two identical symmetric 1D Gaussians (sum 1)."""
    h = gaussian_psf_1d(sigma, taps)
    return np.outer(h, h)


def gaussian_psf_2d_rotated(sigma_x: float, sigma_y: float, angle_deg: float,
                            taps: int, offset_col: float = 0.0,
                            offset_row: float = 0.0) -> np.ndarray:
    """Anisotropic Gaussian, rotated, with its centre shifted: a nonsymmetric PSF.

    Array index [r, c] holds h_{r-m, c-m}; rows are the first image axis.
    """
    if taps % 2 != 1:
        raise ValueError("PSF size must be odd")
    m = taps // 2
    r, c = np.meshgrid(np.arange(-m, m + 1, dtype=np.float64),
                       np.arange(-m, m + 1, dtype=np.float64), indexing="ij")
    x = c - offset_col
    y = r - offset_row
    th = np.deg2rad(angle_deg)
    xr = np.cos(th) * x + np.sin(th) * y
    yr = -np.sin(th) * x + np.cos(th) * y
    h = np.exp(-0.5 * ((xr / sigma_x) ** 2 + (yr / sigma_y) ** 2))
    return h / h.sum()


def signal_1d(rng: np.random.Generator, length: int) -> np.ndarray:
    """Piecewise quadratic (3 random breakpoints) plus sin(2*pi*x*U[1,4]) on x in [0,1]."""
    x = np.linspace(0.0, 1.0, length)
    brk = np.sort(rng.uniform(0.1, 0.9, size=3))
    edges = np.concatenate([[-np.inf], brk, [np.inf]])
    f = np.zeros(length)
    for a, b in zip(edges[:-1], edges[1:]):
        c0, c1, c2 = rng.uniform(-1.0, 1.0, size=3)
        sel = (x >= a) & (x < b)
        f[sel] = c0 + c1 * x[sel] + c2 * x[sel] ** 2
    f += np.sin(2.0 * np.pi * x * rng.uniform(1.0, 4.0))
    return f


def image_2d(rng: np.random.Generator, rows: int, cols: int,
             pieces: int = 20) -> np.ndarray:
    """Sum of ``pieces`` random degree-<=2 polynomials on random rectangles plus a ramp."""
    y, x = np.meshgrid(np.linspace(0.0, 1.0, rows), np.linspace(0.0, 1.0, cols),
                       indexing="ij")
    a, b, c = rng.uniform(-1.0, 1.0, size=3)
    f = a + b * x + c * y
    for _ in range(pieces):
        r0, r1 = np.sort(rng.integers(0, rows, size=2))
        c0, c1 = np.sort(rng.integers(0, cols, size=2))
        r1 = max(r1, r0 + 1)
        c1 = max(c1, c0 + 1)
        k = rng.uniform(-1.0, 1.0, size=6)
        xs, ys = x[r0:r1, c0:c1], y[r0:r1, c0:c1]
        f[r0:r1, c0:c1] += (k[0] + k[1] * xs + k[2] * ys + k[3] * xs * xs
                            + k[4] * xs * ys + k[5] * ys * ys)
    return f


def blur_valid_1d(f_ext: np.ndarray, h: np.ndarray) -> np.ndarray:
    """g_i = sum_j h_j f_{i-j} over the field of view (len(f_ext) - 2m samples)."""
    return np.convolve(f_ext, h, mode="valid")


def blur_valid_2d(f_ext: np.ndarray, h: np.ndarray) -> np.ndarray:
    """2D analogue of :func:`blur_valid_1d` (true convolution, valid part)."""
    from scipy.signal import fftconvolve
    return fftconvolve(f_ext, h, mode="valid")


def add_noise(rng: np.random.Generator, g: np.ndarray, eta: float) -> np.ndarray:
    """g + e with e Gaussian and ||e|| = eta * ||g||."""
    e = rng.standard_normal(g.shape)
    return g + eta * np.linalg.norm(g) / np.linalg.norm(e) * e


def gaussian_psf_3d(sigmas, taps, offsets=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Product of three 1D Gaussians exp(-((j - o_a)/sigma_a)^2 / 2) on masks of the
    given odd sizes (nonsymmetric when an offset is nonzero), normalised to sum 1."""
    axes = []
    for s, p, o in zip(sigmas, taps, offsets):
        if p % 2 != 1:
            raise ValueError("PSF size must be odd")
        j = np.arange(-(p // 2), p // 2 + 1, dtype=np.float64)
        axes.append(np.exp(-0.5 * ((j - o) / s) ** 2))
    h = np.einsum("i,j,k->ijk", *axes)
    return h / h.sum()


def volume_3d(rng: np.random.Generator, n0: int, n1: int, n2: int, pieces: int = 12) -> np.ndarray:
    """Sum of ``pieces`` random degree-<=2 polynomials on random boxes plus a linear ramp."""
    z, y, x = np.meshgrid(np.linspace(0, 1, n0), np.linspace(0, 1, n1), np.linspace(0, 1, n2), indexing="ij")
    a = rng.uniform(-1.0, 1.0, size=4)
    f = a[0] + a[1] * x + a[2] * y + a[3] * z
    for _ in range(pieces):
        lo = [int(rng.integers(0, m)) for m in (n0, n1, n2)]
        hi = [min(m, l0 + 1 + int(rng.integers(0, m))) for l0, m in zip(lo, (n0, n1, n2))]
        sl = tuple(slice(l0, h0) for l0, h0 in zip(lo, hi))
        k = rng.uniform(-1.0, 1.0, size=7)
        xs, ys, zs = x[sl], y[sl], z[sl]
        f[sl] += k[0] + k[1] * xs + k[2] * ys + k[3] * zs + k[4] * xs * ys + k[5] * zs * zs + k[6] * xs * xs
    return f


def problem_3d(seed: int, n0: int, n1: int, n2: int, h: np.ndarray, eta: float, count: int = 1):
    """``count`` seeded 3D problems: the valid part of the blurred extended volume
    plus noise (the 3D form of the data model).  Returns (g[count, n0, n1, n2], f_true)."""
    from scipy.signal import fftconvolve
    rng = np.random.default_rng(seed)
    m = [p // 2 for p in h.shape]
    g = np.empty((count, n0, n1, n2))
    ft = np.empty_like(g)
    for i in range(count):
        f_ext = volume_3d(rng, n0 + 2 * m[0], n1 + 2 * m[1], n2 + 2 * m[2])
        g[i] = add_noise(rng, fftconvolve(f_ext, h, mode="valid"), eta)
        ft[i] = f_ext[m[0]:m[0] + n0, m[1]:m[1] + n1, m[2]:m[2] + n2]
    return g, ft


def mu_grid(k: int, lo: float = 1e-8, hi: float = 1.0) -> np.ndarray:
    """k log-spaced regularisation parameters, endpoints included."""
    if k == 1:
        return np.array([lo], dtype=np.float64)
    return 10.0 ** np.linspace(np.log10(lo), np.log10(hi), k)


def problem_1d(seed: int, n: int, h: np.ndarray, eta: float, count: int = 1):
    """``count`` seeded 1D problems: returns (g[count, n], f_true[count, n])."""
    rng = np.random.default_rng(seed)
    m = len(h) // 2
    g = np.empty((count, n))
    ft = np.empty((count, n))
    for i in range(count):
        f_ext = signal_1d(rng, n + 2 * m)
        g[i] = add_noise(rng, blur_valid_1d(f_ext, h), eta)
        ft[i] = f_ext[m:m + n]
    return g, ft


def problem_2d(seed: int, rows: int, cols: int, h: np.ndarray, eta: float,
               count: int = 1):
    """``count`` seeded 2D problems: returns (g[count, rows, cols], f_true[...])."""
    rng = np.random.default_rng(seed)
    m0, m1 = h.shape[0] // 2, h.shape[1] // 2
    g = np.empty((count, rows, cols))
    ft = np.empty((count, rows, cols))
    for i in range(count):
        f_ext = image_2d(rng, rows + 2 * m0, cols + 2 * m1)
        g[i] = add_noise(rng, blur_valid_2d(f_ext, h), eta)
        ft[i] = f_ext[m0:m0 + rows, m1:m1 + cols]
    return g, ft


def batch_uneven(seed: int, count: int, n_lo: int = 64, n_hi: int = 512, eta: float = 0.01):
    """``count`` square problems of uneven sizes (side log-uniform in [n_lo, n_hi]),
    each with its own isotropic Gaussian PSF (sigma ~ U[1, 4], 2*ceil(3 sigma)+1
    taps) and boundary degree uniform in {1, 2, 3}.

    Returns (items, g_list, h_list): items are (n, n, taps, taps, degree).
    """
    rng = np.random.default_rng(seed)
    items, gs, hs = [], [], []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        sigma = rng.uniform(1.0, 4.0)
        taps = 2 * int(np.ceil(3 * sigma)) + 1
        deg = int(rng.integers(1, 4))
        h1 = gaussian_psf_1d(sigma, taps)
        h = np.outer(h1, h1)
        m = taps // 2
        f_ext = image_2d(rng, n + 2 * m, n + 2 * m)
        # separable PSF: the valid 2D convolution is two valid 1D convolutions
        tmp = np.apply_along_axis(lambda v: np.convolve(v, h1, mode="valid"), 1, f_ext)
        gc = np.apply_along_axis(lambda v: np.convolve(v, h1, mode="valid"), 0, tmp)
        gs.append(add_noise(rng, gc, eta))
        hs.append(h)
        items.append((n, n, taps, taps, deg))
    return items, gs, hs


def disk_psf(radius: float) -> np.ndarray:
    """Uniform disk of the given radius on a (2 ceil(radius) + 1)^2 grid:
    h[r, c] = 1 where (r - m)^2 + (c - m)^2 <= radius^2, normalised to sum 1."""
    m = int(np.ceil(radius))
    j = np.arange(-m, m + 1, dtype=np.float64)
    h = ((j[:, None] ** 2 + j[None, :] ** 2) <= radius * radius).astype(np.float64)
    return h / h.sum()


def motion_defocus_psf(radius: float, length: float, angle_deg: float, taps: int) -> np.ndarray:
    """A nonsymmetric PSF: out-of-focus blur (a disk of ``radius``) combined with a
    one-sided linear motion of ``length`` pixels from the centre at ``angle_deg``
    (the path sampled every 1/8 pixel, spread bilinearly), in a taps x taps array
    (odd), normalised to sum 1."""
    m = taps // 2
    motion = np.zeros((taps, taps))
    a = np.deg2rad(angle_deg)
    for t in np.arange(0.0, length, 0.125):
        x, y = m + t * np.cos(a), m - t * np.sin(a)
        c0, r0 = int(np.floor(x)), int(np.floor(y))
        fx, fy = x - c0, y - r0
        for dr, wr in ((0, 1 - fy), (1, fy)):
            for dc, wc in ((0, 1 - fx), (1, fx)):
                motion[r0 + dr, c0 + dc] += wr * wc
    from scipy.signal import fftconvolve
    h = fftconvolve(motion, disk_psf(radius), mode="same")
    h = np.clip(h, 0.0, None)
    return h / h.sum()


def learned_set(seed: int, count: int, n: int, taps: int = 11, r_lo: float = 1.5, r_hi: float = 5.0,
                eta_lo: float = 1e-3, eta_hi: float = 3e-2):
    """``count`` n x n problems for the learned choice of mu, each with its own
    disk PSF (radius U[r_lo, r_hi], embedded centred in a taps x taps array so
    that one plan serves all) and noise level (log-uniform in [eta_lo, eta_hi]).

    Returns (g[count, n, n], f_true[count, n, n], h[count, taps, taps], eta[count]).
    """
    rng = np.random.default_rng(seed)
    m = taps // 2
    g = np.empty((count, n, n))
    ft = np.empty((count, n, n))
    hs = np.zeros((count, taps, taps))
    etas = np.empty(count)
    for i in range(count):
        r = rng.uniform(r_lo, min(r_hi, m))
        d = disk_psf(r)
        k = d.shape[0] // 2
        hs[i, m - k:m + k + 1, m - k:m + k + 1] = d
        eta = float(np.exp(rng.uniform(np.log(eta_lo), np.log(eta_hi))))
        f_ext = image_2d(rng, n + 2 * m, n + 2 * m)
        g[i] = add_noise(rng, blur_valid_2d(f_ext, hs[i]), eta)
        ft[i] = f_ext[m:m + n, m:m + n]
        etas[i] = eta
    return g, ft, hs, etas
