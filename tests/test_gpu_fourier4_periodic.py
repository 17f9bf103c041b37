"""GPU parity, through the C ABI, of the two families for a nonsymmetric PSF that
run on the FFT path besides FOURIER:
  fourier4  degree 4, Fourier basis (reading R17: the construction of Sec. 3.2 with
            two border columns per side, DFT of order n-4), FP64 only;
  periodic  the classical periodic conditions (Sec. 2, Eq. (eq:permat)): T = F^H,
            the unitary DFT of order n, no border columns, FP64 and FP32;
against the oracle's families 'F4' and 'P' (dense T, LU solves).

Bounds (as for degree 4): every bound that involves the analysis T_X^{-1} scales
with cond(T) (the product over axes in 2D; 1 for periodic)
  eigenvalues            FP64 1e-12 of max; FP32 1e-6 per entry plus a floor
  analysis               max(1e-10 | 1e-5, 64 eps cond(T)) of the largest entry
  G on identical inputs  1e-10 | 1e-5 relative, every mu (no transform involved)
  argmin                 equal, or an index whose oracle G is within tolerance of the minimum
  filter + synthesis     max(flat, 64 eps rb ||T||_2 ||X||_2) on identical inputs
  whole path             the analysis error, at most 64 eps cond(T) max|ghat|, magnified
                         by the filter (kappa) and ||T||_2
and closed forms that need no oracle: with a nonsymmetric PSF the degree-4 Fourier
family returns a sampled quartic unchanged under the Laplacian for every mu
(A p = p, L p = 0); the periodic family blurs a 2D complex exponential of a grid
frequency into itself times z(-theta).
"""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth
import parity_utils as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402

TOL = {"fp64": 1e-10, "fp32": 1e-5}
EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
LETTER = {"fourier4": "F4", "periodic": "P"}
DEG = {"fourier4": 4, "periodic": 0}


def _dt(prec):
    return (np.float64, torch.float64) if prec == "fp64" else (np.float32, torch.float32)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _round(x, dt):
    if np.iscomplexobj(x):
        return x.real.astype(dt).astype(np.float64) + 1j * x.imag.astype(dt).astype(np.float64)
    return x.astype(dt).astype(np.float64)


def _spec_dev(a, dt):
    return _dev(np.stack([a.real, a.imag], axis=-1), dt)


def _spec_np(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def _cond(F, shape):
    out = 1.0
    for n in shape:
        out *= np.linalg.cond(O.transform_matrix(F, n))
    return out


CASES = [("fourier4", "fp64", 1, (13,), 5), ("fourier4", "fp64", 1, (40,), 7),
         ("fourier4", "fp64", 2, (12, 15), (5, 5)), ("fourier4", "fp64", 2, (20, 17), (5, 5)),
         ("periodic", "fp64", 1, (13,), 5), ("periodic", "fp64", 1, (64,), 9),
         ("periodic", "fp64", 2, (12, 15), (5, 5)), ("periodic", "fp64", 2, (33, 40), (7, 7)),
         ("periodic", "fp32", 1, (40,), 7), ("periodic", "fp32", 2, (12, 15), (5, 5)),
         ("periodic", "fp32", 2, (33, 40), (7, 7))]


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam,prec,ndim,n,taps", CASES)
def test_steps_and_whole_path(fam, prec, ndim, n, taps, L):
    F = LETTER[fam]
    dt, tdt = _dt(prec)
    eps, tol = EPS[prec], TOL[prec]
    h = P.psf_for(F, ndim, taps)
    h = _round(h / h.sum(), dt)
    batch = 3
    g, _ = P.problems(ndim, n, h, batch, 5)
    g = _round(g, dt)
    mus = synth.mu_grid(16, 1e-6, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, DEG[fam], mus, L=L, prec=prec, family=fam, psf_symmetric=False,
                     batch=batch)
    assert plan.family == fam and plan.spec_complex
    S = plan.spec_elems
    assert S == len(P.stored_t(F, n[-1], True)) * (n[0] if ndim == 2 else 1)
    c = _cond(F, n)
    sT = P.sigma(F, n)
    rb = 16.0 * P.log2_fft(F, n) + 2.0 * sum(np.sqrt(v) for v in n)
    orc = [P.oracle_steps(F, ndim, h, g[b], L, mus) for b in range(batch)]

    # eigenvalues and analysis from the inputs
    d_d = torch.empty((1, S, 2), dtype=tdt, device="cuda")
    plan.eigenvalues(_dev(h[None], dt), d_d)
    gh_d = torch.empty((batch, S, 2), dtype=tdt, device="cuda")
    plan.analysis(_dev(g, dt), gh_d)
    dg, gh = _spec_np(d_d)[0], _spec_np(gh_d)
    dref = P.to_layout(F, orc[0][1]).reshape(-1)
    floor = 64 * 2.0 ** -53 * np.abs(h).sum()
    if prec == "fp64":
        assert np.abs(dg - dref).max() <= max(1e-12 * np.abs(dref).max(), floor), "eigenvalues"
    else:
        assert np.all(np.abs(dg - dref) <= 1e-6 * np.abs(dref) + floor), "eigenvalues"
    atol = max(tol, 64 * eps * c)
    for b in range(batch):
        ref = P.to_layout(F, orc[b][0]).reshape(-1)
        err = np.abs(gh[b] - ref).max() / np.abs(ref).max()
        assert err <= atol, f"analysis item {b}: {err:.3e} > {atol:.3e}"

    # GCV, filter + synthesis and synthesis on identical (rounded oracle) inputs;
    # the stored half stands for the whole spectrum of a real image
    gin = np.stack([_round(P.to_layout(F, orc[b][0]).reshape(-1), dt) for b in range(batch)])
    din = _round(P.to_layout(F, orc[0][1]).reshape(-1), dt)[None]
    G_d = torch.empty((batch, len(mus)), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.gcv(_spec_dev(gin, dt), _spec_dev(din, dt), G_d, mi_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    shape = n if ndim == 2 else (n[0],)
    mi_fix = np.array([orc[b][4] for b in range(batch)], dtype=np.int32)
    f_d = torch.empty((batch,) + shape, dtype=tdt, device="cuda")
    plan.filter_synthesis(_spec_dev(gin, dt), _spec_dev(din, dt), _dev(mi_fix, np.int32), f_d)
    f = f_d.cpu().numpy()
    for b in range(batch):
        ghat_o, d_o, s_o, G_o, k_o = orc[b]
        # the oracle's G on the rounded inputs: round the full spectrum entrywise
        full_g, full_d = _round(ghat_o, dt), _round(d_o, dt)
        Gref = O.gcv_curve(full_g, full_d, s_o, mus)
        gerr = np.max(np.abs(G[b] - Gref) / np.abs(Gref))
        assert gerr <= tol + 8 * eps, f"G item {b}: {gerr:.3e}"
        kref = O.gcv_argmin(Gref)
        assert mi[b] == kref or Gref[mi[b]] <= (1 + tol) * Gref.min(), "argmin"
        X = O.filter_factors(full_d, s_o, mus[mi_fix[b]]) * full_g
        fref = P.oracle_filtered(F, ndim, full_g, full_d, s_o, mus[mi_fix[b]])
        bound = max(tol * np.abs(fref).max(), 64 * eps * rb * sT * np.linalg.norm(X))
        assert np.abs(f[b] - fref).max() <= bound, f"filter+synthesis item {b}"

    # synthesis of the analysis gives g back
    y_d = torch.empty((batch,) + shape, dtype=tdt, device="cuda")
    plan.synthesis(gh_d, y_d)
    yerr = np.abs(y_d.cpu().numpy() - g).max() / np.abs(g).max()
    assert yerr <= max(tol, 64 * eps * c * rb), f"round trip {yerr:.3e}"

    # the one-call deblur equals the step sequence bit for bit
    f1 = torch.empty((batch,) + shape, dtype=tdt, device="cuda")
    m1 = torch.empty(batch, dtype=torch.int32, device="cuda")
    G1 = torch.empty((batch, len(mus)), dtype=torch.float64, device="cuda")
    plan.gcv(gh_d, d_d, G1, m1)
    plan.filter_synthesis(gh_d, d_d, m1, f1)
    f2 = torch.empty_like(f1)
    m2 = torch.empty_like(m1)
    G2 = torch.empty_like(G1)
    plan.deblur(_dev(g, dt), _dev(h[None], dt), f2, m2, G2)
    assert torch.equal(f1, f2) and torch.equal(m1, m2) and torch.equal(G1, G2)

    # the whole path from g against the oracle
    f2n, m2n = f2.cpu().numpy(), m2.cpu().numpy()
    for b in range(batch):
        ghat_o, d_o, s_o, G_o, k_o = orc[b]
        k = int(m2n[b])
        delta = 64 * eps * c * np.abs(ghat_o).max() * np.sqrt(ghat_o.size)
        kappa = P.amplification(d_o, s_o, mus[k])
        fo = P.oracle_filtered(F, ndim, ghat_o, d_o, s_o, mus[k])
        X = O.filter_factors(d_o, s_o, mus[k]) * ghat_o
        bound = max(tol * np.abs(fo).max(), 64 * eps * rb * sT * np.linalg.norm(X) + sT * kappa * delta)
        assert np.abs(f2n[b] - fo).max() <= bound, f"whole path item {b}"
        if prec == "fp64" and k != k_o:   # a different index only where the curves are within the error
            assert G_o[k] <= (1 + 1e-6) * G_o.min(), f"whole-path argmin {k} vs {k_o}"


@pytest.mark.parametrize("ndim,n", [(1, (14,)), (2, (12, 13))])
def test_fourier4_quartics_come_back_unchanged(ndim, n):
    """A_X of the degree-4 Fourier family preserves sampled quartics for a
    nonsymmetric PSF and the Laplacian annihilates them, so the reblurred Tikhonov
    solution with L = Laplacian returns them for every mu."""
    taps = 5 if ndim == 1 else (5, 5)
    h = P.psf_for("F4", ndim, taps)
    h = h / h.sum()
    t0 = np.linspace(-1.0, 1.5, n[0])
    p0 = 0.3 - 0.8 * t0 + 0.5 * t0 ** 2 + 0.7 * t0 ** 3 - 0.4 * t0 ** 4
    if ndim == 1:
        g = p0[None]
    else:
        t1 = np.linspace(0.2, 1.1, n[1])
        g = np.outer(p0, 1.0 - t1 + 0.3 * t1 ** 4)[None]
    mus = synth.mu_grid(8, 1e-4, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, 4, mus, L="lap", prec="fp64", family="fourier4", psf_symmetric=False)
    f_d = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    plan.deblur(_dev(g, np.float64), _dev(h[None], np.float64), f_d)
    err = np.abs(f_d.cpu().numpy() - g).max() / np.abs(g).max()
    assert err <= max(TOL["fp64"], 64 * EPS["fp64"] * _cond("F4", n)), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_blur_of_a_grid_exponential(prec):
    """Closed form of the periodic conditions: the circulant blur of
    exp(2 pi i (k0 i0 / n0 + k1 i1 / n1)) is the same exponential times
    z(-theta) (the symbol at the grid frequency), so the analysis of the real
    part of the blurred exponential has a single nonzero stored entry, z(-theta)
    sqrt(n0 n1) / 2 (its conjugate partner lies in the half that is not stored),
    and the eigenvalue stored there is z(-theta)."""
    dt, tdt = _dt(prec)
    n0, n1 = 12, 16
    h = _round(P.psf_for("P", 2, (5, 5)), dt)
    k0, k1 = 3, 5
    i0, i1 = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    e = np.exp(2j * np.pi * (k0 * i0 / n0 + k1 * i1 / n1))
    m = 2
    z = sum(h[j0 + m, j1 + m] * np.exp(-2j * np.pi * (k0 * j0 / n0 + k1 * j1 / n1))
            for j0 in range(-m, m + 1) for j1 in range(-m, m + 1))
    g = (z * e).real[None]
    mus = synth.mu_grid(4)
    plan = hobc.Plan(2, (n0, n1), h.shape, 0, mus, prec=prec, family="periodic", psf_symmetric=False)
    gh_d = torch.empty((1, plan.spec_elems, 2), dtype=tdt, device="cuda")
    plan.analysis(_dev(g, dt), gh_d)
    gh = _spec_np(gh_d)[0].reshape(n1 // 2 + 1, n0)            # [c][t0], c = t1
    tol = 1e-12 if prec == "fp64" else 2e-6
    scale = np.sqrt(n0 * n1) / 2                                   # unitary DFT of the real part
    assert abs(gh[k1, k0] - z * scale) <= tol * scale * 4
    gh[k1, k0] = 0
    assert np.abs(gh).max() <= tol * scale * 4
    d_d = torch.empty((1, plan.spec_elems, 2), dtype=tdt, device="cuda")
    plan.eigenvalues(_dev(h[None], dt), d_d)
    d = _spec_np(d_d)[0].reshape(n1 // 2 + 1, n0)
    assert abs(d[k1, k0] - z) <= tol * 4


def test_new_families_outside_the_plain_path_are_rejected():
    """The learned, binned and refined choices, the exact functional and the 3D
    plans do not take these families; FP32 degree 4 is refused (cond(T))."""
    mus = synth.mu_grid(8)
    for fam, deg, prec in (("fourier4", 4, "fp64"), ("periodic", 0, "fp32")):
        plan = hobc.Plan(2, (16, 16), (5, 5), deg, mus, prec=prec, family=fam, psf_symmetric=False)
        dt, tdt = _dt(prec)
        S = plan.spec_elems
        gh = torch.zeros((1, S, 2), dtype=tdt, device="cuda")
        mi = torch.zeros(1, dtype=torch.int32, device="cuda")
        for call in (lambda: plan.gcv_binned(gh, gh, mi), lambda: plan.gcv_exact(gh, gh,
                     torch.empty((1, len(mus)), dtype=torch.float64, device="cuda"), mi)):
            with pytest.raises(hobc.HobcError) as e:
                call()
            assert e.value.status == 2
        with pytest.raises(hobc.HobcError) as e:
            hobc.Volume((8, 10, 10), (3, 3, 3), deg, mus, prec=prec, family=fam, psf_symmetric=False)
        assert e.value.status == 2
    with pytest.raises(hobc.HobcError) as e:
        hobc.Plan(2, (16, 16), (5, 5), 4, mus, prec="fp32", family="fourier4", psf_symmetric=False)
    assert e.value.status == 2
