"""Parity of the continuous refinement of mu* (include/hobc_refine.h) with the
FP64 oracle (oracle/refine_oracle.py, oracle/hobc_oracle.py).

On identical inputs (the oracle's spectra rounded to the working precision go
to both sides, with the oracle's grid argmin as the starting index):
  mu*       inside the bracket of the grid neighbours, a value of the working
            precision, and as good as the oracle's: G(mu_gpu) <= (1 + 10 tol)
            G(mu_oracle), both evaluated by the oracle (a flat minimum admits
            several correct points, so G decides, not the point)
  G(mu*)    the reported value within tol of the oracle's G at that mu
  FP64      where the oracle's last round has a clear minimiser, the same point
Filter at given mu (hobc_filter_synthesis_mu): the oracle's f at the oracle's
own refined mu, within the elementwise bound of an FFT synthesis.
Whole path (hobc_deblur_refined): grid index equal to hobc_deblur's, mu* equal
to hobc_gcv_refine's on the plan's own spectra, f bit-equal to
hobc_filter_synthesis_mu at that mu.
"""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from oracle import refine_oracle as R
from paper_0906_2704_gb300 import synth
import parity_utils as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402

DEG = {"sine": 1, "cosine": 2, "fourier": 2, "sine3": 3}
TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _round(x, dt):
    if np.iscomplexobj(x):
        return x.real.astype(dt).astype(np.float64) + 1j * x.imag.astype(dt).astype(np.float64)
    return x.astype(dt).astype(np.float64)


def _case(ndim, fam, prec, L, K=48, batch=4, seed=5):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    mus = synth.mu_grid(K)
    if ndim == 1:
        n, taps = (70,), 7
    else:
        n, taps = (36, 42), (7, 7)
    h = _round(P.psf_for(F, ndim, taps), dt)
    h = _round(h / h.sum(), dt)
    g, _ = P.problems(ndim, n, h, batch, seed, 0.01)
    g = _round(g, dt)
    plan = hobc.Plan(ndim, n, h.shape, DEG[fam], mus, L=L, prec=prec, family=fam, psf_symmetric=F != "F",
                     batch=batch)
    return F, dt, mus, n, h, g, plan


def _identical_inputs(F, ndim, h, g, L, mus, dt, plan):
    batch = g.shape[0]
    orc = [P.oracle_steps(F, ndim, h, g[b], L, mus) for b in range(batch)]
    cplx = plan.spec_complex
    gin = np.zeros((batch, plan.spec_elems), dtype=complex if cplx else float)
    din = np.zeros_like(gin)
    full = []
    for b in range(batch):
        gr, dr = _round(orc[b][0], dt), _round(orc[b][1], dt)
        full.append((gr, dr, orc[b][2]))
        cast = (lambda a: a) if cplx else np.real
        gin[b] = cast(P.to_layout(F, gr).reshape(-1))
        din[b] = cast(P.to_layout(F, dr).reshape(-1))

    def spec(a):
        return _dev(np.stack([a.real, a.imag], axis=-1) if cplx else a.real, dt)
    return full, spec(gin), spec(din)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_refinement_matches_oracle_on_identical_inputs(ndim, fam, L, prec):
    F, dt, mus, n, h, g, plan = _case(ndim, fam, prec, L)
    batch, K = g.shape[0], len(mus)
    tol = TOL[prec]
    full, gh_d, d_d = _identical_inputs(F, ndim, h, g, L, mus, dt, plan)
    k_o = np.array([O.gcv_argmin(O.gcv_curve(gr, dr, s, mus)) for gr, dr, s in full], dtype=np.int32)
    mi = torch.from_numpy(k_o).cuda()
    mu_d = torch.full((batch,), -1.0, dtype=torch.float64, device="cuda")
    G_d = torch.full((batch,), -1.0, dtype=torch.float64, device="cuda")
    plan.gcv_refine(gh_d, d_d, mi, mu_d, G_d)
    mu_g, G_g = mu_d.cpu().numpy(), G_d.cpu().numpy()
    for b, (gr, dr, s) in enumerate(full):
        k = int(k_o[b])
        lo = float(np.asarray(mus[max(k - 1, 0)], dtype=dt))
        hi = float(np.asarray(mus[min(k + 1, K - 1)], dtype=dt))
        assert lo * (1 - 1e-6) <= mu_g[b] <= hi * (1 + 1e-6), f"item {b}: mu {mu_g[b]} outside [{lo}, {hi}]"
        assert float(np.asarray(mu_g[b], dtype=dt)) == mu_g[b]
        mu_o, G_o, hist = R.refine(gr, dr, s, mus, k, point_dtype=dt)
        G_at = O.gcv_curve(gr, dr, s, np.array([mu_g[b], mu_o]))
        assert G_at[0] <= (1 + 10 * tol) * G_at[1], f"item {b}: G {G_at[0]:.12e} vs oracle {G_at[1]:.12e}"
        assert abs(G_g[b] - G_at[0]) <= 10 * tol * G_at[0], f"item {b}: reported G"
        assert G_at[0] <= (1 + 10 * tol) * O.gcv_curve(gr, dr, s, mus).min()
        if prec == "fp64":
            pts, Gl, j = hist[-1]
            Gs = np.sort(Gl)
            if Gs[1] - Gs[0] > 1e3 * tol * Gs[0]:
                assert abs(np.log10(mu_g[b]) - np.log10(mu_o)) <= 1e-12, f"item {b}: point"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
def test_filter_at_given_mu_matches_oracle(fam, prec):
    ndim, L = 2, "lap"
    F, dt, mus, n, h, g, plan = _case(ndim, fam, prec, L)
    batch = g.shape[0]
    full, gh_d, d_d = _identical_inputs(F, ndim, h, g, L, mus, dt, plan)
    mu_o = np.array([R.refine(gr, dr, s, mus, O.gcv_argmin(O.gcv_curve(gr, dr, s, mus)), point_dtype=dt)[0]
                     for gr, dr, s in full])
    f_d = torch.empty(g.shape, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    plan.filter_synthesis_mu(gh_d, d_d, torch.from_numpy(mu_o).cuda(), f_d)
    f = f_d.cpu().numpy().astype(np.float64)
    eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    # the filter+synthesis bound of the layered parity test: the GPU's FFT
    # (16 log2 M roundings) plus the oracle's dense products (2 sqrt(n) per axis)
    rb = 16.0 * P.log2_fft(F, n) + 2.0 * sum(np.sqrt(v) for v in n)
    sT = P.sigma(F, n)
    for b, (gr, dr, s) in enumerate(full):
        fo = P.oracle_filtered(F, ndim, gr, dr, s, mu_o[b])
        X = O.filter_factors(dr, s, mu_o[b]) * gr
        bound = max(TOL[prec] * np.abs(fo).max(), rb * eps * sT * np.linalg.norm(X))
        err = np.abs(f[b] - fo).max()
        assert err <= bound, f"item {b}: {err:.3e} > {bound:.3e}"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["cosine", "fourier"])
def test_deblur_refined_composes_the_steps(fam, prec):
    F, dt, mus, n, h, g, plan = _case(2, fam, prec, "I", K=64, batch=5, seed=8)
    batch = g.shape[0]
    tdt = torch.float64 if prec == "fp64" else torch.float32
    g_d, h_d = _dev(g, dt), _dev(h, dt)
    f1 = torch.empty(g.shape, dtype=tdt, device="cuda")
    m1 = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.deblur(g_d, h_d, f1, m1)
    f2 = torch.empty_like(f1)
    m2 = torch.empty_like(m1)
    mu2 = torch.empty(batch, dtype=torch.float64, device="cuda")
    plan.deblur_refined(g_d, h_d, f2, m2, mu2)
    assert torch.equal(m1, m2)
    gh = torch.empty((batch, plan.spec_elems * (2 if plan.spec_complex else 1)), dtype=tdt, device="cuda")
    dd = torch.empty((1, plan.spec_elems * (2 if plan.spec_complex else 1)), dtype=tdt, device="cuda")
    plan.analysis(g_d, gh)
    plan.eigenvalues(h_d, dd)
    mu3 = torch.empty_like(mu2)
    plan.gcv_refine(gh, dd, m2, mu3)
    assert torch.equal(mu2, mu3)
    f3 = torch.empty_like(f1)
    plan.filter_synthesis_mu(gh, dd, mu3, f3)
    assert torch.equal(f2, f3)
    # the refined choice is never worse than the grid's (as the oracle evaluates G)
    for b in range(batch):
        ghat, d, s, Go, ko = P.oracle_steps(F, 2, h, g[b], "I", mus)
        Gr = O.gcv_curve(ghat, d, s, np.array([mu2[b].item()]))[0]
        assert Gr <= (1 + 10 * TOL[prec]) * Go[ko]


def test_refine_rejects_a_decreasing_grid():
    mus = synth.mu_grid(8)[::-1].copy()
    plan = hobc.Plan(1, 40, 5, 2, mus, family="cosine", psf_symmetric=True)
    t = torch.zeros(40, dtype=torch.float64, device="cuda")
    mi = torch.zeros(1, dtype=torch.int32, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hobc.HobcError, match="increasing"):
        plan.gcv_refine(t, t, mi, mu)


def test_refine_single_grid_value_keeps_it():
    """K = 1: the bracket collapses to the grid value; mu* is that value up to the rounding of
    10^(log10 mu) in the working precision."""
    mus = np.array([2e-3])
    h = np.array([0.25, 0.5, 0.25])
    g, _ = synth.problem_1d(1, 40, h, 0.01, count=2)
    for prec, dt in (("fp64", np.float64), ("fp32", np.float32)):
        plan = hobc.Plan(1, 40, 3, 2, mus, prec=prec, family="cosine", psf_symmetric=True, batch=2)
        f = torch.empty((2, 40), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        mu = torch.empty(2, dtype=torch.float64, device="cuda")
        mi = torch.empty(2, dtype=torch.int32, device="cuda")
        plan.deblur_refined(_dev(g, dt), _dev(h, dt), f, mi, mu)
        assert np.all(mi.cpu().numpy() == 0)
        assert np.allclose(mu.cpu().numpy(), 2e-3, rtol=4 * float(np.finfo(dt).eps), atol=0)
