"""Parity of the exact GCV functional (include/hobc_exact.h) with the FP64
oracle (oracle/exact_gcv_oracle.py): the spectral form ||T_X sigma ghat||^2 /
(sum sigma)^2 with T_X applied densely.

On identical inputs (the oracle's spectra rounded to the working precision go
to both sides):
  G_ex      every entry of T P is formed as a short sum of terms and every
            line sum runs over at most n entries, so |delta(T P)| <= n eps
            |T_0| |P| |T_1|^T entrywise and the relative error of ||T P||^2 is
            at most 4 n eps ||(|T_0||P||T_1|^T)|| / ||T P||, never below 1e-10
            (FP64) or 1e-5 (FP32).  The ratio is cond(T)-like: large for
            degree 3 (reading R6) and for the cosine family at large n.
  mu*       the same index, or one whose oracle G_ex is within the tolerance
            of the minimum.
Whole path: hobc_deblur_exact equals its steps bit for bit.
"""
import numpy as np
import pytest

from oracle import exact_gcv_oracle as X
from oracle import hobc_oracle as O
from paper_0906_2704_gb300 import synth
import parity_utils as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402

DEG = {"sine": 1, "cosine": 2, "fourier": 2, "sine3": 3}


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _round(x, dt):
    if np.iscomplexobj(x):
        return x.real.astype(dt).astype(np.float64) + 1j * x.imag.astype(dt).astype(np.float64)
    return x.astype(dt).astype(np.float64)


def _spec(a, dt, cplx):
    """Stored-layout spectra -> device tensor (interleaved pairs for the Fourier family)."""
    if cplx:
        return _dev(np.stack([a.real, a.imag], axis=-1), dt)
    return _dev(a.real, dt)


def _bound(F, n, gr, dr, s, mus, prec):
    """Per grid value: 4 n eps ||(|T_0| |P| |T_1|^T)|| / ||T P|| (each entry of
    T P is formed as a short sum of terms, each line sum runs over at most n
    entries), never below the flat tolerance (1e-10 FP64, 1e-5 FP32)."""
    eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    floor = 1e-10 if prec == "fp64" else 1e-5
    Ts = [O.transform_matrix(F, m) for m in n]
    out = []
    for mu in mus:
        sig = np.abs(s) ** 2 / (np.abs(dr) ** 2 + mu * np.abs(s) ** 2)
        Pm = sig * gr
        if len(n) == 1:
            mag = np.linalg.norm(np.abs(Ts[0]) @ np.abs(Pm))
            tp = np.linalg.norm(Ts[0] @ Pm)
        else:
            mag = np.linalg.norm(np.abs(Ts[0]) @ np.abs(Pm) @ np.abs(Ts[1]).T)
            tp = np.linalg.norm(Ts[0] @ Pm @ Ts[1].T)
        out.append(4 * max(n) * eps * mag / tp)
    return np.maximum(np.array(out), floor)


def _case(ndim, fam, prec, L, K=40, batch=3, seed=2):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    mus = synth.mu_grid(K, 1e-7, 1.0)
    n, taps = ((66,), 7) if ndim == 1 else ((40, 46), (7, 7))
    h = _round(P.psf_for(F, ndim, taps), dt)
    h = _round(h / h.sum(), dt)
    g, ft = P.problems(ndim, n, h, batch, seed, 0.01)
    g = _round(g, dt)
    plan = hobc.Plan(ndim, n, h.shape, DEG[fam], mus, L=L, prec=prec, family=fam, psf_symmetric=F != "F",
                     batch=batch)
    return F, dt, mus, n, h, g, ft, plan


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_exact_curve_matches_oracle_on_identical_inputs(ndim, fam, L, prec):
    F, dt, mus, n, h, g, _, plan = _case(ndim, fam, prec, L)
    batch, K = g.shape[0], len(mus)
    cplx = plan.spec_complex
    gin = np.zeros((batch, plan.spec_elems), dtype=complex)
    din = np.zeros((1, plan.spec_elems), dtype=complex)
    full = []
    for b in range(batch):
        ghat, d, s, _, _ = P.oracle_steps(F, ndim, h, g[b], L, mus)
        gr, dr = _round(ghat if cplx else ghat.real, dt), _round(d if cplx else d.real, dt)
        full.append((gr, dr, s))
        gin[b] = P.to_layout(F, gr).reshape(-1)
        din[0] = P.to_layout(F, dr).reshape(-1)
    G_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.gcv_exact(_spec(gin, dt, cplx), _spec(din, dt, cplx), G_d, mi_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    for b, (gr, dr, s) in enumerate(full):
        Go = X.gcv_exact_curve(F, gr, dr, s, mus)
        bound = _bound(F, n, gr, dr, s, mus, prec)
        rel = np.abs(G[b] - Go) / Go
        assert np.all(rel <= bound), f"item {b}: G_ex {np.max(rel / bound):.2f} of bound"
        k, ko = int(mi[b]), int(np.argmin(Go))
        assert k == ko or Go[k] <= (1 + bound[k] + bound[ko]) * Go.min()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier"])
def test_deblur_exact_composes_the_steps(fam, prec):
    F, dt, mus, n, h, g, _, plan = _case(2, fam, prec, "lap", batch=4, seed=7)
    batch = g.shape[0]
    tdt = torch.float64 if prec == "fp64" else torch.float32
    g_d, h_d = _dev(g, dt), _dev(h, dt)
    f1 = torch.empty(g.shape, dtype=tdt, device="cuda")
    m1 = torch.empty(batch, dtype=torch.int32, device="cuda")
    G1 = torch.empty((batch, len(mus)), dtype=torch.float64, device="cuda")
    plan.deblur_exact(g_d, h_d, f1, m1, G1)
    cs = (2,) if plan.spec_complex else ()
    gh = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    dd = torch.empty((1, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    plan.analysis(g_d, gh)
    plan.eigenvalues(h_d, dd)
    G2 = torch.empty_like(G1)
    m2 = torch.empty_like(m1)
    plan.gcv_exact(gh, dd, G2, m2)
    f2 = torch.empty_like(f1)
    plan.filter_synthesis(gh, dd, m2, f2)
    assert torch.equal(G1, G2) and torch.equal(m1, m2) and torch.equal(f1, f2)


def test_orthogonal_conditions_give_the_approximate_functional():
    """Reflective and periodic (dense split-BF16 plans): T orthogonal, rank 0, G_ex = G."""
    n = (36, 40)
    h = np.outer(synth.gaussian_psf_1d(1.3, 5), synth.gaussian_psf_1d(1.1, 5)).astype(np.float32)
    g, _ = synth.problem_2d(3, n[0], n[1], h.astype(np.float64), 0.01, count=2)
    mus = synth.mu_grid(24, 1e-6, 1.0)
    for fam in ("reflective", "periodic"):
        plan = hobc.Plan(2, n, h.shape, 0, mus, L="I", prec="split_bf16", family=fam, psf_symmetric=True, batch=2)
        gh = torch.empty((2, plan.spec_elems), dtype=torch.float32, device="cuda")
        dd = torch.empty((1, plan.spec_elems), dtype=torch.float32, device="cuda")
        plan.analysis(_dev(g, np.float32), gh)
        plan.eigenvalues(_dev(h, np.float32), dd)
        Ga = torch.empty((2, len(mus)), dtype=torch.float64, device="cuda")
        Gx = torch.empty_like(Ga)
        mi = torch.empty(2, dtype=torch.int32, device="cuda")
        plan.gcv(gh, dd, Ga, mi)
        plan.gcv_exact(gh, dd, Gx, mi)
        assert torch.allclose(Gx, Ga, rtol=2e-5, atol=0), fam


def test_full_size_1024_cosine_fp32_at_sampled_mu():
    """The dense-workload shape (1024 x 1024, cosine family, Laplacian, 256 mu) on
    identical inputs: G_ex at five grid values against the oracle's dense
    evaluation there (T_C at n = 1024 has condition ~2e4, where the Gram form
    of the numerator loses every digit in FP32)."""
    n = (1024, 1024)
    h = synth.gaussian_psf_2d_separable(2.5, 15).astype(np.float32).astype(np.float64)
    g, _ = synth.problem_2d(11, n[0], n[1], h, 0.005, count=1)
    g = g[0].astype(np.float32).astype(np.float64)
    mus = synth.mu_grid(256)
    plan = hobc.Plan(2, n, h.shape, 2, mus, L="lap", prec="fp32", family="cosine", psf_symmetric=True, batch=1)
    ghat = _round(O.analysis_2d("C", g), np.float32)
    d = _round(O.eigenvalues_2d("C", h, n[0], n[1]).real, np.float32)
    s = O.smoothing_2d("C", n[0], n[1], "lap")
    G_d = torch.empty((1, 256), dtype=torch.float64, device="cuda")
    mi = torch.empty(1, dtype=torch.int32, device="cuda")
    plan.gcv_exact(_dev(P.to_layout("C", ghat).reshape(1, -1), np.float32),
                   _dev(P.to_layout("C", d).reshape(1, -1), np.float32), G_d, mi)
    js = [0, 40, 85, 170, 255]
    Go = X.gcv_exact_curve("C", ghat, d, s, mus[js])
    bound = _bound("C", n, ghat, d, s, mus[js], "fp32")
    rel = np.abs(G_d.cpu().numpy()[0, js] - Go) / Go
    assert np.all(rel <= bound), f"{rel} > {bound}"


def test_full_size_1024_fourier_fp32_at_sampled_mu():
    """The bench's headline shape (1024 x 1024, Fourier family, nonsymmetric rotated
    Gaussian, L = I, 256 mu) on identical inputs: G_ex at three grid values against
    the oracle's dense complex evaluation there (half spectrum on the GPU)."""
    n = (1024, 1024)
    h = synth.gaussian_psf_2d_rotated(3.0, 1.5, 30.0, 21, 2.0, -1.0).astype(np.float32).astype(np.float64)
    g, _ = synth.problem_2d(12, n[0], n[1], h, 0.005, count=1)
    g = g[0].astype(np.float32).astype(np.float64)
    mus = synth.mu_grid(256)
    plan = hobc.Plan(2, n, h.shape, 2, mus, L="I", prec="fp32", family="fourier", batch=1)
    ghat = _round(O.analysis_2d("F", g), np.float32)
    d = _round(O.eigenvalues_2d("F", h, n[0], n[1]), np.float32)
    s = O.smoothing_2d("F", n[0], n[1], "I")
    G_d = torch.empty((1, 256), dtype=torch.float64, device="cuda")
    mi = torch.empty(1, dtype=torch.int32, device="cuda")
    plan.gcv_exact(_spec(P.to_layout("F", ghat).reshape(1, -1), np.float32, True),
                   _spec(P.to_layout("F", d).reshape(1, -1), np.float32, True), G_d, mi)
    js = [0, 128, 255]
    Go = X.gcv_exact_curve("F", ghat, d, s, mus[js])
    bound = _bound("F", n, ghat, d, s, mus[js], "fp32")
    rel = np.abs(G_d.cpu().numpy()[0, js] - Go) / Go
    assert np.all(rel <= bound), f"{rel} > {bound}"


@pytest.mark.parametrize("fam,n", [("sine", 6), ("cosine", 6), ("fourier", 6), ("sine3", 8)])
def test_exact_smallest_field_of_view_and_single_mu(fam, n):
    """n = 6 (8 for degree 3) in 1D and 2D, K = 1 and K = 3: the curve against the oracle."""
    F = P.FAM_LETTER[fam]
    h = np.array([0.25, 0.5, 0.25])
    for K in (1, 3):
        mus = synth.mu_grid(K, 1e-3, 1.0)
        g, _ = synth.problem_1d(2, n, h, 0.01)
        plan = hobc.Plan(1, n, 3, DEG[fam], mus, family=fam, psf_symmetric=True, batch=1)
        G = torch.empty((1, K), dtype=torch.float64, device="cuda")
        f = torch.empty((1, n), dtype=torch.float64, device="cuda")
        plan.deblur_exact(_dev(g, np.float64), _dev(h, np.float64), f, None, G)
        ghat, d, s = O.analysis_1d(F, g[0]), O.eigenvalues_1d(F, h, n), O.smoothing_1d(F, n, "I")
        assert np.allclose(G.cpu().numpy()[0], X.gcv_exact_curve(F, ghat, d, s, mus), rtol=1e-10, atol=0)
        h2 = np.outer(h, h)
        g2, _ = synth.problem_2d(3, n, n + 1, h2, 0.01)
        plan2 = hobc.Plan(2, (n, n + 1), (3, 3), DEG[fam], mus, family=fam, psf_symmetric=True, batch=1)
        G2 = torch.empty((1, K), dtype=torch.float64, device="cuda")
        f2 = torch.empty((1, n, n + 1), dtype=torch.float64, device="cuda")
        plan2.deblur_exact(_dev(g2, np.float64), _dev(h2, np.float64), f2, None, G2)
        gh2 = O.analysis_2d(F, g2[0])
        d2, s2 = O.eigenvalues_2d(F, h2, n, n + 1), O.smoothing_2d(F, n, n + 1, "I")
        assert np.allclose(G2.cpu().numpy()[0], X.gcv_exact_curve(F, gh2, d2, s2, mus), rtol=1e-9, atol=0)
