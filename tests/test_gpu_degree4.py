"""GPU parity of the degree-4 cosine family (family "cosine4", reading R16: the
construction of Sec. 3.1 with two border columns per side) through the C ABI.

T_X is ill-conditioned (cond(T) ~ n^3.5), so every bound that involves the
analysis T_X^{-1} scales with cond(T) (the product over axes in 2D):
  eigenvalues            FP64 1e-12 of max; FP32 1e-6 per entry plus a floor
  analysis               max(1e-10 | 1e-5, 64 eps cond(T)) of the largest entry
  G on identical inputs  1e-10 | 1e-5 relative, every mu (no transform involved)
  argmin                 equal, or an index whose oracle G is within tolerance of the minimum
  filter + synthesis     max(flat, 64 eps rb ||T||_2 ||X||_2) on identical inputs
  whole path             the analysis error, at most 64 eps cond(T) max|ghat|, magnified
                         by the filter (kappa) and ||T||_2
and closed forms that need no oracle: a sampled quartic deblurred with the
Laplacian comes back unchanged for every mu (A p = p, L p = 0), and the delta
PSF with L = I gives f = g / (1 + mu*) with the smallest mu chosen.
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

TOL = {"fp64": 1e-10, "fp32": 1e-5}
EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


def _dt(prec):
    return (np.float64, torch.float64) if prec == "fp64" else (np.float32, torch.float32)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _round(x, dt):
    return x.astype(dt).astype(np.float64)


def _cond(shape):
    out = 1.0
    for n in shape:
        out *= np.linalg.cond(O.transform_matrix("C4", n))
    return out


CASES = [(1, (13,), 5), (1, (40,), 7), (2, (12, 15), (5, 3)), (2, (20, 17), (5, 5))]


@pytest.mark.parametrize("prec", ["fp64"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("ndim,n,taps", CASES)
def test_degree4_steps_and_whole_path(ndim, n, taps, L, prec):
    dt, tdt = _dt(prec)
    eps, tol = EPS[prec], TOL[prec]
    h = P.psf_for("C", ndim, taps)
    h = _round(h / h.sum(), dt)
    batch = 3
    g, _ = P.problems(ndim, n, h, batch, 5)
    g = _round(g, dt)
    mus = synth.mu_grid(16, 1e-6, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, 4, mus, L=L, prec=prec, family="cosine4", psf_symmetric=True,
                     batch=batch)
    assert plan.family == "cosine4" and not plan.spec_complex
    S = plan.spec_elems
    c = _cond(n)
    sT = P.sigma("C4", n)
    rb = 16.0 * P.log2_fft("C4", n) + 2.0 * sum(np.sqrt(v) for v in n)
    orc = [P.oracle_steps("C4", ndim, h, g[b], L, mus) for b in range(batch)]

    # eigenvalues and analysis from the inputs
    d_d = torch.empty((1, S), dtype=tdt, device="cuda")
    plan.eigenvalues(_dev(h[None], dt), d_d)
    gh_d = torch.empty((batch, S), dtype=tdt, device="cuda")
    plan.analysis(_dev(g, dt), gh_d)
    dg, gh = d_d.cpu().numpy()[0], gh_d.cpu().numpy()
    dref = P.to_layout("C4", orc[0][1]).reshape(-1).real
    floor = 64 * 2.0 ** -53 * np.abs(h).sum()
    if prec == "fp64":
        assert np.abs(dg - dref).max() <= max(1e-12 * np.abs(dref).max(), floor), "eigenvalues"
    else:
        assert np.all(np.abs(dg - dref) <= 1e-6 * np.abs(dref) + floor), "eigenvalues"
    atol = max(tol, 64 * eps * c)
    for b in range(batch):
        ref = P.to_layout("C4", orc[b][0]).reshape(-1).real
        err = np.abs(gh[b] - ref).max() / np.abs(ref).max()
        assert err <= atol, f"analysis item {b}: {err:.3e} > {atol:.3e}"

    # GCV, filter + synthesis and synthesis on identical (rounded oracle) inputs
    gin = np.stack([_round(P.to_layout("C4", orc[b][0]).reshape(-1).real, dt) for b in range(batch)])
    din = _round(P.to_layout("C4", orc[0][1]).reshape(-1).real, dt)[None]
    G_d = torch.empty((batch, len(mus)), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.gcv(_dev(gin, dt), _dev(din, dt), G_d, mi_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    shape = n if ndim == 2 else (n[0],)
    mi_fix = np.array([orc[b][4] for b in range(batch)], dtype=np.int32)
    f_d = torch.empty((batch,) + shape, dtype=tdt, device="cuda")
    plan.filter_synthesis(_dev(gin, dt), _dev(din, dt), _dev(mi_fix, np.int32), f_d)
    y_d = torch.empty((batch,) + shape, dtype=tdt, device="cuda")
    plan.synthesis(_dev(gin, dt), y_d)
    f, y = f_d.cpu().numpy(), y_d.cpu().numpy()
    for b in range(batch):
        s_o = orc[b][2]
        full_g = gin[b].reshape(orc[b][0].T.shape).T if ndim == 2 else gin[b]
        full_d = din[0].reshape(orc[b][1].T.shape).T if ndim == 2 else din[0]
        Gref = O.gcv_curve(full_g, full_d, s_o, mus)
        gerr = np.max(np.abs(G[b] - Gref) / np.abs(Gref))
        assert gerr <= tol, f"G item {b}: {gerr:.3e}"
        kref = O.gcv_argmin(Gref)
        assert mi[b] == kref or Gref[mi[b]] <= (1 + tol) * Gref.min(), "argmin"
        X = O.filter_factors(full_d, s_o, mus[mi_fix[b]]) * full_g
        fref = P.oracle_filtered("C4", ndim, full_g, full_d, s_o, mus[mi_fix[b]])
        bound = max(tol * np.abs(fref).max(), 64 * eps * rb * sT * np.linalg.norm(X))
        assert np.abs(f[b] - fref).max() <= bound, f"filter+synthesis item {b}"
        yref = (O.synthesis_1d("C4", full_g) if ndim == 1 else O.synthesis_2d("C4", full_g)).real
        ybound = max(tol * np.abs(yref).max(), 64 * eps * rb * sT * np.linalg.norm(full_g))
        assert np.abs(y[b] - yref).max() <= ybound, f"synthesis item {b}"

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
        fo = P.oracle_filtered("C4", ndim, ghat_o, d_o, s_o, mus[k])
        X = O.filter_factors(d_o, s_o, mus[k]) * ghat_o
        bound = max(tol * np.abs(fo).max(), 64 * eps * rb * sT * np.linalg.norm(X) + sT * kappa * delta)
        assert np.abs(f2n[b] - fo).max() <= bound, f"whole path item {b}"
        if prec == "fp64" and k != k_o:   # a different index only where the curves are within the error
            assert G_o[k] <= (1 + 1e-6) * G_o.min(), f"whole-path argmin {k} vs {k_o}"


@pytest.mark.parametrize("ndim,prec,n", [(1, "fp64", (14,)), (2, "fp64", (12, 13))])
def test_quartics_come_back_unchanged(ndim, prec, n):
    """A sampled quartic is preserved by A_X and annihilated by the Laplacian, so the
    reblurred Tikhonov solution with L = Laplacian returns it for every mu."""
    dt, tdt = _dt(prec)
    taps = 5 if ndim == 1 else (5, 5)
    h = P.psf_for("C", ndim, taps)
    h = _round(h / h.sum(), dt)
    t0 = np.linspace(-1.0, 1.5, n[0])
    p0 = 0.3 - 0.8 * t0 + 0.5 * t0 ** 2 + 0.7 * t0 ** 3 - 0.4 * t0 ** 4
    if ndim == 1:
        g = p0[None]
    else:
        t1 = np.linspace(0.2, 1.1, n[1])
        g = np.outer(p0, 1.0 - t1 + 0.3 * t1 ** 4)[None]
    g = _round(g, dt)
    mus = synth.mu_grid(8, 1e-4, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, 4, mus, L="lap", prec=prec, family="cosine4", psf_symmetric=True)
    f_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    plan.deblur(_dev(g, dt), _dev(h[None], dt), f_d)
    err = np.abs(f_d.cpu().numpy() - g).max() / np.abs(g).max()
    assert err <= max(TOL[prec], 64 * EPS[prec] * _cond(n)), err


@pytest.mark.parametrize("prec", ["fp64"])
def test_delta_psf_closed_form(prec):
    """h = delta: d = 1, so G is the same for every mu (to rounding) and f = g/(1+mu*)
    at whichever grid value is chosen."""
    dt, tdt = _dt(prec)
    n = (11, 16)
    g = _round(np.random.default_rng(4).standard_normal((2,) + n), dt)
    mus = synth.mu_grid(6, 1e-3, 1.0)
    plan = hobc.Plan(2, n, (1, 1), 4, mus, L="I", prec=prec, family="cosine4", psf_symmetric=True, batch=2)
    f_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    mi_d = torch.empty(2, dtype=torch.int32, device="cuda")
    G_d = torch.empty((2, len(mus)), dtype=torch.float64, device="cuda")
    plan.deblur(_dev(g, dt), _dev(np.ones((1, 1, 1)), dt), f_d, mi_d, G_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    tol = max(TOL[prec], 64 * EPS[prec] * _cond(n))
    for b in range(2):
        assert np.abs(G[b] / G[b].mean() - 1).max() <= tol
        err = np.abs(f_d.cpu().numpy()[b] - g[b] / (1 + mus[mi[b]])).max() / np.abs(g[b]).max()
        assert err <= tol, err


def test_degree4_outside_the_plain_path_is_rejected():
    """Degree 4 needs a symmetric PSF and FP64 (cond(T) >= 644 puts the FP32 rounding
    bound 64 eps32 cond(T) above 1e-3 at every size); the dense engine and 3D plans
    reject it."""
    mus = synth.mu_grid(4)
    for n in ((8,), (12, 15), (40,)):
        with pytest.raises(hobc.HobcError) as e:
            hobc.Plan(len(n), n, (3,) * len(n), 4, mus, prec="fp32", family="cosine4", psf_symmetric=True)
        assert e.value.status == 2
    with pytest.raises(hobc.HobcError) as e:
        hobc.Plan(2, (16, 16), (5, 5), 4, mus, prec="fp32", family="auto", psf_symmetric=False)
    assert e.value.status == 2
    with pytest.raises(hobc.HobcError) as e:
        hobc.Plan(2, (16, 16), (5, 5), 4, mus, prec="split_bf16", family="cosine4", psf_symmetric=True)
    assert e.value.status == 2
    with pytest.raises(hobc.HobcError) as e:
        hobc.Plan(1, 7, 3, 4, mus, prec="fp64", family="cosine4", psf_symmetric=True)   # n >= 8
    assert e.value.status == 3
    with pytest.raises(hobc.HobcError) as e:
        hobc.Volume((8, 10, 10), (3, 3, 3), 4, mus, prec="fp64", family="cosine4", psf_symmetric=True)
    assert e.value.status == 2


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("ndim,n,taps", [(1, (14,), 5), (2, (12, 13), (3, 5))])
def test_degree4_exact_gcv_matches_oracle(ndim, n, taps, L):
    """The exact GCV functional (Eq. (eq:gcv), T_X kept in the numerator) on identical
    FP64 inputs against the oracle's dense synthesis per mu, within 64 eps cond(T)."""
    h = P.psf_for("C", ndim, taps)
    h = h / h.sum()
    g, _ = P.problems(ndim, n, h, 2, 9)
    mus = synth.mu_grid(12, 1e-6, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, 4, mus, L=L, prec="fp64", family="cosine4", psf_symmetric=True, batch=2)
    gin = np.zeros((2, plan.spec_elems))
    full = []
    for b in range(2):
        ghat, d, s, _, _ = P.oracle_steps("C4", ndim, h, g[b], L, mus)
        full.append((ghat.real, d.real, s))
        gin[b] = P.to_layout("C4", ghat.real).reshape(-1)
    din = P.to_layout("C4", full[0][1]).reshape(-1)[None]
    G_d = torch.empty((2, len(mus)), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(2, dtype=torch.int32, device="cuda")
    plan.gcv_exact(_dev(gin, np.float64), _dev(din, np.float64), G_d, mi_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    tol = max(1e-10, 64 * EPS["fp64"] * _cond(n))
    for b, (gr, dr, s) in enumerate(full):
        Go = X.gcv_exact_curve("C4", gr, dr, s, mus)
        assert np.all(np.abs(G[b] - Go) <= tol * Go), np.max(np.abs(G[b] - Go) / Go)
        k, ko = int(mi[b]), int(np.argmin(Go))
        assert k == ko or Go[k] <= (1 + 2 * tol) * Go.min()
