"""Parity of the 3D path (include/hobc_volume.h) with the FP64 oracle
(oracle/volume_oracle.py), layer by layer as in the 2D parity test:
  eigenvalues   FP64 1e-12 of max (plus 64 eps sum|h|); FP32 1e-6 per entry plus that floor
  analysis, synthesis   max(flat, 256 eps cond0 cond1 cond2) of max, cond_a = cond(T_a)
                (FFT rounding through three axes; degree 3 is badly conditioned, reading R6)
  G(mu_j) on identical inputs (the oracle's spectra rounded to the working
                precision): 1e-10 / 1e-5 relative; mu* equal or within that of the minimum
  filter + synthesis on identical inputs at the oracle's mu index: as synthesis
The one-call deblur equals the steps bit for bit; per-volume PSFs equal
single-volume plans.
"""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from oracle import volume_oracle as V
from paper_0906_2704_gb300 import synth
import parity_utils as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402

DEG = {"sine": 1, "cosine": 2, "fourier": 2, "sine3": 3}
TOL = {"fp64": 1e-10, "fp32": 1e-5}
EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _round(x, dt):
    if np.iscomplexobj(x):
        return x.real.astype(dt).astype(np.float64) + 1j * x.imag.astype(dt).astype(np.float64)
    return x.astype(dt).astype(np.float64)


def layout(F, full):
    """Oracle volume spectrum [t0][t1][t2] -> stored [c][t1][t0] (flattened)."""
    ts = P.stored_t(F, full.shape[2], True)
    return np.transpose(full[:, :, ts], (2, 1, 0)).reshape(-1)


def _spec(a, dt, cplx):
    return _dev(np.stack([a.real, a.imag], axis=-1), dt) if cplx else _dev(a.real, dt)


def _np(t, cplx):
    a = t.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1] if cplx else a


def _cond3(F, n):
    return float(np.prod([np.linalg.cond(O.transform_matrix(F, m)) for m in n]))


def _case(fam, prec, L, batch=2, seed=1, psf_per_item=False):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    n = (9, 10, 11) if F == "S3" else (7, 9, 10)
    if F == "F":
        hs = [synth.gaussian_psf_3d((0.9, 1.2, 0.8), (3, 5, 3), (0.3, -0.2, 0.1 * i)) for i in range(batch)]
    else:
        hs = [synth.gaussian_psf_3d((0.8 + 0.1 * i, 1.0, 0.7), (3, 3, 3)) for i in range(batch)]
    hs = [_round(h, dt) for h in hs]
    g = np.stack([synth.problem_3d(seed + i, *n, hs[i if psf_per_item else 0], 0.01)[0][0] for i in range(batch)])
    g = _round(g, dt)
    mus = synth.mu_grid(24, 1e-6, 1.0)
    plan = hobc.Volume(n, hs[0].shape, DEG[fam], mus, L=L, prec=prec, family=fam, psf_symmetric=F != "F",
                       batch=batch, psf_per_item=psf_per_item)
    return F, dt, n, hs, g, mus, plan


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
def test_volume_steps_match_oracle(fam, L, prec):
    F, dt, n, hs, g, mus, plan = _case(fam, prec, L)
    B, S, cplx = g.shape[0], plan.spec_elems, plan.spec_complex
    cs = (2,) if cplx else ()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    tol = TOL[prec]
    ttol = max(tol, 256 * EPS[prec] * _cond3(F, n))
    h = hs[0]
    # eigenvalues
    d_d = torch.empty((1, S) + cs, dtype=tdt, device="cuda")
    plan.eigenvalues(_dev(h, dt), d_d)
    d_o = V.eigenvalues_3d(F, h, *n)
    dref = layout(F, d_o if cplx else d_o.real)
    dg = _np(d_d, cplx)[0]
    floor = 64 * 2.0 ** -53 * np.abs(h).sum()
    if prec == "fp64":
        assert np.abs(dg - dref).max() <= max(1e-12 * np.abs(dref).max(), floor)
    else:
        assert np.all(np.abs(dg - dref) <= 1e-6 * np.abs(dref) + floor)
    # analysis from the volumes
    gh_d = torch.empty((B, S) + cs, dtype=tdt, device="cuda")
    plan.analysis(_dev(g, dt), gh_d)
    gh = _np(gh_d, cplx)
    s_o = V.smoothing_3d(F, *n, L)
    full = []
    for b in range(B):
        ref_full = V.analysis_3d(F, g[b])
        ref = layout(F, ref_full if cplx else ref_full.real)
        assert np.abs(gh[b] - ref).max() <= ttol * np.abs(ref).max(), f"analysis item {b}"
        full.append((_round(ref_full if cplx else ref_full.real, dt), _round(d_o if cplx else d_o.real, dt)))
    # GCV, filter + synthesis and synthesis on identical inputs
    gin = np.stack([layout(F, gr) for gr, _ in full])
    din = layout(F, full[0][1])[None]
    G_d = torch.empty((B, len(mus)), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(B, dtype=torch.int32, device="cuda")
    plan.gcv(_spec(gin, dt, cplx), _spec(din, dt, cplx), G_d, mi_d)
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    k_o = []
    for b, (gr, dr) in enumerate(full):
        Go = O.gcv_curve(gr, dr, s_o, mus)
        assert np.max(np.abs(G[b] - Go) / Go) <= tol, f"G item {b}"
        ko = O.gcv_argmin(Go)
        k_o.append(ko)
        assert mi[b] == ko or Go[mi[b]] <= (1 + tol) * Go.min()
    f_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    plan.filter_synthesis(_spec(gin, dt, cplx), _spec(din, dt, cplx), _dev(np.array(k_o, dtype=np.int32), np.int32),
                          f_d)
    y_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    plan.synthesis(_spec(gin, dt, cplx), y_d)
    f, y = f_d.cpu().numpy(), y_d.cpu().numpy()
    for b, (gr, dr) in enumerate(full):
        fo = V.synthesis_3d(F, O.filter_factors(dr, s_o, mus[k_o[b]]) * gr).real
        assert np.abs(f[b] - fo).max() <= ttol * np.abs(fo).max(), f"filter+synthesis item {b}"
        yo = V.synthesis_3d(F, gr).real
        assert np.abs(y[b] - yo).max() <= ttol * np.abs(yo).max(), f"synthesis item {b}"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["cosine", "fourier"])
def test_volume_deblur_equals_its_steps(fam, prec):
    F, dt, n, hs, g, mus, plan = _case(fam, prec, "lap", batch=3, seed=4)
    B, S, cplx = g.shape[0], plan.spec_elems, plan.spec_complex
    cs = (2,) if cplx else ()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    g_d, h_d = _dev(g, dt), _dev(hs[0], dt)
    f1 = torch.empty(g.shape, dtype=tdt, device="cuda")
    m1 = torch.empty(B, dtype=torch.int32, device="cuda")
    G1 = torch.empty((B, len(mus)), dtype=torch.float64, device="cuda")
    plan.deblur(g_d, h_d, f1, m1, G1)
    assert plan.last_launch_count > 0
    d_d = torch.empty((1, S) + cs, dtype=tdt, device="cuda")
    gh = torch.empty((B, S) + cs, dtype=tdt, device="cuda")
    plan.eigenvalues(h_d, d_d)
    plan.analysis(g_d, gh)
    G2 = torch.empty_like(G1)
    m2 = torch.empty_like(m1)
    plan.gcv(gh, d_d, G2, m2)
    f2 = torch.empty_like(f1)
    plan.filter_synthesis(gh, d_d, m2, f2)
    assert torch.equal(G1, G2) and torch.equal(m1, m2) and torch.equal(f1, f2)


def test_volume_per_item_psf_equals_single_plans():
    F, dt, n, hs, g, mus, plan = _case("cosine", "fp64", "lap", batch=3, seed=6, psf_per_item=True)
    B = g.shape[0]
    f = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    G = torch.empty((B, len(mus)), dtype=torch.float64, device="cuda")
    plan.deblur(_dev(g, dt), _dev(np.stack(hs), dt), f, None, G)
    for b in range(B):
        one = hobc.Volume(n, hs[b].shape, 2, mus, L="lap", prec="fp64", family="cosine", psf_symmetric=True, batch=1)
        f1 = torch.empty((1,) + n, dtype=torch.float64, device="cuda")
        G1 = torch.empty((1, len(mus)), dtype=torch.float64, device="cuda")
        one.deblur(_dev(g[b:b + 1], dt), _dev(hs[b], dt), f1, None, G1)
        assert torch.allclose(G[b], G1[0], rtol=1e-12, atol=0)
        assert torch.allclose(f[b], f1[0], rtol=0, atol=1e-12 * float(f1.abs().max()))


def test_volume_rejects_what_it_does_not_support():
    mus = synth.mu_grid(8)
    with pytest.raises(hobc.HobcError) as e:
        hobc.Volume((8, 8, 8), (3, 3, 3), 2, mus, prec="split_bf16", family="cosine", psf_symmetric=True)
    assert e.value.status == hobc.STATUS.index("HOBC_ERR_UNSUPPORTED")
    with pytest.raises(hobc.HobcError) as e:
        hobc.Volume((8, 8, 8), (7, 3, 3), 2, mus, family="cosine", psf_symmetric=True)
    assert e.value.status == hobc.STATUS.index("HOBC_ERR_SIZE")
    with pytest.raises(hobc.HobcError) as e:
        hobc.Volume((1024, 8, 8), (3, 3, 3), 2, mus, family="cosine", psf_symmetric=True, batch=64)
    assert e.value.status == hobc.STATUS.index("HOBC_ERR_SIZE")


@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier"])
def test_volume_smallest_field_of_view_and_single_mu(fam):
    """6 x 6 x 7 volumes, a 3-tap PSF per axis, K = 1: the whole path against the oracle."""
    F = P.FAM_LETTER[fam]
    n = (6, 6, 7)
    h = synth.gaussian_psf_3d((0.8, 0.9, 0.7), (3, 3, 3), (0.2, 0.0, -0.1) if F == "F" else (0, 0, 0))
    g, _ = synth.problem_3d(5, *n, h, 0.01, count=1)
    mus = np.array([3e-3])
    plan = hobc.Volume(n, h.shape, DEG[fam], mus, L="lap", prec="fp64", family=fam, psf_symmetric=F != "F")
    f = torch.empty((1,) + n, dtype=torch.float64, device="cuda")
    G = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    mi = torch.empty(1, dtype=torch.int32, device="cuda")
    plan.deblur(_dev(g, np.float64), _dev(h, np.float64), f, mi, G)
    fo, Go, ko, _ = V.deblur_3d(F, h, g[0], "lap", mus)
    assert int(mi[0]) == 0 and abs(G[0, 0].item() - Go[0]) <= 1e-10 * Go[0]
    assert np.abs(f[0].cpu().numpy() - fo).max() <= 1e-9 * np.abs(fo).max()
