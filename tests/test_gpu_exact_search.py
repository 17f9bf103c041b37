"""Parity of the coarse-to-fine search of the exact GCV minimiser
(hobc_gcv_exact_search, include/hobc_exact.h) with the oracle's search
(oracle/exact_search_oracle.py) on the oracle's exact GCV curve.

On identical inputs (the oracle's spectra rounded to the working precision go
to both sides):
  values    every G_ex the search evaluated is within the bound of the exact
            functional's parity test (4 n eps ||(|T_0||P||T_1|^T)|| / ||T P||,
            never below 1e-10 / 1e-5) of the oracle's curve, NaN elsewhere;
  mu*       the oracle's search on the oracle curve picks the same index, or one
            whose oracle G_ex is within the tolerance of the other's;
  K <= 32   the full scan of hobc_gcv_exact, bit for bit.
Whole path: hobc_deblur_exact_search equals its steps bit for bit and equals
hobc_deblur_exact wherever the two choose the same index.
"""
import numpy as np
import pytest

from oracle import exact_gcv_oracle as X
from oracle import exact_search_oracle as S
import parity_utils as P
from paper_0906_2704_gb300 import synth
from test_gpu_exact import _bound, _dev, _round, _spec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402

DEG = {"sine": 1, "cosine": 2, "fourier": 2, "sine3": 3, "cosine4": 4}


def _case(ndim, fam, prec, L, K, batch=3, seed=4):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    mus = synth.mu_grid(K)
    n, taps = ((70,), 7) if ndim == 1 else ((40, 46), (7, 7))
    h = _round(P.psf_for(F if F != "C4" else "C", ndim, taps), dt)
    h = _round(h / h.sum(), dt)
    g, _ = P.problems(ndim, n, h, batch, seed, 0.01)
    g = _round(g, dt)
    plan = hobc.Plan(ndim, n, h.shape, DEG[fam], mus, L=L, prec=prec, family=fam, psf_symmetric=F != "F",
                     batch=batch)
    return F, dt, mus, n, h, g, plan


CASES = [(nd, fam, prec, L) for nd in (1, 2) for fam in ("sine", "cosine", "fourier", "sine3")
         for prec in ("fp64", "fp32") for L in ("I", "lap")] + [(2, "cosine4", "fp64", "lap")]


@pytest.mark.parametrize("ndim,fam,prec,L", CASES)
def test_search_matches_the_oracle_search_on_identical_inputs(ndim, fam, prec, L):
    K = 256
    F, dt, mus, n, h, g, plan = _case(ndim, fam, prec, L, K)
    batch = g.shape[0]
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
    plan.gcv_exact_search(_spec(gin, dt, cplx), _spec(din, dt, cplx), G_d, mi_d)
    launches = plan.last_launch_count
    G, mi = G_d.cpu().numpy(), mi_d.cpu().numpy()
    for b, (gr, dr, s) in enumerate(full):
        Go = X.gcv_exact_curve(F, gr, dr, s, mus)
        bound = _bound(F, n, gr, dr, s, mus, prec)
        done = ~np.isnan(G[b])
        assert 16 <= done.sum() <= 30, done.sum()
        rel = np.abs(G[b][done] - Go[done]) / Go[done]
        assert np.all(rel <= bound[done]), f"item {b}: G_ex {np.max(rel / bound[done]):.2f} of bound"
        ko, seen = S.exact_search(lambda j: Go[j], K)
        k = int(mi[b])
        assert done[k]
        assert k == ko or Go[k] <= (1 + bound[k] + bound[ko]) * Go[ko], (k, ko)
        # the oracle search evaluates the same grid values (unless rounding moved the path)
        if k == ko:
            assert set(np.flatnonzero(done)) == set(seen)
    assert launches <= 1 + 3 * (2 + (4 if ndim == 2 else 1))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_grids_run_the_full_scan(prec):
    F, dt, mus, n, h, g, plan = _case(2, "fourier", prec, "I", K=24)
    batch = g.shape[0]
    g_d, h_d = _dev(g, dt), _dev(h[None], dt)
    f1, f2 = torch.empty_like(g_d), torch.empty_like(g_d)
    m1 = torch.empty(batch, dtype=torch.int32, device="cuda")
    m2 = torch.empty_like(m1)
    G1 = torch.empty((batch, 24), dtype=torch.float64, device="cuda")
    G2 = torch.empty_like(G1)
    plan.deblur_exact(g_d, h_d, f1, m1, G1)
    plan.deblur_exact_search(g_d, h_d, f2, m2, G2)
    assert torch.equal(G1, G2) and torch.equal(m1, m2) and torch.equal(f1, f2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["cosine", "fourier"])
def test_deblur_exact_search_composes_the_steps(fam, prec):
    F, dt, mus, n, h, g, plan = _case(2, fam, prec, "lap", K=256, batch=4, seed=9)
    batch = g.shape[0]
    g_d, h_d = _dev(g, dt), _dev(h[None], dt)
    f = torch.empty_like(g_d)
    mi = torch.empty(batch, dtype=torch.int32, device="cuda")
    G = torch.empty((batch, 256), dtype=torch.float64, device="cuda")
    plan.deblur_exact_search(g_d, h_d, f, mi, G)
    S_ = plan.spec_elems
    cs = (2,) if plan.spec_complex else ()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    gh = torch.empty((batch, S_) + cs, dtype=tdt, device="cuda")
    d = torch.empty((1, S_) + cs, dtype=tdt, device="cuda")
    plan.eigenvalues(h_d, d)
    plan.analysis(g_d, gh)
    mi2 = torch.empty_like(mi)
    G2 = torch.empty_like(G)
    plan.gcv_exact_search(gh, d, G2, mi2)
    f2 = torch.empty_like(f)
    plan.filter_synthesis(gh, d, mi2, f2)
    assert torch.equal(mi, mi2) and torch.equal(f, f2)
    assert torch.equal(torch.isnan(G), torch.isnan(G2))
    # against the full exact scan: same index, or a G within the FP tolerance
    mi3 = torch.empty_like(mi)
    G3 = torch.empty_like(G)
    f3 = torch.empty_like(f)
    plan.deblur_exact(g_d, h_d, f3, mi3, G3)
    tol = 1e-10 if prec == "fp64" else 1e-5
    for b in range(batch):
        k, k3 = int(mi[b]), int(mi3[b])
        if k == k3:
            assert torch.equal(f[b], f3[b])
        else:
            assert G3[b, k] <= (1 + 10 * tol) * G3[b, k3]
