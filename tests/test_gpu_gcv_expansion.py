"""The GCV curve by bin expansion (hobc_plan_set_gcv_mode(EXPANSION),
include/hobc.h) against the direct scan and the oracle.

G(mu_j) of Eq. (eq:gcv2) is evaluated through per-bin moments of the entries
(bins uniform in log a = log |d|^2/|s|^2, the series of 1/(a+mu)^k about each
bin's centre cut after the 7th power).  Checked, on FP32 plans:
  * G against the oracle on identical inputs (the oracle's spectra rounded to
    FP32): within the FP32 scan tolerance 1e-5 at every grid value; the argmin
    equal to the oracle's, or an index whose oracle G is within it;
  * G against the direct scan of the same plan on the same spectra, every family
    with an FFT-path FP32 mode, L = I and Laplacian, up to 1024 x 1024;
  * the truncation bound reported for the grid (3.3e-9 on [1e-8, 1]);
  * two runs give the same bits (fixed summation orders), and hobc_deblur in
    this mode equals its steps bit for bit;
  * plans it does not serve are refused: FP64, 1D, one PSF per problem, and a
    grid spanning so many decades that the bound would pass 1e-8.
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

TOL = 1e-5
DEG = {"sine": 1, "cosine": 2, "fourier": 2, "sine3": 3, "periodic": 0}


def _letter(fam):
    return "P" if fam == "periodic" else P.FAM_LETTER[fam]


def _plan(fam, n, taps, L, K, batch, prec="fp32", lo=1e-8, hi=1.0):
    F = _letter(fam)
    h = P.psf_for(F, 2, taps)
    h = h / h.sum()
    mus = synth.mu_grid(K, lo, hi)
    plan = hobc.Plan(2, n, h.shape, DEG[fam], mus, L=L, prec=prec, family=fam,
                     psf_symmetric=F not in ("F", "P"), batch=batch)
    return F, h, mus, plan


def _curves(plan, gh, d, K, batch):
    G = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    mi = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.gcv(gh, d, G, mi)
    torch.cuda.synchronize()
    return G, mi


@pytest.mark.parametrize("fam,L", [("fourier", "I"), ("cosine", "lap"), ("sine", "I"), ("sine3", "lap"),
                                   ("periodic", "lap")])
def test_expansion_matches_the_oracle_on_identical_inputs(fam, L):
    n, taps, K, batch = (40, 46), (7, 7), 64, 3
    F, h, mus, plan = _plan(fam, n, taps, L, K, batch)
    plan.set_gcv_mode("expansion")
    assert plan.gcv_mode == "expansion" and 0 < plan.gcv_expansion_bound < 1e-8
    g, _ = P.problems(2, n, h, batch, 3, 0.01)
    cplx = plan.spec_complex

    def rounded(x):
        re = x.real.astype(np.float32).astype(np.float64)
        return re + 1j * x.imag.astype(np.float32).astype(np.float64) if cplx else re

    def dev(full):
        lay = P.to_layout(F, full).reshape(-1)
        arr = np.stack([lay.real, lay.imag], axis=-1) if cplx else lay.real
        return arr.astype(np.float32)

    orc = [P.oracle_steps(F, 2, h, g[b], L, mus) for b in range(batch)]
    gh_full = [rounded(o[0]) for o in orc]
    d_full = rounded(orc[0][1])
    gh = torch.from_numpy(np.stack([dev(x) for x in gh_full])).cuda()
    d = torch.from_numpy(dev(d_full)[None]).cuda()
    G, mi = _curves(plan, gh, d, K, batch)
    Gn, mn = G.cpu().numpy(), mi.cpu().numpy()
    for b in range(batch):
        Gref = O.gcv_curve(gh_full[b], d_full, orc[b][2], mus)
        rel = np.max(np.abs(Gn[b] - Gref) / Gref)
        assert rel <= TOL, f"item {b}: {rel:.3e}"
        k = int(mn[b])
        assert k == O.gcv_argmin(Gref) or Gref[k] <= (1 + TOL) * Gref.min()


@pytest.mark.parametrize("fam,n,L,K", [("fourier", (66, 130), "I", 256), ("cosine", (96, 80), "lap", 128),
                                       ("sine3", (72, 64), "I", 100), ("periodic", (64, 81), "I", 256),
                                       ("fourier", (1024, 1024), "I", 256)])
def test_expansion_matches_the_direct_scan(fam, n, L, K):
    """Both modes on the same spectra: G within the FP32 scan tolerance, the same
    index or one whose direct G is within it; the curve is deterministic."""
    batch = 2 if n[0] == 1024 else 4
    taps = (21, 21) if n[0] == 1024 else (9, 9)
    F, h, mus, plan = _plan(fam, n, taps, L, K, batch)
    g, _ = P.problems(2, n, h, batch, 7, 0.005)
    g_d = torch.from_numpy(g.astype(np.float32)).cuda()
    h_d = torch.from_numpy(h[None].astype(np.float32)).cuda()
    cs = (2,) if plan.spec_complex else ()
    gh = torch.empty((batch, plan.spec_elems) + cs, dtype=torch.float32, device="cuda")
    d = torch.empty((1, plan.spec_elems) + cs, dtype=torch.float32, device="cuda")
    plan.eigenvalues(h_d, d)
    plan.analysis(g_d, gh)
    G0, m0 = _curves(plan, gh, d, K, batch)
    plan.set_gcv_mode("expansion")
    G1, m1 = _curves(plan, gh, d, K, batch)
    G2, m2 = _curves(plan, gh, d, K, batch)
    assert torch.equal(G1, G2) and torch.equal(m1, m2)
    rel = ((G1 - G0).abs() / G0.abs()).max().item()
    assert rel <= 2 * TOL, rel             # two curves, each within TOL of the exact one
    for b in range(batch):
        k0, k1 = int(m0[b]), int(m1[b])
        assert k0 == k1 or G0[b, k1] <= (1 + 2 * TOL) * G0[b, k0]
    plan.set_gcv_mode("direct")
    G3, m3 = _curves(plan, gh, d, K, batch)
    assert torch.equal(G3, G0) and torch.equal(m3, m0)


def test_deblur_in_expansion_mode_equals_its_steps():
    F, h, mus, plan = _plan("fourier", (64, 70), (9, 9), "lap", 128, 3)
    plan.set_gcv_mode("expansion")
    g, _ = P.problems(2, (64, 70), h, 3, 5, 0.01)
    g_d = torch.from_numpy(g.astype(np.float32)).cuda()
    h_d = torch.from_numpy(h[None].astype(np.float32)).cuda()
    f = torch.empty_like(g_d)
    mi = torch.empty(3, dtype=torch.int32, device="cuda")
    G = torch.empty((3, 128), dtype=torch.float64, device="cuda")
    plan.deblur(g_d, h_d, f, mi, G)
    gh = torch.empty((3, plan.spec_elems, 2), dtype=torch.float32, device="cuda")
    d = torch.empty((1, plan.spec_elems, 2), dtype=torch.float32, device="cuda")
    plan.eigenvalues(h_d, d)
    plan.analysis(g_d, gh)
    G2, mi2 = _curves(plan, gh, d, 128, 3)
    f2 = torch.empty_like(f)
    plan.filter_synthesis(gh, d, mi2, f2)
    assert torch.equal(G, G2) and torch.equal(mi, mi2) and torch.equal(f, f2)


def test_plans_the_expansion_does_not_serve_are_refused():
    for kw in (dict(prec="fp64"),):
        _, _, _, plan = _plan("cosine", (32, 32), (5, 5), "I", 16, 1, **kw)
        with pytest.raises(hobc.HobcError) as e:
            plan.set_gcv_mode("expansion")
        assert e.value.status == 2
        assert plan.gcv_mode == "direct" and plan.gcv_expansion_bound == -1.0
    plan = hobc.Plan(1, 64, 5, 2, synth.mu_grid(16), prec="fp32", family="cosine", psf_symmetric=True)
    with pytest.raises(hobc.HobcError) as e:
        plan.set_gcv_mode("expansion")
    assert e.value.status == 2
    plan = hobc.Plan(2, (32, 32), (5, 5), 2, synth.mu_grid(16), prec="fp32", family="cosine", psf_symmetric=True,
                     batch=2, psf_per_item=True)
    with pytest.raises(hobc.HobcError) as e:
        plan.set_gcv_mode("expansion")
    assert e.value.status == 2
    _, _, _, plan = _plan("cosine", (32, 32), (5, 5), "I", 16, 1, lo=1e-18, hi=1e12)
    with pytest.raises(hobc.HobcError) as e:           # 36 decades: the bound passes 1e-8
        plan.set_gcv_mode("expansion")
    assert e.value.status == 2 and plan.gcv_mode == "direct"


@pytest.mark.parametrize("chunks", [1, 3, 8])
def test_host_calls_in_expansion_mode_equal_the_device_call(chunks):
    """hobc_deblur_host cuts the batch into chunks and prepares the expansion's
    eigenvalue steps once per call: every problem's curve, mu index and f equal
    those of hobc_deblur on device buffers, bit for bit, for any chunk count."""
    F, h, mus, plan = _plan("fourier", (48, 66), (7, 7), "I", 64, 6)
    plan.set_gcv_mode("expansion")
    g, _ = P.problems(2, (48, 66), h, 6, 2, 0.01)
    g32, h32 = g.astype(np.float32), h[None].astype(np.float32)
    f_d = torch.empty((6, 48, 66), dtype=torch.float32, device="cuda")
    mi_d = torch.empty(6, dtype=torch.int32, device="cuda")
    G_d = torch.empty((6, 64), dtype=torch.float64, device="cuda")
    plan.deblur(torch.from_numpy(g32).cuda(), torch.from_numpy(h32).cuda(), f_d, mi_d, G_d)
    plan.set_host_chunks(chunks)
    f_h = np.empty_like(g32)
    mi_h = np.empty(6, dtype=np.int32)
    G_h = np.empty((6, 64), dtype=np.float64)
    for _ in range(2):                              # a second call reuses the staging
        plan.deblur_host(g32, h32, f_h, mi_h, G_h)
        assert np.array_equal(f_h, f_d.cpu().numpy()) and np.array_equal(mi_h, mi_d.cpu().numpy())
        assert np.array_equal(G_h, G_d.cpu().numpy())
    with pytest.raises(hobc.HobcError):
        plan.set_host_chunks(9)
