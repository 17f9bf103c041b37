"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Seeded inputs at small sizes that span several FFT groups, Bluestein and
power-of-two lengths, odd and non-square shapes, odd batches (ragged line
pairs), shared and per-problem PSFs; plus the full-size configurations.

Layer 1 -- each step on identical inputs (the oracle's own values rounded to the
working precision are given to both sides), element by element, relative to the
largest reference entry:
  eigenvalues  FP64 1e-12;  FP32 1e-6 per entry (summed in FP64, stored in FP32)
  analysis     FP64 1e-10;  FP32 1e-5
  G(mu_j)      FP64 1e-10;  FP32 1e-5   (relative, every mu)
  argmin       equal, or an index whose oracle G is within the G tolerance of the minimum
  filter+synthesis, synthesis   max(flat, eps rb sigma(T) ||X||_2): the norm-wise
                    rounding bound of an FFT-based product, rb = 16 log2(M) + 2 sum_axes
                    sqrt(n) (GPU FFT + the oracle's dense products), sigma(T) = ||T||_2
Layer 2 -- the one-call deblur equals the GPU's own step sequence bit for bit.
Layer 3 -- the whole path from g: forward-error bounds from the arithmetic
(reading R13), never below the flat tolerance: the analysis error norm
delta = min(eps rb ||T^{-1}|| ||g||, the layer-1 analysis tolerance) is magnified
by the filter factor kappa = max|d|/(|d|^2+mu|s|^2) and by ||T||;
eps = 2^-53 (FP64) or 2^-24 (FP32).  Where the problem's own
conditioning exceeds the flat tolerance (tiny mu* with T_X of condition ~1e4),
the derived bound is the one that applies.
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
from paper_0906_2704_gb300 import hobc  # noqa: E402  (raises if the library is missing)

TOL = {"fp64": 1e-10, "fp32": 1e-5}
C_FFT = 16.0     # Bluestein: two FFTs of length M plus the chirp products
C_DOT = 2.0      # the oracle's dense products: ~sqrt(n) roundings per axis


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _spec_dev(a, plan, dt):
    """Complex layout array -> device tensor (interleaved for the Fourier family)."""
    if plan.spec_complex:
        a = np.stack([a.real, a.imag], axis=-1)
    return _dev(a.real if not plan.spec_complex else a, dt)


def _spec_np(t, plan):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1] if plan.spec_complex else a


def _round(x, dt):
    """The value a working-precision buffer holds (complex parts rounded separately)."""
    if np.iscomplexobj(x):
        return x.real.astype(dt).astype(np.float64) + 1j * x.imag.astype(dt).astype(np.float64)
    return x.astype(dt).astype(np.float64)


def run_case(ndim, fam_name, n, taps, L, prec, batch, psf_per_item=False, K=24, seed=0, mus=None, h0=None,
             eta=0.01, check_items=None):
    fam = P.FAM_LETTER[fam_name]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    eps = 2.0 ** -53 if prec == "fp64" else P.EPS32
    n = (n,) if ndim == 1 else tuple(n)
    base = P.psf_for(fam, ndim, taps) if h0 is None else h0
    hs = []
    for b in range(batch if psf_per_item else 1):
        h = base ** (1.0 + 0.15 * b) if psf_per_item else base
        hs.append(_round(h / h.sum(), dt))
    g, _ = P.problems(ndim, n, hs[0], batch, seed, eta)
    g = _round(g, dt)
    mus = synth.mu_grid(K, 1e-6, 1.0) if mus is None else mus
    K = len(mus)
    deg = {"S": 1, "C": 2, "F": 2, "S3": 3}[fam]
    plan = hobc.Plan(ndim, n, hs[0].shape, deg, mus, L=L, prec=prec, family=fam_name,
                     psf_symmetric=fam != "F", batch=batch, psf_per_item=psf_per_item)
    S = plan.spec_elems
    cs = (2,) if plan.spec_complex else ()
    npsf = len(hs)
    tol = TOL[prec]
    l2m = P.log2_fft(fam, n)
    # rounding budget (units of eps) of a transform applied by both sides: the
    # GPU's FFT (C_FFT log2 M) plus the oracle's dense products (C_DOT sqrt(n) per axis)
    rb = C_FFT * l2m + C_DOT * sum(np.sqrt(v) for v in n)
    items = range(batch) if check_items is None else check_items

    # ---- oracle answers (FP64) on the rounded inputs
    orc = [P.oracle_steps(fam, ndim, hs[b if psf_per_item else 0], g[b], L, mus) for b in items]

    # ---- layer 1a: eigenvalues and analysis from the seeded inputs
    psf_d = _dev(np.stack(hs), dt)
    d_d = torch.empty((npsf, S) + cs, dtype=tdt, device="cuda")
    plan.eigenvalues(psf_d, d_d)
    g_d = _dev(g, dt)
    gh_d = torch.empty((batch, S) + cs, dtype=tdt, device="cuda")
    plan.analysis(g_d, gh_d)
    dg = _spec_np(d_d, plan)
    gh = _spec_np(gh_d, plan)
    for i, b in enumerate(items):
        ghat_o, d_o = orc[i][0], orc[i][1]
        ref = P.to_layout(fam, ghat_o).reshape(gh[b].shape)
        err = np.abs(gh[b] - ref).max() / np.abs(ref).max()
        assert err <= tol, f"analysis item {b}: {err:.3e}"
        dref = P.to_layout(fam, d_o).reshape(dg[0].shape)
        dgot = dg[b if psf_per_item else 0]
        # both sides sum in FP64 (in different orders): absolute floor ~ eps64 * sum|h|;
        # FP32 storage adds one rounding relative to each entry
        floor = 64 * 2.0 ** -53 * np.abs(hs[b if psf_per_item else 0]).sum()
        if prec == "fp64":
            assert np.abs(dgot - dref).max() <= max(1e-12 * np.abs(dref).max(), floor), "eigenvalues"
        else:
            assert np.all(np.abs(dgot - dref) <= 1e-6 * np.abs(dref) + floor), "eigenvalues"

    # ---- layer 1b: GCV, filter+synthesis and synthesis on identical (rounded oracle) inputs
    sT = P.sigma(fam, n)
    gin = np.zeros((batch, S), dtype=complex if plan.spec_complex else float)
    din = np.zeros((npsf, S), dtype=gin.dtype)
    full_in = {}
    for i, b in enumerate(items):
        ghat_o, d_o = orc[i][0], orc[i][1]
        gr, dr = _round(ghat_o, dt), _round(d_o, dt)
        full_in[b] = (gr, dr)
        cast = (lambda a: a) if plan.spec_complex else np.real
        gin[b] = cast(P.to_layout(fam, gr).reshape(-1))
        din[b if psf_per_item else 0] = cast(P.to_layout(fam, dr).reshape(-1))
    G_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    gin_d = _spec_dev(gin, plan, dt)
    din_d = _spec_dev(din, plan, dt)
    plan.gcv(gin_d, din_d, G_d, mi_d)
    mi_fix = np.array([orc[list(items).index(b)][4] if b in items else 0 for b in range(batch)], dtype=np.int32)
    f_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    plan.filter_synthesis(gin_d, din_d, _dev(mi_fix, np.int32), f_d)
    y_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    plan.synthesis(gin_d, y_d)
    G, mi, f, y = G_d.cpu().numpy(), mi_d.cpu().numpy(), f_d.cpu().numpy(), y_d.cpu().numpy()
    for i, b in enumerate(items):
        s_o = orc[i][2]
        gr, dr = full_in[b]
        Gref = O.gcv_curve(gr, dr, s_o, mus)
        gerr = np.max(np.abs(G[b] - Gref) / np.abs(Gref))
        assert gerr <= tol, f"G (identical inputs) item {b}: {gerr:.3e}"
        k = int(mi[b])
        kref = O.gcv_argmin(Gref)
        assert k == kref or Gref[k] <= (1 + tol) * Gref.min(), f"argmin {k} vs {kref}"
        X = O.filter_factors(dr, s_o, mus[mi_fix[b]]) * gr
        fref = P.oracle_filtered(fam, ndim, gr, dr, s_o, mus[mi_fix[b]])
        bound = max(tol * np.abs(fref).max(), rb * eps * sT * np.linalg.norm(X))
        ferr = np.abs(f[b] - fref).max()
        assert ferr <= bound, f"filter+synthesis item {b}: {ferr:.3e} > {bound:.3e}"
        yref = (O.synthesis_1d(fam, gr) if ndim == 1 else O.synthesis_2d(fam, gr)).real
        ybound = max(tol * np.abs(yref).max(), rb * eps * sT * np.linalg.norm(gr))
        yerr = np.abs(y[b] - yref).max()
        assert yerr <= ybound, f"synthesis item {b}: {yerr:.3e} > {ybound:.3e}"

    # ---- layer 2: the one-call path equals the GPU's own step sequence, bit for bit
    f1_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    mi1_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    G1_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    plan.gcv(gh_d, d_d, G1_d, mi1_d)
    plan.filter_synthesis(gh_d, d_d, mi1_d, f1_d)
    f2_d = torch.empty(g.shape, dtype=tdt, device="cuda")
    mi2_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    G2_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    plan.deblur(g_d, psf_d, f2_d, mi2_d, G2_d)
    assert torch.equal(f2_d, f1_d) and torch.equal(mi2_d, mi1_d) and torch.equal(G2_d, G1_d)

    # ---- layer 3: the whole path from g against the oracle.  The analysis error
    # norm is bounded by what layer 1 asserted (tol * max|ghat| per entry) and by the
    # FFT bound through ||T^{-1}||; it is magnified by the filter (kappa) and by T.
    f2, mi2, G2 = f2_d.cpu().numpy(), mi2_d.cpu().numpy(), G2_d.cpu().numpy()
    sTi = P.sigma(fam, n, inverse=True)
    for i, b in enumerate(items):
        ghat_o, d_o, s_o, G_o, k_o = orc[i]
        delta = min(rb * eps * sTi * np.linalg.norm(g[b]), tol * np.abs(ghat_o).max() * np.sqrt(ghat_o.size))
        k = int(mi2[b])
        a2 = np.abs(d_o) ** 2
        gbs = []
        for j, mu in enumerate(mus):
            sig = np.abs(s_o) ** 2 / (a2 + mu * np.abs(s_o) ** 2)
            num = np.sum(sig * sig * np.abs(ghat_o) ** 2)
            gb = max(tol, (2 * np.sqrt(np.sum(sig ** 4 * np.abs(ghat_o) ** 2)) * delta + sig.max() ** 2 * delta ** 2)
                     / num + (tol if prec == "fp32" else 0.0))
            gbs.append(gb)
            assert abs(G2[b, j] - G_o[j]) <= gb * G_o[j], f"end-to-end G mu {j}: bound {gb:.2e}"
        assert k == k_o or G_o[k] <= (1 + 2 * max(gbs)) * G_o.min(), "end-to-end argmin"
        fo = P.oracle_filtered(fam, ndim, ghat_o, d_o, s_o, mus[k])
        kappa = P.amplification(d_o, s_o, mus[k])
        X = O.filter_factors(d_o, s_o, mus[k]) * ghat_o
        bound = max(tol * np.abs(fo).max(), rb * eps * sT * np.linalg.norm(X) + sT * kappa * delta)
        ferr = np.abs(f2[b] - fo).max()
        assert ferr <= bound, f"end-to-end f item {b}: {ferr:.3e} > {bound:.3e}"
    return plan


CASES_1D = [(37, 5), (66, 7), (130, 5)]
CASES_2D = [((19, 34), (5, 5)), ((34, 21), (7, 7)), ((66, 40), (5, 5))]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("n,taps", CASES_1D)
def test_parity_1d(fam, n, taps, L, prec):
    run_case(1, fam, n, taps, L, prec, batch=5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("n,taps", CASES_2D)
def test_parity_2d(fam, n, taps, L, prec):
    run_case(2, fam, n, taps, L, prec, batch=3)


@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_parity_per_item_psf(fam, ndim):
    if ndim == 1:
        run_case(1, fam, 45, 5, "lap", "fp64", batch=4, psf_per_item=True)
    else:
        run_case(2, fam, (23, 30), (5, 5), "I", "fp32", batch=3, psf_per_item=True)


def test_identity_psf_closed_form():
    """h = delta, L = I: f = g/(1+mu*) exactly (d = 1), up to the rounding of a
    transform pair of condition number cond(T) (2e4 for degree 3 at n = 50)."""
    n = 50
    g = np.random.default_rng(3).standard_normal((4, n))
    mus = synth.mu_grid(8)
    for fam, deg in (("sine", 1), ("cosine", 2), ("fourier", 2), ("sine3", 3)):
        plan = hobc.Plan(1, n, 1, deg, mus, family=fam, psf_symmetric=True, batch=4)
        f = torch.empty((4, n), dtype=torch.float64, device="cuda")
        mi = torch.empty(4, dtype=torch.int32, device="cuda")
        plan.deblur(_dev(g, np.float64), _dev(np.ones(1), np.float64), f, mi)
        k = mi.cpu().numpy()
        cond = np.linalg.cond(O.transform_matrix(P.FAM_LETTER[fam], n))
        atol = 64 * 2.0 ** -53 * cond * np.abs(g).max()
        assert np.allclose(f.cpu().numpy(), g / (1 + mus[k])[:, None], rtol=0, atol=atol), fam


def test_zero_input_and_single_mu():
    """g = 0 gives G = 0 for every mu, mu* = index 0, f = 0; K = 1 works."""
    for K in (1, 5):
        mus = synth.mu_grid(K)
        plan = hobc.Plan(2, (20, 24), (5, 5), 2, mus, L="lap", family="cosine", psf_symmetric=True, batch=2)
        h = P.psf_for("C", 2, (5, 5))
        g = torch.zeros((2, 20, 24), dtype=torch.float64, device="cuda")
        f = torch.full_like(g, 7.0)
        mi = torch.full((2,), -1, dtype=torch.int32, device="cuda")
        G = torch.full((2, K), -1.0, dtype=torch.float64, device="cuda")
        plan.deblur(g, _dev(h, np.float64), f, mi, G)
        assert torch.all(f == 0) and torch.all(mi == 0) and torch.all(G == 0)


def test_minimum_size_and_host_entry_point():
    """Smallest field of view (n = 6, or 8 for degree 3, with a 3-tap PSF) and the host-buffer call."""
    mus = synth.mu_grid(6, 1e-4, 1.0)
    for fam, deg, n in (("sine", 1, 6), ("cosine", 2, 6), ("fourier", 2, 6), ("sine3", 3, 8)):
        h = np.array([0.25, 0.5, 0.25])
        g, _ = synth.problem_1d(1, n, h, 0.01, count=3)
        plan = hobc.Plan(1, n, 3, deg, mus, family=fam, psf_symmetric=True, batch=3)
        f = np.empty_like(g)
        mi = np.empty(3, dtype=np.int32)
        G = np.empty((3, 6))
        plan.deblur_host(g, h, f, mi, G)
        for b in range(3):
            fo, Go, ko, _ = O.deblur_1d(P.FAM_LETTER[fam], h, g[b], "I", mus)
            assert np.allclose(G[b], Go, rtol=1e-10)
            assert mi[b] == ko
            assert np.abs(f[b] - fo).max() <= 1e-10 * np.abs(fo).max()


@pytest.mark.parametrize("psf_per_item", [False, True])
@pytest.mark.parametrize("batch", [1, 4, 7])
def test_host_entry_point_equals_device_entry_point(batch, psf_per_item):
    """The chunked, two-stream host-buffer call gives the device call's results bit for bit."""
    n, taps, K = (30, 36), (5, 5), 12
    mus = synth.mu_grid(K)
    h0 = P.psf_for("F", 2, taps)
    hs = np.stack([h0 ** (1 + 0.1 * b) / (h0 ** (1 + 0.1 * b)).sum() for b in range(batch if psf_per_item else 1)])
    g, _ = P.problems(2, n, h0, batch, 8)
    plan = hobc.Plan(2, n, taps, 2, mus, family="fourier", batch=batch, psf_per_item=psf_per_item)
    f_h = torch.empty(g.shape, dtype=torch.float64).pin_memory().numpy()
    g_h = torch.from_numpy(g).pin_memory().numpy()
    mi_h = np.empty(batch, dtype=np.int32)
    G_h = np.empty((batch, K))
    plan.deblur_host(g_h, np.ascontiguousarray(hs), f_h, mi_h, G_h)
    f_d = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    G_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    plan.deblur(_dev(g, np.float64), _dev(hs, np.float64), f_d, mi_d, G_d)
    assert np.array_equal(f_h, f_d.cpu().numpy())
    assert np.array_equal(mi_h, mi_d.cpu().numpy())
    assert np.array_equal(G_h, G_d.cpu().numpy())
    assert plan.last_launch_count >= 7


@pytest.mark.parametrize("batch", [1, 4, 7])
def test_async_host_calls_overlap_and_equal_device_calls(batch):
    """Consecutive asynchronous host-buffer calls on one plan (different inputs and
    outputs, then the same output buffers again) give each call's device results
    bit for bit: a chunk's input and output slots are not reused before the
    previous call has read them."""
    n, taps, K = (30, 36), (5, 5), 12
    mus = synth.mu_grid(K)
    h0 = P.psf_for("F", 2, taps)
    hs = np.ascontiguousarray(h0[None])
    plan = hobc.Plan(2, n, taps, 2, mus, family="fourier", batch=batch)
    calls = 4
    gs = [P.problems(2, n, h0, batch, 20 + c)[0] for c in range(calls)]
    g_h = [torch.from_numpy(g).pin_memory().numpy() for g in gs]
    f_h = [torch.empty(gs[0].shape, dtype=torch.float64).pin_memory().numpy() for _ in range(calls)]
    mi_h = [torch.empty(batch, dtype=torch.int32).pin_memory().numpy() for _ in range(calls)]
    G_h = [torch.empty((batch, K), dtype=torch.float64).pin_memory().numpy() for _ in range(calls)]
    for c in range(calls):
        plan.deblur_host_async(g_h[c], hs, f_h[c], mi_h[c], G_h[c])
    plan.wait()
    f_same = torch.empty(gs[0].shape, dtype=torch.float64).pin_memory().numpy()
    mi_same = torch.empty(batch, dtype=torch.int32).pin_memory().numpy()
    for c in range(calls):                    # the same output buffers for every call: the last one wins
        plan.deblur_host_async(g_h[c], hs, f_same, mi_same, None)
    plan.wait()
    for c in range(calls):
        f_d = torch.empty(gs[0].shape, dtype=torch.float64, device="cuda")
        mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
        G_d = torch.empty((batch, K), dtype=torch.float64, device="cuda")
        plan.deblur(_dev(gs[c], np.float64), _dev(hs, np.float64), f_d, mi_d, G_d)
        assert np.array_equal(f_h[c], f_d.cpu().numpy()), c
        assert np.array_equal(mi_h[c], mi_d.cpu().numpy()), c
        assert np.array_equal(G_h[c], G_d.cpu().numpy()), c
        if c == calls - 1:
            assert np.array_equal(f_same, f_d.cpu().numpy())
            assert np.array_equal(mi_same, mi_d.cpu().numpy())


def test_caller_mu_index_out_of_range_is_clamped():
    """A caller-supplied mu index outside the grid is clamped on the device."""
    mus = synth.mu_grid(4, 1e-3, 1.0)
    h = P.psf_for("C", 1, 5)
    g, _ = synth.problem_1d(2, 40, h, 0.01, count=2)
    plan = hobc.Plan(1, 40, 5, 2, mus, family="cosine", psf_symmetric=True, batch=2)
    gh = torch.empty((2, plan.spec_elems), dtype=torch.float64, device="cuda")
    d = torch.empty((1, plan.spec_elems), dtype=torch.float64, device="cuda")
    plan.analysis(_dev(g, np.float64), gh)
    plan.eigenvalues(_dev(h, np.float64), d)
    f_bad = torch.empty((2, 40), dtype=torch.float64, device="cuda")
    f_ok = torch.empty_like(f_bad)
    plan.filter_synthesis(gh, d, _dev(np.array([-5, 99], np.int32), np.int32), f_bad)
    plan.filter_synthesis(gh, d, _dev(np.array([0, 3], np.int32), np.int32), f_ok)
    assert torch.equal(f_bad, f_ok)


# ------------------------------------------------------------ full-size configurations


def test_full_size_1d_signals_fp64():
    """1D: n = 256, symmetric Gaussian sigma 2 (9 taps), antireflective (degree 1), L = I,
    64 mu in [1e-8, 1], 1% noise, the 65,536-signal batch; 16 sampled signals vs the oracle."""
    h = synth.gaussian_psf_1d(2.0, 9)
    mus = synth.mu_grid(64)
    idx = [0, 1, 777, 4096, 30000, 65535] + list(range(10, 20))
    run_case(1, "sine", 256, 9, "I", "fp64", batch=65536, mus=mus, h0=h, check_items=idx)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_512_cosine_laplacian(prec):
    """2D 512 x 512, separable Gaussian 15 x 15 (sigma 2.5), degree 2 (cosine), Laplacian, 256 mu."""
    h = synth.gaussian_psf_2d_separable(2.5, 15)
    run_case(2, "cosine", (512, 512), (15, 15), "lap", prec, batch=1, mus=synth.mu_grid(256), h0=h, eta=0.005)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_1024_fourier(prec):
    """2D 1024 x 1024, rotated anisotropic Gaussian 21 x 21, degree 2 (Fourier), L = I, 256 mu --
    the benchmark workload, in the benchmark's launch configuration (batch of 2 here)."""
    h = synth.gaussian_psf_2d_rotated(3.0, 1.5, 30.0, 21, 2.0, -1.0)
    run_case(2, "fourier", (1024, 1024), (21, 21), "I", prec, batch=2, mus=synth.mu_grid(256), h0=h, eta=0.005,
             check_items=[1])
