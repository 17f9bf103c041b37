"""Parity of the binned choice of mu (include/hobc_binned.h) with the FP64
oracle (oracle/binned_oracle.py, oracle/hobc_oracle.py).

On identical inputs (the oracle's spectra rounded to the working precision go
to both sides):
  k_hat     the oracle's binned curve at the GPU's k_hat is within 1e-3 of its
            minimum (bins are decided in the working precision on the GPU, so an
            entry within rounding of an edge may land in the neighbouring bin,
            and G_bin is evaluated in FP32)
  mu*, flag the oracle's bracket rule around the GPU's k_hat gives the same grid
            index and fallback flag, unless the bracket's two smallest exact G
            values are within the G tolerance of each other
Whole path: where the binned index equals hobc_deblur's, f is bit-equal.
"""
import numpy as np
import pytest

from oracle import binned_oracle as Bn
from oracle import hobc_oracle as O
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


def _disk_problems(n, batch, seed, taps=9):
    rng = np.random.default_rng(seed)
    m = taps // 2
    g = np.empty((batch,) + tuple(n))
    hs = np.zeros((batch, taps, taps))
    for b in range(batch):
        d = synth.disk_psf(1.5 + 2.5 * ((b * 0.37) % 1.0))
        k = d.shape[0] // 2
        hs[b, m - k:m + k + 1, m - k:m + k + 1] = d
        f = synth.image_2d(rng, n[0] + 2 * m, n[1] + 2 * m)
        g[b] = synth.add_noise(rng, synth.blur_valid_2d(f, hs[b]), 10.0 ** (-3 + 1.5 * ((b * 0.61) % 1.0)))
    return g, hs


def _case(ndim, fam, prec, L, K=64, batch=5, seed=3):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    mus = synth.mu_grid(K)
    if ndim == 1:
        n, taps = (70,), 7
        h = P.psf_for(F, 1, taps)
        hs = np.stack([h] * batch)
        g, _ = synth.problem_1d(seed, n[0], h, 0.01, count=batch)
    else:
        n, taps = (40, 46), 9
        g, hs = _disk_problems(n, batch, seed, taps)
        if F == "F":                       # a nonsymmetric PSF for the Fourier family
            hs = np.stack([P.psf_for("F", 2, (taps, taps))] * batch)
    hs = np.stack([_round(h / h.sum(), dt) for h in hs])
    g = _round(g, dt)
    plan = hobc.Plan(ndim, n, (taps,) * ndim, DEG[fam], mus, L=L, prec=prec, family=fam,
                     psf_symmetric=F != "F", batch=batch, psf_per_item=True)
    return F, dt, tdt, mus, n, g, hs, plan


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_binned_choice_matches_oracle_on_identical_inputs(ndim, fam, L, prec):
    F, dt, tdt, mus, n, g, hs, plan = _case(ndim, fam, prec, L)
    batch, K = g.shape[0], len(mus)
    tol = TOL[prec]
    orc = [P.oracle_steps(F, ndim, hs[b] if ndim == 2 else hs[b], g[b], L, mus) for b in range(batch)]
    cplx = plan.spec_complex
    gin = np.zeros((batch, plan.spec_elems), dtype=complex if cplx else float)
    din = np.zeros_like(gin)
    full = []
    for b in range(batch):
        gr, dr = _round(orc[b][0], dt), _round(orc[b][1], dt)
        full.append((gr, dr))
        cast = (lambda a: a) if cplx else np.real
        gin[b] = cast(P.to_layout(F, gr).reshape(-1))
        din[b] = cast(P.to_layout(F, dr).reshape(-1))
    def spec(a):
        return _dev(np.stack([a.real, a.imag], axis=-1) if cplx else a.real, dt)
    mi = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
    fb = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
    kh = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
    plan.gcv_binned(spec(gin), spec(din), mi, fb, kh)
    mi, fb, kh = mi.cpu().numpy(), fb.cpu().numpy(), kh.cpu().numpy()
    checked = 0
    for b in range(batch):
        gr, dr = full[b]
        s_o = orc[b][2]
        Gbin = Bn.binned_curve(*Bn.histogram(gr, dr, s_o), mus)
        assert 0 <= kh[b] < K
        assert Gbin[kh[b]] <= (1 + 1e-3) * np.nanmin(Gbin), f"item {b}: k_hat {kh[b]} vs {Bn.first_argmin(Gbin)}"
        G_at = lambda m_, gr=gr, dr=dr, s_o=s_o: O.gcv_curve(gr, dr, s_o, np.atleast_1d(m_))
        onehot = np.ones(K)
        onehot[kh[b]] = 0.0
        k_o, fb_o, _ = Bn.binned_choice(G_at, onehot, mus)
        span = min(9, K)
        k0 = max(0, min(int(kh[b]) - span // 2, K - span))
        Gb = np.sort(G_at(mus[k0:k0 + span]))
        if (Gb[1] - Gb[0]) <= 10 * tol * Gb[0]:
            continue
        checked += 1
        assert fb[b] == int(fb_o), f"item {b}: fell_back {fb[b]} vs {fb_o}"
        if fb_o:
            Gf = G_at(mus)
            assert mi[b] == k_o or Gf[mi[b]] <= (1 + 10 * tol) * Gf.min(), f"item {b}: fallback index"
        else:
            assert mi[b] == k_o, f"item {b}: index {mi[b]} vs {k_o}"
    assert checked >= batch - 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
def test_deblur_binned_equals_full_scan_where_the_choice_agrees(fam, prec):
    F, dt, tdt, mus, n, g, hs, plan = _case(2, fam, prec, "lap", K=96, batch=8, seed=9)
    batch = g.shape[0]
    g_d, h_d = _dev(g, dt), _dev(hs, dt)
    f1 = torch.empty(g.shape, dtype=tdt, device="cuda")
    f2 = torch.empty_like(f1)
    m1 = torch.empty(batch, dtype=torch.int32, device="cuda")
    m2 = torch.empty_like(m1)
    fb = torch.empty_like(m1)
    plan.deblur(g_d, h_d, f1, m1)
    plan.deblur_binned(g_d, h_d, f2, m2, fb)
    m1, m2, f1, f2 = m1.cpu().numpy(), m2.cpu().numpy(), f1.cpu().numpy(), f2.cpu().numpy()
    same = m1 == m2
    assert same.mean() >= 0.75, f"binned index agrees with the full scan on {same.mean():.2f} of the problems"
    for b in np.nonzero(same)[0]:
        assert np.array_equal(f1[b], f2[b])
    # again: deterministic
    f3 = torch.empty_like(torch.from_numpy(f2)).cuda()
    m3 = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.deblur_binned(g_d, h_d, f3, m3)
    assert np.array_equal(m3.cpu().numpy(), m2) and np.array_equal(f3.cpu().numpy(), f2)


def test_binned_rejects_a_decreasing_grid():
    mus = synth.mu_grid(8)[::-1].copy()
    plan = hobc.Plan(1, 40, 5, 2, mus, family="cosine", psf_symmetric=True)
    t = torch.zeros(40, dtype=torch.float64, device="cuda")
    mi = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(hobc.HobcError, match="increasing"):
        plan.deblur_binned(t, torch.ones(5, dtype=torch.float64, device="cuda"), t, mi)
