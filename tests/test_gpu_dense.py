"""Parity of the dense split-BF16 mode (HOBC_SPLIT_BF16, include/hobc_tc.h)
with the FP64 oracle.

Each transform pass is a product with T_X^{-1} or T_X whose operands carry
about 16 bits (bf16 hi + lo), so each pass has an elementwise error of at most
(2^-14 + K 2^-24) |T||X| plus 2^-16 of its value when its output is split
again.  Two passes (2D) stay below 2^-11 of the absolute product:

  analysis          |ghat - oracle| <= 2^-11 |T^{-1}| |g| |T^{-1}|^T  (elementwise)
  synthesis         |y - oracle|    <= 2^-11 |T| |c| |T|^T
  filter+synthesis  as synthesis with c the filtered spectrum
  whole path        G within 1e-2 relative; mu* an index whose oracle G is within
                    that of the minimum; f within the analysis bound carried
                    through the filter and |T| plus the synthesis bound.
The Fourier family runs each complex product as a real product on (re, im)
pairs, so every output sums twice the terms and a complex entry has two
rounded parts: its bounds are four times those above (on the modulus).
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

DEG = {"sine": 1, "cosine": 2, "sine3": 3, "reflective": 0, "periodic": 0, "fourier": 2}
EPS = 2.0 ** -11


def _eps(F):
    return 4 * EPS if F == "F" else EPS


def _stored(F, full):
    """Oracle spectrum (full layout) -> the stored layout as float32 (re, im pairs for F)."""
    lay = P.to_layout(F, full).reshape(-1)
    if F == "F":
        return np.stack([lay.real, lay.imag], axis=-1)
    return lay.real


def _complex(F, arr):
    return arr[..., 0] + 1j * arr[..., 1] if F == "F" else arr


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _r32(x):
    return x.astype(np.float32).astype(np.float64)


def _case(ndim, fam, n, taps, L, batch=3, K=24, seed=0):
    F = P.FAM_LETTER[fam]
    n = (n,) if ndim == 1 else tuple(n)
    h = _r32(P.psf_for(F, ndim, taps))
    h = h / h.sum()
    g, ft = P.problems(ndim, n, h, batch, seed, 0.01)
    g = _r32(g)
    mus = synth.mu_grid(K, 1e-6, 1.0)
    plan = hobc.Plan(ndim, n, h.shape, DEG[fam], mus, L=L, prec="split_bf16", family=fam, psf_symmetric=True,
                     batch=batch)
    return F, n, h, g, mus, plan


def _status(plan):
    plan.status()


@pytest.mark.parametrize("L", ["I", "lap"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "sine3", "reflective", "periodic", "fourier"])
@pytest.mark.parametrize("ndim,n,taps", [(1, 70, 5), (1, 130, 7), (2, (40, 52), (5, 5)), (2, (66, 34), (7, 7))])
def test_dense_steps_match_oracle(ndim, n, taps, fam, L):
    F, n, h, g, mus, plan = _case(ndim, fam, n, taps, L)
    batch = g.shape[0]
    S = plan.spec_elems
    cs = (2,) if plan.spec_complex else ()
    g_d = _dev(g)
    gh_d = torch.empty((batch, S) + cs, dtype=torch.float32, device="cuda")
    plan.analysis(g_d, gh_d)
    y_d = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(1)
    c = _r32(rng.standard_normal((batch,) + n))                 # a spectrum in the oracle's full layout
    if F == "F":                                                # the half spectrum of a real signal
        c = np.stack([O.analysis_1d(F, c[b]) if ndim == 1 else O.analysis_2d(F, c[b]) for b in range(batch)])
        c = _r32(c.real) + 1j * _r32(c.imag)
    c_d = _dev(np.stack([_stored(F, c[b]) for b in range(batch)]))
    plan.synthesis(c_d, y_d)
    _status(plan)
    gh, y = _complex(F, gh_d.cpu().numpy().astype(np.float64)), y_d.cpu().numpy().astype(np.float64)
    eps = _eps(F)
    for b in range(batch):
        ref = O.analysis_1d(F, g[b]) if ndim == 1 else O.analysis_2d(F, g[b])
        bound = eps * P.abs_apply(F, g[b], inverse=True) + 1e-30
        want = P.to_layout(F, ref if F == "F" else ref.real)
        got = gh[b].reshape(want.shape)
        assert np.all(np.abs(got - want) <= P.to_layout(F, bound)), \
            f"analysis item {b}: {np.max(np.abs(got - want) / P.to_layout(F, bound)):.2f} of bound"
        yref = (O.synthesis_1d(F, c[b]) if ndim == 1 else O.synthesis_2d(F, c[b])).real
        ybound = eps * P.abs_apply(F, c[b]) + 1e-30
        assert np.all(np.abs(y[b] - yref) <= ybound), \
            f"synthesis item {b}: {np.max(np.abs(y[b] - yref) / ybound):.2f} of bound"


@pytest.mark.parametrize("fam", ["sine", "cosine", "sine3", "reflective", "periodic", "fourier"])
@pytest.mark.parametrize("ndim,n,taps", [(1, 90, 5), (2, (48, 40), (5, 5))])
def test_dense_deblur_matches_oracle(ndim, n, taps, fam):
    F, n, h, g, mus, plan = _case(ndim, fam, n, taps, "lap", batch=4, K=32, seed=3)
    batch = g.shape[0]
    f_d = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mi_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    G_d = torch.empty((batch, len(mus)), dtype=torch.float64, device="cuda")
    plan.deblur(_dev(g), _dev(h), f_d, mi_d, G_d)
    _status(plan)
    f, mi, G = f_d.cpu().numpy().astype(np.float64), mi_d.cpu().numpy(), G_d.cpu().numpy()
    for b in range(batch):
        ghat, d, s, Go, ko = P.oracle_steps(F, ndim, h, g[b], "lap", mus)
        assert np.all(np.abs(G[b] - Go) <= 1e-2 * Go), f"G item {b}"
        k = int(mi[b])
        assert k == ko or Go[k] <= (1 + 2e-2) * Go.min(), f"mu* item {b}"
        phi = np.abs(O.filter_factors(d, s, mus[k]))
        dg = _eps(F) * P.abs_apply(F, g[b], inverse=True)
        X = O.filter_factors(d, s, mus[k]) * ghat
        bound = P.abs_apply(F, phi * dg) + _eps(F) * P.abs_apply(F, X) + 1e-30
        fo = P.oracle_filtered(F, ndim, ghat, d, s, mus[k])
        assert np.all(np.abs(f[b] - fo) <= bound), f"f item {b}: {np.max(np.abs(f[b] - fo) / bound):.2f} of bound"


@pytest.mark.parametrize("ndim,n,taps", [(1, 64, 5), (2, (40, 44), (5, 5))])
def test_dense_host_call_equals_device_call(ndim, n, taps):
    """The chunked two-stream host call uses per-chunk operand workspace: bit-equal results."""
    F, n, h, g, mus, plan = _case(ndim, "cosine", n, taps, "lap", batch=7, K=16, seed=5)
    f_h = torch.empty(g.shape, dtype=torch.float32).pin_memory().numpy()
    g_h = torch.from_numpy(g.astype(np.float32)).pin_memory().numpy()
    mi_h = np.empty(7, dtype=np.int32)
    plan.deblur_host(g_h, np.ascontiguousarray(h, dtype=np.float32), f_h, mi_h)
    f_d = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mi_d = torch.empty(7, dtype=torch.int32, device="cuda")
    plan.deblur(_dev(g), _dev(h), f_d, mi_d)
    _status(plan)
    assert np.array_equal(f_h, f_d.cpu().numpy()) and np.array_equal(mi_h, mi_d.cpu().numpy())


def test_comparison_families_need_the_dense_mode_and_degree_zero():
    for prec in ("fp32", "fp64"):
        with pytest.raises(hobc.HobcError):
            hobc.Plan(2, (32, 32), (5, 5), 0, synth.mu_grid(8), prec=prec, family="reflective", psf_symmetric=True)
    with pytest.raises(hobc.HobcError):
        hobc.Plan(2, (32, 32), (5, 5), 2, synth.mu_grid(8), prec="split_bf16", family="periodic", psf_symmetric=True)
    with pytest.raises(hobc.HobcError):
        hobc.Plan(2, (32, 32), (5, 5), 0, synth.mu_grid(8), prec="split_bf16", family="periodic")


def test_dense_fourier_plan_for_a_nonsymmetric_psf():
    plan = hobc.Plan(2, (32, 32), (5, 5), 2, synth.mu_grid(8), prec="split_bf16", family="auto")
    assert plan.family == "fourier" and plan.spec_complex
