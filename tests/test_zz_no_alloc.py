"""hobc_gcv_noalloc -- the GCV scan for callers that cannot allocate device
memory (their process runs under an allocator they do not own, or a fixed
device-memory budget, or a path that cannot take cudaMalloc's synchronisation)
-- must give the answer of hobc_gcv, the plan-based call, on the same spectra.
Both run the same kernels with the same chunking, so the answer must be the
same bit for bit; one case also checks it against the oracle on identical
inputs (the oracle's spectra rounded to the working precision).

Its scratch is one static device array shared by every call and never
cleared, so each case runs the allocation-free call twice in a row, and one
test alternates between two problem shapes.  This file is collected last on
purpose: if it fails, a run that stops at the first failure has already run
every other test.  It also passes alone, in a fresh process.
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


def _setup(ndim, n, fam, L, prec, batch, K, seed):
    """Spectra, eigenvalues and the plan-based GCV answer for one case."""
    letter = "P" if fam == "periodic" else P.FAM_LETTER[fam]     # periodic: the FFT-path family
    sym = letter not in ("F", "F4", "P")
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    taps = 5 if ndim == 1 else (5, 5)
    h = P.psf_for(letter, ndim, taps)
    g, _ = P.problems(ndim, (n,) if ndim == 1 else n, h, batch, seed)
    mus = synth.mu_grid(K, 1e-6, 1.0)
    deg = {"S": 1, "F4": 4, "P": 0}.get(letter, 2)
    plan = hobc.Plan(ndim, n, h.shape, deg, mus, L=L, prec=prec, family=fam, psf_symmetric=sym, batch=batch)
    cs = (2,) if plan.spec_complex else ()
    gh = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    d = torch.empty((1, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    plan.analysis(torch.from_numpy(g.astype(dt)).cuda(), gh)
    plan.eigenvalues(torch.from_numpy(h.astype(dt)).cuda(), d)
    G_ref = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    mi_ref = torch.empty(batch, dtype=torch.int32, device="cuda")
    plan.gcv(gh, d, G_ref, mi_ref)
    desc = hobc.make_desc(ndim, n, deg, K, L=L, prec=prec, family=fam, psf_symmetric=sym, batch=batch)
    mu_d = torch.from_numpy(mus).cuda()
    return desc, gh, d, mu_d, G_ref, mi_ref


def _noalloc(case):
    desc, gh, d, mu_d, G_ref, _ = case
    G = torch.full_like(G_ref, -1.0)
    mi = torch.full((G_ref.shape[0],), -1, dtype=torch.int32, device="cuda")
    hobc.gcv_noalloc(desc, gh, d, mu_d, G, mi)
    torch.cuda.synchronize()
    return G, mi


def _check(case, got, prec):
    G_ref, mi_ref = case[4], case[5]
    G, mi = got
    assert torch.equal(G, G_ref), f"G differs from hobc_gcv by {((G - G_ref).abs() / G_ref.abs()).max().item():.3e}"
    assert torch.equal(mi, mi_ref)


CASES = [
    (1, 77, "sine", "I", "fp64", 5, 24),
    (2, (34, 21), "cosine", "lap", "fp64", 3, 17),
    (2, (66, 40), "fourier", "I", "fp32", 4, 256),
    (2, (20, 17), "fourier4", "lap", "fp64", 2, 32),
    (1, 50, "periodic", "I", "fp32", 3, 40),
    (2, (33, 40), "periodic", "lap", "fp32", 3, 64),
]


@pytest.mark.parametrize("ndim,n,fam,L,prec,batch,K", CASES)
def test_noalloc_matches_plan_gcv_twice(ndim, n, fam, L, prec, batch, K):
    case = _setup(ndim, n, fam, L, prec, batch, K, seed=3)
    for _ in range(2):
        _check(case, _noalloc(case), prec)


def test_noalloc_alternating_shapes_do_not_see_stale_scratch():
    a = _setup(2, (66, 40), "fourier", "lap", "fp32", 6, 64, seed=5)
    b = _setup(1, 130, "cosine", "I", "fp64", 9, 31, seed=6)
    for _ in range(2):
        _check(a, _noalloc(a), "fp32")
        _check(b, _noalloc(b), "fp64")


def test_noalloc_rejects_requests_beyond_its_scratch():
    limit = hobc.gcv_noalloc_max_bytes()
    assert limit == 16 << 20
    desc = hobc.make_desc(2, (1024, 1024), 2, 256, prec="fp32", family="fourier", batch=64)
    with pytest.raises(hobc.HobcError) as ei:
        hobc.gcv_noalloc(desc, 16, 16, 16, None, 16)   # rejected before any device access
    assert hobc.STATUS[ei.value.status] == "HOBC_ERR_SIZE"
    assert "maximum" in str(ei.value)


@pytest.mark.parametrize("ndim,n,fam,L,prec", [
    (2, (34, 21), "fourier", "lap", "fp32"),
    (1, 90, "sine3", "I", "fp64"),
    (2, (20, 17), "periodic", "lap", "fp64"),
    (1, 30, "fourier4", "I", "fp64"),
])
def test_noalloc_against_the_oracle(ndim, n, fam, L, prec):
    """G of the allocation-free scan against the oracle's Eq. (eq:gcv2) on identical
    inputs: the oracle's spectrum and eigenvalues, rounded to the working precision,
    go to the GPU, and the oracle evaluates G on the same rounded values."""
    letter = "P" if fam == "periodic" else P.FAM_LETTER[fam]     # periodic: the FFT-path family
    sym = letter not in ("F", "F4", "P")
    dt = np.float64 if prec == "fp64" else np.float32
    shape = (n,) if ndim == 1 else n
    taps = 5 if ndim == 1 else (5, 5)
    h = P.psf_for(letter, ndim, taps)
    batch, K = 3, 40
    g, _ = P.problems(ndim, shape, h, batch, seed=11)
    mus = synth.mu_grid(K, 1e-7, 1.0)
    deg = {"S": 1, "C": 2, "F": 2, "S3": 3, "P": 0, "F4": 4}[letter]
    orc = [P.oracle_steps(letter, ndim, h, g[b], L, mus) for b in range(batch)]

    cplx = not sym                # the other families keep real spectra (the symbol's
                                  # imaginary rounding residue of a symmetric PSF is dropped)

    def rounded(full):
        re = full.real.astype(dt).astype(np.float64)
        return re + 1j * full.imag.astype(dt).astype(np.float64) if cplx else re

    def stored(full):
        lay = P.to_layout(letter, full).reshape(-1)
        if cplx:
            return np.stack([lay.real, lay.imag], axis=-1).astype(dt)
        return lay.real.astype(dt)

    gh_full = [rounded(o[0]) for o in orc]
    d_full = rounded(orc[0][1])
    gh = torch.from_numpy(np.stack([stored(x) for x in gh_full])).cuda()
    d = torch.from_numpy(stored(d_full)[None]).cuda()
    desc = hobc.make_desc(ndim, shape, deg, K, L=L, prec=prec, family=fam, psf_symmetric=sym, batch=batch)
    G = torch.empty((batch, K), dtype=torch.float64, device="cuda")
    mi = torch.empty(batch, dtype=torch.int32, device="cuda")
    for _ in range(2):
        hobc.gcv_noalloc(desc, gh, d, torch.from_numpy(mus).cuda(), G, mi)
        torch.cuda.synchronize()
        Gn, min_ = G.cpu().numpy(), mi.cpu().numpy()
        for b in range(batch):
            Gref = O.gcv_curve(gh_full[b], d_full, orc[b][2], mus)
            rel = np.max(np.abs(Gn[b] - Gref) / np.abs(Gref))
            assert rel <= TOL[prec], f"item {b}: G differs from the oracle by {rel:.3e}"
            k = int(min_[b])
            assert k == O.gcv_argmin(Gref) or Gref[k] <= (1 + TOL[prec]) * Gref.min()
