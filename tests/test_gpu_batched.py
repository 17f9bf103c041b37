"""Batched deblurring of 2D problems of uneven sizes, degrees and PSFs
(hobc_deblur_batched) against the single-geometry plan path -- itself pinned
to the oracle -- and directly against the oracle's G curve, mu* and f."""
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

FAM = {1: "sine", 2: "cosine", 3: "sine3"}
ITEMS = [(16, 20, 5, 3, 1), (33, 33, 7, 7, 2), (40, 28, 5, 5, 3), (9, 12, 3, 3, 1),
         (66, 31, 9, 5, 2), (25, 64, 5, 9, 3), (18, 18, 1, 1, 2)]


def _problems(items, seed):
    rng = np.random.default_rng(seed)
    gs, hs = [], []
    for (n0, n1, p0, p1, deg) in items:
        h = np.outer(synth.gaussian_psf_1d(rng.uniform(0.7, 1.6), p0), synth.gaussian_psf_1d(rng.uniform(0.7, 1.6), p1))
        h /= h.sum()
        g, _ = synth.problem_2d(int(rng.integers(1 << 30)), n0, n1, h, 0.01, count=1)
        gs.append(g[0])
        hs.append(h)
    return gs, hs


def _run(batch, gs, hs, dt, K):
    g = torch.from_numpy(np.concatenate([x.ravel() for x in gs]).astype(dt)).cuda()
    h = torch.from_numpy(np.concatenate([x.ravel() for x in hs]).astype(dt)).cuda()
    f = torch.empty_like(g)
    mi = torch.empty(len(gs), dtype=torch.int32, device="cuda")
    G = torch.empty((len(gs), K), dtype=torch.float64, device="cuda")
    batch.deblur(g, h, f, mi, G)
    torch.cuda.synchronize()
    return f.cpu().numpy(), mi.cpu().numpy(), G.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", ["I", "lap"])
def test_batched_matches_plan_and_oracle(prec, L):
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    K = 24
    mus = synth.mu_grid(K, 1e-6, 1.0)
    gs, hs = _problems(ITEMS, 11)
    gs = [x.astype(dt).astype(np.float64) for x in gs]
    hs = [x.astype(dt).astype(np.float64) for x in hs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = hobc.Batch(ITEMS, mus, L=L, prec=prec, stream=stream)
        f, mi, G = _run(batch, gs, hs, dt, K)
    assert batch.last_launch_count >= 5
    for i, (n0, n1, p0, p1, deg) in enumerate(ITEMS):
        fb = f[batch.img_off[i]:batch.img_off[i + 1]].reshape(n0, n1)
        # the single-geometry plan path on the same problem
        plan = hobc.Plan(2, (n0, n1), (p0, p1), deg, mus, L=L, prec=prec, family=FAM[deg], psf_symmetric=True)
        fp = torch.empty((1, n0, n1), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        mp = torch.empty(1, dtype=torch.int32, device="cuda")
        Gp = torch.empty((1, K), dtype=torch.float64, device="cuda")
        plan.deblur(torch.from_numpy(gs[i][None].astype(dt)).cuda(), torch.from_numpy(hs[i].astype(dt)).cuda(),
                    fp, mp, Gp)
        torch.cuda.synchronize()
        # the two paths sum the eigenvalues differently (cosine recurrence here, complex
        # tables there) before rounding them to the working precision, so an FP32 d may
        # differ by an ulp, which the GCV terms carry: G is compared at 4 tol in FP32
        gtol_plan = tol if prec == "fp64" else 4 * tol
        assert np.max(np.abs(G[i] - Gp.cpu().numpy()[0]) / Gp.cpu().numpy()[0]) <= gtol_plan, f"G vs plan, item {i}"
        assert mi[i] == mp.cpu().numpy()[0], f"mu* vs plan, item {i}"
        # the two paths differ only in how the eigenvalues are summed (cosine recurrence
        # here, complex tables there); the difference is magnified by cond(T0) cond(T1)
        fam = P.FAM_LETTER[FAM[deg]]
        cond = np.linalg.cond(O.transform_matrix(fam, n0)) * np.linalg.cond(O.transform_matrix(fam, n1))
        eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
        fpn = fp.cpu().numpy()[0]
        ftol = max(1e3 * tol, 64 * eps * cond)
        assert np.abs(fb - fpn).max() <= ftol * max(1.0, np.abs(fpn).max()), f"f vs plan, item {i}"
        # the oracle
        ghat, d, s, Go, ko = P.oracle_steps(fam, 2, hs[i], gs[i], L, mus)
        if prec == "fp64":
            gtol = max(1e-8, 1e-14 * cond)
            assert np.max(np.abs(G[i] - Go) / Go) <= gtol, f"G vs oracle, item {i}"
            assert mi[i] == ko or Go[mi[i]] <= (1 + gtol) * Go.min(), f"mu* vs oracle, item {i}"
            fo = P.oracle_filtered(fam, 2, ghat, d, s, mus[mi[i]])
            assert np.abs(fb - fo).max() <= max(1e-10, 1e-13 * cond) * max(1.0, np.abs(fo).max()), \
                f"f vs oracle, item {i}"


def test_graph_replay_equals_direct_launch_and_repeats():
    K = 16
    mus = synth.mu_grid(K, 1e-6, 1.0)
    gs, hs = _problems(ITEMS, 5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        graphed = hobc.Batch(ITEMS, mus, L="lap", prec="fp64", stream=stream)
        a = _run(graphed, gs, hs, np.float64, K)
        b = _run(graphed, gs, hs, np.float64, K)
    direct = hobc.Batch(ITEMS, mus, L="lap", prec="fp64", stream=None)
    c = _run(direct, gs, hs, np.float64, K)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_batched_rejects_bad_items():
    mus = synth.mu_grid(4)
    for bad, status in (((16, 16, 5, 5, 4), "HOBC_ERR_UNSUPPORTED"), ((16, 600, 5, 5, 1), "HOBC_ERR_SIZE"),
                        ((12, 12, 9, 9, 3), "HOBC_ERR_SIZE"), ((12, 12, 4, 3, 2), "HOBC_ERR_SIZE")):
        with pytest.raises(hobc.HobcError) as ei:
            hobc.Batch([(20, 20, 3, 3, 2), bad], mus)
        assert hobc.STATUS[ei.value.status] == status


BIG = [(130, 140, 5, 5, 1), (200, 150, 7, 7, 2), (150, 100, 5, 5, 3), (96, 257, 3, 9, 2), (64, 64, 3, 3, 1)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_schedule_radix8_matches_radix16_and_the_oracle(prec):
    """A schedule that runs every FFT of length >= 256 in radix 8 (hobc_batch_create_tuned)
    gives the default (radix 16) results to rounding, and the oracle's in FP64."""
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    K = 24
    mus = synth.mu_grid(K, 1e-6, 1.0)
    gs, hs = _problems(BIG, 23)
    gs = [x.astype(dt).astype(np.float64) for x in gs]
    hs = [x.astype(dt).astype(np.float64) for x in hs]
    kinds = sorted({(deg, hobc.fft_length(deg, n)) for (n0, n1, _, _, deg) in BIG for n in (n0, n1)})
    assert any(M >= 256 for _, M in kinds)
    sched8 = [(deg, M, 8) for deg, M in kinds if M >= 256]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b16 = hobc.Batch(BIG, mus, L="lap", prec=prec, stream=stream)
        b8 = hobc.Batch(BIG, mus, L="lap", prec=prec, stream=stream, schedule=sched8)
        f16, m16, G16 = _run(b16, gs, hs, dt, K)
        f8, m8, G8 = _run(b8, gs, hs, dt, K)
    assert b8.last_launch_count <= 7
    for i, (n0, n1, p0, p1, deg) in enumerate(BIG):
        fam = P.FAM_LETTER[FAM[deg]]
        cond = np.linalg.cond(O.transform_matrix(fam, n0)) * np.linalg.cond(O.transform_matrix(fam, n1))
        eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
        assert np.max(np.abs(G8[i] - G16[i]) / G16[i]) <= max(tol, 64 * eps * cond), f"G item {i}"
        assert m8[i] == m16[i] or G16[i][m8[i]] <= (1 + tol) * G16[i].min(), f"mu* item {i}"
        a = f8[b8.img_off[i]:b8.img_off[i + 1]]
        c = f16[b16.img_off[i]:b16.img_off[i + 1]]
        if m8[i] == m16[i]:
            assert np.abs(a - c).max() <= max(1e3 * tol, 64 * eps * cond) * max(1.0, np.abs(c).max()), f"f item {i}"
        if prec == "fp64":
            ghat, d, s, Go, ko = P.oracle_steps(fam, 2, hs[i], gs[i], "lap", mus)
            gtol = max(1e-8, 1e-14 * cond)
            assert np.max(np.abs(G8[i] - Go) / Go) <= gtol, f"G vs oracle, item {i}"
            fo = P.oracle_filtered(fam, 2, ghat, d, s, mus[m8[i]])
            assert np.abs(a.reshape(n0, n1) - fo).max() <= max(1e-10, 1e-13 * cond) * max(1.0, np.abs(fo).max())


def test_schedule_entries_are_checked():
    mus = synth.mu_grid(4)
    for bad in ((4, 512, 8), (2, 500, 8), (2, 512, 4)):
        with pytest.raises(hobc.HobcError) as ei:
            hobc.Batch([(20, 20, 3, 3, 2)], mus, schedule=[bad])
        assert hobc.STATUS[ei.value.status] == "HOBC_ERR_ARG"


def test_autotuner_writes_and_reuses_its_table(tmp_path):
    from paper_0906_2704_gb300 import autotune
    items = [(n, n, 3, 3, deg) for deg in (1, 2) for n in (130, 200, 300)]
    mus = synth.mu_grid(16)
    cache = str(tmp_path / "sched.json")
    sched, rec = autotune.tune_batched(items, mus, L="lap", prec="fp32", cache=cache, per_kind=8, reps=2, warmup=1)
    kinds = {(deg, hobc.fft_length(deg, n)) for (n, _, _, _, deg) in items}
    assert {(d_, M) for d_, M, _ in sched} == {k for k in kinds if k[1] >= 256}
    assert all(r in (8, 16) for _, _, r in sched)
    for name, v in rec.items():
        assert v["radix"] == (16 if v["ms_radix16"] <= v["ms_radix8"] else 8)
    sched2, _ = autotune.tune_batched(items, mus, L="lap", prec="fp32", cache=cache)   # from the cache
    assert sched2 == sched
    b = hobc.Batch(items, mus, L="lap", prec="fp32", stream=torch.cuda.current_stream(), schedule=sched)
    assert b.last_launch_count >= 0


@pytest.mark.parametrize("L", ["I", "lap"])
def test_batched_gcv_expansion_matches_the_direct_scan_and_the_oracle(L):
    """The batch's curve by bin expansion (gcv_mode="expansion"): every problem's G
    within the FP32 tolerance of the term-by-term batch curve (itself pinned to the
    plan path and the oracle above; two curves, each within 1e-5 of the exact one),
    the same mu index or one within it, f equal where the index is; the graph and a
    direct launch give the same bits; FP64 and over-wide grids refused."""
    K = 64
    mus = synth.mu_grid(K, 1e-8, 1.0)
    items = ITEMS + BIG
    gs, hs = _problems(items, 31)
    gs = [x.astype(np.float32).astype(np.float64) for x in gs]
    hs = [x.astype(np.float32).astype(np.float64) for x in hs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bd = hobc.Batch(items, mus, L=L, prec="fp32", stream=stream)
        bx = hobc.Batch(items, mus, L=L, prec="fp32", stream=stream, gcv_mode="expansion")
        fd, md, Gd = _run(bd, gs, hs, np.float32, K)
        fx, mx, Gx = _run(bx, gs, hs, np.float32, K)
        fx2, mx2, Gx2 = _run(bx, gs, hs, np.float32, K)
    direct = hobc.Batch(items, mus, L=L, prec="fp32", stream=None, gcv_mode="expansion")
    fx3, mx3, Gx3 = _run(direct, gs, hs, np.float32, K)
    for a, b, c in ((fx, fx2, fx3), (mx, mx2, mx3), (Gx, Gx2, Gx3)):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.max(np.abs(Gx - Gd) / Gd) <= 2e-5
    for i, (n0, n1, p0, p1, deg) in enumerate(items):
        k, kd = int(mx[i]), int(md[i])
        assert k == kd or Gd[i, k] <= (1 + 2e-5) * Gd[i, kd], (i, k, kd)
    same = mx == md
    off = np.concatenate([[0], np.cumsum([n0 * n1 for (n0, n1, *_r) in items])])
    for i in np.flatnonzero(same):
        assert np.array_equal(fx[off[i]:off[i + 1]], fd[off[i]:off[i + 1]])
    with pytest.raises(hobc.HobcError) as ei:
        hobc.Batch(ITEMS, mus, prec="fp64", gcv_mode="expansion")
    assert hobc.STATUS[ei.value.status] == "HOBC_ERR_UNSUPPORTED"
    with pytest.raises(hobc.HobcError) as ei:
        hobc.Batch(ITEMS, synth.mu_grid(8, 1e-18, 1e12), prec="fp32", gcv_mode="expansion")
    assert hobc.STATUS[ei.value.status] == "HOBC_ERR_UNSUPPORTED"
