"""Parity of the learned choice of mu (include/hobc_learned.h) with the FP64
oracle (oracle/mlp_oracle.py, oracle/hobc_oracle.py).

  features      per bin, |x_gpu - x_oracle| <= 1e-5 + log10(1 + (2 sqrt(m) delta + delta^2) / m),
                m the oracle's bin mean of |ghat|^2 (|d|^2), delta the per-entry
                tolerance the analysis (eigenvalue) parity asserts
  network       forward and gradients against the oracle with the weight matrices
                rounded to bfloat16 (what the GPU multiplies by), FP32 accumulation
                bounds; AdamW steps on the same footing
  deblur        mu* and the fallback flag equal the oracle's bracket rule applied to
                the GPU's own prediction (decisions within rounding of a threshold
                are skipped); f against the oracle's filter at that mu* with the
                end-to-end bound of the plain path; a forced fallback equals
                hobc_deblur bit for bit
"""
import numpy as np
import pytest

from oracle import hobc_oracle as O
from oracle import mlp_oracle as M
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


def _spec_np(t, plan):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1] if plan.spec_complex else a


def _problems(n, batch, seed, taps=9, dt=np.float64):
    """Images blurred by disk PSFs of growing radius and noise of growing level."""
    rng = np.random.default_rng(seed)
    m = taps // 2
    g = np.empty((batch,) + tuple(n))
    hs = np.zeros((batch, taps, taps))
    for b in range(batch):
        d = synth.disk_psf(1.5 + 2.5 * b / max(1, batch - 1))
        k = d.shape[0] // 2
        hs[b, m - k:m + k + 1, m - k:m + k + 1] = d
        hs[b] = hs[b].astype(dt).astype(np.float64)
        f = synth.image_2d(rng, n[0] + 2 * m, n[1] + 2 * m)
        eta = 10.0 ** (-3 + 1.5 * b / max(1, batch - 1))
        g[b] = synth.add_noise(rng, synth.blur_valid_2d(f, hs[b]), eta)
    return g.astype(dt).astype(np.float64), hs


def _plan(fam, n, batch, prec, mus, taps=9):
    return hobc.Plan(2, n, (taps, taps), DEG[fam], mus, L="lap", prec=prec, family=fam, psf_symmetric=True,
                     batch=batch, psf_per_item=True)


def _bin_means(fam, n, a):
    b = M.radial_bins(fam, n[0], n[1]).ravel()
    cnt = np.bincount(b, minlength=M.NBINS)
    s = np.bincount(b, weights=np.abs(a.ravel()) ** 2, minlength=M.NBINS)
    return np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)


# --------------------------------------------------------------------- features

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
@pytest.mark.parametrize("n", [(40, 52), (66, 34)])
def test_features_match_oracle(fam, prec, n):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    batch = 3
    g, hs = _problems(n, batch, 11, dt=dt)
    plan = _plan(fam, n, batch, prec, synth.mu_grid(16))
    cs = (2,) if plan.spec_complex else ()
    D = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    G = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
    plan.eigenvalues(_dev(hs, dt), D)
    plan.analysis(_dev(g, dt), G)
    X = torch.empty((batch, 2 * M.NBINS), dtype=torch.float32, device="cuda")
    plan.features(G, D, X)
    x = X.cpu().numpy().astype(np.float64)
    tol = TOL[prec]
    for b in range(batch):
        ghat = O.analysis_2d(F, g[b])
        d = O.eigenvalues_2d(F, hs[b], n[0], n[1])
        xo = M.features(F, ghat, d)
        dg = tol * np.abs(ghat).max()
        dd = (1e-12 if prec == "fp64" else 1e-6) * np.abs(d).max() + 64 * 2.0 ** -53 * np.abs(hs[b]).sum()
        for part, (arr, delta) in enumerate(((ghat, dg), (d, dd))):
            m = _bin_means(F, n, arr)
            sl = slice(part * M.NBINS, (part + 1) * M.NBINS)
            with np.errstate(divide="ignore"):
                bound = 1e-5 + np.log10(1 + (2 * np.sqrt(m) * delta + delta ** 2 + 1e-37) / np.maximum(m, 1e-300))
            err = np.abs(x[b, sl] - xo[sl])
            assert np.all(err <= bound), f"item {b} part {part}: worst {np.max(err - bound):.3e} over bound"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam,ndim", [("cosine", 2), ("fourier", 2), ("sine3", 2), ("sine", 1), ("fourier", 1)])
def test_hist_features_match_oracle(fam, ndim, prec):
    """Histogram features on identical inputs (the oracle's spectra rounded to the
    working precision): shares within the mass of the entries whose a lies within
    rounding of a bin edge (they may land on either side) plus 1e-5 relative."""
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    eps = 2.0 ** -53 if prec == "fp64" else P.EPS32
    batch = 3
    n = (40, 52) if ndim == 2 else (130,)
    if ndim == 2:
        g, hs = _problems(n, batch, 13, dt=dt)
        plan = _plan(fam, n, batch, prec, synth.mu_grid(16))
    else:
        h = P.psf_for(F, 1, 7).astype(dt).astype(np.float64)
        hs = np.stack([h] * batch)
        g, _ = P.problems(1, n, h, batch, 13)
        g = g.astype(dt).astype(np.float64)
        plan = hobc.Plan(1, n, 7, DEG[fam], synth.mu_grid(16), L="lap", prec=prec, family=fam,
                         psf_symmetric=F != "F", batch=batch, psf_per_item=True)
    cplx = plan.spec_complex

    def stored(full):
        lay = P.to_layout(F, full).reshape(-1)
        return np.stack([lay.real, lay.imag], axis=-1) if cplx else lay.real

    def rnd(x):
        return x.real.astype(dt).astype(np.float64) + (1j * x.imag.astype(dt).astype(np.float64) if cplx else 0)
    full = []
    for b in range(batch):
        ghat, d, s, _, _ = P.oracle_steps(F, ndim, hs[b], g[b], "lap", synth.mu_grid(16))
        full.append((rnd(ghat), rnd(d), s))
    G = _dev(np.stack([stored(x[0]) for x in full]), dt)
    D = _dev(np.stack([stored(x[1]) for x in full]), dt)
    X = torch.empty((batch, 2 * M.NBINS), dtype=torch.float32, device="cuda")
    plan.features_hist(G, D, X)
    x = X.cpu().numpy().astype(np.float64)
    from oracle import binned_oracle as Bo
    edges = Bo.bin_edges(M.NBINS)[1:-1]
    for b, (gr, dr, s) in enumerate(full):
        xo = M.hist_features(gr, dr, s)
        m, a = Bo.a_values(dr.ravel(), s.ravel())
        e = np.abs(gr.ravel()[m]) ** 2
        near = np.min(np.abs(a[:, None] / edges[None, :] - 1.0), axis=1) < 16 * eps
        amb = {"E": e[near].sum() / e.sum(), "W": near.sum() / len(a)}
        for part, key in ((0, "E"), (1, "W")):
            sl = slice(part * M.NBINS, (part + 1) * M.NBINS)
            sg, so = 10.0 ** x[b, sl], 10.0 ** xo[sl]
            bound = 2 * amb[key] + 1e-5 * so + 1e-11
            assert np.all(np.abs(sg - so) <= bound), f"item {b} part {key}: {np.max(np.abs(sg - so) - bound):.3e}"


def test_fit_scaling_matches_mean_and_std():
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((1000, 128)) * rng.uniform(0.1, 3, 128) + rng.uniform(-5, 5, 128)).astype(np.float32)
    net = hobc.MLP(128, 32)
    net.fit_scaling(_dev(X, np.float32))
    torch.cuda.synchronize()
    flat = net.get_params()
    _, mean, scale = hobc.unpack_params(flat, 128, 32)
    X64 = X.astype(np.float64)
    assert np.allclose(mean, X64.mean(axis=0), rtol=1e-6, atol=1e-6)
    assert np.allclose(scale, X64.std(axis=0) + 1e-3, rtol=1e-6, atol=1e-6)
    net.set_feature_kind("hist")
    assert net.feature_kind == "hist"


# ---------------------------------------------------------------------- network

def _net_case(n_in, nh, B, seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(rng, n_in, nh)
    p["b1"] = 0.1 * rng.standard_normal(nh)
    p["b2"] = 0.1 * rng.standard_normal(nh)
    p["b3"] = np.array([0.3])
    mean = rng.standard_normal(n_in)
    scale = rng.uniform(0.5, 2.0, n_in)
    X = (rng.standard_normal((B, n_in)) * scale + mean).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    flat = hobc.pack_params(p, mean, scale)
    p32, mean32, scale32 = hobc.unpack_params(flat, n_in, nh)
    return flat, p32, mean32, scale32, X, t


def _bf16_weights(p):
    q = {k: v.copy() for k, v in p.items()}
    for k in ("W1", "W2", "w3"):
        q[k] = M.bf16_round(p[k])
    return q


@pytest.mark.parametrize("n_in,nh,B", [(128, 256, 37), (12, 40, 70), (128, 64, 1), (128, 256, 300)])
def test_mlp_forward_and_gradients_match_oracle(n_in, nh, B):
    flat, p32, mean, scale, X, t = _net_case(n_in, nh, B, 7)
    net = hobc.MLP(n_in, nh)
    assert net.param_count == nh * n_in + nh + nh * nh + nh + nh + 1
    net.set_params(flat)
    assert np.array_equal(net.get_params(), flat)
    x_d, t_d = _dev(X, np.float32), _dev(t, np.float32)
    y_d = torch.empty(B, dtype=torch.float32, device="cuda")
    net.forward(x_d, y_d)
    pb = _bf16_weights(p32)
    Xs = (X.astype(np.float64) - mean) / scale
    yo, (_, z1, h1, z2, h2) = M.forward(pb, Xs, mm=M.bf16_matmul)
    # FP32 accumulation: ~ (terms) * 2^-24 of the absolute sums, through two layers
    scale_y = np.abs(h2) @ np.abs(pb["w3"]) + 1.0
    assert np.all(np.abs(y_d.cpu().numpy() - yo) <= 2e-4 * scale_y)
    grad_d = torch.empty(net.param_count, dtype=torch.float32, device="cuda")
    loss_d = torch.empty(1, dtype=torch.float32, device="cuda")
    net.gradients(x_d, t_d, grad_d, loss_d)
    lo, go = M.loss_and_grads(pb, Xs, t.astype(np.float64), mm=M.bf16_matmul)
    assert abs(loss_d.item() - lo) <= 1e-4 * (1 + lo)
    got, _, _ = hobc.unpack_params(np.concatenate([grad_d.cpu().numpy(), np.zeros(2 * n_in)]), n_in, nh)
    for k in go:
        ref = np.asarray(go[k]).reshape(got[k].shape)
        err = np.abs(got[k] - ref).max()
        assert err <= 2e-3 * np.abs(ref).max() + 1e-7, f"grad {k}: {err:.3e} vs max {np.abs(ref).max():.3e}"


def test_adamw_steps_match_oracle():
    """Two AdamW steps against the oracle's optimiser fed the same gradients (the
    GPU's own, read before each step; their parity with the oracle's gradients is
    the test above): the update arithmetic agrees to FP32 rounding."""
    n_in, nh, B = 128, 64, 96
    flat, p32, mean, scale, X, t = _net_case(n_in, nh, B, 3)
    net = hobc.MLP(n_in, nh)
    net.set_params(flat)
    x_d, t_d = _dev(X, np.float32), _dev(t, np.float32)
    lr, wd = 1e-3, 1e-2
    po = {k: v.astype(np.float64).copy() for k, v in p32.items()}
    m = {k: np.zeros_like(v) for k, v in po.items()}
    v = {k: np.zeros_like(x) for k, x in po.items()}
    grad_d = torch.empty(net.param_count, dtype=torch.float32, device="cuda")
    loss_d = torch.empty(1, dtype=torch.float32, device="cuda")
    for step in (1, 2):
        net.gradients(x_d, t_d, grad_d, loss_d)
        g, _, _ = hobc.unpack_params(np.concatenate([grad_d.cpu().numpy(), np.zeros(2 * n_in)]), n_in, nh)
        g = {k: np.asarray(x, dtype=np.float64).reshape(po[k].shape) for k, x in g.items()}
        net.train_step(x_d, t_d, lr, wd)
        M.adamw_step(po, g, m, v, step, lr, wd=wd)
    got, _, _ = hobc.unpack_params(net.get_params(), n_in, nh)
    for k in po:
        diff = np.abs(got[k] - po[k])
        assert np.all(diff <= 1e-3 * lr + 2e-6 * np.abs(po[k])), (k, float(diff.max()))


def test_mlp_checkpoint_round_trip(tmp_path):
    n_in, nh = 128, 32
    flat, _, _, _, X, t = _net_case(n_in, nh, 40, 5)
    net = hobc.MLP(n_in, nh)
    net.set_params(flat)
    net.train_step(_dev(X, np.float32), _dev(t, np.float32), 1e-3)
    path = str(tmp_path / "net.bin")
    net.save(path)
    other = hobc.MLP(n_in, nh)
    other.load(path)
    assert np.array_equal(other.get_params(), net.get_params())
    y1 = torch.empty(40, dtype=torch.float32, device="cuda")
    y2 = torch.empty(40, dtype=torch.float32, device="cuda")
    net.forward(_dev(X, np.float32), y1)
    other.forward(_dev(X, np.float32), y2)
    assert torch.equal(y1, y2)
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0x01
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(hobc.HobcError):
        other.load(bad)
    with pytest.raises(hobc.HobcError):
        hobc.MLP(n_in, nh + 1).load(path)
    with pytest.raises(hobc.HobcError):
        other.load(str(tmp_path / "missing.bin"))


# ---------------------------------------------------------------- learned deblur

def _set_constant(net, n_in, nh, c):
    p = {"W1": np.zeros((nh, n_in)), "b1": np.zeros(nh), "W2": np.zeros((nh, nh)), "b2": np.zeros(nh),
         "w3": np.zeros(nh), "b3": np.array([c])}
    net.set_params(hobc.pack_params(p, np.zeros(n_in), np.ones(n_in)))


def _run_learned(plan, net, g, hs, dt, tdt):
    batch = g.shape[0]
    f = torch.empty(g.shape, dtype=tdt, device="cuda")
    mu = torch.empty(batch, dtype=torch.float64, device="cuda")
    fb = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
    plan.deblur_learned(net, _dev(g, dt), _dev(hs, dt), f, mu, fb)
    return f.cpu().numpy(), mu.cpu().numpy(), fb.cpu().numpy()


@pytest.mark.parametrize("kind", ["radial", "hist"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", ["sine", "cosine", "fourier", "sine3"])
def test_deblur_learned_matches_oracle(fam, prec, kind):
    F = P.FAM_LETTER[fam]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    eps = 2.0 ** -53 if prec == "fp64" else P.EPS32
    tol = TOL[prec]
    n, batch, K = (48, 56), 6, 48
    mus = synth.mu_grid(K, 1e-8, 1.0)
    g, hs = _problems(n, batch, 21, dt=dt)
    plan = _plan(fam, n, batch, prec, mus)
    orc = [P.oracle_steps(F, 2, hs[b], g[b], "lap", mus) for b in range(batch)]
    sT, sTi = P.sigma(F, n), P.sigma(F, n, inverse=True)
    rb = 16.0 * P.log2_fft(F, n) + 2.0 * sum(np.sqrt(v) for v in n)
    # a network with random weights, inputs standardised on these problems' features
    nh = 48
    rng = np.random.default_rng(2)
    p = M.init_params(rng, 2 * M.NBINS, nh)
    if kind == "radial":
        xo = np.stack([M.features(F, orc[b][0], orc[b][1]) for b in range(batch)])
    else:
        xo = np.stack([M.hist_features(orc[b][0], orc[b][1], orc[b][2]) for b in range(batch)])
    c0 = np.log10(mus[orc[0][4]])
    p["b3"] = np.array([c0])
    net = hobc.MLP(2 * M.NBINS, nh)
    net.set_params(hobc.pack_params(p, xo.mean(axis=0), xo.std(axis=0) + 1e-3))
    net.set_feature_kind(kind)
    checked = 0
    for case in ("random", "constant", "low", "high"):
        if case == "constant":
            _set_constant(net, 2 * M.NBINS, nh, c0 + 0.03)
        elif case == "low":
            _set_constant(net, 2 * M.NBINS, nh, -30.0)
        elif case == "high":
            _set_constant(net, 2 * M.NBINS, nh, 30.0)
        f, mu, fb = _run_learned(plan, net, g, hs, dt, tdt)
        # the GPU's own prediction for these problems
        cs = (2,) if plan.spec_complex else ()
        D = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
        G = torch.empty((batch, plan.spec_elems) + cs, dtype=tdt, device="cuda")
        plan.eigenvalues(_dev(hs, dt), D)
        plan.analysis(_dev(g, dt), G)
        X = torch.empty((batch, 2 * M.NBINS), dtype=torch.float32, device="cuda")
        if kind == "radial":
            plan.features(G, D, X)
        else:
            plan.features_hist(G, D, X)
        y = torch.empty(batch, dtype=torch.float32, device="cuda")
        net.forward(X, y)
        y = y.cpu().numpy().astype(np.float64)
        for b in range(batch):
            ghat_o, d_o, s_o, G_o, k_o = orc[b]
            Gat = lambda m_, gh=ghat_o, dd=d_o, ss=s_o: O.gcv_curve(gh, dd, ss, np.atleast_1d(m_))
            mu_o, fb_o = M.learned_choice(Gat, mus, y[b])
            # skip decisions that sit within rounding of a threshold
            lg = np.log10(mus)
            l = min(max(y[b], lg[0]), lg[-1])
            mh = 10.0 ** l
            kn = int(np.argmin(np.abs(lg - l)))
            span = min(17, K)
            k0 = max(0, min(kn - span // 2, K - span))
            Gb = Gat(mus[k0:k0 + span])
            srt = np.sort(Gb)
            gtol = 1e3 * tol
            near = (abs(Gat(mh)[0] / Gb.min() - 1.05) < gtol or (srt[1] - srt[0]) / srt[0] < gtol
                    or np.sort(np.abs(lg - l))[1] - np.abs(lg - l)[kn] < 1e-9)
            if near:
                continue
            checked += 1
            assert fb[b] == int(fb_o), f"{case} item {b}: fell_back {fb[b]} vs {fb_o}"
            if fb_o:
                assert G_o[np.searchsorted(mus, mu[b])] <= (1 + gtol) * G_o.min(), f"{case} item {b}: fallback mu"
                assert np.any(mus == mu[b]), "a fallback mu is a grid value"
            else:
                assert abs(mu[b] - mu_o) <= 1e-12 * mu_o, f"{case} item {b}: mu {mu[b]} vs {mu_o}"
            # f against the oracle's filter at the GPU's mu*
            delta = min(rb * eps * sTi * np.linalg.norm(g[b]), tol * np.abs(ghat_o).max() * np.sqrt(ghat_o.size))
            fo = P.oracle_filtered(F, 2, ghat_o, d_o, s_o, mu[b])
            kappa = P.amplification(d_o, s_o, mu[b])
            Xf = O.filter_factors(d_o, s_o, mu[b]) * ghat_o
            bound = max(tol * np.abs(fo).max(), rb * eps * sT * np.linalg.norm(Xf) + sT * kappa * delta)
            ferr = np.abs(f[b] - fo).max()
            assert ferr <= bound, f"{case} item {b}: f {ferr:.3e} > {bound:.3e}"
        if case == "constant":
            assert fb[0] == 0, "a prediction next to the GCV minimum is kept"
        if case in ("low", "high"):
            # forced fallback (unless the minimum is at that end of the grid): equals hobc_deblur
            f2 = torch.empty(g.shape, dtype=tdt, device="cuda")
            mi = torch.empty(batch, dtype=torch.int32, device="cuda")
            plan.deblur(_dev(g, dt), _dev(hs, dt), f2, mi)
            mi, f2 = mi.cpu().numpy(), f2.cpu().numpy()
            fell = 0
            for b in range(batch):
                if fb[b] == 1:
                    fell += 1
                    assert mu[b] == mus[mi[b]]
                    assert np.array_equal(f[b], f2[b]), f"{case} item {b}: not bit-equal to hobc_deblur"
            assert fell >= 1, f"{case}: a prediction at the end of the grid never fell back"
    assert checked >= 2 * batch       # a 17-wide bracket on a flat curve has more near-ties to skip


def test_deblur_learned_rejects_bad_shapes():
    mus = synth.mu_grid(8)
    plan1 = hobc.Plan(1, 40, 5, 2, mus, family="cosine", psf_symmetric=True)
    net = hobc.MLP(2 * M.NBINS, 16)
    t = torch.zeros(40, dtype=torch.float64, device="cuda")
    with pytest.raises(hobc.HobcError):
        plan1.deblur_learned(net, t, t, t)
    plan2 = _plan("cosine", (20, 24), 1, "fp64", mus, taps=5)
    small = hobc.MLP(12, 16)
    g = torch.zeros((1, 20, 24), dtype=torch.float64, device="cuda")
    with pytest.raises(hobc.HobcError):
        plan2.deblur_learned(small, g, torch.zeros(25, dtype=torch.float64, device="cuda"), g)
    plan3 = _plan("cosine", (20, 24), 1, "fp64", mus[::-1].copy(), taps=5)
    with pytest.raises(hobc.HobcError, match="increasing"):
        plan3.deblur_learned(net, g, torch.zeros(25, dtype=torch.float64, device="cuda"), g)


def test_features_and_learned_path_are_deterministic():
    """Same input, same features and mu* bit for bit (no order-dependent sums)."""
    n, batch = (64, 70), 4
    mus = synth.mu_grid(32)
    g, hs = _problems(n, batch, 5, dt=np.float32)
    plan = _plan("cosine", n, batch, "fp32", mus)
    D = torch.empty((batch, plan.spec_elems), dtype=torch.float32, device="cuda")
    G = torch.empty((batch, plan.spec_elems), dtype=torch.float32, device="cuda")
    plan.eigenvalues(_dev(hs, np.float32), D)
    plan.analysis(_dev(g, np.float32), G)
    X1 = torch.empty((batch, 2 * M.NBINS), dtype=torch.float32, device="cuda")
    X2 = torch.empty_like(X1)
    plan.features(G, D, X1)
    plan.features(G, D, X2)
    assert torch.equal(X1, X2)
    net = hobc.MLP(2 * M.NBINS, 32)
    p = M.init_params(np.random.default_rng(0), 2 * M.NBINS, 32)
    x = X1.cpu().numpy().astype(np.float64)
    net.set_params(hobc.pack_params(p, x.mean(axis=0), x.std(axis=0) + 1e-3))
    a = _run_learned(plan, net, g, hs, np.float32, torch.float32)
    b = _run_learned(plan, net, g, hs, np.float32, torch.float32)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
