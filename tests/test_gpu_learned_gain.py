"""What the trained network gains over the method without it (include/hobc_learned.h).

The plain method scans G (Eq. (eq:gcv2)) at all K grid values.  The learned
path evaluates G at the network's prediction and the 17 grid values around it
and scans in full only when the prediction fails the bracket rule (reading R9).
A network trained on GCV labels of problems drawn like the held-out ones
(64 x 64, cosine family, disk PSFs of random radius, random noise level,
Laplacian, 128 mu) must
  * fall back on well under half of the held-out problems, and on far fewer than a
    network that predicts the mean label for every problem (the same bracket
    without learning);
  * so evaluate G at far fewer grid values per problem than the full scan;
  * keep G (at the grid value nearest its mu*) within 2% of the full scan's
    minimum on average where it keeps the prediction;
  * and reconstruct as well as the full scan (mean relative error within 2%).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc, learned as LR, synth  # noqa: E402


def test_trained_network_beats_the_untrained_bracket_and_the_full_scan():
    n, K, taps, B = 64, 128, 11, 512
    mus = synth.mu_grid(K)
    plan = hobc.Plan(2, (n, n), (taps, taps), 2, mus, L="lap", prec="fp32", family="cosine", psf_symmetric=True,
                     batch=B, psf_per_item=True)
    Xtr, ttr = LR.training_set(plan, 16384, 1, "disk", taps, kind="hist")
    net = LR.init_network(Xtr, 256, seed=0, kind="hist")
    LR.fit(net, Xtr, ttr, epochs=30, batch=256, lr=1e-3)
    # the same bracket without learning: every prediction the mean training label
    base = LR.init_network(Xtr, 256, seed=0, kind="hist")
    p, mean, scale = hobc.unpack_params(base.get_params(), 128, 256)
    flat = {k: np.zeros_like(v) for k, v in p.items()}
    flat["b3"] = np.array([float(ttr.mean())])
    base.set_params(hobc.pack_params(flat, mean, scale))

    dev = torch.device("cuda", 0)
    count = 1024
    g, h, ft, _ = LR.gpu_problems(count, n, 2 * 1000003, dev, psf="disk", taps=taps, truth=True)
    out = {}
    for name, nt in (("learned", net), ("untrained", base)):
        f = torch.empty_like(g)
        mu = torch.empty(count, dtype=torch.float64, device=dev)
        fb = torch.empty(count, dtype=torch.int32, device=dev)
        for s in range(0, count, B):
            plan.deblur_learned(nt, g[s:s + B], h[s:s + B], f[s:s + B], mu[s:s + B], fb[s:s + B])
        out[name] = (f, mu.cpu().numpy(), fb.cpu().numpy())
    # the plain method: full scan, its G curve and its f
    f_g = torch.empty_like(g)
    mi = torch.empty(count, dtype=torch.int32, device=dev)
    G = torch.empty((count, K), dtype=torch.float64, device=dev)
    for s in range(0, count, B):
        plan.deblur(g[s:s + B], h[s:s + B], f_g[s:s + B], mi[s:s + B], G[s:s + B])
    G = G.cpu().numpy()
    Gmin = G.min(axis=1)

    f_l, mu_l, fb_l = out["learned"]
    fb_u = out["untrained"][2]
    rate_l, rate_u = fb_l.mean(), fb_u.mean()
    assert rate_l < 0.5, f"learned fallback rate {rate_l:.3f}"
    assert rate_l < 0.6 * rate_u, f"learned {rate_l:.3f} vs untrained {rate_u:.3f}"
    evals = 18 + rate_l * K
    assert evals < 0.6 * K, f"{evals:.1f} evaluations per problem against {K}"
    # G near mu*: the kept prediction's G is within 5% of its bracket's minimum; compare the
    # grid value nearest to mu* with the full scan's minimum
    kept = fb_l == 0
    ratio = []
    for b in np.flatnonzero(kept):
        k = int(np.argmin(np.abs(np.log10(mus) - np.log10(mu_l[b]))))
        ratio.append(G[b, k] / Gmin[b])
    ratio = np.array(ratio)
    assert np.mean(ratio) < 1.02, f"mean G ratio {np.mean(ratio):.4f}"

    def rre(f):
        d = (f.double() - ft.double()).flatten(1)
        return (d.norm(dim=1) / ft.double().flatten(1).norm(dim=1)).cpu().numpy()
    r_l, r_g = rre(f_l), rre(f_g)
    assert r_l.mean() <= 1.02 * r_g.mean(), f"RRE {r_l.mean():.4f} vs full scan {r_g.mean():.4f}"
