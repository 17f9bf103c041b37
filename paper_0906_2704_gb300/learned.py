"""Training and use of the mu-predicting network (include/hobc_learned.h).

Everything numeric of the method runs in the library: the labels are the GCV
choice of the plain path (hobc_gcv), the inputs its features (hobc_features or
hobc_features_hist), the input scaling hobc_mlp_fit_scaling, and the network
is trained with hobc_mlp_train_step.  This module moves batches around (device
tensors; torch is used for allocation and indexing) and, for training sets
too large to build on the host, draws seeded synthetic problems on the GPU
with the recipe of synth.py (gpu_problems): that is input generation, not a
step of the method.
"""
from __future__ import annotations

import numpy as np

from . import hobc


def _torch():
    import torch
    return torch


def gpu_problems(count: int, n: int, seed: int, device, psf: str = "disk", taps: int = 11,
                 eta=(1e-3, 3e-2), truth: bool = False):
    """``count`` seeded n x n problems drawn on the GPU with the recipe of synth.py:
    per image a linear ramp plus 20 random degree-<=2 polynomials on random
    rectangles of the field of view extended by m = taps // 2 on each side, its
    valid convolution with the image's own PSF, and noise of relative level
    log-uniform in ``eta`` (e scaled to eta ||g|| / ||e||).  PSFs: "disk" --
    a uniform disk of radius U[1.5, min(5, m)] centred in the taps x taps array;
    "rotated" -- an anisotropic Gaussian with sigma_x U[2, 4], sigma_y U[1, 2],
    angle U[0, 180) degrees and a centre offset U[-2, 2]^2 (nonsymmetric).
    Returns float32 device tensors g [count, n, n], h [count, taps, taps] and, if
    ``truth``, f [count, n, n] (the image on the field of view), with eta [count]."""
    torch = _torch()
    import torch.nn.functional as Fn
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 7919 + 17)
    m = taps // 2
    ne = n + 2 * m
    B = count
    dt = torch.float32
    lin = torch.linspace(0.0, 1.0, ne, device=device, dtype=dt)
    y, x = lin[:, None], lin[None, :]
    ramp = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(B, 3)).astype(np.float32)).to(device)
    f = ramp[:, 0, None, None] + ramp[:, 1, None, None] * x + ramp[:, 2, None, None] * y
    idx = torch.arange(ne, device=device)
    for _ in range(20):
        rr = np.sort(rng.integers(0, ne, size=(B, 2)), axis=1)
        cc = np.sort(rng.integers(0, ne, size=(B, 2)), axis=1)
        rr[:, 1] = np.maximum(rr[:, 1], rr[:, 0] + 1)
        cc[:, 1] = np.maximum(cc[:, 1], cc[:, 0] + 1)
        k = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(B, 6)).astype(np.float32)).to(device)
        r = torch.from_numpy(rr).to(device)
        c = torch.from_numpy(cc).to(device)
        mask = (((idx[None, :, None] >= r[:, 0, None, None]) & (idx[None, :, None] < r[:, 1, None, None]))
                & ((idx[None, None, :] >= c[:, 0, None, None]) & (idx[None, None, :] < c[:, 1, None, None])))
        poly = (k[:, 0, None, None] + k[:, 1, None, None] * x + k[:, 2, None, None] * y
                + k[:, 3, None, None] * x * x + k[:, 4, None, None] * x * y + k[:, 5, None, None] * y * y)
        f = f + mask.to(dt) * poly
    j = torch.arange(-m, m + 1, device=device, dtype=dt)
    jr, jc = j[:, None], j[None, :]
    if psf == "disk":
        rad = torch.from_numpy(rng.uniform(1.5, min(5.0, m), size=B).astype(np.float32)).to(device)
        h = ((jr * jr + jc * jc)[None] <= (rad * rad)[:, None, None]).to(dt)
    else:
        sx = torch.from_numpy(rng.uniform(2.0, 4.0, size=B).astype(np.float32)).to(device)[:, None, None]
        sy = torch.from_numpy(rng.uniform(1.0, 2.0, size=B).astype(np.float32)).to(device)[:, None, None]
        th = torch.from_numpy(np.deg2rad(rng.uniform(0.0, 180.0, size=B)).astype(np.float32)).to(device)[:, None, None]
        off = torch.from_numpy(rng.uniform(-2.0, 2.0, size=(B, 2)).astype(np.float32)).to(device)
        xx = jc[None] - off[:, 0, None, None]
        yy = jr[None] - off[:, 1, None, None]
        xr = torch.cos(th) * xx + torch.sin(th) * yy
        yr = -torch.sin(th) * xx + torch.cos(th) * yy
        h = torch.exp(-0.5 * ((xr / sx) ** 2 + (yr / sy) ** 2))
    h = h / h.sum(dim=(1, 2), keepdim=True)
    # g_i = sum_j h_j f_{i-j}: a cross-correlation with the flipped mask, one group per image
    g = Fn.conv2d(f[None], torch.flip(h, dims=(1, 2))[:, None], groups=B)[0]
    etas = np.exp(rng.uniform(np.log(eta[0]), np.log(eta[1]), size=B)).astype(np.float32)
    e = torch.randn(g.shape, generator=gen, device=device, dtype=dt)
    scale = torch.from_numpy(etas).to(device) * g.flatten(1).norm(dim=1) / e.flatten(1).norm(dim=1)
    g = (g + scale[:, None, None] * e).contiguous()
    ft = f[:, m:m + n, m:m + n].contiguous() if truth else None
    return g, h.contiguous(), ft, etas


def features_and_labels(plan: "hobc.Plan", g_dev, psf_dev, kind: str = "radial"):
    """Features [batch, 128] and labels log10(mu_GCV) [batch] (float32, device) of
    the problems of one plan-sized batch.  kind: "radial" (hobc_features) or
    "hist" (hobc_features_hist)."""
    torch = _torch()
    dt = torch.float64 if plan.prec == "fp64" else torch.float32
    shape = (plan.batch, plan.spec_elems) + ((2,) if plan.spec_complex else ())
    npsf = plan.batch if plan.psf_per_item else 1
    D = torch.empty((npsf,) + shape[1:], dtype=dt, device=g_dev.device)
    G = torch.empty(shape, dtype=dt, device=g_dev.device)
    X = torch.empty((plan.batch, 2 * hobc.FEATURE_BINS), dtype=torch.float32, device=g_dev.device)
    gcv = torch.empty((plan.batch, len(plan.mu_grid)), dtype=torch.float64, device=g_dev.device)
    mi = torch.empty(plan.batch, dtype=torch.int32, device=g_dev.device)
    plan.eigenvalues(psf_dev, D)
    plan.analysis(g_dev, G)
    if kind == "hist":
        plan.features_hist(G, D, X)
    else:
        plan.features(G, D, X)
    plan.gcv(G, D, gcv, mi)
    lg = torch.from_numpy(np.log10(plan.mu_grid).astype(np.float32)).to(g_dev.device)
    return X, lg[mi.long()], mi


def init_network(X, n_hidden: int = 256, seed: int = 0, stream=None, kind: str = "radial") -> "hobc.MLP":
    """A network with scaled-normal weights whose input standardisation is the
    per-feature mean and standard deviation of the training features X (computed
    on the GPU by hobc_mlp_fit_scaling); kind: the features it reads."""
    rng = np.random.default_rng(seed)
    n_in = X.shape[1]
    p = {
        "W1": rng.standard_normal((n_hidden, n_in)) * np.sqrt(2.0 / n_in),
        "b1": np.zeros(n_hidden),
        "W2": rng.standard_normal((n_hidden, n_hidden)) * np.sqrt(2.0 / n_hidden),
        "b2": np.zeros(n_hidden),
        "w3": rng.standard_normal(n_hidden) * np.sqrt(1.0 / n_hidden),
        "b3": np.zeros(1),
    }
    net = hobc.MLP(n_in, n_hidden, stream=stream)
    net.set_params(hobc.pack_params(p, np.zeros(n_in), np.ones(n_in)))
    net.fit_scaling(X)
    net.set_feature_kind(kind)
    return net


def fit(net: "hobc.MLP", X, t, epochs: int = 60, batch: int = 256, lr: float = 1e-3, weight_decay: float = 1e-4,
        seed: int = 0):
    """AdamW on the mean squared error of log10(mu); the learning rate drops
    tenfold for the last fifth of the epochs.  Returns the mean minibatch loss
    of every epoch."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    history = []
    for ep in range(epochs):
        rate = lr if ep < 0.8 * epochs else 0.1 * lr
        perm = torch.from_numpy(rng.permutation(n)).to(X.device)
        total = torch.zeros(1, dtype=torch.float32, device=X.device)
        steps = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            net.train_step(X.index_select(0, idx).contiguous(), t.index_select(0, idx).contiguous(), rate,
                           weight_decay, loss)
            total += loss
            steps += 1
        history.append(float(total.item()) / max(1, steps))
    return history


def predict(net: "hobc.MLP", X):
    torch = _torch()
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    net.forward(X, y)
    return y


def training_set(plan: "hobc.Plan", count: int, seed: int, psf: str, taps: int, kind: str = "hist",
                 chunk: int = 2048, eta=(1e-3, 3e-2)):
    """Features and GCV labels of ``count`` problems drawn on the GPU (gpu_problems)
    and run through the plan in plan-sized batches.  Returns (X, t) on the device."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = plan.n[0]
    B = plan.batch
    dt = torch.float64 if plan.prec == "fp64" else torch.float32
    Xs, ts = [], []
    for c0 in range(0, count, chunk):
        cnt = min(chunk, count - c0)
        cnt -= cnt % B
        if cnt <= 0:
            break
        g, h, _, _ = gpu_problems(cnt, n, seed * 1000003 + c0, dev, psf=psf, taps=taps, eta=eta)
        g, h = g.to(dt), h.to(dt)
        for s in range(0, cnt, B):
            psf_b = h[s:s + B] if plan.psf_per_item else h[s:s + 1]
            X, t, _ = features_and_labels(plan, g[s:s + B].contiguous(), psf_b.contiguous(), kind)
            Xs.append(X)
            ts.append(t)
        del g, h
    return torch.cat(Xs), torch.cat(ts)
