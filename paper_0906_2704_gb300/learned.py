"""Training and use of the mu-predicting network (include/hobc_learned.h).

Everything numeric runs in the library: the labels are the GCV choice of the
plain path (hobc_gcv), the inputs its radial features (hobc_features), and the
network is trained with hobc_mlp_train_step.  This module only moves batches
around (device tensors; torch is used for allocation and indexing).
"""
from __future__ import annotations

import numpy as np

from . import hobc


def _torch():
    import torch
    return torch


def features_and_labels(plan: "hobc.Plan", g_dev, psf_dev):
    """Features [batch, 128] and labels log10(mu_GCV) [batch] (float32, device) of
    the problems of one plan-sized batch."""
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
    plan.features(G, D, X)
    plan.gcv(G, D, gcv, mi)
    lg = torch.from_numpy(np.log10(plan.mu_grid).astype(np.float32)).to(g_dev.device)
    return X, lg[mi.long()], mi


def init_network(X, n_hidden: int = 256, seed: int = 0, stream=None) -> "hobc.MLP":
    """A network with scaled-normal weights whose input standardisation is the
    per-feature mean and standard deviation of the training features X."""
    torch = _torch()
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
    Xh = X.detach().to("cpu", torch.float64).numpy()
    mean = Xh.mean(axis=0)
    scale = Xh.std(axis=0) + 1e-3
    net = hobc.MLP(n_in, n_hidden, stream=stream)
    net.set_params(hobc.pack_params(p, mean, scale))
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
