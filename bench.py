#!/usr/bin/env python
"""Throughput of spectral Tikhonov deblurring with high-order boundary conditions
and GCV (Donatelli, arXiv:0906.2704) on 1024 x 1024 images.

Workload (the 1024^2 configuration): 2D images 1024 x 1024, nonsymmetric PSF
21 x 21 (anisotropic Gaussian sigma_x = 3, sigma_y = 1.5, rotated 30 degrees,
centre offset (+2 col, -1 row), sum 1), degree-2 boundary condition (Fourier
family T_F), L = I, GCV over 256 log-spaced mu in [1e-8, 1], 0.5% noise,
seeded synthetic images.  One step = one deblur call on a batch of images
(eigenvalues, analysis transform, GCV scan + argmin, filter + synthesis).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank deblurs its own batch (independent problems,
no collective in the data path); the timed region is bracketed by a barrier
and a device synchronisation, and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1024² deblurs/s: GCV scan vs learned-μ, equal rel. error; % HBM roofline"
N_SIDE = 1024
K_MU = 256
ETA = 0.005
WORKLOAD = ("2D 1024x1024, nonsymmetric 21x21 rotated anisotropic Gaussian PSF, degree-2 BC "
            "(Fourier family), L=I, GCV over 256 mu in [1e-8,1], 0.5% noise")


def psf():
    from paper_0906_2704_gb300 import synth
    return synth.gaussian_psf_2d_rotated(3.0, 1.5, 30.0, 21, 2.0, -1.0)


def make_inputs(batch: int, seed: int, distinct: int = 4):
    """``batch`` noisy observations built from ``distinct`` seeded clean images."""
    from paper_0906_2704_gb300 import synth
    h = psf()
    clean, truth = synth.problem_2d(seed, N_SIDE, N_SIDE, h, 0.0, count=min(batch, distinct))
    rng = np.random.default_rng(seed + 1)
    g = np.empty((batch, N_SIDE, N_SIDE))
    ft = np.empty_like(g)
    for i in range(batch):
        g[i] = synth.add_noise(rng, clean[i % len(clean)], ETA)
        ft[i] = truth[i % len(clean)]
    return h, g, ft


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_seconds_per_image(h, g, mus, count: int, keep: list | None = None):
    """The FP64 oracle (separable dense mode) on ``count`` images; seconds per image.
    keep: if a list, each image's (f, G, argmin, ghat) is appended to it."""
    from oracle import hobc_oracle as O
    t0 = time.perf_counter()
    for i in range(count):
        out = O.deblur_2d("F", h, g[i], "I", mus)
        if keep is not None:
            keep.append(out)
    return (time.perf_counter() - t0) / count


def rel2(a, b) -> float:
    """||a - b||_2 / ||b||_2 over the whole array."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_f_2d(family: str, h, ghat, L: str, mu: float):
    """The oracle's f at a given mu from its own spectrum (Eq. (eq:freg))."""
    from oracle import hobc_oracle as O
    n0, n1 = ghat.shape
    d = O.eigenvalues_2d(family, h, n0, n1)
    s = O.smoothing_2d(family, n0, n1, L)
    return O.synthesis_2d(family, O.filter_factors(d, s, mu) * ghat).real


def esz_of(prec: str) -> int:
    """Bytes of one real value of the plan's I/O and spectra (split-BF16 plans keep FP32 I/O)."""
    return 8 if prec == "fp64" else 4


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank: int) -> int:
    """Each rank deblurs its own independent images (weak scaling, no data exchange)."""
    return 100 + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time: the only collective of the benchmark (timing only)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_by_weight(weights, world: int, rank: int):
    """Contiguous share [lo, hi) of a batch of independent problems for one rank:
    the batch is cut where the running sum of the weights (pixels per problem)
    crosses each multiple of total/world, so every problem goes to exactly one
    rank and the ranks' pixel counts differ by at most one problem's."""
    w = np.asarray(weights, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return len(w)
        # first index whose cumulative weight reaches r/world of the total
        return int(np.searchsorted(cum, total * r / world, side="left"))
    return cut(rank), cut(rank + 1)


def whole_job_rate(world: int, batch: int, steps: int, seconds: float) -> float:
    """Images deblurred by all ranks per second of the slowest rank."""
    return world * batch * steps / seconds


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, one image per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_0906_2704_gb300 import synth
    h, g, _ = make_inputs(2, seed=11, distinct=2)
    mus = synth.mu_grid(K_MU)
    for i in range(args.warmup):
        oracle_seconds_per_image(h, g[i % 2:i % 2 + 1], mus, 1)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_seconds_per_image(h, g[i % 2:i % 2 + 1], mus, 1)
    el = time.perf_counter() - t0
    value = args.steps / el
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "deblurs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "deblurs/s", "cores": cores, "kind": "oracle",
                         "sample": "one 1024x1024 image per step (dense FP64 oracle, separable mode)"},
        "e2e": {"value": value, "unit": "deblurs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_0906_2704_gb300 import hobc, synth

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    B = args.batch
    prec = args.prec
    npdt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    h, g, ft = make_inputs(B, seed=rank_seed(rank))
    mus = synth.mu_grid(K_MU)
    stream = torch.cuda.current_stream()
    plan = hobc.Plan(2, (N_SIDE, N_SIDE), h.shape, 2, mus, L="I", prec=prec, family="fourier", batch=B,
                     stream=stream)
    # FP32 / split-BF16: the curve by bin expansion (every grid value, within the
    # stated truncation bound of the term-by-term scan, which is timed below as the
    # "direct_scan" arm); FP64 plans keep the term-by-term scan
    if prec != "fp64":
        plan.set_gcv_mode("expansion")
    g_d = torch.from_numpy(g.astype(npdt)).to(dev)
    h_d = torch.from_numpy(h.astype(npdt)).to(dev)
    f_d = torch.empty_like(g_d)
    mi_d = torch.empty(B, dtype=torch.int32, device=dev)

    def step():
        plan.deblur(g_d, h_d, f_d, mi_d, None)

    for _ in range(max(args.warmup, 3)):
        step()
    launches_per_step = plan.last_launch_count
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = whole_job_rate(world, B, args.steps, ms / 1e3)
    clocks = clk.summary()

    # per-step breakdown through the step entry points (same kernels)
    S = plan.spec_elems
    ghat = torch.empty((B, S, 2), dtype=tdt, device=dev)
    dbuf = torch.empty((1, S, 2), dtype=tdt, device=dev)
    G_d = torch.empty((B, K_MU), dtype=torch.float64, device=dev)
    steps_ms = {}
    calls = {
        "eigenvalues": lambda: plan.eigenvalues(h_d, dbuf),
        "analysis": lambda: plan.analysis(g_d, ghat),
        "gcv": lambda: plan.gcv(ghat, dbuf, G_d, mi_d),
        "filter_synthesis": lambda: plan.filter_synthesis(ghat, dbuf, mi_d, f_d),
    }
    for name, fn in calls.items():
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        steps_ms[name] = a.elapsed_time(b) / args.steps

    # the binned choice of mu (histogram localises, exact G decides) on the same batch
    f_b = torch.empty_like(g_d)
    mi_b = torch.empty(B, dtype=torch.int32, device=dev)
    fb_b = torch.empty(B, dtype=torch.int32, device=dev)
    ms_b, clk_b = _timed(lambda: plan.deblur_binned(g_d, h_d, f_b, mi_b, fb_b), stream, args.steps, args.warmup)
    binned_launches = plan.last_launch_count
    ms_b = max_over_ranks(ms_b, dist, dev)

    def rre(f):
        d = (f.cpu().numpy().astype(np.float64) - ft).reshape(B, -1)
        return np.linalg.norm(d, axis=1) / np.linalg.norm(ft.reshape(B, -1), axis=1)

    # the same method with the curve evaluated term by term (hobc_gcv's direct scan)
    direct = None
    f_dir = mi_dir = G_dir = None
    if plan.gcv_mode == "expansion":
        G_e = torch.empty((B, K_MU), dtype=torch.float64, device=dev)
        mi_e = torch.empty(B, dtype=torch.int32, device=dev)
        plan.gcv(ghat, dbuf, G_e, mi_e)
        plan.set_gcv_mode("direct")
        f_dir = torch.empty_like(g_d)
        mi_dir = torch.empty(B, dtype=torch.int32, device=dev)
        ms_dir, clk_dir = _timed(lambda: plan.deblur(g_d, h_d, f_dir, mi_dir), stream, args.steps, args.warmup)
        dir_launches = plan.last_launch_count
        ms_dir = max_over_ranks(ms_dir, dist, dev)
        G_dir = torch.empty_like(G_e)
        mi_d2 = torch.empty_like(mi_e)
        ms_dg, _ = _timed(lambda: plan.gcv(ghat, dbuf, G_dir, mi_d2), stream, args.steps, args.warmup)
        plan.set_gcv_mode("expansion")
        torch.cuda.synchronize()
        direct = {"value": whole_job_rate(world, B, args.steps, ms_dir / 1e3), "unit": "deblurs/s",
                  "ms_per_step": ms_dir / args.steps, "gpu_launches": dir_launches * args.steps,
                  "gcv_ms": ms_dg / args.steps, "clocks": clk_dir,
                  "expansion_vs_direct": {
                      "truncation_bound": plan.gcv_expansion_bound,
                      "G_rel_diff_max": float(((G_e - G_dir).abs() / G_dir.abs()).max()),
                      "index_agreement": float((mi_e == mi_d2).float().mean())}}

    # the grid argmin refined over continuous mu (5 rounds of 9 points in its bracket)
    f_r = torch.empty_like(g_d)
    mi_r = torch.empty(B, dtype=torch.int32, device=dev)
    mu_r = torch.empty(B, dtype=torch.float64, device=dev)
    ms_r, clk_r = _timed(lambda: plan.deblur_refined(g_d, h_d, f_r, mi_r, mu_r), stream, args.steps, args.warmup)
    refined_launches = plan.last_launch_count
    ms_r = max_over_ranks(ms_r, dist, dev)
    G_grid = torch.empty((B, K_MU), dtype=torch.float64, device=dev)
    G_ref = torch.empty(B, dtype=torch.float64, device=dev)
    plan.gcv(ghat, dbuf, G_grid, mi_d)
    plan.gcv_refine(ghat, dbuf, mi_d, mu_r, G_ref)
    g_min = G_grid.min(dim=1).values

    # the exact GCV functional of Eq. (eq:gcv) (T_X kept in the numerator)
    f_x = torch.empty_like(g_d)
    mi_x = torch.empty(B, dtype=torch.int32, device=dev)
    ms_x, clk_x = _timed(lambda: plan.deblur_exact(g_d, h_d, f_x, mi_x), stream, args.steps, args.warmup)
    exact_launches = plan.last_launch_count
    ms_x = max_over_ranks(ms_x, dist, dev)
    G_x = torch.empty((B, K_MU), dtype=torch.float64, device=dev)
    plan.deblur_exact(g_d, h_d, f_x, mi_x, G_x)
    # the same functional, its grid minimiser found by the coarse-to-fine search
    f_xs = torch.empty_like(g_d)
    mi_xs = torch.empty(B, dtype=torch.int32, device=dev)
    ms_xs, clk_xs = _timed(lambda: plan.deblur_exact_search(g_d, h_d, f_xs, mi_xs), stream, args.steps,
                           args.warmup)
    search_launches = plan.last_launch_count
    ms_xs = max_over_ranks(ms_xs, dist, dev)

    plan.deblur(g_d, h_d, f_d, mi_d, None)
    r_full, r_bin = rre(f_d), rre(f_b)
    r_ref = rre(f_r)
    r_x = rre(f_x)
    exact = {"value": whole_job_rate(world, B, args.steps, ms_x / 1e3), "unit": "deblurs/s",
             "ms_per_step": ms_x / args.steps, "gpu_launches": exact_launches * args.steps,
             "index_agreement_with_approximation": float((mi_x == mi_d).float().mean()),
             "mu_median": {"approximate": float(np.median(mus[mi_d.cpu().numpy()])),
                           "exact": float(np.median(mus[mi_x.cpu().numpy()]))},
             "rre_mean": {"approximate": float(r_full.mean()), "exact": float(r_x.mean())},
             "clocks": clk_x}
    # the learned choice of mu (histogram features), its network trained here, outside
    # the timed region, on GCV labels of problems drawn on the GPU like this workload
    # (rotated anisotropic Gaussian PSFs of random shape, noise log-uniform in [1e-3, 3e-2])
    from paper_0906_2704_gb300 import learned as LR
    t_tr = time.time()
    plan_tr = hobc.Plan(2, (N_SIDE, N_SIDE), h.shape, 2, mus, L="I", prec="fp32" if prec != "fp64" else "fp64",
                        family="fourier", batch=16, psf_per_item=True, stream=stream)
    Xtr, ttr = LR.training_set(plan_tr, args.learned_train, 5, "rotated", h.shape[0], kind="hist", chunk=128)
    net = LR.init_network(Xtr, 256, seed=0, stream=stream.cuda_stream, kind="hist")
    hist_l = LR.fit(net, Xtr, ttr, epochs=40, batch=256, lr=1e-3)
    plan_tr.close()
    torch.cuda.synchronize()
    t_tr = time.time() - t_tr
    f_l = torch.empty_like(g_d)
    mu_l = torch.empty(B, dtype=torch.float64, device=dev)
    fb_l = torch.empty(B, dtype=torch.int32, device=dev)
    ms_l, clk_l = _timed(lambda: plan.deblur_learned(net, g_d, h_d, f_l, mu_l, fb_l), stream, args.steps,
                         args.warmup)
    learned_launches = plan.last_launch_count
    ms_l = max_over_ranks(ms_l, dist, dev)
    r_l = rre(f_l)
    grid_mu = torch.from_numpy(mus).to(dev)[mi_d.long()]
    learned_arm = {"value": whole_job_rate(world, B, args.steps, ms_l / 1e3), "unit": "deblurs/s",
                   "ms_per_step": ms_l / args.steps, "gpu_launches": learned_launches * args.steps,
                   "fallback_rate": float(fb_l.float().mean()),
                   "mu_ratio_to_full_scan": {"median": float((mu_l / grid_mu).median()),
                                             "max_abs_log10": float((mu_l / grid_mu).log10().abs().max())},
                   "rre_mean": {"full_scan": float(r_full.mean()), "learned": float(r_l.mean())},
                   "rre_ratio_to_full_scan": float(r_l.mean() / r_full.mean()),
                   "speedup_vs_full_scan": ms / ms_l,
                   "train": {"problems": int(Xtr.shape[0]), "seconds": t_tr, "epochs": 40,
                             "loss_first": hist_l[0], "loss_last": hist_l[-1], "features": "hist"},
                   "clocks": clk_l}
    del Xtr, ttr

    r_xs = rre(f_xs)
    exact_search = {"value": whole_job_rate(world, B, args.steps, ms_xs / 1e3), "unit": "deblurs/s",
                    "ms_per_step": ms_xs / args.steps, "gpu_launches": search_launches * args.steps,
                    "evaluations_per_image": int(np.isfinite(G_xs_probe(plan, g_d, h_d, B)).sum() // B),
                    "index_agreement_with_full_exact_scan": float((mi_xs == mi_x).float().mean()),
                    "rre_mean": {"full_exact_scan": float(r_x.mean()), "search": float(r_xs.mean())},
                    "rre_ratio_to_full_exact_scan": float(r_xs.mean() / r_x.mean()),
                    "clocks": clk_xs}
    refined = {"value": whole_job_rate(world, B, args.steps, ms_r / 1e3), "unit": "deblurs/s",
               "ms_per_step": ms_r / args.steps, "gpu_launches": refined_launches * args.steps,
               "G_ratio_to_grid_min": {"mean": float((G_ref / g_min).mean()), "max": float((G_ref / g_min).max())},
               "mu_ratio_to_grid": {"min": float((mu_r / torch.from_numpy(mus).to(dev)[mi_d.long()]).min()),
                                    "max": float((mu_r / torch.from_numpy(mus).to(dev)[mi_d.long()]).max())},
               "rre_mean": {"full_scan": float(r_full.mean()), "refined": float(r_ref.mean())},
               "clocks": clk_r}
    binned = {"value": whole_job_rate(world, B, args.steps, ms_b / 1e3), "unit": "deblurs/s",
              "ms_per_step": ms_b / args.steps, "gpu_launches": binned_launches * args.steps,
              "fallback_rate": float(fb_b.float().mean()),
              "index_agreement_with_full_scan": float((mi_b == mi_d).float().mean()),
              "rre_mean": {"full_scan": float(r_full.mean()), "binned": float(r_bin.mean())},
              "clocks": clk_b}
    if direct is not None:
        direct["rre_mean"] = {"direct": float(rre(f_dir).mean()), "expansion": float(r_full.mean())}

    # end to end through the host-buffer entry point (pinned host memory)
    g_h = torch.from_numpy(g.astype(npdt)).pin_memory().numpy()
    h_h = np.ascontiguousarray(h.astype(npdt))
    f_h = torch.empty(g.shape, dtype=tdt).pin_memory().numpy()
    mi_h = torch.empty(B, dtype=torch.int32).pin_memory().numpy()
    plan.deblur_host(g_h, h_h, f_h, mi_h)
    # the pipeline's chunk count, picked by a short untimed trial of 2, 4 and 8
    trial = {}
    for nc in (2, 4, 8):
        plan.set_host_chunks(nc)
        plan.deblur_host(g_h, h_h, f_h, mi_h)
        t0 = time.perf_counter()
        for _ in range(3):
            plan.deblur_host_async(g_h, h_h, f_h, mi_h)
        plan.wait()
        trial[nc] = time.perf_counter() - t0
    chunks = min(trial, key=trial.get)
    plan.set_host_chunks(chunks)
    plan.deblur_host(g_h, h_h, f_h, mi_h)
    barrier()
    # consecutive calls overlap (each step's uploads run during the previous
    # step's kernels); every step's copies are inside the timed region
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.deblur_host_async(g_h, h_h, f_h, mi_h)
    plan.wait()
    barrier()
    el = max_over_ranks(time.perf_counter() - t0, dist, dev)
    esz = np.dtype(npdt).itemsize
    e2e = {"value": whole_job_rate(world, B, args.steps, el), "unit": "deblurs/s",
           "h2d_bytes_per_step": B * N_SIDE * N_SIDE * esz + h.size * esz,
           "d2h_bytes_per_step": B * N_SIDE * N_SIDE * esz + B * 4, "host_chunks": chunks}

    # roofline of the term-by-term GCV scan (k_gcv_partials + k_gcv_finalize): evaluations
    # of sigma = 1/(a + mu) per launch over the time of the gcv call in direct mode
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    evals = B * S * K_MU
    gcv_s = (direct["gcv_ms"] if direct is not None else steps_ms["gcv"]) / 1e3
    achieved = evals / gcv_s / 1e9
    # the method's arithmetic per evaluation is one division and four FMA-class
    # operations (sigma = s^2/(|d|^2 + mu s^2), the two products and the two sums);
    # at five FP32-pipe operations per evaluation the 128 FP32 lanes of each of
    # the 152 SMs bound the scan at 128/5 evaluations per SM-clock.  This peak is
    # derived from unit counts and the clock, not measured (the measured peaks
    # cover HBM and bf16 tensor throughput only).
    peak = 152 * (128 / 5.0) * sm_max * 1e6 / 1e9
    # DRAM traffic of one k_gcv_partials launch: ncu on the 8-image case read 37.92 MB and
    # wrote 0.002 MB (eight spectra of 4.2107 MB plus the shared eigenvalues, no re-reads),
    # so a launch over B images moves B spectra plus one eigenvalue array
    spec_bytes = S * 2 * esz_of(prec)
    traffic = B * spec_bytes + spec_bytes if prec == "fp32" else None
    scan_roofline = {"bound": "alu", "kernel": "k_gcv_partials", "achieved": achieved, "peak": peak,
                     "unit": "Geval/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read+write of an 8-image launch (37.92 MB), scaled per image",
                     "peak_source": f"derived, not measured: 152 SMs x 128 FP32 lanes / 5 operations per "
                                    f"evaluation (1 division + 4 FMA) x {sm_max:.0f} MHz ({peak_kind} max clock)"}
    if prec == "fp64":
        # FP64 scan: 2 FP64 operations per SM-clock on this part (1.25 TFLOP/s), five per evaluation
        peak = 152 * (2 / 5.0) * sm_max * 1e6 / 1e9
        scan_roofline.update({"peak": peak, "frac": achieved / peak, "traffic": None,
                              "peak_source": f"derived, not measured: 152 SMs x 2 FP64 operations per clock / "
                                             f"5 per evaluation x {sm_max:.0f} MHz ({peak_kind} max clock)"})
    # the headline step's dominant call: with the direct scan the scan; with the
    # expansion a transform pass (its row and column kernels), bound by HBM by the
    # method's bytes (the spectrum in or out, the image out or in, per image)
    dom = max(("analysis", "filter_synthesis", "gcv"), key=lambda k: steps_ms[k])
    if dom == "gcv":
        roofline = dict(scan_roofline)
    else:
        esz = np.dtype(npdt).itemsize
        call_bytes = B * (S * 2 * esz_of(prec) + N_SIDE * N_SIDE * esz) + (S * 2 * esz_of(prec) if
                                                                          dom == "filter_synthesis" else 0)
        t_call = steps_ms[dom] / 1e3
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        flops = B * 2.5 * N_SIDE * N_SIDE * np.log2(float(N_SIDE * N_SIDE))   # one 2D transform per image
        fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        # DRAM traffic of the two kernels of each call, ncu on the 8-image case (FP32):
        # filter + synthesis 38.01 + 0.78 + 33.79 + 0.44 MB, analysis 33.67 + 1.28 + 33.80 + 0.18 MB
        per_img = {"filter_synthesis": 73.02e6 / 8, "analysis": 68.93e6 / 8}[dom]
        roofline = {"bound": "hbm", "kernel": ("k_cplx_synthesis + k_pair_synthesis (filter + synthesis call)"
                                               if dom == "filter_synthesis" else
                                               "k_pair_analysis + k_cplx_analysis (analysis call)"),
                    "achieved": call_bytes / t_call / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": call_bytes / t_call / 1e9 / hbm_peak,
                    "traffic": B * per_img if prec == "fp32" else None,
                    "traffic_source": "ncu dram__bytes_read+write of the two kernels on the 8-image case, "
                                      "scaled per image",
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                    "bytes_per_launch": call_bytes,
                    "alu_view": {"flops_per_launch": flops, "achieved_tflops": flops / t_call / 1e12,
                                 "fp32_peak_tflops": fp32_peak, "frac": flops / t_call / 1e12 / fp32_peak,
                                 "flops_source": "2.5 N^2 log2(N^2) per 2D transform per image; FP32 peak "
                                                 "derived, not measured: 152 SMs x 128 lanes x 2 x max clock"}}
    transform_roofline = None
    if prec == "split_bf16":
        # the four transform products of a step on the tensor cores (real form of the
        # complex Fourier products): 3 split products x 2 M N K each, padded tile shapes
        tm, tn, tk = hobc.tc_tiles()
        pad = lambda x, t: -(-x // t) * t
        n, W = N_SIDE, S // N_SIDE
        shapes = [(n, 2 * W, pad(n, tk)), (W, 2 * n, 2 * pad(n, tk)),
                  (2 * n, W, pad(2 * n, tk)), (n, n, 2 * pad(W, tk))]
        flops = sum(3 * 2.0 * pad(m_, tm) * pad(n_, tn) * k_ for m_, n_, k_ in shapes) * B
        t_tr = (steps_ms["analysis"] + steps_ms["filter_synthesis"]) / 1e3
        pk = peaks.get("bf16_tflops", 1900.0)
        transform_roofline = {"bound": "tensor", "kernel": "k_gemm_split (4 products per step)",
                              "achieved": flops / t_tr / 1e12, "peak": pk, "unit": "TFLOP/s",
                              "frac": flops / t_tr / 1e12 / pk, "peak_kind": peak_kind,
                              "flops_per_step": flops,
                              "note": "analysis and filter + synthesis calls, their split and filter kernels included"}
    hbm_bytes = B * N_SIDE * N_SIDE * esz * 2 + h.size * esz
    hbm_frac = hbm_bytes / (ms / args.steps / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)
    hbm = {"algorithmic_bytes_per_step": hbm_bytes,
           "achieved_gbs": hbm_bytes / (ms / args.steps / 1e3) / 1e9,
           "peak_gbs": peaks.get("hbm_gbs", 6800.0), "peak_kind": peak_kind, "frac": hbm_frac,
           "target_frac": 0.60, "target_met": bool(hbm_frac >= 0.60),
           "note": "g in and f out per deblur; the scan (FP32 pipe) and the transforms (latency) bind, not HBM"}

    cpu = None
    oracle_error = None
    if rank == 0 and not args.no_cpu_baseline:
        n_img = 3
        kept = []
        sec = oracle_seconds_per_image(h, g, mus, n_img, keep=kept)
        cpu = {"value": 1.0 / sec, "unit": "deblurs/s", "cores": blas_threads(), "kind": "oracle",
               "sample": f"{n_img} images of the same workload, dense FP64 oracle (separable mode)"}
        sec1 = single_core_oracle_seconds(1)
        cpu["single_core"] = {"value": (1.0 / sec1) if sec1 else None, "unit": "deblurs/s", "cores": 1,
                              "sample": "1 image of the same workload, one BLAS thread"}
        oracle_error = default_oracle_error(kept, h, mus, f_d, mi_d, G_grid, f_b, mi_b, f_r, mu_r, G_ref,
                                            f_x, mi_x, G_x, f_xs, mi_xs, f_dir, mi_dir)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "deblurs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "split_bf16": "bf16x3 (split) / f32"}[prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_gpu": B, "n": N_SIDE, "n_mu": K_MU,
                       "l2": "inputs+outputs %.0f MB per step > 129 MB L2 (no flush)" % (2 * B * N_SIDE ** 2 * esz / 1e6)},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "roofline": roofline,
            "gcv_mode": plan.gcv_mode, "direct_scan": direct, "scan_roofline": scan_roofline,
            "hbm_roofline": hbm, "steps_ms": steps_ms, "cpu_baseline": cpu, "clocks": clocks,
            "learned_mu": learned_arm,
            "binned_mu": binned, "refined_mu": refined, "exact_gcv": exact, "exact_gcv_search": exact_search,
            "oracle_error": oracle_error, "precision": prec, "transform_roofline": transform_roofline,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    plan.close()
    return 0


def G_xs_probe(plan, g_d, h_d, B):
    """G_ex at the grid values the coarse-to-fine search evaluated (NaN elsewhere)."""
    import torch
    G = torch.empty((B, K_MU), dtype=torch.float64, device=g_d.device)
    f = torch.empty_like(g_d)
    plan.deblur_exact_search(g_d, h_d, f, None, G)
    return G.cpu().numpy()


def default_oracle_error(kept, h, mus, f_d, mi_d, G_grid, f_b, mi_b, f_r, mu_r, G_ref, f_x, mi_x, G_x, f_xs,
                         mi_xs, f_dir=None, mi_dir=None):
    """Error of every arm of the 1024^2 line against the FP64 oracle on the images
    the CPU baseline ran: f in relative 2-norm at the mu the arm chose (the oracle
    filters its own spectrum at that mu), and G where the arm reports one."""
    from oracle import exact_gcv_oracle as X
    from oracle import hobc_oracle as O
    n = len(kept)
    fs = {k: v.cpu().numpy()[:n] for k, v in (("full", f_d), ("binned", f_b), ("refined", f_r), ("exact", f_x),
                                              ("search", f_xs))}
    ks = {k: v.cpu().numpy()[:n] for k, v in (("full", mi_d), ("binned", mi_b), ("exact", mi_x), ("search", mi_xs))}
    Gg, Gr, Gx, mr = G_grid.cpu().numpy(), G_ref.cpu().numpy(), G_x.cpu().numpy(), mu_r.cpu().numpy()
    d = O.eigenvalues_2d("F", h, N_SIDE, N_SIDE)
    s = O.smoothing_2d("F", N_SIDE, N_SIDE, "I")
    out = {"images": n, "reference": "dense FP64 oracle (separable mode) on the same g",
           "measure": "f: ||f_gpu - f_oracle(mu)||_2 / ||f_oracle(mu)||_2 at the arm's mu; G: max relative"}
    arms = {"full_scan": [], "binned_mu": [], "refined_mu": [], "exact_gcv": [], "exact_gcv_search": []}
    g_err, g_ref_err, g_ex_err, agree, agree_e = [], [], [], [], []
    for i, (f_o, G_o, k_o, ghat) in enumerate(kept):
        cache = {int(k_o): f_o}

        def f_at_index(k):
            if k not in cache:
                cache[k] = oracle_f_2d("F", h, ghat, "I", float(mus[k]))
            return cache[k]
        arms["full_scan"].append(rel2(fs["full"][i], f_at_index(int(ks["full"][i]))))
        arms["binned_mu"].append(rel2(fs["binned"][i], f_at_index(int(ks["binned"][i]))))
        arms["refined_mu"].append(rel2(fs["refined"][i], oracle_f_2d("F", h, ghat, "I", float(mr[i]))))
        arms["exact_gcv"].append(rel2(fs["exact"][i], f_at_index(int(ks["exact"][i]))))
        arms["exact_gcv_search"].append(rel2(fs["search"][i], f_at_index(int(ks["search"][i]))))
        if f_dir is not None:
            ke = int(mi_dir.cpu().numpy()[i])
            arms.setdefault("direct_scan", []).append(rel2(f_dir.cpu().numpy()[i], f_at_index(ke)))
            agree_e.append(ke == int(k_o))
        g_err.append(float(np.max(np.abs(Gg[i] - G_o) / G_o)))
        agree.append(int(ks["full"][i]) == int(k_o))
        G_at = O.gcv_curve(ghat, d, s, np.array([mr[i]]))[0]
        g_ref_err.append(abs(Gr[i] - G_at) / G_at)
        kx = int(ks["exact"][i])
        Gx_o = X.gcv_exact_curve("F", ghat, d, s, np.array([mus[kx]]))[0]
        g_ex_err.append(abs(Gx[i][kx] - Gx_o) / Gx_o)
    out["full_scan"] = {"f_rel_2norm_max": max(arms["full_scan"]), "G_rel_max": max(g_err),
                        "mu_index_agreement": float(np.mean(agree))}
    out["binned_mu"] = {"f_rel_2norm_max": max(arms["binned_mu"])}
    out["refined_mu"] = {"f_rel_2norm_max": max(arms["refined_mu"]), "G_rel_at_mu_max": float(max(g_ref_err))}
    out["exact_gcv"] = {"f_rel_2norm_max": max(arms["exact_gcv"]), "G_rel_at_mu_max": float(max(g_ex_err))}
    out["exact_gcv_search"] = {"f_rel_2norm_max": max(arms["exact_gcv_search"])}
    if f_dir is not None:
        out["direct_scan"] = {"f_rel_2norm_max": max(arms["direct_scan"]),
                              "mu_index_agreement": float(np.mean(agree_e))}
    return out


def _timed(step, stream, steps, warmup):
    """Device time of ``steps`` calls of step() after ``warmup`` untimed ones (ms)."""
    import torch
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
    return a.elapsed_time(b), clk.summary()


def oracle_error_items(samples, K):
    """Errors of sampled problems of a workload against the FP64 oracle.  samples:
    (family letter, h, g, L, mus, f_gpu, k_gpu, G_gpu or None) per problem (1D, 2D or
    3D); the oracle deblurs g, then filters its own spectrum at the GPU's grid index."""
    from oracle import hobc_oracle as O
    from oracle import volume_oracle as V
    f_err, g_err, agree = [], [], []
    for fam, h, g, L, mus, f_gpu, k_gpu, G_gpu in samples:
        if g.ndim == 1:
            f_o, G_o, k_o, ghat = O.deblur_1d(fam, h, g, L, mus)
        elif g.ndim == 2:
            f_o, G_o, k_o, ghat = O.deblur_2d(fam, h, g, L, mus)
        else:
            f_o, G_o, k_o, ghat = V.deblur_3d(fam, h, g, L, mus)
        if int(k_gpu) != int(k_o):
            if g.ndim == 1:
                d, s_ = O.eigenvalues_1d(fam, h, g.shape[0]), O.smoothing_1d(fam, g.shape[0], L)
                f_o = O.synthesis_1d(fam, O.filter_factors(d, s_, mus[k_gpu]) * ghat).real
            elif g.ndim == 2:
                f_o = oracle_f_2d(fam, h, ghat, L, float(mus[k_gpu]))
            else:
                d, s_ = V.eigenvalues_3d(fam, h, *g.shape), V.smoothing_3d(fam, *g.shape, L)
                f_o = V.synthesis_3d(fam, O.filter_factors(d, s_, mus[k_gpu]) * ghat).real
        f_err.append(rel2(f_gpu, f_o))
        agree.append(int(k_gpu) == int(k_o))
        if G_gpu is not None:
            g_err.append(float(np.max(np.abs(np.asarray(G_gpu) - G_o) / G_o)))
    out = {"problems": len(samples), "reference": "dense FP64 oracle on the same g",
           "f_rel_2norm_max": max(f_err), "mu_index_agreement": float(np.mean(agree))}
    if g_err:
        out["G_rel_max"] = max(g_err)
    return out


def single_core_oracle_seconds(n_img: int = 1) -> float | None:
    """The 1024^2 oracle deblur on one host core: a child process with every BLAS
    pool held to one thread (the pools read these variables when numpy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    code = ("import sys, time; sys.path.insert(0, %r); import bench; from paper_0906_2704_gb300 import synth; "
            "h, g, _ = bench.make_inputs(%d, seed=11, distinct=%d); mus = synth.mu_grid(bench.K_MU); "
            "print(bench.oracle_seconds_per_image(h, g, mus, %d))") % (ROOT, n_img, n_img, n_img)
    try:
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        return float(res.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def run_other(args):
    """The other configurations, on one GPU, one JSON line each (not the headline):
    batched  -- 4096 square problems, side log-uniform in [64, 512], own Gaussian
                PSF (sigma U[1,4]) and degree in {1,2,3}, Laplacian, 128 mu, 1% noise
    signals1d -- 65,536 signals n = 256, Gaussian sigma 2 (9 taps), antireflective,
                L = I, 64 mu in [1e-8, 1], 1% noise
    volume128 -- 8 volumes 128^3, separable Gaussian 9^3 sigma 1.5, degree 2 (cosine),
                Laplacian, 128 mu, 1% noise (the tensor-product transform of Sec. 6)
    cosine512 -- 512 x 512, separable Gaussian 15 x 15 sigma 2.5, degree 2 (cosine),
                Laplacian, 256 mu, 0.5% noise, batch 32"""
    import torch
    from paper_0906_2704_gb300 import hobc, synth
    world, rank, local = dist_env()
    dist = None
    if world > 1 and args.workload == "batched":
        # independent problems sharded over the ranks, no data exchange (weak scaling)
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif world > 1:
        if rank != 0:
            return 0
        torch.cuda.set_device(local)
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = args.prec
    npdt = np.float64 if prec == "fp64" else np.float32
    stream = torch.cuda.Stream()
    extra = {}
    with torch.cuda.stream(stream):
        if args.workload == "batched":
            # count problems per rank: the whole job is count x world problems, cut
            # into contiguous pixel-balanced shards (one per rank)
            total = args.count * max(world, 1)
            items, gs, hs = synth.batch_uneven(7, total)
            lo, hi = shard_by_weight([it[0] * it[1] for it in items], world, rank)
            items, gs, hs = items[lo:hi], gs[lo:hi], hs[lo:hi]
            count = len(items)
            K = 128
            # the FFT schedule (radix per degree and FFT length), measured on this GPU by
            # the autotuner (outside the timed region; cached as JSON for later runs);
            # --no-autotune keeps the default schedule (radix 16 from FFT length 256 up)
            schedule, tuned, t_tune = None, None, 0.0
            if not args.no_autotune:
                from paper_0906_2704_gb300 import autotune
                t_tune = time.time()
                cache = os.path.join(tempfile.gettempdir(), "hobc_bench_fft_schedule.json")
                schedule, tuned = autotune.tune_batched(items, synth.mu_grid(K), L="lap", prec=prec, cache=cache,
                                                        refresh=True)
                t_tune = time.time() - t_tune
            # FP32: the curve by bin expansion (the line's value); the term-by-term scan beside it
            gmode = "expansion" if prec == "fp32" else "direct"
            batch = hobc.Batch(items, synth.mu_grid(K), L="lap", prec=prec, stream=stream, schedule=schedule,
                               gcv_mode=gmode)
            g = torch.from_numpy(np.concatenate([x.ravel() for x in gs]).astype(npdt)).to(dev)
            h = torch.from_numpy(np.concatenate([x.ravel() for x in hs]).astype(npdt)).to(dev)
            f = torch.empty_like(g)
            mi = torch.empty(count, dtype=torch.int32, device=dev)
            if dist is not None:
                dist.barrier()
            ms, clocks = _timed(lambda: batch.deblur(g, h, f, mi), stream, args.steps, args.warmup)
            ms = max_over_ranks(ms, dist, dev)
            units, unit = total, "images/s"
            launches = batch.last_launch_count
            pixels = int(g.numel())
            extra = {"pixels_per_step": pixels, "pixels_per_s": pixels * args.steps / (ms / 1e3),
                     "degrees": np.bincount([it[4] for it in items], minlength=4)[1:].tolist(),
                     "graph": True, "persistent": True, "gcv_mode": gmode}
            if gmode == "expansion":
                mi_line = mi.clone()
                direct = hobc.Batch(items, synth.mu_grid(K), L="lap", prec=prec, stream=stream, schedule=schedule)
                ms_dir, _ = _timed(lambda: direct.deblur(g, h, f, mi), stream, args.steps, args.warmup)
                ms_dir = max_over_ranks(ms_dir, dist, dev)
                direct.close()
                extra["direct_scan"] = {"value": total / (ms_dir / args.steps / 1e3), "unit": "images/s",
                                        "index_agreement_with_line": float((mi_line == mi).float().mean())}
            if tuned is not None:
                # the same batch with the default schedule (radix 16 from FFT length 256 up)
                default = hobc.Batch(items, synth.mu_grid(K), L="lap", prec=prec, stream=stream, gcv_mode=gmode)
                ms_def, _ = _timed(lambda: default.deblur(g, h, f, mi), stream, args.steps, args.warmup)
                default.close()
                extra["autotune"] = {"seconds": t_tune, "schedule": tuned}
                extra["default_schedule"] = {"value": total / (ms_def / args.steps / 1e3), "unit": "images/s"}
            cfg = {"workload": f"{args.count} uneven 2D problems per GPU (side log-uniform in [64,512], own "
                               f"Gaussian PSF, degree 1/2/3, Laplacian, 128 mu, 1% noise), one CUDA-graph launch",
                   "count": total, "parallelism": f"dp{max(world, 1)} (pixel-balanced contiguous shards)"}
            io_bytes = 2 * pixels * np.dtype(npdt).itemsize
        elif args.workload == "signals1d":
            B, n, K = 65536, 256, 64
            hh = synth.gaussian_psf_1d(2.0, 9)
            gg, _ = synth.problem_1d(3, n, hh, 0.01, count=B)
            plan = hobc.Plan(1, n, 9, 1, synth.mu_grid(K), L="I", prec=prec, family="sine", batch=B, stream=stream)
            g = torch.from_numpy(gg.astype(npdt)).to(dev)
            h = torch.from_numpy(hh.astype(npdt)).to(dev)
            f = torch.empty_like(g)
            mi = torch.empty(B, dtype=torch.int32, device=dev)
            ms, clocks = _timed(lambda: plan.deblur(g, h, f, mi), stream, args.steps, args.warmup)
            units, unit, launches = B, "signals/s", plan.last_launch_count
            cfg = {"workload": "65536 1D signals n=256, Gaussian sigma 2 (9 taps), antireflective, L=I, 64 mu, 1% noise",
                   "batch": B}
            io_bytes = 2 * B * n * np.dtype(npdt).itemsize
        elif args.workload == "volume128":
            n, B, K = 128, 8, 128
            hh = synth.gaussian_psf_3d((1.5, 1.5, 1.5), (9, 9, 9))
            gg, _ = synth.problem_3d(9, n, n, n, hh, 0.01, count=B)
            vol = hobc.Volume((n, n, n), hh.shape, 2, synth.mu_grid(K), L="lap", prec=prec, family="cosine",
                              psf_symmetric=True, batch=B, stream=stream)
            g = torch.from_numpy(gg.astype(npdt)).to(dev)
            h = torch.from_numpy(hh.astype(npdt)).to(dev)
            f = torch.empty_like(g)
            mi = torch.empty(B, dtype=torch.int32, device=dev)
            ms, clocks = _timed(lambda: vol.deblur(g, h, f, mi), stream, args.steps, args.warmup)
            units, unit, launches = B, "volumes/s", vol.last_launch_count
            cfg = {"workload": f"{B} volumes {n}^3, separable Gaussian 9^3 sigma 1.5, degree 2 (cosine), Laplacian, "
                               f"{K} mu, 1% noise", "batch": B}
            io_bytes = 2 * B * n ** 3 * np.dtype(npdt).itemsize
            S = vol.spec_elems
            gh = torch.empty((B, S), dtype=g.dtype, device=dev)
            ms_a, _ = _timed(lambda: vol.analysis(g, gh), stream, args.steps, 2)
            ms_s, _ = _timed(lambda: vol.synthesis(gh, f), stream, args.steps, 2)
            extra = {"transform_ms_per_step": {"analysis": ms_a / args.steps, "synthesis": ms_s / args.steps}}
        else:
            n = 1024 if args.workload == "cosine1024" else 512
            B, K = (16 if n == 1024 else 32), 256
            hh = synth.gaussian_psf_2d_separable(2.5, 15)
            clean, truth = synth.problem_2d(4, n, n, hh, 0.0, count=4)
            rng = np.random.default_rng(5)
            gg = np.stack([synth.add_noise(rng, clean[i % 4], 0.005) for i in range(B)])
            ftrue = np.stack([truth[i % 4] for i in range(B)])
            plan = hobc.Plan(2, (n, n), (15, 15), 2, synth.mu_grid(K), L="lap", prec=prec, family="cosine",
                             batch=B, stream=stream)
            g = torch.from_numpy(gg.astype(npdt)).to(dev)
            h = torch.from_numpy(hh.astype(npdt)).to(dev)
            f = torch.empty_like(g)
            mi = torch.empty(B, dtype=torch.int32, device=dev)
            # term-by-term scan first, then (FP32 / split-BF16) the curve by bin expansion,
            # which is the line's value where it applies
            ms_dir, _ = _timed(lambda: plan.deblur(g, h, f, mi), stream, args.steps, args.warmup)
            plan.status()
            mi_dir = mi.clone()
            if prec != "fp64":
                plan.set_gcv_mode("expansion")
            ms, clocks = _timed(lambda: plan.deblur(g, h, f, mi), stream, args.steps, args.warmup)
            plan.status()
            units, unit, launches = B, "deblurs/s", plan.last_launch_count
            cfg = {"workload": f"{n}x{n}, separable Gaussian 15x15 sigma 2.5, degree 2 (cosine), Laplacian, 256 mu, "
                               "0.5% noise", "batch": B}
            io_bytes = 2 * B * n * n * np.dtype(npdt).itemsize
            # the transform passes alone (analysis + synthesis), and for the dense mode their tensor-core rate
            S = plan.spec_elems
            gh = torch.empty((B, S), dtype=g.dtype, device=dev)
            ms_a, _ = _timed(lambda: plan.analysis(g, gh), stream, args.steps, 2)
            ms_s, _ = _timed(lambda: plan.synthesis(gh, f), stream, args.steps, 2)
            extra = {"transform_ms_per_step": {"analysis": ms_a / args.steps, "synthesis": ms_s / args.steps},
                     "gcv_mode": plan.gcv_mode,
                     "direct_scan": {"value": B / (ms_dir / args.steps / 1e3), "unit": "deblurs/s",
                                     "index_agreement_with_line": float((mi_dir == mi).float().mean())}}
            f_b = torch.empty_like(g)
            mi_b = torch.empty(B, dtype=torch.int32, device=dev)
            ms_b, _ = _timed(lambda: plan.deblur_binned(g, h, f_b, mi_b), stream, args.steps, 2)
            plan.status()
            extra["binned_mu"] = {"value": B / (ms_b / args.steps / 1e3), "unit": "deblurs/s",
                                  "index_agreement_with_full_scan": float((mi_b == mi).float().mean())}
            # the exact GCV functional of Eq. (eq:gcv) (T_X kept in the numerator)
            f_x = torch.empty_like(g)
            mi_x = torch.empty(B, dtype=torch.int32, device=dev)
            ms_x, _ = _timed(lambda: plan.deblur_exact(g, h, f_x, mi_x), stream, args.steps, 2)
            x_launches = plan.last_launch_count
            plan.deblur(g, h, f, mi)
            plan.status()

            def rre(t):
                dlt = (t.cpu().numpy().astype(np.float64) - ftrue).reshape(B, -1)
                return np.linalg.norm(dlt, axis=1) / np.linalg.norm(ftrue.reshape(B, -1), axis=1)
            grid = synth.mu_grid(K)
            extra["exact_gcv"] = {"value": B / (ms_x / args.steps / 1e3), "unit": "deblurs/s",
                                  "ms_per_step": ms_x / args.steps, "gpu_launches": x_launches * args.steps,
                                  "index_agreement_with_approximation": float((mi_x == mi).float().mean()),
                                  "mu": {"approximate_median": float(np.median(grid[mi.cpu().numpy()])),
                                         "exact_median": float(np.median(grid[mi_x.cpu().numpy()]))},
                                  "rre_mean": {"approximate": float(rre(f).mean()), "exact": float(rre(f_x).mean())}}
            if prec == "split_bf16":
                # 4 passes x 3 split products x 2 n^3 (the padded tile shape is what the tensor cores run)
                tm, tn, tk = hobc.tc_tiles()
                npad = [-(-n // t) * t for t in (tm, tn, tk)]
                flops = 4 * 3 * 2.0 * npad[0] * npad[1] * npad[2] * B
                t_s = (ms_a + ms_s) / args.steps / 1e3
                pk = measured_peaks()[0].get("bf16_tflops")
                extra["roofline"] = {"bound": "tensor", "kernel": "k_gemm_split (4 passes)",
                                     "achieved": flops / t_s / 1e12, "peak": pk, "unit": "TFLOP/s",
                                     "frac": flops / t_s / 1e12 / pk if pk else None, "traffic": None,
                                     "flops_per_step": flops}
    if rank == 0 and not args.no_cpu_baseline:
        # error against the FP64 oracle on a sample of the workload's problems
        mus_w = synth.mu_grid(K)
        G_d = torch.empty((mi.numel(), K), dtype=torch.float64, device=dev)
        samples = []
        if args.workload == "batched":
            batch.deblur(g, h, f, mi, G_d)
            torch.cuda.synchronize()      # the plan runs on its own stream
            offs = np.concatenate([[0], np.cumsum([it[0] * it[1] for it in items])])
            fam_of = {1: "S", 2: "C", 3: "S3"}
            fn, Gn, kn = f.cpu().numpy(), G_d.cpu().numpy(), mi.cpu().numpy()
            for deg in (1, 2, 3):           # the two smallest problems of each degree
                idx = sorted([i for i, it in enumerate(items) if it[4] == deg], key=lambda i: items[i][0])[:2]
                for i in idx:
                    nn = items[i][0]
                    samples.append((fam_of[deg], hs[i], gs[i], "lap", mus_w,
                                    fn[offs[i]:offs[i + 1]].reshape(nn, nn), kn[i], Gn[i]))
        elif args.workload == "signals1d":
            plan.deblur(g, h, f, mi, G_d)
            torch.cuda.synchronize()      # the plan runs on its own stream
            fn, Gn, kn = f[:8].cpu().numpy(), G_d[:8].cpu().numpy(), mi[:8].cpu().numpy()
            samples = [("S", hh, gg[i], "I", mus_w, fn[i], kn[i], Gn[i]) for i in range(8)]
        elif args.workload == "volume128":
            vol.deblur(g, h, f, mi, G_d)
            torch.cuda.synchronize()      # the plan runs on its own stream
            samples = [("C", hh, gg[0], "lap", mus_w, f[0].cpu().numpy(), int(mi[0]), G_d[0].cpu().numpy())]
        else:
            plan.deblur(g, h, f, mi, G_d)
            torch.cuda.synchronize()      # the plan runs on its own stream
            fn, Gn, kn = f[:2].cpu().numpy(), G_d[:2].cpu().numpy(), mi[:2].cpu().numpy()
            samples = [("C", hh, gg[i], "lap", mus_w, fn[i], kn[i], Gn[i]) for i in range(2)]
        extra["oracle_error"] = oracle_error_items(samples, K)
    peaks, kind = measured_peaks()
    sec = ms / args.steps / 1e3
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    line = {"metric": f"{args.workload} throughput", "value": units / sec, "unit": unit,
            "n_gpus": max(world, 1) if dist is not None else 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "split_bf16": "bf16x3 (split) / f32"}[prec],
            "data": "synthetic", "config": cfg, "gpu_launches": launches * args.steps,
            "hbm_roofline": {"algorithmic_bytes_per_step": io_bytes, "achieved_gbs": io_bytes / sec / 1e9,
                             "peak_gbs": peaks.get("hbm_gbs"), "frac": io_bytes / sec / 1e9 / peaks.get("hbm_gbs")},
            "clocks": clocks, **extra}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_learned(args):
    """Learned choice of mu against the full GCV scan, at equal relative error.

    Problems (drawn on the GPU, learned.gpu_problems): images as in the other 2D
    workloads blurred by out-of-focus disks (radius U[1.5, 5], 11 x 11 PSF array,
    one per image), noise log-uniform in [1e-3, 3e-2]; degree 2 (cosine family),
    Laplacian, 256 mu in [1e-8, 1], FP32.  The network (histogram features,
    hobc_features_hist) is trained here, outside the timed region, on GCV labels
    of ``--train`` problems at 256^2; it is timed on 8192 other problems at 256^2
    and on 8192 at 1024^2 (in chunks of 512, each chunk's three arms timed in
    turn), against the full scan and the binned choice on the same problems."""
    import torch
    from paper_0906_2704_gb300 import hobc, learned, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n, taps, K = 256, 11, 256
    mus = synth.mu_grid(K)
    B = 512
    plan = hobc.Plan(2, (n, n), (taps, taps), 2, mus, L="lap", prec="fp32", family="cosine", psf_symmetric=True,
                     batch=B, psf_per_item=True, stream=stream)
    # ---- training (not timed): data drawn and labelled on the GPU
    t0 = time.time()
    Xtr, ttr = learned.training_set(plan, args.train, 1, "disk", taps, kind="hist")
    torch.cuda.synchronize()
    t_data = time.time() - t0
    t1 = time.time()
    net = learned.init_network(Xtr, 256, seed=0, stream=stream.cuda_stream, kind="hist")
    hist = learned.fit(net, Xtr, ttr, epochs=args.epochs, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t1

    def rre(f, ft):
        d = (f.double() - ft.double()).flatten(1)
        return (d.norm(dim=1) / ft.double().flatten(1).norm(dim=1)).cpu().numpy()

    def evaluate(size, count, batch, seed, steps, net):
        """The three arms on ``count`` problems of one size, chunk by chunk."""
        pl = plan if size == n else hobc.Plan(2, (size, size), (taps, taps), 2, mus, L="lap", prec="fp32",
                                              family="cosine", psf_symmetric=True, batch=batch, psf_per_item=True,
                                              stream=stream)
        chunk = 512
        ms = {"learned": 0.0, "gcv": 0.0, "binned": 0.0}
        r = {"learned": [], "gcv": [], "binned": []}
        fbs, agree_b, lab_err = [], [], []
        clk = {}
        launches = 0
        for c0 in range(0, count, chunk):
            g, h, ft, _ = learned.gpu_problems(chunk, size, seed * 1000003 + c0, dev, psf="disk", taps=taps,
                                               truth=True)
            f_l, f_g, f_b = torch.empty_like(g), torch.empty_like(g), torch.empty_like(g)
            mu_l = torch.empty(chunk, dtype=torch.float64, device=dev)
            fb_l = torch.empty(chunk, dtype=torch.int32, device=dev)
            mi_g = torch.empty(chunk, dtype=torch.int32, device=dev)
            mi_b = torch.empty(chunk, dtype=torch.int32, device=dev)
            fb_b = torch.empty(chunk, dtype=torch.int32, device=dev)
            cs = [slice(s, s + batch) for s in range(0, chunk, batch)]
            arms = {"learned": lambda: [pl.deblur_learned(net, g[c], h[c], f_l[c], mu_l[c], fb_l[c]) for c in cs],
                    "gcv": lambda: [pl.deblur(g[c], h[c], f_g[c], mi_g[c]) for c in cs],
                    "binned": lambda: [pl.deblur_binned(g[c], h[c], f_b[c], mi_b[c], fb_b[c]) for c in cs]}
            for name, fn in arms.items():
                t_ms, c_ = _timed(fn, stream, steps, 3 if c0 == 0 else 1)
                ms[name] += t_ms / steps
                clk.setdefault(name, c_)
                if name == "learned":
                    launches += pl.last_launch_count * len(cs)
            r["learned"].append(rre(f_l, ft))
            r["gcv"].append(rre(f_g, ft))
            r["binned"].append(rre(f_b, ft))
            fbs.append(fb_l.cpu().numpy())
            agree_b.append((mi_b == mi_g).cpu().numpy())
            lab = np.log10(mus)[mi_g.cpu().numpy()]
            lab_err.append(np.abs(np.log10(mu_l.cpu().numpy()) - lab))
            del g, h, ft, f_l, f_g, f_b
        rl, rg, rb = (np.concatenate(r[k]) for k in ("learned", "gcv", "binned"))
        err = np.concatenate(lab_err)
        out = {"images": count, "batch": batch,
               "learned": {"images_per_s": count / (ms["learned"] / 1e3), "fallback_rate": float(np.mean(np.concatenate(fbs))),
                           "rre_mean": float(rl.mean()), "rre_ratio_to_gcv": float(rl.mean() / rg.mean()),
                           "log10_mu_abs_err_vs_gcv": {"median": float(np.median(err)),
                                                       "p90": float(np.quantile(err, 0.9))}},
               "gcv_scan": {"images_per_s": count / (ms["gcv"] / 1e3), "rre_mean": float(rg.mean())},
               "binned_mu": {"images_per_s": count / (ms["binned"] / 1e3), "rre_ratio_to_gcv": float(rb.mean() / rg.mean()),
                             "index_agreement_with_full_scan": float(np.mean(np.concatenate(agree_b)))},
               "speedup_learned_vs_gcv_scan": ms["gcv"] / ms["learned"]}
        return out, ms, clk, launches

    res256, ms256, clk256, launches = evaluate(n, 8192, B, 2, args.steps, net)
    res1024, _, _, _ = evaluate(1024, args.count_1024, 64, 3, max(1, args.steps // 2), net)
    # the 256^2 network does not carry over to 1024^2 (the GCV choice shifts with the size);
    # a second network trained on problems drawn at 1024^2
    t2 = time.time()
    plan_big = hobc.Plan(2, (1024, 1024), (taps, taps), 2, mus, L="lap", prec="fp32", family="cosine",
                         psf_symmetric=True, batch=64, psf_per_item=True, stream=stream)
    Xb, tb = learned.training_set(plan_big, args.train_1024, 4, "disk", taps, kind="hist", chunk=256)
    net_big = learned.init_network(Xb, 256, seed=0, stream=stream.cuda_stream, kind="hist")
    hist_big = learned.fit(net_big, Xb, tb, epochs=40, batch=256, lr=1e-3)
    plan_big.close()
    del Xb, tb
    torch.cuda.synchronize()
    t_big = time.time() - t2
    res1024_own, _, _, _ = evaluate(1024, args.count_1024, 64, 3, max(1, args.steps // 2), net_big)
    res1024_own["train"] = {"problems": args.train_1024, "seconds": t_big, "loss_last": hist_big[-1]}
    peaks, _ = measured_peaks()
    sec_l = ms256["learned"] / 1e3
    io_bytes = 2 * 8192 * n * n * 4
    line = {"metric": "learned-mu deblurs/s at equal relative error (256x256 and 1024x1024, cosine family, disk PSF)",
            "value": res256["learned"]["images_per_s"], "unit": "images/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms256["learned"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (drawn on the GPU)",
            "config": {"workload": "8192 problems 256x256 and 1024x1024, disk PSF r~U[1.5,5] (11x11), noise "
                                   "log-U[1e-3,3e-2], degree 2 (cosine), Laplacian, 256 mu in [1e-8,1], learned mu "
                                   "(histogram features) with bracket check", "batch": B,
                       "train_problems": int(Xtr.shape[0]), "features": "hist"},
            "at_256": res256, "at_1024_network_trained_at_256": res1024, "at_1024": res1024_own,
            "train": {"seconds": t_train, "data_seconds": t_data, "epochs": args.epochs,
                      "loss_first": hist[0], "loss_last": hist[-1]},
            "gpu_launches": launches * args.steps,
            "hbm_roofline": {"algorithmic_bytes_per_step": io_bytes, "achieved_gbs": io_bytes / sec_l / 1e9,
                             "peak_gbs": peaks.get("hbm_gbs"), "frac": io_bytes / sec_l / 1e9 / peaks.get("hbm_gbs")},
            "clocks": clk256.get("learned"), "clocks_gcv_scan": clk256.get("gcv")}
    print(json.dumps(line), flush=True)
    return 0


def run_plain(args):
    """The headline workload's step alone (one plan, hobc_deblur on the 1024^2 batch,
    no other arm, no CPU baseline): the command the kernel profiles use."""
    import torch
    from paper_0906_2704_gb300 import hobc, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    B, prec = args.batch, args.prec
    npdt = np.float64 if prec == "fp64" else np.float32
    h, g, _ = make_inputs(B, seed=rank_seed(0))
    stream = torch.cuda.current_stream()
    plan = hobc.Plan(2, (N_SIDE, N_SIDE), h.shape, 2, synth.mu_grid(K_MU), L="I", prec=prec, family="fourier",
                     batch=B, stream=stream)
    if prec != "fp64" and not args.direct:
        plan.set_gcv_mode("expansion")
    g_d = torch.from_numpy(g.astype(npdt)).to(dev)
    h_d = torch.from_numpy(h.astype(npdt)).to(dev)
    f_d = torch.empty_like(g_d)
    mi_d = torch.empty(B, dtype=torch.int32, device=dev)
    ms, clocks = _timed(lambda: plan.deblur(g_d, h_d, f_d, mi_d), stream, args.steps, args.warmup)
    line = {"metric": f"{WORKLOAD} deblurs/s (the step alone)", "value": B * args.steps / (ms / 1e3),
            "unit": "deblurs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "gcv_mode": plan.gcv_mode,
            "gpu_launches": plan.last_launch_count * args.steps, "batch": B, "precision": prec, "clocks": clocks}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_bccompare(args):
    """The paper's comparison of boundary conditions (its 2D out-of-focus experiment) on
    synthetic images: RRE at the RRE-optimal grid mu, at the GCV mu (the paper's
    approximation, Eq. (eq:gcv2)) and at the exact-GCV mu (Eq. (eq:gcv)) for periodic,
    reflective, antireflective (degree 1), degree-2 (cosine) and degree-3 conditions.
    Images as in the other 2D workloads, out-of-focus (disk) PSF of radius 3.3 in a
    9 x 9 array, 0.1% noise, L = I (the paper's setting) and the Laplacian, 64 mu."""
    import torch
    from paper_0906_2704_gb300 import hobc, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, taps, B, K, eta = 256, 9, 8, 64, 1e-3
    rng = np.random.default_rng(11)
    m = taps // 2
    disk = synth.disk_psf(3.3)
    h = np.zeros((taps, taps))
    k = disk.shape[0] // 2
    h[m - k:m + k + 1, m - k:m + k + 1] = disk
    gs, fts = [], []
    for _ in range(B):
        f_ext = synth.image_2d(rng, n + 2 * m, n + 2 * m)
        gs.append(synth.add_noise(rng, synth.blur_valid_2d(f_ext, h), eta))
        fts.append(f_ext[m:m + n, m:m + n])
    g = np.stack(gs).astype(np.float32)
    ft = np.stack(fts)
    mus = synth.mu_grid(K)
    g_d, h_d = torch.from_numpy(g).to(dev), torch.from_numpy(h.astype(np.float32)).to(dev)
    tables, clocks = {}, None
    for L in ("I", "lap"):
        table = {}
        # classical conditions on the dense tensor-core engine (orthonormal transforms);
        # the high-order families on the FFT engine in FP64 (degree 3 is ill-conditioned)
        for fam, deg, prec in (("periodic", 0, "split_bf16"), ("reflective", 0, "split_bf16"), ("sine", 1, "fp64"),
                               ("cosine", 2, "fp64"), ("sine3", 3, "fp64")):
            dt = torch.float64 if prec == "fp64" else torch.float32
            plan = hobc.Plan(2, (n, n), (taps, taps), deg, mus, L=L, prec=prec, family=fam, psf_symmetric=True,
                             batch=B)
            S = plan.spec_elems
            gg, hh = g_d.to(dt), h_d.to(dt)
            D = torch.empty((1, S), dtype=dt, device=dev)
            G = torch.empty((B, S), dtype=dt, device=dev)
            f = torch.empty_like(gg)
            mi = torch.empty(B, dtype=torch.int32, device=dev)
            ms, clocks = _timed(lambda: plan.deblur(gg, hh, f, mi), torch.cuda.current_stream(), args.steps,
                                args.warmup)
            plan.eigenvalues(hh, D)
            plan.analysis(gg, G)
            rre = np.empty((K, B))
            for j in range(K):
                plan.filter_synthesis(G, D, torch.full((B,), j, dtype=torch.int32, device=dev), f)
                d = (f.cpu().numpy().astype(np.float64) - ft).reshape(B, -1)
                rre[j] = np.linalg.norm(d, axis=1) / np.linalg.norm(ft.reshape(B, -1), axis=1)
            plan.gcv(G, D, torch.empty((B, K), dtype=torch.float64, device=dev), mi)
            plan.status()
            kg = mi.cpu().numpy()
            # the exact functional of Eq. (eq:gcv): T_X kept in the numerator
            plan.gcv_exact(G, D, None, mi)
            plan.status()
            kx = mi.cpu().numpy()
            table[fam] = {"rre_opt": float(rre.min(axis=0).mean()), "rre_gcv": float(rre[kg, np.arange(B)].mean()),
                          "rre_gcv_exact": float(rre[kx, np.arange(B)].mean()),
                          "mu_gcv_median": float(np.median(mus[kg])), "mu_gcv_exact_median": float(np.median(mus[kx])),
                          "engine": prec, "deblurs_per_s": B / (ms / args.steps / 1e3)}
        tables[L] = table
    # nonsymmetric PSF (the paper's last 2D experiment, and its 1D moving-blur example):
    # out-of-focus combined with a one-sided motion; with no symmetry only the Fourier
    # families and the periodic conditions have fast transforms, all on the FFT engine
    # in FP64 (degree 4 is ill-conditioned)
    tn = 15
    hn = synth.motion_defocus_psf(2.3, 6.0, 30.0, tn)
    mn = tn // 2
    eta_n = 1e-2
    gs, fts = [], []
    for _ in range(B):
        f_ext = synth.image_2d(rng, n + 2 * mn, n + 2 * mn)
        gs.append(synth.add_noise(rng, synth.blur_valid_2d(f_ext, hn), eta_n))
        fts.append(f_ext[mn:mn + n, mn:mn + n])
    gn_d = torch.from_numpy(np.stack(gs)).to(dev)
    hn_d = torch.from_numpy(hn).to(dev)
    ftn = np.stack(fts)
    tables_ns = {}
    for L in ("I", "lap"):
        table = {}
        for fam, deg in (("periodic", 0), ("fourier", 2), ("fourier4", 4)):
            plan = hobc.Plan(2, (n, n), (tn, tn), deg, mus, L=L, prec="fp64", family=fam, psf_symmetric=False,
                             batch=B)
            S = plan.spec_elems
            D = torch.empty((1, S, 2), dtype=torch.float64, device=dev)
            G = torch.empty((B, S, 2), dtype=torch.float64, device=dev)
            f = torch.empty_like(gn_d)
            mi = torch.empty(B, dtype=torch.int32, device=dev)
            ms, clocks = _timed(lambda: plan.deblur(gn_d, hn_d, f, mi), torch.cuda.current_stream(), args.steps,
                                args.warmup)
            plan.eigenvalues(hn_d, D)
            plan.analysis(gn_d, G)
            rre = np.empty((K, B))
            for j in range(K):
                plan.filter_synthesis(G, D, torch.full((B,), j, dtype=torch.int32, device=dev), f)
                d = (f.cpu().numpy() - ftn).reshape(B, -1)
                rre[j] = np.linalg.norm(d, axis=1) / np.linalg.norm(ftn.reshape(B, -1), axis=1)
            plan.gcv(G, D, torch.empty((B, K), dtype=torch.float64, device=dev), mi)
            plan.status()
            kg = mi.cpu().numpy()
            row = {"rre_opt": float(rre.min(axis=0).mean()), "rre_gcv": float(rre[kg, np.arange(B)].mean()),
                   "mu_gcv_median": float(np.median(mus[kg])), "engine": "fp64",
                   "deblurs_per_s": B / (ms / args.steps / 1e3)}
            if fam == "fourier":           # the exact functional is built for the degree-2 family
                plan.gcv_exact(G, D, None, mi)
                plan.status()
                kx = mi.cpu().numpy()
                row["rre_gcv_exact"] = float(rre[kx, np.arange(B)].mean())
            table[fam] = row
        tables_ns[L] = table
    table = tables["I"]
    line = {"metric": "RRE at mu_opt / mu_GCV by boundary condition (2D out-of-focus blur, 0.1% noise, L=I)",
            "value": table["reflective"]["rre_opt"] / table["cosine"]["rre_opt"],
            "unit": "RRE(reflective) / RRE(degree 2) at mu_opt", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3 (split) / f32", "data": "synthetic",
            "config": {"workload": f"{B} images {n}x{n}, disk PSF r=3.3 (9x9), 0.1% noise, {K} mu in [1e-8,1]; "
                                   "periodic/reflective on the dense split-BF16 engine, degrees 1-3 on the FFT "
                                   "engine in FP64", "batch": B},
            "rre": tables,
            "rre_nonsymmetric": {"config": f"{B} images {n}x{n}, out-of-focus r=2.3 plus one-sided motion of 6 px "
                                           f"at 30 degrees ({tn}x{tn}), 1% noise, {K} mu; FFT engine, FP64",
                                 **tables_ns},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp32", "fp64", "split_bf16"], default="fp32")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--direct", action="store_true",
                    help="fourier1024_step: the term-by-term GCV scan instead of the expansion")
    ap.add_argument("--workload", choices=["fourier1024", "fourier1024_step", "batched", "signals1d", "cosine512",
                                           "cosine1024",
                                           "learned", "bccompare", "volume128"],
                    default="fourier1024")
    ap.add_argument("--train", type=int, default=200000, help="training problems of the learned workload")
    ap.add_argument("--epochs", type=int, default=30, help="training epochs of the learned workload")
    ap.add_argument("--count-1024", dest="count_1024", type=int, default=8192,
                    help="1024^2 problems of the learned workload")
    ap.add_argument("--train-1024", dest="train_1024", type=int, default=16384,
                    help="training problems at 1024^2 of the learned workload")
    ap.add_argument("--learned-train", dest="learned_train", type=int, default=16384,
                    help="training problems of the default line's learned arm")
    ap.add_argument("--count", type=int, default=4096, help="problems of the batched workload")
    ap.add_argument("--no-autotune", dest="no_autotune", action="store_true",
                    help="batched workload: the default FFT schedule, no autotuning run")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "bccompare":
        return run_bccompare(args)
    if args.workload == "fourier1024_step":
        return run_plain(args)
    if args.workload != "fourier1024":
        return run_other(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
