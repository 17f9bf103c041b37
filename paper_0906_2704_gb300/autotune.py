"""Autotuner of the batched path's FFT schedule (include/hobc.h, hobc_fft_schedule).

For every kind of line a batch holds -- a boundary-condition degree and an FFT
length -- the FFT stages can run in radix 16 (16 values a thread) or radix 8
(8 values a thread, twice the threads a line pair).  tune_batched measures both
on the GPU for every kind with a choice (FFT length >= 256): a batch of problems
of that kind alone, each schedule timed with CUDA events after warm-up, the
faster kept.  The table is cached as JSON, keyed by precision, smoothing
operator and grid size, so a later batch with the same kinds of line reuses it.
Everything timed runs in the library; this module only builds batches and
reads clocks.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hobc


def _torch():
    import torch
    return torch


def default_cache_path() -> str:
    base = os.environ.get("HOBC_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "hobc_gb300")
    return os.path.join(base, "batched_fft_schedule.json")


def line_kinds(items):
    """(degree, FFT length) -> the sizes n of the batch's lines of that kind."""
    kinds = {}
    for n0, n1, _, _, deg in items:
        for n in (n0, n1):
            kinds.setdefault((int(deg), hobc.fft_length(deg, n)), set()).add(int(n))
    return kinds


def _time_batch(items, mus, L, prec, schedule, reps, warmup):
    torch = _torch()
    stream = torch.cuda.current_stream()
    b = hobc.Batch(items, mus, L=L, prec=prec, stream=stream, schedule=schedule)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(0)
    g = torch.from_numpy(rng.standard_normal(int(b.img_off[-1]))).to("cuda", dt)
    h = torch.zeros(int(b.psf_off[-1]), dtype=dt, device="cuda")
    for i, (_, _, p0, p1, _) in enumerate(items):         # a centred delta: any symmetric PSF would do
        h[int(b.psf_off[i]) + (p0 // 2) * p1 + p1 // 2] = 1.0
    f = torch.empty_like(g)
    for _ in range(warmup):
        b.deblur(g, h, f)
    torch.cuda.synchronize()
    a_, z_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(3):
        a_.record(stream)
        for _ in range(reps):
            b.deblur(g, h, f)
        z_.record(stream)
        torch.cuda.synchronize()
        best = min(best, a_.elapsed_time(z_) / reps)
    b.close()
    return best


def tune_batched(items, mus, L: str = "lap", prec: str = "fp32", cache: str | None = None, per_kind: int = 64,
                 reps: int = 5, warmup: int = 3, refresh: bool = False):
    """The FFT schedule (a list of (degree, FFT length, radix)) for a batch of these
    items, and a record of the measurements.  Each kind of line with a choice is
    timed on a batch of up to per_kind square problems of the kind's sizes (PSF
    3 x 3), in radix 16 and in radix 8."""
    cache = cache or default_cache_path()
    key = f"{prec}/{L}/K{len(mus)}"
    table = {}
    if os.path.exists(cache) and not refresh:
        with open(cache) as fh:
            table = json.load(fh)
    entries = table.setdefault(key, {})
    record = {}
    for (deg, M), sizes in sorted(line_kinds(items).items()):
        if M < 256:
            continue
        name = f"{deg}/{M}"
        if name not in entries:
            sz = sorted(sizes)
            pick = [sz[int(i)] for i in np.linspace(0, len(sz) - 1, min(per_kind, len(sz)))]
            sub = [(n, n, 3, 3, deg) for n in (pick * (per_kind // len(pick) + 1))[:per_kind]]
            t16 = _time_batch(sub, mus, L, prec, [(deg, M, 16)], reps, warmup)
            t8 = _time_batch(sub, mus, L, prec, [(deg, M, 8)], reps, warmup)
            entries[name] = {"radix": 16 if t16 <= t8 else 8, "ms_radix16": t16, "ms_radix8": t8,
                             "problems": len(sub)}
        record[name] = entries[name]
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tmp = cache + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache)
    schedule = [(int(k.split("/")[0]), int(k.split("/")[1]), v["radix"]) for k, v in record.items()]
    return schedule, record
