"""The C-ABI library loads, exports every function include/hobc.h declares, and
rejects bad problem descriptions on the host before touching the GPU.  CPU only:
no call here reaches a kernel or allocates device memory."""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_0906_2704_gb300", "libhobc.so")


@pytest.fixture(scope="module")
def hobc():
    if not os.path.exists(LIB):
        from paper_0906_2704_gb300 import build
        build.build()
    from paper_0906_2704_gb300 import hobc as mod
    return mod


def test_library_exports_every_declared_function(hobc):
    names = hobc.declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(hobc.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(hobc):
    lib = hobc.library()
    for code, name in enumerate(hobc.STATUS):
        assert lib.hobc_status_str(code).decode() == name


def _create(hobc, **kw):
    args = dict(ndim=1, n=64, psf=5, bc_degree=2, mu_grid=[1e-3, 1e-2], psf_symmetric=True)
    args.update(kw)
    return hobc.Plan(**args)


@pytest.mark.parametrize("kw,status", [
    (dict(n=5), "HOBC_ERR_SIZE"),                       # n < 6
    (dict(n=2048), "HOBC_ERR_SIZE"),                    # n > 1024
    (dict(psf=4), "HOBC_ERR_SIZE"),                     # even PSF
    (dict(n=8, psf=7), "HOBC_ERR_SIZE"),                # 2m+1 > n-2
    (dict(bc_degree=5), "HOBC_ERR_UNSUPPORTED"),
    (dict(family="cosine4", bc_degree=4, psf_symmetric=False), "HOBC_ERR_UNSUPPORTED"),   # needs symmetry
    (dict(family="fourier4", bc_degree=2), "HOBC_ERR_UNSUPPORTED"),
    (dict(family="fourier4", bc_degree=4, prec="fp32", psf_symmetric=False), "HOBC_ERR_UNSUPPORTED"),
    (dict(family="fourier4", bc_degree=4, n=7, psf=1), "HOBC_ERR_SIZE"),   # N = n - 4 >= 4
    (dict(family="periodic", bc_degree=2), "HOBC_ERR_UNSUPPORTED"),       # periodic: degree 0
    (dict(family="cosine4", bc_degree=2), "HOBC_ERR_UNSUPPORTED"),
    (dict(bc_degree=4, n=9, psf=7), "HOBC_ERR_SIZE"),               # 2m+1 <= n-4 for degree 4
    (dict(prec="split_bf16", bc_degree=4), "HOBC_ERR_UNSUPPORTED"),  # no dense matrices for degree 4
    (dict(bc_degree=3, psf_symmetric=False), "HOBC_ERR_UNSUPPORTED"),   # cubic sine family needs symmetry
    (dict(family="sine3", bc_degree=2), "HOBC_ERR_UNSUPPORTED"),
    (dict(bc_degree=3, n=9, psf=7), "HOBC_ERR_SIZE"),               # 2m+1 <= n-4 for degree 3
    (dict(bc_degree=1, psf_symmetric=False), "HOBC_ERR_UNSUPPORTED"),   # antireflective needs symmetry
    (dict(family="sine", bc_degree=2), "HOBC_ERR_UNSUPPORTED"),
    (dict(family="fourier", bc_degree=1), "HOBC_ERR_UNSUPPORTED"),
    (dict(mu_grid=[1e-3, 0.0]), "HOBC_ERR_ARG"),        # mu > 0 (Eq. (eq:mintik))
    (dict(mu_grid=[1e-3, float("nan")]), "HOBC_ERR_NONFINITE"),
    (dict(mu_grid=[1e-3, float("inf")]), "HOBC_ERR_NONFINITE"),
    (dict(batch=0), "HOBC_ERR_ARG"),
    (dict(prec="fp32", mu_grid=[1e-20, 1.0]), "HOBC_ERR_ARG"),   # FP32 pairs grid values: mu >= 1e-18
    (dict(ndim=3), "HOBC_ERR_ARG"),
])
def test_plan_validation_rejects_bad_descriptions(hobc, kw, status):
    with pytest.raises(hobc.HobcError) as ei:
        _create(hobc, **kw)
    assert hobc.STATUS[ei.value.status] == status


def test_null_arguments_rejected(hobc):
    lib = hobc.library()
    out = ctypes.c_void_p()
    assert lib.hobc_plan_create(None, None, None, ctypes.byref(out)) == 1
    assert lib.hobc_deblur(None, None, None, None, None, None) == 1
    assert lib.hobc_deblur_host(None, None, None, None, None, None) == 1
    assert lib.hobc_deblur_host_async(None, None, None, None, None, None) == 1
    assert lib.hobc_plan_wait(None) == 1
    assert lib.hobc_analysis(None, None, None) == 1
    assert lib.hobc_gcv(None, None, None, None, None) == 1


def test_binding_has_no_cpu_fallback(hobc):
    """The binding only marshals: it refuses host tensors for device entry points."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        hobc._ptr(torch.zeros(4))
    with pytest.raises(ValueError):
        hobc._hptr(np.zeros((4, 4))[:, ::2])


def test_learned_entry_points_reject_bad_arguments_on_the_host(hobc):
    """The learned-mu calls of include/hobc_learned.h check their arguments
    before any CUDA call (no device needed)."""
    lib = hobc.library()
    out = ctypes.c_void_p()
    arg = hobc.STATUS.index("HOBC_ERR_ARG")
    assert lib.hobc_mlp_create(0, 16, None, ctypes.byref(out)) == arg
    assert lib.hobc_mlp_create(128, 0, None, ctypes.byref(out)) == arg
    assert lib.hobc_mlp_create(5000, 16, None, ctypes.byref(out)) == arg
    assert lib.hobc_mlp_create(128, 16, None, None) == arg
    assert lib.hobc_mlp_param_count(None) == 0
    assert lib.hobc_mlp_last_launch_count(None) == 0
    assert lib.hobc_mlp_set_params(None, None) == arg
    assert lib.hobc_mlp_get_params(None, None) == arg
    assert lib.hobc_mlp_forward(None, None, 1, None) == arg
    assert lib.hobc_mlp_gradients(None, None, None, 1, None, None) == arg
    assert lib.hobc_mlp_train_step(None, None, None, 1, 1e-3, 0.0, None) == arg
    assert lib.hobc_mlp_save(None, b"x") == arg
    assert lib.hobc_mlp_load(None, b"x") == arg
    assert lib.hobc_features(None, None, None, None) == arg
    assert lib.hobc_deblur_learned(None, None, None, None, None, None, None) == arg
    assert lib.hobc_gcv_binned(None, None, None, None, None, None) == arg
    assert lib.hobc_deblur_binned(None, None, None, None, None, None) == arg
    assert lib.hobc_gcv_refine(None, None, None, None, None, None) == arg
    assert lib.hobc_deblur_refined(None, None, None, None, None, None) == arg
    assert lib.hobc_filter_synthesis_mu(None, None, None, None, None) == arg
    assert lib.hobc_gcv_exact(None, None, None, None, None) == arg
    assert lib.hobc_volume_create(None, None, None, None) == arg
    assert lib.hobc_volume_deblur(None, None, None, None, None, None) == arg
    assert lib.hobc_volume_analysis(None, None, None) == arg
    assert lib.hobc_volume_launch_count(None) == 0
    lib.hobc_volume_destroy(None)
    assert lib.hobc_deblur_exact(None, None, None, None, None, None) == arg
    lib.hobc_mlp_destroy(None)


@pytest.mark.parametrize("kw", [
    dict(n=5), dict(n=2048), dict(bc_degree=5), dict(family="cosine4", bc_degree=4, psf_symmetric=False),
    dict(family="fourier4", bc_degree=4, prec="fp32", n=16, psf=3), dict(family="periodic", bc_degree=2),
    dict(family="cosine4", bc_degree=2), dict(bc_degree=3, psf_symmetric=False),
    dict(family="sine3", bc_degree=2), dict(bc_degree=1, psf_symmetric=False),
    dict(family="sine", bc_degree=2), dict(family="fourier", bc_degree=1), dict(batch=0),
    dict(ndim=3), dict(family="sine3", bc_degree=3, n=7, psf=1), dict(family="cosine4", bc_degree=4, n=6, psf=1),
    dict(bc_degree=3, n=7, psf=1), dict(bc_degree=4, n=7, psf=1),
    dict(bc_degree=4, prec="fp32", n=16, psf=3),                   # degree 4 is FP64 only
    dict(family="reflective", bc_degree=0, prec="fp64"),           # reflective: dense engine only
])
def test_noalloc_rejects_what_plan_create_rejects(hobc, kw):
    """hobc_gcv_noalloc checks a description as hobc_plan_create does (the PSF
    extents aside), so no geometry that a plan refuses runs there."""
    with pytest.raises(hobc.HobcError) as ei:
        _create(hobc, **kw)
    args = dict(ndim=1, n=64, bc_degree=2, psf_symmetric=True)
    args.update({k: v for k, v in kw.items() if k != "psf"})
    ndim = args.pop("ndim")
    n = args.pop("n")
    deg = args.pop("bc_degree")
    desc = hobc.make_desc(ndim, n, deg, 2, **args)
    lib = hobc.library()
    got = lib.hobc_gcv_noalloc(ctypes.byref(desc), ctypes.c_void_p(256), ctypes.c_void_p(256),
                               ctypes.c_void_p(256), None, ctypes.c_void_p(256), None)
    assert got == ei.value.status, (kw, hobc.STATUS[got], hobc.STATUS[ei.value.status])


def test_fp32_degree4_rejected(hobc):
    """Degree 4 is offered in FP64 only: its cond(T) is 644 at the smallest field of
    view (n = 8), so the FP32 rounding bound 64 eps32 cond(T) is above 1e-3 at every size."""
    for n in (8, 12, 64):
        with pytest.raises(hobc.HobcError) as ei:
            _create(hobc, n=n, psf=3, bc_degree=4, prec="fp32")
        assert hobc.STATUS[ei.value.status] == "HOBC_ERR_UNSUPPORTED"


def test_fft_length_and_schedule_validation(hobc):
    """FFT lengths of the batched path's lines (host arithmetic, no device): the
    core DFT (N = n - 2, n - 4 for degree 3; 2(N + 1) for degrees 1 and 3) if it is
    a power of two, else the chirp-z padding 2^k >= 2 L - 1."""
    assert hobc.fft_length(2, 66) == 64          # N = 64
    assert hobc.fft_length(2, 512) == 1024       # L = 510 -> 2^k >= 1019
    assert hobc.fft_length(1, 129) == 256        # L = 2 * 128 = 256
    assert hobc.fft_length(1, 130) == 1024       # L = 258 -> 2^k >= 515
    assert hobc.fft_length(3, 100) == 512        # N = 96, L = 194 -> 2^k >= 387
    assert hobc.fft_length(4, 100) == 0 and hobc.fft_length(2, 5) == 0
    lib = hobc.library()
    bad = (hobc.FftSchedule * 1)()
    bad[0].bc_degree, bad[0].fft_length, bad[0].radix = 2, 500, 8
    out = ctypes.c_void_p()
    d = hobc.BatchDesc()
    d.count, d.n_mu = 1, 1
    it = (hobc.BatchItem * 1)()
    mu = (ctypes.c_double * 1)(1e-2)
    assert lib.hobc_batch_create_tuned(ctypes.byref(d), it, mu, bad, 1, None, ctypes.byref(out)) == 1


def test_gcv_mode_and_host_chunk_calls_reject_bad_arguments_on_the_host(hobc):
    """The curve-by-expansion and host-chunk calls check their arguments before
    any CUDA call; a batch description with an unknown gcv_mode, the expansion on
    an FP64 batch, or a grid whose truncation bound would pass 1e-8 is refused
    before any device work."""
    lib = hobc.library()
    assert lib.hobc_plan_set_gcv_mode(None, hobc.GCV_MODE["expansion"]) == 1
    assert lib.hobc_plan_gcv_mode(None) == -1
    assert lib.hobc_gcv_expansion_bound(None) == -1.0
    assert lib.hobc_plan_set_host_chunks(None, 2) == 1
    items = (hobc.BatchItem * 2)()
    for it, n in zip(items, (32, 48)):
        it.n[0], it.n[1], it.psf[0], it.psf[1], it.bc_degree = n, n, 5, 5, 2
    cases = [("fp32", 7, (1e-8, 1.0), 1),                           # unknown mode: HOBC_ERR_ARG
             ("fp64", hobc.GCV_MODE["expansion"], (1e-8, 1.0), 2),  # FP64: HOBC_ERR_UNSUPPORTED
             ("fp32", hobc.GCV_MODE["expansion"], (1e-18, 1e12), 2)]  # 36 decades: bound > 1e-8
    for prec, mode, (lo, hi), status in cases:
        mus = np.geomspace(lo, hi, 16)
        desc = hobc.BatchDesc(count=2, L=1, prec=hobc.PRECISION[prec], n_mu=16, gcv_mode=mode)
        out = ctypes.c_void_p()
        got = lib.hobc_batch_create(ctypes.byref(desc), items,
                                    mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, ctypes.byref(out))
        assert got == status, (prec, mode, lo, hi, got)
        assert not out.value
