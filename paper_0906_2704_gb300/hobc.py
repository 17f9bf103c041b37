"""Python binding of the C ABI in include/hobc.h, include/hobc_learned.h and
include/hobc_binned.h (ctypes; marshalling only).

Every step of the method runs in the CUDA library ``libhobc.so`` built in this
package directory by ``paper_0906_2704_gb300.build``.  There is no fallback: if
the library is missing, importing this module raises.

Device buffers are passed as torch CUDA tensors (or raw integer addresses);
host buffers for :meth:`Plan.deblur_host` as NumPy arrays.  Shapes and dtypes
are checked here only to produce clear errors before the C call.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhobc.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "hobc.h")
HEADER_PATHS = [HEADER_PATH, os.path.join(os.path.dirname(_HERE), "include", "hobc_learned.h"),
                os.path.join(os.path.dirname(_HERE), "include", "hobc_binned.h"),
                os.path.join(os.path.dirname(_HERE), "include", "hobc_tc.h"),
                os.path.join(os.path.dirname(_HERE), "include", "hobc_refine.h"),
                os.path.join(os.path.dirname(_HERE), "include", "hobc_exact.h"),
                os.path.join(os.path.dirname(_HERE), "include", "hobc_volume.h")]

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_0906_2704_gb300.build`")

_lib = ctypes.CDLL(LIB_PATH)

FAMILY = {"auto": 0, "sine": 1, "cosine": 2, "fourier": 3, "sine3": 4, "reflective": 5, "periodic": 6,
          "cosine4": 7, "fourier4": 8}
FAMILY_NAME = {v: k for k, v in FAMILY.items()}
SMOOTHING = {"I": 0, "identity": 0, "lap": 1, "laplacian": 1}
PRECISION = {"fp64": 0, "fp32": 1, "split_bf16": 2}
STATUS = ["HOBC_OK", "HOBC_ERR_ARG", "HOBC_ERR_UNSUPPORTED", "HOBC_ERR_SIZE",
          "HOBC_ERR_NONFINITE", "HOBC_ERR_CUDA", "HOBC_ERR_TIMEOUT"]


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 2),
        ("psf", ctypes.c_int * 2),
        ("bc_degree", ctypes.c_int),
        ("family", ctypes.c_int),
        ("psf_symmetric", ctypes.c_int),
        ("L", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("n_mu", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("psf_per_item", ctypes.c_int),
    ]


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_lib.hobc_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_double), _vp,
                                  ctypes.POINTER(_vp)]
_lib.hobc_plan_create.restype = ctypes.c_int
_lib.hobc_plan_destroy.argtypes = [_vp]
_lib.hobc_plan_destroy.restype = None
_lib.hobc_plan_family.argtypes = [_vp]
_lib.hobc_plan_family.restype = ctypes.c_int
_lib.hobc_plan_set_host_chunks.argtypes = [_vp, ctypes.c_int]
_lib.hobc_plan_set_host_chunks.restype = ctypes.c_int
_lib.hobc_plan_set_gcv_mode.argtypes = [_vp, ctypes.c_int]
_lib.hobc_plan_set_gcv_mode.restype = ctypes.c_int
_lib.hobc_plan_gcv_mode.argtypes = [_vp]
_lib.hobc_plan_gcv_mode.restype = ctypes.c_int
_lib.hobc_gcv_expansion_bound.argtypes = [_vp]
_lib.hobc_gcv_expansion_bound.restype = ctypes.c_double
GCV_MODE = {"direct": 0, "expansion": 1}
_lib.hobc_spectrum_size.argtypes = [_vp, ctypes.POINTER(_sz), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_sz)]
_lib.hobc_spectrum_size.restype = ctypes.c_int
for _name, _n in (("hobc_deblur", 6), ("hobc_deblur_host", 6), ("hobc_deblur_host_async", 6), ("hobc_plan_wait", 1),
                  ("hobc_analysis", 3), ("hobc_synthesis", 3),
                  ("hobc_eigenvalues", 3), ("hobc_gcv", 5), ("hobc_filter_synthesis", 5)):
    getattr(_lib, _name).argtypes = [_vp] * _n
    getattr(_lib, _name).restype = ctypes.c_int
_lib.hobc_gcv_noalloc.argtypes = [ctypes.POINTER(PlanDesc)] + [_vp] * 6
_lib.hobc_gcv_noalloc.restype = ctypes.c_int
_lib.hobc_gcv_noalloc_max_bytes.argtypes = []
_lib.hobc_gcv_noalloc_max_bytes.restype = _sz
class BatchItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 2), ("psf", ctypes.c_int * 2), ("bc_degree", ctypes.c_int)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("L", ctypes.c_int), ("prec", ctypes.c_int), ("n_mu", ctypes.c_int),
                ("gcv_mode", ctypes.c_int)]


_lib.hobc_batch_create.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(BatchItem),
                                   ctypes.POINTER(ctypes.c_double), _vp, ctypes.POINTER(_vp)]
_lib.hobc_batch_create.restype = ctypes.c_int
class FftSchedule(ctypes.Structure):
    _fields_ = [("bc_degree", ctypes.c_int), ("fft_length", ctypes.c_int), ("radix", ctypes.c_int)]


_lib.hobc_batch_create_tuned.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(BatchItem),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(FftSchedule), ctypes.c_int,
                                         _vp, ctypes.POINTER(_vp)]
_lib.hobc_batch_create_tuned.restype = ctypes.c_int
_lib.hobc_fft_length.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.hobc_fft_length.restype = ctypes.c_int
_lib.hobc_batch_destroy.argtypes = [_vp]
_lib.hobc_batch_destroy.restype = None
_lib.hobc_batch_offsets.argtypes = [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]
_lib.hobc_batch_offsets.restype = ctypes.c_int
_lib.hobc_batch_launch_count.argtypes = [_vp]
_lib.hobc_batch_launch_count.restype = ctypes.c_int
_lib.hobc_deblur_batched.argtypes = [_vp] * 6
_lib.hobc_deblur_batched.restype = ctypes.c_int
_lib.hobc_last_launch_count.argtypes = [_vp]
_lib.hobc_last_launch_count.restype = ctypes.c_int
_lib.hobc_status_str.argtypes = [ctypes.c_int]
_lib.hobc_status_str.restype = ctypes.c_char_p
_lib.hobc_last_error.argtypes = []
_lib.hobc_last_error.restype = ctypes.c_char_p
class TcOperand(ctypes.Structure):
    _fields_ = [("hi", _vp), ("lo", _vp), ("ld", ctypes.c_longlong), ("batch_stride", ctypes.c_longlong)]


class TcOutput(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("f32", _vp), ("hi", _vp), ("lo", _vp), ("ld", ctypes.c_longlong),
                ("batch_stride", ctypes.c_longlong), ("rows", ctypes.c_int), ("cols", ctypes.c_int)]


TC_OUT = {"f32": 0, "f32_t": 1, "split": 2, "split_t": 3}
_lib.hobc_tc_gemm.argtypes = [ctypes.POINTER(TcOperand), ctypes.POINTER(TcOperand), ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.POINTER(TcOutput), _vp, _vp]
_lib.hobc_tc_gemm.restype = ctypes.c_int
_lib.hobc_tc_split.argtypes = [_vp, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _vp, _vp,
                               ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _vp]
_lib.hobc_tc_split.restype = ctypes.c_int
for _name in ("hobc_tc_tile_m", "hobc_tc_tile_n", "hobc_tc_tile_k"):
    getattr(_lib, _name).argtypes = []
    getattr(_lib, _name).restype = ctypes.c_int
_lib.hobc_plan_status.argtypes = [_vp]
_lib.hobc_plan_status.restype = ctypes.c_int
_lib.hobc_gcv_binned.argtypes = [_vp] * 6
_lib.hobc_gcv_binned.restype = ctypes.c_int
_lib.hobc_deblur_binned.argtypes = [_vp] * 6
_lib.hobc_deblur_binned.restype = ctypes.c_int
_lib.hobc_gcv_refine.argtypes = [_vp] * 6
_lib.hobc_gcv_refine.restype = ctypes.c_int
_lib.hobc_deblur_refined.argtypes = [_vp] * 6
_lib.hobc_deblur_refined.restype = ctypes.c_int
_lib.hobc_filter_synthesis_mu.argtypes = [_vp] * 5
_lib.hobc_filter_synthesis_mu.restype = ctypes.c_int
_lib.hobc_gcv_exact.argtypes = [_vp] * 5
_lib.hobc_gcv_exact.restype = ctypes.c_int
_lib.hobc_deblur_exact.argtypes = [_vp] * 6
_lib.hobc_deblur_exact.restype = ctypes.c_int
_lib.hobc_features_hist.argtypes = [_vp] * 4
_lib.hobc_features_hist.restype = ctypes.c_int
_lib.hobc_mlp_set_feature_kind.argtypes = [_vp, ctypes.c_int]
_lib.hobc_mlp_set_feature_kind.restype = ctypes.c_int
_lib.hobc_mlp_feature_kind.argtypes = [_vp]
_lib.hobc_mlp_feature_kind.restype = ctypes.c_int
_lib.hobc_mlp_fit_scaling.argtypes = [_vp, _vp, ctypes.c_int]
_lib.hobc_mlp_fit_scaling.restype = ctypes.c_int
_lib.hobc_gcv_exact_search.argtypes = [_vp] * 5
_lib.hobc_gcv_exact_search.restype = ctypes.c_int
_lib.hobc_deblur_exact_search.argtypes = [_vp] * 6
_lib.hobc_deblur_exact_search.restype = ctypes.c_int
_lib.hobc_features.argtypes = [_vp] * 4
_lib.hobc_features.restype = ctypes.c_int
_lib.hobc_deblur_learned.argtypes = [_vp] * 7
_lib.hobc_deblur_learned.restype = ctypes.c_int
_lib.hobc_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.hobc_mlp_create.restype = ctypes.c_int
_lib.hobc_mlp_destroy.argtypes = [_vp]
_lib.hobc_mlp_destroy.restype = None
_lib.hobc_mlp_param_count.argtypes = [_vp]
_lib.hobc_mlp_param_count.restype = ctypes.c_int
_lib.hobc_mlp_last_launch_count.argtypes = [_vp]
_lib.hobc_mlp_last_launch_count.restype = ctypes.c_int
for _name in ("hobc_mlp_set_params", "hobc_mlp_get_params"):
    getattr(_lib, _name).argtypes = [_vp, _vp]
    getattr(_lib, _name).restype = ctypes.c_int
for _name in ("hobc_mlp_save", "hobc_mlp_load"):
    getattr(_lib, _name).argtypes = [_vp, ctypes.c_char_p]
    getattr(_lib, _name).restype = ctypes.c_int
_lib.hobc_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int, _vp]
_lib.hobc_mlp_forward.restype = ctypes.c_int
_lib.hobc_mlp_gradients.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
_lib.hobc_mlp_gradients.restype = ctypes.c_int
_lib.hobc_mlp_train_step.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float, _vp]
_lib.hobc_mlp_train_step.restype = ctypes.c_int

FEATURE_BINS = 64


class HobcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        name = _lib.hobc_status_str(status).decode()
        detail = _lib.hobc_last_error().decode()
        super().__init__(f"{what}: {name}" + (f" ({detail})" if detail else ""))


def _check(status: int, what: str) -> None:
    if status != 0:
        raise HobcError(status, what)


def declared_functions() -> list[str]:
    """Names of the functions declared in include/hobc.h and include/hobc_learned.h."""
    text = ""
    for path in HEADER_PATHS:
        with open(path) as fh:
            text += fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hobc_[a-z_0-9]+)\s*\(", text)))


def library() -> ctypes.CDLL:
    return _lib


def _ptr(x) -> int | None:
    """Device address of a torch tensor (or an int address / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _hptr(a) -> int | None:
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous NumPy array")
    return a.ctypes.data


def make_desc(ndim: int, n, bc_degree: int, n_mu: int, L: str = "I", prec: str = "fp64",
              family: str = "auto", psf_symmetric: bool = False, batch: int = 1,
              psf_per_item: bool = False, psf=None) -> PlanDesc:
    """Fill a hobc_plan_desc (the PSF size is only needed by hobc_plan_create)."""
    n = [int(n)] if np.isscalar(n) else [int(v) for v in n]
    psf = [1] * len(n) if psf is None else ([int(psf)] if np.isscalar(psf) else [int(v) for v in psf])
    d = PlanDesc()
    d.ndim = ndim
    for i in range(2):
        d.n[i] = n[i] if i < len(n) else 0
        d.psf[i] = psf[i] if i < len(psf) else 0
    d.bc_degree = bc_degree
    d.family = FAMILY[family]
    d.psf_symmetric = int(bool(psf_symmetric))
    d.L = SMOOTHING[L]
    d.prec = PRECISION[prec]
    d.n_mu = n_mu
    d.batch = batch
    d.psf_per_item = int(bool(psf_per_item))
    return d


def gcv_noalloc(desc: PlanDesc, ghat, d, mu, gcv, mu_index, stream=None) -> None:
    """hobc_gcv_noalloc: the GCV scan with no plan and no device allocation
    (scratch in the library's static array of gcv_noalloc_max_bytes() bytes)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(_lib.hobc_gcv_noalloc(ctypes.byref(desc), _ptr(ghat), _ptr(d), _ptr(mu), _ptr(gcv), _ptr(mu_index),
                                 _vp(stream)), "hobc_gcv_noalloc")


def tc_tiles():
    """(tile_m, tile_n, tile_k) of the tensor-core GEMM."""
    return _lib.hobc_tc_tile_m(), _lib.hobc_tc_tile_n(), _lib.hobc_tc_tile_k()


def tc_gemm(a_hi, a_lo, a_ld, b_hi, b_lo, b_ld, m, n, k, out, mode="f32", out_lo=None, out_ld=None,
            batch=1, a_bs=0, b_bs=0, out_bs=0, err=None, stream=None) -> None:
    """C = A . B^T on the tensor cores (include/hobc_tc.h); device tensors."""
    A = TcOperand(_ptr(a_hi), _ptr(a_lo), a_ld, a_bs)
    B = TcOperand(_ptr(b_hi), _ptr(b_lo), b_ld, b_bs)
    md = TC_OUT[mode]
    O = TcOutput(md, _ptr(out) if md < 2 else None, _ptr(out) if md >= 2 else None, _ptr(out_lo),
                 out_ld if out_ld is not None else (n if md in (0, 2) else m), out_bs, m, n)
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(_lib.hobc_tc_gemm(ctypes.byref(A), ctypes.byref(B), m, n, k, batch, ctypes.byref(O), _ptr(err),
                             _vp(st)), "hobc_tc_gemm")


def tc_split(src, src_ld, src_bs, rows, cols, hi, lo, ld, bs, rows_padded, batch=1, stream=None) -> None:
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(_lib.hobc_tc_split(_ptr(src), src_ld, src_bs, rows, cols, _ptr(hi), _ptr(lo), ld, bs, rows_padded,
                              batch, _vp(st)), "hobc_tc_split")


def fft_length(bc_degree: int, n: int) -> int:
    """FFT length of a line of n samples under a boundary-condition degree (hobc_fft_length)."""
    return int(_lib.hobc_fft_length(int(bc_degree), int(n)))


def gcv_noalloc_max_bytes() -> int:
    return int(_lib.hobc_gcv_noalloc_max_bytes())


class Plan:
    """A plan of the C ABI: problem geometry, tables and workspace on one GPU."""

    def __init__(self, ndim: int, n, psf, bc_degree: int, mu_grid, L: str = "I",
                 prec: str = "fp64", family: str = "auto", psf_symmetric: bool = False,
                 batch: int = 1, psf_per_item: bool = False, stream=None):
        n = [int(n)] if np.isscalar(n) else [int(v) for v in n]
        psf = [int(psf)] if np.isscalar(psf) else [int(v) for v in psf]
        d = PlanDesc()
        d.ndim = ndim
        for i in range(2):
            d.n[i] = n[i] if i < len(n) else 0
            d.psf[i] = psf[i] if i < len(psf) else 0
        d.bc_degree = bc_degree
        d.family = FAMILY[family]
        d.psf_symmetric = int(bool(psf_symmetric))
        d.L = SMOOTHING[L]
        d.prec = PRECISION[prec]
        mu = np.ascontiguousarray(mu_grid, dtype=np.float64)
        d.n_mu = len(mu)
        d.batch = batch
        d.psf_per_item = int(bool(psf_per_item))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        self._handle = _vp()
        _check(_lib.hobc_plan_create(ctypes.byref(d), mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     _vp(stream), ctypes.byref(self._handle)), "hobc_plan_create")
        self.ndim, self.n, self.psf_shape = ndim, tuple(n[:ndim]), tuple(psf[:ndim])
        self.batch, self.mu_grid, self.prec, self.L = batch, mu, prec, L
        self.psf_per_item = bool(psf_per_item)
        self.family = FAMILY_NAME[_lib.hobc_plan_family(self._handle)]
        spec, cplx, psfn = _sz(), ctypes.c_int(), _sz()
        _check(_lib.hobc_spectrum_size(self._handle, ctypes.byref(spec), ctypes.byref(cplx), ctypes.byref(psfn)),
               "hobc_spectrum_size")
        self.spec_elems, self.spec_complex, self.psf_elems = spec.value, bool(cplx.value), psfn.value

    # geometry helpers -------------------------------------------------------
    @property
    def spectrum_shape(self):
        """Per-item stored spectrum shape (see the spectrum layout in include/hobc.h)."""
        if self.ndim == 1:
            return (self.spec_elems,)
        return (self.spec_elems // self.n[0], self.n[0])

    @property
    def real_dtype(self):
        return np.float64 if self.prec == "fp64" else np.float32

    def status(self) -> None:
        """Synchronise and raise if a bounded tensor-core wait gave up (split_bf16 plans)."""
        _check(_lib.hobc_plan_status(self._handle), "hobc_plan_status")

    @property
    def last_launch_count(self) -> int:
        return _lib.hobc_last_launch_count(self._handle)

    @property
    def gcv_mode(self) -> str:
        return {v: k for k, v in GCV_MODE.items()}[_lib.hobc_plan_gcv_mode(self._handle)]

    def set_gcv_mode(self, mode: str) -> None:
        """'direct' (default) or 'expansion' (include/hobc.h, hobc_plan_set_gcv_mode)."""
        _check(_lib.hobc_plan_set_gcv_mode(self._handle, GCV_MODE[mode]), "hobc_plan_set_gcv_mode")

    def set_host_chunks(self, chunks: int) -> None:
        """Chunks of the host-buffer pipeline (1..8; 0: the default)."""
        _check(_lib.hobc_plan_set_host_chunks(self._handle, int(chunks)), "hobc_plan_set_host_chunks")

    @property
    def gcv_expansion_bound(self) -> float:
        return _lib.hobc_gcv_expansion_bound(self._handle)

    # C ABI calls --------------------------------------------------------------
    def deblur(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_deblur(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(gcv)),
               "hobc_deblur")

    def deblur_host(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_deblur_host(self._handle, _hptr(g), _hptr(psf), _hptr(f), _hptr(mu_index), _hptr(gcv)),
               "hobc_deblur_host")

    def deblur_host_async(self, g, psf, f, mu_index=None, gcv=None) -> None:
        """Queue deblur_host without waiting; the host arrays must stay alive and
        untouched until wait()."""
        _check(_lib.hobc_deblur_host_async(self._handle, _hptr(g), _hptr(psf), _hptr(f), _hptr(mu_index),
                                           _hptr(gcv)), "hobc_deblur_host_async")

    def wait(self) -> None:
        _check(_lib.hobc_plan_wait(self._handle), "hobc_plan_wait")

    def analysis(self, g, ghat) -> None:
        _check(_lib.hobc_analysis(self._handle, _ptr(g), _ptr(ghat)), "hobc_analysis")

    def synthesis(self, c, y) -> None:
        _check(_lib.hobc_synthesis(self._handle, _ptr(c), _ptr(y)), "hobc_synthesis")

    def eigenvalues(self, psf, d) -> None:
        _check(_lib.hobc_eigenvalues(self._handle, _ptr(psf), _ptr(d)), "hobc_eigenvalues")

    def gcv(self, ghat, d, gcv, mu_index) -> None:
        _check(_lib.hobc_gcv(self._handle, _ptr(ghat), _ptr(d), _ptr(gcv), _ptr(mu_index)), "hobc_gcv")

    def filter_synthesis(self, ghat, d, mu_index, f) -> None:
        _check(_lib.hobc_filter_synthesis(self._handle, _ptr(ghat), _ptr(d), _ptr(mu_index), _ptr(f)),
               "hobc_filter_synthesis")

    def gcv_binned(self, ghat, d, mu_index, fell_back=None, k_hat=None) -> None:
        _check(_lib.hobc_gcv_binned(self._handle, _ptr(ghat), _ptr(d), _ptr(mu_index), _ptr(fell_back), _ptr(k_hat)),
               "hobc_gcv_binned")

    def deblur_binned(self, g, psf, f, mu_index=None, fell_back=None) -> None:
        _check(_lib.hobc_deblur_binned(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(fell_back)),
               "hobc_deblur_binned")

    def gcv_refine(self, ghat, d, mu_index, mu, gcv=None) -> None:
        """Refined mu* (double, per problem) from the grid argmin mu_index; gcv: G at mu*."""
        _check(_lib.hobc_gcv_refine(self._handle, _ptr(ghat), _ptr(d), _ptr(mu_index), _ptr(mu), _ptr(gcv)),
               "hobc_gcv_refine")

    def filter_synthesis_mu(self, ghat, d, mu, f) -> None:
        """Filter at mu[item] (double, device) and synthesis."""
        _check(_lib.hobc_filter_synthesis_mu(self._handle, _ptr(ghat), _ptr(d), _ptr(mu), _ptr(f)),
               "hobc_filter_synthesis_mu")

    def gcv_exact(self, ghat, d, gcv, mu_index) -> None:
        """The exact GCV functional of Eq. (eq:gcv) on the grid and its argmin."""
        _check(_lib.hobc_gcv_exact(self._handle, _ptr(ghat), _ptr(d), _ptr(gcv), _ptr(mu_index)), "hobc_gcv_exact")

    def deblur_exact(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_deblur_exact(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(gcv)),
               "hobc_deblur_exact")

    def gcv_exact_search(self, ghat, d, gcv, mu_index) -> None:
        """Grid minimiser of G_ex by the coarse-to-fine search (strides 16, 4, 1)."""
        _check(_lib.hobc_gcv_exact_search(self._handle, _ptr(ghat), _ptr(d), _ptr(gcv), _ptr(mu_index)),
               "hobc_gcv_exact_search")

    def deblur_exact_search(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_deblur_exact_search(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index),
                                             _ptr(gcv)), "hobc_deblur_exact_search")

    def deblur_refined(self, g, psf, f, mu_index=None, mu=None) -> None:
        _check(_lib.hobc_deblur_refined(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(mu)),
               "hobc_deblur_refined")

    def features(self, ghat, d, x) -> None:
        _check(_lib.hobc_features(self._handle, _ptr(ghat), _ptr(d), _ptr(x)), "hobc_features")

    def features_hist(self, ghat, d, x) -> None:
        """Shares of the GCV terms over log10 a (include/hobc_learned.h)."""
        _check(_lib.hobc_features_hist(self._handle, _ptr(ghat), _ptr(d), _ptr(x)), "hobc_features_hist")

    def deblur_learned(self, net: "MLP", g, psf, f, mu=None, fell_back=None) -> None:
        _check(_lib.hobc_deblur_learned(self._handle, net._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu),
                                        _ptr(fell_back)), "hobc_deblur_learned")

    def close(self) -> None:
        if getattr(self, "_handle", None):
            _lib.hobc_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VolumeDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("psf", ctypes.c_int * 3),
        ("bc_degree", ctypes.c_int),
        ("family", ctypes.c_int),
        ("psf_symmetric", ctypes.c_int),
        ("L", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("n_mu", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("psf_per_item", ctypes.c_int),
    ]


_lib.hobc_volume_create.argtypes = [ctypes.POINTER(VolumeDesc), ctypes.POINTER(ctypes.c_double), _vp,
                                    ctypes.POINTER(_vp)]
_lib.hobc_volume_create.restype = ctypes.c_int
_lib.hobc_volume_destroy.argtypes = [_vp]
_lib.hobc_volume_destroy.restype = None
_lib.hobc_volume_spectrum_size.argtypes = [_vp, ctypes.POINTER(_sz), ctypes.POINTER(ctypes.c_int)]
_lib.hobc_volume_spectrum_size.restype = ctypes.c_int
for _name, _n in (("hobc_volume_analysis", 3), ("hobc_volume_synthesis", 3), ("hobc_volume_eigenvalues", 3),
                  ("hobc_volume_gcv", 5), ("hobc_volume_filter_synthesis", 5), ("hobc_volume_deblur", 6)):
    getattr(_lib, _name).argtypes = [_vp] * _n
    getattr(_lib, _name).restype = ctypes.c_int
_lib.hobc_volume_launch_count.argtypes = [_vp]
_lib.hobc_volume_launch_count.restype = ctypes.c_int


class Volume:
    """A plan for 3D arrays [n0][n1][n2] (Sec. 6): tensor-product transforms,
    3D symbol eigenvalues, GCV and filter per spectral entry."""

    def __init__(self, n, psf, bc_degree: int, mu_grid, L: str = "I", prec: str = "fp64", family: str = "auto",
                 psf_symmetric: bool = False, batch: int = 1, psf_per_item: bool = False, stream=None):
        d = VolumeDesc()
        for i in range(3):
            d.n[i] = int(n[i])
            d.psf[i] = int(psf[i])
        d.bc_degree = int(bc_degree)
        d.family = FAMILY[family]
        d.psf_symmetric = int(psf_symmetric)
        d.L = SMOOTHING[L]
        d.prec = PRECISION[prec]
        mus = np.ascontiguousarray(mu_grid, dtype=np.float64)
        d.n_mu = len(mus)
        d.batch = int(batch)
        d.psf_per_item = int(psf_per_item)
        self.desc = d
        self.mu_grid = mus
        h = _vp()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.hobc_volume_create(ctypes.byref(d), mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       _vp(stream), ctypes.byref(h)), "hobc_volume_create")
        self._handle = h
        spec, cplx = _sz(), ctypes.c_int()
        _check(_lib.hobc_volume_spectrum_size(h, ctypes.byref(spec), ctypes.byref(cplx)), "hobc_volume_spectrum_size")
        self.spec_elems = int(spec.value)
        self.spec_complex = bool(cplx.value)

    @property
    def last_launch_count(self) -> int:
        return _lib.hobc_volume_launch_count(self._handle)

    def analysis(self, g, ghat) -> None:
        _check(_lib.hobc_volume_analysis(self._handle, _ptr(g), _ptr(ghat)), "hobc_volume_analysis")

    def synthesis(self, c, y) -> None:
        _check(_lib.hobc_volume_synthesis(self._handle, _ptr(c), _ptr(y)), "hobc_volume_synthesis")

    def eigenvalues(self, psf, d) -> None:
        _check(_lib.hobc_volume_eigenvalues(self._handle, _ptr(psf), _ptr(d)), "hobc_volume_eigenvalues")

    def gcv(self, ghat, d, gcv, mu_index) -> None:
        _check(_lib.hobc_volume_gcv(self._handle, _ptr(ghat), _ptr(d), _ptr(gcv), _ptr(mu_index)), "hobc_volume_gcv")

    def filter_synthesis(self, ghat, d, mu_index, f) -> None:
        _check(_lib.hobc_volume_filter_synthesis(self._handle, _ptr(ghat), _ptr(d), _ptr(mu_index), _ptr(f)),
               "hobc_volume_filter_synthesis")

    def deblur(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_volume_deblur(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(gcv)),
               "hobc_volume_deblur")

    def close(self) -> None:
        if getattr(self, "_handle", None):
            _lib.hobc_volume_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch plan: many 2D problems of uneven sizes, each with its own
    symmetric PSF and boundary degree (1, 2, 3), deblurred in one call."""

    def __init__(self, items, mu_grid, L: str = "lap", prec: str = "fp64", stream=None, schedule=None,
                 gcv_mode: str = "direct"):
        """items: sequence of (n0, n1, psf0, psf1, bc_degree); schedule: optional
        sequence of (bc_degree, fft_length, radix) (hobc_batch_create_tuned);
        gcv_mode: "direct" or "expansion" (FP32)."""
        arr = (BatchItem * len(items))()
        for i, (n0, n1, p0, p1, deg) in enumerate(items):
            arr[i].n[0], arr[i].n[1], arr[i].psf[0], arr[i].psf[1], arr[i].bc_degree = n0, n1, p0, p1, deg
        d = BatchDesc()
        d.count, d.L, d.prec = len(items), SMOOTHING[L], PRECISION[prec]
        d.gcv_mode = GCV_MODE[gcv_mode]
        mu = np.ascontiguousarray(mu_grid, dtype=np.float64)
        d.n_mu = len(mu)
        if stream is None:
            stream = 0
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        self._handle = _vp()
        sched = list(schedule or [])
        sarr = (FftSchedule * max(1, len(sched)))()
        for i, (deg, M, rad) in enumerate(sched):
            sarr[i].bc_degree, sarr[i].fft_length, sarr[i].radix = int(deg), int(M), int(rad)
        _check(_lib.hobc_batch_create_tuned(ctypes.byref(d), arr, mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            sarr, len(sched), _vp(stream), ctypes.byref(self._handle)),
               "hobc_batch_create_tuned")
        self.items, self.mu_grid, self.prec, self.L = list(items), mu, prec, L
        self.schedule, self.gcv_mode = sched, gcv_mode
        io = (_sz * (len(items) + 1))()
        po = (_sz * (len(items) + 1))()
        _check(_lib.hobc_batch_offsets(self._handle, io, po), "hobc_batch_offsets")
        self.img_off = np.array(io[:], dtype=np.int64)
        self.psf_off = np.array(po[:], dtype=np.int64)

    @property
    def last_launch_count(self) -> int:
        return _lib.hobc_batch_launch_count(self._handle)

    def deblur(self, g, psf, f, mu_index=None, gcv=None) -> None:
        _check(_lib.hobc_deblur_batched(self._handle, _ptr(g), _ptr(psf), _ptr(f), _ptr(mu_index), _ptr(gcv)),
               "hobc_deblur_batched")

    def close(self) -> None:
        if getattr(self, "_handle", None):
            _lib.hobc_batch_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The mu-predicting network of include/hobc_learned.h on one GPU."""

    def __init__(self, n_in: int = 2 * FEATURE_BINS, n_hidden: int = 256, stream=None):
        if stream is None:
            stream = 0
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        self._handle = _vp()
        _check(_lib.hobc_mlp_create(n_in, n_hidden, _vp(stream), ctypes.byref(self._handle)), "hobc_mlp_create")
        self.n_in, self.n_hidden = n_in, n_hidden
        self.param_count = _lib.hobc_mlp_param_count(self._handle)

    def fit_scaling(self, x) -> None:
        """Input mean and scale from training features x [rows, n_in] (device)."""
        _check(_lib.hobc_mlp_fit_scaling(self._handle, _ptr(x), int(x.shape[0])), "hobc_mlp_fit_scaling")

    @property
    def feature_kind(self) -> str:
        return {0: "radial", 1: "hist"}[int(_lib.hobc_mlp_feature_kind(self._handle))]

    def set_feature_kind(self, kind: str) -> None:
        """'radial' (hobc_features) or 'hist' (hobc_features_hist)."""
        _check(_lib.hobc_mlp_set_feature_kind(self._handle, {"radial": 0, "hist": 1}[kind]),
               "hobc_mlp_set_feature_kind")

    @property
    def last_launch_count(self) -> int:
        return _lib.hobc_mlp_last_launch_count(self._handle)

    def set_params(self, flat) -> None:
        """flat: float32 host array of param_count + 2 n_in values (parameters, mean, scale)."""
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.param_count + 2 * self.n_in:
            raise ValueError("wrong parameter vector length")
        _check(_lib.hobc_mlp_set_params(self._handle, a.ctypes.data), "hobc_mlp_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.param_count + 2 * self.n_in, dtype=np.float32)
        _check(_lib.hobc_mlp_get_params(self._handle, a.ctypes.data), "hobc_mlp_get_params")
        return a

    def forward(self, x, y) -> None:
        _check(_lib.hobc_mlp_forward(self._handle, _ptr(x), int(x.shape[0]), _ptr(y)), "hobc_mlp_forward")

    def gradients(self, x, t, grad=None, loss=None) -> None:
        _check(_lib.hobc_mlp_gradients(self._handle, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(grad), _ptr(loss)),
               "hobc_mlp_gradients")

    def train_step(self, x, t, lr: float, weight_decay: float = 1e-4, loss=None) -> None:
        _check(_lib.hobc_mlp_train_step(self._handle, _ptr(x), _ptr(t), int(x.shape[0]), lr, weight_decay,
                                        _ptr(loss)), "hobc_mlp_train_step")

    def save(self, path: str) -> None:
        _check(_lib.hobc_mlp_save(self._handle, path.encode()), "hobc_mlp_save")

    def load(self, path: str) -> None:
        _check(_lib.hobc_mlp_load(self._handle, path.encode()), "hobc_mlp_load")

    def close(self) -> None:
        if getattr(self, "_handle", None):
            _lib.hobc_mlp_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_params(p: dict, mean, scale) -> np.ndarray:
    """Flat float32 vector (W1, b1, W2, b2, w3, b3, mean, scale) in the ABI's layout."""
    parts = [p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], p["b3"], mean, scale]
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts]).astype(np.float32)


def unpack_params(flat, n_in: int, n_hidden: int):
    """Inverse of pack_params: (params dict, mean, scale) as float64 arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    sizes = [("W1", (n_hidden, n_in)), ("b1", (n_hidden,)), ("W2", (n_hidden, n_hidden)), ("b2", (n_hidden,)),
             ("w3", (n_hidden,)), ("b3", (1,))]
    out, o = {}, 0
    for k, shp in sizes:
        cnt = int(np.prod(shp))
        out[k] = flat[o:o + cnt].reshape(shp)
        o += cnt
    return out, flat[o:o + n_in], flat[o + n_in:o + 2 * n_in]
