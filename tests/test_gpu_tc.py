"""The tensor-core GEMM of include/hobc_tc.h against an exact FP64 evaluation
of the same split products.

Inputs are random FP32 matrices; the test splits them the way the kernels do
(hi = bf16(x), lo = bf16(x - hi), oracle/mlp_oracle.bf16_round) and forms
hi.hi + hi.lo + lo.hi in FP64, so what remains is the kernel's FP32
accumulation: |C - ref| <= K 2^-23 (|A| |B|^T) per entry.  The split itself is
checked against the same rounding bit for bit, and the whole product against
the unsplit one within the header's bound (2^-14 + K 2^-24) (|A| |B|^T).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_0906_2704_gb300 import hobc  # noqa: E402


def _split(x):
    hi = M.bf16_round(x)
    lo = M.bf16_round((x.astype(np.float32) - hi.astype(np.float32)).astype(np.float32))
    return hi, lo


def _bf16_dev(a):
    """float64 array holding bf16 values -> device bfloat16 tensor (exact)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def _pad(x, rows, cols):
    out = np.zeros(x.shape[:-2] + (rows, cols), dtype=x.dtype)
    out[..., :x.shape[-2], :x.shape[-1]] = x
    return out


@pytest.mark.parametrize("mode", ["f32", "f32_t", "split", "split_t"])
@pytest.mark.parametrize("m,n,k,batch,shared_b", [(128, 256, 64, 1, False), (200, 300, 128, 1, False),
                                                  (70, 40, 64, 3, True), (256, 512, 1024, 2, False)])
def test_tc_gemm_matches_exact_split_products(m, n, k, batch, shared_b, mode):
    tm, tn, tk = hobc.tc_tiles()
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.standard_normal((batch, m, k)).astype(np.float32)
    B = rng.standard_normal((1 if shared_b else batch, n, k)).astype(np.float32)
    mp, np_, kp = -(-m // tm) * tm, -(-n // tn) * tn, -(-k // tk) * tk
    ah, al = _split(A.astype(np.float64))
    bh, bl = _split(B.astype(np.float64))
    d_ah, d_al = _bf16_dev(_pad(ah, mp, kp)), _bf16_dev(_pad(al, mp, kp))
    d_bh, d_bl = _bf16_dev(_pad(bh, np_, kp)), _bf16_dev(_pad(bl, np_, kp))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    t = mode.endswith("_t")
    shape = (batch, n, m) if t else (batch, m, n)
    if mode.startswith("f32"):
        out = torch.full(shape, np.nan, dtype=torch.float32, device="cuda")
        out_lo = None
    else:
        out = torch.zeros(shape, dtype=torch.bfloat16, device="cuda")
        out_lo = torch.zeros(shape, dtype=torch.bfloat16, device="cuda")
    hobc.tc_gemm(d_ah, d_al, kp, d_bh, d_bl, kp, m, n, kp, out, mode=mode, out_lo=out_lo, batch=batch,
                 a_bs=mp * kp, b_bs=0 if shared_b else np_ * kp, out_bs=m * n, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    Bb = np.broadcast_to(bh, (batch, n, k)), np.broadcast_to(bl, (batch, n, k))
    ref = ah @ Bb[0].transpose(0, 2, 1) + ah @ Bb[1].transpose(0, 2, 1) + al @ Bb[0].transpose(0, 2, 1)
    mag = np.abs(A.astype(np.float64)) @ np.abs(np.broadcast_to(B, (batch, n, k)).astype(np.float64)).transpose(0, 2, 1)
    if mode.startswith("f32"):
        got = out.cpu().numpy().astype(np.float64)
    else:
        got = out.float().cpu().numpy().astype(np.float64) + out_lo.float().cpu().numpy().astype(np.float64)
    if t:
        got = got.transpose(0, 2, 1)
    tol = k * 2.0 ** -23 * mag + (0 if mode.startswith("f32") else 2.0 ** -16 * np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol), f"max excess {np.max(np.abs(got - ref) - tol):.3e}"
    # against the unsplit product: the header's bound
    exact = A.astype(np.float64) @ np.broadcast_to(B, (batch, n, k)).astype(np.float64).transpose(0, 2, 1)
    bound = (2.0 ** -14 + k * 2.0 ** -24) * mag + (0 if mode.startswith("f32") else 2.0 ** -16 * np.abs(exact))
    assert np.all(np.abs(got - exact) <= bound)


def test_tc_split_matches_bf16_rounding():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal((2, 37, 50)) * 10.0 ** rng.uniform(-3, 3, (2, 37, 50))).astype(np.float32)
    src = torch.from_numpy(x).cuda()
    hi = torch.full((2, 64, 64), 7.0, dtype=torch.bfloat16, device="cuda")
    lo = torch.full_like(hi, 7.0)
    hobc.tc_split(src, 50, 37 * 50, 37, 50, hi, lo, 64, 64 * 64, 64, batch=2)
    eh, el = _split(x.astype(np.float64))
    h, l = hi.float().cpu().numpy(), lo.float().cpu().numpy()
    assert np.array_equal(h[:, :37, :50], eh) and np.array_equal(l[:, :37, :50], el)
    assert np.all(h[:, 37:, :] == 0) and np.all(h[:, :, 50:] == 0) and np.all(l[:, 37:, :] == 0)


def test_tc_gemm_rejects_bad_shapes():
    t = torch.zeros(64 * 128, dtype=torch.bfloat16, device="cuda")
    out = torch.zeros(128 * 256, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(hobc.HobcError):       # K not a multiple of the tile
        hobc.tc_gemm(t, t, 64, t, t, 64, 128, 256, 48, out, err=err)
    with pytest.raises(hobc.HobcError):       # rows not 16-byte aligned
        hobc.tc_gemm(t, t, 60, t, t, 64, 128, 256, 64, out, err=err)
