"""The tensor-core building blocks (tcgen05.mma kind::tf32 with FP32
accumulation in tensor memory, K-major 128-byte-swizzled operands, the 3-term
TF32 split) through the library's probe: one 128 x N tile D = A B^T against the
FP64 product of the same FP32 inputs.

Bounds, from the arithmetic.  A TF32 operand keeps 10 explicit mantissa bits:
read from an FP32 value it is off by less than 2^-10 of it (truncation, the
worst case), so a plain product is off by <= (2^-9 + 2^-20) |a||b|.  With the
split x = hi + lo + e (hi, lo rounded to nearest TF32: |x - hi| <= 2^-11 |x|,
|e| <= 2^-22 |x|), hi*hi' + hi*lo' + lo*hi' misses x*x' by
lo*lo' + e-terms <= 2^-21 (1 + 2^-10) |x||x'| (+ 2^-43 terms).  Products of TF32
values are exact in FP32; the 3k (or k) products of an entry are added in FP32,
each addition off by at most one FP32 ulp (2^-23) of a partial sum bounded by
sum |a||b| (no rounding mode assumed)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


def _inputs(n_cols, k, seed, wide):
    g = torch.Generator().manual_seed(seed)
    A = torch.rand(128, k, generator=g, dtype=torch.float64) * 2 - 1
    B = torch.rand(n_cols, k, generator=g, dtype=torch.float64) * 2 - 1
    if wide:  # magnitudes over 2^-12 .. 2^12: exercises the exponent handling of the split
        A = A * torch.pow(2.0, torch.randint(-12, 13, A.shape, generator=g).double())
        B = B * torch.pow(2.0, torch.randint(-12, 13, B.shape, generator=g).double())
    return A.float(), B.float()


@pytest.mark.parametrize("n_cols,k,split,wide", [(128, 32, 0, False), (256, 64, 0, False), (16, 32, 0, False),
                                                 (128, 64, 1, False), (256, 32, 1, True), (48, 64, 1, True)])
def test_umma_tile_against_fp64_product(n_cols, k, split, wide):
    A, B = _inputs(n_cols, k, seed=700 + n_cols + k + split, wide=wide)
    D = tk.tk_umma_probe(A.cuda(), B.cuda(), split=bool(split)).double().cpu().numpy()
    a, b = A.double().numpy(), B.double().numpy()
    ref = a @ b.T
    absd = np.abs(a) @ np.abs(b).T
    per_product = 2.0 ** -21 * (1 + 2.0 ** -10) if split else 2.0 ** -9 + 2.0 ** -20
    adds = (3 if split else 1) * k
    tol = (per_product + adds * 2.0 ** -23) * absd
    err = np.abs(D - ref)
    print(f"\nN={n_cols} k={k} split={split}: max err/tol {float(np.max(err / tol)):.3e}, "
          f"max err/sum|ab| {float(np.max(err / absd)):.3e}")
    assert np.all(np.isfinite(D))
    assert np.all(err <= tol), float(np.max(err / tol))
