"""GPU parity of the packed build against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, U64, UBF16, as_f64, tc_build_rel

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.fixture(params=["simt", "tensor_cores"])
def path(request):
    """Which kernel builds FP32 / BF16 storage (FP64 always takes the SIMT build)."""
    tk.tk_build_set_config(1 if request.param == "tensor_cores" else -1)
    yield request.param
    assert tk.tk_build_status() == tk.TK_OK
    tk.tk_build_set_config(0)


def linear_rel(d, m, storage, path):
    """Relative bound of the linear build: the SIMT build's FP32 (or FP64) sum of
    d products of m factors, gamma_{d+m+2}; the tensor-core build's arithmetic
    (gpu_util.tc_build_rel)."""
    if storage != "f64" and path == "tensor_cores":
        return tc_build_rel(d, m)
    u = U64 if storage == "f64" else U32
    return 1.01 * (d + m + 2) * u


def build_bound(Kabs, d, m, storage, Khat=None, path="simt"):
    """|K_computed - K_exact| <= rel * sum_k prod_j |x|; BF16 adds the final rounding."""
    acc = linear_rel(d, m, storage, path) * Kabs
    if storage == "bf16":
        return acc + UBF16 * (np.abs(Khat) + acc)
    return acc + 1e-300


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,d", [(2, 1, 1), (2, 70, 3), (4, 1, 2), (4, 5, 3), (4, 64, 17),
                                   (4, 65, 16), (4, 130, 5), (6, 21, 4), (8, 7, 3), (3, 40, 2)])
def test_build_matches_oracle(m, n, d, storage, path):
    X = synth.small_problem(m, n, d, salt=31 * n + d)
    K_ref = oracle.build(X, m)
    K_abs = oracle.build(np.abs(X), m)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage=storage)
    Kh = as_f64(K)
    err = np.abs(Kh - K_ref)
    tol = build_bound(K_abs, d, m, storage, Kh, path)
    assert np.all(err <= tol), float(np.max(err / tol))


def test_build_ranges_are_bit_identical(path):
    m, n, d = 4, 70, 6
    X = torch.tensor(synth.small_problem(m, n, d, salt=3), device="cuda")
    full = tk.tk_build_packed(X, m, storage="f32")
    N = full.numel()
    cuts = [0, 1, 999, 40000, N - 3, N]
    parts = [tk.tk_build_packed(X, m, storage="f32", off_lo=lo, off_hi=hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
    assert torch.equal(torch.cat(parts), full)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("feat,deg", [("poly", 2), ("poly", 3), ("exp", 1)])
def test_build_feature_maps(feat, deg, storage, path):
    # The epilogue maps the accumulated linear sum s_hat (|s_hat - s| <= e, the
    # linear build's bound) through t -> t^deg (deg - 1 rounded products) or
    # t -> exp(t) (CUDA's exp: at most 2 ulp in FP32, 1 ulp in FP64), then
    # rounds to the storage type.  Propagated:
    #   power: |s_hat^deg - s^deg| <= deg (|s| + e)^(deg-1) e,  plus (deg-1) u |K|
    #   exp:   |exp(s_hat) - exp(s)| <= exp(s + e)(exp(e) - 1),  plus 4 u |K|
    m, n, d = 4, 12, 3
    X = 0.5 * synth.small_problem(m, n, d, salt=17)
    code = oracle.FEAT_POLY if feat == "poly" else oracle.FEAT_EXP
    K_ref = oracle.build(X, m, feat=code, degree=deg)
    s_lin = oracle.build(X, m)
    K_abs = oracle.build(np.abs(X), m)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage=storage, feat=feat, degree=deg)
    Kh = as_f64(K)
    u = U64 if storage == "f64" else U32
    e = linear_rel(d, m, storage, path) * K_abs
    if feat == "poly":
        tol = deg * (np.abs(s_lin) + e) ** (deg - 1) * e + 1.01 * (deg - 1) * u * np.abs(K_ref)
    else:
        tol = np.exp(s_lin + e) * np.expm1(e) + 4 * u * np.abs(K_ref)
    if storage == "bf16":
        tol = tol + UBF16 * (np.abs(Kh) + tol)
    tol = tol + 1e-300
    err = np.abs(Kh - K_ref)
    assert np.all(err <= tol), float(np.max(err / tol))
