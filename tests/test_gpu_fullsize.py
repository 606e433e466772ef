"""Parity at the workload sizes, in the launch configuration the benchmark uses:
sampled entries of the built tensor against the oracle one by one, and whole
contractions against the linear-kernel closed form K[a^{m-1}] = X (X^T a)^{m-1}
(which holds at any size)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, UBF16, accumulation_depth, as_f64, build_rel, max_warp_triangles

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")

U = {"f32": U32, "bf16": UBF16}


def _workloads():
    c2 = synth.full_fp32()
    c3 = synth.higher_order()
    c4 = synth.nystrom_bf16(n_train=3000, n_test=10)  # landmark rows share the AR(1) law
    idx = oracle.nystrom_select(3000, 600, c4["select_seed"])
    return [("full_fp32", c2["X"], 4, "f32"), ("higher_order", c3["X"], 6, "f32"),
            ("nystrom_bf16", c4["X_train"][idx], 4, "bf16")]


@pytest.fixture(scope="module", params=_workloads(), ids=lambda w: w[0])
def built(request):
    name, X, m, storage = request.param
    Xd = torch.tensor(X, device="cuda")
    K = tk.tk_build_packed(Xd, m, storage=storage)
    torch.cuda.synchronize()
    yield name, X, m, storage, K
    del K
    torch.cuda.empty_cache()


def test_sampled_entries(built):
    name, X, m, storage, K = built
    n, d = X.shape
    N = tk.tk_packed_size(m, n)
    rng = np.random.default_rng(42)
    offs = np.unique(np.concatenate([rng.integers(0, N, size=1500), [0, 1, N - 2, N - 1]]))
    got = as_f64(K[torch.tensor(offs, device="cuda")])
    for o, g in zip(offs, got):
        ref = oracle.build(X, m, int(o), int(o) + 1)[0]
        rabs = oracle.build(np.abs(X), m, int(o), int(o) + 1)[0]
        tol = build_rel(d, m, storage, tk.tk_build_uses_tensor_cores(d, storage)) * rabs
        if storage == "bf16":
            tol += UBF16 * (abs(g) + tol)
        assert abs(g - ref) <= tol, (int(o), g, ref)


def test_contraction_closed_form(built):
    name, X, m, storage, K = built
    n, d = X.shape
    for salt, scale in ((1, 1.0), (2, 0.01)):
        a = synth.alpha_like(n, salt=salt, scale=scale)
        G, S = tk.tk_contract(K, m, n, torch.tensor(a, device="cuda"))
        u = X.T @ a
        g_ref = X @ u ** (m - 1)
        S_ref = float(np.sum(u ** m))
        uabs = np.abs(X).T @ np.abs(a)
        g_abs = np.abs(X) @ uabs ** (m - 1)
        S_abs = float(np.sum(uabs ** m))
        # storage rounding + build accumulation + contraction accumulation
        rel = build_rel(d, m, storage, tk.tk_build_uses_tensor_cores(d, storage)) + \
            1.01 * accumulation_depth(n, max_warp_triangles(m, n, storage)) * U32
        if storage == "bf16":
            rel += 1.01 * U[storage]
        err = np.abs(G.cpu().numpy() - g_ref)
        assert np.all(err <= rel * g_abs), float(np.max(err / (rel * g_abs)))
        assert abs(float(S[0]) - S_ref) <= rel * S_abs
    assert tk.tk_status_read(tk.workspace(m, n)) == 0


def test_hvp_closed_form(built):
    name, X, m, storage, K = built
    n, d = X.shape
    a = synth.alpha_like(n, salt=5)
    v = synth.alpha_like(n, salt=6)
    HV, _ = tk.tk_contract(K, m, n, torch.tensor(a, device="cuda"), r=m - 2, V=torch.tensor(v, device="cuda"))
    u = X.T @ a
    hv_ref = X @ (u ** (m - 2) * (X.T @ v))
    uabs = np.abs(X).T @ np.abs(a)
    hv_abs = np.abs(X) @ (uabs ** (m - 2) * (np.abs(X).T @ np.abs(v)))
    rel = build_rel(d, m, storage, tk.tk_build_uses_tensor_cores(d, storage)) + \
        1.01 * 2 * accumulation_depth(n, max_warp_triangles(m, n, storage, dual=True)) * U32
    if storage == "bf16":
        rel += 1.01 * U[storage]
    err = np.abs(HV.cpu().numpy() - hv_ref)
    assert np.all(err <= rel * hv_abs), float(np.max(err / (rel * hv_abs)))


def test_dexter_shaped_build_and_contraction():
    # few points, very many sparse features: the build is d-heavy (2d flops per entry)
    p = synth.dexter_like()
    m, X = p["m"], p["X"]
    n, d = X.shape
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f32")
    a = synth.alpha_like(n, salt=31)
    G, S = tk.tk_contract(K, m, n, torch.tensor(a, device="cuda"))
    u = X.T @ a
    g_ref = X @ u ** (m - 1)
    uabs = np.abs(X).T @ np.abs(a)
    g_abs = np.abs(X) @ uabs ** (m - 1)
    rel = build_rel(d, m, "f32", tk.tk_build_uses_tensor_cores(d, "f32")) + \
        1.01 * accumulation_depth(n, max_warp_triangles(m, n, "f32")) * U32
    err = np.abs(G.cpu().numpy() - g_ref)
    assert np.all(err <= rel * g_abs + 1e-30), float(np.max(err / (rel * g_abs + 1e-30)))
    assert abs(float(S[0]) - float(np.sum(u ** m))) <= rel * float(np.sum(uabs ** m))
