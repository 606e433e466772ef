"""One-pass batched contraction (B > 1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, as_f64, batched_accumulation_depth, batched_bound, build_rel, round_storage, \
    tc_batched_bound, tc_batched_rel

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,d,B", [(4, 37, 4, 5), (4, 70, 3, 70), (6, 19, 3, 33), (2, 150, 3, 64), (4, 80, 2, 200),
                                     (3, 300, 2, 130), (2, 520, 2, 3)])
def test_batched_contraction_matches_oracle(m, n, d, B, storage):
    X = synth.small_problem(m, n, d, salt=800 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = synth.alpha_like(n, salt=801, batch=B)
    G, S = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(A, device="cuda"))
    G = G.cpu().numpy()
    S = S.cpu().numpy()
    pick = sorted(set([0, B - 1, B // 2, min(B - 1, 33), min(B - 1, 64)]))
    for b in pick:
        g_ref, S_ref = oracle.contract(Kr, A[b], m)
        g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(A[b]), m)
        tol = batched_bound(g_abs, storage, n, m)
        assert np.all(np.abs(G[b] - g_ref) <= tol), (b, float(np.max(np.abs(G[b] - g_ref) / tol)))
        assert abs(S[b] - S_ref) <= float(batched_bound(np.array([S_abs]), storage, n, m)[0])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,d,B", [(4, 41, 3, 9), (6, 17, 3, 40), (3, 300, 2, 64)])
def test_batched_hvp_matches_oracle(m, n, d, B, storage):
    X = synth.small_problem(m, n, d, salt=820 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = synth.alpha_like(n, salt=821, batch=B)
    V = synth.alpha_like(n, salt=822, batch=B)
    HV, _ = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(A, device="cuda"), r=m - 2,
                           V=torch.tensor(V, device="cuda"))
    HV = HV.cpu().numpy()
    for b in sorted(set([0, B // 2, B - 1])):
        ref = oracle.hvp(Kr, A[b], V[b], m)
        hab = oracle.hvp(np.abs(Kr), np.abs(A[b]), np.abs(V[b]), m)
        tol = batched_bound(hab, storage, n, m, dual=True)
        assert np.all(np.abs(HV[b] - ref) <= tol), (b, float(np.max(np.abs(HV[b] - ref) / tol)))


@pytest.fixture(scope="module")
def path_tensor():
    """The batched workload's packed tensor: m = 4 over n' = 300 landmarks of
    20,000 points (d = 80), FP32 storage (344,291,325 entries)."""
    p = synth.batched_path()
    idx = oracle.nystrom_select(p["X"].shape[0], p["n_prime"], p["select_seed"])
    X = p["X"][idx]
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), p["m"], storage="f32")
    torch.cuda.synchronize()
    yield p["m"], X, K
    del K
    torch.cuda.empty_cache()


def test_batched_full_width_against_closed_form(path_tensor):
    # every element of all 512 vectors of one pass, against the linear
    # kernel's closed forms K[a^3] = X (X^T a)^3, K[a^4] = sum (X^T a)^4 and
    # K[a^2, v] = X ((X^T a)^2 * X^T v); bound: the build's accumulation and
    # storage rounding plus the batched kernel's depth, times sum |terms|
    m, X, K = path_tensor
    n, d = X.shape
    B = 512
    A = synth.alpha_like(n, salt=830, batch=B)
    V = synth.alpha_like(n, salt=831, batch=B)
    Ad, Vd = torch.tensor(A, device="cuda"), torch.tensor(V, device="cuda")
    tk.tk_batched_set_config(tensor_cores=-1)  # the SIMT batched kernel (the tensor-core pass has its own test)
    try:
        cfg = tk.tk_batched_get_config(m, n, "f32", False, B)
        assert cfg["vpl"] > 0 and cfg["tensor_cores"] == 0  # the SIMT kernel serves this shape in one launch
        G, S = tk.tk_contract(K, m, n, Ad)
        HV, _ = tk.tk_contract(K, m, n, Ad, r=m - 2, V=Vd)
    finally:
        tk.tk_batched_set_config(reset=True)
    G, S, HV = G.cpu().numpy(), S.cpu().numpy(), HV.cpu().numpy()
    U = A @ X                       # B x d: X^T a_b
    Ua = np.abs(A) @ np.abs(X)
    W = V @ X
    Wa = np.abs(V) @ np.abs(X)
    g_ref, g_abs = (U ** 3) @ X.T, (Ua ** 3) @ np.abs(X).T
    S_ref, S_abs = np.sum(U ** 4, axis=1), np.sum(Ua ** 4, axis=1)
    h_ref, h_abs = (U ** 2 * W) @ X.T, (Ua ** 2 * Wa) @ np.abs(X).T
    e_build = build_rel(d, m, "f32", tk.tk_build_uses_tensor_cores(d, "f32"))
    rel = e_build + 1.01 * batched_accumulation_depth(n, m) * U32
    rel_h = e_build + 1.01 * batched_accumulation_depth(n, m, dual=True) * U32
    assert np.all(np.abs(G - g_ref) <= rel * g_abs), float(np.max(np.abs(G - g_ref) / (rel * g_abs)))
    assert np.all(np.abs(S - S_ref) <= rel * S_abs)
    assert np.all(np.abs(HV - h_ref) <= rel_h * h_abs), float(np.max(np.abs(HV - h_ref) / (rel_h * h_abs)))


@pytest.fixture
def tensor_cores():
    """Route batched K[a^{m-1}] passes to the tensor-core kernel wherever it covers them."""
    tk.tk_batched_set_config(tensor_cores=1)
    yield
    tk.tk_batched_set_config(reset=True)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,d,B,vdt", [(4, 70, 3, 130, torch.float64), (3, 130, 2, 128, torch.float32),
                                         (4, 33, 4, 256, torch.float64), (2, 150, 3, 200, torch.float64),
                                         (4, 101, 3, 300, torch.float32), (5, 24, 3, 129, torch.float64),
                                         (4, 5, 2, 128, torch.float64)])
def test_tensor_core_contraction_matches_oracle(tensor_cores, m, n, d, B, vdt, storage):
    # the tcgen05 pass (TF32 with the 3-term split, FP32 and FP64 partials)
    # element by element against the oracle, for vectors of every slice of
    # 128, including a partial last slice
    X = synth.small_problem(m, n, d, salt=840 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = synth.alpha_like(n, salt=841, batch=B)
    assert tk.tk_batched_get_config(m, n, storage, False, B)["tensor_cores"] == 1
    Ad = torch.tensor(A, device="cuda").to(vdt)
    a_used = Ad.double().cpu().numpy()
    G, S = tk.tk_contract(Kt.cuda(), m, n, Ad)
    G, S = G.double().cpu().numpy(), S.cpu().numpy()
    assert np.all(np.isfinite(G)) and np.all(np.isfinite(S))
    pick = sorted(set([0, 1, 127, min(B - 1, 128), B // 2, B - 2, B - 1]))
    for b in pick:
        g_ref, S_ref = oracle.contract(Kr, a_used[b], m)
        g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a_used[b]), m)
        tol = tc_batched_bound(g_abs, n, m)
        if vdt == torch.float32:
            tol = tol + U32 * np.abs(g_ref)  # G rounded to the vector type
        assert np.all(np.abs(G[b] - g_ref) <= tol), (b, float(np.max(np.abs(G[b] - g_ref) / tol)))
        assert abs(S[b] - S_ref) <= float(tc_batched_bound(np.array([S_abs]), n, m)[0]), b


def test_tensor_core_full_width_against_closed_form(path_tensor, tensor_cores):
    # all 512 vectors of the batched workload (m = 4, n' = 300, FP32) in one
    # tensor-core pass against the closed forms, and the time of one pass
    # beside the SIMT batched kernel's
    m, X, K = path_tensor
    n, d = X.shape
    B = 512
    A = synth.alpha_like(n, salt=850, batch=B)
    Ad = torch.tensor(A, device="cuda")
    assert tk.tk_batched_get_config(m, n, "f32", False, B)["tensor_cores"] == 1
    G, S = tk.tk_contract(K, m, n, Ad)
    G, S = G.cpu().numpy(), S.cpu().numpy()
    U, Ua = A @ X, np.abs(A) @ np.abs(X)
    g_ref, g_abs = (U ** 3) @ X.T, (Ua ** 3) @ np.abs(X).T
    S_ref, S_abs = np.sum(U ** 4, axis=1), np.sum(Ua ** 4, axis=1)
    rel = build_rel(d, m, "f32", tk.tk_build_uses_tensor_cores(d, "f32")) + 2.0 * tc_batched_rel(n, m)
    err = np.abs(G - g_ref) / g_abs
    print(f"\ntensor-core pass: max |err| / sum|terms| = {float(np.max(err)):.3e} (bound {rel:.3e})")
    assert np.all(np.abs(G - g_ref) <= rel * g_abs), float(np.max(np.abs(G - g_ref) / (rel * g_abs)))
    assert np.all(np.abs(S - S_ref) <= rel * S_abs)
    times = {}
    for mode in (1, -1):
        tk.tk_batched_set_config(tensor_cores=mode)
        tk.tk_contract(K, m, n, Ad)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            tk.tk_contract(K, m, n, Ad)
        e1.record()
        e1.synchronize()
        times[mode] = e0.elapsed_time(e1) / 3
    print(f"one B=512 pass: tensor cores {times[1]:.2f} ms, SIMT batched kernel {times[-1]:.2f} ms")
