"""GPU parity of the packed contraction kernels against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import as_f64, contraction_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")

# (m, n, d): one-entry rows, sizes that span several 32-column chunks with a
# ragged tail, every order the library supports
CASES = [(2, 1, 3), (2, 37, 4), (2, 300, 3), (4, 1, 2), (4, 2, 3), (4, 5, 3), (4, 33, 4),
         (4, 37, 5), (4, 64, 3), (4, 97, 4), (6, 3, 2), (6, 23, 3), (8, 9, 2), (3, 20, 3),
         (5, 12, 3)]


def _setup(m, n, d, storage, salt):
    X = synth.small_problem(m, n, d, salt=salt)
    K64 = oracle.build(X, m)
    Kt = round_storage(K64, storage)
    Kr = as_f64(Kt)  # the exact values the GPU sees
    return X, Kr, Kt.cuda()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,d", CASES)
def test_contract_matches_oracle(m, n, d, storage):
    X, Kr, Kd = _setup(m, n, d, storage, salt=1000 * m + n)
    a = synth.alpha_like(n, salt=n + 7)
    g_ref, S_ref = oracle.contract(Kr, a, m)
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a), m)
    for vdt in (torch.float64, torch.float32):
        A = torch.tensor(a, dtype=vdt, device="cuda")
        a_used = A.double().cpu().numpy()
        if vdt == torch.float32:
            g_ref, S_ref = oracle.contract(Kr, a_used, m)
            g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a_used), m)
        G, S = tk.tk_contract(Kd, m, n, A)
        torch.cuda.synchronize()
        g = G.double().cpu().numpy()
        tol = contraction_bound(n, g_abs, storage, m)
        if vdt == torch.float32:
            tol = tol + 2.0 ** -24 * np.abs(g_ref)  # output rounded to FP32
        err = np.abs(g - g_ref)
        assert np.all(err <= tol), (np.max(err / tol), storage, vdt)
        if storage == "f64" and vdt == torch.float64:
            # the stated FP64 target: relative 1e-10
            assert np.allclose(g, g_ref, rtol=1e-10, atol=1e-10 * np.max(np.abs(g_ref)))
            assert float(S[0]) == pytest.approx(S_ref, rel=1e-10, abs=1e-10 * S_abs)
        assert abs(float(S[0]) - S_ref) <= float(contraction_bound(n, np.array([S_abs]), storage, m)[0])
    assert tk.tk_status_read(tk.workspace(m, n)) == 0


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,d", [(2, 37, 3), (4, 5, 2), (4, 41, 4), (6, 17, 3), (4, 1, 2)])
def test_hvp_matches_oracle(m, n, d, storage):
    X, Kr, Kd = _setup(m, n, d, storage, salt=77 * m + n)
    a = synth.alpha_like(n, salt=3 * n)
    v = synth.alpha_like(n, salt=3 * n + 1)
    hv_ref = oracle.hvp(Kr, a, v, m)
    hv_abs = oracle.hvp(np.abs(Kr), np.abs(a), np.abs(v), m)
    A = torch.tensor(a, device="cuda")
    V = torch.tensor(v, device="cuda")
    HV, _ = tk.tk_contract(Kd, m, n, A, r=m - 2, V=V)
    hv = HV.cpu().numpy()
    tol = 2 * contraction_bound(n, hv_abs, storage, m, dual=True)
    assert np.all(np.abs(hv - hv_ref) <= tol), np.max(np.abs(hv - hv_ref) / tol)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batch_and_objective(storage):
    m, n, d, B = 4, 29, 3, 3
    X, Kr, Kd = _setup(m, n, d, storage, salt=5)
    A = synth.alpha_like(n, salt=9, batch=B)
    y = synth.alpha_like(n, salt=10)
    lam = np.array([0.1, 1.0, 3.0])
    At = torch.tensor(A, device="cuda")
    G, S = tk.tk_contract(Kd, m, n, At)
    F, grad, gn = tk.tk_objective(Kd, m, n, At, torch.tensor(y, device="cuda"),
                                  torch.tensor(lam, device="cuda"))
    for b in range(B):
        g_ref, S_ref = oracle.contract(Kr, A[b], m)
        g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(A[b]), m)
        tol = contraction_bound(n, g_abs, storage, m)
        assert np.all(np.abs(G[b].cpu().numpy() - g_ref) <= tol)
        F_ref = oracle.dual_objective(S_ref, A[b], y, lam[b], m)
        gr_ref = oracle.dual_gradient(g_ref, A[b], y, lam[b])
        assert np.all(np.abs(grad[b].cpu().numpy() - gr_ref) <= tol + 1e-13 * np.abs(gr_ref))
        assert float(F[b]) == pytest.approx(F_ref, abs=float(contraction_bound(n, np.array([S_abs]), storage, m)[0]) / m + 1e-12 * abs(F_ref))
        assert float(gn[b]) == pytest.approx(np.linalg.norm(gr_ref), abs=np.linalg.norm(tol) + 1e-12)


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_range_shards_add_up(storage):
    m, n, d = 4, 45, 3
    X, Kr, Kd = _setup(m, n, d, storage, salt=11)
    a = synth.alpha_like(n, salt=12)
    A = torch.tensor(a, device="cuda")
    N = tk.tk_packed_size(m, n)
    cuts = [0] + [tk.tk_row_align(m, n, c) for c in (N // 5, N // 2, (4 * N) // 5)] + [N]
    G = torch.zeros(n, dtype=torch.float64, device="cuda")
    S = 0.0
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        Kpart = Kd[lo:hi].clone()  # a shard in its own (aligned) allocation
        g, s = tk.tk_contract(Kpart, m, n, A, off_lo=lo, off_hi=hi)
        g_ref, s_ref = oracle.contract(Kr[lo:hi], a, m, lo=lo)
        g_abs, _ = oracle.contract(np.abs(Kr[lo:hi]), np.abs(a), m, lo=lo)
        assert np.all(np.abs(g.cpu().numpy() - g_ref) <= contraction_bound(n, g_abs, storage, m, lo, hi))
        G += g
        S += float(s[0])
    g_ref, S_ref = oracle.contract(Kr, a, m)
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a), m)
    assert np.all(np.abs(G.cpu().numpy() - g_ref) <= 4 * contraction_bound(n, g_abs, storage, m))


def test_rejects_bad_arguments():
    m, n = 4, 10
    K = torch.zeros(tk.tk_packed_size(m, n), dtype=torch.float32, device="cuda")
    A = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(tk.TKError):
        tk.tk_contract(K, m, n, A, r=1)  # r must be m-1 or m-2
    with pytest.raises(tk.TKError):
        tk.tk_contract(K, m, n, A, off_lo=1, off_hi=tk.tk_packed_size(m, n))  # not a row start
    with pytest.raises(tk.TKError):
        tk.tk_contract(K, 10, n, A)  # order above the supported maximum
    with pytest.raises(tk.TKError):
        tk.tk_contract(K[1:], m, n, A)  # K not 16-byte aligned


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_objective_with_host_buffers(storage):
    # one C-ABI call: host alpha in, host [F, |grad|, grad] out; the same pass as tk_objective
    m, n, d = 4, 33, 3
    X, Kr, Kd = _setup(m, n, d, storage, salt=21)
    a = synth.alpha_like(n, salt=22)
    y = torch.tensor(synth.alpha_like(n, salt=23), device="cuda")
    lam = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    out = tk.tk_objective_host(Kd, m, n, torch.tensor(a).pin_memory(), y, lam)
    F, grad, gn = tk.tk_objective(Kd, m, n, torch.tensor(a, device="cuda"), y, lam)
    assert out[0].item() == F.item() and out[1].item() == gn.item()
    assert torch.equal(out[2:], grad.reshape(n).cpu())
    g_ref, S_ref = oracle.contract(Kr, a, m)
    F_ref = oracle.dual_objective(S_ref, a, y.cpu().numpy(), 0.7, m)
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a), m)
    assert abs(out[0].item() - F_ref) <= float(contraction_bound(n, np.array([S_abs]), storage, m)[0]) / m + 1e-12 * abs(F_ref)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_largest_point_count(storage):
    # n = TK_MAX_POINTS: 32 column chunks per lane, the widest register configuration
    m, n, d = 2, 1024, 3
    X, Kr, Kd = _setup(m, n, d, storage, salt=41)
    a = synth.alpha_like(n, salt=42)
    v = synth.alpha_like(n, salt=43)
    G, S = tk.tk_contract(Kd, m, n, torch.tensor(a, device="cuda"))
    g_ref, S_ref = oracle.contract(Kr, a, m)
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a), m)
    assert np.all(np.abs(G.cpu().numpy() - g_ref) <= contraction_bound(n, g_abs, storage, m))
    assert abs(float(S[0]) - S_ref) <= float(contraction_bound(n, np.array([S_abs]), storage, m)[0])
    HV, _ = tk.tk_contract(Kd, m, n, torch.tensor(a, device="cuda"), r=m - 2, V=torch.tensor(v, device="cuda"))
    hv_ref = oracle.hvp(Kr, a, v, m)
    hv_abs = oracle.hvp(np.abs(Kr), np.abs(a), np.abs(v), m)
    assert np.all(np.abs(HV.cpu().numpy() - hv_ref) <= 2 * contraction_bound(n, hv_abs, storage, m, dual=True))


def test_point_count_above_the_limit_is_refused():
    m, n = 2, 1025
    K = torch.zeros(tk.tk_packed_size(m, n), dtype=torch.float32, device="cuda")
    A = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(tk.TKError):
        tk.tk_contract(K, m, n, A)


def test_empty_shard_contributes_nothing():
    m, n, d = 4, 20, 3
    X, Kr, Kd = _setup(m, n, d, "f32", salt=44)
    lo = tk.tk_row_align(m, n, tk.tk_packed_size(m, n) // 2)
    A = torch.tensor(synth.alpha_like(n, salt=45), device="cuda")
    G, S = tk.tk_contract(Kd[lo:lo + 1].clone(), m, n, A, off_lo=lo, off_hi=lo)
    assert torch.count_nonzero(G).item() == 0 and float(S[0]) == 0.0


def test_bounded_wait_times_out_and_the_context_stays_usable():
    # a device wait that runs out reports TK_ETIMEOUT through the status word;
    # the wait ends by itself (no fault, no hang) and the next call works
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    tk.tk_check_bounded_wait(ws, budget_cycles=1 << 20)
    assert tk.tk_status_read(ws) == tk.TK_ETIMEOUT
    assert tk.tk_status_read(ws) == tk.TK_OK  # reading clears it
    m, n, d = 4, 12, 3
    X, Kr, Kd = _setup(m, n, d, "f64", salt=46)
    a = synth.alpha_like(n, salt=47)
    G, S = tk.tk_contract(Kd, m, n, torch.tensor(a, device="cuda"))
    g_ref, _ = oracle.contract(Kr, a, m)
    assert np.allclose(G.cpu().numpy(), g_ref, rtol=1e-10, atol=1e-12)
