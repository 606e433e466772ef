"""Autograd of K[a^m]: backward m K[a^{m-1}] and double backward m(m-1) K[a^{m-2}, v]
from the packed kernels, against finite differences and the closed form."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")
from paper_2003_10482_gb300 import autograd as tka  # noqa: E402


def test_gradcheck_fp64():
    m, n, d = 4, 9, 3
    X = synth.small_problem(m, n, d, salt=60)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    a = torch.tensor(synth.alpha_like(n, salt=61), device="cuda", requires_grad=True)
    f = lambda x: tka.energy(x, K, m)
    assert torch.autograd.gradcheck(f, (a,), eps=1e-6, atol=1e-8, rtol=1e-7)
    assert torch.autograd.gradgradcheck(f, (a,), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_higher_order_fp32_against_fd_and_closed_form():
    # the m = 6 workload: n = 80, d = 50, FP32 storage; FD step 1e-4
    p = synth.higher_order()
    m, X = p["m"], p["X"]
    n = X.shape[0]
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f32")
    a0 = synth.alpha_like(n, salt=62, scale=0.05)
    v = synth.alpha_like(n, salt=63)
    a = torch.tensor(a0, device="cuda", requires_grad=True)
    S = tka.energy(a, K, m)
    (g,) = torch.autograd.grad(S, a, create_graph=True)
    (hv,) = torch.autograd.grad(g, a, grad_outputs=torch.tensor(v, device="cuda"))
    g, hv = g.detach().cpu().numpy(), hv.cpu().numpy()
    # closed forms of the linear kernel
    u = X.T @ a0
    S_cf = float(np.sum(u ** m))
    g_cf = m * X @ u ** (m - 1)
    hv_cf = m * (m - 1) * X @ (u ** (m - 2) * (X.T @ v))
    assert float(S) == pytest.approx(S_cf, rel=1e-4)
    assert np.linalg.norm(g - g_cf) <= 1e-4 * np.linalg.norm(g_cf)
    assert np.linalg.norm(hv - hv_cf) <= 1e-4 * np.linalg.norm(hv_cf)
    # central finite differences with step 1e-4 through the kernels themselves
    h = 1e-4
    e_idx = [0, 17, 55, 79]
    for i in e_idx:
        e = np.zeros(n)
        e[i] = h
        Sp = float(tka.energy(torch.tensor(a0 + e, device="cuda"), K, m))
        Sm = float(tka.energy(torch.tensor(a0 - e, device="cuda"), K, m))
        assert (Sp - Sm) / (2 * h) == pytest.approx(g[i], rel=2e-3, abs=2e-3 * np.abs(g).max())
    gp, _ = tk.tk_contract(K, m, n, torch.tensor(a0 + h * v, device="cuda"))
    gm, _ = tk.tk_contract(K, m, n, torch.tensor(a0 - h * v, device="cuda"))
    fd = m * (gp - gm).cpu().numpy() / (2 * h)
    assert np.linalg.norm(fd - hv) <= 2e-3 * np.linalg.norm(hv)


def test_batched_energy_and_dual_objective():
    m, n, d = 4, 15, 3
    X = synth.small_problem(m, n, d, salt=64)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A = torch.tensor(synth.alpha_like(n, salt=65, batch=3), device="cuda", requires_grad=True)
    y = torch.tensor(synth.alpha_like(n, salt=66), device="cuda")
    F = tka.dual_objective(A, K, m, y, 0.5)
    F.sum().backward()
    Kr = oracle.build(X, m)
    for b in range(3):
        g_ref, S_ref = oracle.contract(Kr, A[b].detach().cpu().numpy(), m)
        gr_ref = oracle.dual_gradient(g_ref, A[b].detach().cpu().numpy(), y.cpu().numpy(), 0.5)
        assert np.allclose(A.grad[b].cpu().numpy(), gr_ref, rtol=1e-10, atol=1e-10)
        assert float(F[b]) == pytest.approx(oracle.dual_objective(S_ref, A[b].detach().cpu().numpy(),
                                                                  y.cpu().numpy(), 0.5, m), rel=1e-10)


def test_dual_objective_gradcheck_fp64():
    # F = K[a^m]/m + lam/2 |a|^2 - <y, a>: value and gradient from tk_objective,
    # Hessian-vector products from tk_dual_hvp, checked by finite differences
    m, n, d = 4, 8, 3
    X = synth.small_problem(m, n, d, salt=67)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    y = torch.tensor(synth.alpha_like(n, salt=68), device="cuda")
    a = torch.tensor(synth.alpha_like(n, salt=69, batch=2), device="cuda", requires_grad=True)
    f = lambda x: tka.dual_objective(x, K, m, y, 0.3)
    assert torch.autograd.gradcheck(f, (a,), eps=1e-6, atol=1e-8, rtol=1e-7)
    assert torch.autograd.gradgradcheck(f, (a,), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_dual_hvp_matches_oracle(storage):
    m, n, d, B = 4, 23, 4, 3
    X = synth.small_problem(m, n, d, salt=90)
    K64 = oracle.build(X, m)
    Kt = torch.from_numpy(K64).to(torch.float64 if storage == "f64" else torch.float32)
    Kr = Kt.double().numpy()
    A = synth.alpha_like(n, salt=91, batch=B)
    V = synth.alpha_like(n, salt=92, batch=B)
    lam = np.array([0.1, 1.0, 7.0])
    HV = tk.tk_dual_hvp(Kt.cuda(), m, n, torch.tensor(A, device="cuda"), torch.tensor(V, device="cuda"),
                        torch.tensor(lam, device="cuda")).cpu().numpy()
    from gpu_util import contraction_bound
    for b in range(B):
        ref = (m - 1) * oracle.hvp(Kr, A[b], V[b], m) + lam[b] * V[b]
        hab = (m - 1) * oracle.hvp(np.abs(Kr), np.abs(A[b]), np.abs(V[b]), m) + lam[b] * np.abs(V[b])
        # the dual-number pass carries two accumulation chains; the finish is
        # two FP64 operations
        tol = 2 * contraction_bound(n, hab, storage, m, dual=True) + 4 * 2.0 ** -53 * hab
        assert np.all(np.abs(HV[b] - ref) <= tol), float(np.max(np.abs(HV[b] - ref) / tol))
