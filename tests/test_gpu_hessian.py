"""The full Hessian pass (tk_hessian): K[a^{m-2}] as a dense n x n matrix from one
pass over the packed tensor, element by element against the FP64 oracle's
dense Hessian (the second derivative of eq. dual_tensor_kernel's tensor term),
and the full-Hessian Newton solver built on it."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import as_f64, hessian_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,d", [(2, 70, 3), (3, 41, 2), (4, 1, 2), (4, 37, 5), (4, 100, 3), (6, 19, 3),
                                   (8, 9, 2), (4, 33, 2)])
def test_hessian_matches_oracle(m, n, d, storage):
    X = synth.small_problem(m, n, d, salt=700 + n + m)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    a = synth.alpha_like(n, salt=701 + n)
    H = tk.tk_hessian(Kt.cuda(), m, n, torch.tensor(a, device="cuda")).cpu().numpy()
    H_ref = oracle.hessian(Kr, a, m)
    H_abs = oracle.hessian(np.abs(Kr), np.abs(a), m)
    tol = hessian_bound(n, m, H_abs, storage)
    err = np.abs(H - H_ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    # symmetric up to the order of its last sums
    assert np.all(np.abs(H - H.T) <= 2 * tol)


def test_hessian_times_alpha_is_the_gradient_contraction():
    # Euler's identity: K[a^{m-2}] a = K[a^{m-1}], a . K[a^{m-1}] = K[a^m]
    m, n, d = 4, 150, 6
    X = synth.small_problem(m, n, d, salt=710)
    Kd = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    a = torch.tensor(synth.alpha_like(n, salt=711), device="cuda")
    H = tk.tk_hessian(Kd, m, n, a)
    G, S = tk.tk_contract(Kd, m, n, a)
    assert torch.allclose(H @ a, G, rtol=1e-11, atol=1e-11 * float(G.abs().max()))
    assert float(a @ H @ a) == pytest.approx(float(S[0]), rel=1e-11)


def test_full_newton_plain_fp64():
    # the plain FP64 configuration solved with the full Hessian: every accepted
    # Newton step costs one pass (its Hessian pass also gives F and grad F)
    p = synth.plain_fp64()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    n = X.shape[0]
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], method="newton_full", tol=1e-10)
    assert rc == tk.TK_OK and rep[0]["status"] == tk.TK_OK, rep
    assert rep[0]["gradnorm"] <= 1e-10
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-10)
    assert np.linalg.norm(A[0].cpu().numpy() - a_ref) <= (rep[0]["gradnorm"] + info["gradnorm"]) / lam + 1e-12
    assert rep[0]["passes"] <= 15, rep


def test_full_newton_masked_batch_matches_subproblems():
    m, n, d = 4, 30, 5
    X = synth.small_problem(m, n, d, salt=720)
    y = X @ synth.thesis_weights(synth.rng_for(9), d, 2) + 0.05 * synth.alpha_like(n, salt=721)
    lams = np.array([0.05, 1.0, 10.0])
    masks = np.ones((3, n), dtype=np.uint8)
    masks[1, : n // 2] = 0
    masks[2, ::3] = 0
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), lams, method="newton_full",
                                  mask=torch.tensor(masks, device="cuda"), tol=1e-10)
    assert rc == tk.TK_OK, rep
    A = A.cpu().numpy()
    for b in range(3):
        keep = masks[b].astype(bool)
        assert np.all(A[b][~keep] == 0.0)
        sub, info = oracle.solve_dual_newton(oracle.build(X[keep], m), y[keep], lams[b], m, tol=1e-10)
        assert np.linalg.norm(A[b][keep] - sub) <= (rep[b]["gradnorm"] + info["gradnorm"]) / lams[b] + 1e-12


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_full_newton_low_precision(storage):
    # the stored tensor is rounded; the returned point's exact gradient bounds
    # its distance to the exact minimiser (strong convexity)
    m, n, d = 4, 60, 8
    X = synth.small_problem(m, n, d, salt=730, dist="uniform")
    y = X @ synth.thesis_weights(synth.rng_for(8), d, 3) + 0.05 * synth.alpha_like(n, salt=731)
    lam = 1.0 / 0.86
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage=storage)
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], method="newton_full",
                                  tol=0.0, rel_gap=1e-9, max_iter=40)
    a = A[0].cpu().numpy()
    u = X.T @ a
    ge = np.linalg.norm(X @ u ** (m - 1) + lam * a - y)
    # the oracle stops at its own rounding floor (about 3e-8 here, reached in 7
    # iterations); the bound uses the gradient norm it reached
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-12, max_iter=15)
    assert np.linalg.norm(a - a_ref) <= ge / lam + info["gradnorm"] / lam + 1e-12
    assert ge <= (1e-4 if storage == "f32" else 3e-2) * np.linalg.norm(y)
