"""GPU dual solver (tk_solve_dual) against the FP64 oracle and the problem's own
optimality conditions.  F is lambda-strongly convex, so for any point a
|a - a*| <= |grad F(a)| / lambda: the checks below bound the distance to the
oracle's minimiser by the gradient norms both sides report."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


def _exact_grad(X, y, lam, m, a):
    """grad F at a for the exact (FP64, linear-kernel) problem, closed form."""
    u = X.T @ a
    return X @ u ** (m - 1) + lam * a - y


def test_plain_fp64_solves_to_tolerance():
    p = synth.plain_fp64()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    n = X.shape[0]
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], tol=1e-10)
    assert rc == tk.TK_OK and rep[0]["status"] == tk.TK_OK
    assert rep[0]["gradnorm"] <= 1e-10
    a = A[0].cpu().numpy()
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-10)
    assert np.linalg.norm(a - a_ref) <= (rep[0]["gradnorm"] + info["gradnorm"]) / lam + 1e-12
    # optimality of the exact problem at the GPU's point, and zero duality gap
    assert np.linalg.norm(_exact_grad(X, y, lam, m, a)) <= 1e-9
    w = oracle.primal_from_dual(X, a, m)
    Fd = oracle.dual_objective(float(np.sum((X.T @ a) ** m)), a, y, lam, m)
    assert oracle.primal_objective(X, y, w, lam, m) + Fd == pytest.approx(0.0, abs=1e-8)
    assert rep[0]["F"] == pytest.approx(info["F"], rel=1e-10, abs=1e-12)


def test_order_two_is_ridge():
    X = synth.small_problem(2, 25, 4, salt=40)
    y = synth.alpha_like(25, salt=41)
    lam = 0.7
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), 2, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, 2, 25, torch.tensor(y, device="cuda"), [lam], tol=1e-12)
    a_ref = np.linalg.solve(X @ X.T + lam * np.eye(25), y)
    assert np.allclose(A[0].cpu().numpy(), a_ref, rtol=1e-9, atol=1e-11)


def test_masked_batch_matches_subproblems():
    m, n, d = 4, 30, 5
    X = synth.small_problem(m, n, d, salt=42)
    y = X @ synth.thesis_weights(synth.rng_for(7), d, 2) + 0.05 * synth.alpha_like(n, salt=43)
    lams = np.array([0.1, 1.0, 10.0])
    masks = np.ones((3, n), dtype=np.uint8)
    masks[1, : n // 2] = 0
    masks[2, ::3] = 0
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), lams,
                                  mask=torch.tensor(masks, device="cuda"), tol=1e-10)
    assert rc == tk.TK_OK
    A = A.cpu().numpy()
    for b in range(3):
        keep = masks[b].astype(bool)
        assert np.all(A[b][~keep] == 0.0)
        sub, info = oracle.solve_dual_newton(oracle.build(X[keep], m), y[keep], lams[b], m, tol=1e-10)
        assert np.linalg.norm(A[b][keep] - sub) <= (rep[b]["gradnorm"] + info["gradnorm"]) / lams[b] + 1e-12


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_low_precision_storage_solution_error(storage):
    # the stored tensor is a rounded copy of K; the solver finds the minimiser of
    # that problem.  Its distance to the exact minimiser is bounded a posteriori
    # by the exact gradient at the returned point.
    m, n, d = 4, 60, 8
    X = synth.small_problem(m, n, d, salt=44, dist="uniform")
    y = X @ synth.thesis_weights(synth.rng_for(8), d, 3) + 0.05 * synth.alpha_like(n, salt=45)
    lam = 1.0 / 0.86
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage=storage)
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], tol=1e-7)
    a = A[0].cpu().numpy()
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-12, max_iter=15)
    ge = np.linalg.norm(_exact_grad(X, y, lam, m, a))
    assert np.linalg.norm(a - a_ref) <= ge / lam + info["gradnorm"] / lam + 1e-12
    # and the stored-precision perturbation keeps it small in absolute terms
    assert ge <= (1e-4 if storage == "f32" else 3e-2) * np.linalg.norm(y)


def test_gradient_descent_method():
    m, n, d = 4, 20, 4
    X = synth.small_problem(m, n, d, salt=46)
    y = synth.alpha_like(n, salt=47)
    lam = 2.0
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], method="gd_bt",
                                  tol=1e-8, max_iter=5000)
    assert rc == tk.TK_OK, rep
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-12, max_iter=15)
    assert np.linalg.norm(A[0].cpu().numpy() - a_ref) <= (1e-8 + info["gradnorm"]) / lam + 1e-12


def test_batch_solves_each_problem_as_alone():
    # The line search runs in lockstep over the batch: a problem that accepts
    # its step while another still backtracks must keep it (and a compacted
    # pass over the problems still searching must not disturb it).  With FP64
    # storage a batch does, problem by problem, the arithmetic of a solve of
    # that problem alone, up to the rounding of kernels that differ between the
    # full and the compacted passes.
    m, n, d = 4, 26, 4
    X = synth.small_problem(m, n, d, salt=61)
    y = X @ synth.thesis_weights(synth.rng_for(8), d, 2) + 0.05 * synth.alpha_like(n, salt=62)
    lams = np.array([1e-2, 10.0, 0.3])  # the small lambda backtracks, the large one does not
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    yt = torch.tensor(y, device="cuda")
    for it in (1, 2, 3):
        A, rep, _ = tk.tk_solve_dual(K, m, n, yt, lams, tol=1e-10, max_iter=it)
        for b in range(3):
            A1, rep1, _ = tk.tk_solve_dual(K, m, n, yt, lams[b:b + 1], tol=1e-10, max_iter=it)
            assert rep1[0]["passes"] == rep[b]["passes"]
            assert np.allclose(A[b].cpu().numpy(), A1[0].cpu().numpy(), rtol=1e-12, atol=1e-13), (it, b)
    A, rep, rc = tk.tk_solve_dual(K, m, n, yt, lams, tol=1e-10)
    assert rc == tk.TK_OK
    for b in range(3):
        A1, rep1, rc1 = tk.tk_solve_dual(K, m, n, yt, lams[b:b + 1], tol=1e-10)
        assert rc1 == tk.TK_OK
        dist = float((A[b] - A1[0]).norm())
        assert dist <= (rep[b]["gradnorm"] + rep1[0]["gradnorm"]) / lams[b] + 1e-12


def test_relative_gap_stop():
    # Newton decrement stop: F - F* ~ -<grad F, p>/2 <= rel_gap max(1, |F|)
    p = synth.plain_fp64()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    n = X.shape[0]
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, m, n, torch.tensor(y, device="cuda"), [lam], tol=0.0, rel_gap=1e-8)
    assert rc == tk.TK_OK and rep[0]["status"] == tk.TK_OK
    a_ref, info = oracle.solve_dual_newton(oracle.build(X, m), y, lam, m, tol=1e-12, max_iter=15)
    assert abs(rep[0]["F"] - info["F"]) <= 1e-7 * max(1.0, abs(info["F"]))


@pytest.mark.parametrize("method", ["newton_full", "newton_cg"])
def test_batched_solve_through_tensor_cores(method):
    # 72 problems (lambda in [0.3, 3]) at n = 96: the objective and gradient
    # passes of the batch take the tensor-core batched contraction while at
    # least 64 problems are active, then the SIMT kernels.  Every returned point
    # is judged by its exact (FP64, closed-form) gradient, which bounds its
    # distance to the exact minimiser (strong convexity).
    m, n, d, B = 4, 96, 6, 72
    X = synth.small_problem(m, n, d, salt=91, dist="uniform")
    y = X @ synth.thesis_weights(synth.rng_for(5), d, 3) + 0.05 * synth.alpha_like(n, salt=92)
    lams = np.geomspace(0.3, 3.0, B)
    K = tk.tk_build_packed(torch.tensor(X, device="cuda"), m, storage="f32")
    yt = torch.tensor(y, device="cuda")
    tk.tk_batched_set_config(tensor_cores=1)
    try:
        assert tk.tk_batched_get_config(m, n, "f32", False, B)["tensor_cores"] == 1
        A, rep, rc = tk.tk_solve_dual(K, m, n, yt, lams, method=method, tol=0.0, rel_gap=1e-9, max_iter=40,
                                      K_hvp=K if method == "newton_full" else None)
    finally:
        tk.tk_batched_set_config(reset=True)
    A = A.cpu().numpy()
    for b in range(B):
        ge = np.linalg.norm(_exact_grad(X, y, lams[b], m, A[b]))
        assert ge <= 1e-4 * np.linalg.norm(y), (b, ge, rep[b])

