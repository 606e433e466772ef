"""Pins of the oracle's dual solver, primal recovery and Nystrom selection."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from brute import full_tensor


def test_duality_maps_invert():
    # Section 4: J_p o J_q = Id for 1/p + 1/q = 1
    z = synth.alpha_like(50, salt=1, scale=3.0)
    for q in (2.0, 4.0, 6.0):
        p = q / (q - 1.0)
        assert np.allclose(oracle.J(oracle.J(z, q), p), z, rtol=1e-12, atol=1e-12)


def test_conjugate_identity():
    # Section 4, eq. tensor_sub_jq: u.J_q(u) - (1/p)|J_q(u)|_p^p = (1/q)|u|_q^q
    u = synth.alpha_like(40, salt=2, scale=2.0)
    for q in (4.0, 6.0):
        p = q / (q - 1.0)
        jq = oracle.J(u, q)
        lhs = float(u @ jq) - float(np.sum(np.abs(jq) ** p)) / p
        assert lhs == pytest.approx(float(np.sum(np.abs(u) ** q)) / q, rel=1e-12)


def test_order_two_is_ridge_regression():
    # m = 2 (p = q = 2): the dual is kernel ridge regression, whose minimiser is
    # (X X^T + lam I)^{-1} y (textbook closed form)
    X = synth.small_problem(2, 15, 4, salt=3)
    y = synth.alpha_like(15, salt=4)
    lam = 0.3
    K = oracle.build(X, 2)
    a, info = oracle.solve_dual_newton(K, y, lam, 2, tol=1e-12)
    a_ref = np.linalg.solve(X @ X.T + lam * np.eye(15), y)
    assert np.allclose(a, a_ref, rtol=1e-10, atol=1e-12)
    assert info["iters"] <= 2


def _solved_plain():
    p = synth.plain_fp64()
    K = oracle.build(p["X"], p["m"])
    a, info = oracle.solve_dual_newton(K, p["y"], p["lam"], p["m"], tol=1e-10)
    return p, K, a, info


def test_plain_fp64_kkt_and_duality_gap():
    p, K, a, info = _solved_plain()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    assert info["gradnorm"] <= 1e-10
    # dual optimality (eq. jq) written with the closed form X J_q(X^T a)
    u = X.T @ a
    grad = X @ u ** (m - 1) + lam * a - y
    assert np.linalg.norm(grad) <= 1e-9
    # representer map and primal optimality (eq. jp_4):
    # X^T (X w - y) + gamma^{-1} J_p(w) = 0 with gamma = 1/lam
    w = oracle.primal_from_dual(X, a, m)
    pp = m / (m - 1.0)
    kkt = X.T @ (X @ w - y) + lam * oracle.J(w, pp)
    assert np.linalg.norm(kkt) <= 1e-8 * max(1.0, np.linalg.norm(X.T @ y))
    # strong duality (Section 4, min F = -min Lambda): P(w*) + F(a*) = 0
    Fd = oracle.dual_objective(float(np.sum(u ** m)), a, y, lam, m)
    Pp = oracle.primal_objective(X, y, w, lam, m)
    assert Pp + Fd == pytest.approx(0.0, abs=1e-9 * max(1.0, abs(Pp)))


def test_newton_converges_quadratically():
    _, _, _, info = _solved_plain()
    g = [h[1] for h in info["history"]]
    assert info["iters"] < 40
    # above the rounding floor the gradient norm falls quadratically:
    # |grad_{k+1}| <= C |grad_k|^2 for the last steps with |grad_k| < 1e-3
    tail = [(g0, g1) for g0, g1 in zip(g[:-1], g[1:]) if 1e-8 < g0 < 1e-3]
    assert len(tail) >= 2
    for g0, g1 in tail:
        assert g1 <= 100.0 * g0 * g0


def test_prediction_equals_tensor_kernel_sum():
    # Section 4, eq. tensor_1: <w, x> = sum_{i_1..i_{q-1}} k(x_{i_1},..,x_{i_{q-1}}, x) a_{i_1}..a_{i_{q-1}}
    m, n, d = 4, 5, 3
    X = synth.small_problem(m, n, d, salt=11)
    Xt = synth.small_problem(m, 3, d, salt=12)
    a = synth.alpha_like(n, salt=13)
    w = oracle.primal_from_dual(X, a, m)
    for x in Xt:
        Z = np.vstack([X, x])
        T = full_tensor(Z, m)
        s = 0.0
        for idx in itertools.product(range(n), repeat=m - 1):
            s += T[idx + (n,)] * np.prod(a[list(idx)])
        assert float(oracle.predict(x[None, :], w)[0]) == pytest.approx(s, rel=1e-12)


def test_threshold_support():
    w = np.zeros(100)
    w[[3, 50, 77]] = [5.0, -4.0, 6.0]
    w += 1e-3 * synth.alpha_like(100, salt=5)
    assert list(oracle.threshold_support(w)) == [3, 50, 77]
    assert oracle.mse(np.array([1.0, 2.0]), np.array([0.0, 0.0])) == 2.5


def test_nystrom_properties():
    idx = oracle.nystrom_select(50_000, 600, 123)
    assert idx.shape == (600,)
    assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < 50_000
    assert np.array_equal(oracle.nystrom_select(10, 10, 5), np.arange(10))
    assert oracle.nystrom_select(10, 0, 5).shape == (0,)
    assert np.array_equal(oracle.nystrom_select(1000, 30, 7), oracle.nystrom_select(1000, 30, 7))
    assert not np.array_equal(oracle.nystrom_select(1000, 30, 7), oracle.nystrom_select(1000, 30, 8))
    with pytest.raises(ValueError):
        oracle.nystrom_select(5, 6, 1)


def test_nystrom_subsets_are_uniform():
    # every 3-subset of 7 points is equally likely (chi-square, 35 cells)
    counts = {}
    trials = 35 * 400
    for s in range(trials):
        key = tuple(oracle.nystrom_select(7, 3, s))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.comb(7, 3)
    exp = trials / 35
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    # 34 degrees of freedom: P(chi2 > 70) < 1e-3
    assert chi2 < 70


def test_dexter_shaped_generator():
    # 0.5 % density, w* supported on features that occur in some row, thesis-rule values
    p = synth.dexter_like()
    X, w = p["X"], p["w_true"]
    assert X.shape == (200, 20_000)
    assert abs(np.mean(X != 0.0) - 0.005) < 0.0005
    sup = np.flatnonzero(w)
    assert sup.size == 20 and np.all(np.any(X[:, sup] != 0.0, axis=0))
    assert np.all((np.abs(w[sup]) >= 0.7) & (np.abs(w[sup]) <= 1.0))
    assert np.allclose(p["y"], X @ w, atol=0.05 * 6)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_dual_objective_floor(m):
    # For an exact tensor of even order K[a^m] >= 0, so
    # F(a) >= (lam/2)|a|^2 - <y, a> >= -|y|^2/(2 lam), with equality only at
    # a = y/lam when K[(y/lam)^m] = 0 (y orthogonal to the features' span).
    # The GPU solver stops a problem whose computed F goes below this floor.
    n, d, lam = 9, 3, 0.37
    X = synth.small_problem(m, n, d, salt=140 + m)
    K = oracle.build(X, m)
    rng = np.random.default_rng(141)
    y = rng.standard_normal(n)
    floor = -float(y @ y) / (2 * lam)
    for _ in range(50):
        a = rng.standard_normal(n) * rng.choice([1e-2, 1.0, 30.0])
        _, S = oracle.contract(K, a, m)
        assert S >= 0.0
        assert oracle.dual_objective(S, a, y, lam, m) >= floor
    # the floor is attained where the tensor vanishes: y in the null space of X^T
    Q, _ = np.linalg.qr(X, mode="complete")
    y0 = Q[:, d:] @ rng.standard_normal(n - d)  # X^T y0 = 0
    a0 = y0 / lam
    _, S0 = oracle.contract(K, a0, m)
    assert abs(S0) <= 1e-12 * float(a0 @ a0) ** (m / 2) * np.abs(X).sum() ** m
    assert oracle.dual_objective(S0, a0, y0, lam, m) == pytest.approx(-float(y0 @ y0) / (2 * lam), rel=1e-9)
