"""Pins of the oracle's packed build and contractions against the full tensor."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from brute import contract_full, full_tensor

CASES = [(2, 5, 3), (4, 5, 3), (4, 6, 2), (6, 4, 3), (2, 1, 4), (4, 1, 2), (4, 3, 1), (8, 3, 2)]


def _expand(Kp, m, n):
    """Dense tensor from packed entries: T[idx] = Kp[rank(sorted(idx))]."""
    T = np.zeros((n,) * m)
    for idx in itertools.product(range(n), repeat=m):
        T[idx] = Kp[oracle.rank(m, n, sorted(idx))]
    return T


@pytest.mark.parametrize("m,n,d", CASES)
def test_build_matches_full_tensor(m, n, d):
    X = synth.small_problem(m, n, d, salt=m * 100 + n)
    Kp = oracle.build(X, m)
    T = full_tensor(X, m)
    assert np.allclose(_expand(Kp, m, n), T, rtol=1e-13, atol=1e-13)
    # Section 4 symmetry: every permutation of the indices gives the same value
    for perm in itertools.permutations(range(m)):
        assert np.array_equal(np.transpose(T, perm), T) or \
            np.allclose(np.transpose(T, perm), T, rtol=1e-14, atol=1e-14)


def test_build_ranges_concatenate():
    X = synth.small_problem(4, 7, 3, salt=1)
    full = oracle.build(X, 4)
    N = full.shape[0]
    cuts = [0, 1, 17, 100, N - 5, N]
    parts = [oracle.build(X, 4, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
    assert np.array_equal(np.concatenate(parts), full)


def test_polynomial_kernel_is_linear_kernel_on_monomials():
    # Section 4 polynomial tensor kernel of degree 2: (sum_j prod_l x_lj)^2 equals
    # the linear tensor kernel on the explicit degree-2 monomial features x (x) x.
    X = synth.small_problem(4, 5, 3, salt=7)
    X2 = np.einsum("ij,ik->ijk", X, X).reshape(5, 9)
    assert np.allclose(oracle.build(X, 4, feat=oracle.FEAT_POLY, degree=2),
                       oracle.build(X2, 4), rtol=1e-12, atol=1e-12)


def test_exponential_kernel_brute_force():
    X = 0.3 * synth.small_problem(4, 4, 3, salt=8)
    Kp = oracle.build(X, 4, feat=oracle.FEAT_EXP)
    assert np.allclose(_expand(Kp, 4, 4), full_tensor(X, 4, feat=2), rtol=1e-13)


@pytest.mark.parametrize("m,n,d", CASES)
def test_contraction_matches_full_tensor(m, n, d):
    X = synth.small_problem(m, n, d, salt=m * 10 + n)
    a = synth.alpha_like(n, salt=m + n)
    Kp = oracle.build(X, m)
    g, S = oracle.contract(Kp, a, m)
    T = full_tensor(X, m)
    g_ref = contract_full(T, a, m - 1)
    S_ref = float(g_ref @ a)
    assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
    assert S == pytest.approx(S_ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("m,n,d", [(4, 30, 7), (6, 12, 5), (2, 50, 4), (4, 3, 9)])
def test_contraction_closed_form_linear_kernel(m, n, d):
    # linear kernel: K[a^m] = sum_k (X^T a)_k^m and K[a^{m-1}] = X (X^T a)^{m-1}
    X = synth.small_problem(m, n, d, salt=n)
    a = synth.alpha_like(n, salt=n + 1)
    u = X.T @ a
    g, S = oracle.contract(oracle.build(X, m), a, m)
    assert S == pytest.approx(float(np.sum(u ** m)), rel=1e-12)
    assert np.allclose(g, X @ u ** (m - 1), rtol=1e-11, atol=1e-11 * np.abs(g).max())
    # Euler: a . K[a^{m-1}] = K[a^m]; positive semidefinite: K[a^m] >= 0 (even m)
    assert float(a @ g) == pytest.approx(S, rel=1e-12)
    assert S >= 0.0


def test_gradient_and_hvp_finite_differences():
    m, n, d = 4, 9, 4
    X = synth.small_problem(m, n, d, salt=3)
    Kp = oracle.build(X, m)
    a = synth.alpha_like(n, salt=4)
    v = synth.alpha_like(n, salt=5)
    g, S = oracle.contract(Kp, a, m)
    h = 1e-5
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        Sp = oracle.contract(Kp, a + e, m)[1]
        Sm = oracle.contract(Kp, a - e, m)[1]
        # d K[a^m] / d a_i = m K[a^{m-1}]_i
        assert (Sp - Sm) / (2 * h) == pytest.approx(m * g[i], rel=1e-7, abs=1e-7)
    gp = oracle.contract(Kp, a + h * v, m)[0]
    gm = oracle.contract(Kp, a - h * v, m)[0]
    hv = oracle.hvp(Kp, a, v, m)
    # d K[a^{m-1}] / d a . v = (m-1) K[a^{m-2}, v]
    assert np.allclose((gp - gm) / (2 * h), (m - 1) * hv, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("m,n,d", [(2, 4, 3), (4, 5, 3), (6, 4, 2), (4, 1, 3)])
def test_hessian_and_hvp_match_full_tensor(m, n, d):
    X = synth.small_problem(m, n, d, salt=20 + m)
    a = synth.alpha_like(n, salt=21)
    v = synth.alpha_like(n, salt=22)
    Kp = oracle.build(X, m)
    T = full_tensor(X, m)
    H_ref = contract_full(T, a, m - 2)
    H = oracle.hessian(Kp, a, m)
    assert np.allclose(H, H_ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.hvp(Kp, a, v, m), H_ref @ v, rtol=1e-12, atol=1e-12)


def test_contraction_ranges_add_up():
    m, n = 4, 8
    X = synth.small_problem(m, n, 3, salt=9)
    a = synth.alpha_like(n, salt=10)
    Kp = oracle.build(X, m)
    g, S = oracle.contract(Kp, a, m)
    N = Kp.shape[0]
    gs, Ss = np.zeros(n), 0.0
    cuts = [0, 5, 77, 200, N]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        gi, Si = oracle.contract(Kp[lo:hi], a, m, lo=lo)
        gs += gi
        Ss += Si
    assert np.allclose(gs, g, rtol=1e-13, atol=1e-13)
    assert Ss == pytest.approx(S, rel=1e-13)
