"""Plain FP64 CPU oracle for the packed tensor-kernel method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2003_10482_gb300``) and never imports it.

Thesis: F. Hibraj, "Efficient Tensor Kernel methods for sparse regression".

What each function follows:

* ``packed_size``            -- Section 5, b_matrix / b_cube / b_tensor4 (the
                                 number of sorted index tuples).
* ``rank`` / ``unrank`` / ``enumerate_tuples``
                              -- Section 5 nested-loop storage order.
* ``build``                  -- Section 4, tensor kernel k = sum_k prod_j phi_k.
* ``contract``               -- Section 4, eq. dual_tensor_kernel: K[a^m] and
                                 K[a^{m-1}] over all n^m tuples, via multiplicities.
* ``hessian`` / ``hvp``      -- second derivative of the same polynomial.
* ``dual_objective`` / ``dual_gradient``
                              -- Section 4, eq. dual_tensor / dual_tensor_kernel and
                                 eq. jq, with lambda = 1/gamma.
* ``primal_from_dual``       -- Section 4, eq. tensor_representer, w = J_q(X^T a).
* ``primal_objective``       -- Section 4, eq. tensor_primal.
* ``solve_dual_newton``      -- the thesis names no algorithm; damped Newton
                                 with a dense Hessian and Armijo backtracking.
* ``nystrom_select``         -- Section 6.1 uniform subsampling (SplitMix64 +
                                 Floyd's algorithm as the stated generator).
* ``predict`` / ``mse``      -- Section 4 test-phase estimate; Section 6.1 MSE.
* ``threshold_support``      -- Section 6.3, keep |w_j| > 2 std(w).

Every function has a pin in ``tests/test_oracle_*.py`` that does not go through
the oracle itself (thesis numbers, brute force over all n^m tuples, closed forms,
finite differences, duality).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libtk_oracle.so")
_lock = threading.Lock()
_lib = None

FEAT_LINEAR, FEAT_POLY, FEAT_EXP = 0, 1, 2


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/ (plain -O2, no OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            i64, i32, dbl, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            P = ctypes.c_void_p
            lib.or_multichoose.restype = i64
            lib.or_multichoose.argtypes = [i64, i32]
            lib.or_packed_size.restype = i64
            lib.or_packed_size.argtypes = [i32, i64]
            lib.or_rank.restype = i64
            lib.or_rank.argtypes = [i32, i64, P]
            lib.or_unrank.restype = None
            lib.or_unrank.argtypes = [i32, i64, i64, P]
            lib.or_enumerate.restype = i64
            lib.or_enumerate.argtypes = [i32, i64, P, i64]
            lib.or_build.restype = None
            lib.or_build.argtypes = [i32, i64, i64, P, i32, i32, i64, i64, P]
            lib.or_contract.restype = None
            lib.or_contract.argtypes = [i32, i64, P, i64, i64, P, P, P]
            lib.or_hessian.restype = None
            lib.or_hessian.argtypes = [i32, i64, P, i64, i64, P, P]
            lib.or_hvp.restype = None
            lib.or_hvp.argtypes = [i32, i64, P, i64, i64, P, P, P]
            lib.or_nystrom_select.restype = i32
            lib.or_nystrom_select.argtypes = [i64, i64, u64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- layout
def packed_size(m: int, n: int) -> int:
    """Number of stored entries: the multiset coefficient C(n+m-1, m)."""
    return math.comb(n + m - 1, m)


def rank(m: int, n: int, t) -> int:
    """Offset of a sorted tuple in the nested-loop storage order."""
    a = np.ascontiguousarray(t, dtype=np.int32)
    assert a.shape == (m,) and np.all(np.diff(a) >= 0)
    return int(_L().or_rank(m, n, _ptr(a)))


def unrank(m: int, n: int, off: int) -> np.ndarray:
    t = np.zeros(m, dtype=np.int32)
    _L().or_unrank(m, n, int(off), _ptr(t))
    return t


def enumerate_tuples(m: int, n: int) -> np.ndarray:
    """All sorted tuples in storage order, shape (N, m)."""
    N = packed_size(m, n)
    out = np.zeros((N, m), dtype=np.int32)
    k = _L().or_enumerate(m, n, _ptr(out), N)
    assert k == N
    return out


# ----------------------------------------------------------------- tensor
def build(X, m: int, lo: int = 0, hi: int | None = None,
          feat: int = FEAT_LINEAR, degree: int = 1) -> np.ndarray:
    """Packed entries K[lo:hi] of the order-m tensor kernel over the rows of X."""
    X = _f64(X)
    n, d = X.shape
    N = packed_size(m, n)
    hi = N if hi is None else hi
    K = np.zeros(max(hi - lo, 0), dtype=np.float64)
    _L().or_build(m, n, d, _ptr(X), feat, degree, lo, hi, _ptr(K))
    return K


def contract(K, alpha, m: int, lo: int = 0):
    """(g, S) with g = K[alpha^{m-1}] (n-vector) and S = K[alpha^m], summed over
    the stored entries K (offsets lo .. lo+len(K)-1)."""
    K = _f64(K)
    a = _f64(alpha)
    n = a.shape[0]
    g = np.zeros(n)
    S = np.zeros(1)
    _L().or_contract(m, n, _ptr(K), lo, lo + K.shape[0], _ptr(a), _ptr(g), _ptr(S))
    return g, float(S[0])


def hessian(K, alpha, m: int, lo: int = 0) -> np.ndarray:
    """K[alpha^{m-2}] as a dense symmetric n x n matrix."""
    K = _f64(K)
    a = _f64(alpha)
    n = a.shape[0]
    H = np.zeros((n, n))
    _L().or_hessian(m, n, _ptr(K), lo, lo + K.shape[0], _ptr(a), _ptr(H))
    return H


def hvp(K, alpha, v, m: int, lo: int = 0) -> np.ndarray:
    """K[alpha^{m-2}, v] (n-vector)."""
    K = _f64(K)
    a = _f64(alpha)
    vv = _f64(v)
    n = a.shape[0]
    out = np.zeros(n)
    _L().or_hvp(m, n, _ptr(K), lo, lo + K.shape[0], _ptr(a), _ptr(vv), _ptr(out))
    return out


# ----------------------------------------------------------------- dual problem
def dual_objective(S: float, alpha, y, lam: float, m: int) -> float:
    """F(a) = K[a^m]/m + (lam/2)|a|^2 - <y, a>, lam = 1/gamma (eq. dual_tensor_kernel)."""
    a = _f64(alpha)
    return S / m + 0.5 * lam * float(a @ a) - float(_f64(y) @ a)


def dual_gradient(g, alpha, y, lam: float) -> np.ndarray:
    """grad F = K[a^{m-1}] + lam a - y (eq. jq with X J_q(X^T a) = K[a^{m-1}])."""
    return _f64(g) + lam * _f64(alpha) - _f64(y)


def solve_dual_newton(K, y, lam: float, m: int, tol: float = 1e-10,
                      max_iter: int = 100, alpha0=None):
    """Damped Newton on the dual: Hessian (m-1) K[a^{m-2}] + lam I, Cholesky
    solve, Armijo backtracking (c = 1e-4, halving), start a = 0, stop at
    |grad F|_2 <= tol.  Returns (alpha, info)."""
    y = _f64(y)
    n = y.shape[0]
    a = np.zeros(n) if alpha0 is None else _f64(alpha0).copy()
    hist = []

    def fg(x):
        g, S = contract(K, x, m)
        return dual_objective(S, x, y, lam, m), dual_gradient(g, x, y, lam)

    F, G = fg(a)
    it = 0
    for it in range(max_iter + 1):
        gn = float(np.linalg.norm(G))
        hist.append((F, gn))
        if gn <= tol or it == max_iter:
            break
        H = (m - 1) * hessian(K, a, m) + lam * np.eye(n)
        L = np.linalg.cholesky(H)
        p = -np.linalg.solve(L.T, np.linalg.solve(L, G))
        slope = float(G @ p)
        t = 1.0
        while True:
            Fn, Gn = fg(a + t * p)
            if Fn <= F + 1e-4 * t * slope or t < 1e-20:
                break
            t *= 0.5
        a = a + t * p
        F, G = Fn, Gn
    return a, {"iters": it, "F": F, "gradnorm": float(np.linalg.norm(G)),
               "history": hist}


# ----------------------------------------------------------------- primal side
def J(z, r: float) -> np.ndarray:
    """Duality map J_r(z) = sign(z) |z|^{r-1}, the gradient of (1/r)|z|_r^r."""
    z = _f64(z)
    return np.sign(z) * np.abs(z) ** (r - 1.0)


def primal_from_dual(X, alpha, m: int) -> np.ndarray:
    """Representer map w = J_q(X^T a) with q = m (eq. tensor_representer)."""
    return J(_f64(X).T @ _f64(alpha), float(m))


def primal_objective(X, y, w, lam: float, m: int) -> float:
    """P(w) = (gamma/2)|Xw - y|^2 + (1/p)|w|_p^p, gamma = 1/lam, p = m/(m-1)
    (eq. tensor_primal)."""
    p = m / (m - 1.0)
    r = _f64(X) @ _f64(w) - _f64(y)
    return 0.5 / lam * float(r @ r) + float(np.sum(np.abs(w) ** p)) / p


def predict(Xtest, w) -> np.ndarray:
    """<w, x> for each test row (Section 4 test-phase estimate, linear kernel)."""
    return _f64(Xtest) @ _f64(w)


def mse(yhat, y) -> float:
    """Mean squared error over the evaluated points (Section 6.1)."""
    d = _f64(yhat) - _f64(y)
    return float(d @ d) / d.shape[0]


def threshold_support(w) -> np.ndarray:
    """Indices j with |w_j| > 2 std(w) (adaptive threshold of Section 6.3)."""
    w = _f64(w)
    return np.nonzero(np.abs(w) > 2.0 * np.std(w))[0]


# ----------------------------------------------------------------- Nystrom
def nystrom_select(N: int, n_prime: int, seed: int) -> np.ndarray:
    """n' of N indices, uniform without replacement, sorted ascending."""
    out = np.zeros(max(n_prime, 0), dtype=np.int64)
    rc = _L().or_nystrom_select(N, n_prime, ctypes.c_uint64(seed & (2**64 - 1)), _ptr(out))
    if rc != 0:
        raise ValueError("n_prime must be in [0, N]")
    return out
