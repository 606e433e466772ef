"""Seeded synthetic inputs shaped like the thesis's sparse-regression workloads.

This module only draws random numbers; it holds none of the method's
arithmetic.  Both the oracle side (tests, CPU baseline) and the CUDA side
(tests, bench) take their inputs from here, so the two see identical data.

Generator (Section 5.4 of the thesis): X with i.i.d. entries, a sparse w* whose
s nonzero positions are drawn at random and whose values are sign(h)(1 - 0.3u)
with h ~ N(0,1), u ~ U(0,1), and y = X w* + sigma * eps with eps ~ N(0,1)
(the thesis writes eps in R^d; it must be R^n).  The five workloads below
follow that recipe with the shapes of the thesis's experiments; the thesis
datasets (Wpbc, Dexter) are not available and these draws stand in for them.

All draws use numpy's PCG64 seeded with 2003_10482 + workload index.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2003_10482


def rng_for(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + index, salt]))


def thesis_weights(rng: np.random.Generator, d: int, s: int) -> np.ndarray:
    """Sparse w*: s random positions with values sign(h)(1 - 0.3u)."""
    w = np.zeros(d)
    pos = rng.choice(d, size=s, replace=False)
    h = rng.standard_normal(s)
    u = rng.uniform(0.0, 1.0, size=s)
    w[pos] = np.where(h >= 0, 1.0, -1.0) * (1.0 - 0.3 * u)
    return w


def ar1_gaussian(rng: np.random.Generator, rows: int, d: int, rho: float) -> np.ndarray:
    """Rows ~ N(0, Sigma) with Sigma_ij = rho^|i-j|, drawn exactly as the AR(1)
    recursion x_1 = z_1, x_j = rho x_{j-1} + sqrt(1 - rho^2) z_j."""
    z = rng.standard_normal((rows, d))
    x = np.empty_like(z)
    x[:, 0] = z[:, 0]
    c = np.sqrt(1.0 - rho * rho)
    for j in range(1, d):
        x[:, j] = rho * x[:, j - 1] + c * z[:, j]
    return x


def plain_fp64(index: int = 0) -> dict:
    """m=4, n=40, d=10, X ~ N(0,1); w* has 3 entries of value +-1 at random
    positions; y = X w* + N(0, 0.01^2); lambda = 1e-2."""
    rng = rng_for(index)
    n, d = 40, 10
    X = rng.standard_normal((n, d))
    w = np.zeros(d)
    pos = rng.choice(d, size=3, replace=False)
    w[pos] = np.where(rng.standard_normal(3) >= 0, 1.0, -1.0)
    y = X @ w + 0.01 * rng.standard_normal(n)
    return dict(name="plain_fp64_m4_n40_d10", m=4, X=X, y=y, w_true=w, lam=1e-2,
                storage="f64")


def full_fp32(index: int = 1) -> dict:
    """m=4, n=400, d=100, X ~ U(-1,1); w* has 10 entries ~ N(0,1); noise at
    20 dB SNR (sigma = std(X w*)/10); gamma = 0.86 as in the thesis's synthetic
    runs, i.e. lambda = 1/0.86."""
    rng = rng_for(index)
    n, d = 400, 100
    X = rng.uniform(-1.0, 1.0, size=(n, d))
    w = np.zeros(d)
    pos = rng.choice(d, size=10, replace=False)
    w[pos] = rng.standard_normal(10)
    clean = X @ w
    y = clean + (np.std(clean) / 10.0) * rng.standard_normal(n)
    return dict(name="full_fp32_m4_n400_d100", m=4, X=X, y=y, w_true=w,
                lam=1.0 / 0.86, storage="f32")


def higher_order(index: int = 2) -> dict:
    """m=6, n=80, d=50, X ~ N(0,1); w* has 5 thesis-rule entries; sigma = 0.05."""
    rng = rng_for(index)
    n, d = 80, 50
    X = rng.standard_normal((n, d))
    w = thesis_weights(rng, d, 5)
    y = X @ w + 0.05 * rng.standard_normal(n)
    return dict(name="higher_order_m6_n80_d50", m=6, X=X, y=y, w_true=w,
                lam=1.0 / 0.86, storage="f32")


def nystrom_bf16(index: int = 3, n_train: int = 50_000, n_test: int = 10_000,
                 d: int = 200, n_prime: int = 600) -> dict:
    """N = 50,000 training and 10,000 held-out points, d = 200, rows ~ N(0, Sigma)
    with Sigma_ij = 0.5^|i-j|; w* has 20 thesis-rule entries; sigma = 0.05;
    n' = 600 landmarks (selected by the library's Nystrom call, seed below)."""
    rng = rng_for(index)
    X = ar1_gaussian(rng, n_train + n_test, d, 0.5)
    w = thesis_weights(rng, d, 20)
    y = X @ w + 0.05 * rng.standard_normal(n_train + n_test)
    return dict(name="nystrom_bf16_m4_N50000_d200_np600", m=4,
                X_train=X[:n_train], y_train=y[:n_train],
                X_test=X[n_train:], y_test=y[n_train:], w_true=w,
                n_prime=n_prime, select_seed=SEED_BASE + index, lam=1.0 / 0.86,
                storage="bf16")


def batched_path(index: int = 4, n_points: int = 20_000, d: int = 80,
                 n_prime: int = 300, n_lambda: int = 64, n_folds: int = 8) -> dict:
    """m=4, n' = 300 landmarks of N = 20,000 points, d = 80; w* has 10
    thesis-rule entries; sigma = 0.05; 64 lambdas log-spaced in [1e-4, 1] times
    8 cross-validation folds = 512 problems.  Fold f keeps the landmarks whose
    position in a seeded permutation is not congruent to f mod 8."""
    rng = rng_for(index)
    X = rng.standard_normal((n_points, d))
    w = thesis_weights(rng, d, 10)
    y = X @ w + 0.05 * rng.standard_normal(n_points)
    perm = rng.permutation(n_prime)
    fold_of = np.empty(n_prime, dtype=np.int64)
    fold_of[perm] = np.arange(n_prime) % n_folds
    lambdas = np.logspace(-4.0, 0.0, n_lambda)
    masks = np.zeros((n_lambda * n_folds, n_prime), dtype=np.uint8)
    lam_b = np.zeros(n_lambda * n_folds)
    for i, lam in enumerate(lambdas):
        for f in range(n_folds):
            b = i * n_folds + f
            masks[b] = (fold_of != f).astype(np.uint8)
            lam_b[b] = lam
    return dict(name="batched_path_m4_np300_d80_B512", m=4, X=X, y=y, w_true=w,
                n_prime=n_prime, select_seed=SEED_BASE + index, lambdas=lam_b,
                masks=masks, storage="f32")


def dexter_like(index: int = 5, n: int = 200, d: int = 20_000, density: float = 0.005, s: int = 20) -> dict:
    """Shaped like the thesis's Dexter runs (few points, very many sparse
    features): n = 200 rows of d = 20,000 features, each feature nonzero with
    probability 0.5 % (values ~ N(0, 1)); w* has s = 20 thesis-rule entries
    among the features that have a nonzero in some row; sigma = 0.05; m = 4;
    lambda = 1 (the thesis does not state its Dexter lambda)."""
    rng = rng_for(index)
    X = np.where(rng.random((n, d)) < density, rng.standard_normal((n, d)), 0.0)
    used = np.flatnonzero(np.any(X != 0.0, axis=0))
    w = np.zeros(d)
    pos = rng.choice(used, size=min(s, used.size), replace=False)
    h = rng.standard_normal(pos.size)
    u = rng.random(pos.size)
    w[pos] = np.sign(h) * (1.0 - 0.3 * u)
    y = X @ w + 0.05 * rng.standard_normal(n)
    return dict(name="dexter_like_m4_n200_d20000", m=4, X=X, y=y, w_true=w, lam=1.0, storage="f32")


def alpha_like(n: int, salt: int, scale: float = 1.0, batch: int | None = None) -> np.ndarray:
    """Seeded dual vector(s) ~ N(0, scale^2) for contraction tests."""
    rng = rng_for(99, salt)
    shape = (n,) if batch is None else (batch, n)
    return scale * rng.standard_normal(shape)


def small_problem(m: int, n: int, d: int, salt: int, dist: str = "normal") -> np.ndarray:
    """Seeded n x d data matrix for parity tests of odd sizes."""
    rng = rng_for(98, salt)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=(n, d))
    return rng.standard_normal((n, d))
