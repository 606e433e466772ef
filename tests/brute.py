"""Brute-force references over the FULL n^m tensor (tiny n only).

These go through numpy's einsum on the dense tensor and never touch the packed
layout, so they pin the oracle's packed routines from outside.
"""
import string

import numpy as np


def full_tensor(X, m, feat=0, degree=1):
    """T[i_1..i_m] = k(x_{i_1}, ..., x_{i_m}) as a dense array."""
    letters = string.ascii_lowercase[:m]
    spec = ",".join(f"{c}z" for c in letters) + "->" + letters
    T = np.einsum(spec, *([X] * m))
    if feat == 1:
        T = T ** degree
    elif feat == 2:
        T = np.exp(T)
    return T


def contract_full(T, a, times):
    """Contract the last `times` slots of T with a."""
    for _ in range(times):
        T = T @ a
    return T
