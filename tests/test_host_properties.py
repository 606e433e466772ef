"""Property-based checks (no GPU): the library's host logic -- the ranking
bijection, row alignment and the cost-balanced cut of a range, on random
orders, point counts, offsets and piece counts -- and the oracle's packed
contraction and HVP against the dense n^m tensor on random tiny data."""
import math

import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

tk = pytest.importorskip("paper_2003_10482_gb300")


def _lib_or_skip():
    try:
        tk.lib()
    except ImportError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(str(e))


@settings(max_examples=200, deadline=None)
@given(m=st.integers(1, 8), n=st.integers(1, 60), u=st.floats(0.0, 1.0, exclude_max=True))
def test_rank_unrank_roundtrip_and_order(m, n, u):
    _lib_or_skip()
    N = tk.tk_packed_size(m, n)
    assert N == math.comb(n + m - 1, m)
    off = int(u * N)
    t = tk.tk_unrank(m, n, off)
    assert all(0 <= a <= b < n for a, b in zip(t[:-1], t[1:])) and 0 <= t[0] and t[-1] < n
    assert tk.tk_rank(m, n, t) == off
    assert t == list(oracle.unrank(m, n, off))
    if off + 1 < N:  # lexicographic successor
        assert tuple(tk.tk_unrank(m, n, off + 1)) > tuple(t)


@settings(max_examples=200, deadline=None)
@given(m=st.integers(2, 6), n=st.integers(1, 40), u=st.floats(0.0, 1.0))
def test_row_align_gives_the_next_row_start(m, n, u):
    _lib_or_skip()
    N = tk.tk_packed_size(m, n)
    off = int(u * N)
    r = tk.tk_row_align(m, n, off)
    assert off <= r <= N
    if r < N:
        t = tk.tk_unrank(m, n, r)
        assert t[-1] == t[-2]  # a row starts where the last two indices meet
    for o in range(off, min(r, off + 64)):  # nothing between off and r starts a row
        t = tk.tk_unrank(m, n, o)
        assert t[-1] != t[-2]


@settings(max_examples=120, deadline=None)
@given(m=st.integers(2, 6), n=st.integers(1, 30), pieces=st.integers(1, 64), a=st.floats(0.0, 1.0),
       b=st.floats(0.0, 1.0), rc=st.integers(1, 512), tc=st.integers(0, 4096))
def test_plan_cuts_are_ordered_row_starts(m, n, pieces, a, b, rc, tc):
    _lib_or_skip()
    N = tk.tk_packed_size(m, n)
    lo = tk.tk_row_align(m, n, int(min(a, b) * N))
    hi = tk.tk_row_align(m, n, int(max(a, b) * N))
    cuts = tk.tk_contract_plan(m, n, lo, hi, pieces, rc, tc)
    assert len(cuts) == pieces + 1 and cuts[0] == lo and cuts[-1] == hi
    assert all(x <= y for x, y in zip(cuts[:-1], cuts[1:]))
    for c in cuts:
        assert c == N or tk.tk_row_align(m, n, c) == c


@settings(max_examples=60, deadline=None)
@given(m=st.integers(2, 5), n=st.integers(1, 5), d=st.integers(1, 3), seed=st.integers(0, 2**31 - 1))
def test_oracle_contraction_equals_the_full_tensor(m, n, d, seed):
    # the packed contraction (multiplicity-weighted) against the dense n^m tensor, any data
    import numpy as np

    from brute import contract_full, full_tensor
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    a = rng.standard_normal(n)
    v = rng.standard_normal(n)
    K = oracle.build(X, m)
    g, S = oracle.contract(K, a, m)
    T = full_tensor(X, m)
    g_ref = contract_full(T, a, m - 1)
    scale = max(1.0, float(np.abs(g_ref).max()))
    assert np.allclose(g, g_ref, rtol=1e-11, atol=1e-11 * scale)
    assert abs(S - float(g_ref @ a)) <= 1e-11 * max(1.0, abs(float(g_ref @ a)))
    hv_ref = contract_full(T, a, m - 2) @ v
    assert np.allclose(oracle.hvp(K, a, v, m), hv_ref, rtol=1e-11, atol=1e-11 * max(1.0, float(np.abs(hv_ref).max())))
