"""Pins of the oracle's packed layout against the thesis (Section 5) and brute force."""
import itertools
import math

import numpy as np
import pytest

import oracle


def test_entry_count_table(golden):
    # Section 5, Table t_size: n^2/b_mat, n^3/b_cube, n^4/b_tensor4 and %reduce
    for row in golden("t_size.txt"):
        n = int(row[0])
        vals = [float(v) for v in row[1:]]
        for k, m in enumerate((2, 3, 4)):
            full, packed, reduce_pct = vals[3 * k], vals[3 * k + 1], vals[3 * k + 2]
            assert n ** m == full
            assert oracle.packed_size(m, n) == packed
            assert round(100.0 * (1.0 - packed / full), 2) == pytest.approx(reduce_pct, abs=1e-9)


def test_entry_count_table_by_enumeration(golden):
    # the same counts reached by walking the nested loops (small n only)
    for row in golden("t_size.txt"):
        n = int(row[0])
        if n > 30:
            continue
        for m, col in ((2, 2), (3, 5), (4, 8)):
            assert oracle.enumerate_tuples(m, n).shape[0] == int(float(row[col]))


def test_counts_quoted_in_text(golden):
    for kind, n, val in golden("entry_counts.txt"):
        n = int(n)
        if kind == "full":
            assert n ** 4 == int(val)
        elif kind == "packed":
            assert oracle.packed_size(4, n) == int(val)
        elif kind == "packed_min":
            assert oracle.packed_size(4, n) > int(val)
        elif kind == "packed_max":
            assert oracle.packed_size(4, n) < int(val)
        elif kind == "old_matrix_GB":
            assert (n * n) ** 2 * 8 / 2 ** 30 == pytest.approx(float(val), abs=0.005)
        elif kind == "max_points_full_8GB":
            lim = 8 * 2 ** 30
            assert int(val) ** 4 * 8 <= lim < (int(val) + 1) ** 4 * 8
        elif kind == "max_points_packed_8GB":
            lim = 8 * 2 ** 30
            k = int(val)
            assert oracle.packed_size(4, k) * 8 <= lim < oracle.packed_size(4, k + 1) * 8


def test_memory_gain(golden):
    # Section 5.1: n^4 * 8 B and C(n+3,4) * 8 B in units of 2^30 bytes
    for n, full_gb, packed_gb, rel in golden("memory_gain.txt"):
        n = int(n)
        assert n ** 4 * 8 / 2 ** 30 == pytest.approx(float(full_gb), rel=0.005)
        assert oracle.packed_size(4, n) * 8 / 2 ** 30 == pytest.approx(float(packed_gb),
                                                                         rel=float(rel))


def test_index_2d_worked_example(golden):
    # Section 5, eqs. index_2d / skip_2d worked on a 9 x 9 matrix
    for n, r, c, full, skip, packed in golden("index_2d.txt"):
        n, r, c = int(n), int(r), int(c)
        assert r * n + c == int(full)
        assert r * (r + 1) // 2 == int(skip)
        assert oracle.rank(2, n, [r, c]) == int(packed)


def _thesis_index_formulas(n):
    """v_2d, v_3d, v_4d as printed in Section 5 (eqs. index_2d, v3d, skip_3d, v4d),
    with the readings this build takes where the print is inconsistent:
    skip_3d(0) = 0 as the base case, the cube tuple read as (d <= r <= c), and
    t * n^3 in v_4d where the print has t * n^4."""
    skip2 = lambda r: r * (r + 1) // 2
    v2 = lambda r, c: r * n - skip2(r) + c
    s3 = {0: 0}
    for d in range(1, n + 1):
        s3[d] = n * n - (n - d) ** 2 + skip2(n - d - 1) + s3[d - 1]
    v3 = lambda r, c, d: d * n * n - s3[d] + v2(r, c)
    s3inv = {n: 0}
    for d in range(n - 1, -1, -1):
        s3inv[d] = n * n - (n - d) ** 2 + skip2(n - d - 1) + s3inv[d + 1]
    s4 = {0: 0}
    for t in range(1, n + 1):
        s4[t] = t * n * n + s3inv[t] + s4[t - 1]
    v4 = lambda r, c, d, t: t * n ** 3 - s4[t] + v3(r, c, d)
    return v2, v3, v4


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_rank_matches_thesis_formulas(n):
    v2, v3, v4 = _thesis_index_formulas(n)
    for r, c in itertools.combinations_with_replacement(range(n), 2):
        assert oracle.rank(2, n, [r, c]) == v2(r, c)
    for d, r, c in itertools.combinations_with_replacement(range(n), 3):
        assert oracle.rank(3, n, [d, r, c]) == v3(r, c, d)
    for t, d, r, c in itertools.combinations_with_replacement(range(n), 4):
        assert oracle.rank(4, n, [t, d, r, c]) == v4(r, c, d, t)


@pytest.mark.parametrize("m,n", [(1, 5), (2, 7), (3, 6), (4, 6), (5, 4), (6, 5), (8, 3)])
def test_enumeration_is_nested_loop_order(m, n):
    # Python's combinations_with_replacement yields exactly the nested loops
    # i_1 <= i_2 <= ... with the first index slowest
    ref = np.array(list(itertools.combinations_with_replacement(range(n), m)), dtype=np.int32)
    got = oracle.enumerate_tuples(m, n)
    assert np.array_equal(got, ref)
    for off, t in enumerate(ref):
        assert oracle.rank(m, n, t) == off
        assert np.array_equal(oracle.unrank(m, n, off), t)


def test_rank_large_sizes_against_sums():
    # at configuration sizes: first/last tuples, and rank of a row start equals
    # the count of tuples with a smaller prefix (hand-summed with math.comb)
    for m, n in ((4, 400), (4, 603 - 3), (6, 80), (4, 300)):
        N = oracle.packed_size(m, n)
        assert oracle.rank(m, n, [0] * m) == 0
        assert oracle.rank(m, n, [n - 1] * m) == N - 1
        assert list(oracle.unrank(m, n, N - 1)) == [n - 1] * m
        # tuples whose first index is < a: sum over v < a of C(n - v + m - 2, m - 1)
        for a in (1, n // 3, n - 1):
            want = sum(math.comb(n - v + m - 2, m - 1) for v in range(a))
            assert oracle.rank(m, n, [a] * m) == want


def test_multiplicities_count_all_full_tuples():
    # sum over stored tuples of the number of orderings = n^m
    for m, n in ((2, 6), (4, 5), (6, 4), (3, 7)):
        tot = 0
        for t in oracle.enumerate_tuples(m, n):
            _, cnt = np.unique(t, return_counts=True)
            tot += math.factorial(m) // int(np.prod([math.factorial(c) for c in cnt]))
        assert tot == n ** m
