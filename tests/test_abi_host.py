"""Host-side checks of libtk that need no GPU: the library loads, exports every
symbol include/tk.h declares, and its layout helpers agree with the oracle."""
import subprocess

import numpy as np
import pytest

import oracle

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.fixture(scope="module")
def L():
    try:
        return tk.lib()
    except ImportError:
        from paper_2003_10482_gb300 import build_lib
        build_lib.build()
        return tk.lib()


def test_exports_every_declared_symbol(L):
    declared = tk.exported_symbols()
    assert "tk_contract" in declared and "tk_build_packed" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", tk.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(L, s)


@pytest.mark.parametrize("m,n", [(1, 5), (2, 9), (3, 7), (4, 40), (4, 400), (6, 80), (4, 600), (8, 12)])
def test_packed_size(L, m, n):
    assert tk.tk_packed_size(m, n) == oracle.packed_size(m, n)
    assert tk.tk_packed_bytes(m, n, "bf16") == 2 * oracle.packed_size(m, n)


def test_packed_size_overflow_and_errors(L):
    assert L.tk_packed_size(8, 10**9) == -1
    assert L.tk_packed_size(0, 5) == -1
    assert L.tk_packed_size(4, -1) == -1
    with pytest.raises(tk.TKError):
        tk.tk_rank(4, 5, [0, 2, 1, 3])       # not sorted
    with pytest.raises(tk.TKError):
        tk.tk_unrank(4, 5, tk.tk_packed_size(4, 5))  # offset == N


@pytest.mark.parametrize("m,n", [(2, 7), (3, 6), (4, 6), (6, 5), (8, 3)])
def test_rank_unrank_bit_exact(L, m, n):
    tuples = oracle.enumerate_tuples(m, n)
    for off, t in enumerate(tuples):
        assert tk.tk_rank(m, n, t) == off
        assert tk.tk_unrank(m, n, off) == list(t)


@pytest.mark.parametrize("m,n", [(4, 400), (4, 600), (6, 80), (4, 300), (2, 1000)])
def test_rank_unrank_config_sizes(L, m, n):
    N = oracle.packed_size(m, n)
    rng = np.random.default_rng(5)
    for off in list(rng.integers(0, N, size=200)) + [0, N - 1, N // 2]:
        t = tk.tk_unrank(m, n, int(off))
        assert t == list(oracle.unrank(m, n, int(off)))
        assert tk.tk_rank(m, n, t) == off


def test_row_align(L):
    m, n = 4, 7
    tuples = oracle.enumerate_tuples(m, n)
    N = len(tuples)
    starts = [o for o, t in enumerate(tuples) if t[-1] == t[-2]] + [N]
    for off in range(N + 1):
        want = min(s for s in starts if s >= off)
        assert tk.tk_row_align(m, n, off) == want


def _row_costs(m, n, lo, hi, rc, tc):
    """(offset, cost) of every row start in [lo, hi), by enumeration."""
    tuples = oracle.enumerate_tuples(m, n)
    rows = []
    prev_q = None
    for o in range(lo, hi):
        t = tuples[o]
        if t[-1] == t[-2]:
            q = tuple(t[:-2])
            cost = (n - t[-2]) + rc + (tc if q != prev_q else 0)
            rows.append((o, cost))
            prev_q = q
    return rows


@pytest.mark.parametrize("m,n,pieces", [(4, 9, 7), (2, 30, 5), (6, 6, 13), (4, 12, 40), (3, 10, 3)])
def test_contract_plan_is_row_aligned_and_balanced(L, m, n, pieces):
    N = tk.tk_packed_size(m, n)
    for lo, hi in ((0, N), (tk.tk_row_align(m, n, N // 3), tk.tk_row_align(m, n, (2 * N) // 3))):
        rc, tc = 5, 11
        b = tk.tk_contract_plan(m, n, lo, hi, pieces, rc, tc)
        assert b[0] == lo and b[-1] == hi and len(b) == pieces + 1
        assert all(x <= y for x, y in zip(b[:-1], b[1:]))
        rows = _row_costs(m, n, lo, hi, rc, tc)
        starts = {o for o, _ in rows} | {hi}
        assert all(x in starts for x in b)
        total = sum(c for _, c in rows)
        big = max(c for _, c in rows) if rows else 0
        for x, y in zip(b[:-1], b[1:]):
            piece = sum(c for o, c in rows if x <= o < y)
            assert piece <= total / pieces + big + tc


@pytest.mark.parametrize("N,np_,seed", [(50_000, 600, 2003_10485), (20_000, 300, 2003_10486), (7, 3, 1),
                                        (10, 10, 5), (10, 0, 5), (1, 1, 0), (1000, 999, 2**63 + 7)])
def test_nystrom_select_matches_oracle(L, N, np_, seed):
    assert tk.tk_nystrom_select(N, np_, seed) == list(oracle.nystrom_select(N, np_, seed))


def test_nystrom_select_rejects_bad_sizes(L):
    with pytest.raises(tk.TKError):
        tk.tk_nystrom_select(5, 6, 1)


def test_batched_config_validation():
    tk = pytest.importorskip("paper_2003_10482_gb300")
    for bad in (dict(vpl=3), dict(block_bytes=1000), dict(block_bytes=4100), dict(nbuf=5), dict(slice_mult=3),
                dict(min_batch=-1), dict(tensor_cores=2), dict(tensor_cores=-2)):
        with pytest.raises(tk.TKError):
            tk.tk_batched_set_config(**bad)
    tk.tk_batched_set_config(vpl=1, block_bytes=8320, nbuf=2, slice_mult=2, min_batch=4, tensor_cores=-1)
    tk.tk_batched_set_config(reset=True)
