"""tk_contract_noalloc: the contraction for callers that cannot allocate device
memory -- code recorded into a CUDA graph (an allocation cannot be captured),
runtimes whose device memory is all reserved up front, hosts that only lend the
library their own tensors.  Its scratch is a static device array inside libtk.

Checked here, through the C ABI: the result against the FP64 oracle on two
calls in a row (the second reuses what the first left in the array); that a
call allocates no device memory; that a call recorded into a CUDA graph replays
correctly, and that a replay after the array was re-planned for another shape
writes nothing and reports it; that a first call under capture is refused
without breaking the capture; that a launch whose scratch does not fit is
refused.  The file is collected last, so a run that stops at the first failure
has run every other test before it."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, as_f64, contraction_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


def _case(m, n, d, storage, vdt, salt):
    X = synth.small_problem(m, n, d, salt=salt)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = torch.tensor(synth.alpha_like(n, salt=salt + 1), dtype=vdt, device="cuda")
    a_used = A.double().cpu().numpy()  # the vector the kernel sees
    g_ref, S_ref = oracle.contract(Kr, a_used, m)
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a_used), m)
    tol = contraction_bound(n, g_abs, storage, m)
    if vdt == torch.float32:  # G is rounded to the vector type on output
        tol = tol + U32 * np.abs(g_ref)
    s_tol = float(contraction_bound(n, np.array([S_abs]), storage, m)[0])
    return Kt.cuda(), A, g_ref, S_ref, tol, s_tol


def _check(G, S, g_ref, S_ref, tol, s_tol):
    g = G.double().cpu().numpy()
    assert np.all(np.isfinite(g))
    assert np.all(np.abs(g - g_ref) <= tol), float(np.max(np.abs(g - g_ref) / tol))
    assert abs(float(S[0]) - S_ref) <= s_tol


@pytest.mark.parametrize("m,n,d,storage,vdt", [(4, 37, 5, "f32", torch.float64),
                                               (6, 23, 3, "bf16", torch.float32),
                                               (4, 120, 4, "f64", torch.float64),
                                               (2, 301, 3, "f32", torch.float32)])
def test_noalloc_matches_oracle_twice(m, n, d, storage, vdt):
    Kd, A, g_ref, S_ref, tol, s_tol = _case(m, n, d, storage, vdt, salt=500 + n)
    for _ in range(2):
        G = torch.full((n,), float("nan"), dtype=vdt, device="cuda")
        S = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        tk.tk_contract_noalloc(Kd, m, n, A, G, S)
        torch.cuda.synchronize()
        _check(G, S, g_ref, S_ref, tol, s_tol)
    assert tk.tk_contract_noalloc_status() == tk.TK_OK


def test_noalloc_allocates_no_device_memory():
    m, n = 4, 64
    Kd, A, g_ref, S_ref, tol, s_tol = _case(m, n, 4, "f32", torch.float64, salt=510)
    G = torch.empty(n, dtype=torch.float64, device="cuda")
    S = torch.empty(1, dtype=torch.float64, device="cuda")
    tk.tk_contract_noalloc(Kd, m, n, A, G, S)  # first call: loads the kernel, plans the scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        tk.tk_contract_noalloc(Kd, m, n, A, G, S)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check(G, S, g_ref, S_ref, tol, s_tol)


def test_noalloc_graph_replay_and_stale_plan():
    m, n = 4, 45
    Kd, A, g_ref, S_ref, tol, s_tol = _case(m, n, 4, "f32", torch.float64, salt=520)
    G = torch.empty(n, dtype=torch.float64, device="cuda")
    S = torch.empty(1, dtype=torch.float64, device="cuda")
    tk.tk_contract_noalloc(Kd, m, n, A, G, S)  # plans the scratch outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tk.tk_contract_noalloc(Kd, m, n, A, G, S)
    G.fill_(float("nan"))
    S.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    _check(G, S, g_ref, S_ref, tol, s_tol)
    assert tk.tk_contract_noalloc_status() == tk.TK_OK

    # another shape re-plans the scratch; the old graph must not read that plan
    m2, n2 = 4, 29
    Kd2, A2, g_ref2, S_ref2, tol2, s_tol2 = _case(m2, n2, 3, "f32", torch.float64, salt=530)
    G2 = torch.empty(n2, dtype=torch.float64, device="cuda")
    S2 = torch.empty(1, dtype=torch.float64, device="cuda")
    tk.tk_contract_noalloc(Kd2, m2, n2, A2, G2, S2)
    torch.cuda.synchronize()
    _check(G2, S2, g_ref2, S_ref2, tol2, s_tol2)
    G.fill_(float("nan"))
    S.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.isnan(G).all() and torch.isnan(S).all()  # nothing written
    assert tk.tk_contract_noalloc_status() == tk.TK_EINVAL
    assert tk.tk_contract_noalloc_status() == tk.TK_OK  # reading clears it

    # re-planned for the first shape outside capture, the graph works again
    tk.tk_contract_noalloc(Kd, m, n, A, G, S)
    G.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    _check(G, S, g_ref, S_ref, tol, s_tol)


def test_noalloc_first_call_under_capture_is_refused():
    m, n = 4, 53  # a shape no earlier call used: the scratch would need a new plan
    Kd, A, g_ref, S_ref, tol, s_tol = _case(m, n, 3, "f32", torch.float64, salt=540)
    G = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(graph):
        try:
            tk.tk_contract_noalloc(Kd, m, n, A, G, S)
        except tk.TKError as e:
            refused = e
    # the refusal issued nothing, so the capture ended without being invalidated
    assert refused is not None and refused.code == tk.TK_EINVAL
    tk.tk_contract_noalloc(Kd, m, n, A, G, S)
    torch.cuda.synchronize()
    _check(G, S, g_ref, S_ref, tol, s_tol)


def test_noalloc_scratch_too_small_is_refused():
    m, n = 4, 37
    Kd, A, *_ = _case(m, n, 3, "f32", torch.float64, salt=550)
    G = torch.empty(n, dtype=torch.float64, device="cuda")
    try:
        # two blocks per SM double the work plan beyond the static array's records
        tk.tk_contract_set_config(ctas_per_sm=2)
        with pytest.raises(tk.TKError) as e:
            tk.tk_contract_noalloc(Kd, m, n, A, G)
        assert e.value.code == tk.TK_ENOMEM
    finally:
        tk.tk_contract_set_config(reset=True)
