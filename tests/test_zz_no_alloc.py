"""tk_contract_noalloc: the contraction for callers that cannot allocate device
memory (graph capture, pre-reserved memory pools, hosts that only lend their own
tensors).  Its scratch is a static device array inside libtk; this file checks
through the C ABI that it returns what tk_contract returns, on two calls in a row
(the second call reuses the array the first one left behind).  It sits in a file
of its own, collected last."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, as_f64, contraction_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.mark.parametrize("m,n,d,storage,vdt", [(4, 37, 5, "f32", torch.float64),
                                               (6, 23, 3, "bf16", torch.float32),
                                               (4, 120, 4, "f64", torch.float64),
                                               (2, 301, 3, "f32", torch.float32)])
def test_noalloc_matches_contract(m, n, d, storage, vdt):
    X = synth.small_problem(m, n, d, salt=500 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    Kd = Kt.cuda()
    A = torch.tensor(synth.alpha_like(n, salt=501 + n), dtype=vdt, device="cuda")
    a_used = A.double().cpu().numpy()
    g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(a_used), m)
    G_ref, S_ref = tk.tk_contract(Kd, m, n, A)
    torch.cuda.synchronize()
    g_ref = G_ref.double().cpu().numpy()
    # both results carry the contraction's accumulation error; the outputs
    # are rounded to the vector type
    tol = 2 * contraction_bound(n, g_abs, storage, m)
    if vdt == torch.float32:
        tol = tol + 2 * U32 * np.abs(g_ref)
    s_tol = 2 * float(contraction_bound(n, np.array([S_abs]), storage, m)[0])
    for _ in range(2):
        G = torch.full((n,), float("nan"), dtype=vdt, device="cuda")
        S = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        tk.tk_contract_noalloc(Kd, m, n, A, G, S)
        torch.cuda.synchronize()
        g = G.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.all(np.abs(g - g_ref) <= tol), float(np.max(np.abs(g - g_ref) / tol))
        assert abs(float(S[0]) - float(S_ref[0])) <= s_tol
