"""One-pass batched contraction (B > 1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import as_f64, batched_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,d,B", [(4, 37, 4, 5), (4, 70, 3, 70), (6, 19, 3, 33), (2, 150, 3, 64), (4, 80, 2, 200),
                                     (3, 300, 2, 130), (2, 520, 2, 3)])
def test_batched_contraction_matches_oracle(m, n, d, B, storage):
    X = synth.small_problem(m, n, d, salt=800 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = synth.alpha_like(n, salt=801, batch=B)
    G, S = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(A, device="cuda"))
    G = G.cpu().numpy()
    S = S.cpu().numpy()
    pick = sorted(set([0, B - 1, B // 2, min(B - 1, 33), min(B - 1, 64)]))
    for b in pick:
        g_ref, S_ref = oracle.contract(Kr, A[b], m)
        g_abs, S_abs = oracle.contract(np.abs(Kr), np.abs(A[b]), m)
        # the batched kernel flushes its FP32 accumulators every 2048 rows
        tol = 4 * batched_bound(g_abs, storage, n)
        assert np.all(np.abs(G[b] - g_ref) <= tol), (b, float(np.max(np.abs(G[b] - g_ref) / tol)))
        assert abs(S[b] - S_ref) <= 4 * float(batched_bound(np.array([S_abs]), storage, n)[0])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,d,B", [(4, 41, 3, 9), (6, 17, 3, 40), (3, 300, 2, 64)])
def test_batched_hvp_matches_oracle(m, n, d, B, storage):
    X = synth.small_problem(m, n, d, salt=820 + n)
    Kt = round_storage(oracle.build(X, m), storage)
    Kr = as_f64(Kt)
    A = synth.alpha_like(n, salt=821, batch=B)
    V = synth.alpha_like(n, salt=822, batch=B)
    HV, _ = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(A, device="cuda"), r=m - 2,
                           V=torch.tensor(V, device="cuda"))
    HV = HV.cpu().numpy()
    for b in sorted(set([0, B // 2, B - 1])):
        ref = oracle.hvp(Kr, A[b], V[b], m)
        hab = oracle.hvp(np.abs(Kr), np.abs(A[b]), np.abs(V[b]), m)
        tol = 8 * batched_bound(hab, storage, n)
        assert np.all(np.abs(HV[b] - ref) <= tol), (b, float(np.max(np.abs(HV[b] - ref) / tol)))
