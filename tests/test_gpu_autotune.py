"""The autotuner picks launch configurations by measurement; results under the
tuned configuration still match the FP64 oracle within the same bounds."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import as_f64, batched_bound, contraction_bound, round_storage

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")
from paper_2003_10482_gb300 import autotune  # noqa: E402


def test_tuned_single_vector_contraction_matches_oracle():
    m, n, d = 4, 90, 3
    X = synth.small_problem(m, n, d, salt=901)
    Kt = round_storage(oracle.build(X, m), "f32")
    Kr = as_f64(Kt)
    try:
        rep = autotune.tune_contract(Kt.cuda(), m, n, reps=2,
                                     candidates=[dict(warps=16), dict(warps=12, nbuf=3), dict(schedule=2)])
        assert rep["best"] in [t[0] for t in rep["trials"]] and len(rep["trials"]) >= 2
        a = synth.alpha_like(n, salt=902)
        G, S = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(a, device="cuda"))
        g_ref, _ = oracle.contract(Kr, a, m)
        g_abs, _ = oracle.contract(np.abs(Kr), np.abs(a), m)
        # the tuned schedule may be the shared-ticket one, under which a warp
        # may enter every triangle
        tol = contraction_bound(n, g_abs, "f32", m, dynamic=True)
        assert np.all(np.abs(G.cpu().numpy() - g_ref) <= tol)
        assert autotune.apply("contract", m, n, "f32")
    finally:
        tk.tk_contract_set_config(reset=True)


def test_tuned_batched_contraction_matches_oracle():
    m, n, d, B = 4, 80, 2, 64
    X = synth.small_problem(m, n, d, salt=903)
    Kt = round_storage(oracle.build(X, m), "f32")
    Kr = as_f64(Kt)
    try:
        rep = autotune.tune_batched(Kt.cuda(), m, n, B, reps=1,
                                    candidates=[dict(vpl=1), dict(vpl=2, nbuf=2), dict(vpl=2, slice_mult=2)])
        best = rep["best"]
        assert best["min_batch"] >= 2 and len(rep["trials"]) >= 2
        A = synth.alpha_like(n, salt=904, batch=B)
        G, S = tk.tk_contract(Kt.cuda(), m, n, torch.tensor(A, device="cuda"))
        G = G.cpu().numpy()
        for b in (0, B // 2, B - 1):
            g_ref, _ = oracle.contract(Kr, A[b], m)
            g_abs, _ = oracle.contract(np.abs(Kr), np.abs(A[b]), m)
            assert np.all(np.abs(G[b] - g_ref) <= batched_bound(g_abs, "f32", n, m))
    finally:
        tk.tk_batched_set_config(reset=True)
