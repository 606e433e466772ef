"""Primal recovery, prediction and Nystrom selection on the GPU path against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


@pytest.mark.parametrize("m,n,d,B", [(4, 40, 10, 1), (6, 13, 7, 3), (2, 70, 300, 2)])
def test_primal_and_predict(m, n, d, B):
    X = synth.small_problem(m, n, d, salt=70 + n)
    Xt = synth.small_problem(m, 33, d, salt=71 + n)
    A = synth.alpha_like(n, salt=72, batch=B)
    W = tk.tk_primal(torch.tensor(X, device="cuda"), torch.tensor(A, device="cuda"), m).cpu().numpy()
    for b in range(B):
        w_ref = oracle.primal_from_dual(X, A[b], m)
        assert np.allclose(W[b], w_ref, rtol=1e-12, atol=1e-14 * np.abs(w_ref).max())
    Y = tk.tk_predict(torch.tensor(Xt, device="cuda"), torch.tensor(W, device="cuda")).cpu().numpy()
    for b in range(B):
        assert np.allclose(Y[b], oracle.predict(Xt, W[b]), rtol=1e-12, atol=1e-12 * np.abs(Y[b]).max())


def test_nystrom_pipeline_small():
    # Section 6.1 on a small draw: select landmarks, build over them, solve,
    # recover w and predict held-out points; compare every stage with the oracle
    c = synth.nystrom_bf16(n_train=2000, n_test=300, d=30, n_prime=40)
    idx = tk.tk_nystrom_select(2000, 40, c["select_seed"])
    assert idx == list(oracle.nystrom_select(2000, 40, c["select_seed"]))
    XL, yL = c["X_train"][idx], c["y_train"][idx]
    K = tk.tk_build_packed(torch.tensor(XL, device="cuda"), 4, storage="f64")
    A, rep, rc = tk.tk_solve_dual(K, 4, 40, torch.tensor(yL, device="cuda"), [c["lam"]], tol=1e-10)
    assert rc == tk.TK_OK
    a_ref, info = oracle.solve_dual_newton(oracle.build(XL, 4), yL, c["lam"], 4, tol=1e-10)
    assert np.linalg.norm(A[0].cpu().numpy() - a_ref) <= (rep[0]["gradnorm"] + info["gradnorm"]) / c["lam"] + 1e-12
    W = tk.tk_primal(torch.tensor(XL, device="cuda"), A[0], 4)
    yhat = tk.tk_predict(torch.tensor(c["X_test"], device="cuda"), W).cpu().numpy()
    yref = oracle.predict(c["X_test"], oracle.primal_from_dual(XL, a_ref, 4))
    assert np.allclose(yhat, yref, rtol=1e-6, atol=1e-8)
    assert oracle.mse(yhat, c["y_test"]) == pytest.approx(oracle.mse(yref, c["y_test"]), rel=1e-6)


@pytest.mark.parametrize("d,B", [(1, 1), (7, 3), (200, 2), (20_000, 1)])
def test_support_threshold_matches_oracle(d, B):
    # Section 6.3: keep |w_j| > 2 std(w); computed on the device in FP64.  The
    # draws are heavy-tailed so that some weights pass and most do not.
    rng = synth.rng_for(97, d)
    W = rng.standard_normal((B, d)) ** 3
    keep, cnt = tk.tk_support_threshold(torch.tensor(W, device="cuda"))
    keep, cnt = keep.cpu().numpy(), cnt.cpu().numpy()
    for b in range(B):
        ref = oracle.threshold_support(W[b])
        got = np.flatnonzero(keep[b])
        # a weight within rounding of the threshold could go either way
        thr = 2.0 * np.std(W[b])
        near = np.abs(np.abs(W[b]) - thr) <= 1e-12 * max(thr, 1e-300)
        assert set(got[~near[got]]) == set(ref[~near[ref]])
        assert cnt[b] == got.size
    assert tk.support_threshold(torch.tensor(W[0], device="cuda")) == list(np.flatnonzero(keep[0]))
