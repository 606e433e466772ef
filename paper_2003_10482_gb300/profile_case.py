"""Small, repeatable launches of one kernel, for profiler captures.

    python -m paper_2003_10482_gb300.profile_case contract --m 4 --n 350 --storage f32 --reps 5
    python -m paper_2003_10482_gb300.profile_case batched --m 4 --n 300 --B 512 --reps 3
    python -m paper_2003_10482_gb300.profile_case build --m 4 --n 300 --d 80 --reps 2
    python -m paper_2003_10482_gb300.profile_case dexter
    python -m paper_2003_10482_gb300.profile_case nystrom

The `dexter` case is the Dexter-shaped run (n = 200 points, d = 20,000
features at 0.5 % density, m = 4, FP32 storage): it times the packed build and
a full Newton-CG dual solve (build once, solve to |grad F| <= 1e-6) and
checks the solution against the closed-form gradient X (X^T a)^{o3} + lambda a - y.
The `nystrom` case runs the Nystrom configuration end to end for FP64, FP32
and BF16 storage: 600 landmarks of 50,000 points (d = 200), build, Newton-CG
solve to a 1e-7 relative gap (at most 40 iterations), primal
w = J_q(X^T a), prediction of 10,000 held-out points; it prints each
solution's objective under the FP64 tensor, test MSE, the recovered support
(|w_j| > 2 std(w)) against w*'s, and timings.

Inputs are the seeded synthetic ones of the benchmarks (X ~ U(-1, 1) rows of
the full FP32 workload, or N(0, 1) rows of the batched workload's points);
each case builds its packed tensor once, then launches the kernel `--reps`
more times after one warm-up launch (skip it with `ncu -s 1`).  Prints the
mean CUDA-event time per timed launch.
"""
from __future__ import annotations

import argparse

import torch

import paper_2003_10482_gb300 as tk
import synth


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["contract", "hvp", "batched", "batched_hvp", "build", "dexter", "nystrom"])
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--n", type=int, default=300)
    ap.add_argument("--d", type=int, default=80)
    ap.add_argument("--B", type=int, default=512)
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    if args.case == "dexter":
        return dexter()
    if args.case == "nystrom":
        return nystrom()
    if args.case in ("contract", "hvp"):
        X = synth.full_fp32()["X"][: args.n]
    else:
        X = synth.batched_path()["X"][: args.n, : args.d]
    Xd = torch.tensor(X, device="cuda")
    m, n = args.m, Xd.shape[0]
    K = tk.tk_build_packed(Xd, m, storage=args.storage)
    B = 1 if args.case in ("contract", "hvp") else args.B
    A = torch.tensor(synth.alpha_like(n, salt=1, batch=B), device="cuda")
    V = torch.tensor(synth.alpha_like(n, salt=2, batch=B), device="cuda")
    ws = tk.workspace(m, n, B)
    if args.case == "build":
        def run():
            tk.tk_build_packed(Xd, m, storage=args.storage)
    elif args.case in ("contract", "batched"):
        def run():
            tk.tk_contract(K, m, n, A, work=ws)
    else:
        def run():
            tk.tk_contract(K, m, n, A, r=m - 2, V=V, work=ws)
    run()  # warm-up: module load, work plan (the profiler's -s 1 skips this launch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(f"{args.case} m={m} n={n} B={B} {args.storage}: {ms:.3f} ms per launch "
          f"({K.numel():,} packed entries, status {tk.tk_status_read(ws)})")


def dexter() -> None:
    import time

    import numpy as np
    p = synth.dexter_like()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    n, d = X.shape
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    tk.tk_build_packed(Xd[:8], m, storage="f32")  # warm-up (module load)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    K = tk.tk_build_packed(Xd, m, storage="f32")
    e1.record()
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    A, rep, rc = tk.tk_solve_dual(K, m, n, yd, [lam], tol=1e-6, max_iter=100)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    a = A[0].cpu().numpy()
    u = X.T @ a
    g_exact = X @ u ** (m - 1) + lam * a - y
    print(f"dexter-shaped m={m} n={n} d={d} (density {np.mean(X != 0):.4f}), {K.numel():,} packed FP32 entries: "
          f"build {build_ms:.1f} ms ({2 * d * K.numel() / build_ms / 1e9:.1f} TFLOP/s at 2d flop per entry); "
          f"solve {solve_s:.3f} s, {rep[0]['iters']} Newton iterations, {rep[0]['passes']} passes, "
          f"|grad F| {rep[0]['gradnorm']:.2e} (closed form at the solution {np.linalg.norm(g_exact):.2e}), rc {rc}")


def nystrom() -> None:
    import time

    import numpy as np
    c = synth.nystrom_bf16()
    m, lam = c["m"], c["lam"]
    N = c["X_train"].shape[0]
    idx = tk.tk_nystrom_select(N, c["n_prime"], c["select_seed"])
    XL = torch.tensor(c["X_train"][idx], device="cuda")
    yL = torch.tensor(c["y_train"][idx], device="cuda")
    Xt = torch.tensor(c["X_test"], device="cuda")
    n = XL.shape[0]
    true_support = set(np.flatnonzero(c["w_true"]).tolist())
    lam_t = torch.tensor([lam], dtype=torch.float64, device="cuda")
    K64 = None
    F_ref = None
    for storage in ("f64", "f32", "bf16"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        K = tk.tk_build_packed(XL, m, storage=storage)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        A, rep, rc = tk.tk_solve_dual(K, m, n, yL, [lam], tol=0.0, rel_gap=1e-7, max_iter=40)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        if storage == "f64":
            K64 = K
            F_ref = rep[0]["F"]
        F64, _, _ = tk.tk_objective(K64, m, n, A[0].contiguous(), yL, lam_t)
        W = tk.tk_primal(XL, A[0], m)
        yhat = tk.tk_predict(Xt, W).cpu().numpy().reshape(-1)
        mse = float(np.mean((yhat - c["y_test"]) ** 2))
        sup = set(int(j) for j in tk.support_threshold(W))
        hit = len(sup & true_support)
        print(f"nystrom {storage}: {K.numel():,} entries ({K.numel() * K.element_size() / 1e9:.1f} GB); build "
              f"{t_build:.2f} s; solve {t_solve:.2f} s ({rep[0]['iters']} iterations, {rep[0]['passes']} passes, "
              f"|grad F| {rep[0]['gradnorm']:.1e}, rc {rc}); F under the FP64 tensor {float(F64[0]):.9f} "
              f"(rel. to the FP64 solve {(float(F64[0]) - F_ref) / abs(F_ref):+.1e}); test MSE {mse:.6f}; "
              f"support {len(sup)} found, {hit} of {len(true_support)} true", flush=True)
        if storage != "f64":
            del K
    torch.cuda.empty_cache()


if __name__ == "__main__":
    main()
