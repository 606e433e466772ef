"""Benchmark of the packed tensor-kernel hot path on GB300.

Workload: the full-tensor FP32 configuration -- order m = 4, n = 400 points,
d = 100 features, X ~ U(-1, 1) (seeded), linear tensor kernel; the packed
tensor has C(403, 4) = 1,082,740,100 FP32 entries (4.33 GB, far above the
129 MB L2, so no flush between steps is needed).

One step = one dual-solver iteration's pass over the packed tensor:
tk_objective, i.e. the streaming contraction kernel (K[a^3] and K[a^4] in one
read of K) followed by the FP64 assembly of F, grad F and |grad F| on the
device.  value = algorithmic bytes streamed per step (N x 4 B) / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (the only reference: the thesis
ships no runnable code) on bounded samples of the same workload, on the host
cores.  Under torchrun (N > 1) every rank builds and contracts its own
row-aligned shard and the partial contractions are summed with one NCCL
all-reduce per step; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("packed K[α^{m−1}] contraction HBM GB/s (% of peak); "
          "dual solves/sec batched vs plain FP64")
WORKLOAD = "full_fp32_m4_n400_d100"
FALLBACK_HBM_GBS = 6800.0


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _kernel_hash() -> str:
    h = hashlib.sha256()
    for name in ("tk_contract_impl.cuh", "tk_contract.cu"):
        with open(os.path.join(ROOT, "paper_2003_10482_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profile_traffic(bytes_per_launch_alg: float):
    """dram traffic per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "contract_full_fp32_n400.json")
    try:
        with open(path) as f:
            prof = json.load(f)
    except Exception:
        return None
    if prof.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    return prof.get("dram_bytes_per_launch")


def _oracle_sample(target_s: float, max_entries: int = 40_000_000):
    """Calibrate the oracle's contraction rate, then build (untimed) a prefix
    sample of the packed tensor sized for about target_s seconds of work."""
    import oracle
    import synth
    p = synth.full_fp32()
    X, m = p["X"], p["m"]
    a = synth.alpha_like(X.shape[0], salt=1)
    K0 = oracle.build(X, m, 0, 100_000)
    t0 = time.perf_counter()
    oracle.contract(K0, a, m)
    rate = 100_000 / max(time.perf_counter() - t0, 1e-6)
    S = int(min(max(rate * target_s, 10_000), max_entries))
    # the sample is built on every host thread (untimed setup)
    import concurrent.futures as cf

    import numpy as np
    T = _host_threads()
    cuts = [S * i // T for i in range(T + 1)]
    with cf.ThreadPoolExecutor(max_workers=T) as ex:
        parts = list(ex.map(lambda i: oracle.build(X, m, cuts[i], cuts[i + 1]), range(T)))
    return np.concatenate(parts), a, m


def _time_oracle(K, a, m, threads: int = 1):
    """Wall time of the oracle's contraction of K (as it stands), on `threads`
    host threads each contracting one contiguous chunk (the C oracle releases
    the interpreter lock while it runs; the chunk sums are added afterwards)."""
    import concurrent.futures as cf

    import oracle
    t0 = time.perf_counter()
    if threads <= 1:
        oracle.contract(K, a, m)
    else:
        N = K.shape[0]
        cuts = [N * i // threads for i in range(threads + 1)]
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            parts = list(ex.map(lambda i: oracle.contract(K[cuts[i]:cuts[i + 1]], a, m, lo=cuts[i]),
                                range(threads)))
        g = sum(pp[0] for pp in parts)
        S = sum(pp[1] for pp in parts)
        del g, S
    return time.perf_counter() - t0


def _host_threads() -> int:
    return len(os.sched_getaffinity(0))


def _sample_text(S, threads):
    return (f"first {S:,} packed entries of the n=400 m=4 tensor (built by the oracle, untimed); "
            f"FP64 oracle contraction K[a^3] and K[a^4] on {threads} host thread(s), contiguous chunks; "
            f"value = entries/s x 4 B (the FP32 storage the GPU streams)")


def _config():
    """The workload both arms report (the reference arm runs it on samples)."""
    import math
    N = math.comb(400 + 3, 4)
    return {"workload": WORKLOAD, "m": 4, "n": 400, "d": 100, "storage": "f32", "packed_entries": N,
            "packed_bytes": N * 4}


def cpu_baseline_leg(target_s: float = 2.5) -> dict:
    """The FP64 oracle's contraction on a prefix of the same packed tensor, on
    all host cores and on one; and the oracle's full dual solve of the plain
    FP64 configuration."""
    import oracle
    import synth
    K, a, m = _oracle_sample(target_s)
    T = _host_threads()
    dt1 = _time_oracle(K, a, m, 1)
    dtT = _time_oracle(K, a, m, T)
    c1 = synth.plain_fp64()
    Kc1 = oracle.build(c1["X"], c1["m"])
    t0 = time.perf_counter()
    _, info = oracle.solve_dual_newton(Kc1, c1["y"], c1["lam"], c1["m"], tol=1e-10)
    solve_s = time.perf_counter() - t0
    return {"value": K.shape[0] / dtT * 4 / 1e9, "unit": "GB/s", "cores": T, "kind": "oracle",
            "sample": _sample_text(K.shape[0], T), "entries_per_s": K.shape[0] / dtT, "seconds": dtT,
            "single_thread": {"value": K.shape[0] / dt1 * 4 / 1e9, "unit": "GB/s", "seconds": dt1},
            "host_cores": os.cpu_count(), "affinity_cores": T,
            "oracle_solve_plain_fp64": {"seconds": solve_s, "newton_iterations": info["iters"],
                                        "gradnorm": info["gradnorm"],
                                        "workload": "plain FP64: m=4, n=40, d=10, dense-Hessian Newton to 1e-10"}}


def run_reference(args) -> None:
    """Reference arm: the oracle on all host cores, one bounded sample per step,
    the whole run sized to about half a minute of timed work."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    steps = max(args.steps, 1)
    T = _host_threads()
    K, a, m = _oracle_sample(max(0.02, 30.0 * T / steps))
    for _ in range(args.warmup):
        _time_oracle(K[: max(1, K.shape[0] // 10)], a, m, T)
    times = [_time_oracle(K, a, m, T) for _ in range(steps)]
    per = statistics.mean(times)
    v = K.shape[0] / per * 4 / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * per,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": T, "kind": "oracle",
                             "sample": _sample_text(K.shape[0], T)},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(dev) -> dict:
    """Dual solves/s of the batched FP32 path against plain FP64 solves, on the
    whole lambda path, and the batched contraction pass behind it.

    Workload: m = 4, n' = 300 Nystrom landmarks (uniform without replacement,
    tk_nystrom_select) of 20,000 points, d = 80; lambda in logspace(-4, 0, 64)
    x 8 cross-validation folds (masks) = 512 problems.  Both arms use the
    full-Hessian Newton method (FP64 Cholesky on the device) to the same
    relative-gap target (1e-7), at most 30 iterations, and the same
    continuation along the path: the 64 lambdas are taken largest first in 8
    stages of 8; stage 0 starts from the best multiple of y, every later
    problem from the same fold's solution at the previous stage's smallest
    lambda.  Batched = one tk_solve_dual call per stage over its 64 problems
    on the FP32 tensor (objective and gradient of the active problems from one
    batched contraction pass, the Newton matrix of each new point from its
    Hessian pass); plain = one call per problem on the FP64 tensor (F, grad F
    and the Newton matrix all from FP64 passes), for fold 0 of every lambda
    (64 problems).  A problem whose Newton matrix fails to factorise stops
    there (its stored tensor's rounding has made the form indefinite).  Accuracy: F of
    each fold-0 batched solution under the FP64 tensor against its plain FP64
    solve, per lambda, with the convergence and passes of every fold."""
    import torch

    import paper_2003_10482_gb300 as tk
    import synth
    p = synth.batched_path()
    m = p["m"]
    idx = tk.tk_nystrom_select(p["X"].shape[0], p["n_prime"], p["select_seed"])
    X = torch.tensor(p["X"][idx], device=dev)
    y = torch.tensor(p["y"][idx], device=dev)
    n = X.shape[0]
    lam = torch.tensor(p["lambdas"], device=dev)
    mask = torch.tensor(p["masks"], device=dev)
    B = lam.numel()
    folds, nlam = 8, B // 8
    K32 = tk.tk_build_packed(X, m, storage="f32")
    K64 = tk.tk_build_packed(X, m, storage="f64")
    gap, iters = 1e-7, 30

    # the batched contraction pass itself at B = 512: tensor cores vs SIMT
    A512 = torch.tensor(synth.alpha_like(n, salt=5, batch=B), device=dev)
    passes = {}
    for mode, name in ((1, "tensor_cores"), (-1, "simt")):
        tk.tk_batched_set_config(tensor_cores=mode)
        tk.tk_contract(K32, m, n, A512)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            tk.tk_contract(K32, m, n, A512)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 3
        passes[name] = {"ms": ms, "tflops": 4.0 * B * K32.numel() / ms / 1e9}
    tk.tk_batched_set_config(reset=True)
    tf32_peak = 1879.2 * 1.1 / 2.25  # measured bf16 burst x nominal TF32/BF16 ratio
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            tf32_peak = json.load(f)["bf16_tflops"] * 1.1 / 2.25
    except (OSError, KeyError, ValueError):
        pass
    contraction = {"B": B, "entries": int(K32.numel()), "flops_per_entry": 4 * B, **passes,
                   "speedup_tensor_cores": passes["simt"]["ms"] / passes["tensor_cores"]["ms"],
                   "tf32_peak_tflops": tf32_peak,
                   "frac_of_tf32_peak": passes["tensor_cores"]["tflops"] / tf32_peak,
                   "peak_note": "measured bf16 burst x nominal TF32/BF16 ratio (1.1 / 2.25); the pass does 3 TF32 "
                                "products per FP32 product (the split), so useful flops are a third of the tensor work"}

    order = list(range(nlam - 1, -1, -1))           # lambda indices, largest first
    stages = [order[k:k + 8] for k in range(0, nlam, 8)]
    def probs(st):
        return [8 * i + f for i in st for f in range(folds)]

    # warm-up (library load, plans, workspaces) on the problems of each arm's
    # first timed call, two iterations deep so that the Newton-matrix path runs
    w0 = probs(stages[0])
    tk.tk_solve_dual(K32, m, n, y, lam[w0], mask=mask[w0], method="newton_full", tol=0.0, rel_gap=gap,
                     max_iter=2, K_hvp=K32, start_on_y=True)
    j0 = 8 * stages[0][0]
    tk.tk_solve_dual(K64, m, n, y, lam[j0:j0 + 1], mask=mask[j0:j0 + 1], method="newton_full", tol=0.0,
                     rel_gap=gap, max_iter=2, K_hvp=K64, start_on_y=True)
    torch.cuda.synchronize()

    # batched arm: one call per stage
    A32 = torch.zeros(B, n, dtype=torch.float64, device=dev)
    rep = [None] * B
    t_batched = 0.0
    t_stage_b, t_stage_p = [], []
    prev = None
    for st in stages:
        js = probs(st)
        a0 = None if prev is None else torch.stack([A32[8 * prev + (j % 8)] for j in js])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A, r, _ = tk.tk_solve_dual(K32, m, n, y, lam[js], alpha0=a0, mask=mask[js], method="newton_full", tol=0.0,
                                   rel_gap=gap, max_iter=iters, K_hvp=K32, start_on_y=prev is None)
        torch.cuda.synchronize()
        t_stage_b.append(time.perf_counter() - t0)
        t_batched += t_stage_b[-1]
        A32[js] = A
        for j, rr in zip(js, r):
            rep[j] = rr
        prev = st[-1]
    # plain FP64 arm: fold 0, one problem per call, the same starts
    t_plain, F64, rep64 = 0.0, {}, {}
    A64 = {}
    prev = None
    for st in stages:
        t_stage_p.append(0.0)
        for i in st:
            j = 8 * i
            a0 = None if prev is None else A64[8 * prev].reshape(1, n)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A, r64, _ = tk.tk_solve_dual(K64, m, n, y, lam[j:j + 1], alpha0=a0, mask=mask[j:j + 1],
                                         method="newton_full", tol=0.0, rel_gap=gap, max_iter=iters, K_hvp=K64,
                                         start_on_y=prev is None)
            torch.cuda.synchronize()
            t_stage_p[-1] += time.perf_counter() - t0
            t_plain += time.perf_counter() - t0
            A64[j] = A[0]
            F64[j] = r64[0]["F"]
            rep64[j] = r64[0]
        prev = st[-1]
    plain = sorted(F64)
    # the batched solutions of those problems judged under the FP64 tensor
    Fb, _, _ = tk.tk_objective(K64, m, n, A32[plain].contiguous(), y, lam[plain].contiguous())
    Fb = Fb.cpu().numpy()
    errs = {j: abs(float(Fb[i]) - F64[j]) / max(abs(F64[j]), 1e-300) for i, j in enumerate(plain)}
    per_lambda = []
    lam_h = p["lambdas"]
    for i in range(nlam):
        js = range(8 * i, 8 * i + 8)
        per_lambda.append({"lambda": float(lam_h[8 * i]),
                           "rel_obj_diff_vs_fp64_fold0": errs[8 * i],
                           "fp32_reaches_fp64_within_1e-6": errs[8 * i] <= 1e-6,
                           "fp64_fold0_converged": rep64[8 * i]["status"] == 0,
                           "fp64_fold0_passes": rep64[8 * i]["passes"],
                           "fp32_converged_folds": sum(rep[j]["status"] == 0 for j in js),
                           "fp32_passes_max": max(rep[j]["passes"] for j in js)})
    ok = [j for j in plain if errs[j] <= 1e-6]
    lam_ok = [float(lam_h[j]) for j in ok]
    held_out = float(A32[~mask.bool()].abs().max()) if bool((~mask.bool()).any()) else 0.0
    # equal accuracy: the lambdas whose FP32 solutions reach the FP64 objective,
    # and the stages made only of such lambdas (timed as a whole in both arms)
    ok_set = {j // 8 for j in ok}
    eq_b = [j for j in range(B) if j // 8 in ok_set]
    eq_stages = [k for k, st in enumerate(stages) if all(i in ok_set for i in st)]
    tb = sum(t_stage_b[k] for k in eq_stages)
    tp = sum(t_stage_p[k] for k in eq_stages)
    eq_speedup = (64 * len(eq_stages) / tb) / (8 * len(eq_stages) / tp) if eq_stages else None
    return {"workload": "batched_path_m4_np300_d80: 64 lambdas in [1e-4, 1] x 8 folds = 512 problems",
            "problems": B, "method": "newton_full (Hessian pass + FP64 Cholesky per problem and iteration), "
                                     "continuation in 8 stages of 8 lambdas, largest first",
            "stage_seconds": {"batched_fp32": t_stage_b, "plain_fp64_fold0": t_stage_p},
            "batched_contraction_pass": contraction,
            "batched_fp32": {"solves_per_s": B / t_batched, "seconds": t_batched,
                             "converged": sum(r["status"] == 0 for r in rep),
                             "passes_total": sum(r["passes"] for r in rep),
                             "max_passes": max(r["passes"] for r in rep)},
            "plain_fp64": {"solves_per_s": len(plain) / t_plain, "seconds": t_plain, "timed_problems": len(plain),
                           "problems": "fold 0 of every lambda",
                           "converged": sum(r["status"] == 0 for r in rep64.values()),
                           "passes_total": sum(r["passes"] for r in rep64.values())},
            "speedup": (B / t_batched) / (len(plain) / t_plain),
            "target": f"relative objective gap {gap:g} (Newton decrement), at most {iters} Newton iterations",
            "equal_accuracy": {"lambdas": len(ok_set), "lambda_min": min(lam_ok) if lam_ok else None,
                               "problems": len(eq_b), "stages": eq_stages,
                               "batched_solves_per_s": 64 * len(eq_stages) / tb if eq_stages else None,
                               "plain_fp64_solves_per_s": 8 * len(eq_stages) / tp if eq_stages else None,
                               "speedup": eq_speedup,
                               "note": "lambdas whose fold-0 FP32 solution is within 1e-6 of the FP64 objective; "
                                       "below them the FP32 tensor's rounding (indefinite along null(X^T), where "
                                       "alpha grows like 1/lambda) decides the FP32 solution"},
            "fold0_within_1e-6_of_fp64": len(ok),
            "fold0_max_rel_obj_diff_vs_fp64": max(errs.values()), "held_out_max_abs_alpha": held_out,
            "per_lambda": per_lambda}


def dexter_leg(dev) -> dict:
    """The Dexter-shaped workload (few points, very many sparse features): the
    packed build (d-heavy: 2d flops per entry) and a full dual solve, timed;
    the solution checked against the linear kernel's closed-form gradient."""
    import numpy as np
    import torch

    import paper_2003_10482_gb300 as tk
    import synth
    p = synth.dexter_like()
    m, Xh, yh, lam = p["m"], p["X"], p["y"], p["lam"]
    n, d = Xh.shape
    X = torch.tensor(Xh, device=dev)
    y = torch.tensor(yh, device=dev)
    tk.tk_build_packed(X[:8], m, storage="f32")  # warm-up
    build = {}
    K = None
    for mode, name in ((1, "tensor_cores"), (0, "default")):
        tk.tk_build_set_config(mode)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        K = tk.tk_build_packed(X, m, storage="f32", K=K)
        e1.record()
        torch.cuda.synchronize()
        build[name] = e0.elapsed_time(e1)
    tk.tk_build_set_config(0)
    build_ms = build["default"]
    out = {"workload": f"dexter_like_m4_n{n}_d{d} (0.5 % dense features, FP32 storage)",
           "packed_entries": int(K.numel()), "build_ms": build_ms,
           "build_path": "tensor cores" if tk.tk_build_uses_tensor_cores(d, "f32") else "simt",
           "build_ms_tensor_cores": build["tensor_cores"], "build_status": tk.tk_build_status(),
           "build_tflops_at_2d_flop_per_entry": 2 * d * K.numel() / build_ms / 1e9}
    for method in ("newton_full", "newton_cg"):
        tk.tk_solve_dual(K, m, n, y, [lam], method=method, tol=1e-6, max_iter=1)  # warm-up: kernels, plans
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A, rep, rc = tk.tk_solve_dual(K, m, n, y, [lam], method=method, tol=1e-6, max_iter=100)
        torch.cuda.synchronize()
        a = A[0].cpu().numpy()
        u = Xh.T @ a
        g_exact = float(np.linalg.norm(Xh @ u ** (m - 1) + lam * a - yh))
        out[method] = {"solve_s": time.perf_counter() - t0, "iterations": rep[0]["iters"],
                       "passes": rep[0]["passes"], "gradnorm": rep[0]["gradnorm"],
                       "closed_form_gradnorm": g_exact, "status": rep[0]["status"]}
    return out


def methods_leg(dev) -> dict:
    """Full-Hessian Newton against Newton-CG on the plain FP64 workload (m = 4,
    n = 40, d = 10, lambda = 1e-2) to |grad F| <= 1e-10, and on the first stage
    of the lambda path (the 64 problems with lambda in [0.41, 1], FP32 storage,
    one batched call from the best multiple of y) to a 1e-7 relative gap:
    passes over K, iterations and time of each method (CUDA-synchronised wall
    clock, after a warm-up call)."""
    import torch

    import paper_2003_10482_gb300 as tk
    import synth
    out = {}
    p = synth.plain_fp64()
    m, X, y, lam = p["m"], p["X"], p["y"], p["lam"]
    n = X.shape[0]
    K = tk.tk_build_packed(torch.tensor(X, device=dev), m, storage="f64")
    yt = torch.tensor(y, device=dev)
    plain = {}
    for method in ("newton_full", "newton_cg"):
        tk.tk_solve_dual(K, m, n, yt, [lam], method=method, tol=1e-10, max_iter=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A, rep, rc = tk.tk_solve_dual(K, m, n, yt, [lam], method=method, tol=1e-10, max_iter=100)
        torch.cuda.synchronize()
        plain[method] = {"seconds": time.perf_counter() - t0, "iterations": rep[0]["iters"],
                         "passes": rep[0]["passes"], "gradnorm": rep[0]["gradnorm"], "status": rep[0]["status"]}
    out["plain_fp64_m4_n40_d10"] = plain
    bp = synth.batched_path()
    idx = tk.tk_nystrom_select(bp["X"].shape[0], bp["n_prime"], bp["select_seed"])
    Xb = torch.tensor(bp["X"][idx], device=dev)
    yb = torch.tensor(bp["y"][idx], device=dev)
    nb = Xb.shape[0]
    lamb = torch.tensor(bp["lambdas"], device=dev)
    maskb = torch.tensor(bp["masks"], device=dev)
    js = list(range(8 * 56, 8 * 64))  # the 8 largest lambdas x 8 folds
    K32 = tk.tk_build_packed(Xb, bp["m"], storage="f32")
    stage = {}
    for method in ("newton_full", "newton_cg"):
        kw = {"K_hvp": K32, "start_on_y": True} if method == "newton_full" else {"start_on_y": True}
        tk.tk_solve_dual(K32, bp["m"], nb, yb, lamb[js], mask=maskb[js], method=method, tol=0.0, rel_gap=1e-7,
                         max_iter=1, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A, rep, rc = tk.tk_solve_dual(K32, bp["m"], nb, yb, lamb[js], mask=maskb[js], method=method, tol=0.0,
                                      rel_gap=1e-7, max_iter=40, **kw)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        stage[method] = {"seconds": sec, "solves_per_s": len(js) / sec,
                         "converged": sum(r["status"] == 0 for r in rep),
                         "passes_total": sum(r["passes"] for r in rep), "passes_max": max(r["passes"] for r in rep),
                         "iterations_max": max(r["iters"] for r in rep)}
    out["lambda_path_stage0_fp32_64_problems"] = stage
    return out


def peaks_leg() -> dict:
    """Measured vector multiply-add rates (the denominators of the rooflines of
    the kernels bound by vector arithmetic)."""
    import paper_2003_10482_gb300 as tk
    return {"fp32_simt_tflops": tk.tk_fma_probe("f32", iters=1 << 16) / 1e12,
            "fp64_simt_tflops": tk.tk_fma_probe("f64", iters=1 << 12) / 1e12,
            "how": "tk_fma_probe: 8 x SMs blocks of 256 threads, 16 independent FMA chains each, CUDA events, best of 3"}


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2003_10482_gb300 as tk
    import synth
    from paper_2003_10482_gb300 import build_lib, parallel

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()

    p = synth.full_fp32()
    m = p["m"]
    npts = args.n if args.n > 0 else p["X"].shape[0]
    X = torch.tensor(p["X"][:npts], device=dev)
    n = X.shape[0]
    workload = WORKLOAD if npts == p["X"].shape[0] else WORKLOAD.replace("n400", f"n{npts}")
    N = tk.tk_packed_size(m, n)
    lo, hi = (0, N) if world == 1 else parallel.my_range(m, n, rank, world)
    K = tk.tk_build_packed(X, m, storage="f32", off_lo=lo, off_hi=hi)
    y = torch.tensor(p["y"][:npts], device=dev)
    lam = torch.tensor([p["lam"]], dtype=torch.float64, device=dev)
    A = torch.tensor(synth.alpha_like(n, salt=1, scale=0.1), device=dev)
    work = tk.workspace(m, n, 1, dev)
    esize = K.element_size()
    alg_bytes = (hi - lo) * esize  # algorithmic bytes of one pass over this rank's shard

    def step():
        if world == 1:
            return tk.tk_objective(K, m, n, A, y, lam, work=work)
        return parallel.sharded_objective(K, lo, hi, m, n, A, y, lam, work=work)

    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    ms = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    total_ms = float(ms[0])
    ms_per_step = total_ms / args.steps
    bytes_all = N * esize
    value = bytes_all / (ms_per_step * 1e-3) / 1e9
    status = tk.tk_status_read(work)

    # end to end through the public API: host (pinned) alpha in, F and grad out
    A_host = torch.tensor(synth.alpha_like(n, salt=1, scale=0.1)).pin_memory()
    out_host = torch.empty(n + 1, dtype=torch.float64).pin_memory()
    out_host2 = torch.empty(n + 2, dtype=torch.float64).pin_memory()
    if world == 1:
        tk.tk_objective_host(K, m, n, A_host, y, lam, out_host=out_host2)  # warm-up (workspace, plan)
    e2e_steps = max(10, args.steps // 4)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        if world == 1:
            # one C-ABI call with host buffers: alpha in, [F, |grad|, grad] out
            tk.tk_objective_host(K, m, n, A_host, y, lam, out_host=out_host2)
        else:
            Ad = A_host.to(dev, non_blocking=True)
            F, grad, gn = parallel.sharded_objective(K, lo, hi, m, n, Ad, y, lam, work=work)
            out_host[:n].copy_(grad.reshape(n), non_blocking=True)
            out_host[n:].copy_(F.reshape(1), non_blocking=True)
            torch.cuda.current_stream().synchronize()
    e2e_s = (time.perf_counter() - w0) / e2e_steps
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_s = float(e2e_t[0])

    if rank == 0:
        peak, peak_kind = _peaks()
        achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
        traffic = _profile_traffic(alg_bytes) if npts == p["X"].shape[0] else None
        cfg = tk.tk_contract_get_config(m, n, "f32")
        cfg_line = _config() if npts == p["X"].shape[0] else {
            "workload": workload, "m": m, "n": n, "d": int(X.shape[1]), "storage": "f32", "packed_entries": N,
            "packed_bytes": bytes_all}
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg_line,
            "setup": {"step": "tk_objective: one streaming pass (K[a^3], K[a^4]) + FP64 F/grad/|grad|",
                      "l2": "inputs (4.33 GB) larger than L2 (129 MB); no flush",
                      "parallelism": f"packed-range shards x{world}" if world > 1 else "1 GPU",
                      "launch": cfg},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "kernel": "contract_kernel (its last block runs the fixed-order FP64 reduction)",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "e2e": {"value": bytes_all / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": n * 8,
                    "d2h_bytes_per_step": (n + 2) * 8 if world == 1 else (n + 1) * 8,
                    "call": "tk_objective_host (pinned host alpha in, F, |grad|, grad out)" if world == 1
                    else "host alpha -> device, sharded objective, grad and F -> host"},
            "clocks": clocks,
            # one contraction kernel per step (+ the assembly kernel after the
            # all-reduce when sharded); the memset of the ticket is not a kernel
            "gpu_launches": (1 if world == 1 else 2) * args.steps,
            "device_status": status,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_leg()
        if world == 1 and not args.no_batched:
            line["peaks"] = peaks_leg()
            line["batched"] = batched_leg(dev)
            line["dexter_shaped"] = dexter_leg(dev)
            line["methods"] = methods_leg(dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_case(args) -> None:
    """One kernel a few times, for profiler captures.  On the batched
    workload's tensor (m = 4, n' = 300 landmarks, FP32): `hessian` runs
    tk_hessian, `batched_pass` the B-vector contraction (tensor-core pass
    unless --tc -1), `build` the packed build (SIMT unless --tc 1).  On the
    first --n points of the full FP32 workload (m = 4, d = 100): `hvp` runs the
    single-vector Hessian-vector pass.  `higher_order` runs the single pass on
    the m = 6, n = 80 FP32 tensor; `bf16` the single pass (the Hessian-vector
    pass with --dual) on a BF16 tensor over the first --n Nystrom landmarks
    (default 400).  Prints the mean CUDA-event time per call."""
    import torch

    import paper_2003_10482_gb300 as tk
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    storage = "f32"
    if args.case == "hvp":
        q = synth.full_fp32()
        n = args.n if args.n > 0 else q["X"].shape[0]
        X = torch.tensor(q["X"][:n], device=dev)
        m = q["m"]
    elif args.case == "higher_order":
        q = synth.higher_order()
        X = torch.tensor(q["X"], device=dev)
        m, n = q["m"], q["X"].shape[0]
    elif args.case == "bf16":
        q = synth.nystrom_bf16(n_test=10)
        idx = tk.tk_nystrom_select(q["X_train"].shape[0], q["n_prime"], q["select_seed"])
        n = args.n if args.n > 0 else 400
        X = torch.tensor(q["X_train"][idx[:n]], device=dev)
        m, storage = q["m"], "bf16"
    else:
        p = synth.batched_path()
        m = p["m"]
        idx = tk.tk_nystrom_select(p["X"].shape[0], p["n_prime"], p["select_seed"])
        X = torch.tensor(p["X"][idx], device=dev)
        n = X.shape[0]
    if args.case == "build":
        tk.tk_build_set_config(1 if args.build_tc else -1)
    K = tk.tk_build_packed(X, m, storage=storage)
    if args.case == "build":
        call = lambda: tk.tk_build_packed(X, m, storage="f32", K=K)  # noqa: E731
    elif args.case == "hvp" or (args.case == "bf16" and args.dual):
        a = torch.tensor(synth.alpha_like(n, salt=7), device=dev)
        v = torch.tensor(synth.alpha_like(n, salt=8), device=dev)
        call = lambda: tk.tk_contract(K, m, n, a, r=m - 2, V=v)  # noqa: E731
    elif args.case in ("higher_order", "bf16"):
        a = torch.tensor(synth.alpha_like(n, salt=7), device=dev)
        call = lambda: tk.tk_contract(K, m, n, a)  # noqa: E731
    elif args.case == "hessian":
        a = torch.tensor(synth.alpha_like(n, salt=3), device=dev)
        call = lambda: tk.tk_hessian(K, m, n, a)  # noqa: E731
    else:
        tk.tk_batched_set_config(tensor_cores=args.tc)
        A = torch.tensor(synth.alpha_like(n, salt=5, batch=args.B), device=dev)
        call = lambda: tk.tk_contract(K, m, n, A)  # noqa: E731
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        call()
    e1.record()
    e1.synchronize()
    batched = args.case == "batched_pass"
    print(json.dumps({"case": args.case, "B": args.B if batched else 1, "tensor_cores": args.tc if batched else None,
                      "ms_per_call": e0.elapsed_time(e1) / 3, "entries": int(K.numel()),
                      "TB_per_s": K.numel() * K.element_size() / (e0.elapsed_time(e1) / 3) / 1e9}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-FP64 dual-solve comparison")
    ap.add_argument("--n", type=int, default=0,
                    help="points of the workload (default: all 400); smaller n for profiler captures")
    ap.add_argument("--case", choices=["hessian", "batched_pass", "build", "hvp", "higher_order", "bf16"],
                    default=None,
                    help="run one kernel a few times (profiler captures) and exit")
    ap.add_argument("--build-tc", action="store_true", help="--case build: the tensor-core build")
    ap.add_argument("--dual", action="store_true", help="--case bf16: the Hessian-vector pass")
    ap.add_argument("--B", type=int, default=128, help="vectors of --case batched_pass")
    ap.add_argument("--tc", type=int, default=1, choices=[1, -1], help="--case batched_pass: tensor cores or SIMT")
    args = ap.parse_args()
    if args.case is not None:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(_spawn_ranks(args.gpus))
    else:
        run_ours(args)


def _spawn_ranks(nproc: int) -> int:
    """`--gpus N` without a launcher: start N ranks on this node the way
    torchrun would (one process per GPU, rendezvous on 127.0.0.1); rank 0
    prints the JSON line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


if __name__ == "__main__":
    main()
