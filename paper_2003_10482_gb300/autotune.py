"""Autotuner of the contraction launch configurations, by measurement.

The launch shape of both contraction kernels is a process-wide setting of the
library (tk_contract_set_config, tk_batched_set_config).  `tune_contract`
times the single-vector pass over a few warp counts, staging-buffer sizes,
buffer counts and schedules; `tune_batched` times the batched pass over batch
widths per lane (vectors per lane), staging-buffer sizes, buffer counts and
slices per group, and the smallest batch that takes the batched kernel.  Each
candidate runs on the caller's own packed tensor with seeded dual vectors,
timed by CUDA events after a warm-up call; the fastest one is set and kept per
shape key, so `apply` restores it later without measuring again.

Candidates the library rejects for the shape (shared memory, register
budget) are skipped.  Tuning changes only the order in which partial sums
meet, not what is computed; the static schedule keeps results
bit-reproducible for a given configuration.
"""
from __future__ import annotations

import itertools

import torch

import paper_2003_10482_gb300 as tk

_best: dict = {}


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _vectors(n: int, B: int, seed: int) -> torch.Tensor:
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(B, n, generator=g, dtype=torch.float64).mul_(0.1).cuda()


def tune_contract(K: torch.Tensor, m: int, n: int, dual: bool = False, reps: int = 3,
                  candidates: list[dict] | None = None) -> dict:
    """Time the single-vector contraction over `candidates` (launch-config
    dicts, 0 = library choice) and keep the fastest.  Returns
    {"best": cfg, "ms": t, "trials": [(cfg, ms), ...]}."""
    storage = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}[K.dtype]
    if candidates is None:
        candidates = [dict(warps=w, block_bytes=bb, nbuf=nb, schedule=sc)
                      for w, bb, nb, sc in itertools.product((14, 16), (0, 4224), (2, 3), (1, 2))]
        candidates += [dict(pieces_per_warp=pp) for pp in (8, 12)] + [dict(row_cost=256, tri_cost=4096)]
    A = _vectors(n, 1, 1)[0]
    V = _vectors(n, 1, 2)[0]
    ws = tk.workspace(m, n)
    run = (lambda: tk.tk_contract(K, m, n, A, r=m - 2, V=V, work=ws)) if dual else \
          (lambda: tk.tk_contract(K, m, n, A, work=ws))
    trials = []
    for cfg in candidates:
        try:
            tk.tk_contract_set_config(**cfg)
            got = tk.tk_contract_get_config(m, n, storage, dual)
            if cfg.get("warps") and got["warps"] != cfg["warps"]:
                continue  # the library capped the warps: an equivalent candidate exists
            trials.append((cfg, _time(run, reps)))
        except tk.TKError:
            continue
    if not trials:
        tk.tk_contract_set_config(reset=True)
        raise tk.TKError(tk.TK_EUNSUPPORTED, "no candidate configuration runs for this shape")
    cfg, ms = min(trials, key=lambda t: t[1])
    tk.tk_contract_set_config(**cfg)
    _best[("contract", m, n, storage, dual)] = ("contract", cfg)
    return {"best": cfg, "ms": ms, "trials": trials}


def tune_batched(K: torch.Tensor, m: int, n: int, B: int, dual: bool = False, reps: int = 2,
                 candidates: list[dict] | None = None) -> dict:
    """Time the batched contraction of B vectors over `candidates` (batched
    launch-config dicts) and keep the fastest; also finds the smallest batch
    that the batched kernel serves faster than one single-vector pass per
    vector (min_batch)."""
    storage = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}[K.dtype]
    if candidates is None:
        candidates = [dict(vpl=v, block_bytes=bb, nbuf=nb, slice_mult=sm)
                      for v, bb, nb, sm in itertools.product((1, 2), (8320, 16512), (2, 3), (1, 2))]
    A = _vectors(n, B, 3)
    V = _vectors(n, B, 4)
    ws = tk.workspace(m, n, B)

    def run_for(X, Y):
        if dual:
            return lambda: tk.tk_contract(K, m, n, X, r=m - 2, V=Y, work=ws)
        return lambda: tk.tk_contract(K, m, n, X, work=ws)

    trials = []
    for cfg in candidates:
        try:
            tk.tk_batched_set_config(**dict(cfg, min_batch=1))
            got = tk.tk_batched_get_config(m, n, storage, dual, B)
            if got["vpl"] == 0 or got["vpl"] != cfg.get("vpl", got["vpl"]):
                continue
            trials.append((cfg, _time(run_for(A, V), reps)))
        except tk.TKError:
            continue
    if not trials:
        tk.tk_batched_set_config(reset=True)
        raise tk.TKError(tk.TK_EUNSUPPORTED, "the batched kernel does not cover this shape")
    cfg, ms = min(trials, key=lambda t: t[1])
    # crossover: one batched pass of b vectors against b single-vector passes
    tk.tk_batched_set_config(**dict(cfg, min_batch=1))
    t_batched_small = _time(run_for(A[:8].contiguous(), V[:8].contiguous()), reps)
    tk.tk_batched_set_config(**dict(cfg, min_batch=1 << 30))
    t_single = _time(run_for(A[:1].contiguous(), V[:1].contiguous()), reps)
    min_batch = max(2, int(t_batched_small / max(t_single, 1e-9)) + 1)
    best = dict(cfg, min_batch=min_batch)
    tk.tk_batched_set_config(**best)
    _best[("batched", m, n, storage, dual)] = ("batched", best)
    return {"best": best, "ms": ms, "trials": trials, "single_vector_ms": t_single,
            "batched_floor_ms": t_batched_small}


def apply(kind: str, m: int, n: int, storage: str, dual: bool = False) -> bool:
    """Set the configuration a previous tune_* call found for this shape."""
    hit = _best.get((kind, m, n, storage, dual))
    if hit is None:
        return False
    what, cfg = hit
    if what == "contract":
        tk.tk_contract_set_config(**cfg)
    else:
        tk.tk_batched_set_config(**cfg)
    return True
