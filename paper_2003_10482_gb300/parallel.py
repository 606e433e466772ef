"""Sharding of the packed tensor over several processes (one per GPU).

The packed array is cut into row-aligned, cost-balanced shards (the same cut
the contraction uses for its warps, tk_contract_plan).  Each rank builds and
holds only its shard; per solver pass it contracts the shard and the ranks sum
their partial K[a^{m-1}] (n values) and K[a^m] (1 value) with one all-reduce.
The dual vector and the data matrix are replicated.  Everything here is host
logic around the C ABI: the contraction itself runs in libtk.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

import paper_2003_10482_gb300 as tk


def shard_bounds(m: int, n: int, world: int, row_cost: int = 256, tri_cost: int = 1024) -> list[int]:
    """world+1 row-aligned offsets cutting [0, N) into near-equal-cost shards."""
    N = tk.tk_packed_size(m, n)
    return tk.tk_contract_plan(m, n, 0, N, world, row_cost, tri_cost)


def my_range(m: int, n: int, rank: int, world: int) -> tuple[int, int]:
    b = shard_bounds(m, n, world)
    return b[rank], b[rank + 1]


def allreduce_partials(G: torch.Tensor, S: torch.Tensor, group=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Sum the ranks' partial contractions: one all-reduce of the B x (n+1) FP64 block."""
    B = S.numel()
    buf = torch.cat([G.reshape(B, -1).to(torch.float64), S.reshape(B, 1).to(torch.float64)], dim=1)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[:, :-1].reshape(G.shape), buf[:, -1].contiguous()


def sharded_objective(K_shard: torch.Tensor, lo: int, hi: int, m: int, n: int, A: torch.Tensor,
                      y: torch.Tensor, lam, work=None, group=None):
    """Dual objective and gradient with the packed tensor split over ranks."""
    G, S = tk.tk_contract(K_shard, m, n, A.to(torch.float64), off_lo=lo, off_hi=hi, work=work)
    G, S = allreduce_partials(G, S, group)
    return tk.tk_assemble_objective(m, n, G, S, A, y, lam)
