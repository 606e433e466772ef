"""Sharded contraction across processes (the multi-GPU design) with world_size 2
on CPU: each rank takes its row-aligned, cost-balanced shard of the packed range
(paper_2003_10482_gb300.parallel), computes the partial contraction of its shard
with the oracle, and the ranks sum the partials with one gloo all-reduce.  The
sum must equal the unsharded contraction."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

tk = pytest.importorskip("paper_2003_10482_gb300")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, m, n, d, q):
    import oracle
    import synth
    from paper_2003_10482_gb300 import parallel
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = synth.small_problem(m, n, d, salt=90)
    a = synth.alpha_like(n, salt=91)
    lo, hi = parallel.my_range(m, n, rank, world)
    K = oracle.build(X, m, lo, hi)
    g, S = oracle.contract(K, a, m, lo=lo)
    G, St = parallel.allreduce_partials(torch.tensor(g).reshape(1, n), torch.tensor([S], dtype=torch.float64))
    q.put((rank, lo, hi, G.numpy(), float(St[0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("m,n,d", [(4, 17, 3), (6, 8, 2), (2, 40, 3)])
def test_two_rank_shards_sum_to_full_contraction(m, n, d):
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, m, n, d, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    N = oracle.packed_size(m, n)
    assert out[0][1] == 0 and out[0][2] == out[1][1] and out[1][2] == N  # the shards tile [0, N)
    X = synth.small_problem(m, n, d, salt=90)
    a = synth.alpha_like(n, salt=91)
    g_ref, S_ref = oracle.contract(oracle.build(X, m), a, m)
    for _, lo, hi, G, S in out:
        assert np.allclose(G.reshape(n), g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
        assert S == pytest.approx(S_ref, rel=1e-12)
