"""The sharded path through the real kernels: two processes (the ranks of the
multi-GPU design, here sharing the one GPU of the test machine; their kernels
never wait on each other) each build their row-aligned shard of the packed
tensor with tk_build_packed_range, contract it with tk_contract_range, and the
ranks sum the partial contractions with one gloo all-reduce
(parallel.allreduce_partials).  The sum must equal the oracle's unsharded
contraction within the contraction's bound."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

tk = pytest.importorskip("paper_2003_10482_gb300")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, m, n, d, storage, q):
    import synth
    from paper_2003_10482_gb300 import parallel
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    X = torch.tensor(synth.small_problem(m, n, d, salt=95), device="cuda")
    a = torch.tensor(synth.alpha_like(n, salt=96), device="cuda")
    lo, hi = parallel.my_range(m, n, rank, world)
    K = tk.tk_build_packed(X, m, storage=storage, off_lo=lo, off_hi=hi)
    G, S = tk.tk_contract(K, m, n, a, off_lo=lo, off_hi=hi)
    torch.cuda.synchronize()
    G, S = parallel.allreduce_partials(G.reshape(1, n).cpu(), S.cpu())
    q.put((rank, lo, hi, G.numpy().reshape(n), float(S[0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("m,n,d,storage", [(4, 90, 4, "f64"), (4, 121, 3, "f32"), (6, 23, 2, "f32")])
def test_two_process_shards_through_the_kernels(m, n, d, storage):
    import oracle
    import synth
    from gpu_util import contraction_bound, round_storage
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, m, n, d, storage, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    N = oracle.packed_size(m, n)
    assert out[0][1] == 0 and out[0][2] == out[1][1] and out[1][2] == N
    X = synth.small_problem(m, n, d, salt=95)
    a = synth.alpha_like(n, salt=96)
    # the GPU contracts its own build of K, which differs from the oracle's
    # rounded build by the build's accumulation error and at most one rounding
    # of the storage type per entry; each shard then carries its own
    # contraction bound (its plan), and the FP64 all-reduce adds nothing
    Kr = round_storage(oracle.build(X, m), storage).double().numpy()
    g_ref, S_ref = oracle.contract(Kr, a, m)
    g_abs, S_abs = oracle.contract(oracle.build(np.abs(X), m), np.abs(a), m)
    u = 2.0 ** -53 if storage == "f64" else 2.0 ** -24
    e_build = (1.01 * (d + m + 2) + 1) * u
    shard = [contraction_bound(n, g_abs, storage, m, lo=o[1], hi=o[2]) for o in out]
    s_shard = [float(contraction_bound(n, np.array([S_abs]), storage, m, lo=o[1], hi=o[2])[0]) for o in out]
    tol = e_build * g_abs + np.maximum(shard[0], shard[1])
    s_tol = e_build * S_abs + max(s_shard)
    for _, lo, hi, G, S in out:
        assert np.all(np.abs(G - g_ref) <= tol), float(np.max(np.abs(G - g_ref) / tol))
        assert abs(S - S_ref) <= s_tol
