"""The data-parallel decomposition behind pinn_set_global_counts, on the CPU with two
gloo ranks: each rank evaluates the FP64 oracle on its own shard with every mean taken
over the whole batch's counts; an all-reduce of those shares gives the whole-batch loss
and gradient."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard(b, rank, ws):
    def cut(n):
        return n * rank // ws, n * (rank + 1) // ws
    r0, r1 = cut(b.n_res)
    i0, i1 = cut(b.x_ic.shape[1])
    c0, c1 = cut(b.x_bc.shape[1])
    return type(b)(b.x_res[:, r0:r1], b.x_ic[:, i0:i1], b.g_ic[:, i0:i1], b.ic_mask,
                   b.x_bc[:, c0:c1], b.g_bc[:, c0:c1], b.bc_mask)


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    from synth import make_workload
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, p, B, b = make_workload("burgers1d_4x64", n_res=301, n_ic=37, n_bc=53, random_bias=0.1)
        lam = (1.0, 0.7, 1.3)
        s = _shard(b, rank, ws)
        # the shard's share: its sums over the whole batch's counts = its means scaled by its fraction
        f = (s.n_res / b.n_res, s.x_ic.shape[1] / b.x_ic.shape[1], s.x_bc.shape[1] / b.x_bc.shape[1])
        m = oracle.Model.from_spec(w.spec)
        t, g = oracle.loss_and_grad(m, p, B, s, w.problem.nu, tuple(l * fi for l, fi in zip(lam, f)))
        share = torch.tensor(np.concatenate([[t["total"]], g]), dtype=torch.float64)
        dist.all_reduce(share)
        out.put((rank, share.numpy()))
    finally:
        dist.destroy_process_group()


def test_sharded_oracle_all_reduce_equals_the_whole_batch():
    import oracle
    from synth import make_workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, pp, B, b = make_workload("burgers1d_4x64", n_res=301, n_ic=37, n_bc=53, random_bias=0.1)
    t, g = oracle.loss_and_grad(oracle.Model.from_spec(w.spec), pp, B, b, w.problem.nu, (1.0, 0.7, 1.3))
    full = np.concatenate([[t["total"]], g])
    for _, share in res:
        np.testing.assert_allclose(share, full, rtol=1e-12, atol=1e-14 * np.max(np.abs(full)))
