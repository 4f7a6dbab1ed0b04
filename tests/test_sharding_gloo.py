"""Event sharding across ranks (the multi-GPU design), checked on CPU ranks.

Events are independent given rho^t, so one MLEM update over the whole list
equals the sum over ranks of the updates over each rank's share of the events
(Eq. iter is a sum over j); only rho_new needs an all-reduce.  Two gloo ranks
run the FP64 oracle on their shares and all-reduce; the result must equal the
single-process update.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_iter, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from oracle import Setup
    from synth import make_workload
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w, n_threads=1)
    s = oracle.sensitivity(st)
    mine = [e[rank::world] for e in ev]
    rho = np.ones((w.ny, w.nz))
    for _ in range(n_iter):
        part, stats = oracle.mlem(st, mine, 1, rho0=rho, s=s)
        t = torch.from_numpy(part.copy())
        dist.all_reduce(t)
        rho = t.numpy()
        used = torch.tensor([stats.n_used], dtype=torch.int64)
        dist.all_reduce(used)
    if rank == 0:
        q.put((rho, int(used.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_update_equals_whole():
    import oracle
    from oracle import Setup
    from synth import make_workload
    n_iter = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_iter, q)) for r in range(2)]
    for p in procs:
        p.start()
    rho_sh, used = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w)
    rho, stats = oracle.mlem(st, ev, n_iter)
    np.testing.assert_allclose(rho_sh, rho, rtol=1e-12, atol=1e-300)
    assert used == stats.n_used
