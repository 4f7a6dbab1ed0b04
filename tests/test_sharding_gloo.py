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


class _OracleShard:
    """Stand-in for a Recon holding one rank's share of the events, with the
    FP64 oracle doing the arithmetic: backproject returns A = sum_j P_jl / D_j
    over the share (one oracle update of rho divided by rho, 0 where rho = 0);
    apply_update multiplies the image."""

    def __init__(self, st, events, s):
        import oracle
        self._oracle = oracle
        self.st, self.events, self.s = st, events, s
        self.rho = np.ones((st.ny, st.nz))
        self.calls = []

    def backproject(self, out=None):
        nxt, _ = self._oracle.mlem(self.st, self.events, 1, rho0=self.rho, s=self.s)
        A = np.divide(nxt, self.rho, out=np.zeros_like(nxt), where=self.rho > 0)
        self.calls.append("backproject")
        if out is None:
            return torch.from_numpy(A)
        out.copy_(torch.from_numpy(A))
        return out

    def apply_update(self, A):
        self.rho = self.rho * A.numpy()
        self.calls.append("apply_update")


def _loop_worker(rank, world, port, n_iter, q):
    """Each rank drives the package's sharded loop over its share."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from oracle import Setup
    from paper_1502_07478_gb300.shard import sharded_iterate
    from synth import make_workload
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w, n_threads=1)
    s = oracle.sensitivity(st)
    # uneven contiguous shares: rank 0 a third, rank 1 the rest
    cut = len(ev[0]) // 3
    mine = [e[:cut] for e in ev] if rank == 0 else [e[cut:] for e in ev]
    shard = _OracleShard(st, mine, s)
    sharded_iterate(shard, n_iter, dist.all_reduce)
    assert shard.calls == ["backproject", "apply_update"] * n_iter
    q.put((rank, shard.rho))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_loop_equals_whole():
    """paper_1502_07478_gb300.shard.sharded_iterate over two gloo ranks with
    uneven shares: both ranks end with the single-process oracle image."""
    import oracle
    from oracle import Setup
    from synth import make_workload
    n_iter = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_loop_worker, args=(r, 2, port, n_iter, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    rho, _ = oracle.mlem(Setup.from_workload(w), ev, n_iter)
    for r in (0, 1):
        np.testing.assert_allclose(got[r], rho, rtol=1e-12, atol=1e-300)


class _OracleAdjShard:
    """Stand-in for a Recon holding one rank's share of the events, with the
    FP64 oracle's log-likelihood and gradients (Recon.loglik_grad's quantities)."""

    def __init__(self, st, events, s, rho):
        import oracle
        self._oracle = oracle
        self.st, self.events, self.s, self.rho = st, events, s, rho

    def loglik_grad(self):
        L, g, gs = self._oracle.loglik_grad(self.st, self.events, self.rho, s=self.s)
        return L, torch.from_numpy(np.asarray(g).reshape(self.rho.shape).copy()), np.asarray(gs)

    def compute_sensitivity(self):
        return torch.from_numpy(np.asarray(self.s).reshape(self.rho.shape).copy())

    def read_image(self, which=0):
        return torch.from_numpy(self.rho * (np.asarray(self.s).reshape(self.rho.shape)
                                            if which == 1 else 1.0))


def _adj_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from oracle import Setup
    from paper_1502_07478_gb300.shard import sharded_loglik_grad
    from synth import make_workload
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w, n_threads=1)
    s = oracle.sensitivity(st)
    rho = np.random.Generator(np.random.PCG64(11)).uniform(0.5, 2.0, (w.ny, w.nz))
    cut = len(ev[0]) // 3
    mine = [e[:cut] for e in ev] if rank == 0 else [e[cut:] for e in ev]
    L, g, gs = sharded_loglik_grad(_OracleAdjShard(st, mine, s, rho), dist.all_reduce, world)
    q.put((rank, L, g.numpy(), gs))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_loglik_grad_equals_whole():
    """paper_1502_07478_gb300.shard.sharded_loglik_grad over two gloo ranks with
    uneven shares: L, g_rho and g_sigma of the whole list on both ranks (the
    image terms of L and g_rho counted once)."""
    import oracle
    from oracle import Setup
    from synth import make_workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_adj_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {r: (L, g, gs) for r, L, g, gs in (q.get(timeout=300) for _ in range(2))}
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    w = make_workload("small_5mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w)
    rho = np.random.Generator(np.random.PCG64(11)).uniform(0.5, 2.0, (w.ny, w.nz))
    L, g, gs = oracle.loglik_grad(st, ev, rho)
    for r in (0, 1):
        Lr, gr, gsr = got[r]
        assert Lr == pytest.approx(L, rel=1e-12)
        np.testing.assert_allclose(gr.ravel(), np.asarray(g).ravel(), rtol=1e-10,
                                   atol=1e-12 * float(np.abs(g).max()))
        np.testing.assert_allclose(gsr, gs, rtol=1e-10)
