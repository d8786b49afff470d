"""One problem split over ranks (paper Sec. 3 subdomains in a row, the update of
Sec. 2.5 across rank boundaries): paper_2203_10477_gb300/split.py.

CPU: the partition; two and three gloo ranks whose parts are solved by the
oracle (the same part, the whole grid's coefficients), gathered and compared
bit for bit with the oracle's monolithic solve of the whole grid.
GPU: three ranks as threads of one process, each with its part plan on the one
GPU (the library), exchanging through in-process mailboxes; bit for bit
against the oracle.  No kernel waits on another: the host orders every round.
"""
from __future__ import annotations

import os
import queue
import socket
import threading

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs
from paper_2203_10477_gb300.split import partition

F32, F64 = 0, 1


def test_partition_covers_the_grid_once():
    for nx, N, world, h in [(2001, 8, 2, 8), (2001, 8, 3, 8), (10_007, 17, 5, 32), (1 << 20, 256, 8, 32)]:
        blocks = partition(nx, N, world, h)
        assert blocks[0].c0 == 0 and blocks[-1].c1 == nx
        for a, b in zip(blocks, blocks[1:]):
            assert a.c1 == b.c0 and a.i1 == b.i0
            assert a.hi - a.c1 == h and b.c0 - b.lo == h  # halos beside every cut
        assert blocks[0].lo == 0 and blocks[-1].hi == nx
        counts = [b.i1 - b.i0 for b in blocks]
        assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        partition(100, 4, 5, 8)  # more ranks than subdomains
    with pytest.raises(ValueError):
        partition(100, 10, 10, 11)  # a rank owning fewer points than the halo


class OracleSolver:
    """Test stand-in for the part plan: the oracle's monolithic leapfrog on the
    part's points, with the whole grid's coefficients (the oracle derives them
    from nx and runs the first nx_run points: the part's data is given as its
    own state and boundary samples, so the part's place in the grid does not
    matter)."""

    def __init__(self, xa, xb, a, nx, dt, blk, overlap, dtype, device):
        import oracle

        oracle.build()
        self.oracle = oracle
        self.args = (xa, xb, a, nx, dt)
        self.m = blk.hi - blk.lo
        self.form, self.prec = (0, "f64") if dtype == F64 else (1, "f32")

    def run(self, fA, fB, steps, u, w, out, j_r=None):
        import torch

        xa, xb, a, nx, dt = self.args
        r = self.oracle.leapfrog(nx, steps, a, dt, fA.numpy(), fB.numpy(), form=self.form, prec=self.prec,
                                 q0=u.numpy(), q1=w.numpy(), nx_run=self.m, xa=xa, xb=xb,
                                 rec_j=[] if j_r is None else [j_r])
        out[0].copy_(torch.from_numpy(r["u"]))
        out[1].copy_(torch.from_numpy(r["w"]))
        return None if j_r is None else torch.from_numpy(r["rec"][0])


def split_case(seed):
    """nx = 2001, N = 12 subdomains, overlap 16, CFL 0.9, 300 steps; a boundary
    pulse on each end and a smooth initial state, so every point is active."""
    nx, N, ov, T = 2001, 12, 16, 300
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=13.0)
    fB = -0.5 * inputs.ramped_sine(T, dt, freq=7.0)
    q0 = inputs.smooth_random_state(nx, seed=seed)
    return nx, N, ov, T, dt, fA, fB, q0


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, dtype, halo, q):
    import torch
    import torch.distributed as dist

    from paper_2203_10477_gb300.split import SplitPlan

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, N, ov, T, dt, fA, fB, q0 = split_case(3)
        sp = SplitPlan(0.0, 1.0, 1.0, nx, dt, N, ov, rank, world, dist, dtype=dtype, halo=halo,
                       device="cpu", solver=OracleSolver)
        res = sp.run(fA, fB, T, q0=q0, j_r=777)
        u = sp.gather(res["u"])
        w = sp.gather(res["w"])
        if rank == 0:
            q.put((u.numpy(), w.numpy(), res["recv"].numpy(), sp.exchanged_bytes))
        else:
            q.put(None)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dtype,halo", [(2, F64, None), (3, F64, None), (3, F32, None), (2, F64, 40)])
def test_gloo_ranks_equal_the_monolithic_oracle(oracle_mod, world, dtype, halo):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, dtype, halo, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u, w, recv, nbytes = next(r for r in res if r is not None)
    nx, N, ov, T, dt, fA, fB, q0 = split_case(3)
    form, prec = (0, "f64") if dtype == F64 else (1, "f32")
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=form, prec=prec, q0=q0, rec_j=[777])
    assert np.array_equal(u, ref["u"]) and np.array_equal(w, ref["w"])
    assert np.array_equal(recv, ref["rec"][0])
    assert nbytes > 0


def test_gloo_split_catches_a_missing_exchange(oracle_mod, monkeypatch):
    """The comparison above is sensitive: without the exchange the halos go
    stale and the gathered state differs (checked in one process with a
    single-rank plan per part and no exchange)."""
    import torch

    from paper_2203_10477_gb300.split import SplitPlan

    nx, N, ov, T, dt, fA, fB, q0 = split_case(3)
    parts = []
    for r in range(2):
        sp = SplitPlan(0.0, 1.0, 1.0, nx, dt, N, ov, r, 2, None, dtype=F64, device="cpu", solver=OracleSolver)
        monkeypatch.setattr(sp, "_exchange", lambda u, w: None)
        parts.append(sp.run(fA, fB, T, q0=q0)["u"])
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, q0=q0)
    assert not np.array_equal(torch.cat(parts).numpy(), ref["u"])


class MailDist:
    """Point-to-point messages between ranks that are threads of one process
    (the calls of torch.distributed that SplitPlan makes).  A message is a
    copy made on the sender's stream and read on the receiver's; both are the
    device's default stream here, so the copies are ordered."""

    class _Done:
        def wait(self):
            return None

    class _Recv:
        def __init__(self, box, buf):
            self.box, self.buf = box, buf

        def wait(self):
            self.buf.copy_(self.box.get(timeout=120))

    class P2POp:
        def __init__(self, op, tensor, peer):
            self.op, self.tensor, self.peer = op, tensor, peer

    def __init__(self, boxes, rank, world):
        self.boxes, self.rank, self.world = boxes, rank, world

    def batch_isend_irecv(self, ops):
        return [o.op(o.tensor, o.peer) for o in ops]

    def isend(self, t, dst):
        self.boxes[(self.rank, dst)].put(t.clone())
        return self._Done()

    def irecv(self, buf, src):
        return self._Recv(self.boxes[(src, self.rank)], buf)

    def send(self, t, dst):
        self.boxes[(self.rank, dst)].put(t.clone())

    def recv(self, buf, src):
        buf.copy_(self.boxes[(src, self.rank)].get(timeout=120))

    def broadcast(self, t, src):
        if self.rank == src:
            for r in range(self.world):
                if r != src:
                    self.send(t, r)
        else:
            self.recv(t, src)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,halo", [(F64, None), (F32, None), (F64, 64), (F32, 48)])
def test_three_thread_ranks_on_one_gpu_equal_the_oracle(oracle_mod, dtype, halo):
    import torch

    from paper_2203_10477_gb300 import build
    from paper_2203_10477_gb300.split import SplitPlan

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    nx, N, ov, T = 30_001, 12, 32, 400
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=13.0)
    fB = -0.5 * inputs.ramped_sine(T, dt, freq=7.0)
    q0 = inputs.smooth_random_state(nx, seed=5)
    world = 3
    boxes = {(s, d): queue.Queue() for s in range(world) for d in range(world)}
    results, errors = {}, []

    def rank_main(r):
        try:
            torch.cuda.set_device(0)
            sp = SplitPlan(0.0, 1.0, 1.0, nx, dt, N, ov, r, world, MailDist(boxes, r, world), dtype=dtype,
                           halo=halo, device="cuda:0")
            res = sp.run(fA, fB, T, q0=q0, j_r=12_345)
            u, w = sp.gather(res["u"]), sp.gather(res["w"])
            torch.cuda.synchronize()
            if r == 0:
                results.update(u=u.cpu().numpy(), w=w.cpu().numpy(), recv=res["recv"].cpu().numpy())
        except Exception as e:  # reported below
            errors.append((r, repr(e)))

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    form, prec = (0, "f64") if dtype == F64 else (1, "f32")
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=form, prec=prec, q0=q0, rec_j=[12_345])
    assert np.array_equal(results["u"], ref["u"]), "state differs from the oracle"
    assert np.array_equal(results["w"], ref["w"]), "second component differs from the oracle"
    assert np.array_equal(results["recv"], ref["rec"][0]), "receiver trace differs from the oracle"
