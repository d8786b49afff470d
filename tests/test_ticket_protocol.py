"""A CPU model of the persistent span kernel's scheduling protocol.

The warp-specialised span kernel (csrc/span_kernel.cuh: producer_loop and the
compute warps of span_kernel_ws) hands out (span k, tile i) tickets in
span-major order from one counter; a ticket's window may be loaded once tile i
and its neighbours in the same problem have published span k-1; a finished
tile's core is stored into the other state buffer and then published.  The
producer keeps two stages: it fetches the ticket after next while the current
one computes, and it publishes a finished tile before it waits for the
neighbours of the next one.

This model replays that protocol step by step under random interleavings of
many CTAs (each a producer and a compute process sharing two stages) and
checks, at every window load, that each core it reads holds exactly the
state of span k in buffer k & 1 (no read before the write was published, no
overwrite by span k + 2 before the read), that every ticket completes without
a timeout, and that a tile which never publishes (the host-injected fault of
rswr_plan_inject_missing_flag) ends the run with a latched error instead of a
hang.  Waits are bounded by a poll budget, like the kernel's time limit.
The persistent adjoint sweep (adj_producer in csrc/adjoint_kernel.cu) runs the
same protocol with its spans taken last first, i.e. the same tickets in
dependency order, so the model covers it as well.
"""
from __future__ import annotations

import random

import pytest

PENDING = "pending"


class Protocol:
    def __init__(self, problem_tiles, nspans, nctas, seed, inject=None, poll_limit=20000):
        self.tiles = [(p, j) for p, nt in enumerate(problem_tiles) for j in range(nt)]
        self.nt = problem_tiles
        self.ntiles = len(self.tiles)
        self.nspans = nspans
        self.total = nspans * self.ntiles
        self.counter = 0
        self.done = [0] * self.ntiles
        # version[b][i]: the span whose state buffer b holds for tile i's core
        self.version = [[0] * self.ntiles, [None] * self.ntiles]
        self.err = False
        self.inject = inject  # (tile, span) whose completion is never published
        self.poll_limit = poll_limit
        self.rng = random.Random(seed)
        self.computed = set()
        self.violations = []
        self.nctas = nctas

    # ---- the device operations ------------------------------------------
    def grab(self):
        if self.err:
            return -1
        t = self.counter
        self.counter += 1
        return t if t < self.total else -1

    def window(self, i):
        p, j = self.tiles[i]
        return [i + d for d in (-1, 0, 1) if 0 <= j + d < self.nt[p]]

    def ready(self, t):
        k, i = divmod(t, self.ntiles)
        return k == 0 or all(self.done[n] >= k for n in self.window(i))

    def load(self, t):
        k, i = divmod(t, self.ntiles)
        for n in self.window(i):
            v = self.version[k & 1][n]
            if v != k:
                self.violations.append(("read", t, n, v))

    def store(self, t):
        k, i = divmod(t, self.ntiles)
        self.version[(k + 1) & 1][i] = (PENDING, k + 1)

    def publish(self, t):
        k, i = divmod(t, self.ntiles)
        self.version[(k + 1) & 1][i] = k + 1
        if self.inject == (i, k):
            return
        self.done[i] = k + 1

    # ---- processes (generators; each yield lets another process run) -----
    def wait(self, cond):
        """Bounded poll; True when cond held, False on timeout or a latched error."""
        polls = 0
        while not cond():
            if self.err:
                return False
            polls += 1
            if polls > self.poll_limit:
                self.err = True
                return False
            yield
        return True

    def producer(self, st):
        def arm(y, t):
            if t >= 0:
                self.load(t)
            st[y]["ticket"] = t
            st[y]["full"] = True

        y = 0
        t = self.grab()
        yield
        if t >= 0:
            ok = yield from self.wait(lambda: self.ready(t))
            if not ok:
                t = -1
        arm(0, t)
        tn, tn_armed = -1, True
        if t >= 0:
            tn = self.grab()
            tn_armed = tn < 0 or self.ready(tn)
            if tn_armed:
                arm(1, tn)
        while t >= 0:
            yield
            tnn = self.grab() if tn >= 0 else -1
            ok = yield from self.wait(lambda: st[y]["empty"])
            if not ok:
                if not tn_armed:
                    arm(y ^ 1, -1)
                break
            st[y]["empty"] = False
            self.store(t)
            yield
            published = False
            if not tn_armed:
                self.publish(t)
                published = True
                ok = yield from self.wait(lambda: self.ready(tn))
                if not ok:
                    arm(y ^ 1, -1)
                    break
                arm(y ^ 1, tn)
                tn_armed = True
            if tn < 0:
                if not published:
                    self.publish(t)
                break
            yield
            tnn_armed = tnn < 0 or self.ready(tnn)
            if tnn_armed:
                arm(y, tnn)
            if not published:
                self.publish(t)
            t, tn, tn_armed = tn, tnn, tnn_armed
            y ^= 1

    def compute(self, st):
        x = 0
        while True:
            ok = yield from self.wait(lambda: st[x]["full"])
            if not ok:
                return
            st[x]["full"] = False
            t = st[x]["ticket"]
            if t < 0:
                return
            for _ in range(self.rng.randint(0, 6)):
                yield
            self.computed.add(t)
            st[x]["empty"] = True
            x ^= 1

    def run(self):
        procs = []
        for _ in range(self.nctas):
            st = [{"ticket": -1, "full": False, "empty": False} for _ in range(2)]
            procs += [self.producer(st), self.compute(st)]
        live = list(procs)
        while live:
            p = self.rng.choice(live)
            try:
                next(p)
            except StopIteration:
                live.remove(p)
        return self


def configs(n, seed):
    r = random.Random(seed)
    for _ in range(n):
        nprob = r.randint(1, 3)
        yield [r.randint(1, 9) for _ in range(nprob)], r.randint(1, 6), r.randint(1, 7), r.randrange(1 << 30)


@pytest.mark.parametrize("problem_tiles,nspans,nctas,seed", list(configs(150, 2203)))
def test_every_ticket_completes_and_reads_published_state(problem_tiles, nspans, nctas, seed):
    sim = Protocol(problem_tiles, nspans, nctas, seed).run()
    assert not sim.violations, sim.violations[:3]
    assert not sim.err
    assert sim.computed == set(range(sim.total))
    assert sim.done == [nspans] * sim.ntiles


@pytest.mark.parametrize("seed", range(40))
def test_a_missing_publish_ends_in_a_latched_error_not_a_hang(seed):
    r = random.Random(seed)
    problem_tiles = [r.randint(2, 8) for _ in range(r.randint(1, 2))]
    nspans = r.randint(2, 5)
    ntiles = sum(problem_tiles)
    inject = (r.randrange(ntiles), r.randrange(nspans - 1))  # a span some ticket still needs
    sim = Protocol(problem_tiles, nspans, r.randint(1, 5), seed, inject=inject, poll_limit=2000).run()
    assert sim.err
    assert not sim.violations, sim.violations[:3]
    assert len(sim.computed) < sim.total


class OwnTileOnly(Protocol):
    """A planted protocol error: a ticket waits for its own tile only."""

    def ready(self, t):
        k, i = divmod(t, self.ntiles)
        return k == 0 or self.done[i] >= k


class PublishBeforeStore(Protocol):
    """A planted protocol error: the flag is raised before the core is stored."""

    def store(self, t):
        pass

    def publish(self, t):
        k, i = divmod(t, self.ntiles)
        self.done[i] = k + 1
        self.version[(k + 1) & 1][i] = (PENDING, k + 1)

    def load(self, t):
        super().load(t)
        # a pending store becomes visible some time after the flag
        for i in range(self.ntiles):
            for b in (0, 1):
                v = self.version[b][i]
                if isinstance(v, tuple) and self.rng.random() < 0.3:
                    self.version[b][i] = v[1]


@pytest.mark.parametrize("broken", [OwnTileOnly, PublishBeforeStore])
def test_the_model_catches_planted_protocol_errors(broken):
    caught = 0
    for problem_tiles, nspans, nctas, seed in configs(60, 7):
        sim = broken(problem_tiles, nspans, max(nctas, 3), seed, poll_limit=2000).run()
        caught += bool(sim.violations)
    assert caught > 0
