"""One problem split over the ranks of a process group (one GPU per rank).

The paper puts the N subdomains of a problem in a row (Sec. 3), and its
update step (Sec. 2.5) hands every subdomain the state that its neighbours
computed.  Here the N subdomains are dealt to the ranks in contiguous blocks,
and the update across a rank boundary is a point-to-point exchange.

Rank r owns the subdomains [i0, i1) of the problem's decomposition, that is
the core points [c0, c1) = [b_i0, b_i1) with b_i = floor(i nx / N).  It keeps
the part [lo, hi) = [max(c0 - h, 0), min(c1 + h, nx)) of the grid: its owned
points plus a halo of h points beside each cut.  A round advances the part by
s <= h steps from the true state through a part plan
(rswr_plan_create_part: the whole grid's coefficients, the part's own
subdomains).  The end node of the part at a cut holds a guess: its level-0
value is the true one, later levels are 0.  A guess travels one point per
step, so after s <= h steps every owned point is exact: the Waveform Time Span
Theorem (Sec. 2.4) with the part as the window.  Then each rank sends the h
owned points beside each cut, both state components, to the neighbour that
keeps them as halo, and receives its own halos.  With h = floor(overlap / 2)
a round is one span of the paper's loop and the exchange is its update step.

The owned points of every rank then equal the whole-grid run, and so the
monolithic solve, bit for bit.

The local solver is the library (a part plan on the rank's GPU).  A caller
may pass another solver with the same ``run`` method; the CPU tests pass the
oracle running the same part, so that the partition and the exchange are
checked on gloo ranks without a GPU.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Block:
    """The share of one rank: subdomains [i0, i1), owned points [c0, c1),
    kept part [lo, hi)."""
    i0: int
    i1: int
    c0: int
    c1: int
    lo: int
    hi: int


def partition(nx: int, n_sub: int, world: int, halo: int) -> list[Block]:
    """Contiguous blocks of subdomains, one per rank, as even in subdomain
    count as possible (the subdomains of the decomposition have equal sizes up
    to one point).  Every rank must own at least `halo` points, so that its
    halos come from its two neighbours only."""
    if world < 1 or n_sub < world:
        raise ValueError("need 1 <= world <= n_sub")
    if halo < 1:
        raise ValueError("halo must be >= 1")
    b = lambda i: i * nx // n_sub
    out = []
    for r in range(world):
        i0, i1 = r * n_sub // world, (r + 1) * n_sub // world
        c0, c1 = b(i0), b(i1)
        if c1 - c0 < halo:
            raise ValueError(f"rank {r} owns {c1 - c0} points, fewer than the halo of {halo}")
        out.append(Block(i0, i1, c0, c1, max(c0 - halo, 0), min(c1 + halo, nx)))
    return out


class PartSolver:
    """The library on the rank's GPU: a part plan for [blk.lo, blk.hi) with the
    rank's own subdomains (one per owned subdomain; the halos widen the first
    and the last)."""

    def __init__(self, xa, xb, a, nx, dt, blk: Block, overlap: int, dtype, device):
        from . import rswr

        self.plan = rswr.Plan.part(xa, xb, a, nx, dt, blk.lo, blk.hi, blk.i1 - blk.i0, overlap, dtype=dtype,
                                   device=device)
        # every round passes other state buffers: launch directly, no graph capture
        self.plan.set_graph(False)

    def run(self, fA, fB, steps, u, w, out, j_r=None):
        """`steps` steps of the part from (u, w) into out = (u', w'); returns the
        receiver trace (levels 0..steps) at local point j_r, or None."""
        r = self.plan.run(fA, fB, steps, q0=u, q1=w, j_r=j_r, out=out)
        return r["recv"]


class SplitPlan:
    """One problem, (xa, xb, a, nx, dt) with n_sub subdomains sharing `overlap`
    points, split over the `world` ranks of torch.distributed (`dist` is the
    torch.distributed module, already initialised; None for one rank).

    halo: the h of the module docstring (default floor(overlap / 2)); a round
    advances h steps.  solver: the local solver (default PartSolver on
    `device`); it is constructed as solver(xa, xb, a, nx, dt, block, overlap,
    dtype, device)."""

    def __init__(self, xa, xb, a, nx, dt, n_sub, overlap, rank, world, dist=None, dtype=None, halo=None,
                 device=None, solver=None):
        import torch

        from . import rswr

        self.xa, self.xb, self.a, self.nx, self.dt = xa, xb, a, nx, dt
        self.n_sub, self.overlap = n_sub, overlap
        self.rank, self.world, self.dist = rank, world, dist
        self.dtype = rswr.F64 if dtype is None else dtype
        self.halo = overlap // 2 if halo is None else int(halo)
        self.blocks = partition(nx, n_sub, world, self.halo)
        self.blk = self.blocks[rank]
        self.device = torch.device("cuda" if device is None else device)
        self.tdtype = torch.float64 if self.dtype == rswr.F64 else torch.float32
        make = PartSolver if solver is None else solver
        self.solver = make(xa, xb, a, nx, dt, self.blk, overlap, self.dtype, self.device)
        self.exchanged_bytes = 0

    @classmethod
    def from_problem(cls, p, rank, world, dist=None, **kw):
        return cls(p.xa, p.xb, p.a, p.nx, p.dt, p.n_sub, p.overlap, rank, world, dist, **kw)

    # ---- the exchange of the update step across rank boundaries ----------

    def _exchange(self, u, w):
        """Send the h owned points beside each cut (both components) to the
        neighbour that keeps them as halo; receive this rank's halos."""
        import torch

        if self.world == 1:
            return
        b, h, r = self.blk, self.halo, self.rank
        dist = self.dist
        ops, recv = [], []
        if r > 0:  # left neighbour: my first h owned points; my left halo is its last h
            send = torch.stack([u[b.c0 - b.lo:b.c0 - b.lo + h], w[b.c0 - b.lo:b.c0 - b.lo + h]]).contiguous()
            buf = torch.empty((2, h), dtype=u.dtype, device=u.device)
            ops += [dist.P2POp(dist.isend, send, r - 1), dist.P2POp(dist.irecv, buf, r - 1)]
            recv.append((0, buf, send))
        if r + 1 < self.world:  # right neighbour: my last h owned points; my right halo is its first h
            send = torch.stack([u[b.c1 - b.lo - h:b.c1 - b.lo], w[b.c1 - b.lo - h:b.c1 - b.lo]]).contiguous()
            buf = torch.empty((2, h), dtype=u.dtype, device=u.device)
            ops += [dist.P2POp(dist.isend, send, r + 1), dist.P2POp(dist.irecv, buf, r + 1)]
            recv.append((b.c1 - b.lo, buf, send))
        # one group: with NCCL, separately posted sends and receives between
        # neighbours could wait on each other
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for at, buf, send in recv:
            u[at:at + h].copy_(buf[0])
            w[at:at + h].copy_(buf[1])
            self.exchanged_bytes += 2 * send.numel() * send.element_size()

    # ---- the run -----------------------------------------------------------

    def run(self, fA, fB, T, q0=None, q1=None, j_r=None):
        """T steps from the state pair (q0, q1) (whole-grid arrays; None: zero
        data at rest) with the Dirichlet samples fA, fB (T+1 each; None: 0).
        Returns dict(u, w) of this rank's owned points [c0, c1) and, when j_r is
        given, recv: the receiver trace u^n_{j_r}, n = 0..T, on every rank."""
        import torch

        b, h, dev, td = self.blk, self.halo, self.device, self.tdtype
        n = b.hi - b.lo
        as_t = lambda x: None if x is None else torch.as_tensor(x).to(device=dev, dtype=td).contiguous()
        fA_t = as_t(fA) if fA is not None else torch.zeros(T + 1, dtype=td, device=dev)
        fB_t = as_t(fB) if fB is not None else torch.zeros(T + 1, dtype=td, device=dev)
        u = torch.zeros(n, dtype=td, device=dev) if q0 is None else as_t(q0)[b.lo:b.hi].clone()
        if q1 is not None:
            w = as_t(q1)[b.lo:b.hi].clone()
        elif q0 is not None and self._canonical():
            w = u.clone()  # at rest: u^{-1} = u^0
        else:
            w = torch.zeros(n, dtype=td, device=dev)
        if q0 is None:
            # zero data: the boundary nodes carry the level-0 samples
            if b.lo == 0:
                u[0] = fA_t[0]
                if self._canonical():
                    w[0] = fA_t[0]
            if b.hi == self.nx:
                u[-1] = fB_t[0]
                if self._canonical():
                    w[-1] = fB_t[0]
        out = (torch.empty_like(u), torch.empty_like(w))
        # the guesses at the cuts: the true value at level 0, then 0
        gL = torch.zeros(h + 1, dtype=td, device=dev)
        gR = torch.zeros(h + 1, dtype=td, device=dev)
        own_recv = j_r is not None and b.c0 <= j_r < b.c1
        recv = torch.zeros(T + 1, dtype=td, device=dev) if j_r is not None else None
        n0 = 0
        while n0 < T:
            s = min(h, T - n0)
            if b.lo == 0:
                fa = fA_t[n0:n0 + s + 1]
            else:
                gL[0] = u[0]
                fa = gL[:s + 1]
            if b.hi == self.nx:
                fb = fB_t[n0:n0 + s + 1]
            else:
                gR[0] = u[-1]
                fb = gR[:s + 1]
            tr = self.solver.run(fa, fb, s, u, w, out, j_r=(j_r - b.lo) if own_recv else None)
            if own_recv:
                recv[n0:n0 + s + 1] = tr
            u, out = out[0], (u, out[1])
            w, out = out[1], (out[0], w)
            self._exchange(u, w)
            n0 += s
        if recv is not None and self.world > 1:
            owner = next(r for r, blk in enumerate(self.blocks) if blk.c0 <= j_r < blk.c1)
            self.dist.broadcast(recv, owner)
        return {"u": u[b.c0 - b.lo:b.c1 - b.lo], "w": w[b.c0 - b.lo:b.c1 - b.lo], "recv": recv}

    def _canonical(self) -> bool:
        from . import rswr

        return self.dtype == rswr.F64 if self.form is None else self.form == rswr.FORM_CANONICAL

    form = None  # the state form: None = the library default of the dtype

    def gather(self, x, dst=0):
        """The whole grid's array on rank dst from every rank's owned part x
        (point-to-point; other ranks get None)."""
        import torch

        if self.world == 1:
            return x.clone()
        if self.rank != dst:
            self.dist.send(x.contiguous(), dst)
            return None
        full = torch.empty(self.nx, dtype=x.dtype, device=x.device)
        for r, blk in enumerate(self.blocks):
            if r == dst:
                full[blk.c0:blk.c1] = x
            else:
                buf = torch.empty(blk.c1 - blk.c0, dtype=x.dtype, device=x.device)
                self.dist.recv(buf, r)
                full[blk.c0:blk.c1] = buf
        return full
