"""Element partition of a box into y-slabs for several GPUs (one process per
GPU), after Sec. 3.1 of the paper: non-overlapping partitions of whole
element columns, with one exchange of partition-face contributions per pass
of the right-hand side (the communication step of Alg. 3).

A domain of nel_y element rows is cut into ``parts`` slabs of consecutive
rows.  Slab r is an ordinary library context over its own elements whose y
nodes run from its lower face to its upper face, both included (the face
nodes are held by both neighbours).  xg_partition_set marks each end that
is a partition face; a periodic domain is a ring (slab 0's lower neighbour
is the last slab).  Between the two halves of every stage
(xg_partition_stage) each face is crossed by one array per direction: the
upper slab's partial face value and the lower slab's one-sided row, each
5 n_x n_z values.  Exchanges are point-to-point (torch.distributed
isend/irecv: NCCL between GPUs, gloo on the CPU); they are ordered by face
index so that two faces between the same pair of ranks (two slabs in a
ring) match in NCCL's issue order.

This module holds the host logic only: slab geometry, scattering and
gathering the global state, the exchange, and the driver of a partitioned
context.  Every step of the path runs in the library's kernels.
"""

from dataclasses import dataclass

import numpy as np


def slab_ranges(nel_y, parts):
    """[(e0, e1)] element-row ranges of the slabs, as even as possible
    (the first nel_y % parts slabs get one row more)."""
    if parts < 1 or nel_y < parts:
        raise ValueError("need 1 <= parts <= nel_y (got %d parts for %d rows)" % (parts, nel_y))
    q, r = divmod(nel_y, parts)
    out, e = [], 0
    for k in range(parts):
        n = q + (1 if k < r else 0)
        out.append((e, e + n))
        e += n
    return out


@dataclass(frozen=True)
class Slab:
    """Slab `rank` of `parts`: element rows [e0, e1) of a domain of
    nel = (nel_x, nel_y, nel_z) order-N elements over [lo, hi]."""
    rank: int
    parts: int
    e0: int
    e1: int
    nel: tuple
    N: int
    lo: tuple
    hi: tuple
    periodic: tuple

    @property
    def partitioned(self):
        return self.parts > 1

    @property
    def open_lo(self):
        return self.partitioned and (self.rank > 0 or self.periodic[1])

    @property
    def open_hi(self):
        return self.partitioned and (self.rank < self.parts - 1 or self.periodic[1])

    @property
    def lower(self):
        """Rank across the lower face (None at a wall)."""
        return (self.rank - 1) % self.parts if self.open_lo else None

    @property
    def upper(self):
        return (self.rank + 1) % self.parts if self.open_hi else None

    @property
    def faces(self):
        """Global indices of the faces at the slab's lower and upper ends
        (face f separates slab f - 1 from slab f; the ring's face 0 separates
        the last slab from slab 0)."""
        return self.rank, (self.rank + 1) % self.parts if self.periodic[1] else self.rank + 1

    @property
    def local_nel(self):
        return (self.nel[0], self.e1 - self.e0, self.nel[2])

    @property
    def local_periodic(self):
        return (self.periodic[0], self.periodic[1] and not self.partitioned, self.periodic[2])

    @property
    def local_lo_hi(self):
        h = (self.hi[1] - self.lo[1]) / self.nel[1]
        lo = (self.lo[0], self.lo[1] + self.e0 * h, self.lo[2])
        hi = (self.hi[0], self.lo[1] + self.e1 * h if self.e1 < self.nel[1] else self.hi[1],
              self.hi[2])
        return lo, hi

    def node_counts(self):
        """(global n_x, n_y, n_z) and the slab's local n_y."""
        n = [self.N * self.nel[d] + (0 if self.periodic[d] else 1) for d in range(3)]
        local_ny = self.N * (self.e1 - self.e0) + (0 if self.local_periodic[1] else 1)
        return n, local_ny

    def y_nodes(self):
        """Global y node index of each local y node (the periodic ring's last
        slab ends on global node 0)."""
        n, ny = self.node_counts()
        return (self.N * self.e0 + np.arange(ny)) % n[1]

    @property
    def face_values(self):
        """Values of one face array (5 variables x n_x x n_z)."""
        n, _ = self.node_counts()
        return 5 * n[0] * n[2]


def slab(rank, parts, nel, N, lo, hi, periodic):
    e0, e1 = slab_ranges(nel[1], parts)[rank]
    return Slab(rank, parts, e0, e1, tuple(int(v) for v in nel), int(N), tuple(lo), tuple(hi),
                tuple(bool(p) for p in periodic))


def scatter(q, s):
    """The slab's part [V][Np_local] of a global nodal array q [V][Np] (V
    variables, x fastest; numpy or torch)."""
    n, ny = s.node_counts()
    gy = s.y_nodes()
    qv = q.reshape(q.shape[0], n[2], n[1], n[0])
    idx = gy if isinstance(q, np.ndarray) else _torch_index(q, gy)
    return qv[:, :, idx, :].reshape(q.shape[0], -1)


def gather(parts, slabs):
    """The global array from every slab's part (face nodes from the lower
    slab's copy; both copies are equal after a partitioned pass)."""
    s0 = slabs[0]
    n, _ = s0.node_counts()
    v = parts[0].shape[0]
    out = np.empty((v, n[2], n[1], n[0]), dtype=np.asarray(parts[0]).dtype)
    for p, s in zip(parts[::-1], slabs[::-1]):
        _, ny = s.node_counts()
        out[:, :, s.y_nodes(), :] = np.asarray(p).reshape(v, n[2], ny, n[0])
    return out.reshape(v, -1)


def _torch_index(t, idx):
    import torch
    return torch.as_tensor(idx, device=t.device)


def exchange(s, send_lo, recv_lo, send_hi, recv_hi, group=None):
    """Swap the face arrays with the neighbours: recv_lo <- lower neighbour's
    send_hi, recv_hi <- upper neighbour's send_lo (torch tensors on the
    process group's device).  The operations are issued in ascending face
    order, so two faces shared by the same pair of ranks pair up correctly
    under in-order matching; the tag is the face index."""
    import torch.distributed as dist
    f_lo, f_hi = s.faces
    items = []
    if s.open_lo:
        items.append((f_lo, s.lower, send_lo, recv_lo))
    if s.open_hi:
        items.append((f_hi, s.upper, send_hi, recv_hi))
    items.sort(key=lambda it: it[0])
    ops = []
    for face, peer, snd, rcv in items:
        ops.append(dist.P2POp(dist.isend, snd, peer, group, tag=face))
        ops.append(dist.P2POp(dist.irecv, rcv, peer, group, tag=face))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


class PartitionedContext:
    """A library context over one slab with its exchange buffers: the
    partitioned counterpart of xg_step / xg_rhs.  ``exchanger(ctx)`` swaps
    the face arrays (by default :func:`exchange` over torch.distributed)."""

    def __init__(self, s, desc_kw, device, precision=0, exchanger=None):
        import torch
        from . import xg
        self.xg, self.torch, self.s = xg, torch, s
        self.dev = torch.device(device)
        lo, hi = s.local_lo_hi
        self.ctx = xg.xg_mesh_create(xg.mesh_desc(s.local_nel, s.N, lo, hi, s.local_periodic,
                                                  precision=precision, **desc_kw))
        self.np = xg.xg_mesh_np(self.ctx)
        nf = s.face_values
        buf = lambda: torch.zeros(nf, dtype=torch.float64, device=self.dev)
        self.send_lo, self.recv_lo, self.send_hi, self.recv_hi = buf(), buf(), buf(), buf()
        if s.partitioned:
            xg.xg_partition_set(self.ctx, s.open_lo, s.open_hi,
                                self.send_lo if s.open_lo else None, self.recv_lo if s.open_lo else None,
                                self.send_hi if s.open_hi else None, self.recv_hi if s.open_hi else None)
        self.exchanger = exchanger or (lambda c: exchange(c.s, c.send_lo, c.recv_lo, c.send_hi, c.recv_hi))

    def set_state(self, q_global, rho0, rhotheta0, S_global=None):
        t = self.torch
        dev = lambda a: t.as_tensor(np.ascontiguousarray(a), dtype=t.float64).to(self.dev)
        self.xg.xg_set_state(self.ctx, dev(scatter(q_global, self.s)), dev(rho0), dev(rhotheta0))
        if S_global is not None:
            self.xg.xg_set_forcing(self.ctx, dev(scatter(np.asarray(S_global)[None], self.s)[0]))

    def half(self, h, stage, dt=0.0, dqdt=None):
        self.xg.xg_partition_stage(self.ctx, h, stage, dt, dqdt)

    def state(self):
        out = self.torch.empty((5, self.np), dtype=self.torch.float64, device=self.dev)
        self.xg.xg_get_state(self.ctx, out)
        return out

    def close(self):
        if self.ctx:
            self.xg.xg_destroy(self.ctx)
            self.ctx = None


def step(ctxs, dt, nsteps):
    """nsteps SSP-RK3 steps of the slabs held by this process: each stage
    runs half 0 on every slab, the exchange, then half 1 on every slab."""
    for _ in range(nsteps):
        for stage in range(3):
            for c in ctxs:
                c.half(0, stage, dt)
            _exchange_all(ctxs)
            for c in ctxs:
                c.half(1, stage, dt)


def rhs(ctxs, outs):
    """dq/dt of every slab into outs (device tensors [5][Np_local])."""
    for c in ctxs:
        c.half(0, -1)
    _exchange_all(ctxs)
    for c, o in zip(ctxs, outs):
        c.half(1, -1, 0.0, o)


def _exchange_all(ctxs):
    seen = set()
    for c in ctxs:
        key = id(c.exchanger)
        if getattr(c.exchanger, "all_at_once", False):
            if key not in seen:
                seen.add(key)
                c.exchanger(None)
        else:
            c.exchanger(c)


class LocalExchange:
    """The exchange between slabs that live in one process (several
    contexts on one device): device copies of each face array to the
    neighbour's receive buffer, after every slab has run half 0 (nothing
    waits on a kernel of another slab)."""

    all_at_once = True

    def __init__(self):
        self.ctxs = []

    def add(self, c):
        self.ctxs.append(c)

    def __call__(self, _):
        by_rank = {c.s.rank: c for c in self.ctxs}
        for c in self.ctxs:
            if c.s.open_lo:
                c.recv_lo.copy_(by_rank[c.s.lower].send_hi)
            if c.s.open_hi:
                c.recv_hi.copy_(by_rank[c.s.upper].send_lo)
