"""The element partition's host logic (paper_2504_08157_gb300/partition.py) on
the CPU: slab geometry, scatter/gather, and the face exchange between two
gloo ranks driving the oracle's partitioned right-hand side.

Sec. 3.1 partitions the elements (whole columns) and Alg. 3 exchanges the
partition-face partial sums once per right-hand side.  Here each rank holds
one y-slab, computes the oracle's pointwise S(q) and partial DSS sums R, M
over its own elements, sends the partial sums of its two face planes to the
neighbours with partition.exchange and adds what it receives, then divides
by M and applies the walls: the two-rank right-hand side, and ten SSP-RK3
steps with an exchange in every stage, equal the single-domain oracle's to
rounding (1e-14: a slab's oracle mesh computes its node coordinates, and so
its metric terms, from its own corners)."""

import os
import socket

import numpy as np
import pytest

from paper_2504_08157_gb300 import partition as P


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CASES = {
    # periodic in y: a ring of two slabs (both faces shared by the same pair)
    "ring": dict(kind="tc", nel=(4, 6, 3)),
    # walls in y: one interior face; uneven slabs (5 rows into 3 + 2)
    "walled": dict(kind="box", nel=(3, 5, 2)),
}


def _workload(case):
    from inputs import workloads as W
    c = CASES[case]
    if c["kind"] == "tc":
        return W.tc(nel=c["nel"], state="random")
    nel = c["nel"]
    return W.box(nel, 4, (0.0, 0.0, 0.0), tuple(1000.0 * n for n in nel), (True, False, False),
                 seed=5)


# ------------------------------------------------------------------ geometry (one process)

@pytest.mark.parametrize("parts", [1, 2, 3, 5])
@pytest.mark.parametrize("periodic_y", [False, True])
def test_slabs_cover_the_domain(parts, periodic_y):
    nel, N = (3, 7, 2), 4
    lo, hi = (0.0, -3.5e3, 0.0), (3e3, 3.5e3, 2e3)
    per = (True, periodic_y, False)
    slabs = [P.slab(r, parts, nel, N, lo, hi, per) for r in range(parts)]
    rows = [r for s in slabs for r in range(s.e0, s.e1)]
    assert rows == list(range(nel[1]))
    assert max(s.e1 - s.e0 for s in slabs) - min(s.e1 - s.e0 for s in slabs) <= 1
    h = (hi[1] - lo[1]) / nel[1]
    for s in slabs:
        llo, lhi = s.local_lo_hi
        assert np.isclose(llo[1], lo[1] + s.e0 * h) and np.isclose(lhi[1], lo[1] + s.e1 * h)
        assert s.local_periodic[1] == (periodic_y and parts == 1)
        _, ny = s.node_counts()
        assert len(s.y_nodes()) == ny
        if parts > 1:
            assert s.open_lo == (s.rank > 0 or periodic_y)
            assert s.open_hi == (s.rank < parts - 1 or periodic_y)
    # every global node is in some slab; face nodes in exactly two
    n, _ = slabs[0].node_counts()
    count = np.zeros(n[1], dtype=int)
    for s in slabs:
        np.add.at(count, s.y_nodes(), 1)
    assert np.all(count >= 1)
    assert np.all(count <= (2 if parts > 1 else 1))
    # scatter / gather round trip
    q = np.random.default_rng(1).normal(size=(5, n[0] * n[1] * n[2]))
    parts_q = [P.scatter(q, s) for s in slabs]
    assert np.array_equal(P.gather(parts_q, slabs), q)


def test_ring_faces_are_ordered_for_in_order_matching():
    """Two slabs in a ring share both faces; each rank lists its face
    operations in ascending face order, and the sender's order on every
    channel equals the receiver's."""
    s0 = P.slab(0, 2, (2, 4, 2), 4, (0, 0, 0), (1, 1, 1), (True, True, False))
    s1 = P.slab(1, 2, (2, 4, 2), 4, (0, 0, 0), (1, 1, 1), (True, True, False))
    assert s0.faces == (0, 1) and s1.faces == (1, 0)
    assert s0.lower == s0.upper == 1 and s1.lower == s1.upper == 0
    # rank 0 sends over faces (0: its send_lo, 1: its send_hi); rank 1
    # receives over faces (0: its recv_hi, 1: its recv_lo): matched in order
    sends0 = sorted([(s0.faces[0], "lo"), (s0.faces[1], "hi")])
    recvs1 = sorted([(s1.faces[0], "lo"), (s1.faces[1], "hi")])
    assert [f for f, _ in sends0] == [f for f, _ in recvs1]
    assert [side for _, side in sends0] == ["lo", "hi"] and [side for _, side in recvs1] == ["hi", "lo"]


# ------------------------------------------------------------------ two gloo ranks

def _partitioned_rhs_factory(case, rank, world):
    """dq/dt of this rank's slab: the oracle's partial sums over the slab's
    elements, the face planes exchanged with partition.exchange."""
    import torch
    from oracle import euler as E, mesh as M
    wl = _workload(case)
    s = P.slab(rank, world, wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    llo, lhi = s.local_lo_hi
    m = M.build_mesh(s.local_nel, wl["N"], llo, lhi, s.local_periodic)
    phys = E.Physics(**wl["phys"])
    base = E.Base(wl["rho0"], wl["Theta0"])
    S = P.scatter(wl["S_theta"][None], s)[0] if wl["S_theta"] is not None else None
    n, ny = s.node_counts()
    nx, nz = n[0], n[2]

    def planes(a, y):   # a [V][Np_local] -> [V][n_z][n_x] of local plane y
        return a.reshape(a.shape[0], nz, ny, nx)[:, :, y, :]

    def exchange_sum(A):
        v = A.shape[0]
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x).reshape(-1))
        send_lo, send_hi = t(planes(A, 0)), t(planes(A, ny - 1))
        recv_lo, recv_hi = torch.zeros_like(send_lo), torch.zeros_like(send_hi)
        P.exchange(s, send_lo, recv_lo, send_hi, recv_hi)
        A = A.reshape(v, nz, ny, nx).copy()
        if s.open_lo:
            A[:, :, 0, :] += recv_lo.numpy().reshape(v, nz, nx)
        if s.open_hi:
            A[:, :, ny - 1, :] += recv_hi.numpy().reshape(v, nz, nx)
        return A.reshape(v, -1)

    _, Mloc = E.assemble(m, np.zeros((1,) + m.intma.shape))
    Mass = exchange_sum(Mloc[None])[0]
    walls_y = m.wall_nodes(1)
    gy = np.arange(m.Np) // nx % ny
    if s.open_lo:
        walls_y &= gy != 0
    if s.open_hi:
        walls_y &= gy != ny - 1

    def L(q):
        Sl = E.local_tendency(m, q, base, S, phys)
        R, _ = E.assemble(m, Sl)
        out = exchange_sum(R) / Mass[None]
        out[1][m.wall_nodes(0)] = 0.0
        out[2][walls_y] = 0.0
        out[3][m.wall_nodes(2)] = 0.0
        return out

    return wl, s, L


def _worker(case, rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import euler as E, mesh as M, ssprk3
        wl, s, L = _partitioned_rhs_factory(case, rank, world)
        q0 = P.scatter(wl["q"], s)
        r = L(q0)
        qs = ssprk3.run(L, q0, wl["dt"], 10)
        m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
        phys, base = E.Physics(**wl["phys"]), E.Base(wl["rho0"], wl["Theta0"])
        Lg = lambda x: E.rhs(m, x, base, wl["S_theta"], phys)
        ref_r = P.scatter(Lg(wl["q"]), s)
        ref_q = P.scatter(ssprk3.run(Lg, wl["q"], wl["dt"], 10), s)
        rel = lambda a, b: [float(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300))
                            for v in range(5)]
        inc = lambda a, b: rel(a - q0, b - q0)
        q.put((rank, rel(r, ref_r), rel(qs, ref_q), inc(qs, ref_q)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_gloo_ranks_match_the_single_domain_oracle(case):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(case, r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for _ in range(2):
        rank, e_rhs, e_state, e_inc = q.get(timeout=10)
        # to rounding: a slab's oracle mesh computes its node coordinates
        # (hence its metric terms) from its own corners
        assert max(e_rhs) <= 1e-14, (rank, e_rhs)
        assert max(e_state) <= 1e-14, (rank, e_state)
        assert max(e_inc) <= 1e-13, (rank, e_inc)
