"""Shared helpers of the tests: oracle set-up, the GPU path through the C ABI
(torch tensors for device memory), and the relative L2 metric."""

import numpy as np

from inputs import workloads as W  # noqa: F401
from oracle import euler as E, mesh as M, ssprk3


def rel_l2(a, b):
    """||a - b|| / ||b|| over nodes for one variable; the absolute norm when
    ||b|| is (numerically) zero."""
    nb = np.linalg.norm(b)
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    return d / nb if nb > 1e-300 else d


def rel_l2_per_var(a, b):
    return np.array([rel_l2(a[v], b[v]) for v in range(a.shape[0])])


def oracle_of(wl, elements=None):
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], elements=elements)
    phys = E.Physics(**wl["phys"])
    base = E.Base(wl["rho0"], wl["Theta0"])
    return m, phys, base


def oracle_rhs(wl, q=None):
    m, phys, base = oracle_of(wl)
    return E.rhs(m, wl["q"] if q is None else q, base, wl["S_theta"], phys)


def oracle_of_extended(wl, elements=None):
    """The oracle's mesh, physics and reference state for an evaluation in
    extended precision (np.longdouble): the same definitions with rounding
    far below FP64's, the reference where a tendency is a small residual of
    cancelling parts (the pure-vortex state)."""
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], elements=elements,
                     dtype=np.longdouble)
    return m, E.Physics(**wl["phys"]), E.Base(wl["rho0"], wl["Theta0"])


def _ld(a):
    return None if a is None else np.asarray(a, dtype=np.longdouble)


def oracle_rhs_extended(wl, q=None):
    """E.rhs in extended precision, returned as float64."""
    m, phys, base = oracle_of_extended(wl)
    return E.rhs(m, _ld(wl["q"] if q is None else q), base, _ld(wl["S_theta"]), phys).astype(np.float64)


def oracle_rhs_at_nodes_extended(wl, nodes, q=None):
    """E.rhs_at_nodes in extended precision on the elements around the nodes."""
    el = M.elements_around(wl["nel"], wl["N"], wl["periodic"], nodes)
    m, phys, base = oracle_of_extended(wl, elements=el)
    return E.rhs_at_nodes(m, _ld(wl["q"] if q is None else q), base, _ld(wl["S_theta"]), phys,
                          nodes).astype(np.float64)


def oracle_steps(wl, nsteps, q=None):
    m, phys, base = oracle_of(wl)
    L = lambda s: E.rhs(m, s, base, wl["S_theta"], phys)
    return ssprk3.run(L, wl["q"] if q is None else q, wl["dt"], nsteps)


class GpuContext:
    """One library context for a workload, inputs resident on cuda:0."""

    def __init__(self, wl, device="cuda:0", precision=0):
        import torch
        from paper_2504_08157_gb300 import xg
        self.xg, self.torch, self.wl = xg, torch, wl
        self.dev = torch.device(device)
        ph = wl["phys"]
        self.ctx = xg.xg_mesh_create(xg.mesh_desc(
            wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], f=ph["f"], g=ph["g"],
            R=ph["R"], cp=ph["cp"], cv=ph["cv"], p_a=ph["p_a"], precision=precision))
        self.np = xg.xg_mesh_np(self.ctx)
        self.set_state(wl["q"], with_base=True)
        if wl["S_theta"] is not None:
            xg.xg_set_forcing(self.ctx, torch.from_numpy(np.ascontiguousarray(wl["S_theta"])).to(self.dev))

    def set_state(self, q, with_base=False):
        t = self.torch
        qd = t.from_numpy(np.ascontiguousarray(q)).to(self.dev)
        if with_base:
            self.xg.xg_set_state(self.ctx, qd, t.from_numpy(self.wl["rho0"]).to(self.dev),
                                 t.from_numpy(self.wl["Theta0"]).to(self.dev))
        else:
            self.xg.xg_set_state(self.ctx, qd)
        self.torch.cuda.synchronize()

    def rhs(self):
        out = self.torch.empty((5, self.np), dtype=self.torch.float64, device=self.dev)
        self.xg.xg_rhs(self.ctx, out)
        return out.cpu().numpy()

    def step(self, nsteps, dt=None):
        self.xg.xg_step(self.ctx, self.wl["dt"] if dt is None else dt, nsteps)

    def state(self):
        out = self.torch.empty((5, self.np), dtype=self.torch.float64, device=self.dev)
        self.xg.xg_get_state(self.ctx, out)
        return out.cpu().numpy()

    def close(self):
        if self.ctx:
            self.xg.xg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchRun:
    """A batch of XG_FP32 instances (the batched persistent form), one per
    workload, inputs resident on cuda:0."""

    def __init__(self, wls, device="cuda:0"):
        import torch
        from paper_2504_08157_gb300 import xg
        self.xg, self.torch, self.wls = xg, torch, list(wls)
        self.dev = torch.device(device)
        descs = []
        for wl in self.wls:
            ph = wl["phys"]
            descs.append(xg.mesh_desc(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"],
                                      f=ph["f"], g=ph["g"], R=ph["R"], cp=ph["cp"], cv=ph["cv"],
                                      p_a=ph["p_a"], precision=xg.XG_FP32))
        self.b = xg.xg_batch_create(descs)
        self.ctx = [xg.xg_batch_instance(self.b, i) for i in range(len(self.wls))]
        self.np = [xg.xg_mesh_np(c) for c in self.ctx]
        for c, wl in zip(self.ctx, self.wls):
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)
            xg.xg_set_state(c, t(wl["q"]), t(wl["rho0"]), t(wl["Theta0"]))
            if wl["S_theta"] is not None:
                xg.xg_set_forcing(c, t(wl["S_theta"]))
        torch.cuda.synchronize()

    @property
    def dts(self):
        return [wl["dt"] for wl in self.wls]

    def rhs(self):
        outs = [self.torch.empty((5, n), dtype=self.torch.float64, device=self.dev) for n in self.np]
        self.xg.xg_batch_rhs(self.b, outs)
        return [o.cpu().numpy() for o in outs]

    def step(self, nsteps):
        self.xg.xg_batch_step(self.b, self.dts, nsteps)

    def states(self):
        outs = []
        for c, n in zip(self.ctx, self.np):
            o = self.torch.empty((5, n), dtype=self.torch.float64, device=self.dev)
            self.xg.xg_get_state(c, o)
            outs.append(o)
        return [o.cpu().numpy() for o in outs]

    def close(self):
        if self.b:
            self.xg.xg_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
