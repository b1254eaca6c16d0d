"""The element partition on the GPU: a box cut into y-slabs (Sec. 3.1), each
slab its own context, with the partition-face rows exchanged between the two
halves of every stage (Alg. 3's communication step).  The slabs run in one
process on one GPU here, and the exchange is a device copy done after every
slab's first half (LocalExchange: no kernel waits on another slab's).  The
partitioned right-hand side and five SSP-RK3 steps equal the single-domain
context's bit for bit, in both FP64-accurate precisions, for a periodic ring
of slabs and for a walled domain, with two and three slabs of uneven size."""

import numpy as np
import pytest

from inputs import workloads as W
from paper_2504_08157_gb300 import partition as P

from helpers import GpuContext

pytestmark = pytest.mark.gpu

CASES = {
    "ring": lambda: W.tc(nel=(8, 6, 3), state="random"),
    "walled": lambda: W.box((3, 7, 2), 4, (0.0, 0.0, 0.0), (3000.0, 7000.0, 2000.0),
                            (True, False, False), seed=13),
}


def _desc_kw(wl):
    ph = wl["phys"]
    return dict(f=ph["f"], g=ph["g"], R=ph["R"], cp=ph["cp"], cv=ph["cv"], p_a=ph["p_a"])


def _slabs(wl, parts, prec):
    ex = P.LocalExchange()
    ctxs = []
    for r in range(parts):
        s = P.slab(r, parts, wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
        c = P.PartitionedContext(s, _desc_kw(wl), "cuda:0", prec, exchanger=ex)
        ex.add(c)
        c.set_state(wl["q"], wl["rho0"], wl["Theta0"], wl["S_theta"])
        ctxs.append(c)
    return ctxs


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
@pytest.mark.parametrize("case,parts", [("ring", 2), ("ring", 3), ("walled", 2), ("walled", 3)])
def test_partitioned_equals_single_domain(cuda_device, prec, case, parts):
    import torch
    wl = CASES[case]()
    with GpuContext(wl, precision=prec) as g:
        r_ref = g.rhs()
        g.step(5)
        q_ref = g.state()
    ctxs = _slabs(wl, parts, prec)
    try:
        slabs = [c.s for c in ctxs]
        outs = [torch.empty((5, c.np), dtype=torch.float64, device=cuda_device) for c in ctxs]
        P.rhs(ctxs, outs)
        torch.cuda.synchronize()
        r_part = [o.cpu().numpy() for o in outs]
        for o, s in zip(r_part, slabs):       # every slab's copy of its nodes, faces included
            assert np.array_equal(o, P.scatter(r_ref, s))
        assert np.array_equal(P.gather(r_part, slabs), r_ref)
        P.step(ctxs, wl["dt"], 5)
        q_part = [c.state().cpu().numpy() for c in ctxs]
        for o, s in zip(q_part, slabs):
            assert np.array_equal(o, P.scatter(q_ref, s))
    finally:
        for c in ctxs:
            c.close()


def test_partition_set_checks(cuda_device):
    """A partitioned context refuses the unpartitioned calls; the FP32 form,
    a periodic y direction and a missing buffer are rejected."""
    import torch
    from paper_2504_08157_gb300 import xg
    wl = CASES["walled"]()
    s = P.slab(0, 2, wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    c = P.PartitionedContext(s, _desc_kw(wl), "cuda:0", 0)
    try:
        c.set_state(wl["q"], wl["rho0"], wl["Theta0"])
        with pytest.raises(xg.XgError) as e:
            xg.xg_step(c.ctx, 0.01, 1)
        assert e.value.status == xg.XG_ERR_UNSUPPORTED
        with pytest.raises(xg.XgError) as e:
            xg.xg_rhs(c.ctx, torch.empty((5, c.np), dtype=torch.float64, device=cuda_device))
        assert e.value.status == xg.XG_ERR_UNSUPPORTED
        with pytest.raises(xg.XgError) as e:
            xg.xg_partition_set(c.ctx, 0, 1, None, None, None, None)
        assert e.value.status == xg.XG_ERR_ARG
        xg.xg_partition_set(c.ctx, 0, 0)                 # back to a walled context
        xg.xg_step(c.ctx, 0.01, 1)
    finally:
        c.close()
    with GpuContext(W.tc(nel=(4, 4, 2)), precision=1) as g:
        buf = torch.zeros(5 * 16 * 9, dtype=torch.float64, device=cuda_device)
        with pytest.raises(xg.XgError) as e:                # periodic in y
            xg.xg_partition_set(g.ctx, 1, 0, buf, buf)
        assert e.value.status == xg.XG_ERR_ARG
    wl = CASES["walled"]()
    with GpuContext(wl, precision=1) as g:
        buf = torch.zeros(5 * 13 * 9, dtype=torch.float64, device=cuda_device)
        with pytest.raises(xg.XgError) as e:                # FP32 form
            xg.xg_partition_set(g.ctx, 1, 0, buf, buf)
        assert e.value.status == xg.XG_ERR_UNSUPPORTED
