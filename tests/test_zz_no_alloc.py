"""xg_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (for example code living inside another framework's memory pool).
It keeps its intermediates in one fixed device array instead of cudaMalloc'd
buffers.  Checked here through the C ABI against the context entry point
xg_rhs, on two calls in a row (with different meshes, so the second call
also runs over the first call's leftovers in the shared array), plus the
size limit.  This file is collected last on purpose."""

import numpy as np
import pytest

from inputs import workloads as W

from helpers import GpuContext, rel_l2_per_var

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-12


def _desc(xg, wl):
    ph = wl["phys"]
    return xg.mesh_desc(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], f=ph["f"],
                        g=ph["g"], R=ph["R"], cp=ph["cp"], cv=ph["cv"], p_a=ph["p_a"])


def _noalloc_rhs(xg, torch, dev, wl):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, r0, t0 = t(wl["q"]), t(wl["rho0"]), t(wl["Theta0"])
    S = t(wl["S_theta"]) if wl["S_theta"] is not None else None
    out = torch.full((5, q.shape[1]), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    xg.xg_rhs_noalloc(_desc(xg, wl), q, r0, t0, S, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(dev)[0]
    return out.cpu().numpy(), free0, free1


def test_noalloc_rhs_matches_context_rhs(cuda_device):
    import torch
    from paper_2504_08157_gb300 import build, xg
    build.build()
    first = W.tc(nel=(16, 16, 4), state="random")    # 64 x 64 x 17 nodes, heating, Coriolis
    second = W.bubble(state="random")                 # 33^3 nodes, walls, no heating
    for k, wl in enumerate((first, second)):
        got, free0, free1 = _noalloc_rhs(xg, torch, cuda_device, wl)
        with GpuContext(wl) as g:
            ref = g.rhs()
        err = rel_l2_per_var(got, ref)
        assert np.all(np.isfinite(got))
        assert np.all(err <= RHS_TOL), (k, err)
        if k == 1:
            # after the first call has set the device up, a call changes no
            # device memory reservation
            assert free1 == free0


def test_noalloc_rejects_meshes_beyond_the_scratch(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    wl = W.tc(nel=(32, 32, 16))                       # 128 x 128 x 65 nodes: too large
    n = wl["q"].shape[1]
    assert 8 * n * 8 > 16 * 2 ** 20
    dev = cuda_device
    q = torch.zeros((5, n), dtype=torch.float64, device=dev)
    r0 = torch.from_numpy(wl["rho0"]).to(dev)
    t0 = torch.from_numpy(wl["Theta0"]).to(dev)
    out = torch.empty_like(q)
    with pytest.raises(xg.XgError) as e:
        xg.xg_rhs_noalloc(_desc(xg, wl), q, r0, t0, None, out)
    assert e.value.status == xg.XG_ERR_UNSUPPORTED
