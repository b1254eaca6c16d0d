"""Hyper-diffusion, the sponge and the RI-velocity diagnostic
(include/xg_dynamics.h) against the oracle (oracle/dynamics.py): the extra
tendency, the right-hand side and SSP-RK3 steps with the terms set (FP64
bars: 1e-12 per evaluation, 1e-10 after the steps), and the diagnostic on
FP64 and FP32 contexts."""

import numpy as np
import pytest

from inputs import workloads as W
from oracle import dynamics as Y, euler as E, ssprk3

from helpers import GpuContext, oracle_of, rel_l2_per_var

pytestmark = pytest.mark.gpu

C = (2.0, 1.0, 1.0)       # largest element size (y here) first; x and z tie
DT_H = 0.5
DEPTH, GAMMA = 1200.0, 0.05


def _case(N=4, per=(True, False, False), seed=51):
    return W.box((3, 2, 2), N, (0.0, 0.0, 0.0), (3000.0, 3000.0, 2000.0), per, seed=seed)


def _oracle_terms(wl, q=None):
    m, phys, base = oracle_of(wl)
    tau = Y.viscosity_tensor(m, C, DT_H)
    q = wl["q"] if q is None else q
    return m, phys, base, tau, Y.hyperdiffusion(m, q, tau) + Y.sponge(m, q, DEPTH, GAMMA)


@pytest.mark.parametrize("N,per", [(3, (True, False, False)), (4, (False, False, False)),
                                   (5, (True, True, False))])
def test_extra_tendency_matches_oracle(cuda_device, N, per):
    import torch
    wl = _case(N, per)
    with GpuContext(wl) as g:
        g.xg.xg_set_dynamics(g.ctx, C, DT_H, DEPTH, GAMMA)
        out = torch.empty((5, g.np), dtype=torch.float64, device=cuda_device)
        g.xg.xg_dynamics_tendency(g.ctx, out)
        got = out.cpu().numpy()
    ref = _oracle_terms(wl)[4]
    err = rel_l2_per_var(got, ref)
    assert np.all(err <= 1e-12), err


def test_rhs_and_steps_with_the_terms(cuda_device):
    """Steps with explicit hyper-diffusion need c small enough for the
    explicit step: grid-scale damping nu^2 k^4 dt grows with the clustering
    of the LGL nodes (here c ~ 1e-6 at the step size)."""
    wl = _case(4, (True, False, False), seed=53)
    m, phys, base = oracle_of(wl)
    c = (2e-6, 1e-6, 1e-6)
    tau = Y.viscosity_tensor(m, c, wl["dt"])

    def L(s):
        extra = Y.hyperdiffusion(m, s, tau) + Y.sponge(m, s, DEPTH, GAMMA)
        return E.apply_walls(m, E.rhs(m, s, base, wl["S_theta"], phys) + extra)

    with GpuContext(wl) as g:
        g.xg.xg_set_dynamics(g.ctx, c, wl["dt"], DEPTH, GAMMA)
        r = g.rhs()
        assert np.all(rel_l2_per_var(r, L(wl["q"])) <= 1e-12)
        g.step(10)
        q = g.state()
    ref = ssprk3.run(L, wl["q"], wl["dt"], 10)
    assert np.all(rel_l2_per_var(q, ref) <= 1e-10)
    assert np.all(rel_l2_per_var(q - wl["q"], ref - wl["q"]) <= 1e-10)


def test_terms_off_and_unsupported(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    wl = _case()
    with GpuContext(wl) as g:
        plain = g.rhs()
        xg.xg_set_dynamics(g.ctx, C, DT_H, DEPTH, GAMMA)
        xg.xg_set_dynamics(g.ctx, off=True)
        assert np.array_equal(g.rhs(), plain)
        out = torch.ones((5, g.np), dtype=torch.float64, device=cuda_device)
        xg.xg_dynamics_tendency(g.ctx, out)
        assert torch.count_nonzero(out) == 0
        for bad in (dict(hyper_c=(-1.0, 0.0, 0.0)), dict(hyper_c=(1.0, 1.0, 1.0), hyper_dt=0.0),
                    dict(sponge_depth=5000.0, sponge_gamma=0.1)):
            with pytest.raises(xg.XgError) as e:
                xg.xg_set_dynamics(g.ctx, **bad)
            assert e.value.status == xg.XG_ERR_ARG
    for prec in (1, 2):
        with GpuContext(wl, precision=prec) as g:
            with pytest.raises(xg.XgError) as e:
                xg.xg_set_dynamics(g.ctx, C, DT_H)
            assert e.value.status == xg.XG_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_ri_velocity_matches_oracle(cuda_device, prec):
    wl = W.tc(nel=(12, 12, 4), state="initial")
    with GpuContext(wl, precision=prec) as g:
        u, cent, means = g.xg.xg_ri_velocity(g.ctx, 50)
        q = g.state()
    m, _, _ = oracle_of(wl)
    ru, rcent, rmeans = Y.ri_velocity(m, q, wl["rho0"], nstrips=50)
    assert abs(u - ru) <= 1e-12 * ru
    assert np.allclose(cent, rcent, rtol=0, atol=1e-9 * 1e6)
    assert np.allclose(means, rmeans, rtol=1e-12, atol=1e-12)
    assert 5.0 < u < 20.0          # the 15 m/s vortex, averaged over strips
