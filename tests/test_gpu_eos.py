"""Both branches of the equation of state (Sec. 2.1, Eq. 3) on the GPU, in
every precision, against the FP64 oracle.

The kernels evaluate p' = p_0 ((1 + x)^gamma - 1), x = Theta'/Theta_0, by a
binomial series for |x| < x_max and by expm1(gamma log1p(x)) beyond.  The
workload ``eos_span`` puts |x| between 1e-7 and 0.25, so one right-hand side
runs both; the library's own x_max (about 0.0169 for gamma = 1.4) is checked
to lie inside that range.  The switch itself is checked node by node through
the test hook xg_pressure_perturbation on a ladder of x a few ulps either
side of +-x_max: both sides agree with the oracle's p' to the precision's
rounding, so p' is continuous across the switch."""

import numpy as np
import pytest

from inputs import workloads as W
from oracle import euler as E

from helpers import GpuContext, oracle_rhs, rel_l2_per_var

pytestmark = pytest.mark.gpu

FP64, FP32, DF64 = 0, 1, 2
PRECS = pytest.mark.parametrize("prec", [FP64, DF64, FP32], ids=["fp64", "df64", "fp32"])
RHS_BAR = {FP64: 1e-12, DF64: 1e-12, FP32: 1e-5}
P_BAR = {FP64: 2e-15, DF64: 5e-14, FP32: 2.5e-7}   # relative error of p' itself


def _x_of(wl):
    n_xy = (wl["N"] * wl["nel"][0] + 1) * (wl["N"] * wl["nel"][1] + 1)
    gz = np.arange(wl["q"].shape[1]) // n_xy
    return wl["q"][4] / wl["Theta0"][gz], gz


@PRECS
def test_rhs_across_the_eos_switch(cuda_device, prec):
    import torch
    wl = W.eos_span()
    x, _ = _x_of(wl)
    with GpuContext(wl, precision=prec) as g:
        tp = torch.from_numpy(wl["q"][4].copy()).to(g.dev)
        out = torch.empty_like(tp)
        xmax = g.xg.xg_pressure_perturbation(g.ctx, tp, out)
        got = g.rhs()
    assert 0.005 < xmax < 0.1
    assert np.count_nonzero(np.abs(x) < xmax) > 100
    assert np.count_nonzero(np.abs(x) > xmax) > 100
    err = rel_l2_per_var(got, oracle_rhs(wl))
    assert np.all(err <= RHS_BAR[prec]), err


@PRECS
def test_pressure_perturbation_continuous_at_the_switch(cuda_device, prec):
    import torch
    wl = W.box((2, 2, 2), 4, (0.0, 0.0, 0.0), (2000.0, 2000.0, 2000.0), (False, False, False))
    with GpuContext(wl, precision=prec) as g:
        n = g.np
        tp0 = torch.zeros(n, dtype=torch.float64, device=g.dev)
        out = torch.empty_like(tp0)
        xmax = g.xg.xg_pressure_perturbation(g.ctx, tp0, out)
        # ladders of x around +-x_max: float-ulp steps (the FP32 and double-
        # float forms test x rounded to float) and FP64-ulp steps
        k = np.arange(-8, 9, dtype=np.float64)
        lad = np.concatenate([xmax * (1.0 + k * 2.0 ** -23), xmax * (1.0 + k * 2.0 ** -50)])
        lad = np.concatenate([lad, -lad])
        _, gz = _x_of(wl)
        x = np.resize(lad, n)
        Th0 = wl["Theta0"][gz]
        theta_p = x * Th0
        g.xg.xg_pressure_perturbation(g.ctx, torch.from_numpy(theta_p).to(g.dev), out)
        got = out.cpu().numpy()
    ref = E.pressure_perturbation(Th0, theta_p, E.Physics(**wl["phys"]))
    rel = np.abs(got - ref) / np.abs(ref)
    xr = theta_p / Th0
    below, above = np.abs(xr) < xmax, np.abs(xr) > xmax
    assert below.any() and above.any()
    assert rel[below].max() <= P_BAR[prec], rel[below].max()
    assert rel[above].max() <= P_BAR[prec], rel[above].max()
