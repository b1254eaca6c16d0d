"""IMEX ARK2 with matrix-free GMRES (include/xg_imex.h) against the oracle
(oracle/imex.py): the linear operator, steps at the explicit step and at a
step the explicit scheme cannot take, the solver statistics, the bounded
solve and the unsupported precision.  L, GMRES and the combinations are
FP64 in every supported precision; in the mixed XG_DF64 context the
explicit part is the mixed stage in right-hand-side mode."""

import numpy as np
import pytest

from inputs import workloads as W
from oracle import euler as E, imex as X

from helpers import GpuContext, oracle_of, rel_l2_per_var

pytestmark = pytest.mark.gpu


def _case(per=(True, False, False), N=3, seed=31):
    return W.box((2, 2, 2), N, (0.0, 0.0, 0.0), (2000.0, 2000.0, 2000.0), per, f=1e-4, seed=seed)


def _oracle(wl):
    m, phys, base = oracle_of(wl)
    S = lambda s: E.rhs(m, s, base, wl["S_theta"], phys)
    L = lambda s: X.linear_operator(m, s, base, phys)
    return m, S, L


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
@pytest.mark.parametrize("per,N", [((True, False, False), 3), ((False, False, False), 4),
                                   ((True, True, True), 5)])
def test_linear_operator_matches_oracle(cuda_device, per, N, prec):
    import torch
    wl = _case(per, N)
    _, _, L = _oracle(wl)
    with GpuContext(wl, precision=prec) as g:
        v = torch.from_numpy(wl["q"]).to(cuda_device)
        out = torch.empty_like(v)
        g.xg.xg_linear_operator(g.ctx, v, out)
        got = out.cpu().numpy()
    assert np.all(rel_l2_per_var(got, L(wl["q"])) <= 1e-12)


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
@pytest.mark.parametrize("factor", [1.0, 20.0])
def test_steps_match_oracle(cuda_device, factor, prec):
    """Three steps at the explicit step and at 20 times it (beyond the
    explicit scheme's acoustic limit)."""
    wl = _case()
    _, S, L = _oracle(wl)
    dt = wl["dt"] * factor
    with GpuContext(wl, precision=prec) as g:
        st = g.xg.xg_step_imex(g.ctx, dt, 3, tol=1e-12)
        q = g.state()
    ref = wl["q"]
    for _ in range(3):
        ref = X.ark2_step(S, L, ref, dt)
    assert st.solves == 6 and st.iterations >= 6 and st.max_residual <= 1e-12
    err = rel_l2_per_var(q, ref)
    inc = rel_l2_per_var(q - wl["q"], ref - wl["q"])
    assert np.all(err <= 1e-10), err
    assert np.all(inc <= 1e-8), inc


def test_imex_takes_steps_the_explicit_scheme_cannot(cuda_device):
    wl = _case(seed=33)
    dt = wl["dt"] * 40.0
    with GpuContext(wl) as g:
        g.xg.xg_step_imex(g.ctx, dt, 20, tol=1e-10)
        q = g.state()
        assert np.all(np.isfinite(q)) and np.abs(q[1:3]).max() < 10.0
    with GpuContext(wl) as g:
        with pytest.raises(g.xg.XgError) as e:
            g.xg.xg_step(g.ctx, dt, 20)
        assert e.value.status == g.xg.XG_ERR_NONFINITE


def test_bounded_solve_reports_timeout_and_keeps_the_state(cuda_device):
    wl = _case()
    with GpuContext(wl) as g:
        before = g.state()
        with pytest.raises(g.xg.XgError) as e:
            g.xg.xg_step_imex(g.ctx, wl["dt"] * 20, 1, tol=1e-15, krylov=1, max_restarts=1)
        assert e.value.status == g.xg.XG_ERR_TIMEOUT
        assert np.array_equal(g.state(), before)
        g.xg.xg_step_imex(g.ctx, wl["dt"], 1)          # still usable


def test_imex_arguments_and_precisions(cuda_device):
    from paper_2504_08157_gb300 import xg
    wl = _case()
    with GpuContext(wl) as g:
        for kw in (dict(tol=0.0), dict(tol=1.0), dict(krylov=0), dict(krylov=65), dict(max_restarts=0)):
            with pytest.raises(xg.XgError) as e:
                xg.xg_step_imex(g.ctx, 0.1, 1, **kw)
            assert e.value.status == xg.XG_ERR_ARG
        with pytest.raises(xg.XgError) as e:
            xg.xg_step_imex(g.ctx, -0.1, 1)
        assert e.value.status == xg.XG_ERR_ARG
    with GpuContext(wl, precision=1) as g:
        with pytest.raises(xg.XgError) as e:
            xg.xg_step_imex(g.ctx, 0.1, 1)
        assert e.value.status == xg.XG_ERR_UNSUPPORTED
