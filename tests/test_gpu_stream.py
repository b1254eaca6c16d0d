"""xg_step_stream: independent host states streamed through one context,
the uploads and downloads overlapping the steps on the context's copy
streams.  Its outputs equal xg_set_state + xg_step + xg_get_state of each
input bit for bit (the same kernels in the same order), in every precision;
a repeated output pointer keeps the latest output, the context holds the
last output's state, and count 0 is a no-op."""

import numpy as np
import pytest

from inputs import workloads as W

from helpers import GpuContext

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "fp32", "df64"])
def test_step_stream_equals_sequential_calls(cuda_device, prec):
    import torch
    wl = W.tc(nel=(6, 5, 4), state="random")
    rng = np.random.default_rng(17)
    ins = [np.ascontiguousarray(wl["q"] * (1.0 + 0.05 * k) + 1e-4 * rng.normal(size=wl["q"].shape)
                                * np.abs(wl["q"]).max(axis=1, keepdims=True)) for k in range(3)]
    with GpuContext(wl, precision=prec) as g:
        xg = g.xg
        refs = []
        for q in ins:
            xg.xg_set_state(g.ctx, q)
            xg.xg_step(g.ctx, wl["dt"], 2)
            out = np.empty_like(q)
            xg.xg_get_state(g.ctx, out)
            refs.append(out)
        pin_in = [torch.from_numpy(q).pin_memory() for q in ins]
        outs = [torch.empty(q.shape, dtype=torch.float64).pin_memory() for q in ins]
        xg.xg_step_stream(g.ctx, pin_in, outs, wl["dt"], 2)
        for o, r in zip(outs, refs):
            assert np.array_equal(o.numpy(), r)
        assert np.array_equal(g.state(), refs[-1])
        same = torch.empty(ins[0].shape, dtype=torch.float64).pin_memory()
        xg.xg_step_stream(g.ctx, ins, [same, same, same], wl["dt"], 2)   # pageable inputs too
        assert np.array_equal(same.numpy(), refs[-1])
        xg.xg_step_stream(g.ctx, [], [], wl["dt"], 2)
        assert np.array_equal(g.state(), refs[-1])


def test_step_stream_checks(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    wl = W.tc(nel=(4, 4, 2))
    with GpuContext(wl) as g:
        dev_q = torch.zeros(wl["q"].shape, dtype=torch.float64, device=cuda_device)
        with pytest.raises(ValueError):
            xg.xg_step_stream(g.ctx, [dev_q], [wl["q"].copy()], wl["dt"])
        with pytest.raises(ValueError):
            xg.xg_step_stream(g.ctx, [wl["q"][:, :10].copy()], [wl["q"].copy()], wl["dt"])
        with pytest.raises(xg.XgError) as e:
            xg.xg_step_stream(g.ctx, [wl["q"]], [wl["q"].copy()], float("nan"))
        assert e.value.status == xg.XG_ERR_ARG
        a, b = wl["q"].copy(), wl["q"].copy()
        with pytest.raises(xg.XgError) as e:                 # an output that is a later input
            xg.xg_step_stream(g.ctx, [a, b], [b, b], wl["dt"])
        assert e.value.status == xg.XG_ERR_ARG


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
def test_step_stream_array_rotation(cuda_device, prec):
    """FP64-state contexts step the inputs where they were uploaded and move
    the state between six arrays: odd and even step counts, more inputs
    than arrays, and plain calls afterwards all give the sequential results."""
    import torch
    wl = W.tc(nel=(5, 4, 3), state="random")
    ins = [np.ascontiguousarray(wl["q"] * (1.0 + 0.03 * k)) for k in range(7)]
    with GpuContext(wl, precision=prec) as g:
        xg = g.xg

        def sequential(nsteps):
            refs = []
            for q in ins:
                xg.xg_set_state(g.ctx, q)
                xg.xg_step(g.ctx, wl["dt"], nsteps)
                out = np.empty_like(q)
                xg.xg_get_state(g.ctx, out)
                refs.append(out)
            return refs

        ref1, ref2 = sequential(1), sequential(2)
        pin_in = [torch.from_numpy(q).pin_memory() for q in ins]
        for nsteps, refs in ((1, ref1), (2, ref2), (1, ref1), (0, ins)):
            outs = [torch.empty(q.shape, dtype=torch.float64).pin_memory() for q in ins]
            xg.xg_step_stream(g.ctx, pin_in, outs, wl["dt"], nsteps)
            for o, r in zip(outs, refs):
                assert np.array_equal(o.numpy(), r)
            assert np.array_equal(g.state(), refs[-1])
        xg.xg_step(g.ctx, wl["dt"], 1)                 # the context goes on from the last output
        xg.xg_set_state(g.ctx, ins[2])
        xg.xg_step(g.ctx, wl["dt"], 2)
        assert np.array_equal(g.state(), ref2[2])
