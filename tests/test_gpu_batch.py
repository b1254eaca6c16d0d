"""The batched persistent form (include/xg_batch.h): many XG_FP32 instances
of different sizes and orders advanced by one persistent launch.

Each instance is checked against the FP64 oracle at the precision form's
bar (relative L2 per variable <= 1e-5 per RHS), and against a single XG_FP32
context of the same description bit for bit: batching changes the
scheduling, never the arithmetic.  Every schedule and tile choice gives the
same bits; the autotuner leaves the states untouched; the bounded grid
barrier reports a starved wait as XG_ERR_TIMEOUT and the batch stays
usable."""

import numpy as np
import pytest

from inputs import workloads as W

from helpers import BatchRun, GpuContext, oracle_rhs, oracle_steps, rel_l2_per_var

pytestmark = pytest.mark.gpu

FP32 = 1
RHS_TOL32 = 1e-5


def small_batch():
    """Five instances: orders 3-6, mixed boundaries, a scaled cyclone box."""
    wls = [
        W.box((3, 4, 2), 3, (0.0, 0.0, 0.0), (3000.0, 4000.0, 2000.0), (True, True, False), seed=61),
        W.box((2, 3, 3), 4, (0.0, 0.0, 0.0), (2000.0, 3000.0, 3000.0), (True, False, False), seed=62),
        W.box((2, 2, 2), 5, (0.0, 0.0, 0.0), (2000.0, 2000.0, 2000.0), (False, True, False), seed=63),
        W.box((1, 2, 3), 6, (0.0, 0.0, 0.0), (1000.0, 2000.0, 3000.0), (True, True, True), seed=64),
        W.batch_instance(dict(W.batch_specs(1, seed=7)[0], nel=(5, 4, 4), N=4), state="random"),
    ]
    return wls


@pytest.fixture(scope="module")
def wls():
    return small_batch()


def test_batch_rhs_matches_oracle(cuda_device, wls):
    with BatchRun(wls) as b:
        got = b.rhs()
    for g, wl in zip(got, wls):
        err = rel_l2_per_var(g, oracle_rhs(wl))
        assert np.all(err <= RHS_TOL32), (wl["N"], wl["nel"], err)


def test_batch_is_bitwise_the_single_context(cuda_device, wls):
    with BatchRun(wls) as b:
        r = b.rhs()
        b.step(3)
        q = b.states()
    for i, wl in enumerate(wls):
        with GpuContext(wl, precision=FP32) as g:
            r1 = g.rhs()
            g.step(3)
            q1 = g.state()
        assert np.array_equal(r[i], r1), (i, np.abs(r[i] - r1).max())
        assert np.array_equal(q[i], q1), (i, np.abs(q[i] - q1).max())


@pytest.mark.parametrize("sched", [0, 1, 2], ids=["round_robin", "lpt", "dynamic"])
@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("cps", [1, 2])
def test_every_schedule_gives_the_same_bits(cuda_device, wls, sched, half, cps):
    with BatchRun(wls) as b:
        b.xg.xg_batch_set_tuning(b.b, sched, half, cps)
        b.step(2)
        q = b.states()
    with BatchRun(wls) as ref:
        ref.xg.xg_batch_set_tuning(ref.b, 1, 0, 2)
        ref.step(2)
        q0 = ref.states()
    for a, c in zip(q, q0):
        assert np.array_equal(a, c)


def test_batch_steps_match_oracle(cuda_device, wls):
    n = 10
    with BatchRun(wls) as b:
        b.step(n)
        q = b.states()
    for g, wl in zip(q, wls):
        ref = oracle_steps(wl, n)
        assert np.all(rel_l2_per_var(g, ref) <= 1e-5), (wl["N"], rel_l2_per_var(g, ref))


def test_odd_and_even_step_counts_chain(cuda_device, wls):
    """1 + 2 steps equal 3 steps (q^n and q^{n+1} trade places every step)."""
    with BatchRun(wls) as b:
        b.step(1)
        b.step(2)
        q = b.states()
    with BatchRun(wls) as b:
        b.step(3)
        q3 = b.states()
    for a, c in zip(q, q3):
        assert np.array_equal(a, c)


def test_autotune_keeps_the_states(cuda_device, wls):
    with BatchRun(wls) as b:
        before = b.states()
        t = b.xg.xg_batch_autotune(b.b, b.dts, trial_steps=1)
        after = b.states()
        assert t.schedule in (0, 1, 2) and t.plane_tile in (0, 1) and t.ctas_per_sm in (1, 2)
        assert t.ms_per_step > 0.0
        got = b.xg.xg_batch_get_tuning(b.b)
        assert (got.schedule, got.plane_tile, got.ctas_per_sm) == (t.schedule, t.plane_tile,
                                                                 t.ctas_per_sm)
        b.step(2)
        q = b.states()
    for a, c in zip(before, after):
        assert np.array_equal(a, c)
    with BatchRun(wls) as ref:
        ref.step(2)
        q0 = ref.states()
    for a, c in zip(q, q0):
        assert np.array_equal(a, c)


def test_starved_barrier_times_out_and_batch_stays_usable(cuda_device, wls):
    with BatchRun(wls) as b:
        s = b.xg.xg_batch_barrier_selftest(b.b, spin_limit=2000)
        assert s == b.xg.XG_ERR_TIMEOUT
        b.step(1)
        q = b.states()
    with BatchRun(wls) as ref:
        ref.step(1)
        q0 = ref.states()
    for a, c in zip(q, q0):
        assert np.array_equal(a, c)


def test_nonfinite_state_is_reported(cuda_device, wls):
    import torch
    with BatchRun(wls) as b:
        q = wls[2]["q"].copy()
        q[4, 7] = np.nan
        b.xg.xg_set_state(b.ctx[2], torch.from_numpy(q).to(cuda_device))
        with pytest.raises(b.xg.XgError) as e:
            b.step(1)
        assert e.value.status == b.xg.XG_ERR_NONFINITE


def test_step_needs_every_state(cuda_device):
    from paper_2504_08157_gb300 import xg
    wl = W.box((2, 2, 2), 4, (0.0, 0.0, 0.0), (2000.0, 2000.0, 2000.0), (True, True, False))
    d = xg.mesh_desc(wl["nel"], 4, wl["lo"], wl["hi"], wl["periodic"], precision=xg.XG_FP32)
    b = xg.xg_batch_create([d, d])
    try:
        with pytest.raises(xg.XgError) as e:
            xg.xg_batch_step(b, [0.1, 0.1], 1)
        assert e.value.status == xg.XG_ERR_ARG
    finally:
        xg.xg_batch_destroy(b)


@pytest.mark.slow
def test_full_batch_rhs_is_the_single_contexts(cuda_device):
    """The 96-instance batch: every instance's right-hand side equals its
    single XG_FP32 context's bit for bit, and the two smallest instances are
    within the precision form's bar of the oracle."""
    specs = W.batch_specs()
    wls = [W.batch_instance(s, state="random", seed=i + 1) for i, s in enumerate(specs)]
    with BatchRun(wls) as b:
        b.xg.xg_batch_autotune(b.b, b.dts, trial_steps=1)
        got = b.rhs()
    for i, wl in enumerate(wls):
        with GpuContext(wl, precision=FP32) as g:
            assert np.array_equal(got[i], g.rhs()), i
    sizes = np.argsort([g.shape[1] for g in got])
    for i in sizes[:2]:
        err = rel_l2_per_var(got[i], oracle_rhs(wls[i]))
        assert np.all(err <= RHS_TOL32), (i, err)
