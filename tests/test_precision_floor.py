"""What storing the state in FP32 costs by itself, computed by the oracle
alone (no GPU): the oracle's right-hand side of the cyclone box's pure-vortex
state against its right-hand side of the same state rounded to FP32.

At this state the rho' and Theta' tendencies are residuals of cancelling x
and y flux derivatives (the vortex is horizontally non-divergent), so the
per-node rounding of the momentum to 24 significand bits, differentiated and
no longer cancelling, moves them by more than 1e-5 relative L2: no
computation that holds the state in FP32 can be within 1e-5 of the FP64
oracle there.  The horizontal momentum tendencies, which do not cancel, move
by less than 1e-6, and at a perturbed state every variable moves by less
than 5e-6.  Rounding to the
double-float format (48 significand bits) instead moves every tendency by
less than 5e-13."""

import numpy as np

from inputs import workloads as W

from helpers import oracle_rhs, rel_l2_per_var


def _df_round(q):
    h = q.astype(np.float32).astype(np.float64)
    return h + (q - h).astype(np.float32).astype(np.float64)


def test_fp32_state_rounding_floor_at_the_vortex():
    wl = W.tc(nel=(16, 16, 16))
    ref = oracle_rhs(wl)
    e32 = rel_l2_per_var(oracle_rhs(wl, q=wl["q"].astype(np.float32).astype(np.float64)), ref)
    assert np.all(e32[[0, 4]] > 1e-5), e32
    assert np.all(e32[1:3] < 1e-6), e32
    edf = rel_l2_per_var(oracle_rhs(wl, q=_df_round(wl["q"])), ref)
    assert np.all(edf < 5e-13), edf


def test_fp32_state_rounding_at_a_perturbed_state():
    wl = W.tc(nel=(16, 16, 16), state="random")
    ref = oracle_rhs(wl)
    e32 = rel_l2_per_var(oracle_rhs(wl, q=wl["q"].astype(np.float32).astype(np.float64)), ref)
    assert np.all(e32 < 5e-6), e32


def test_state_rounding_floors_at_full_size():
    """The full cyclone box (17 M nodes) at ~600 sampled nodes, against the
    oracle in extended precision: there the rho' and Theta' residuals are
    smaller relative to their cancelling parts than on the 16^3 sample, and
    rounding the state to the double-float format (48 significand bits)
    already moves them by more than 1e-12; rounding to FP32 by more than
    1e-4 (rho').  The momentum tendencies move by less than 1e-12 and 1e-5."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    import test_gpu_parity as P
    from helpers import oracle_rhs_at_nodes_extended
    wl = W.tc()
    nodes = P._sample_nodes((512, 512, 65), np.random.default_rng(2504), 600)
    refx = oracle_rhs_at_nodes_extended(wl, nodes)
    edf = rel_l2_per_var(oracle_rhs_at_nodes_extended(wl, nodes, q=_df_round(wl["q"])), refx)
    assert np.all(edf[[0, 4]] > 1e-12), edf
    assert np.all(edf[1:3] < 1e-12), edf
    e32 = rel_l2_per_var(oracle_rhs_at_nodes_extended(
        wl, nodes, q=wl["q"].astype(np.float32).astype(np.float64)), refx)
    assert e32[0] > 1e-4 and np.all(e32[1:3] < 1e-5), e32
