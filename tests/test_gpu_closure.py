"""The learned closure's kernels (include/xg_closure.h) against the oracle:
features and restriction of fields, the training arithmetic (loss,
back-propagated gradient, Adam, column statistics) against float64, the
FP32 and bfloat16 tensor-core forward passes, and the closure inside the
right-hand side (the correction added before the wall condition)."""

import numpy as np
import pytest

from inputs import rng, workloads as W
from oracle import closure as OC, euler as E

from helpers import GpuContext, oracle_of, rel_l2

pytestmark = pytest.mark.gpu

FP32 = 1


def _t(a, dev, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype=dtype)


def _random_net(seed, n, scale=0.5):
    """Parameters, features, targets and normalisation of a seeded problem
    (inputs of the oracle and of the kernels alike)."""
    P = OC.param_count()
    u = rng.uniform(seed, P + n * 26 + 26, -1.0, 1.0)
    p = u[:P] * scale
    X = (u[P:P + 21 * n].reshape(21, n) * 3.0 + 0.5).astype(np.float32)
    T = u[P + 21 * n:P + 26 * n].reshape(5, n).astype(np.float32)
    mean = (0.1 * u[-26:-5]).astype(np.float32)
    scale_in = (0.5 + 0.25 * (u[-26:-5] + 1.0)).astype(np.float32)
    out_scale = (1.0 + np.arange(5) * 0.5).astype(np.float32)
    return p.astype(np.float32), X, T, mean, scale_in, out_scale


def test_features_match_oracle(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    for N, per in ((3, (True, False, False)), (4, (False, True, False)), (6, (True, True, True))):
        wl = W.box((3, 2, 2), N, (0.0, 0.0, 0.0), (3000.0, 2000.0, 2000.0), per, seed=70 + N)
        with GpuContext(wl, precision=FP32) as g:
            X = torch.empty((21, g.np), dtype=torch.float32, device=cuda_device)
            xg.xg_features(g.ctx, X)
            q32 = g.state()                       # the FP32 state the kernel saw
            got = X.cpu().numpy().astype(np.float64)
        m, _, _ = oracle_of(wl)
        S32 = wl["S_theta"].astype(np.float32).astype(np.float64)
        ref = OC.features(m, q32, S32)
        for f in range(21):
            assert rel_l2(got[f], ref[f]) <= 1e-5, (N, f, rel_l2(got[f], ref[f]))


@pytest.mark.parametrize("per", [(False, False, False), (True, True, False)])
def test_restriction_matches_oracle(cuda_device, per):
    import torch
    from paper_2504_08157_gb300 import xg
    N = 4
    fine = W.box((4, 6, 4), N, (0.0, 0.0, 0.0), (2000.0, 3000.0, 2000.0), per, seed=81)
    coarse = W.box((2, 3, 2), N, (0.0, 0.0, 0.0), (2000.0, 3000.0, 2000.0), per, seed=82)
    with GpuContext(fine) as gf, GpuContext(coarse) as gc:
        src = _t(fine["q"], cuda_device)
        dst = torch.empty((5, gc.np), dtype=torch.float64, device=cuda_device)
        xg.xg_restrict(gf.ctx, gc.ctx, src, dst)
        got = dst.cpu().numpy()
    axes = lambda wl: [(wl["nel"][d], N, wl["lo"][d], wl["hi"][d], wl["periodic"][d]) for d in range(3)]
    ref = OC.restrict(axes(fine), axes(coarse), fine["q"])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_loss_and_gradient_match_oracle(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    n = 1000
    p, X, T, mean, sin, sout = _random_net(3, n)
    d = cuda_device
    grad = torch.empty(OC.param_count(), dtype=torch.float32, device=d)
    loss = xg.xg_mlp_loss_grad(_t(p, d), _t(X, d), _t(T, d), _t(mean, d), _t(sin, d), _t(sout, d), grad)
    Xn = OC.normalise(X.T, mean, sin)
    Tn = T.T.astype(np.float64) / sout.astype(np.float64)
    ref_loss, ref_grad = OC.loss_and_grad(p.astype(np.float64), Xn, Tn)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) <= 1e-5 * np.linalg.norm(ref_grad)
    # a subset of the samples through the leading dimension
    loss2 = xg.xg_mlp_loss_grad(_t(p, d), _t(X, d), _t(T, d), _t(mean, d), _t(sin, d), _t(sout, d),
                                grad, n=333)
    ref2, rg2 = OC.loss_and_grad(p.astype(np.float64), Xn[:333], Tn[:333])
    assert abs(loss2 - ref2) <= 1e-5 * ref2
    assert np.linalg.norm(grad.cpu().numpy() - rg2) <= 1e-5 * np.linalg.norm(rg2)


def test_gradient_is_deterministic(cuda_device):
    import torch
    from paper_2504_08157_gb300 import xg
    p, X, T, mean, sin, sout = _random_net(4, 5000)
    d = cuda_device
    args = [_t(a, d) for a in (p, X, T, mean, sin, sout)]
    g1 = torch.empty(OC.param_count(), dtype=torch.float32, device=d)
    g2 = torch.empty_like(g1)
    l1 = xg.xg_mlp_loss_grad(*args, g1)
    l2 = xg.xg_mlp_loss_grad(*args, g2)
    assert l1 == l2 and torch.equal(g1, g2)


def test_adam_matches_oracle(cuda_device):
    from paper_2504_08157_gb300 import xg
    u = rng.uniform(9, 4 * 700, -1.0, 1.0).reshape(4, 700)
    p, m, v, g = (a.astype(np.float32) for a in (u[0], 0.1 * u[1], 0.01 * np.abs(u[2]), u[3]))
    d = cuda_device
    tp, tm, tv, tg = (_t(a, d) for a in (p, m, v, g))
    xg.xg_mlp_adam(tp, tm, tv, tg, 7, lr=3e-3)
    rp, rm, rv = OC.adam_step(p.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                              g.astype(np.float64), 7, lr=3e-3)
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-6, atol=1e-7)   # FP32 coefficients
    assert np.allclose(tv.cpu().numpy(), rv, rtol=2e-6, atol=1e-9)
    assert np.allclose(tp.cpu().numpy(), rp, rtol=1e-6, atol=1e-7)


def test_column_stats(cuda_device):
    from paper_2504_08157_gb300 import xg
    X = (rng.uniform(11, 3 * 10007, -2.0, 5.0).reshape(3, 10007)).astype(np.float32)
    mean, std = xg.xg_column_stats(_t(X, cuda_device), n=10000)
    x = X[:, :10000].astype(np.float64)
    assert np.allclose(mean, x.mean(axis=1), rtol=1e-12)
    assert np.allclose(std, x.std(axis=1), rtol=1e-10)


# 150,000 samples are 1,172 tiles of 128: more than one per persistent CTA
@pytest.mark.parametrize("n", [1, 127, 1000, 150_000])
def test_forward_fp32_and_bf16_match_oracle(cuda_device, n):
    import torch
    from paper_2504_08157_gb300 import xg
    p, X, T, mean, sin, sout = _random_net(5, n)
    d = cuda_device
    args = [_t(a, d) for a in (p, X)] + [_t(a, d) for a in (mean, sin, sout)]
    Y32 = torch.empty((5, n), dtype=torch.float32, device=d)
    Y16 = torch.empty((5, n), dtype=torch.float32, device=d)
    xg.xg_mlp_forward(*args, Y32, precision=xg.XG_MLP_FP32)
    xg.xg_mlp_forward(*args, Y16, precision=xg.XG_MLP_BF16)
    Xn = OC.normalise(X.T, mean, sin)
    ref = OC.forward(p.astype(np.float64), Xn) * sout.astype(np.float64)
    ref16 = OC.forward_bf16(p, Xn) * sout.astype(np.float64)
    got32, got16 = Y32.cpu().numpy().T, Y16.cpu().numpy().T
    assert np.linalg.norm(got32 - ref) <= 1e-5 * np.linalg.norm(ref)
    # bfloat16 inference: the oracle rounds at the same points; what remains
    # is FP32 accumulation order (and the rare rounding flip it causes)
    assert np.linalg.norm(got16 - ref16) <= 3e-3 * np.linalg.norm(ref16)
    assert np.linalg.norm(got16 - ref) <= 5e-2 * np.linalg.norm(ref)


def test_closure_in_the_rhs(cuda_device):
    """xg_rhs with the closure = plain RHS + bfloat16 correction of the
    state's features (wall-normal momentum still zero at walls); disabling
    it restores the plain RHS bit for bit."""
    import torch
    from paper_2504_08157_gb300 import xg
    wl = W.box((3, 2, 2), 4, (0.0, 0.0, 0.0), (3000.0, 2000.0, 2000.0), (True, False, False), seed=97)
    p, _, _, _, _, _ = _random_net(6, 1, scale=0.3)
    mean = np.zeros(21, np.float32)
    sin = np.ones(21, np.float32)
    sin[5:20] = 1e2            # gradients are O(1e-2) per metre
    sout = np.full(5, 1e-3, np.float32)
    d = cuda_device
    with GpuContext(wl, precision=FP32) as g:
        plain = g.rhs()
        xg.xg_closure_set(g.ctx, _t(p, d), _t(mean, d), _t(sin, d), _t(sout, d))
        withc = g.rhs()
        q32 = g.state()
        xg.xg_closure_set(g.ctx, None)
        again = g.rhs()
    assert np.array_equal(plain, again)
    m, _, _ = oracle_of(wl)
    S32 = wl["S_theta"].astype(np.float32).astype(np.float64)
    feats = OC.features(m, q32, S32)
    corr = (OC.forward_bf16(p, OC.normalise(feats.T, mean, sin)) * sout).T
    corr = E.apply_walls(m, corr)
    diff = withc - plain
    for v in range(5):
        assert rel_l2(diff[v], corr[v]) <= 2e-2, (v, rel_l2(diff[v], corr[v]))
    for d_ in range(3):
        assert np.all(diff[1 + d_][m.wall_nodes(d_)] == 0.0)


def test_prescribed_correction_in_the_rhs(cuda_device):
    """xg_correction_set: xg_rhs = plain RHS + C (C rounded to FP32, the
    wall-normal momentum still zero at walls), replacing an enabled network;
    removing it restores the plain RHS bit for bit; FP32 contexts only."""
    import torch
    from paper_2504_08157_gb300 import xg
    wl = W.box((3, 2, 2), 4, (0.0, 0.0, 0.0), (3000.0, 2000.0, 2000.0), (True, False, False), seed=97)
    d = cuda_device
    p, _, _, _, _, _ = _random_net(6, 1, scale=0.3)
    ones = np.ones(21, np.float32)
    with GpuContext(wl, precision=FP32) as g:
        plain = g.rhs()
        C = 0.5 * plain.std(axis=1, keepdims=True) * np.random.default_rng(3).normal(size=plain.shape)
        xg.xg_closure_set(g.ctx, _t(p, d), _t(np.zeros(21, np.float32), d), _t(ones, d),
                          _t(np.full(5, 1e-3, np.float32), d))
        xg.xg_correction_set(g.ctx, _t(C, d, torch.float64))
        withc = g.rhs()
        xg.xg_correction_set(g.ctx, None)
        again = g.rhs()
    assert np.array_equal(plain, again)
    m, _, _ = oracle_of(wl)
    want = E.apply_walls(m, C.astype(np.float32).astype(np.float64))
    diff = withc - plain
    for v in range(5):
        bar = 1e-5 * (1.0 + np.linalg.norm(plain[v]) / np.linalg.norm(want[v]))
        assert rel_l2(diff[v], want[v]) <= bar, (v, rel_l2(diff[v], want[v]))
    for d_ in range(3):
        assert np.all(diff[1 + d_][m.wall_nodes(d_)] == 0.0)
    with GpuContext(wl, precision=0) as g:
        with pytest.raises(xg.XgError) as e:
            xg.xg_correction_set(g.ctx, _t(C, d, torch.float64))
        assert e.value.status == xg.XG_ERR_UNSUPPORTED


def test_closure_target_is_the_scaled_difference(cuda_device):
    """xg_closure_target: out = s (a - b), elementwise in FP64 (bit for bit
    the same IEEE operations as numpy's), also in place."""
    import torch
    from paper_2504_08157_gb300 import xg
    r = np.random.default_rng(5)
    a, b = r.normal(size=(5, 1001)), r.normal(size=(5, 1001))
    ta, tb = _t(a, cuda_device, torch.float64), _t(b, cuda_device, torch.float64)
    out = xg.xg_closure_target(ta, tb, 0.25)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), 0.25 * (a - b))
    xg.xg_closure_target(ta, tb, 1.0 / 0.0125, out=ta)
    torch.cuda.synchronize()
    assert np.array_equal(ta.cpu().numpy(), (1.0 / 0.0125) * (a - b))


def test_closure_only_on_fp32(cuda_device):
    from paper_2504_08157_gb300 import xg
    wl = W.box((2, 2, 2), 4, (0.0, 0.0, 0.0), (2000.0, 2000.0, 2000.0), (True, True, False))
    import torch
    z = torch.zeros(OC.param_count(), dtype=torch.float32, device=cuda_device)
    o = torch.ones(21, dtype=torch.float32, device=cuda_device)
    with GpuContext(wl, precision=0) as g:
        with pytest.raises(xg.XgError) as e:
            xg.xg_closure_set(g.ctx, z, o, o, o[:5])
        assert e.value.status == xg.XG_ERR_UNSUPPORTED


def test_trained_closure_reduces_the_held_out_tendency_error(cuda_device):
    """A small end-to-end training: refined runs of 20 x 20 x 10 elements
    and their 10 x 10 x 5 coarse meshes (orders 4) generate the targets; the
    closure trained on three runs removes a clear part of the coarse
    tendency's error on a held-out run's snapshots, and a coarse run with it
    stays finite."""
    from paper_2504_08157_gb300 import closure as CL
    X, T = CL.sample_pairs(W.closure_case, seeds=[1, 2, 3, 4], coarse_nel=(10, 10, 5), snapshots=3,
                           steps_between=10, samples=4000, dev=cuda_device)
    assert X.shape == (21, 48000) and T.shape == (5, 48000)
    model = CL.train(X, T, cuda_device, epochs=25, batch=2048, lr=3e-3, holdout=0.25)
    print("held-out loss: zero correction %.4g, trained %.4g" % (model["holdout_zero"], model["holdout"]))
    assert model["holdout"] < 0.8 * model["holdout_zero"]
    ev = CL.evaluate(W.closure_case, 9, (10, 10, 5), model, 20, cuda_device)
    print("state error after 20 steps: plain", ev["plain"], "closure", ev["closure"])
    assert all(np.isfinite(ev["closure"]))
    # the plain right-hand side as fallback: the gain chosen on a validation run is one of
    # the candidates, its validation run is no worse than the plain one (gain 0 competes),
    # and gain 0 reproduces the plain coarse run bit for bit
    g, sel = CL.select_gain(W.closure_case, 10, (10, 10, 5), model, 20, cuda_device,
                            gains=(0.0, 0.1, 1.0))
    assert g in (0.0, 0.1, 1.0) and set(sel) == {0.0, 0.1, 1.0}
    score = lambda e: sum(a / b for a, b in zip(e, sel[0.0])) / 5
    assert score(sel[g]) <= 1.0
    again = CL.evaluate_gains(W.closure_case, 9, (10, 10, 5), model, 20, cuda_device, (0.0,))
    assert again[0.0] == ev["plain"]


def test_tensor_core_wait_times_out_cleanly(cuda_device):
    """A tensor-core wait that nothing completes gives up after its limit,
    frees its tensor memory and reports XG_ERR_TIMEOUT; the device then runs
    the tensor-core inference as before."""
    import torch
    from paper_2504_08157_gb300 import xg
    assert xg.xg_tc_wait_selftest(2_000_000) == xg.XG_ERR_TIMEOUT
    p, X, T, mean, sin, sout = _random_net(3, 300)
    d = cuda_device
    Y = torch.empty((5, 300), dtype=torch.float32, device=d)
    xg.xg_mlp_forward(_t(p, d), _t(X, d), _t(mean, d), _t(sin, d), _t(sout, d), Y, precision=xg.XG_MLP_BF16)
    ref16 = OC.forward_bf16(p, OC.normalise(X.T, mean, sin)) * sout.astype(np.float64)
    got = Y.cpu().numpy().T
    assert np.linalg.norm(got - ref16) <= 3e-3 * np.linalg.norm(ref16)
    with pytest.raises(xg.XgError):
        xg.xg_tc_wait_selftest(0)
