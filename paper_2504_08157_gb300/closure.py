"""Training and evaluation of the learned closure through the C ABI
(include/xg_closure.h).

Orchestration only: the right-hand sides, time steps, restriction, features,
statistics, loss gradients and Adam updates all run in ``libxg.so``; torch
holds the device arrays and gathers the sampled training columns.

A training pair is a refined run and the coarse mesh of the same box (the
refined mesh has twice the elements per direction, same order).  At each
snapshot of the refined run:

    target  = R L_fine(q_fine) - L_coarse(R q_fine)
    features = xg_features of the coarse context holding R q_fine

where R is the restriction (xg_restrict: the fine elements' interpolants at
the coarse nodes).  The closure learns the target from the features; a
coarse run with the closure then adds its prediction to L_coarse.
"""

import numpy as np

from . import xg

P = xg.XG_CLOSURE_PARAMS


def _torch():
    import torch
    return torch


def make_ctx(wl, dev, precision=xg.XG_FP32):
    torch = _torch()
    ph = wl["phys"]
    ctx = xg.xg_mesh_create(xg.mesh_desc(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"],
                                         f=ph["f"], g=ph["g"], R=ph["R"], cp=ph["cp"], cv=ph["cv"],
                                         p_a=ph["p_a"], precision=precision))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    xg.xg_set_state(ctx, t(wl["q"]), t(wl["rho0"]), t(wl["Theta0"]))
    if wl["S_theta"] is not None:
        xg.xg_set_forcing(ctx, t(wl["S_theta"]))
    return ctx


def _state(ctx, dev):
    torch = _torch()
    q = torch.empty((5, xg.xg_mesh_np(ctx)), dtype=torch.float64, device=dev)
    xg.xg_get_state(ctx, q)
    return q


def _rhs(ctx, dev):
    torch = _torch()
    r = torch.empty((5, xg.xg_mesh_np(ctx)), dtype=torch.float64, device=dev)
    xg.xg_rhs(ctx, r)
    return r


def sample_pairs(case, seeds, coarse_nel, snapshots, steps_between, samples, dev, sample_seed=7,
                 target="rhs"):
    """Training set from refined runs: for each seed, a refined run of
    2 x coarse_nel elements advanced ``steps_between`` refined steps between
    ``snapshots`` snapshots (the first at t = 0); at each snapshot
    ``samples`` coarse nodes drawn by the seeded generator.  The target is
    the refined-minus-coarse tendency difference at the snapshot,
    ``target="rhs"``: R L_f(q_f) - L_c(R q_f); or averaged over one coarse
    step, ``target="step"``: (R q_f(t + dt) - S_c(R q_f(t))) / dt with S_c
    one coarse SSP-RK3 step (what a correction added in every stage of that
    step must supply).  Returns float32 CUDA tensors X [21][n], T [5][n]."""
    torch = _torch()
    from inputs import rng
    fine_nel = tuple(2 * n for n in coarse_nel)
    Xs, Ts = [], []
    draw = 0
    for seed in seeds:
        fwl = case(seed, nel=fine_nel)
        cwl = case(seed, nel=coarse_nel)
        fctx = make_ctx(fwl, dev)
        cctx = make_ctx(cwl, dev)
        try:
            npc = xg.xg_mesh_np(cctx)
            X = torch.empty((21, npc), dtype=torch.float32, device=dev)
            qc = torch.empty((5, npc), dtype=torch.float64, device=dev)
            rc_f = torch.empty((5, npc), dtype=torch.float64, device=dev)
            for k in range(snapshots):
                if k:
                    xg.xg_step(fctx, fwl["dt"], steps_between)
                xg.xg_restrict(fctx, cctx, _state(fctx, dev), qc)
                xg.xg_set_state(cctx, qc)
                xg.xg_features(cctx, X)
                if target == "rhs":
                    xg.xg_restrict(fctx, cctx, _rhs(fctx, dev), rc_f)
                    T = xg.xg_closure_target(rc_f, _rhs(cctx, dev))
                else:
                    q_save = _state(fctx, dev)
                    xg.xg_step(fctx, fwl["dt"], 2)          # two refined steps = one coarse step
                    xg.xg_restrict(fctx, cctx, _state(fctx, dev), rc_f)
                    xg.xg_set_state(fctx, q_save)          # the refined run continues unchanged
                    xg.xg_step(cctx, cwl["dt"], 1)
                    T = xg.xg_closure_target(rc_f, _state(cctx, dev), 1.0 / cwl["dt"])
                u = rng.uniform(sample_seed, samples, offset=draw)
                draw += samples
                idx = torch.from_numpy(np.minimum((u * npc).astype(np.int64), npc - 1)).to(dev)
                Xs.append(X[:, idx])
                Ts.append(T[:, idx].to(torch.float32))
        finally:
            xg.xg_destroy(fctx)
            xg.xg_destroy(cctx)
    return torch.cat(Xs, dim=1).contiguous(), torch.cat(Ts, dim=1).contiguous()


def init_params(seed, dev):
    """Seeded uniform initialisation, +-1/sqrt(fan_in) per layer."""
    torch = _torch()
    from inputs import rng
    u = rng.uniform(seed, P, -1.0, 1.0)
    p = np.empty(P)
    k = 0
    for fin, fout in ((21, 64), (64, 64), (64, 5)):
        nw = fin * fout
        p[k:k + nw] = u[k:k + nw] / np.sqrt(fin)
        k += nw
        p[k:k + fout] = 0.0
        k += fout
    return torch.from_numpy(p.astype(np.float32)).to(dev)


def normalisation(X, T, dev):
    """(in_mean, in_scale, out_scale) float32 CUDA tensors from the column
    statistics of the training set (xg_column_stats)."""
    torch = _torch()
    mx, sx = xg.xg_column_stats(X)
    _, st = xg.xg_column_stats(T)
    in_scale = np.where(sx > 0, 1.0 / np.maximum(sx, 1e-30), 1.0)
    out_scale = np.where(st > 0, st, 1.0)
    f = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).to(dev)
    return f(mx), f(in_scale), f(out_scale)


def train(X, T, dev, epochs=20, batch=4096, lr=2e-3, seed=11, holdout=0.1):
    """Adam (cosine-decayed step) on minibatches of the samples in a seeded
    random order; the last ``holdout`` fraction of the set (the last run's
    snapshots) is held out.  Returns a dict with the parameters,
    the normalisation and the loss history (the loss is the normalised MSE;
    the network predicting zero scores the normalised target variance)."""
    torch = _torch()
    from inputs import rng
    n = X.shape[1]
    ntr = int(n * (1.0 - holdout))
    perm = torch.from_numpy(np.argsort(rng.uniform(seed + 1, ntr))).to(dev)
    Xtr, Ttr = X[:, :ntr][:, perm].contiguous(), T[:, :ntr][:, perm].contiguous()
    Xho, Tho = X[:, ntr:].contiguous(), T[:, ntr:].contiguous()
    mean, scale, oscale = normalisation(Xtr, Ttr, dev)
    p = init_params(seed, dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.empty_like(p)
    zero = torch.zeros_like(p)
    hist = []
    t = 0
    base_ho = xg.xg_mlp_loss_grad(zero, Xho, Tho, mean, scale, oscale, g)
    for ep in range(epochs):
        tot = 0.0
        for b0 in range(0, ntr - batch + 1, batch):
            Xb = Xtr[:, b0:b0 + batch]
            Tb = Ttr[:, b0:b0 + batch]
            # minibatch columns as their own contiguous arrays
            Xb = Xb.contiguous()
            Tb = Tb.contiguous()
            tot += xg.xg_mlp_loss_grad(p, Xb, Tb, mean, scale, oscale, g)
            t += 1
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(epochs, 1)))
            xg.xg_mlp_adam(p, m, v, g, t, lr=lr_t)
        ho = xg.xg_mlp_loss_grad(p, Xho, Tho, mean, scale, oscale, g)
        hist.append((ep, tot / max(1, (ntr // batch)), ho))
    return dict(params=p, in_mean=mean, in_scale=scale, out_scale=oscale, history=hist,
                holdout_zero=base_ho, holdout=hist[-1][2] if hist else base_ho)


def centered(model, X, dev):
    """The model with the mean of its correction over the samples X removed
    (the output bias b3 shifted by the mean inference output, per variable):
    a network whose correction drifts the coarse run in one direction loses
    that drift."""
    torch = _torch()
    n = X.shape[1]
    Y = torch.empty((5, n), dtype=torch.float32, device=dev)
    xg.xg_mlp_forward(model["params"], X, model["in_mean"], model["in_scale"], model["out_scale"], Y,
                      precision=xg.XG_MLP_BF16)
    mean = Y.double().mean(dim=1)
    p = model["params"].clone()
    p[P - 5:] -= (mean / model["out_scale"].double()).float()
    return dict(model, params=p)


def evaluate_gains(case, seed, coarse_nel, model, coarse_steps, dev, gains):
    """The refined run once, then one coarse run per gain g: the closure's
    output scaled by g (g = 0 is the plain coarse run), all from the
    restriction of the refined initial field, over ``coarse_steps`` coarse
    steps (twice as many refined steps).  Returns, per gain, the relative L2
    distance of the coarse state from the restricted refined state, per
    variable, relative to the refined run's change over that time."""
    torch = _torch()
    fine_nel = tuple(2 * n for n in coarse_nel)
    fwl = case(seed, nel=fine_nel)
    cwl = case(seed, nel=coarse_nel)
    fctx = make_ctx(fwl, dev)
    ctxs = []
    try:
        probe = make_ctx(cwl, dev)
        ctxs.append(probe)
        npc = xg.xg_mesh_np(probe)
        q0 = torch.empty((5, npc), dtype=torch.float64, device=dev)
        xg.xg_restrict(fctx, probe, _state(fctx, dev), q0)
        xg.xg_step(fctx, fwl["dt"], 2 * coarse_steps)   # the refined step is half the coarse one
        ref = torch.empty((5, npc), dtype=torch.float64, device=dev)
        xg.xg_restrict(fctx, probe, _state(fctx, dev), ref)
        ref0 = ref - q0
        out = {}
        for g in gains:
            c = make_ctx(cwl, dev)
            ctxs.append(c)
            xg.xg_set_state(c, q0)
            if g != 0.0:
                xg.xg_closure_set(c, model["params"], model["in_mean"], model["in_scale"],
                                  model["out_scale"] * float(g))
            try:
                xg.xg_step(c, cwl["dt"], coarse_steps)
                a = _state(c, dev)
                out[g] = [float(torch.linalg.norm(a[v] - ref[v]) /
                                torch.linalg.norm(ref0[v]).clamp_min(1e-300)) for v in range(5)]
            except xg.XgError as e:          # a closure run that blew up
                if e.status != xg.XG_ERR_NONFINITE:
                    raise
                out[g] = [float("inf")] * 5
        return out
    finally:
        for c in [fctx] + ctxs:
            xg.xg_destroy(c)


def evaluate(case, seed, coarse_nel, model, coarse_steps, dev):
    """Refined run vs the plain coarse run vs the coarse run with the
    closure (gain 1); per-variable errors as in evaluate_gains."""
    e = evaluate_gains(case, seed, coarse_nel, model, coarse_steps, dev, (0.0, 1.0))
    return dict(plain=e[0.0], closure=e[1.0],
                what="relative L2 distance of each coarse run's state from the restricted "
                     "refined state after %d coarse steps, per variable, relative to the "
                     "refined run's change over that time" % coarse_steps)


def select_gain(case, seed, coarse_nel, model, coarse_steps, dev,
                gains=(0.0, 0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0)):
    """The plain right-hand side as fallback: the gain, among ``gains``
    (0 = no correction), whose coarse run on a validation run (``seed``, used
    neither for training nor for the final judgement) ends closest to the
    refined run, scored by the mean over the five variables of the error
    relative to the plain run's.  Returns (gain, {gain: errors})."""
    e = evaluate_gains(case, seed, coarse_nel, model, coarse_steps, dev, gains)
    plain = e[0.0]
    score = {g: sum(v / max(p, 1e-300) for v, p in zip(errs, plain)) / 5 for g, errs in e.items()}
    return min(gains, key=lambda g: (score[g], g)), e


def correction_study(case, seed, coarse_nel, coarse_steps, dev, filter_order=2):
    """What the training target is worth in a coarse run, measured with the
    exact target instead of a network: three coarse runs from the
    restriction of the refined initial field over ``coarse_steps`` coarse
    steps, judged as in evaluate_gains --
      plain:     no correction;
      exact:     in every coarse step the exact target of sample_pairs,
                 R L_f(q_f) - L_c(R q_f) at the refined run's state at the
                 start of the step (xg_correction_set);
      filtered:  the same correction passed through a low-pass filter (its
                 interpolant on the same elements at order ``filter_order``,
                 two xg_restrict calls), which keeps most of its norm;
      bf16:      the exact correction rounded to bfloat16, the precision of
                 the network's inference (a data conversion, for the study).
    Returns the per-variable errors of the runs and the filtered
    correction's share of the exact one's norm at t = 0."""
    torch = _torch()
    fine_nel = tuple(2 * n for n in coarse_nel)
    fwl = case(seed, nel=fine_nel)
    cwl = case(seed, nel=coarse_nel)
    mwl = case(seed, nel=coarse_nel, N=filter_order)
    ctxs = []
    try:
        for w in (fwl, cwl, cwl, cwl, cwl, mwl, cwl):
            ctxs.append(make_ctx(w, dev))
        fctx, probe, plain, exact, filt, low, rb16 = ctxs
        npc, npm = xg.xg_mesh_np(probe), xg.xg_mesh_np(low)
        Z = lambda n: torch.empty((5, n), dtype=torch.float64, device=dev)
        Rq, RL, Tm, Tf = Z(npc), Z(npc), Z(npm), Z(npc)
        xg.xg_restrict(fctx, probe, _state(fctx, dev), Rq)
        q0 = Rq.clone()
        for c in (plain, exact, filt, rb16):
            xg.xg_set_state(c, q0)
        xg.xg_step(plain, cwl["dt"], coarse_steps)
        share = None
        for k in range(coarse_steps):
            if k:
                xg.xg_restrict(fctx, probe, _state(fctx, dev), Rq)
            xg.xg_restrict(fctx, probe, _rhs(fctx, dev), RL)
            xg.xg_set_state(probe, Rq)
            T = xg.xg_closure_target(RL, _rhs(probe, dev))
            xg.xg_restrict(probe, low, T, Tm)
            xg.xg_restrict(low, probe, Tm, Tf)
            if share is None:
                share = [float(torch.linalg.norm(Tf[v]) / torch.linalg.norm(T[v]).clamp_min(1e-300))
                         for v in range(5)]
            xg.xg_correction_set(exact, T)
            xg.xg_correction_set(filt, Tf)
            xg.xg_correction_set(rb16, T.to(torch.bfloat16).to(torch.float64).contiguous())
            xg.xg_step(exact, cwl["dt"], 1)
            xg.xg_step(filt, cwl["dt"], 1)
            xg.xg_step(rb16, cwl["dt"], 1)
            xg.xg_step(fctx, fwl["dt"], 2)                 # the refined step is half the coarse one
        xg.xg_restrict(fctx, probe, _state(fctx, dev), Rq)
        ref0 = Rq - q0
        err = lambda c: [float(torch.linalg.norm(_state(c, dev)[v] - Rq[v]) /
                               torch.linalg.norm(ref0[v]).clamp_min(1e-300)) for v in range(5)]
        return dict(plain=err(plain), exact=err(exact), filtered=err(filt), exact_in_bfloat16=err(rb16),
                    filtered_norm_share=share,
                    filter="interpolant of order %d on the same elements" % filter_order,
                    what="relative L2 distance from the restricted refined state after %d coarse "
                         "steps, per variable, relative to the refined run's change, of coarse runs "
                         "with no correction, the exact training target as correction, that "
                         "target low-pass filtered, and that target rounded to bfloat16" % coarse_steps)
    finally:
        for c in ctxs:
            xg.xg_destroy(c)

