"""ctypes binding of the C ABI in ``include/xg.h``, ``include/xg_batch.h``,
``include/xg_closure.h``, ``include/xg_dynamics.h`` and ``include/xg_imex.h``
(same function names).

Argument marshalling only: every step of the path runs in ``libxg.so``.
Arrays may be torch tensors (CUDA tensors are passed as device pointers,
CPU tensors as host pointers), numpy arrays (host) or raw integer
addresses together with an explicit ``where``.  The stream defaults to
torch's current stream for CUDA tensors and to the legacy stream otherwise.
A non-OK status raises ``XgError`` carrying the status code.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxg.so")

XG_OK, XG_ERR_ARG, XG_ERR_CUDA, XG_ERR_OOM, XG_ERR_NONFINITE, XG_ERR_TIMEOUT, \
    XG_ERR_UNSUPPORTED = range(7)
XG_HOST, XG_DEVICE = 0, 1
XG_FP64, XG_FP32, XG_DF64 = 0, 1, 2
XG_SCHED_ROUND_ROBIN, XG_SCHED_LPT, XG_SCHED_DYNAMIC = 0, 1, 2
XG_MLP_FP32, XG_MLP_BF16 = 0, 1
XG_CONTRACT_FMA, XG_CONTRACT_TF32X3, XG_CONTRACT_F16X3 = 0, 1, 2
XG_CLOSURE_IN, XG_CLOSURE_HIDDEN, XG_CLOSURE_OUT, XG_CLOSURE_PARAMS = 21, 64, 5, 5893

__all__ = ["XgError", "xg_mesh_desc", "mesh_desc", "xg_status_str", "xg_mesh_create",
           "xg_mesh_np", "xg_mesh_dims", "xg_set_state", "xg_set_forcing", "xg_rhs",
           "xg_step", "xg_step_stream", "xg_get_state", "xg_set_contraction", "xg_set_fused", "xg_profile", "xg_kernel_times", "xg_rhs_noalloc", "xg_reciprocal", "xg_pressure_perturbation", "xg_partition_set",
           "xg_partition_stage", "xg_diagnostics", "xg_destroy", "library",
           "xg_batch_tuning", "xg_batch_create", "xg_batch_count", "xg_batch_instance",
           "xg_batch_step", "xg_batch_rhs", "xg_batch_autotune", "xg_batch_set_tuning",
           "xg_batch_get_tuning", "xg_batch_barrier_selftest", "xg_batch_destroy",
           "XG_SCHED_ROUND_ROBIN", "XG_SCHED_LPT", "XG_SCHED_DYNAMIC",
           "xg_features", "xg_restrict", "xg_column_stats", "xg_mlp_loss_grad", "xg_mlp_adam",
           "xg_mlp_forward", "xg_closure_set", "xg_correction_set", "xg_closure_target", "xg_tc_wait_selftest", "XG_MLP_FP32", "XG_MLP_BF16", "XG_CLOSURE_IN",
           "XG_CLOSURE_HIDDEN", "XG_CLOSURE_OUT", "XG_CLOSURE_PARAMS",
           "xg_dynamics", "xg_set_dynamics", "xg_dynamics_tendency", "xg_ri_velocity",
           "xg_imex_opts", "xg_imex_stats", "xg_step_imex", "xg_linear_operator", "XG_HOST", "XG_DEVICE",
           "XG_FP64", "XG_FP32", "XG_DF64", "XG_OK", "XG_ERR_ARG", "XG_ERR_CUDA", "XG_ERR_OOM",
           "XG_ERR_NONFINITE", "XG_ERR_TIMEOUT", "XG_ERR_UNSUPPORTED"]


class xg_mesh_desc(ctypes.Structure):
    _fields_ = [("nel", ctypes.c_int * 3), ("order", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("precision", ctypes.c_int),
                ("f_coriolis", ctypes.c_double), ("g", ctypes.c_double),
                ("R", ctypes.c_double), ("cp", ctypes.c_double), ("cv", ctypes.c_double),
                ("p_a", ctypes.c_double)]


class xg_batch_tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("plane_tile", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("ms_per_step", ctypes.c_double)]

    def as_dict(self):
        return dict(schedule=("round_robin", "lpt", "dynamic")[self.schedule],
                    plane_tile=self.plane_tile, ctas_per_sm=self.ctas_per_sm,
                    ms_per_step=self.ms_per_step)


class xg_dynamics(ctypes.Structure):
    _fields_ = [("hyper_c", ctypes.c_double * 3), ("hyper_dt", ctypes.c_double),
                ("sponge_depth", ctypes.c_double), ("sponge_gamma", ctypes.c_double)]


class xg_imex_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("krylov", ctypes.c_int), ("max_restarts", ctypes.c_int)]


class xg_imex_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_longlong), ("max_iterations", ctypes.c_int),
                ("solves", ctypes.c_int), ("max_residual", ctypes.c_double),
                ("reorthogonalised", ctypes.c_longlong)]

    def as_dict(self):
        return dict(iterations=self.iterations, max_iterations=self.max_iterations,
                    solves=self.solves, max_residual=self.max_residual,
                    reorthogonalised=self.reorthogonalised)


class XgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s" % (where, _status_name(status)))


_lib = None


def library():
    """Load libxg.so (once).  Raises when it has not been built: there is no
    fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libxg.so is not built (%s); run "
                           "paper_2504_08157_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.xg_status_str.restype = ctypes.c_char_p
    lib.xg_status_str.argtypes = [I]
    lib.xg_mesh_create.restype = I
    lib.xg_mesh_create.argtypes = [ctypes.POINTER(xg_mesh_desc), ctypes.POINTER(P)]
    lib.xg_mesh_np.restype = I
    lib.xg_mesh_np.argtypes = [P, ctypes.POINTER(LL)]
    lib.xg_mesh_dims.restype = I
    lib.xg_mesh_dims.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.xg_set_state.restype = I
    lib.xg_set_state.argtypes = [P, P, P, P, I, P]
    lib.xg_set_forcing.restype = I
    lib.xg_set_forcing.argtypes = [P, P, I, P]
    lib.xg_rhs.restype = I
    lib.xg_rhs.argtypes = [P, P, I, P]
    lib.xg_step.restype = I
    lib.xg_step.argtypes = [P, D, I, P]
    lib.xg_get_state.restype = I
    lib.xg_get_state.argtypes = [P, P, I, P]
    lib.xg_set_contraction.restype = I
    lib.xg_set_contraction.argtypes = [P, I]
    lib.xg_set_fused.restype = I
    lib.xg_set_fused.argtypes = [P, I]
    lib.xg_step_stream.restype = I
    lib.xg_step_stream.argtypes = [P, I, P, P, D, I, P]
    lib.xg_profile.restype = I
    lib.xg_profile.argtypes = [P, I]
    lib.xg_kernel_times.restype = I
    lib.xg_kernel_times.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(LL), I]
    lib.xg_rhs_noalloc.restype = I
    lib.xg_rhs_noalloc.argtypes = [ctypes.POINTER(xg_mesh_desc), P, P, P, P, P, P]
    lib.xg_reciprocal.restype = I
    lib.xg_reciprocal.argtypes = [P, P, LL, P]
    lib.xg_partition_set.restype = I
    lib.xg_partition_set.argtypes = [P, I, I, P, P, P, P]
    lib.xg_partition_stage.restype = I
    lib.xg_partition_stage.argtypes = [P, I, I, D, P, I, P]
    lib.xg_pressure_perturbation.restype = I
    lib.xg_pressure_perturbation.argtypes = [P, P, P, ctypes.POINTER(D), P]
    lib.xg_diagnostics.restype = I
    lib.xg_diagnostics.argtypes = [P, ctypes.POINTER(D), P]
    lib.xg_destroy.restype = None
    lib.xg_destroy.argtypes = [P]
    TP = ctypes.POINTER(xg_batch_tuning)
    lib.xg_batch_create.restype = I
    lib.xg_batch_create.argtypes = [ctypes.POINTER(xg_mesh_desc), I, ctypes.POINTER(P)]
    lib.xg_batch_count.restype = I
    lib.xg_batch_count.argtypes = [P, ctypes.POINTER(I)]
    lib.xg_batch_instance.restype = P
    lib.xg_batch_instance.argtypes = [P, I]
    lib.xg_batch_step.restype = I
    lib.xg_batch_step.argtypes = [P, ctypes.POINTER(D), I, P]
    lib.xg_batch_rhs.restype = I
    lib.xg_batch_rhs.argtypes = [P, ctypes.POINTER(P), I, P]
    lib.xg_batch_autotune.restype = I
    lib.xg_batch_autotune.argtypes = [P, ctypes.POINTER(D), I, TP, P]
    lib.xg_batch_set_tuning.restype = I
    lib.xg_batch_set_tuning.argtypes = [P, TP]
    lib.xg_batch_get_tuning.restype = I
    lib.xg_batch_get_tuning.argtypes = [P, TP]
    lib.xg_batch_barrier_selftest.restype = I
    lib.xg_batch_barrier_selftest.argtypes = [P, LL, P]
    lib.xg_batch_destroy.restype = None
    lib.xg_batch_destroy.argtypes = [P]
    lib.xg_features.restype = I
    lib.xg_features.argtypes = [P, P, P]
    lib.xg_restrict.restype = I
    lib.xg_restrict.argtypes = [P, P, P, I, P, P]
    lib.xg_column_stats.restype = I
    lib.xg_column_stats.argtypes = [P, I, LL, LL, ctypes.POINTER(D), ctypes.POINTER(D), P]
    lib.xg_mlp_loss_grad.restype = I
    lib.xg_mlp_loss_grad.argtypes = [P, P, P, LL, LL, P, P, P, P, ctypes.POINTER(D), P]
    lib.xg_mlp_adam.restype = I
    lib.xg_mlp_adam.argtypes = [P, P, P, P, I, I, D, D, D, D, P]
    lib.xg_mlp_forward.restype = I
    lib.xg_mlp_forward.argtypes = [P, P, LL, LL, P, P, P, P, LL, I, P]
    lib.xg_tc_wait_selftest.restype = I
    lib.xg_tc_wait_selftest.argtypes = [LL, P]
    lib.xg_closure_set.restype = I
    lib.xg_closure_set.argtypes = [P, P, P, P, P, P]
    lib.xg_correction_set.restype = I
    lib.xg_correction_set.argtypes = [P, P, P]
    lib.xg_closure_target.restype = I
    lib.xg_closure_target.argtypes = [P, P, ctypes.c_double, LL, P, P]
    lib.xg_set_dynamics.restype = I
    lib.xg_set_dynamics.argtypes = [P, ctypes.POINTER(xg_dynamics)]
    lib.xg_dynamics_tendency.restype = I
    lib.xg_dynamics_tendency.argtypes = [P, P, I, P]
    lib.xg_ri_velocity.restype = I
    lib.xg_ri_velocity.argtypes = [P, I, ctypes.POINTER(D), P, P, P]
    lib.xg_step_imex.restype = I
    lib.xg_step_imex.argtypes = [P, D, I, ctypes.POINTER(xg_imex_opts), ctypes.POINTER(xg_imex_stats), P]
    lib.xg_linear_operator.restype = I
    lib.xg_linear_operator.argtypes = [P, P, P, P]
    _lib = lib
    return lib


def _status_name(s):
    try:
        return library().xg_status_str(int(s)).decode()
    except Exception:  # the library itself failed to load
        return "status %d" % int(s)


def _check(s, where):
    if s != XG_OK:
        raise XgError(s, where)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, where=None, writable=False):
    """(address, where, stream-or-None) of an array argument."""
    if a is None:
        return None, where, None
    if isinstance(a, int):
        if where is None:
            raise ValueError("raw addresses need an explicit where")
        return a, where, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        if a.is_cuda:
            return a.data_ptr(), XG_DEVICE, torch.cuda.current_stream(a.device).cuda_stream
        return a.data_ptr(), XG_HOST, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float64")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("output array is read-only")
        return a.ctypes.data, XG_HOST, None
    raise TypeError("unsupported array type %r" % type(a))


def mesh_desc(nel, order, lo, hi, periodic, f=0.0, g=9.81, R=287.0, cp=1004.5, cv=717.5,
              p_a=1.0e5, precision=XG_FP64):
    """Fill an xg_mesh_desc (the problem statement of Sec. 2.1-2.2)."""
    d = xg_mesh_desc()
    for k in range(3):
        d.nel[k] = int(nel[k])
        d.lo[k] = float(lo[k])
        d.hi[k] = float(hi[k])
        d.periodic[k] = int(bool(periodic[k]))
    d.order = int(order)
    d.precision = int(precision)
    d.f_coriolis, d.g, d.R, d.cp, d.cv, d.p_a = float(f), float(g), float(R), float(cp), \
        float(cv), float(p_a)
    return d


def xg_status_str(s):
    return library().xg_status_str(int(s)).decode()


def xg_mesh_create(desc):
    """Returns the context handle (an integer address)."""
    out = ctypes.c_void_p()
    _check(library().xg_mesh_create(ctypes.byref(desc), ctypes.byref(out)), "xg_mesh_create")
    return out.value


def xg_mesh_np(ctx):
    n = ctypes.c_longlong()
    _check(library().xg_mesh_np(ctx, ctypes.byref(n)), "xg_mesh_np")
    return n.value


def xg_mesh_dims(ctx):
    n = (ctypes.c_int * 3)()
    _check(library().xg_mesh_dims(ctx, n), "xg_mesh_dims")
    return tuple(n)


def _stream(stream, implied):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    return implied


def xg_set_state(ctx, q, rho0=None, rhotheta0=None, where=None, stream=None):
    pq, wq, sq = _ptr(q, where)
    pr, wr, _ = _ptr(rho0, wq)
    pt, wt, _ = _ptr(rhotheta0, wq)
    if pr is not None and (wr != wq or wt != wq):
        raise ValueError("q and the reference arrays must all be host or all device")
    _check(library().xg_set_state(ctx, pq, pr, pt, wq, _stream(stream, sq)), "xg_set_state")


def xg_set_forcing(ctx, S_theta, where=None, stream=None):
    p, w, s = _ptr(S_theta, where)
    _check(library().xg_set_forcing(ctx, p, XG_HOST if w is None else w, _stream(stream, s)),
           "xg_set_forcing")


def xg_rhs(ctx, dqdt, where=None, stream=None):
    p, w, s = _ptr(dqdt, where, writable=True)
    _check(library().xg_rhs(ctx, p, w, _stream(stream, s)), "xg_rhs")


def xg_step(ctx, dt, nsteps, stream=None):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    _check(library().xg_step(ctx, float(dt), int(nsteps), _stream(stream, None)), "xg_step")


def xg_get_state(ctx, q, where=None, stream=None):
    p, w, s = _ptr(q, where, writable=True)
    _check(library().xg_get_state(ctx, p, w, _stream(stream, s)), "xg_get_state")


def xg_set_contraction(ctx, mode):
    _check(library().xg_set_contraction(ctx, int(mode)), "xg_set_contraction")


def xg_step_stream(ctx, q_in, q_out, dt, nsteps=1, stream=None):
    """nsteps steps of each host state q_in[k] ([5][Np] float64 CPU tensors or
    arrays, pinned for the full rate) into q_out[k], the copies overlapping
    the steps (see include/xg.h)."""
    if len(q_in) != len(q_out):
        raise ValueError("q_in and q_out need one entry per input")
    n = len(q_in)
    size = 5 * xg_mesh_np(ctx)
    for a in list(q_in) + list(q_out):
        if (a.numel() if _is_torch(a) else np.asarray(a).size) != size:
            raise ValueError("each state needs 5 x Np values")
    pin = (ctypes.c_void_p * max(n, 1))()
    pout = (ctypes.c_void_p * max(n, 1))()
    for k in range(n):
        pi, wi, _ = _ptr(q_in[k])
        po, wo, _ = _ptr(q_out[k], writable=True)
        if wi != XG_HOST or wo != XG_HOST:
            raise ValueError("xg_step_stream takes host arrays")
        pin[k], pout[k] = pi, po
    _check(library().xg_step_stream(ctx, n, pin, pout, float(dt), int(nsteps), _default_stream(stream)),
           "xg_step_stream")


def xg_set_fused(ctx, fused):
    """XG_FP32: one fused column pass per stage where the mesh allows it (1),
    or the plane + z-line kernels (0, the default)."""
    _check(library().xg_set_fused(ctx, int(fused)), "xg_set_fused")


def xg_profile(ctx, enable):
    _check(library().xg_profile(ctx, int(bool(enable))), "xg_profile")


def xg_kernel_times(ctx, reset=False):
    """((ms_x, ms_y, ms_z), (launches_x, launches_y, launches_z))."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_longlong * 3)()
    _check(library().xg_kernel_times(ctx, ms, n, int(bool(reset))), "xg_kernel_times")
    return tuple(ms), tuple(n)


def xg_rhs_noalloc(desc, q, rho0, rhotheta0, S_theta, dqdt, stream=None):
    """Context-free right-hand side that allocates no device memory (all
    arrays are device memory of the current device)."""
    pq, wq, sq = _ptr(q)
    ptrs = [_ptr(a) for a in (rho0, rhotheta0, S_theta, dqdt)]
    if wq != XG_DEVICE or any(p[0] is not None and p[1] != XG_DEVICE for p in ptrs):
        raise ValueError("xg_rhs_noalloc takes device arrays only")
    _check(library().xg_rhs_noalloc(ctypes.byref(desc), pq, ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                    ptrs[3][0], _stream(stream, sq)), "xg_rhs_noalloc")


def xg_reciprocal(x, out, stream=None):
    """The library's FP64 reciprocal applied to device values (test hook)."""
    px, wx, sx = _ptr(x)
    po, wo, _ = _ptr(out, writable=True)
    if wx != XG_DEVICE or wo != XG_DEVICE:
        raise ValueError("xg_reciprocal takes device arrays")
    n = x.numel() if hasattr(x, "numel") else len(x)
    _check(library().xg_reciprocal(px, po, int(n), _stream(stream, sx)), "xg_reciprocal")


def xg_partition_set(ctx, open_lo, open_hi, send_lo=None, recv_lo=None, send_hi=None, recv_hi=None):
    """Mark the context's y ends as partition faces and give the exchange
    buffers (device arrays of 5 n_x n_z values of 8 bytes each, owned by the
    caller and kept alive while the partition is set)."""
    ptrs = []
    for a in (send_lo, recv_lo, send_hi, recv_hi):
        if a is None:
            ptrs.append(None)
            continue
        p, w, _ = _ptr(a, writable=True)
        if w != XG_DEVICE:
            raise ValueError("partition face buffers must be device arrays")
        ptrs.append(p)
    _check(library().xg_partition_set(ctx, int(open_lo), int(open_hi), *ptrs), "xg_partition_set")


def xg_partition_stage(ctx, half, stage, dt=0.0, dqdt=None, stream=None):
    """One half of a partitioned stage (stage 0..2 of an SSP-RK3 step, or -1
    for dq/dt into dqdt)."""
    pd, wd, sd = _ptr(dqdt, writable=True)
    st = _stream(stream, sd) if (stream is not None or sd is not None) else _default_stream(None)
    _check(library().xg_partition_stage(ctx, int(half), int(stage), float(dt), pd,
                                        XG_DEVICE if wd is None else wd, st),
           "xg_partition_stage")


def xg_pressure_perturbation(ctx, theta_p, out, stream=None):
    """p' of Eq. 3 at every node from Theta' (device arrays of Np values),
    through the context's own equation-of-state code (test hook); returns the
    series/fallback switch point x_max."""
    pt, wt, st = _ptr(theta_p)
    po, wo, _ = _ptr(out, writable=True)
    if wt != XG_DEVICE or wo != XG_DEVICE:
        raise ValueError("xg_pressure_perturbation takes device arrays")
    xm = ctypes.c_double(0.0)
    _check(library().xg_pressure_perturbation(ctx, pt, po, ctypes.byref(xm), _stream(stream, st)),
           "xg_pressure_perturbation")
    return xm.value


def xg_diagnostics(ctx, stream=None):
    """FP64 conservation sums sum_I M_I q_v,I, v = 0..4, of the current state."""
    out = (ctypes.c_double * 5)()
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    _check(library().xg_diagnostics(ctx, out, _stream(stream, None)), "xg_diagnostics")
    return tuple(out)


def xg_destroy(ctx):
    if ctx:
        library().xg_destroy(ctx)


# ------------------------------------------------------------------ batched persistent form

def _default_stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    return _stream(stream, None)


def xg_batch_create(descs):
    """Batch of XG_FP32 instances from a sequence of xg_mesh_desc; returns the
    handle (an integer address)."""
    arr = (xg_mesh_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(library().xg_batch_create(arr, len(descs), ctypes.byref(out)), "xg_batch_create")
    return out.value


def xg_batch_count(batch):
    n = ctypes.c_int()
    _check(library().xg_batch_count(batch, ctypes.byref(n)), "xg_batch_count")
    return n.value


def xg_batch_instance(batch, i):
    """The xg_ctx handle of instance i (owned by the batch)."""
    c = library().xg_batch_instance(batch, int(i))
    if not c:
        raise XgError(XG_ERR_ARG, "xg_batch_instance")
    return c


def _dt_array(dt):
    a = np.ascontiguousarray(np.asarray(dt, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def xg_batch_step(batch, dt, nsteps, stream=None):
    """nsteps SSP-RK3 steps of every instance (dt: one value per instance)."""
    a, p = _dt_array(dt)
    if a.size != xg_batch_count(batch):
        raise ValueError("dt needs one value per instance")
    _check(library().xg_batch_step(batch, p, int(nsteps), _default_stream(stream)),
           "xg_batch_step")


def xg_batch_rhs(batch, dqdt, stream=None):
    """Right-hand sides of every instance into dqdt[i] (all host or all
    device float64 arrays)."""
    ptrs = [_ptr(a, writable=True) for a in dqdt]
    where = {p[1] for p in ptrs}
    if len(where) != 1:
        raise ValueError("dqdt arrays must be all host or all device")
    implied = next((p[2] for p in ptrs if p[2] is not None), None)
    arr = (ctypes.c_void_p * len(ptrs))(*[p[0] for p in ptrs])
    _check(library().xg_batch_rhs(batch, arr, where.pop(), _stream(stream, implied) if implied
                                  else _default_stream(stream)), "xg_batch_rhs")


def xg_batch_autotune(batch, dt, trial_steps=2, stream=None):
    a, p = _dt_array(dt)
    t = xg_batch_tuning()
    _check(library().xg_batch_autotune(batch, p, int(trial_steps), ctypes.byref(t),
                                       _default_stream(stream)), "xg_batch_autotune")
    return t


def xg_batch_set_tuning(batch, schedule, plane_tile=0, ctas_per_sm=2):
    t = xg_batch_tuning(int(schedule), int(plane_tile), int(ctas_per_sm), 0.0)
    _check(library().xg_batch_set_tuning(batch, ctypes.byref(t)), "xg_batch_set_tuning")


def xg_batch_get_tuning(batch):
    t = xg_batch_tuning()
    _check(library().xg_batch_get_tuning(batch, ctypes.byref(t)), "xg_batch_get_tuning")
    return t


def xg_batch_barrier_selftest(batch, spin_limit=20000, stream=None):
    """Returns the status of the deliberately starved barrier (XG_ERR_TIMEOUT
    when the bounded wait works)."""
    return library().xg_batch_barrier_selftest(batch, int(spin_limit), _default_stream(stream))


def xg_batch_destroy(batch):
    if batch:
        library().xg_batch_destroy(batch)


# ------------------------------------------------------------------ learned closure
# Arrays are float32 CUDA tensors (device memory); feature and target sets
# are [rows][ld] with the sample index fastest.

def _f32(a, rows=None):
    import torch
    if not (_is_torch(a) and a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if rows is not None and (a.dim() != 2 or a.shape[0] != rows):
        raise ValueError("expected %d rows" % rows)
    return a.data_ptr()


def xg_features(ctx, X, stream=None):
    """Features of an XG_FP32 context's state into X [21][Np] (float32)."""
    _check(library().xg_features(ctx, _f32(X, XG_CLOSURE_IN), _default_stream(stream)), "xg_features")


def xg_restrict(fine, coarse, src, dst, stream=None):
    """Fields src [nv][Np_fine] (float64 CUDA) at the nodes of ``coarse`` into dst [nv][Np_coarse]."""
    ps, ws, _ = _ptr(src)
    pd, wd, _ = _ptr(dst, writable=True)
    if ws != XG_DEVICE or wd != XG_DEVICE:
        raise ValueError("xg_restrict takes device arrays")
    nv = src.shape[0] if src.dim() == 2 else 1
    _check(library().xg_restrict(fine, coarse, ps, int(nv), pd, _default_stream(stream)), "xg_restrict")


def xg_column_stats(X, n=None, stream=None):
    """(mean, std) float64 numpy arrays of the rows of X [ncol][ld] over the
    first n samples."""
    ncol, ld = X.shape
    n = ld if n is None else n
    mean = (ctypes.c_double * ncol)()
    std = (ctypes.c_double * ncol)()
    _check(library().xg_column_stats(_f32(X), int(ncol), int(ld), int(n), mean, std,
                                     _default_stream(stream)), "xg_column_stats")
    return np.array(mean), np.array(std)


def xg_mlp_loss_grad(params, X, T, in_mean, in_scale, out_scale, grad, n=None, stream=None):
    """MSE of the network on the first n samples of X [21][ld] against T
    [5][ld]; writes grad (float32 [5893]) and returns the loss."""
    ld = X.shape[1]
    n = ld if n is None else n
    if T.shape[1] != ld:
        raise ValueError("X and T need the same leading dimension")
    loss = ctypes.c_double()
    _check(library().xg_mlp_loss_grad(_f32(params), _f32(X, XG_CLOSURE_IN), _f32(T, XG_CLOSURE_OUT),
                                      int(ld), int(n), _f32(in_mean), _f32(in_scale), _f32(out_scale),
                                      _f32(grad), ctypes.byref(loss), _default_stream(stream)),
           "xg_mlp_loss_grad")
    return loss.value


def xg_mlp_adam(params, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(library().xg_mlp_adam(_f32(params), _f32(m), _f32(v), _f32(grad), int(params.numel()),
                                 int(t), float(lr), float(beta1), float(beta2), float(eps),
                                 _default_stream(stream)), "xg_mlp_adam")


def xg_mlp_forward(params, X, in_mean, in_scale, out_scale, Y, precision=XG_MLP_BF16, n=None,
                   stream=None):
    ld, ldy = X.shape[1], Y.shape[1]
    n = ld if n is None else n
    _check(library().xg_mlp_forward(_f32(params), _f32(X, XG_CLOSURE_IN), int(ld), int(n),
                                    _f32(in_mean), _f32(in_scale), _f32(out_scale),
                                    _f32(Y, XG_CLOSURE_OUT), int(ldy), int(precision),
                                    _default_stream(stream)), "xg_mlp_forward")


def xg_tc_wait_selftest(limit_ns, stream=None):
    """Status of a tensor-core wait made to run out (XG_ERR_TIMEOUT expected)."""
    st = library().xg_tc_wait_selftest(int(limit_ns), _default_stream(stream))
    if st not in (XG_OK, XG_ERR_TIMEOUT):
        _check(st, "xg_tc_wait_selftest")
    return st


def xg_closure_set(ctx, params=None, in_mean=None, in_scale=None, out_scale=None, stream=None):
    """Enable the closure on an XG_FP32 context (params None disables it)."""
    if params is None:
        _check(library().xg_closure_set(ctx, None, None, None, None, _default_stream(stream)),
               "xg_closure_set")
        return
    _check(library().xg_closure_set(ctx, _f32(params), _f32(in_mean), _f32(in_scale),
                                    _f32(out_scale), _default_stream(stream)), "xg_closure_set")


def xg_correction_set(ctx, C=None, stream=None):
    """A prescribed correction C [5][Np] (float64 CUDA) added to the
    tendency of an XG_FP32 context in every stage (None removes it)."""
    if C is None:
        _check(library().xg_correction_set(ctx, None, _default_stream(stream)), "xg_correction_set")
        return
    p, w, _ = _ptr(C)
    if w != XG_DEVICE or C.dim() != 2 or C.shape[0] != 5:
        raise ValueError("xg_correction_set takes a [5][Np] device array")
    _check(library().xg_correction_set(ctx, p, _default_stream(stream)), "xg_correction_set")


def xg_closure_target(a, b, s=1.0, out=None, stream=None):
    """out = s (a - b) for float64 CUDA arrays of one shape (a new array when
    out is None); returns out."""
    import torch
    if out is None:
        out = torch.empty_like(a)
    for t in (a, b, out):
        if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected contiguous float64 CUDA tensors")
    if a.shape != b.shape or a.shape != out.shape:
        raise ValueError("a, b and out must have one shape")
    _check(library().xg_closure_target(a.data_ptr(), b.data_ptr(), float(s), int(a.numel()), out.data_ptr(),
                                       _default_stream(stream)), "xg_closure_target")
    return out


# ------------------------------------------------------------------ remaining dynamics

def xg_set_dynamics(ctx, hyper_c=(0.0, 0.0, 0.0), hyper_dt=1.0, sponge_depth=0.0, sponge_gamma=0.0,
                    off=False):
    """Hyper-diffusion (c_i, dt of Eq. 16) and the top sponge on an XG_FP64
    context; off=True switches both off."""
    if off:
        _check(library().xg_set_dynamics(ctx, None), "xg_set_dynamics")
        return
    d = xg_dynamics((ctypes.c_double * 3)(*[float(v) for v in hyper_c]), float(hyper_dt),
                    float(sponge_depth), float(sponge_gamma))
    _check(library().xg_set_dynamics(ctx, ctypes.byref(d)), "xg_set_dynamics")


def xg_dynamics_tendency(ctx, out, where=None, stream=None):
    p, w, s = _ptr(out, where, writable=True)
    _check(library().xg_dynamics_tendency(ctx, p, w, _stream(stream, s)), "xg_dynamics_tendency")


def xg_ri_velocity(ctx, nstrips=50, stream=None):
    """(u_RI, centroid [n_z, 2], strip means [n_z, nstrips]) of the state."""
    nz = xg_mesh_dims(ctx)[2]
    u = ctypes.c_double()
    cent = np.zeros((nz, 2))
    means = np.zeros((nz, int(nstrips)))
    _check(library().xg_ri_velocity(ctx, int(nstrips), ctypes.byref(u), cent.ctypes.data,
                                    means.ctypes.data, _default_stream(stream)), "xg_ri_velocity")
    return u.value, cent, means


# ------------------------------------------------------------------ IMEX

def xg_step_imex(ctx, dt, nsteps, tol=1e-10, krylov=20, max_restarts=50, stream=None):
    """nsteps IMEX ARK2 steps; returns the solver statistics."""
    o = xg_imex_opts(float(tol), int(krylov), int(max_restarts))
    st = xg_imex_stats()
    _check(library().xg_step_imex(ctx, float(dt), int(nsteps), ctypes.byref(o), ctypes.byref(st),
                                  _default_stream(stream)), "xg_step_imex")
    return st


def xg_linear_operator(ctx, v, out, stream=None):
    """out = L(v) (device float64 arrays [5][Np])."""
    pv, wv, sv = _ptr(v)
    po, wo, _ = _ptr(out, writable=True)
    if wv != XG_DEVICE or wo != XG_DEVICE:
        raise ValueError("xg_linear_operator takes device arrays")
    _check(library().xg_linear_operator(ctx, pv, po, _stream(stream, sv)), "xg_linear_operator")
