"""Throughput of the explicit CG Euler path on GB300: RK-stage GDOF/s.

Default workload (the cyclone box): 1024 x 1024 x 20 km, 128 x 128 x 16
order-4 elements, doubly periodic sides, no-flux bottom and top
(512 x 512 x 65 = 17,039,360 nodes), stable sounding, f-plane, vortex and
ring-plus-cells heating, dt = 0.1 s.  The timed arm is the FP64-accurate
mixed path (--precision df64, the default: FP64 state, rho' and Theta' on
the FP64 pipe, the momentum in double-float arithmetic on the FP32 pipes);
the same line reports plain native FP64 on the same workload and GPU, the
FP32, batched and closure forms, and the relative L2 errors against the
oracle (at the timed full-size state against its extended-precision
evaluation).  One bench step is one SSP-RK3
step = three passes of the whole hot path (each pass: primitives, fluxes,
sum-factorised derivatives, DSS, inverse mass, sources, walls, stage
update), so

    value = 5 * Np * 3 * K * world / max-over-ranks(time of K steps) / 1e9

in unique-node DOF (the paper's element-local convention, N_e (N+1)^3 x 5,
is reported beside it).  Inputs are resident in HBM before the timed region;
each state buffer (682 MB) is larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xg|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference there is)
on a bounded sample of the same workload.  Under torchrun every rank runs an
independent replica (the path needs no exchange on one box) and rank 0
prints one JSON line.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # one thread per oracle worker process (OracleTeam)

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK-stage GDOF/s vs plain FP64 at stated L2 error; % of HBM roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2504_08157_gb300", "csrc", f)
               for f in ("xg_kernels.cuh", "xg_kernels_df.cuh", "xg_df.cuh", "xg_kernels_f32.cuh",
                         "xg_plane_f32.cuh", "xg_batch.cu", "xg_closure.cu", "xg_tc.cuh", "xg_plane_tc.cuh",
                         "xg_plane_h16.cuh", "xg_column_f32.cuh", "xg_tma.cuh")]
KERNELS = ("k_line_x", "k_line_y", "k_line_z")
# the kernels behind the three timing slots in each precision (the FP32 form
# fuses the x and y passes into one plane kernel; slot 1 stays empty)
KERNEL_NAMES = {0: ("k_line_x", "k_line_y", "k_line_z"),
                2: ("k_df_line_x", "k_df_tline_y", "k_df_tline_z"),
                1: ("k_f_plane_xy", "-", "k_f_tline")}
# the FP32 plane kernel of each tensor-core contraction mode (by --contraction
# name: the mode's constant, the kernel; by mode constant: the kernel)
CONTRACTIONS = {"tf32x3": (lambda xg: xg.XG_CONTRACT_TF32X3, "k_f_plane_xy_tc"),
                "f16x3": (lambda xg: xg.XG_CONTRACT_F16X3, "k_f_plane_xy_h16")}
PLANE_KERNEL_OF = {1: "k_f_plane_xy_tc", 2: "k_f_plane_xy_h16"}
# the FP32 form's opt-in fused pass (order 4, walls at the bottom and top, the
# CUDA-core contraction): the whole stage is one kernel in timing slot 0
COLUMN_NAMES = ("k_f_column", "-", "-")


def fp32_kernel_names(wl, contract=0, fused=False):
    """The kernels behind the FP32 form's timing slots on workload wl."""
    if contract:
        return (PLANE_KERNEL_OF[contract],) + KERNEL_NAMES[1][1:]
    if fused and wl["N"] == 4 and not wl["periodic"][2]:
        return COLUMN_NAMES
    return KERNEL_NAMES[1]
# FP64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x
# 2 flop x 2.07 GHz (maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 instructions (DFMA + DADD + DMUL) per node and launch of the mixed
# path's kernels, from the --set full capture of the 64x64x16 order-4 case
# (profiles/line_kernels_tc.md); the pipe issues 2 per clock per SM.
DF64_FP64_INSTR_PER_NODE = {"k_df_line_x": 17.5, "k_df_tline_y": 14.0, "k_df_tline_z": 20.6}
FP64_PIPE_PEAK_GINSTR = 152 * 2 * 2.07e9 / 1e9


def flops_per_node(kernel, N):
    """Algorithmic FP64 flops per unique node of each kernel (FMA = 2), from
    the arithmetic each performs for N-th order elements (one segment of
    N+1 nodes covers N unique nodes):

    * x: the even/odd contraction of one flux component over a segment,
      2P adds + P (4P + 2e) + e (2P - 1) with P = (N+1)//2, e = [N even];
      face sums 5/N; pointwise rho (1), 1/rho (4 fma), u v w (3),
      Theta'/Theta0 (1), 8-term series (7 fma + 1 mul), p0 * (1), Theta (1),
      x-fluxes (1 fma + 3 mul).
    * y, z: N rows of N+1 fma started from the running tendency, row N
      (1 mul + N fma) and the face addition: 2N^2 + 4N + 2 per component and
      segment; fluxes (3 mul + 1 fma + 1 add).  z adds the sources (3 fma,
      1 add, 1 fma) and the stage update (5 fma in stage 1, 5 x (2 fma +
      1 mul) in stages 2-3, averaged)."""
    P, e = (N + 1) // 2, 1 if N % 2 == 0 else 0
    eo = 2 * P + P * (4 * P + 2 * e) + e * (2 * P - 1)
    folded = 2 * N * N + 4 * N + 2
    if kernel == "k_line_x":
        pointwise = 1 + 8 + 3 + 1 + 15 + 1 + 1 + 1 + 5
        return pointwise + 5.0 * eo / N + 5.0 / N
    if kernel == "k_line_y":
        return 6 + 5.0 * folded / N
    if kernel == "k_line_z":
        return 6 + 5.0 * folded / N + 9 + (10 + 25 + 25) / 3.0
    raise KeyError(kernel)


def kernel_source_sha():
    """sha256 prefix over the kernel sources (a capture is valid only for them)."""
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def stage_traffic(kernels):
    """DRAM bytes of one RK stage (the kernels' per-launch traffic averaged
    over the three stages, summed), from the committed ncu summary if every
    kernel was captured on the current source; else None."""
    vals = [traffic_per_launch(k) for k in kernels]
    if not vals or any(v is None for v in vals):
        return None
    return float(sum(vals))


def traffic_per_launch(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    sha = kernel_source_sha()
    vals = {}
    for line in open(TRAFFIC_FILE):
        p = line.split()
        if len(p) >= 2 and not line.startswith("#"):
            vals[p[0]] = p[1]
    if vals.get("source_sha") != sha:
        return None
    v = vals.get(kernel)
    return float(v) if v is not None else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 50 ms, in a thread."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 8:
                continue
            for k, name in enumerate(names):
                if r[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(self.rows[0][1]),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload(name, nel=None):
    from inputs import workloads as W
    if name == "tc":
        return W.tc() if nel is None else W.tc(nel=tuple(nel))
    if name == "bubble":
        return W.bubble()
    raise SystemExit("unknown workload " + name)


def describe(wl):
    from inputs import workloads as W
    dof_u, dof_p = W.dof_counts(wl["nel"], wl["N"], wl["periodic"])
    per = "".join("p" if p else "w" for p in wl["periodic"])
    return dict(workload="%s %dx%dx%d N=%d FP64 (%s)" % (wl["name"], *wl["nel"], wl["N"], per),
                nel=list(wl["nel"]), N=wl["N"], nodes=dof_u // 5, dof_unique=dof_u,
                dof_paper=dof_p, dt=wl["dt"], periodic=list(wl["periodic"]),
                l2="inputs larger than L2 (each [5][Np] FP64 buffer 682 MB > 129 MB L2)",
                parallelism="replicas")


# ------------------------------------------------------------------ CPU oracle timing

def cpu_sample_workload(name):
    """A bounded sample of the workload for the oracle: the cyclone box with
    16 x 16 x 16 elements (same spacing and order, 266,240 nodes); the
    bubble case is small enough to run whole."""
    from inputs import workloads as W
    if name == "tc":
        return W.tc(nel=(16, 16, 16))
    if name == "batch":
        specs = W.batch_specs()
        sizes = [s["N"] ** 3 * s["nel"][0] * s["nel"][1] * s["nel"][2] for s in specs]
        return W.batch_instance(specs[int(np.argsort(sizes)[len(sizes) // 2])])
    return W.bubble()


def full_size_errors(wl, xg, torch, dev, count=600, seed=2504):
    """Errors of one GPU right-hand side of the timed workload itself (full
    size, the timed state) at `count` seeded nodes, against the oracle in
    extended precision (the FP64 oracle's own rounding is close to 1e-12
    there); per precision, plus the floors that rounding the state to FP32
    or to double-float alone sets."""
    n = [wl["N"] * wl["nel"][d] + (0 if wl["periodic"][d] else 1) for d in range(3)]
    rng = np.random.default_rng(seed)
    nodes = np.unique(rng.integers(0, n[0], count) + n[0] * (rng.integers(0, n[1], count)
                      + n[1] * rng.integers(0, n[2], count)))
    refx = oracle_rhs_extended_at(wl, nodes)
    out = {"nodes": int(nodes.size)}
    for p, v in (("fp64", xg.XG_FP64), ("df64", xg.XG_DF64), ("fp32", xg.XG_FP32)):
        out[p] = rel_err(gpu_rhs(wl, xg, torch, dev, v)[:, nodes], refx)
    h = wl["q"].astype(np.float32).astype(np.float64)
    out["df64_state_rounding_floor"] = rel_err(
        oracle_rhs_extended_at(dict(wl, q=h + (wl["q"] - h).astype(np.float32).astype(np.float64)), nodes), refx)
    out["fp32_state_rounding_floor"] = rel_err(oracle_rhs_extended_at(dict(wl, q=h), nodes), refx)
    out["meets_1e-12"] = {p: bool(max(out[p]) <= 1e-12) for p in ("fp64", "df64")}
    return out


def random_state_errors(name, xg, torch, dev):
    """oracle_error_of_gpu per precision on the CPU sample of the cyclone box
    at a seeded smooth random state plus the vortex (None for the other
    workloads)."""
    from inputs import workloads as W
    if name != "tc":
        return None
    sw = W.tc(nel=(16, 16, 16), state="random")
    out = {p: oracle_error_of_gpu(sw, xg, torch, dev, v)
           for p, v in (("df64", xg.XG_DF64), ("fp64", xg.XG_FP64), ("fp32", xg.XG_FP32))}
    out["fp32_tf32x3_contraction"] = oracle_error_of_gpu(sw, xg, torch, dev, xg.XG_FP32, xg.XG_CONTRACT_TF32X3)
    out["fp32_f16x3_contraction"] = oracle_error_of_gpu(sw, xg, torch, dev, xg.XG_FP32, xg.XG_CONTRACT_F16X3)
    return out


def _oracle_worker(conn, wl, elements, q_name, r_name, slot, np_):
    """One worker of OracleTeam: holds the elements it was given and, on each
    request, writes the oracle's partial DSS sums R (Eqs. 9-11) of those
    elements for the state in shared memory into its own slot."""
    from multiprocessing import shared_memory
    from oracle import euler as E, mesh as M
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], elements=elements)
    phys = E.Physics(**wl["phys"])
    base = E.Base(wl["rho0"], wl["Theta0"])
    qs, rs = shared_memory.SharedMemory(name=q_name), shared_memory.SharedMemory(name=r_name)
    q = np.ndarray((5, np_), dtype=np.float64, buffer=qs.buf)
    R = np.ndarray((slot[1], 6, np_), dtype=np.float64, buffer=rs.buf)[slot[0]]
    _, Mw = E.assemble(m, np.zeros((1,) + m.intma.shape))
    R[5] = Mw
    conn.send("ready")
    while conn.recv() == "rhs":
        S = E.local_tendency(m, q, base, wl["S_theta"], phys)
        R[:5] = E.assemble(m, S)[0]
        conn.send("done")
    del q, R
    qs.close()
    rs.close()


class OracleTeam:
    """The FP64 oracle's right-hand side on all host cores: the elements are
    split into one contiguous chunk per worker process (spawned, so it is safe
    next to a CUDA context), each worker evaluates the oracle's pointwise
    S(q) and partial DSS sums for its chunk, and the partial sums are added in
    worker order before the inverse mass and the walls (Eq. 12).  Same
    functions and arithmetic as the single-process oracle; only the
    summation order of the assembly differs."""

    def __init__(self, wl, workers=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        from oracle import euler as E, mesh as M
        self.workers = workers or os.cpu_count() or 1
        ne = wl["nel"][0] * wl["nel"][1] * wl["nel"][2]
        self.workers = max(1, min(self.workers, ne))
        self.wall_mesh = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"],
                                      elements=[0])
        self.np = self.wall_mesh.Np
        self.qs = shared_memory.SharedMemory(create=True, size=5 * self.np * 8)
        self.rs = shared_memory.SharedMemory(create=True, size=self.workers * 6 * self.np * 8)
        self.q = np.ndarray((5, self.np), dtype=np.float64, buffer=self.qs.buf)
        self.R = np.ndarray((self.workers, 6, self.np), dtype=np.float64, buffer=self.rs.buf)
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for w, el in enumerate(np.array_split(np.arange(ne), self.workers)):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, daemon=True,
                            args=(b, wl, el, self.qs.name, self.rs.name, (w, self.workers), self.np))
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            c.recv()
        self.M = np.zeros(self.np)
        for w in range(self.workers):
            self.M += self.R[w, 5]
        self.E = E

    def rhs(self, q):
        self.q[:] = q
        for c in self.conns:
            c.send("rhs")
        for c in self.conns:
            c.recv()
        R = self.R[0, :5].copy()
        for w in range(1, self.workers):
            R += self.R[w, :5]
        return self.E.apply_walls(self.wall_mesh, R / self.M[None, :])

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=10)
        del self.q, self.R
        self.qs.close()
        self.qs.unlink()
        self.rs.close()
        self.rs.unlink()


def time_oracle(wl, min_seconds=10.0, max_steps=50, team=None):
    """SSP-RK3 steps of the oracle until min_seconds have passed; returns
    (unique-DOF GDOF/s per stage, steps, seconds, final state, worker
    processes).  The right-hand side runs on all host cores (OracleTeam)."""
    from oracle import ssprk3
    from inputs import workloads as W
    own = team is None
    team = team or OracleTeam(wl)
    try:
        q = wl["q"]
        t0 = time.perf_counter()
        steps = 0
        while steps < max_steps:
            q = ssprk3.ssprk3_step(team.rhs, q, wl["dt"])
            steps += 1
            if time.perf_counter() - t0 >= min_seconds:
                break
        dt = time.perf_counter() - t0
    finally:
        if own:
            team.close()
    dof_u, _ = W.dof_counts(wl["nel"], wl["N"], wl["periodic"])
    return dof_u * 3 * steps / dt / 1e9, steps, dt, q, team.workers


def oracle_rhs(wl, q=None):
    """The FP64 oracle's right-hand side of the workload (or of state q)."""
    from oracle import euler as E, mesh as M
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    return E.rhs(m, wl["q"] if q is None else q, E.Base(wl["rho0"], wl["Theta0"]), wl["S_theta"],
                 E.Physics(**wl["phys"]))


def oracle_rhs_extended_at(wl, nodes):
    """The oracle in extended precision (np.longdouble) at the given nodes:
    the reference where the rho' and Theta' tendencies are residuals of
    cancelling parts and the FP64 oracle's own rounding approaches 1e-12."""
    from oracle import euler as E, mesh as M
    el = M.elements_around(wl["nel"], wl["N"], wl["periodic"], nodes)
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], elements=el,
                     dtype=np.longdouble)
    ld = lambda a: None if a is None else np.asarray(a, dtype=np.longdouble)
    return E.rhs_at_nodes(m, ld(wl["q"]), E.Base(wl["rho0"], wl["Theta0"]), ld(wl["S_theta"]),
                          E.Physics(**wl["phys"]), nodes).astype(np.float64)


def rel_err(got, ref):
    return [float("%.3e" % (np.linalg.norm(got[v] - ref[v]) / max(np.linalg.norm(ref[v]), 1e-300)))
            for v in range(5)]


def gpu_rhs(wl, xg, torch, dev, precision, contract=0):
    ctx = make_ctx(xg, torch, wl, dev, precision)
    try:
        if contract:
            xg.xg_set_contraction(ctx, contract)
        out = torch.empty((5, xg.xg_mesh_np(ctx)), dtype=torch.float64, device=dev)
        xg.xg_rhs(ctx, out)
        return out.cpu().numpy()
    finally:
        xg.xg_destroy(ctx)


def oracle_error_of_gpu(wl, xg, torch, dev, precision, contract=0):
    """Relative L2 per variable between one GPU right-hand side and the
    oracle's on the CPU sample (contract: the FP32 contraction arithmetic)."""
    from oracle import euler as E, mesh as M
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    ref = E.rhs(m, wl["q"], E.Base(wl["rho0"], wl["Theta0"]), wl["S_theta"],
                E.Physics(**wl["phys"]))
    ctx = make_ctx(xg, torch, wl, dev, precision)
    try:
        if contract:
            xg.xg_set_contraction(ctx, contract)
        out = torch.empty((5, xg.xg_mesh_np(ctx)), dtype=torch.float64, device=dev)
        xg.xg_rhs(ctx, out)
        got = out.cpu().numpy()
    finally:
        xg.xg_destroy(ctx)
    err = [np.linalg.norm(got[v] - ref[v]) / max(np.linalg.norm(ref[v]), 1e-300) for v in range(5)]
    return [float("%.3e" % e) for e in err]


# ------------------------------------------------------------------ GPU arm

def make_ctx(xg, torch, wl, dev, precision=0):
    ph = wl["phys"]
    ctx = xg.xg_mesh_create(xg.mesh_desc(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"],
                                         f=ph["f"], g=ph["g"], R=ph["R"], cp=ph["cp"],
                                         cv=ph["cv"], p_a=ph["p_a"], precision=precision))
    q = torch.from_numpy(wl["q"]).to(dev)
    xg.xg_set_state(ctx, q, torch.from_numpy(wl["rho0"]).to(dev),
                    torch.from_numpy(wl["Theta0"]).to(dev))
    if wl["S_theta"] is not None:
        xg.xg_set_forcing(ctx, torch.from_numpy(wl["S_theta"]).to(dev))
    torch.cuda.synchronize()
    return ctx


# Values each kernel must move per node given its inputs and outputs (times
# the bytes per stored value): the x pass reads q (5) and writes W (v, w, p'
# and, in FP64 and XG_DF64, theta) and T (5); the y pass reads the momentum
# (3), v, p' and theta, and reads and writes T; the z pass reads q (5), w,
# p' and theta, T (5), S and -- in stages 2 and 3 -- q^n (5), and writes the
# stage output (5).  The FP32 plane pass (x and y fused) reads q and writes
# W (3) and T; its z pass reads w and p' (no theta).
_Z_VALUES = 5 + 3 + 5 + 1 + 5 * 2 / 3 + 5
KERNEL_VALUES_PER_NODE = {"k_line_x": 14, "k_line_y": 16, "k_line_z": _Z_VALUES,
                          # the mixed path's y pass also writes, and its z pass reads, the rows of
                          # the y faces (5 values at one plane in N = 4, the bench order)
                          "k_df_line_x": 14, "k_df_tline_y": 16 + 5 / 4, "k_df_tline_z": _Z_VALUES + 5 / 4,
                          "k_f_plane_xy": 13, "k_f_plane_xy_tc": 13, "k_f_plane_xy_h16": 13,
                          "k_f_tline": _Z_VALUES - 1, "k_f_column": 5 + 1 + 5 * 2 / 3 + 5}
# The method's own traffic per node and stage: q and S in,
# q out, plus q^n in stages 2 and 3.
STAGE_BYTES_PER_NODE = (88 + 128 + 128) / 3.0


def timed_steps(xg, torch, ctx, dt, K, Wm, stream, world, local, sample_clocks):
    """W warm-up steps, then K steps timed with CUDA events on `stream`
    (barrier and synchronize on both sides), with per-kernel event times."""
    xg.xg_step(ctx, dt, Wm, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    xg.xg_profile(ctx, 1)
    xg.xg_kernel_times(ctx, reset=True)
    clocks = ClockSampler(local) if sample_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xg.xg_step(ctx, dt, K, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if clocks else None
    xg.xg_profile(ctx, 0)
    kms, klaunch = xg.xg_kernel_times(ctx, reset=True)
    return reduce_max(e0.elapsed_time(e1), world), kms, klaunch, clk


def run_xg(args, world, rank, local):
    import torch
    from paper_2504_08157_gb300 import build, xg
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    wl = workload(args.workload, args.nel)
    cfg = describe(wl)
    prec = {"fp64": xg.XG_FP64, "df64": xg.XG_DF64, "fp32": xg.XG_FP32}[args.precision]
    stream = torch.cuda.current_stream(dev)
    dt = wl["dt"]
    K, Wm = args.steps, args.warmup
    dof_u, dof_p = cfg["dof_unique"], cfg["dof_paper"]
    gdof = lambda ms, k: dof_u * 3 * k * world / (ms / 1e3) / 1e9

    ctx = make_ctx(xg, torch, wl, dev, prec)
    knames = KERNEL_NAMES[prec]
    if prec == xg.XG_FP32:
        contract = CONTRACTIONS[args.contraction][0](xg) if args.contraction != "fma" else 0
        if contract:
            xg.xg_set_contraction(ctx, contract)
        if args.fused:
            xg.xg_set_fused(ctx, 1)
        knames = fp32_kernel_names(wl, contract, args.fused)
    ms_max, kms, klaunch, clk = timed_steps(xg, torch, ctx, dt, K, Wm, stream, world, local, True)
    value = gdof(ms_max, K)

    # roofline: the method's algorithmic bytes per unique node and RK stage
    # (q and S in, the stage output out, plus q^n in stages 2 and 3: 114.7 B
    # with 8-byte values, 57.3 B with 4-byte values) over the measured stage
    # time, against the measured copy bandwidth; the stage's kernels (x, y, z
    # passes) run back to back, so the stage is the launch sequence the
    # figure belongs to.  kernel_frac: the dominant kernel's own compulsory
    # bytes (its inputs and outputs, intermediates included) over its time.
    k = int(np.argmax(kms))
    name = KERNELS[k]
    kname = knames[k]
    avg_ms = kms[k] / max(klaunch[k], 1)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    per_launch = {knames[i]: round(kms[i] / max(klaunch[i], 1), 4) for i in range(3) if klaunch[i]}
    vb = 4 if prec == xg.XG_FP32 else 8            # bytes per stored value
    stage_s = ms_max / 1e3 / (3 * K)
    stage_bytes = cfg["nodes"] * STAGE_BYTES_PER_NODE * vb / 8
    achieved = stage_bytes / stage_s / 1e9
    traffic = stage_traffic([n for n in knames if n != "-"])
    kbytes = KERNEL_VALUES_PER_NODE[kname] * vb * cfg["nodes"]
    kach = kbytes / (avg_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4),
            "traffic": traffic, "traffic_ratio": (round(traffic / stage_bytes, 3) if traffic else None),
            "scope": "one RK stage (every kernel of the pass); algorithmic bytes "
                     "%.1f B per unique node x %d nodes" % (STAGE_BYTES_PER_NODE * vb / 8, cfg["nodes"]),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy), of measured",
            "stage_ms": round(stage_s * 1e3, 4),
            "dominant_kernel": kname, "share": round(kms[k] / max(sum(kms), 1e-30), 4),
            "kernel_frac": round(kach / hbm, 4),
            "kernel_bytes_per_node": round(KERNEL_VALUES_PER_NODE[kname] * vb, 2),
            "kernel_ms_per_launch": per_launch}
    if prec == xg.XG_FP64:
        flops = flops_per_node(name, wl["N"]) * cfg["nodes"]
        fach = flops / (avg_ms / 1e3) / 1e12
        roof["alu"] = {"kernel": kname, "achieved": round(fach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                       "unit": "TFLOP/s", "frac": round(fach / FP64_PEAK_TFLOPS, 4),
                       "peak_source": "FP64 derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    if prec == xg.XG_DF64 and wl["N"] == 4:
        # the pipe that binds this path: FP64 instructions over the stage and per kernel
        inst = sum(DF64_FP64_INSTR_PER_NODE.values()) * cfg["nodes"]
        per_k = {n: round(DF64_FP64_INSTR_PER_NODE[n] * cfg["nodes"] / (per_launch[n] / 1e3) / 1e9
                          / FP64_PIPE_PEAK_GINSTR, 4) for n in DF64_FP64_INSTR_PER_NODE if n in per_launch}
        ach_i = inst / stage_s / 1e9
        roof["alu"] = {"pipe": "fp64", "achieved": round(ach_i, 1), "peak": round(FP64_PIPE_PEAK_GINSTR, 1),
                       "unit": "G FP64 instructions/s", "frac": round(ach_i / FP64_PIPE_PEAK_GINSTR, 4),
                       "kernel_frac": per_k,
                       "instructions_per_node_and_stage": round(sum(DF64_FP64_INSTR_PER_NODE.values()), 1),
                       "peak_source": "derived: 152 SMs x 2 FP64 instructions/clk x 2.07 GHz (maximum SM "
                                      "clock); instruction counts from the ncu capture in profiles/"}
    hbm_frac = achieved / hbm

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        np_ = xg.xg_mesh_np(ctx)
        h_in = torch.from_numpy(wl["q"]).pin_memory()
        h_out = torch.empty((5, np_), dtype=torch.float64).pin_memory()
        Ke = max(1, min(K, 10))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(Ke):
            xg.xg_set_state(ctx, h_in, stream=stream.cuda_stream)
            xg.xg_step(ctx, dt, 1, stream=stream.cuda_stream)
            xg.xg_get_state(ctx, h_out, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        te_sync = reduce_max(time.perf_counter() - t0, world)
        barrier(world)
        # the same steps through xg_step_stream: every step still uploads its
        # input and downloads its result, on the context's copy streams,
        # overlapping the neighbouring steps
        xg.xg_step_stream(ctx, [h_in], [h_out], dt, 1, stream=stream.cuda_stream)   # staging set up
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        xg.xg_step_stream(ctx, [h_in] * Ke, [h_out] * Ke, dt, 1, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        te = reduce_max(time.perf_counter() - t0, world)
        barrier(world)
        nbytes = 5 * np_ * 8
        e2e = {"value": round(dof_u * 3 * Ke * world / te / 1e9, 4), "unit": "GDOF/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": Ke,
               "api": "xg_step_stream (one host state in and out per step, copies overlapping the "
                      "neighbouring steps)",
               "sequential_calls": {"value": round(dof_u * 3 * Ke * world / te_sync / 1e9, 4),
                                    "api": "xg_set_state + xg_step + xg_get_state per step"}}
    xg.xg_destroy(ctx)

    # the other precisions on the same workload and GPU: plain FP64 (the
    # comparison the metric asks for) and the FP32 precision form
    def side_run(p, dtype, contract=0, fused=False):
        Kp = max(1, min(K, 10))
        c2 = make_ctx(xg, torch, wl, dev, p)
        if contract:
            xg.xg_set_contraction(c2, contract)
        if p == xg.XG_FP32 and fused:
            xg.xg_set_fused(c2, 1)
        names = fp32_kernel_names(wl, contract, fused) if p == xg.XG_FP32 else KERNEL_NAMES[p]
        msp, kmsp, klp, _ = timed_steps(xg, torch, c2, dt, Kp, 3, stream, world, local, False)
        xg.xg_destroy(c2)
        return {"value": round(gdof(msp, Kp), 4), "unit": "GDOF/s", "dtype": dtype,
                "ms_per_step": round(msp / Kp, 4), "steps": Kp,
                "kernel_ms_per_launch": {names[i]: round(kmsp[i] / max(klp[i], 1), 4)
                                         for i in range(3) if klp[i]}}
    plain = side_run(xg.XG_FP64, "f64") if prec != xg.XG_FP64 and not args.no_plain else None
    fp32 = side_run(xg.XG_FP32, "f32") if prec != xg.XG_FP32 and not args.no_plain else None
    if fp32 is not None and wl["N"] == 4:
        # the same form with the x and y contractions on the tensor cores
        fp32["fused_column_pass"] = side_run(xg.XG_FP32, "f32", 0, True)
        fp32["tf32x3_contraction"] = side_run(xg.XG_FP32, "f32", xg.XG_CONTRACT_TF32X3)
        fp32["f16x3_contraction"] = side_run(xg.XG_FP32, "f32", xg.XG_CONTRACT_F16X3)
    batched = None
    if not args.no_plain and not args.no_batch:
        batched = batch_measure(xg, torch, dev, stream, world, local, max(1, min(K, 10)), 3,
                                False, compare=True, oracle_check=rank == 0)
        batched.pop("clocks", None)
    closure_rate = None
    dyn = None
    if not args.no_plain and not args.no_batch:
        closure_rate = closure_throughput(xg, torch, dev, stream, max(1, min(K, 10)), 3)
        dyn = dynamics_measure(xg, torch, dev, stream)

    cpu, l2 = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sw = cpu_sample_workload(args.workload)
        g, steps, secs, _, workers = time_oracle(sw)
        ref = oracle_rhs(sw)
        got = {p: gpu_rhs(sw, xg, torch, dev, v)
               for p, v in (("df64", xg.XG_DF64), ("fp64", xg.XG_FP64), ("fp32", xg.XG_FP32))}
        if sw["N"] == 4:
            got["fp32_tf32x3_contraction"] = gpu_rhs(sw, xg, torch, dev, xg.XG_FP32,
                                                     xg.XG_CONTRACT_TF32X3)
            got["fp32_f16x3_contraction"] = gpu_rhs(sw, xg, torch, dev, xg.XG_FP32,
                                                    xg.XG_CONTRACT_F16X3)
        # the extended-precision oracle at sampled nodes of the sample
        n_all = got["fp64"].shape[1]
        nodes = np.unique(np.concatenate([np.arange(0, n_all, 331),
                                          np.random.default_rng(16).integers(0, n_all, 400)]))
        refx = oracle_rhs_extended_at(sw, nodes)
        ref32 = oracle_rhs(sw, q=sw["q"].astype(np.float32).astype(np.float64))
        l2 = {p: rel_err(v, ref) for p, v in got.items()}
        l2["vs_extended_oracle"] = {p: rel_err(got[p][:, nodes], refx) for p in ("fp64", "df64")}
        l2["fp64_oracle_vs_extended_oracle"] = rel_err(ref[:, nodes], refx)
        l2["meets_1e-12"] = {p: bool(max(l2["vs_extended_oracle"][p]) <= 1e-12 and max(l2[p]) <= 1e-12)
                             for p in ("fp64", "df64")}
        l2["fp32_vs_oracle_of_fp32_rounded_state"] = {
            p: rel_err(got[p], ref32) for p in ("fp32", "fp32_tf32x3_contraction", "fp32_f16x3_contraction")
            if p in got}
        l2["fp32_state_rounding_floor"] = rel_err(ref32, ref)
        # the same sample at a seeded smooth random state plus the vortex, where no
        # tendency is a cancellation residual
        l2["random_state"] = random_state_errors(args.workload, xg, torch, dev)
        # the timed workload itself at sampled nodes
        l2["full_size_timed_state"] = full_size_errors(wl, xg, torch, dev)
        l2["what"] = ("relative L2 difference of one GPU right-hand side from the FP64 oracle on "
                      "the CPU sample at the timed (vortex) state, per variable (rho', rho u, "
                      "rho v, rho w, Theta'); vs_extended_oracle: against the same oracle in "
                      "extended precision at %d sampled nodes (at this state the rho' and "
                      "Theta' tendencies are residuals of cancelling flux derivatives, and the "
                      "FP64 oracle's own rounding is fp64_oracle_vs_extended_oracle); "
                      "fp32_state_rounding_floor: what rounding the state to FP32 alone "
                      "changes in the oracle's RHS" % nodes.size)
        cpu = {"value": round(g, 6), "unit": "GDOF/s", "cores": workers, "nproc": os.cpu_count(),
               "kind": "oracle",
               "sample": "%s %dx%dx%d N=%d, %d SSP-RK3 steps in %.1f s (numpy, %d worker "
                         "processes over element chunks, 1 thread each)"
                         % (sw["name"], *sw["nel"], sw["N"], steps, secs, workers)}

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world,
               "steps": K, "warmup": Wm, "ms_per_step": round(ms_max / K, 4),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": {xg.XG_FP64: "f64", xg.XG_DF64: "f64+f32x2", xg.XG_FP32: "f32"}[prec],
               "precision": args.precision,
               "contraction": args.contraction if prec == xg.XG_FP32 else None,
               "data": "synthetic", "impl": "xg",
               "config": cfg,
               "gdof_paper_convention": round(dof_p * 3 * K * world / (ms_max / 1e3) / 1e9, 4),
               "plain_fp64": plain,
               "speedup_vs_plain_fp64": round(value / plain["value"], 3) if plain else None,
               "fp32_form": fp32,
               "fp32_speedup_vs_plain_fp64": (round(fp32["value"] / plain["value"], 3)
                                              if fp32 and plain else None),
               "batched_form": batched,
               "closure_form": closure_rate,
               "paper_dynamics": dyn,
               "l2_error_vs_oracle": l2,
               "hbm_roofline_frac": round(hbm_frac, 4),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": int(sum(klaunch))}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ batched persistent form

BATCH_BYTES_PER_NODE = 4 * (5 + 3 + 5) + 4 * (5 + 2 + 5 + 1 + 5 * 2 / 3 + 5)   # plane + z passes, FP32


def batch_workloads(count=96):
    from inputs import workloads as W
    return [W.batch_instance(s) for s in W.batch_specs()[:count]]


def make_batch(xg, torch, wls, dev):
    descs = []
    for wl in wls:
        ph = wl["phys"]
        descs.append(xg.mesh_desc(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"],
                                  f=ph["f"], g=ph["g"], R=ph["R"], cp=ph["cp"], cv=ph["cv"],
                                  p_a=ph["p_a"], precision=xg.XG_FP32))
    b = xg.xg_batch_create(descs)
    for i, wl in enumerate(wls):
        c = xg.xg_batch_instance(b, i)
        xg.xg_set_state(c, torch.from_numpy(wl["q"]).to(dev), torch.from_numpy(wl["rho0"]).to(dev),
                        torch.from_numpy(wl["Theta0"]).to(dev))
        if wl["S_theta"] is not None:
            xg.xg_set_forcing(c, torch.from_numpy(wl["S_theta"]).to(dev))
    torch.cuda.synchronize()
    return b


def batch_describe(wls):
    from inputs import workloads as W
    dof_u = sum(W.dof_counts(wl["nel"], wl["N"], wl["periodic"])[0] for wl in wls)
    dof_p = sum(W.dof_counts(wl["nel"], wl["N"], wl["periodic"])[1] for wl in wls)
    orders = {str(n): sum(1 for wl in wls if wl["N"] == n) for n in (3, 4, 5, 6)}
    sizes = [W.dof_counts(wl["nel"], wl["N"], wl["periodic"])[0] // 5 for wl in wls]
    return dict(workload="batch of %d limited-area instances, 512x512x20 km, nel 4..24 x 4..24 x "
                         "4..12, N 3..6, FP32 (ppw)" % len(wls),
                instances=len(wls), nodes=dof_u // 5, dof_unique=dof_u, dof_paper=dof_p,
                orders=orders, nodes_min=min(sizes), nodes_max=max(sizes),
                l2="inputs larger than L2 (the batch's FP32 states total %.0f MB > 129 MB L2)"
                   % (dof_u * 4 / 1e6),
                parallelism="replicas")


def batch_measure(xg, torch, dev, stream, world, local, K, Wm, sample_clocks, compare,
                  oracle_check, count=96):
    """The batched form on the 96-instance workload: autotune, then K steps
    in one persistent launch timed with CUDA events; with ``compare`` also
    the same instances stepped through single contexts (FP32, one launch
    sequence per instance) and in plain FP64."""
    wls = batch_workloads(count)
    cfg = batch_describe(wls)
    dts = [wl["dt"] for wl in wls]
    dof_u = cfg["dof_unique"]
    b = make_batch(xg, torch, wls, dev)
    out = {}
    try:
        tune = xg.xg_batch_autotune(b, dts, trial_steps=2, stream=stream.cuda_stream)
        xg.xg_batch_step(b, dts, Wm, stream=stream.cuda_stream)
        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xg.xg_batch_step(b, dts, K, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = reduce_max(e0.elapsed_time(e1), world)
        out["clocks"] = clocks.stop() if clocks else None
        out["value"] = round(dof_u * 3 * K * world / (ms / 1e3) / 1e9, 4)
        out["unit"] = "GDOF/s"
        out["dtype"] = "f32"
        out["ms_per_step"] = round(ms / K, 4)
        out["steps"] = K
        out["launches_per_call"] = 1
        out["tuning"] = tune.as_dict()
        out["config"] = cfg
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        achieved = BATCH_BYTES_PER_NODE * cfg["nodes"] * 3 * K / (ms / 1e3) / 1e9
        out["roofline"] = {"kernel": "k_batch", "bound": "hbm", "achieved": round(achieved, 1),
                           "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                           "traffic": (lambda b: None if b is None else round(b * cfg["nodes"] * 3 * K))(
                               traffic_per_launch("k_batch_per_node_stage")),
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
                           "bytes_per_node_stage": round(BATCH_BYTES_PER_NODE, 2),
                           "launch": "one persistent launch of %d steps (%d stages)" % (K, 3 * K)}
        if oracle_check:
            # one right-hand side of the whole batch, with the smallest
            # instance set to a seeded smooth random state (at the vortex
            # state several tendencies are cancellation residuals or exactly
            # zero), against the FP64 oracle
            from inputs import workloads as W
            from oracle import euler as E, mesh as M
            outs = [torch.empty((5, xg.xg_mesh_np(xg.xg_batch_instance(b, i))), dtype=torch.float64,
                                device=dev) for i in range(len(wls))]
            i = int(np.argmin([o.shape[1] for o in outs]))
            wl = W.batch_instance(W.batch_specs()[i], state="random", seed=i + 1)
            xg.xg_set_state(xg.xg_batch_instance(b, i), torch.from_numpy(wl["q"]).to(dev),
                            stream=stream.cuda_stream)
            xg.xg_batch_rhs(b, outs, stream=stream.cuda_stream)
            m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
            ref = E.rhs(m, wl["q"], E.Base(wl["rho0"], wl["Theta0"]), wl["S_theta"],
                        E.Physics(**wl["phys"]))
            got = outs[i].cpu().numpy()
            del outs
            out["l2_error_vs_oracle"] = {
                "instance": i, "nel": list(wl["nel"]), "N": wl["N"],
                "rel_l2": [float("%.3e" % (np.linalg.norm(got[v] - ref[v]) /
                                           max(np.linalg.norm(ref[v]), 1e-300))) for v in range(5)],
                "what": "one batched right-hand side (all 96 instances in one launch) of the "
                        "smallest instance, at a seeded smooth random state plus its vortex, vs "
                        "the FP64 oracle, relative L2 per variable"}
    finally:
        xg.xg_batch_destroy(b)
    if compare:
        def sequential(p, Kp):
            ctxs = [make_ctx(xg, torch, wl, dev, p) for wl in wls]
            try:
                for c, wl in zip(ctxs, wls):
                    xg.xg_step(c, wl["dt"], 1, stream=stream.cuda_stream)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for c, wl in zip(ctxs, wls):
                    xg.xg_step(c, wl["dt"], Kp, stream=stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                msq = e0.elapsed_time(e1)
            finally:
                for c in ctxs:
                    xg.xg_destroy(c)
            return {"value": round(dof_u * 3 * Kp / (msq / 1e3) / 1e9, 4), "unit": "GDOF/s",
                    "ms_per_step": round(msq / Kp, 4), "steps": Kp}
        out["per_instance_fp32"] = sequential(xg.XG_FP32, K)
        out["per_instance_fp32"]["what"] = ("the same instances through single XG_FP32 contexts, "
                                            "one xg_step call per instance")
        out["plain_fp64"] = sequential(xg.XG_FP64, max(1, K // 2))
        out["plain_fp64"]["what"] = "the same instances in native FP64, one context per instance"
        out["speedup_vs_plain_fp64"] = round(out["value"] / out["plain_fp64"]["value"], 3)
        out["speedup_vs_per_instance_fp32"] = round(out["value"] / out["per_instance_fp32"]["value"], 3)
    return out


def run_batch(args, world, rank, local):
    import torch
    from paper_2504_08157_gb300 import build, xg
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    stream = torch.cuda.current_stream(dev)
    K, Wm = args.steps, args.warmup
    res = batch_measure(xg, torch, dev, stream, world, local, K, Wm, True,
                        compare=not args.no_plain, oracle_check=rank == 0 and world == 1,
                        count=args.instances)
    cfg = res.pop("config")
    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI: every instance's state from pinned
        # host memory, one batched step, every state back to pinned memory
        wls = batch_workloads(args.instances)
        dts = [wl["dt"] for wl in wls]
        b = make_batch(xg, torch, wls, dev)
        try:
            hin = [torch.from_numpy(wl["q"]).pin_memory() for wl in wls]
            hout = [torch.empty_like(h).pin_memory() for h in hin]
            Ke = max(1, min(K, 5))
            xg.xg_batch_step(b, dts, 1, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(Ke):
                for i, h in enumerate(hin):
                    xg.xg_set_state(xg.xg_batch_instance(b, i), h, stream=stream.cuda_stream)
                xg.xg_batch_step(b, dts, 1, stream=stream.cuda_stream)
                for i, h in enumerate(hout):
                    xg.xg_get_state(xg.xg_batch_instance(b, i), h, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            te = reduce_max(time.perf_counter() - t0, world)
            nbytes = sum(h.numel() * 8 for h in hin)
            e2e = {"value": round(cfg["dof_unique"] * 3 * Ke * world / te / 1e9, 4), "unit": "GDOF/s",
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": Ke}
        finally:
            xg.xg_batch_destroy(b)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sw = cpu_sample_workload("batch")
        g, steps, secs, _, workers = time_oracle(sw)
        cpu = {"value": round(g, 6), "unit": "GDOF/s", "cores": workers, "nproc": os.cpu_count(),
               "kind": "oracle",
               "sample": "batch instance %dx%dx%d N=%d, %d SSP-RK3 steps in %.1f s (numpy, %d "
                         "worker processes over element chunks)"
                         % (*sw["nel"], sw["N"], steps, secs, workers)}
    if rank == 0:
        roof = res.pop("roofline")
        clk = res.pop("clocks")
        out = {"metric": METRIC, "value": res.pop("value"), "unit": "GDOF/s", "n_gpus": world,
               "steps": K, "warmup": Wm, "ms_per_step": res.pop("ms_per_step"),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "precision": "fp32", "data": "synthetic", "impl": "xg", "config": cfg,
               "gdof_paper_convention": None, **res, "roofline": roof, "cpu_baseline": cpu,
               "e2e": e2e, "clocks": clk, "gpu_launches": 1}
        out["gdof_paper_convention"] = round(out["value"] * cfg["dof_paper"] / cfg["dof_unique"], 4)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ the paper's remaining dynamics

def dynamics_measure(xg, torch, dev, stream, K=5):
    """FP64 on the cyclone box: explicit SSP-RK3 at dt = 0.1 s against IMEX
    ARK2 (matrix-free GMRES) at the paper's dt = 0.5 s, with and without
    hyper-diffusion (c = 1e-4 on the three axes) and a 4 km top sponge
    (gamma_max = 0.05 1/s); the same pair in the mixed XG_DF64 context
    (without hyper-diffusion, which is FP64 only); simulated seconds per
    wall-clock second; and the RI-velocity diagnostic's cost."""
    wl = workload("tc")
    out = {}

    def timed(run, ctx):
        run(ctx, 1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = run(ctx, K)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K, res

    ctx = make_ctx(xg, torch, wl, dev, xg.XG_FP64)
    try:
        ms, _ = timed(lambda c, n: xg.xg_step(c, 0.1, n, stream=stream.cuda_stream), ctx)
        out["explicit_fp64"] = {"dt": 0.1, "ms_per_step": round(ms, 3),
                                "simulated_s_per_s": round(0.1 / (ms / 1e3), 2)}
        for name, dyn in (("imex_fp64", None), ("imex_fp64_hyperdiffusion_sponge", True)):
            if dyn:
                xg.xg_set_dynamics(ctx, (1e-4, 1e-4, 1e-4), 0.5, 4000.0, 0.05)
            ms, st = timed(lambda c, n: xg.xg_step_imex(c, 0.5, n, tol=1e-8, stream=stream.cuda_stream), ctx)
            out[name] = {"dt": 0.5, "ms_per_step": round(ms, 3),
                         "simulated_s_per_s": round(0.5 / (ms / 1e3), 2),
                         "gmres": st.as_dict(), "tol": 1e-8}
        xg.xg_set_dynamics(ctx, off=True)
        t0 = time.perf_counter()
        u, _, _ = xg.xg_ri_velocity(ctx, 50)
        out["ri_velocity"] = {"value_m_per_s": round(u, 3), "ms": round(1e3 * (time.perf_counter() - t0), 2),
                              "strips": 50}
    finally:
        xg.xg_destroy(ctx)
    # the mixed context: its SSP-RK3 step against IMEX whose explicit part is
    # the mixed stage (L, GMRES and the combinations FP64 as above)
    ctx = make_ctx(xg, torch, wl, dev, xg.XG_DF64)
    try:
        ms, _ = timed(lambda c, n: xg.xg_step(c, 0.1, n, stream=stream.cuda_stream), ctx)
        out["explicit_df64"] = {"dt": 0.1, "ms_per_step": round(ms, 3),
                                "simulated_s_per_s": round(0.1 / (ms / 1e3), 2)}
        ms, st = timed(lambda c, n: xg.xg_step_imex(c, 0.5, n, tol=1e-8, stream=stream.cuda_stream), ctx)
        out["imex_df64"] = {"dt": 0.5, "ms_per_step": round(ms, 3),
                            "simulated_s_per_s": round(0.5 / (ms / 1e3), 2),
                            "gmres": st.as_dict(), "tol": 1e-8}
    finally:
        xg.xg_destroy(ctx)
    out["config"] = "tc 128x128x16 N=4 FP64 (and the mixed XG_DF64 context)"
    out["speedup_imex_vs_explicit"] = round(out["imex_fp64"]["simulated_s_per_s"] /
                                            out["explicit_fp64"]["simulated_s_per_s"], 3)
    out["speedup_imex_vs_explicit_df64"] = round(out["imex_df64"]["simulated_s_per_s"] /
                                                 out["explicit_df64"]["simulated_s_per_s"], 3)

    # the paper's own timing workload (Table 1): 80 x 80 x 24 elements of order 5 on the
    # 800 x 800 x 20 km box, IMEX ARK2 at dt = 0.5 s with hyper-diffusion and the 4 km sponge
    from inputs import workloads as W
    wp = W.tc_paper()
    ctx = make_ctx(xg, torch, wp, dev, xg.XG_FP64)
    try:
        xg.xg_set_dynamics(ctx, (1e-4, 1e-4, 1e-4), 0.5, 4000.0, 0.05)
        ms, st = timed(lambda c, n: xg.xg_step_imex(c, 0.5, n, tol=1e-8, stream=stream.cuda_stream), ctx)
        dof_u, dof_p = W.dof_counts(wp["nel"], wp["N"], wp["periodic"])
        out["paper_table1_workload"] = {
            "config": "tc_paper 80x80x24 N=5, 800x800x20 km, FP64, IMEX ARK2 dt=0.5 s, "
                      "hyper-diffusion + 4 km sponge, GMRES tol 1e-8",
            "dof_paper": dof_p, "dof_unique": dof_u, "ms_per_step": round(ms, 3),
            "gmres": st.as_dict(), "steps": K,
            "paper": {"ms_per_step": 536.0, "hardware": "4x NVIDIA A100 (one node), FP64, OpenACC; "
                      "mean over 100 steps; GMRES tolerance not stated",
                      "cpu_ms_per_step": 5563.0, "cpu_hardware": "128 cores AMD EPYC 7763"},
            "what": "context, not the target: same grid, order, domain, dt and integrator as the "
                    "paper's Table 1; the sounding, vortex and heating are this build's synthetic "
                    "recipe, so the GMRES work per step may differ"}
    finally:
        xg.xg_destroy(ctx)
    return out


# ------------------------------------------------------------------ learned-closure form

def closure_throughput(xg, torch, dev, stream, K, Wm, nel=(64, 64, 16)):
    """The closure form's step rate on the config-5 coarse mesh (FP32 with
    the bfloat16 tensor-core closure in every stage; a seeded untrained
    network: the rate does not depend on the weights) against plain FP64 on
    the same mesh."""
    from inputs import workloads as W
    from paper_2504_08157_gb300 import closure as CL
    wl = W.closure_case(1, nel=nel)
    dof_u, _ = W.dof_counts(wl["nel"], wl["N"], wl["periodic"])
    out = {}
    for name, prec, with_closure in (("closure_fp32", xg.XG_FP32, True), ("plain_fp32", xg.XG_FP32, False),
                                     ("plain_fp64", xg.XG_FP64, False)):
        ctx = make_ctx(xg, torch, wl, dev, prec)
        if with_closure:
            p = CL.init_params(3, dev)
            one = torch.ones(21, dtype=torch.float32, device=dev)
            xg.xg_closure_set(ctx, p, torch.zeros_like(one), one, one[:5] * 1e-6)
        xg.xg_step(ctx, wl["dt"], Wm, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xg.xg_step(ctx, wl["dt"], K, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        xg.xg_destroy(ctx)
        out[name] = {"value": round(dof_u * 3 * K / (ms / 1e3) / 1e9, 4), "unit": "GDOF/s",
                     "ms_per_step": round(ms / K, 4), "steps": K}
    out["config"] = "closure coarse mesh %dx%dx%d N=4 (10 km cube, walls), %d nodes" % (*nel, dof_u // 5)
    out["speedup_vs_plain_fp64"] = round(out["closure_fp32"]["value"] / out["plain_fp64"]["value"], 3)
    return out


def run_closure(args, world, rank, local):
    """Config 5: train the closure on refined-minus-coarse tendency
    differences of paired runs (coarse 64 x 64 x 16, refined 128 x 128 x 32
    elements, 8 seeded runs, 2e6 samples) with the library's kernels, then
    judge it against the refined run; and the closure form's step rate."""
    import torch
    from inputs import workloads as W
    from paper_2504_08157_gb300 import build, closure as CL, xg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    stream = torch.cuda.current_stream(dev)
    K, Wm = args.steps, args.warmup
    nel = tuple(args.nel) if args.nel else (64, 64, 16)
    if args.rate_only:
        rate = closure_throughput(xg, torch, dev, stream, K, Wm, nel)
        if rank == 0:
            print(json.dumps({"workload": "closure", "closure_form": rate}))
        return
    t0 = time.perf_counter()
    nseeds, snaps = 8, 4
    per_snap = args.samples // (nseeds * snaps)
    X, T = CL.sample_pairs(W.closure_case, seeds=list(range(1, nseeds + 1)), coarse_nel=nel,
                           snapshots=snaps, steps_between=20, samples=per_snap, dev=dev)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = CL.train(X, T, dev, epochs=args.epochs, batch=16384, lr=2e-3, holdout=1.0 / nseeds)
    t_train = time.perf_counter() - t0
    # the plain right-hand side as fallback: the output gain (0 = plain) chosen on a validation
    # run, then the test run judged at gains 0 (plain), 1 (the trained network) and the chosen
    # candidates: the trained network and the same with its mean correction removed
    cands = {"trained": model, "centered": CL.centered(model, X, dev)}
    picks = {k: CL.select_gain(W.closure_case, 101, nel, m, args.eval_steps, dev) for k, m in cands.items()}
    score = lambda e, p: sum(a / max(b, 1e-300) for a, b in zip(e, p)) / 5
    best = min(picks, key=lambda k: score(picks[k][1][picks[k][0]], picks[k][1][0.0]))
    gain = picks[best][0]
    ev = CL.evaluate_gains(W.closure_case, 100, nel, cands[best], args.eval_steps, dev,
                           tuple(sorted({0.0, 1.0, gain})))
    # the target itself as the correction (no network): exact, and low-pass filtered
    study = CL.correction_study(W.closure_case, 101, nel, args.eval_steps, dev)
    vs_refined = {"plain": ev[0.0], "closure": ev[1.0], "closure_at_chosen_gain": ev[gain],
                  "exact_target_as_correction": study,
                  "chosen_gain": gain, "chosen_model": best,
                  "gain_selection": {"validation_run_seed": 101,
                                     "errors": {k: {repr(g): e for g, e in picks[k][1].items()}
                                                for k in picks}},
                  "what": "relative L2 distance of each coarse run's state from the restricted "
                          "refined state after %d coarse steps, per variable, relative to the "
                          "refined run's change (test run seed 100); gain g scales the closure's "
                          "output, g = 0 is the plain coarse run" % args.eval_steps}
    rate = closure_throughput(xg, torch, dev, stream, K, Wm, nel)
    if rank == 0:
        dof_u, dof_p = W.dof_counts(nel, 4, (False, False, False))
        cfg = {"workload": "closure form: coarse %dx%dx%d N=4 FP32 + 21-64-64-5 bf16 closure, 10 km "
                           "cube (walls), refined %dx%dx%d" % (*nel, *(2 * n for n in nel)),
               "nodes": dof_u // 5, "dof_unique": dof_u, "dof_paper": dof_p,
               "training_samples": int(X.shape[1]), "runs": nseeds, "snapshots_per_run": snaps,
               "parallelism": "replicas"}
        out = {"metric": METRIC, "value": rate["closure_fp32"]["value"], "unit": "GDOF/s",
               "n_gpus": world, "steps": K, "warmup": Wm,
               "ms_per_step": rate["closure_fp32"]["ms_per_step"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
               "impl": "xg", "config": cfg, "closure_form": rate,
               "training": {"seconds_data": round(t_data, 2), "seconds_train": round(t_train, 2),
                            "epochs": args.epochs,
                            "holdout_loss_zero_correction": round(model["holdout_zero"], 5),
                            "holdout_loss_trained": round(model["holdout"], 5),
                            "history": [[h[0], round(h[1], 5), round(h[2], 5)] for h in model["history"]],
                            "what": "normalised mean-squared tendency error on the held-out run's "
                                    "samples, without and with the closure"},
               "vs_refined_run": vs_refined, "gpu_launches": None, "roofline": None, "cpu_baseline": None,
               "e2e": None}
        print(json.dumps(out))


def run_paper_imex(args, world, rank, local):
    """The paper's timing workload alone (Table 1: 80 x 80 x 24 elements of
    order 5, IMEX ARK2 at dt = 0.5 s with hyper-diffusion and the sponge, FP64):
    ms per step over K steps after W warm-up steps, with the GMRES counts."""
    import torch
    from inputs import workloads as W
    from paper_2504_08157_gb300 import build, xg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    stream = torch.cuda.current_stream(dev)
    wp = W.tc_paper()
    ctx = make_ctx(xg, torch, wp, dev, xg.XG_FP64)
    try:
        xg.xg_set_dynamics(ctx, (1e-4, 1e-4, 1e-4), 0.5, 4000.0, 0.05)
        xg.xg_step_imex(ctx, 0.5, args.warmup, tol=1e-8, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = xg.xg_step_imex(ctx, 0.5, args.steps, tol=1e-8, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    finally:
        xg.xg_destroy(ctx)
    if rank == 0:
        dof_u, dof_p = W.dof_counts(wp["nel"], wp["N"], wp["periodic"])
        print(json.dumps({"workload": "paper_imex", "ms_per_step": round(ms, 3), "steps": args.steps,
                          "warmup": args.warmup, "gmres": st.as_dict(), "dof_paper": dof_p,
                          "config": "tc_paper 80x80x24 N=5, FP64, IMEX ARK2 dt=0.5 s, hyper-diffusion "
                                    "+ 4 km sponge, GMRES tol 1e-8",
                          "paper_ms_per_step": 536.0}))


def run_reference(args, world, rank, local):
    """The FP64 oracle on the host cores, one bounded sample per step."""
    if rank != 0:
        return
    sw = cpu_sample_workload(args.workload)
    wl_full = workload_desc_only(args.workload)
    K, Wm = args.steps, args.warmup
    per_step = []
    team = OracleTeam(sw)
    try:
        q = sw["q"]
        for i in range(Wm + K):
            _, _, secs, q, workers = time_oracle(dict(sw, q=q), min_seconds=0.0, max_steps=1,
                                                 team=team)
            if i >= Wm:
                per_step.append(secs)
    finally:
        team.close()
    total = sum(per_step)
    from inputs import workloads as W
    dof_u, _ = W.dof_counts(sw["nel"], sw["N"], sw["periodic"])
    value = dof_u * 3 * K / total / 1e9
    sample = ("%s %dx%dx%d N=%d, one SSP-RK3 step per bench step (numpy, %d worker processes "
              "over element chunks, 1 thread each)" % (sw["name"], *sw["nel"], sw["N"], workers))
    out = {"metric": METRIC, "value": round(value, 6), "unit": "GDOF/s", "n_gpus": world,
           "steps": K, "warmup": Wm, "ms_per_step": round(1e3 * total / K, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference", "config": wl_full,
           "cpu_baseline": {"value": round(value, 6), "unit": "GDOF/s", "cores": workers,
                            "nproc": os.cpu_count(), "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def workload_desc_only(name):
    from inputs import workloads as W
    if name == "batch":
        specs = W.batch_specs()
        dof = [W.dof_counts(sp["nel"], sp["N"], (True, True, False)) for sp in specs]
        return dict(workload="batch of %d limited-area instances, 512x512x20 km, nel 4..24 x "
                             "4..24 x 4..12, N 3..6, FP32 (ppw)" % len(specs),
                    instances=len(specs), nodes=sum(d[0] for d in dof) // 5,
                    dof_unique=sum(d[0] for d in dof), dof_paper=sum(d[1] for d in dof),
                    parallelism="replicas")
    if name == "tc":
        nel, N, per, dt = (128, 128, 16), 4, (True, True, False), 0.1
        label = "tc"
    else:
        nel, N, per, dt = (8, 8, 8), 4, (False, False, False), 0.02
        label = "bubble"
    dof_u, dof_p = W.dof_counts(nel, N, per)
    pstr = "".join("p" if p else "w" for p in per)
    return dict(workload="%s %dx%dx%d N=%d FP64 (%s)" % (label, *nel, N, pstr), nel=list(nel),
                N=N, nodes=dof_u // 5, dof_unique=dof_u, dof_paper=dof_p, dt=dt,
                periodic=list(per), parallelism="replicas")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["xg", "reference"], default="xg")
    ap.add_argument("--workload", choices=["tc", "bubble", "batch", "closure", "paper_imex"], default="tc")
    ap.add_argument("--samples", type=int, default=2000000,
                    help="closure workload: training samples")
    ap.add_argument("--epochs", type=int, default=20, help="closure workload: training epochs")
    ap.add_argument("--rate-only", action="store_true",
                    help="closure workload: only the step rates (no training or evaluation)")
    ap.add_argument("--eval-steps", type=int, default=500,
                    help="closure workload: coarse steps of the runs compared with the refined run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "df64", "fp32"], default="df64",
                    help="df64: the FP64-accurate mixed FP64 / double-float path (default); "
                         "fp64: native FP64; fp32: the FP32 precision form")
    ap.add_argument("--contraction", choices=["fma", "tf32x3", "f16x3"], default="fma",
                    help="with --precision fp32: x and y contractions on the CUDA cores (fma) or "
                         "on the tensor cores (tf32x3: TF32 head/tail split; f16x3: half-precision "
                         "head/tail split with a scale per segment; order 4)")
    ap.add_argument("--fused", action="store_true",
                    help="with --precision fp32: the fused column pass (one kernel per stage, TMA "
                         "staging) instead of the plane + z-line kernels")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain-FP64 and FP32-form comparison runs")
    ap.add_argument("--instances", type=int, default=96,
                    help="instances of the batched workload (the first ones of the seeded list)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-form comparison in the cyclone line")
    ap.add_argument("--nel", type=int, nargs=3, default=None,
                    help="element counts of a smaller cyclone box (same spacing), for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    elif args.workload == "batch":
        run_batch(args, world, rank, local)
    elif args.workload == "closure":
        run_closure(args, world, rank, local)
    elif args.workload == "paper_imex":
        run_paper_imex(args, world, rank, local)
    else:
        run_xg(args, world, rank, local)


if __name__ == "__main__":
    main()
