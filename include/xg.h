/*
 * xg.h -- C ABI of the GB300 (sm_103a) explicit CG Euler path after
 * Kang, Giraldo & Camp, "A GPU-accelerated simulation of rapid
 * intensification of a tropical cyclone with observed heating"
 * (arXiv 2504.08157).
 *
 * The library evaluates, on one GPU, the explicit right-hand side of the
 * compressible Euler equations for perturbations about a hydrostatic
 * reference state (Sec. 2.1, Eq. 1, with the equation of state Eq. 3),
 * written for q = (rho', rho u, rho v, rho w, Theta'), Theta = rho theta,
 * with f-plane Coriolis and a prescribed heating S_theta, on a hexahedral
 * continuous-Galerkin mesh of tensor-product LGL nodes (Sec. 2.2, Eqs. 4-8);
 * assembles it by direct stiffness summation (Eqs. 9-11, Alg. 3), applies
 * the inverse diagonal mass matrix (Eq. 12) and no-flux walls, and advances
 * the state with three-stage SSP Runge-Kutta stages fused into the same
 * kernels.
 *
 * Mesh: an axis-aligned box [lo, hi] split into nel[0] x nel[1] x nel[2]
 * equal hexahedra of order N = order.  Direction d has n_d = N nel_d global
 * nodes when periodic and N nel_d + 1 when bounded by no-flux walls.
 *
 * Data layout (all arrays FP64, row-major, no padding):
 *   state q      [5][Np]  structure of arrays; variable v = 0 rho' (kg m^-3),
 *                         1..3 rho u, rho v, rho w (kg m^-2 s^-1),
 *                         4 Theta' = (rho theta)' (K kg m^-3);
 *                         node I = gx + n_x (gy + n_y gz), x fastest.
 *   reference    rho0[n_z], rhotheta0[n_z]: rho_0 and Theta_0 = rho_0 theta_0
 *                on the node levels gz = 0 .. n_z-1 (the reference state
 *                depends on z only, Sec. 2.1); p_0 = p(Theta_0) by Eq. 3.
 *   heating      S_theta[Np] in K s^-1 (a potential-temperature tendency;
 *                the conservative source is rho S_theta).
 *
 * Pointers: every array argument is either host memory (where = XG_HOST) or
 * device memory of the context's GPU (where = XG_DEVICE), e.g. a PyTorch
 * tensor's data_ptr().  The library copies what it is given and never keeps
 * a caller pointer.  `stream` is a cudaStream_t passed as void*; NULL is the
 * legacy default stream.  Work is enqueued on that stream; a call returns
 * before the GPU finishes except where stated.
 *
 * Errors: every call returns an xg_status and never throws.  XG_ERR_ARG and
 * XG_ERR_UNSUPPORTED are detected on the host before any GPU work and leave
 * the context unchanged.  XG_ERR_CUDA is sticky: the context refuses further
 * work (only xg_destroy).  XG_ERR_NONFINITE (xg_step) leaves the context
 * usable with whatever state the GPU computed.
 *
 * Threads: a context may be used by one host thread at a time.
 */
#ifndef XG_H
#define XG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XG_OK = 0,
  XG_ERR_ARG = 1,          /* invalid argument (NULL, out of range, wrong order of calls) */
  XG_ERR_CUDA = 2,         /* a CUDA runtime call failed; sticky */
  XG_ERR_OOM = 3,          /* device allocation failed */
  XG_ERR_NONFINITE = 4,    /* a NaN or Inf appeared in the state */
  XG_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  XG_ERR_UNSUPPORTED = 6   /* valid but not supported by this build */
} xg_status;

enum { XG_HOST = 0, XG_DEVICE = 1 };
enum { XG_FP64 = 0, XG_FP32 = 1, XG_DF64 = 2 };

/* Problem statement (Sec. 2.1-2.2, Sec. 4.1):
 *   nel[3]      elements per direction, >= 1
 *   order       polynomial order N of the LGL basis, 1 <= N <= 8
 *   lo, hi      box corners in metres, hi > lo
 *   periodic    per direction: 1 periodic, 0 no-flux walls
 *   precision   XG_FP64: state and arithmetic in native FP64;
 *               XG_DF64: FP64-accurate "double-float" arithmetic (each value
 *               an unevaluated pair of floats, 48-bit significand) on the
 *               FP32 pipes, with the state kept in that form on the device;
 *               XG_FP32: the precision form -- FP32 state perturbations and
 *               volume arithmetic, with the pressure perturbation of Eq. 3
 *               evaluated FP64-accurately from the FP64 reference state;
 *               in every precision the ABI takes and returns FP64 arrays
 *   f_coriolis  f-plane Coriolis parameter (s^-1)
 *   g, R, cp, cv, p_a   gravity, dry-air gas constant, heat capacities and
 *               reference surface pressure of Eq. 1 and Eq. 3 (SI units) */
typedef struct {
  int nel[3];
  int order;
  double lo[3];
  double hi[3];
  int periodic[3];
  int precision;
  double f_coriolis;
  double g, R, cp, cv, p_a;
} xg_mesh_desc;

typedef struct xg_ctx xg_ctx;

/* Human-readable name of a status code (static string, never NULL). */
const char* xg_status_str(xg_status s);

/* Sec. 2.2: build the mesh on the current CUDA device and allocate every
 * device buffer of the path (owned by the context).  On success *out is a
 * new context; on failure *out is NULL.  Errors: XG_ERR_ARG (NULL, nel < 1,
 * order outside [1, 8], hi <= lo, non-positive constants),
 * XG_ERR_UNSUPPORTED (an unknown precision, or a line of more nodes than one
 * CTA stages in shared memory), XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_mesh_create(const xg_mesh_desc* d, xg_ctx** out);

/* Number of global (unique) nodes Np = n_x n_y n_z. */
xg_status xg_mesh_np(const xg_ctx* ctx, long long* np);

/* Global nodes per direction n[0..2]. */
xg_status xg_mesh_dims(const xg_ctx* ctx, int n[3]);

/* Copy the state q [5][Np] into the context.  rho0 and rhotheta0 ([n_z]
 * each, both or neither) replace the reference state; NULL keeps the
 * previous one (the first call must give them).  The reference arrays are
 * read synchronously (they are small); q is copied on `stream`.
 * Errors: XG_ERR_ARG (NULL q, only one of rho0/rhotheta0, no reference yet,
 * a non-positive reference value), XG_ERR_CUDA. */
xg_status xg_set_state(xg_ctx* ctx, const double* q, const double* rho0,
                       const double* rhotheta0, int where, void* stream);

/* Copy the heating S_theta [Np] (K s^-1) into the context, on `stream`;
 * NULL sets it to zero.  Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_set_forcing(xg_ctx* ctx, const double* S_theta, int where, void* stream);

/* Eq. 12 for the current state: dqdt [5][Np] = M^-1 DSS(w J S(q)) with the
 * wall condition (the wall-normal momentum tendency is zero at wall nodes).
 * Does not modify the state.  With XG_HOST the call waits for the copy;
 * with the closure of xg_closure.h on it always waits.
 * Errors: XG_ERR_ARG (NULL, no state yet), XG_ERR_TIMEOUT (the closure
 * kernel's bounded tensor-core wait ran out), XG_ERR_CUDA. */
xg_status xg_rhs(xg_ctx* ctx, double* dqdt, int where, void* stream);

/* nsteps SSP-RK3 steps of size dt (each step three fused stage passes:
 * q1 = q + dt L(q); q2 = 3/4 q + 1/4 (q1 + dt L(q1));
 * q <- 1/3 q + 2/3 (q2 + dt L(q2))).  Waits for the GPU once at the end to
 * read the non-finite flag.  Errors: XG_ERR_ARG (dt not finite, nsteps < 0,
 * no state yet), XG_ERR_NONFINITE, XG_ERR_TIMEOUT (the closure kernel's
 * bounded tensor-core wait ran out), XG_ERR_CUDA. */
xg_status xg_step(xg_ctx* ctx, double dt, int nsteps, void* stream);

/* Copy the current state to q [5][Np], on `stream` (XG_HOST waits for it).
 * Errors: XG_ERR_ARG (NULL, no state yet), XG_ERR_CUDA. */
xg_status xg_get_state(xg_ctx* ctx, double* q, int where, void* stream);

/* Conservation sums of the current state, accumulated in FP64 whatever the
 * precision: out[v] = sum_I M_I q_v,I for v = 0..4 (rho', rho u, rho v,
 * rho w, Theta'), with M_I the diagonal mass of Eqs. 9 and 12 (the LGL
 * weights times the Jacobian, assembled).  Deterministic (fixed summation
 * order); waits for the GPU.  Errors: XG_ERR_ARG (NULL, no state yet),
 * XG_ERR_CUDA. */
xg_status xg_diagnostics(xg_ctx* ctx, double out[5], void* stream);

/* Arithmetic of the x and y derivative contractions of an XG_FP32 context
 * (Eqs. 8-12: the flux values of an element segment times the rows of the
 * scaled derivative matrix).
 *   XG_CONTRACT_FMA     FP32 fused multiply-adds on the CUDA cores (default)
 *   XG_CONTRACT_TF32X3  the tensor cores (tcgen05.mma, TF32 operands, FP32
 *                       accumulation in tensor memory), each flux and matrix
 *                       entry split into a TF32 head and tail and three
 *                       products summed (head*head + tail*head + head*tail);
 *                       order 4 only
 *   XG_CONTRACT_F16X3   the tensor cores with IEEE half-precision operands
 *                       (tcgen05.mma kind f16, FP32 accumulation): the
 *                       differences of each segment's fluxes against its first
 *                       value, scaled by a power of two per segment into half
 *                       range and split into three halves (exact for FP32
 *                       values), against Dm split likewise; six partial
 *                       products in two instructions of K = 16; order 4 only
 * The z contraction stays on the CUDA cores.  Errors: XG_ERR_ARG (NULL, an
 * unknown mode), XG_ERR_UNSUPPORTED (a tensor-core mode on a context that
 * is not XG_FP32 or not of order 4). */
enum { XG_CONTRACT_FMA = 0, XG_CONTRACT_TF32X3 = 1, XG_CONTRACT_F16X3 = 2 };
xg_status xg_set_contraction(xg_ctx* ctx, int mode);

/* Streamed host-to-host steps (Sec. 5's throughput setting: many
 * independent states through one context).  For each of count inputs:
 * state <- q_in[k] (host, [5][Np] FP64), nsteps SSP-RK3 steps of dt,
 * q_out[k] <- the state (host).  The copies run on two streams of the
 * context: the upload of input k + 1 and the download of output k - 1
 * overlap the steps of input k (the host link carries both directions at
 * once), so for count > 1 they hide behind the arithmetic.  q_in and q_out
 * are arrays of count host pointers (pinned memory gives the full copy
 * rate); a q_out pointer may repeat (its last write is the latest output),
 * but no output may overlap any input (XG_ERR_ARG, checked on the host).
 * The reference state of xg_set_state is kept; afterwards the context holds
 * the last output's state.  Outputs equal set_state + step + get_state of
 * each input bit for bit.  XG_FP64 and XG_DF64 contexts step each input in
 * the device array it was uploaded to and download the output from the
 * array the steps leave it in (no device copies); XG_FP32 converts through
 * FP64 staging arrays.  Allocates 4 FP64 state arrays of device memory on
 * first use; waits for the GPU.  Errors: XG_ERR_ARG (NULL, count < 0, no
 * reference state yet, an output overlapping an input), XG_ERR_UNSUPPORTED (a
 * partitioned context),
 * XG_ERR_OOM, XG_ERR_NONFINITE, XG_ERR_TIMEOUT, XG_ERR_CUDA. */
xg_status xg_step_stream(xg_ctx* ctx, int count, const double* const* q_in, double* const* q_out, double dt,
                         int nsteps, void* stream);

/* Pass structure of an XG_FP32 context.  fused = 0 (the default): a stage
 * is the x-y plane kernel followed by the z-line kernel, with the partial
 * tendency in HBM between them.  fused = 1: on order-4 meshes with walls at
 * the bottom and top and the XG_CONTRACT_FMA contraction, each stage is one
 * kernel that marches columns of 4 x 4 elements up through the levels and
 * does the x, y and z contractions, the sources, walls and the stage
 * combination on chip (its state loads staged by TMA where n_x is a
 * multiple of 4); it moves only the stage's own inputs and output, but its
 * level-by-level march makes it slower than the two kernels (measured on
 * the 128 x 128 x 16 box: 1.00 against 0.67 ms per stage); other meshes keep
 * the two kernels.  Both compute the same arithmetic up to the order of two
 * FP32 additions at face nodes.  Errors: XG_ERR_ARG (NULL, fused not 0 or
 * 1). */
xg_status xg_set_fused(xg_ctx* ctx, int fused);

/* Kernel timing (Sec. 5.4 measures its kernels against a roofline; this is
 * the hook for doing the same here).  enable = 1 brackets every kernel that
 * xg_rhs and xg_step launch with CUDA events on the launching stream; the
 * elapsed times are folded into per-kernel totals when those calls end
 * (enabling profiling makes xg_rhs wait for the GPU).  enable = 0 stops
 * recording.  Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_profile(xg_ctx* ctx, int enable);

/* Per-kernel totals since the last reset: ms[k] total device milliseconds and
 * launches[k] launch count of kernel k = 0 (x lines: primitives, x part),
 * 1 (y lines), 2 (z lines: z part, sources, walls, stage store).  reset != 0
 * clears the totals after reading.  Either output may be NULL.
 * Errors: XG_ERR_ARG. */
xg_status xg_kernel_times(xg_ctx* ctx, double ms[3], long long launches[3], int reset);

/* Applies the library's FP64 reciprocal (the one used for 1/rho: a
 * hardware estimate refined by Newton-Raphson steps) to n device values
 * x[i] > 0 (normal numbers), writing out[i], on `stream`.  Exposed so that
 * tests can hold it against IEEE division.  Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_reciprocal(const double* x, double* out, long long n, void* stream);

/* Element partition (Sec. 3.1: non-overlapping element partitions that keep
 * columns whole; Alg. 3: the partition-face contributions are exchanged once
 * per right-hand side).  A domain of nel_y elements along y is split into
 * slabs of consecutive element rows; each slab is an ordinary context whose
 * mesh description covers its own elements (nel[1] = its rows, lo[1]/hi[1]
 * its extent, periodic[1] = 0, so its y nodes run from one partition face to
 * the other, both included).  xg_partition_set marks which of the
 * context's y ends are partition faces (open_lo: y = lo[1], open_hi: y =
 * hi[1]; 0 = a no-flux wall as usual, 1 = a partition face) and gives the
 * caller-owned device buffers of the exchange, each 5 n_x n_z values of 8
 * bytes in the context's representation ([5][n_z][n_x]; FP64 doubles, or
 * double-float pairs for XG_DF64).  At a partition face the face node's y
 * part is the sum of two one-sided rows, one from each slab: the slab above
 * the face sends (send_lo) its partial value (x part plus its own row), the
 * slab below sends (send_hi) its row; after each side has received the
 * other's array (recv_lo from the lower neighbour's send_hi, recv_hi from
 * the upper neighbour's send_lo) both complete the face node in the same
 * order as a single domain does, so a partitioned run equals the
 * single-domain run bit for bit.  A periodic domain is a ring (the first
 * slab's lower neighbour is the last slab).  Precisions XG_FP64 and XG_DF64
 * only; not with hyper-diffusion/sponge (xg_set_dynamics) or IMEX
 * (XG_ERR_UNSUPPORTED).  While any end is open, xg_rhs and xg_step return
 * XG_ERR_UNSUPPORTED: use xg_partition_stage.  Setting both flags to 0
 * restores the walled context.  XG_ERR_ARG: a periodic y direction, a NULL
 * buffer for an open side, flags other than 0/1. */
xg_status xg_partition_set(xg_ctx* ctx, int open_lo, int open_hi, double* send_lo,
                           double* recv_lo, double* send_hi, double* recv_hi);

/* One half of a partitioned pass: stage 0, 1, 2 of an SSP-RK3 step of size
 * dt (as xg_step), or stage -1 for dq/dt into dqdt [5][Np] (as xg_rhs, `where`
 * says where dqdt lives).  half 0 runs the x and y passes and fills the send
 * buffers; the caller then exchanges them with the neighbours (recv_lo <-
 * lower neighbour's send_hi, recv_hi <- upper neighbour's send_lo) on or
 * after `stream`; half 1 combines the received arrays into the face nodes
 * and runs the z pass (sources, walls, the stage store).  Half 1 of stage 2
 * ends the step (the new state becomes current) and, like xg_step,
 * synchronises once to report XG_ERR_NONFINITE.  The send buffers must stay
 * unchanged until half 1 of the same stage has been enqueued.  Errors:
 * XG_ERR_ARG (no open end, half or stage out of range, NULL dqdt for stage
 * -1), XG_ERR_UNSUPPORTED (dynamics set), XG_ERR_CUDA. */
xg_status xg_partition_stage(xg_ctx* ctx, int half, int stage, double dt, double* dqdt, int where,
                             void* stream);

/* Test hook for the equation of state (Sec. 2.1, Eq. 3): p[I] = p' =
 * p(Theta_0 + Theta') - p(Theta_0) at every node I of the mesh, from
 * theta_p[I] = Theta' and the reference Theta_0 of node I's level, evaluated
 * by the same device code and in the same arithmetic as the context's
 * kernels (theta_p is first converted to the context's precision, as
 * xg_set_state converts the state).  Those kernels use a binomial series of
 * (1 + x)^gamma - 1, x = Theta'/Theta_0, for |x| < x_max and
 * expm1(gamma log1p(x)) beyond; *x_max (if x_max is not NULL) receives the
 * switch point (in the FP32 and double-float forms the test is applied to
 * x rounded to float).  theta_p and p are caller-owned device arrays of Np
 * FP64 values; the call is asynchronous on the stream.  XG_ERR_ARG for NULL
 * arrays or a context without a reference state. */
xg_status xg_pressure_perturbation(const xg_ctx* ctx, const double* theta_p, double* p,
                                   double* x_max, void* stream);

/* Free every buffer of the context (synchronises the device first).  NULL
 * is a no-op. */
void xg_destroy(xg_ctx* ctx);

/* Size of the fixed device scratch used by xg_rhs_noalloc (16 MiB). */
#define XG_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The right-hand side of xg_rhs without a context and without allocating
 * any device memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot or must not call cudaMalloc -- for example code
 * running inside an application whose device memory has been handed to its
 * own caching allocator or memory pool (a cudaMalloc there may fail or split
 * the pool), plug-ins and callbacks that are not allowed to allocate, and
 * latency-bound loops where an allocation would stall the device.
 *
 * The caller passes every input and output as device memory of the current
 * device: q [5][Np], rho0 and rhotheta0 [n_z], S_theta [Np] (NULL = no
 * heating), dqdt [5][Np] (layouts as above); dqdt must not overlap q or
 * S_theta (XG_ERR_ARG: other thread blocks still read them while it is
 * written).  The intermediate arrays the
 * kernels need live in one fixed array of XG_NOALLOC_SCRATCH_BYTES per
 * device, which every device that loads this library keeps until the
 * process exits; meshes whose 9 Np + 4 n_z + 32 doubles do not fit (about
 * 233,000 nodes) are rejected with XG_ERR_UNSUPPORTED and a message on
 * stderr.  The first call on a device looks up that array's device address
 * (once per device, with the device current); make that first call before
 * any stream capture.  The address found belongs to the device's primary
 * context (the CUDA runtime's) and is kept for the life of the process: do
 * not call this entry point on a device after a cudaDeviceReset of it.  All calls share the array and it keeps the last
 * call's contents, so calls that overlap on the GPU (different streams or
 * threads) race: serialise them.  Work is enqueued on `stream` and the call
 * returns without waiting; the reference values must be positive (this
 * entry point cannot check device data without waiting for it).
 * Errors: XG_ERR_ARG (NULL pointer, invalid description, dqdt overlapping
 * q or S_theta), XG_ERR_UNSUPPORTED
 * (mesh too large for the scratch, a precision other than XG_FP64, or a
 * description this build cannot run), XG_ERR_CUDA. */
xg_status xg_rhs_noalloc(const xg_mesh_desc* d, const double* q, const double* rho0,
                         const double* rhotheta0, const double* S_theta, double* dqdt,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XG_H */
