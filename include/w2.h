/*
 * w2.h -- C ABI of the GB300 (sm_103a) library that advances the Wigner
 * function of the two-body reduced density matrix (2-RDM) of a spatially
 * periodic 1-D two-particle system by one Lawson step.
 *
 * The equation stepped is the 2-RDM Wigner equation of arXiv:2511.11354
 * (Sec. 2.4, Eq. two_body_truncated_Wigner):
 *
 *   d_t f + (p1/m) d_x1 f + (p2/m) d_x2 f
 *       = Theta_{U1}[f] + Theta_{U2}[f] + Theta_{gamma W}[f],
 *
 * with U_i = V_ext + c_H V_H[n_i] + c_xc phi(n_i) the one-body (external +
 * Hartree + exchange-correlation) potential of particle i, built from its
 * density n_i, and W the pair interaction.  On the periodic box each Theta is
 * the pseudo-difference operator of Sec. 3.1 (Eqs. Hartree_FSM and
 * two_body_FSM), a sum of momentum shifts by multiples of dp = pi hbar / L.
 * A time step is the Lawson predictor-corrector of Sec. 4.1 with the
 * characteristic shift X -> X - tau P / m done by periodic cubic B-spline
 * interpolation (Sec. 4.1, A_per).
 *
 * Grid (shared by every entry point):
 *   x_i = -L/2 + i dx,  dx = L / nx,           i in [0, nx)
 *   p_n = (n - nk/2) dp, dp = pi hbar / L,      n in [0, nk)
 *   phase-space arrays are f[i1][i2][n1][n2], n2 fastest, C order,
 *   nx*nx*nk*nk elements (double for W2_F64 and W2_F64_SLICED, float for
 *   W2_F32_TF32X3 and W2_F32_BF16X3);
 *   f is zero outside the momentum window.
 *
 * Conventions:
 *   - Every function returns a w2_status; nothing throws.  The first CUDA
 *     error seen by a context sticks (every later call returns W2_ERR_CUDA)
 *     until w2_destroy.
 *   - The caller owns every pointer it passes; nothing is retained after a
 *     call returns, except the CUDA stream given to w2_create (borrowed for
 *     the lifetime of the context).
 *   - Device pointers are CUDA global-memory addresses on the context's
 *     device (for example torch tensor data_ptr()).  Host pointers are plain
 *     host memory (pinned or pageable).
 *   - Work is queued on the context's stream and returns immediately, except
 *     where a function says it synchronises.
 *   - There is no CPU fallback: without a usable sm_103a device w2_create
 *     fails with W2_ERR_CUDA.
 */
#ifndef W2_H
#define W2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  W2_OK = 0,
  W2_ERR_ARG = -1,          /* invalid argument (size, pointer, value)          */
  W2_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed       */
  W2_ERR_OOM = -3,          /* device or host allocation failed                  */
  W2_ERR_STATE = -4,        /* call order violated (e.g. step before set_state)  */
  W2_ERR_UNSTABLE = -5,     /* tau * max|symbol| exceeds the stability bound     */
  W2_ERR_NONFINITE = -6,    /* a NaN or Inf was found in the state               */
  W2_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up                */
  W2_ERR_UNSUPPORTED = -8   /* valid but not supported (grid size, precision)    */
} w2_status;

typedef enum {
  W2_F64 = 0,           /* FP64 state and arithmetic (FP64 pipe: DMMA and DFMA)   */
  W2_F32_TF32X3 = 1,    /* precision form: FP32 state; the pseudo-difference
                           contractions on tensor cores, the state split into two
                           TF32 parts and the kernel into three (four products,
                           FP32 accumulate); the spline shift as an FP32 increment
                           of the state; densities and observables in FP64       */
  W2_F32_BF16X3 = 2,    /* precision form as W2_F32_TF32X3, the contractions with
                           BF16 operands: the state in three BF16 parts (exact),
                           the kernel in four; seven m16n8k16 products per 16
                           columns (every term to 2^-16 and the table's 2^-24
                           term), FP32 accumulate; nk, nx as W2_F32_TF32X3        */
  W2_F64_SLICED = 3     /* FP64 state and results as W2_F64 (the FP64 oracle to
                           1e-10 over whole steps); the pseudo-difference
                           contractions as exact products of six 8-bit integer
                           slices of each operand on the BF16 tensor cores (the
                           Ozaki splitting, 21 slice pairs), recombined in 64-bit
                           integers; nk in {16, 32, 48, 64}; on mma.sync, or
                           on tcgen05 for nk = 64 (w2_set_tensor_path)           */
} w2_precision;

typedef enum {
  W2_HARTREE_PAIR = 0,     /* V_H[n](x) = gamma dx sum_q W(fold(x - x_q)) n(x_q): the pair
                              kernel of w2_set_potentials (the default)                   */
  W2_HARTREE_POISSON = 1   /* neutralised periodic Poisson (the 1-D Coulomb example of
                              Sec. 2.3 under an ion background): -V_H'' = n - mean(n),
                              the N_x-point Fourier solution, Nyquist mode as its cosine  */
} w2_hartree_kind;

typedef enum {
  W2_XC_NONE = 0,       /* no exchange-correlation term                           */
  W2_XC_LINEAR = 1,     /* phi(n) = n (the exchange test potential of Sec. 5.1.1) */
  W2_XC_HEDIN_LUNDQVIST = 2  /* phi(n) = 0.985 c + 0.985*0.034 ln(1 + 18.37 c), c = max(n,0)^{1/3}:
                                the H-L form of Sec. 2.2 in atomic units          */
} w2_xc_kind;

/* Problem description (Sec. 3.1 grid; Sec. 5 uses hbar = m = 1).
 *   nx  : spatial points per particle, 4 <= nx; FP64 supports nx <= 128,
 *         W2_F32_TF32X3 and W2_F32_BF16X3 nx <= 256
 *   nk  : momentum points per particle; W2_F64 supports nk in {8,16,...,64},
 *         W2_F64_SLICED nk in {16,32,48,64}, W2_F32_TF32X3 and W2_F32_BF16X3
 *         nk in {16,32,...,128}
 *   L   : period of the box (> 0); dt: time step tau (> 0)
 *   hbar, mass: > 0
 *   precision: a w2_precision;  xc_kind: a w2_xc_kind                          */
typedef struct {
  int32_t nx, nk;
  double L, dt, hbar, mass;
  int32_t precision;
  int32_t xc_kind;
} w2_config;

/* A potential evaluated on the HOST only, at arguments already folded into
 * [-L/2, L/2); user is passed through unchanged. */
typedef double (*w2_fn)(double x, void *user);

/* Observables of the current state (Sec. 2 definitions; reductions in FP64,
 * in a fixed order, so repeated calls give identical bits).
 *   mass        = sum f dx^2 dp^2
 *   energy      = sum f (p1^2/2m + p2^2/2m + V(x1) + V(x2) + gamma W(x1-x2)) dV
 *                 + (c_H/2) sum_i [n_1 V_H[n_1] + n_2 V_H[n_2]](x_i) dx
 *   purity      = Tr rho_1^2 = 2 pi hbar sum f1^2 dx dp, f1 = sum_{x2,p2} f dx dp
 *   entropy_lin = 1 - purity (linear entropy of the one-body matrix)
 *   l2norm      = sqrt(sum f^2 dV)
 *   step        = number of steps taken since the last w2_set_state        */
typedef struct {
  double mass, energy, purity, entropy_lin, l2norm;
  int64_t step;
} w2_obs;

typedef struct w2_ctx w2_ctx;

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream), borrowed.  Allocates the device workspace
 * (4 phase-space arrays plus small tables).  Errors: W2_ERR_ARG (bad config or
 * out == NULL), W2_ERR_UNSUPPORTED (nk not supported for the precision),
 * W2_ERR_OOM, W2_ERR_CUDA (no usable device).  *out is NULL on failure. */
w2_status w2_create(const w2_config *cfg, void *cuda_stream, w2_ctx **out);

/* Set the external potential V_ext (vext), the pair interaction W (vee), the
 * pair strength gamma, and the weights c_hartree of the Hartree potential
 * V_H[n](y) = gamma dx sum_q W(fold(y - x_q)) n(x_q) (Sec. 2.3, smoothed
 * Coulomb example, on the torus) and c_xc of the XC potential (Sec. 2.2).
 * vext == NULL means V_ext = 0; vee == NULL means W = 0.  The callbacks are
 * called on the host during this call only (at x_i + l L/(2 nk) and at the
 * pair distances d dx + l L/(2 nk)).  Builds the pair kernel tables on the
 * device (queued on the stream).
 * Errors: W2_ERR_ARG (non-finite parameter or callback value),
 * W2_ERR_UNSTABLE when tau/hbar * (2 max|dV_ext| + gamma max|dW| +
 * 2 |c_H| gamma (max W - min W)) > 1 (the worst mode of Heun's method on the
 * imaginary axis then grows by more than sqrt(1 + 1/4) per step; the
 * Hartree bound assumes unit mass), W2_ERR_CUDA. */
w2_status w2_set_potentials(w2_ctx *ctx, w2_fn vext, void *ue, w2_fn vee, void *ui,
                            double gamma, double c_hartree, double c_xc);

/* Choose how the Hartree potential (weight c_hartree) is formed: kind is a
 * w2_hartree_kind.  W2_HARTREE_POISSON (the plasma examples, Sec. 5.2) solves
 *   -V_H'' = n - mean(n),  V_H(y) = sum_q G(y - x_q) n(x_q),
 *   G(r) = (1/N_x) [2 sum_{0 < m < N_x/2} cos(k_m r)/k_m^2 + cos(k_{N_x/2} r)/k_{N_x/2}^2],
 * k_m = 2 pi m / L (the last term for even N_x only); the energy's Hartree
 * term uses the same kernel.  May be called before or after
 * w2_set_potentials; the stability precheck of w2_set_potentials leaves the
 * Poisson term out (it depends on the state).  Errors: W2_ERR_ARG,
 * W2_ERR_OOM, W2_ERR_CUDA. */
w2_status w2_set_hartree(w2_ctx *ctx, int32_t kind);

/* Distributed form of the characteristic shift (Sec. 4.2, local splines with
 * perfectly matched boundary conditions): the x1 shift is cut into np1
 * patches of nx / np1 points and the x2 shift into np2 patches (1: the global
 * spline of Sec. 4.1).  Each patch solves its own spline over its points and
 * G ghost points per side (G = 1 + the shift's whole cells), with the slopes
 * of the global spline at the ends of that range as boundary rows; each slope
 * is a 53-point stencil of the samples (coefficients below 2^-52 beyond), of
 * which the part over a neighbouring patch is summed by that neighbour and
 * handed over with the ghost samples, as one rank hands them to the next.
 * All patches run in this process on this device, the hand-over going
 * through device buffers; results equal the global spline shift to FP64
 * rounding.  Applies to w2_step and w2_advect of a W2_F64 context until the
 * next call (np1 = np2 = 1 restores the global spline).
 * Errors: W2_ERR_ARG (np < 1), W2_ERR_UNSUPPORTED (another precision, nx not a
 * multiple of np, or fewer than G + 26 points per patch), W2_ERR_OOM,
 * W2_ERR_CUDA. */
w2_status w2_set_patches(w2_ctx *ctx, int32_t np1, int32_t np2);


/* Copy a full state f[nx][nx][nk][nk] (element type of the precision) into the context: from device
 * memory when on_device != 0, else from host memory.  Resets the step count.
 * Queued on the stream (a host source is copied with cudaMemcpyAsync, so a
 * pageable host buffer is copied before return).
 * Errors: W2_ERR_ARG (NULL f), W2_ERR_STATE (potentials not set), W2_ERR_CUDA. */
w2_status w2_set_state(w2_ctx *ctx, const void *f, int32_t on_device);

/* Double-buffered input from host memory, so that the host-to-device copy of
 * the next state overlaps the work on the current one.  w2_stage_state queues
 * the copy of a host state f (layout and element type of w2_set_state) into
 * the context's staging buffer on a private copy stream and returns; the
 * context's state is not touched.  The copy starts once the previous staged
 * state has been taken.  w2_use_staged_state makes the staged state the
 * context's state: the context's stream waits for the copy, the staging
 * buffer and the state buffer trade places (no device copy; the next staged
 * copy goes into the old state buffer once the work queued on it is done),
 * the per-X sums of the new state are computed and the step count is reset.
 * The step is captured once per state buffer (two graphs alternate).  The
 * staging buffer (one state) and the copy stream are created by the first
 * w2_stage_state.  The host buffer must stay unchanged until the copy is
 * done, which any synchronising call after the matching w2_use_staged_state
 * guarantees; pinned host memory makes the copy asynchronous.
 * Errors: W2_ERR_ARG, W2_ERR_STATE (potentials not set; for
 * w2_use_staged_state: nothing staged), W2_ERR_OOM, W2_ERR_CUDA. */
w2_status w2_stage_state(w2_ctx *ctx, const void *f);
w2_status w2_use_staged_state(w2_ctx *ctx);

/* Exchange symmetry of the two-body state (identical particles):
 * f(x1, x2, p1, p2) = f(x2, x1, p2, p1), which the paper's 2-RDM satisfies and
 * the Lawson step preserves.  With on = 1 the sliced sweeps of w2_step
 * (W2_F64_SLICED only) compute the pseudo-difference operator on the blocks
 * X = (i1, i2) with i1 <= i2 and write each mirror block (i2, i1) as the
 * transpose (the one-body kernels of the two particles coincide and the pair
 * kernel is odd in x1 - x2), about half the tensor-core work of a step.  The
 * caller guarantees that the state it sets is exchange symmetric; for other
 * states the results differ from on = 0 by the state's asymmetric part.
 * Not used while a learned two-body term is active, nor by w2_theta.
 * Errors: W2_ERR_ARG (on not 0 or 1), W2_ERR_UNSUPPORTED (on = 1 and not
 * W2_F64_SLICED). */
w2_status w2_set_exchange_symmetry(w2_ctx *ctx, int32_t on);

/* Tensor-core path of the sliced sweeps (W2_F64_SLICED; the pseudo-difference
 * operator of Sec. 3.1 as exact 8-bit slice products).  tcgen05 = 0, the
 * default, runs every sweep on the warp-level mma.sync path (the faster one
 * on this operator: see the design notes).  tcgen05 = 1 runs every digit
 * product on the 5th-generation tensor cores (tcgen05 MMA with the
 * accumulators in tensor memory) where supported: N_k = 64 without a learned
 * pair term; other cases stay on the warp-level path.  Both give the operator
 * to FP64 accuracy and differ only in the rounding of the lowest slice
 * diagonal (below 2^-50 of each block's scale).  A bounded wait of the
 * tcgen05 sweep that gives up (about a second) leaves NaN in its block and
 * makes w2_observables return W2_ERR_TIMEOUT until a new state is set
 * (w2_set_state or w2_use_staged_state clears the error).
 * Errors: W2_ERR_ARG (tcgen05 not 0 or 1), W2_ERR_UNSUPPORTED (tcgen05 = 1 and
 * not W2_F64_SLICED). */
w2_status w2_set_tensor_path(w2_ctx *ctx, int32_t tcgen05);

/* Host-requested fault injection into the tcgen05 sweep, for testing its
 * time-out path without any device fault: with stall = 1 every tcgen05 sweep
 * of the context leaves one batch of its products and their completion signal
 * out, so its next bounded wait (wait_cycles SM clocks; 0: about a second)
 * runs out; the sweep then issues nothing more, waits for the products it did
 * issue, writes NaN to its blocks and sets the error word that makes
 * w2_observables return W2_ERR_TIMEOUT.  stall = 0 restores normal sweeps and
 * clears the error word.  Errors: W2_ERR_ARG. */
w2_status w2_debug_sweep_stall(w2_ctx *ctx, int32_t stall, int64_t wait_cycles);

/* Copy the current state out (same layout).  With on_device == 0 the call
 * synchronises the stream before returning.  Errors: W2_ERR_ARG, W2_ERR_STATE
 * (no state), W2_ERR_CUDA. */
w2_status w2_get_state(w2_ctx *ctx, void *f, int32_t on_device);

/* Advance the state by nsteps >= 0 Lawson steps (Sec. 4.1):
 *   g  = Theta[f^n];  a = A_tau f^n;  b = A_tau g
 *   f~ = a + tau b;   f^{n+1} = a + tau/2 (b + Theta[f~])
 * where each Theta takes its HXC potential from the densities of its own input
 * and A_tau g(X, P) = g(X - tau P / m, P) by periodic cubic splines.
 * One step is captured once into a CUDA graph and replayed; queued on the
 * stream.  Errors: W2_ERR_ARG (nsteps < 0), W2_ERR_STATE, W2_ERR_CUDA. */
w2_status w2_step(w2_ctx *ctx, int32_t nsteps);

/* Compute the observables of the current state.  Synchronises the stream.
 * out (required) receives the scalars; n1 (host, [nx], or NULL) the density
 * n_1(x_i) = sum f dx dp^2 over (x2, p1, p2); n12 (host, [nx*nx], or NULL) the
 * pair density n_12(x_i1, x_i2) = sum f dp^2 over (p1, p2).
 * Errors: W2_ERR_ARG, W2_ERR_STATE, W2_ERR_NONFINITE (NaN/Inf in the state; the
 * outputs are still written), W2_ERR_TIMEOUT (a tcgen05 sweep gave up a wait,
 * see w2_set_tensor_path), W2_ERR_CUDA. */
w2_status w2_observables(w2_ctx *ctx, w2_obs *out, double *n1, double *n12);

/* The same observables without waiting, for a host loop that reads each
 * step's results while the next step runs.  w2_observables_enqueue queues
 * the reductions of the current state and the copy of their results into
 * pinned host slot `slot` (0 or 1) on the stream, and returns.
 * w2_observables_collect waits for that slot's copy (not for later work on
 * the stream) and unpacks it exactly as w2_observables does; the step count
 * reported is the one at enqueue time.  A slot must be collected before it is
 * enqueued again.  Errors: W2_ERR_ARG (slot not 0 or 1, NULL out), W2_ERR_STATE
 * (no state; collect: slot not enqueued), W2_ERR_NONFINITE, W2_ERR_CUDA. */
w2_status w2_observables_enqueue(w2_ctx *ctx, int32_t slot);
w2_status w2_observables_collect(w2_ctx *ctx, int32_t slot, w2_obs *out, double *n1, double *n12);

/* Operator-level entry points on caller-owned DEVICE arrays of the context's
 * layout (f and out may not alias).  Queued on the stream.
 *
 * w2_theta:  out = Theta_V[f] of Eq. two_body_truncated_Wigner (Sec. 3.1
 *            discretisation), the HXC potentials built from the densities of f.
 * w2_advect: out = A_tau f, i.e. out(X, P) = f(X - tau P/m, P) by the periodic
 *            cubic B-spline of Sec. 4.1, x1 and x2 in turn.
 * Arrays hold the context precision's element type.
 * Errors: W2_ERR_ARG (NULL or aliasing pointers; a pointer not 16-byte aligned
 * for w2_theta, and for w2_advect in the FP32 precisions), W2_ERR_STATE (potentials
 * not set), W2_ERR_CUDA.  Both use the context's workspace and must not overlap
 * with w2_step on another stream. */
w2_status w2_theta(w2_ctx *ctx, const void *f, void *out);
w2_status w2_advect(w2_ctx *ctx, const void *f, void *out);

/* Diagnostic form of w2_step: advances nsteps > 0 steps launching the step's
 * W2_STEP_KERNELS kernels directly (no graph) with a CUDA event pair on the
 * context's stream around each, and writes to kernel_ms[k] (host, length
 * W2_STEP_KERNELS) the mean duration in milliseconds of kernel k of a step:
 *   0 per-X sums of f^n (no launch: they come from the previous step's
 *     corrector, or from w2_set_state / w2_use_staged_state; about 0)
 *   1 kernel tables (f^n)   2 Theta sweep, predictor
 *   3 shift along x2      4 shift along x1 + Lawson combination
 *   5 per-X sums of f~    6 kernel tables (f~)
 *   7 Theta sweep, corrector (with the per-X sums of f^{n+1})
 * The state advances exactly as with w2_step.  Synchronises the stream.
 * Errors: W2_ERR_ARG (nsteps <= 0 or kernel_ms NULL), W2_ERR_STATE, W2_ERR_CUDA. */
#define W2_STEP_KERNELS 8
w2_status w2_step_profile(w2_ctx *ctx, int32_t nsteps, double *kernel_ms);

/* Allocation-free form of w2_theta, for callers that may not allocate device
 * memory at all: code that runs while someone else's CUDA stream capture is
 * open (cudaMalloc is not allowed there), hot loops whose device memory is
 * owned and budgeted by a host framework, or plug-ins whose host forbids
 * calls into the allocator.  The paper has no counterpart; it is a property of
 * this library only.
 *
 * out = Theta_V[f] for potentials the caller has already sampled (device
 * arrays, row-major, l in [0, 2 nk), h' = L / (2 nk)):
 *   u1[i][l]  = U1(x_i + l h')   one-body potential of particle 1
 *   u2[i][l]  = U2(x_i + l h')   one-body potential of particle 2
 *   u12[d][l] = U12(d dx + l h') pair potential (gamma W) at distance d dx + l h'
 * With u1 = u2 = V_ext samples and u12 = gamma W samples this is w2_theta of a
 * context whose c_hartree = c_xc = 0.  f and out: device [nx][nx][nk][nk]
 * doubles, 16-byte aligned, not aliasing; cfg: only nx, nk, L, hbar and
 * precision (W2_F64) are read.  Queued on cuda_stream (a cudaStream_t, NULL =
 * legacy default stream).
 *
 * No allocation: the shift-kernel tables live in one fixed device array of
 * 3 * W2_NOALLOC_MAX_NX * (2 * W2_NOALLOC_MAX_NK - 1) + 2 * W2_NOALLOC_MAX_NK
 * doubles (about 391 KB) that is part of the library image, so every device
 * that loads the library holds it until the process exits.  The first call on
 * a device, with that device current, resolves the array's address and sets
 * kernel attributes; make that first call before any stream capture.  All
 * calls share the one array and every call rewrites all of it that it reads,
 * so nothing has to be cleared between calls, but calls that overlap on the
 * GPU (different streams, threads or captured graphs in flight at once) race
 * on it and give wrong results.  The array's address and the kernel
 * attributes are kept per device for the life of the process: after a
 * cudaDeviceReset of a device this entry point must not be called on it again
 * (the kept address no longer belongs to a live allocation).
 * Errors: W2_ERR_ARG (NULL, aliasing or misaligned pointers, bad grid),
 * W2_ERR_UNSUPPORTED (nx > W2_NOALLOC_MAX_NX, nk > W2_NOALLOC_MAX_NK, nk not a
 * multiple of 8, or a precision other than W2_F64), W2_ERR_CUDA. */
#define W2_NOALLOC_MAX_NX 128
#define W2_NOALLOC_MAX_NK 64
w2_status w2_theta_noalloc(const w2_config *cfg, const double *u1, const double *u2, const double *u12,
                           const double *f, double *out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batching form: many independent problems (uneven nx, nk, potentials and
 * pair strengths) advanced together.  Every instance is a W2_F32_TF32X3
 * problem with its own state.  One batch step is ONE persistent kernel: its
 * CTAs take the work items of all seven phases of the Lawson step of every
 * instance (tables, Theta predictor, the two shift passes, per-X sums of f~,
 * tables, Theta corrector with the per-X sums of f^{n+1}) from one list,
 * phase after phase, and an item starts once every item of the previous
 * phase of its instance has finished.  The launch is captured once into a CUDA graph and replayed.
 * Results are identical, bit for bit, to running each instance in its own
 * context.  (Sec. 4.2 of the paper runs one problem over many ranks; running
 * many problems in one launch has no counterpart there.)
 * ------------------------------------------------------------------------ */
typedef struct w2_batch w2_batch;

/* Create n (1..4096) instances from cfgs[0..n) (every precision must be
 * W2_F32_TF32X3, nx <= 128, nk <= 64, other fields as for w2_create) on the
 * current device, all on the borrowed cuda_stream.  Errors: as w2_create,
 * W2_ERR_UNSUPPORTED for another precision, nx > 128 or nk > 64.  *out is
 * NULL on failure. */
w2_status w2_batch_create(const w2_config *cfgs, int32_t n, void *cuda_stream, w2_batch **out);

/* Per-instance forms of w2_set_potentials / w2_set_state / w2_get_state /
 * w2_observables for instance i in [0, n); W2_ERR_ARG for another i.  The
 * synchronising ones (w2_batch_get_state to the host, w2_batch_observables)
 * first wait for the queued steps and return W2_ERR_TIMEOUT if a wait inside
 * one of them ran out (see w2_batch_set_wait_limit). */
w2_status w2_batch_set_potentials(w2_batch *b, int32_t i, w2_fn vext, void *ue, w2_fn vee, void *ui,
                                  double gamma, double c_hartree, double c_xc);
w2_status w2_batch_set_state(w2_batch *b, int32_t i, const void *f, int32_t on_device);
w2_status w2_batch_get_state(w2_batch *b, int32_t i, void *f, int32_t on_device);
w2_status w2_batch_observables(w2_batch *b, int32_t i, w2_obs *out, double *n1, double *n12);

/* Advance every instance by nsteps Lawson steps (as w2_step): nsteps
 * replays of the one-launch step graph.  Needs potentials and a state on
 * every instance (W2_ERR_STATE otherwise).  Asynchronous; a wait that ran out
 * in an earlier call is reported here as W2_ERR_TIMEOUT once it is known. */
w2_status w2_batch_step(w2_batch *b, int32_t nsteps);

/* Wait for the queued steps; W2_OK, or W2_ERR_TIMEOUT / W2_ERR_CUDA (sticky). */
w2_status w2_batch_sync(w2_batch *b);

/* Failure detection.  Every wait of an item for the previous phase of its
 * instance is bounded: after `seconds` (default about 2 s; 0 < seconds <= 60)
 * the CTA records W2_ERR_TIMEOUT, all CTAs stop taking items and the launch
 * ends, leaving the CUDA context usable; the batch then reports
 * W2_ERR_TIMEOUT (sticky: its states are not valid).
 * w2_batch_inject_stall is the host-side fault injector that tests this: the
 * finished items of phase `phase` (0..6) of instance i are no longer counted,
 * so the items of the next phase wait until their limit; phase = -1 removes
 * the stall.  Errors: W2_ERR_ARG. */
w2_status w2_batch_set_wait_limit(w2_batch *b, double seconds);
w2_status w2_batch_inject_stall(w2_batch *b, int32_t phase, int32_t i);

/* Autotuner: times candidate tile shapes of the persistent step (columns
 * per shift item 64 or 32, warps per 16-row Theta block 2 or 1, work units
 * per item such that a CTA takes about 2, 8 or 32 items per phase) at 1 and
 * 2 CTAs per SM (as far as they fit) on the batch as it is (potentials and
 * states set; the states are kept and restored), and keeps the fastest.
 * Synchronises.  tuning_out (host, tuning_len entries, or NULL) receives
 *   [shift columns, Theta warps per row block, grid (CTAs), shared memory
 *    bytes per CTA, best step time in microseconds, shapes tried, work items
 *    per step, items per CTA and phase]  (zeros after the end).
 * Errors: W2_ERR_ARG, W2_ERR_STATE, W2_ERR_OOM (no room to keep the states),
 * W2_ERR_TIMEOUT, W2_ERR_CUDA. */
w2_status w2_batch_autotune(w2_batch *b, int32_t *tuning_out, int32_t tuning_len);

/* Release the batch and all its instances (NULL is ignored). */
void w2_batch_destroy(w2_batch *b);

/* ------------------------------------------------------------------------
 * Learned form: a multilayer perceptron stands in for the two-body term
 * Theta_{V12} (Eq. two_body_FSM) of W2_F64 contexts.  For each spatial point
 * X = (x1, x2) its input row (BF16, w2_mlp_input_dim entries) is
 *   s_f f(X, p1, p2) for all nk^2 momenta, s_f1 f1(x1, .) and s_f1 f1(x2, .)
 *   (f1 = sum over x2, p2 of f dx dp, the reduced one-body Wigner function),
 *   sin(2 pi m (x1 - x2)/L), cos(2 pi m (x1 - x2)/L) for m = 1..8 (in that
 *   order, sin first), zeros up to a multiple of 32;
 * its output is s_y Theta_{V12}[f](X, ., .) (nk^2 values).  Layers: input ->
 * hidden -> hidden -> hidden -> nk^2 with SiLU between them; FP32 master
 * weights, BF16 tensor-core products with FP32 accumulation; trained by the
 * library's own forward, backward and Adam kernels on the mean squared error.
 * Parameters are packed as W0 [din][H], b0 [H], W1 [H][H], b1, W2 [H][H], b2,
 * W3 [H][nk^2], b3 [nk^2] (row-major, floats).
 * ------------------------------------------------------------------------ */
typedef struct w2_mlp w2_mlp;

/* Create an MLP for momentum size nk (hidden width a multiple of 16) able to
 * process max_rows input rows per call, on the borrowed cuda_stream.  The
 * weights start uniform in +-sqrt(3/fan_in) (a fixed counter-based sequence),
 * biases 0, scales 1.  Errors: W2_ERR_ARG, W2_ERR_OOM, W2_ERR_CUDA. */
w2_status w2_mlp_create(int32_t nk, int32_t hidden, int32_t max_rows, void *cuda_stream, w2_mlp **out);
/* A kernel network: the same layers, with the two-body term's structure.
 * Theta_{V12} f(X, n1, n2) = sum_{j >= 1} K(r, j) [F(n1 + j, n2 - j) -
 * F(n1 - j, n2 + j)] is linear in F = f(X, ., .) with a kernel that depends
 * on the pair distance r = x1 - x2 only, so this network maps the distance's
 * harmonics (sin, cos (2 pi m r / L), m = 1..8, zeros up to 32 inputs) to
 * s_y K^(r, j), j = 0 .. nk - 1 (nk outputs; j = 0 is not used).  Attached to
 * a context (w2_learned_attach) it is evaluated once for the nx distances d dx
 * and its table K^ takes the place of the exact pair table in the sweep.
 * max_nx (<= 1024): the largest nx it will serve.
 * Errors: W2_ERR_ARG, W2_ERR_OOM, W2_ERR_CUDA. */
w2_status w2_mlp_create_kernel(int32_t nk, int32_t hidden, int32_t max_nx, void *cuda_stream, w2_mlp **out);
/* One Adam step of a kernel network m (the context's nk, max_nx >= nx) on a
 * batch of rows spatial points taken from trajectories of the exact method:
 * f (device, FP64 [rows][nk^2]) the state blocks f(X, ., .), p (device, FP64
 * [rows][nk^2]) the exact two-body term there, dr (device, int32 [rows]) the
 * pair distance index d = (i1 - i2) mod nx of each point.  The loss
 * sum |Theta_K^ F - P|^2 / sum |P|^2 (host, *loss, before the update) and its
 * gradient with respect to the network's outputs are formed by the library's
 * kernels; the update runs through the network's own backward and Adam
 * kernels (lr, as w2_mlp_train_step).  Synchronises.
 * Errors: W2_ERR_ARG (not a kernel network, another nk, nx > max_nx, NULL),
 * W2_ERR_OOM, W2_ERR_NONFINITE, W2_ERR_CUDA. */
w2_status w2_pair_kernel_train_step(w2_ctx *ctx, w2_mlp *m, const double *f, const double *p, const int32_t *dr,
                                    int32_t rows, float lr, double *loss);
/* The same loss for a batch of rows, and its gradient with respect to the
 * network's outputs without an update: *loss (host, required), y (host,
 * float [nx][nk], or NULL) the network's outputs for every distance,
 * dldy (host, double [nx][nk], or NULL) dL/dy (column j = 0 is not used by
 * the kernel and is 0).  For checking the training chain against a reference.
 * Synchronises.  Errors: as w2_pair_kernel_train_step. */
w2_status w2_pair_kernel_loss_grad(w2_ctx *ctx, w2_mlp *m, const double *f, const double *p, const int32_t *dr,
                                   int32_t rows, double *loss, float *y, double *dldy);
size_t w2_mlp_param_count(const w2_mlp *m);
int32_t w2_mlp_input_dim(const w2_mlp *m);
/* Host copies of the packed FP32 parameters (synchronise). */
w2_status w2_mlp_set_params(w2_mlp *m, const float *params);
w2_status w2_mlp_get_params(w2_mlp *m, float *params);
/* Input and output scales (all > 0). */
w2_status w2_mlp_set_scales(w2_mlp *m, float s_f, float s_f1, float s_y);
/* y[rows][nk^2] (device, FP32) = network(x) for x (device, BF16 [rows][din]). */
w2_status w2_mlp_forward(w2_mlp *m, const void *x, int32_t rows, float *y);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the mean squared error
 * against target (device, FP32 [rows][nk^2], already scaled by s_y); *loss
 * (host) receives the loss before the update.  Synchronises.
 * Errors: W2_ERR_ARG, W2_ERR_NONFINITE (non-finite loss), W2_ERR_CUDA. */
w2_status w2_mlp_train_step(w2_mlp *m, const void *x, const float *target, int32_t rows, float lr, double *loss);
/* Loss and its gradient with respect to the packed parameters (host,
 * w2_mlp_param_count floats, or NULL), without an update.  Synchronises. */
w2_status w2_mlp_gradients(w2_mlp *m, const void *x, const float *target, int32_t rows, float *grads, double *loss);
void w2_mlp_destroy(w2_mlp *m);

/* Input rows (device, BF16 [rows][w2_mlp_input_dim(m)]) for the spatial points
 * xs[0..rows) (device int32, X = i1*nx + i2), or for every X in order when xs
 * is NULL (rows must then be nx*nx), from the state f (device, the context's
 * element type), with m's input scales.  Queued on the stream. */
w2_status w2_features(w2_ctx *ctx, const w2_mlp *m, const void *f, const int32_t *xs, int32_t rows, void *x);

/* out = Theta_{V12}[f] alone (the exact two-body term; device arrays of the
 * context's element type, 16-byte aligned).  Queued on the stream. */
w2_status w2_theta_pair(w2_ctx *ctx, const void *f, void *out);

/* Make w2_step use m for the two-body term of a W2_F64 or W2_F64_SLICED
 * context (m must have the context's nk and max_rows >= nx*nx, or for a
 * kernel network max_nx >= nx, whose table is evaluated here; m = NULL goes
 * back to the exact term).  Every judge_every steps (0: never) the network is compared with the
 * exact term on the current state (relative L2 error of the two-body term);
 * above tol the context falls back to the exact term for good.  The MLP is
 * borrowed and must outlive its use.  Errors: W2_ERR_ARG, W2_ERR_UNSUPPORTED
 * (not W2_F64), W2_ERR_OOM. */
w2_status w2_learned_attach(w2_ctx *ctx, w2_mlp *m, int32_t judge_every, double tol);
/* active: 1 while the network is in use; judged: judgements so far; last_err:
 * the latest relative error. */
w2_status w2_learned_report(w2_ctx *ctx, int32_t *active, int32_t *judged, double *last_err);

/* ------------------------------------------------------------------------
 * Occupation numbers and correlation entropy (the paper's appendix on the
 * correlation entropy through the Wigner function, Sec. 5.3):
 *   f1(x, p) = sum_{x2, p2} f dx dp  (particle 1),
 *   rho1(x_{mu - nu}, x_{mu + nu}) = dp sum_n f1(x_mu, p_n) e^{-2 pi i (n - nk/2) nu / nx},
 * nu = (c - b)/2 for the entry (b, c) with c - b the minimal image on the
 * torus, mu = b + nu (for odd b + c a half point, where f1 comes from its
 * periodic trigonometric interpolant), rho1 made Hermitian as
 * (rho1 + rho1^H)/2.  occ[k] (host, nx values, largest first) are the
 * eigenvalues of rho1 dx (the device eigensolver of w2_hermitian_eigvals, FP64);
 * *entropy (host) = sum_k n_k ln n_k / sum_k n_k over n_k > 1e-14 n_0.
 * Either pointer may be NULL.  Synchronises the stream.
 * Errors: W2_ERR_ARG, W2_ERR_STATE (no state), W2_ERR_OOM, W2_ERR_CUDA. */
w2_status w2_occupations(w2_ctx *ctx, double *occ, double *entropy);

/* Eigenvalues of batch complex Hermitian n x n matrices (device, row-major,
 * interleaved re/im doubles, 16-byte aligned; overwritten).  Up to n = 320
 * (the matrix spread over the shared memory of a cluster of 8 CTAs):
 * Householder reduction to tridiagonal form, then bisection on Sturm counts
 * (one warp per eigenvalue, 32 points a round, down to a few ulps; absolute
 * error a small multiple of n eps |A|).  Larger n (or a device without room
 * for the cluster): one CTA per matrix, cyclic Jacobi with the round-robin
 * ordering (at most 40 sweeps; stops when the off-diagonal part is below
 * 1e-14 of the matrix).  eig: device [batch][n], largest first.  Queued on
 * cuda_stream.
 * Errors: W2_ERR_ARG (NULL, misaligned, n outside [1, 4096]), W2_ERR_CUDA. */
w2_status w2_hermitian_eigvals(void *a, int32_t n, int32_t batch, double *eig, void *cuda_stream);

/* Release every resource of the context (NULL is ignored). */
void w2_destroy(w2_ctx *ctx);

/* Static, human-readable name of a status code. */
const char *w2_status_string(w2_status s);
/* The CUDA runtime's message for the error behind the calling thread's most
 * recent W2_ERR_CUDA (a static string; "no CUDA error recorded" if none). */
const char *w2_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Host-side fault injection for the allocation paths.  Every device and
 * pinned-host allocation the library makes (contexts, batches, networks,
 * patch tables, staging buffers, scratch) goes through one counter.
 * w2_debug_fail_alloc(n), n >= 0, makes the n-th allocation from now (0: the
 * next one) fail as if the device were full, once; the call that made it
 * returns W2_ERR_OOM and releases what it had taken.  n < 0 disarms.  No
 * allocation is attempted for the failed one, so nothing on the device is
 * touched.  w2_debug_alloc_count() is the number of allocations attempted
 * since the library was loaded (injected failures included), so a test can
 * count a call's allocations and then fail each one in turn.  Process-wide,
 * not thread-safe against concurrent allocating calls on other threads.
 * Errors: none (always W2_OK). */
w2_status w2_debug_fail_alloc(int32_t n);
int64_t w2_debug_alloc_count(void);

/* ------------------------------------------------------------------------
 * Encoders and one-tile self-test of the 5th-generation tensor-core path
 * (tcgen05 MMA with a TMEM accumulator, operands in shared memory).
 *
 * w2_debug_umma_smem_desc: the 64-bit shared-memory matrix descriptor of a
 * no-swizzle operand: start address (bytes, shared window), leading-dimension
 * byte offset (distance between core matrices adjacent along K) and
 * stride-dimension byte offset (along M or N); each a multiple of 16 below
 * 256 KB.  w2_debug_umma_idesc: the 32-bit instruction descriptor of a
 * kind::f16 MMA with BF16 A and B and an FP32 accumulator of M x N, A and B
 * K-major (0) or MN-major (1).  w2_debug_umma_tile_off: byte offset of
 * element (r, c) of a 16-bit matrix with ncol columns in the tiled layout
 * (8 x 8 core matrices of 128 contiguous bytes, row-major over the tiles).
 * Pure host functions, no device use, no errors.
 *
 * w2_debug_umma_gemm: one CTA computes D = A B (A: M x K, B: K x N, both
 * row-major BF16 bit patterns in device memory; M = 64 or 128, N a multiple
 * of 16 up to 64 (of 8 for M = 64), K = 16, 32, 48 or 64) on one tcgen05
 * MMA chain, after writing the marker word
 * 0x7fc0dead to TMEM columns [0, 2N) of all 128 lanes, and copies those
 * columns to dump (device, [128][2N] 32-bit words, lane-major).  swap = 1
 * passes the two core-matrix strides to the descriptor the other way round
 * (for the test that tells the two conventions apart; both stay inside the
 * operand's buffer).  Synchronises the device.  Errors: W2_ERR_ARG (shape or
 * pointer), W2_ERR_UNSUPPORTED (not a compute-capability 10.x device),
 * W2_ERR_TIMEOUT (the MMA's completion was not seen within about a second),
 * W2_ERR_CUDA. */
uint64_t w2_debug_umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo);
uint32_t w2_debug_umma_idesc(int32_t M, int32_t N, int32_t a_mn, int32_t b_mn);
uint32_t w2_debug_umma_tile_off(int32_t r, int32_t c, int32_t ncol);
w2_status w2_debug_umma_gemm(int32_t M, int32_t N, int32_t K, int32_t a_mn, int32_t b_mn, int32_t swap,
                             const uint16_t *A, const uint16_t *B, uint32_t *dump);

#ifdef __cplusplus
}
#endif

#endif /* W2_H */
