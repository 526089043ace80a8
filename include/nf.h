/*
 * nf.h - C ABI of the GB300 near-field force library (libnf).
 *
 * The library computes the near-field part of the Abacus force split
 * (Garrison et al., "The Abacus Cosmological N-body Code"): particles are
 * binned into a periodic K^3 grid of cells, and every particle receives the
 * spline-softened 1/r^2 acceleration of every particle in the (2R+1)^3 cells
 * around its own cell, with the source image taken in the unwrapped neighbour
 * cell (Sec. "Force Solver": exact near/far split; Sec. "GPU Near-Field
 * Computation": 5^3 neighbour cells for R = 2).
 *
 * Conventions shared by every entry point
 *   - Every pointer named pos, g, acc, grad, rel, perm, cell_offsets or ws is
 *     CUDA device memory owned by the caller.  Host-side arrays are marked
 *     "host".  The library allocates no memory.
 *   - `stream` is a cudaStream_t passed as void*.  Every call only enqueues
 *     work on that stream and returns; none of them synchronises, except
 *     nf_status_read.
 *   - Positions are FP32 [N][3] in box units.  Coordinates outside [0, box)
 *     are taken periodically.  Masses are all 1/N and G = 1 (the paper's
 *     particle state has no mass field, Sec. "Memory Model").
 *   - `eps` is the Plummer-equivalent softening in box units.  Internally the
 *     spline softening length is eps_s = 2.16 eps (Sec. "Force Softening").
 *     The pair force is Eq. (spline):
 *         F(d) = [10 - 15u + 6u^2] d / eps_s^3  for u = |d|/eps_s < 1,
 *         F(d) = d / |d|^3                      otherwise,
 *     with d = x_j - x_i, so the acceleration of i points towards j.
 *   - Arguments are checked on the host before anything is enqueued.  A
 *     rejected call returns NF_ERR_ARG or NF_ERR_WORKSPACE and launches
 *     nothing.  The checks are: N >= 1, N < 2^31; box > 0 and finite;
 *     K >= 2R+1 (else the stencil would count a cell twice) and K^3 < 2^31;
 *     1 <= R <= NF_MAX_R; eps > 0 with 1e-5 w <= eps_s <= R w, w = box/K
 *     (the softening must return to 1/r^2 inside the near field,
 *     Sec. "Force Softening"); non-null pointers; ws_bytes large enough.
 *   - Problems found on the device (non-finite coordinates) are recorded in a
 *     status word inside the workspace; nf_status_read returns it.  A
 *     non-finite particle is placed at the centre of cell 0 so the call
 *     still completes; its outputs and those of its neighbours are then
 *     meaningless.
 *   - Every call is asynchronous and can be captured in a CUDA graph.  Calls
 *     that share a workspace must not run concurrently.
 *   - Return value: an nf_status.  nf_last_error() describes the last
 *     non-OK return of the calling thread.
 */
#ifndef NF_H
#define NF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NF_MAX_R 4

typedef enum {
    NF_OK = 0,
    NF_ERR_ARG = 1,        /* invalid argument (checked on the host, nothing launched) */
    NF_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    NF_ERR_WORKSPACE = 3,  /* ws is NULL or ws_bytes is below the required size */
    NF_ERR_NONFINITE = 4,  /* device status: a coordinate was NaN or infinite */
    NF_ERR_TIMEOUT = 5,    /* device status: a bounded device-side wait gave up */
    NF_ERR_CORRUPT = 6     /* device status (debug mode): a workspace guard block was overwritten */
} nf_status;

/* Message for the last non-OK return on the calling thread ("" if none). */
const char *nf_last_error(void);

/* Library version string. */
const char *nf_version(void);

/* ------------------------------------------------------------------------ */
/* Sizes                                                                     */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace that nf_bin, nf_forces and nf_forces_adjoint need
 * for one box of N particles on a K^3 grid with radius R.  Returns 0 for
 * arguments nf_forces would reject.  The workspace's first 256 bytes hold the
 * device status word read by nf_status_read. */
size_t nf_workspace_bytes(int64_t N, int K, int R);

/* ------------------------------------------------------------------------ */
/* Binning (Sec. "Force Accuracy" overview: FP32 offsets from cell centres;  */
/* Sec. "Two-Stage Execution": the K^3 cell grid)                            */
/* ------------------------------------------------------------------------ */

/* Stable counting sort of N particles into K^3 cells.
 *   pos           [N][3] FP32, box units (input).
 *   cell_offsets  [K^3 + 1] int32 (output): first sorted slot of cell
 *                 c = (cx*K + cy)*K + cz; cell_offsets[K^3] = N.
 *   rel           [N][4] FP32 (output), sorted by cell, input order inside a
 *                 cell: (t_x - c_x - 1/2, t_y - c_y - 1/2, t_z - c_z - 1/2,
 *                 bits of the int32 original index), where t = x K / box is
 *                 formed in FP64 and c = floor(t); each offset is rounded once
 *                 from FP64 to FP32, so it lies in [-1/2, 1/2] cell widths.
 *                 Must be 16-byte aligned.
 *   perm          [N] int32 (output): sorted slot -> original index.
 * The result is bit-exact: it equals the plain CPU definition above. */
int nf_bin(const float *pos, int64_t N, double box, int K,
           int32_t *cell_offsets, float *rel, int32_t *perm,
           void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Forces (Sec. "GPU Near-Field Computation"; Eq. (spline))                  */
/* ------------------------------------------------------------------------ */

/* Near-field accelerations of one periodic box.
 *   pos  [N][3] FP32 box units (input).
 *   acc  [N][3] FP32 (output), original particle order:
 *        a_i = (1/N) sum_{j in N(i)} F(x_j - x_i), the sum running over the
 *        (2R+1)^3 cells around i's cell (j = i included; it adds 0).
 *   net  [3] FP64 (output) or NULL: sum_i (1/N) a_i of the FP32 results,
 *        accumulated in FP64 (zero up to roundoff by Newton's third law).
 * The pair arithmetic runs in FP32 on cell-relative coordinates.  The 2R+1
 * pencil partial sums that reach each particle are added without rounding
 * error into an FP32 (hi, lo) pair (a TwoSum cascade), multiplied by the box
 * scale m/w^2 held as a float pair, and rounded once to FP32. */
int nf_forces(const float *pos, int64_t N, double box, int K, int R, double eps,
              float *acc, double *net, void *ws, size_t ws_bytes, void *stream);

/* nf_forces plus the top-hat density estimate the paper's kernel accumulates
 * as a 4th component of the acceleration (Sec. "Force Kernel": b^2 - r^2 for
 * r < b, "nearly for free" next to the distances the force needs).
 *   b    top-hat radius in box units, 0 < b <= R w (the ball must lie inside
 *        the near field; checked, NF_ERR_ARG otherwise);
 *   acc  as nf_forces (bit-identical to nf_forces for the same inputs);
 *   rho  [N] FP32 (output), original order:
 *        rho_i = sum_{j in N(i), |x_j - x_i| < b} (1 - |x_j - x_i|^2 / b^2),
 *        the particle itself included (it contributes 1). */
int nf_forces_density(const float *pos, int64_t N, double box, int K, int R, double eps,
                      double b, float *acc, float *rho, void *ws, size_t ws_bytes, void *stream);

/* Where nf_forces_density's top-hat term runs (process-wide; not thread-safe
 * against running calls).  Both modes give bit-identical acc and rho; the
 * choice only moves work:
 *   1 fused     the term is added in every pair-kernel stage whose sources
 *               can lie within b of a sink;
 *   2 deferred  those stages track their smallest r^2 (which the softening
 *               test needs anyway) and add the term in a second sweep over
 *               the stage only when some pair is closer than b; cheap for a
 *               small b (the friends-of-friends scale of the paper);
 *   0 auto      (default) deferred for b <= w / 4, fused above.
 * nf_set_density_mode returns NF_ERR_ARG for any other value. */
int nf_set_density_mode(int mode);
int nf_get_density_mode(void);

/* Adjoint of nf_forces: for a loss L with g = dL/da,
 *   g     [N][3] FP32 (input), original order;
 *   grad  [N][3] FP32 (output), original order:
 *         dL/dx_i = (1/N) sum_{j in N(i)} J(x_j - x_i) (g_j - g_i),
 *         J(d) = f(|d|) I + (f'(|d|)/|d|) d d^T the Jacobian of F (F = f d),
 *         J(0) = f(0) I.
 * The cell assignment is the one nf_forces uses for the same positions (the
 * gradient of the piecewise-smooth map with cells held fixed).  It is not
 * in the paper; it is the exact derivative of the sum nf_forces computes.
 * Nothing is stored between the two calls: binning is recomputed. */
int nf_forces_adjoint(const float *pos, const float *g, int64_t N, double box,
                      int K, int R, double eps, float *grad,
                      void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched boxes and tuning                                                  */
/* ------------------------------------------------------------------------ */

/* One box of a batch.  Boxes are packed back to back: box b's particles are
 * rows [pos_offset, pos_offset + N) of pos_cat/acc_cat, and pos_offset must
 * equal the sum of N over the boxes before b. */
typedef struct {
    int64_t N;
    int64_t pos_offset;
    double box;
    double eps;
    int K;
    int R;
} nf_box;

/* Shape of the force kernel's work (picked by the autotuner or by hand).
 *   sinks_per_lane  sinks each lane keeps in registers: 1 to 4
 *                   (a sink chunk is 32 * sinks_per_lane particles);
 *   stage           sources staged in shared memory per step: 64 or 128;
 *   warps_per_block 4 or 8;
 *   blocks_per_sm   resident blocks of the persistent kernel per SM, 0 = as
 *                   many as fit.  Asking for 24 or more warps per SM
 *                   (warps_per_block * blocks_per_sm) with sinks_per_lane <= 2
 *                   selects the register-lean build of the kernel (at most
 *                   85 registers per thread); asking for 1 with stage 128
 *                   and 3 or 4 sinks per lane selects the build that has the
 *                   whole register file (up to 255 registers per thread;
 *                   not for nf_forces_density, which then runs its usual
 *                   build at one block per SM).
 * Unsupported combinations are rejected with NF_ERR_ARG.  The built-in
 * defaults are below. */
typedef struct {
    int sinks_per_lane;
    int stage;
    int warps_per_block;
    int blocks_per_sm;
} nf_tuning;

/* The tunings used when no tuning is given: one for the forward calls
 * (nf_forces, nf_forces_density, nf_forces_batched, the time steps and
 * nf_forces_total) and one for the adjoint calls (nf_forces_adjoint,
 * nf_forces_adjoint_batched).  The built-in defaults, measured best on GB300,
 * are {4, 128, 8, 0} forward and {4, 128, 8, 1} adjoint.
 * nf_set_default_tuning copies *t (validated) into both; NULL restores both
 * built-ins.  nf_set_default_tuning_adjoint sets the adjoint's alone (NULL:
 * its built-in).  All are process-wide and not thread-safe against running
 * calls. */
int nf_set_default_tuning(const nf_tuning *t);
void nf_get_default_tuning(nf_tuning *t);
int nf_set_default_tuning_adjoint(const nf_tuning *t);
void nf_get_default_tuning_adjoint(nf_tuning *t);

/* Workspace for a batch (host array boxes[nboxes]); 0 if the batch is invalid. */
size_t nf_workspace_bytes_batched(const nf_box *boxes, int nboxes);

/* Near-field accelerations of nboxes independent periodic boxes in one pass:
 * one binning over all boxes, one work list, one persistent force launch and
 * one combine.  Each box uses its own N (mass 1/N), box, K, R and eps.
 *   boxes    host array [nboxes];
 *   pos_cat  [sum N][3] FP32 (input), acc_cat [sum N][3] FP32 (output);
 *   net      [nboxes][3] FP64 (output) or NULL: per-box sum of m a;
 *   tune     NULL = default tuning.
 * Equivalent to nf_forces on each box (same arithmetic, bit-identical
 * results for the same tuning). */
int nf_forces_batched(const nf_box *boxes, int nboxes, const float *pos_cat,
                      float *acc_cat, double *net, const nf_tuning *tune,
                      void *ws, size_t ws_bytes, void *stream);

/* Adjoint of nf_forces_batched (same packing; g_cat and grad_cat [sum N][3]). */
int nf_forces_adjoint_batched(const nf_box *boxes, int nboxes, const float *pos_cat,
                              const float *g_cat, float *grad_cat,
                              const nf_tuning *tune, void *ws, size_t ws_bytes,
                              void *stream);

/* ------------------------------------------------------------------------ */
/* Forces without a caller-provided workspace                                */
/* ------------------------------------------------------------------------ */

/* Size of the fixed scratch array behind nf_forces_noalloc (32 MiB). */
#define NF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* nf_forces for callers that cannot allocate device memory.  This entry point
 * is an addition of this library; the paper has no counterpart.
 *
 * Who it is for: code that may only touch the buffers it is handed and cannot
 * call cudaMalloc to make a workspace, for example a plugin inside a host
 * program whose device memory is owned by that program's own pool allocator,
 * or a caller that must not allocate while other work is being captured.
 *
 * What it does: exactly what nf_forces does with the same arguments (pos, acc
 * and net are still the caller's device buffers), but its scratch space is a
 * fixed array of NF_NOALLOC_SCRATCH_BYTES compiled into the library instead
 * of a workspace.  Every GPU that loads the library keeps that array until
 * the process exits.  The call allocates nothing and frees nothing.
 *
 * Limits and rules:
 *   - A problem whose workspace (nf_workspace_bytes with the default tuning)
 *     is larger than the array is rejected with NF_ERR_WORKSPACE and a
 *     message; nothing is launched.  Use nf_forces with your own workspace
 *     for larger boxes.  Other bad arguments give NF_ERR_ARG as for nf_forces.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the one array, and it keeps the contents of the last
 *     call; each call clears the parts that must start at zero itself.  Calls
 *     that can overlap on the GPU (other streams, other host threads) race on
 *     the array and corrupt each other: order them on one stream.
 *   - The array's device status word is not exposed; check the input for
 *     non-finite coordinates on the caller's side if that matters. */
int nf_forces_noalloc(const float *pos, int64_t N, double box, int K, int R, double eps,
                      float *acc, double *net, void *stream);

/* ------------------------------------------------------------------------ */
/* Cell multipoles (Sec. "Computation of the Cell Multipoles")               */
/* ------------------------------------------------------------------------ */

#define NF_MAX_MULTIPOLE_ORDER 16

/* Complete-basis multipoles of every cell, Eq. (multipoles), in FP64:
 *     M[cell][t] = sum over the particles q of the cell of x_q^a y_q^b z_q^c,
 * (x, y, z) the displacement of q from the centre of its cell in box units
 * (unit masses; multiply by the particle mass for mass moments).  Terms t run
 * over a = 0..p, then b = 0..p-a, then c = 0..p-a-b; there are
 * (p+3)(p+2)(p+1)/6 of them.  The particles are binned first (as nf_bin);
 * cells are numbered (cx*K + cy)*K + cz.  M is [K^3][(p+3)(p+2)(p+1)/6]
 * doubles in device memory; 0 <= p <= NF_MAX_MULTIPOLE_ORDER. */
int nf_multipoles(const float *pos, int64_t N, double box, int K, int p, double *M,
                  void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Far field (Sec. "Far-field Computation")                                  */
/* ------------------------------------------------------------------------ */

/* The far field of the paper's near/far split: cell multipoles (Eq.
 * (multipoles)), their convolution over the K^3 grid with the derivatives
 * tensor (by FFT), and the acceleration from the resulting Taylor series of
 * the potential in every cell.  The derivatives include every periodic image
 * of the box, the images of the central and near-field cells included, minus
 * the one image per cell pair that nf_forces computes directly, so
 * nf_forces + nf_far_forces is the periodic (Ewald-summed) force up to the
 * multipole order (same section).  Expansions are truncated at total order p:
 * Taylor index n and multipole index k with |n| + |k| <= p, both in the
 * complete basis of (p+3)(p+2)(p+1)/6 terms (ordered as in nf_multipoles).
 * The uniform background of Ewald summation is included (the mean density
 * exerts no force).  Arithmetic: FP64 for the derivatives; double-float or
 * FP64 for the rest (see nf_far_set_arith).  The 3-D transforms are this
 * library's own kernels: radix-4/2 in double-float for a power-of-two K, and
 * mixed-radix (factors 4, 2, 3, 5, 7 and any larger prime) for any K, in
 * double-float or IEEE FP64. */
#define NF_MAX_FAR_ORDER 12

/* Bytes of a derivatives buffer for grid K and order p (0 if out of range):
 * a 256-byte header, the convolution's tables and the transformed
 * derivatives, (p+3)(p+2)(p+1)/6 FP64 fields of K*K*(K/2+1) values, a
 * second copy as double-float pairs with the pairs' coefficients in that
 * form, and the transforms' twiddles (FP64 and double-float).  The transform
 * of a term of even order is real and of odd order imaginary (the
 * derivatives have definite parity, Sec. "Far-field Computation"), so one
 * real number per term and frequency is kept. */
size_t nf_derivatives_bytes(int K, int p);

/* Workspace bytes of nf_far_forces (N particles) and of nf_derivatives (any
 * N >= 1 will do): the binning, the multipoles and two complex spectra.
 * 0 if the arguments are out of range. */
size_t nf_far_workspace_bytes(int64_t N, int K, int p);

/* Precomputes the derivatives tensor of grid K, near-field radius R, order p
 * and box side box into `derivs` (device memory, caller-owned, 256-byte
 * aligned, at least nf_derivatives_bytes(K, p) bytes); ws is a device
 * workspace of nf_far_workspace_bytes(1, K, p) bytes.  Asynchronous on
 * `stream` (its host-built tables are copied from pageable memory, so the
 * call returns once they are staged).
 * Errors: NF_ERR_ARG for K < 2R+1, R outside 1..NF_MAX_R, p outside
 * 0..NF_MAX_FAR_ORDER, (p+3)(p+2)(p+1)/6 K^3 >= 2^31 (32-bit field offsets;
 * K <= 235 at p = 8), box <= 0 or NULL pointers; NF_ERR_WORKSPACE for a
 * short or misaligned buffer; NF_ERR_CUDA if a launch fails. */
int nf_derivatives(int K, int R, int p, double box, void *derivs, size_t derivs_bytes,
                   void *ws, size_t ws_bytes, void *stream);

/* Far-field accelerations (m = 1/N, G = 1) of N particles (pos FP32 [N][3],
 * box units, wrapped into [0, box) like nf_forces) from a derivatives buffer
 * made by nf_derivatives for the same K, R, p and box:
 *   acc_far  FP64 [N][3] in input order, or NULL;
 *   acc_add  FP32 [N][3] in input order, or NULL: the far acceleration is
 *            added to it (e.g. to the output of nf_forces for the total);
 *   taylors  FP64 [K^3][(p+3)(p+2)(p+1)/6] Taylor coefficients, or NULL:
 *            the potential in cell c is -m sum_t taylors[c][t] x^a y^b z^c,
 *            x the displacement from the cell centre in box units.
 * All device memory, caller-owned; ws holds nf_far_workspace_bytes(N, K, p)
 * bytes.  Asynchronous on `stream` and graph-capturable.  Errors: as
 * nf_derivatives; NF_ERR_ARG also when `derivs` was made for another
 * (K, R, p, box) by this process. */
int nf_far_forces(const float *pos, int64_t N, double box, int K, int R, int p,
                  const void *derivs, size_t derivs_bytes, double *acc_far, float *acc_add,
                  double *taylors, void *ws, size_t ws_bytes, void *stream);

/* The periodic force, near + far, in one call: acc (FP32 [N][3], input
 * order) = nf_forces(pos) + the far field of order p, binning the particles
 * once for both.  derivs from nf_derivatives for (K, R, p, box); ws a
 * near-field workspace (nf_workspace_bytes(N, K, R)), ws_far a far-field one
 * (nf_far_workspace_bytes(N, K, p)).  Errors as nf_forces and nf_far_forces. */
int nf_forces_total(const float *pos, int64_t N, double box, int K, int R, double eps, int p,
                    const void *derivs, size_t derivs_bytes, float *acc, void *ws, size_t ws_bytes,
                    void *ws_far, size_t ws_far_bytes, void *stream);

/* Arithmetic of the far-field call (multipoles, convolution, Taylor
 * evaluation), process-wide.  The paper keeps every internal
 * far-field computation in double precision to avoid round-off build-up.
 * NF_FAR_FP64 does so with IEEE binary64 arithmetic, which GB300 runs at
 * 1/64 of its FP32 rate.  NF_FAR_DOUBLE_FLOAT (the default) keeps each value
 * as an unevaluated sum of two FP32 numbers, held exact by error-free
 * transformations, on the FP32 pipe: about 48 significant bits.  Both modes
 * give the same far field to 1e-12 of its largest value (tested).  In
 * double-float mode the transforms and the k-space product are double-float
 * too; in FP64 mode they are FP64.  The derivatives are FP64 in both.
 * nf_far_set_arith returns
 * NF_ERR_ARG for another mode; calls already enqueued keep the mode they
 * were enqueued with. */
#define NF_FAR_FP64 0
#define NF_FAR_DOUBLE_FLOAT 1
int nf_far_set_arith(int mode);
int nf_far_get_arith(void);

/* Releases what the far-field calls keep between calls.  The transforms are
 * the library's own kernels and keep no plans or tables of their own, so
 * there is nothing to release; kept so that callers written for earlier
 * versions still link.  Always NF_OK. */
int nf_far_release(void);

/* ------------------------------------------------------------------------ */
/* Time stepping (Sec. "Time Stepping": Kick-Drift-Kick leapfrog with a      */
/* global time step, Eq. (timestep))                                         */
/* ------------------------------------------------------------------------ */

/* Parameters of the time-step criterion, Eq. (timestep), written for the time
 * step dt at scale factor a = 1 (da = a H dt):
 *     dt = min(eta_h / hubble, eta_acc * max(min_c [v_rms / a_max]_c,
 *                                            v_rms,global / a_max,global)),
 * v_rms per cell without subtracting the cell's mean velocity (as the paper
 * specifies), a_max the largest |a| in the cell; cells with a_max = 0 are
 * skipped; hubble = 0 drops the Hubble limit.  eta_acc > 0 is required. */
typedef struct {
    double eta_acc;
    double eta_h;
    double hubble;
} nf_step_params;

/* Global time step of the particles (host array prm; dt is ONE double in device
 * memory, written).  Bins pos (same rule as nf_bin) to group the particles by
 * cell, then reduces vel and acc ([N][3] FP32, original order) per cell.
 * If nothing limits the step (all accelerations zero and hubble = 0) dt = +inf. */
int nf_timestep(const float *pos, const float *vel, const float *acc, int64_t N, double box, int K,
                const nf_step_params *prm, double *dt, void *ws, size_t ws_bytes, void *stream);

/* One leapfrog step in place, all on the device:
 *     vel += acc dt/2;  pos = wrap(pos + vel dt) into [0, box);
 *     acc = nf_forces(pos);  vel += acc dt/2;
 * acc must hold the accelerations at the input positions (from nf_forces or
 * the previous step).  dt is ONE double in device memory: it is read for this
 * step and, when prm != NULL, overwritten with the next step's dt from
 * Eq. (timestep) at the new state; so a loop of steps needs no host round trip
 * and can be captured in a CUDA graph.  Arguments as nf_forces otherwise. */
int nf_kdk_step(float *pos, float *vel, float *acc, int64_t N, double box, int K, int R, double eps,
                double *dt, const nf_step_params *prm, void *ws, size_t ws_bytes, void *stream);

/* One leapfrog step with the total force, near + far, all on the device:
 *     vel += acc dt/2;  pos = wrap(pos + vel dt);
 *     acc = nf_forces(pos) + nf_far_forces(pos);  vel += acc dt/2;
 * then, when prm != NULL, dt = Eq. (timestep) at the new state (as
 * nf_kdk_step).  acc (FP32 [N][3]) must hold the total acceleration at the
 * input positions.  derivs comes from nf_derivatives for (K, R, p, box) (the
 * far field, Sec. "Far-field Computation"); ws is
 * a near-field workspace (nf_workspace_bytes(N, K, R)) and ws_far a far-field
 * one (nf_far_workspace_bytes(N, K, p)).  Graph-capturable.  Errors as
 * nf_kdk_step and nf_far_forces. */
int nf_kdk_step_far(float *pos, float *vel, float *acc, int64_t N, double box, int K, int R, double eps,
                    int p, const void *derivs, size_t derivs_bytes, double *dt, const nf_step_params *prm,
                    void *ws, size_t ws_bytes, void *ws_far, size_t ws_far_bytes, void *stream);


/* ------------------------------------------------------------------------ */
/* Status and statistics                                                     */
/* ------------------------------------------------------------------------ */

/* Debug mode (process-wide, off by default): every workspace region is
 * followed by a 256-byte guard block, so workspace sizes grow - size
 * workspaces after switching it.  Each call fills the guards when it starts
 * and checks them when it ends; an overwritten guard (an out-of-bounds write
 * by a kernel, or by anyone else) sets NF_ERR_CORRUPT in the status word.
 * This stands in for a memory checker where none can run. */
int nf_set_debug(int on);

/* Debug mode: checks the guard blocks of `ws` now (enqueued on `stream`);
 * read the result with nf_status_read.  NF_ERR_ARG if debug mode is off. */
int nf_debug_check(void *ws, void *stream);

/* Synchronises `stream`, then returns the device status word of the last call
 * that used `ws` (NF_OK, NF_ERR_NONFINITE, NF_ERR_TIMEOUT or NF_ERR_CORRUPT),
 * or NF_ERR_CUDA if synchronisation failed.  Every call clears the word when
 * it starts. */
int nf_status_read(void *ws, void *stream);

/* Statistics of the last call that used `ws`, copied to the host after a
 * stream synchronisation (host array out[4]):
 *   out[0] = pair interactions computed, P = sum_c n_c S_c (self pairs
 *            included), summed over boxes;
 *   out[1] = work items (sink chunks) in the persistent queue;
 *   out[2] = largest cell occupancy;
 *   out[3] = sink lanes issued (32 * sinks_per_lane rounded up per chunk),
 *            so out[0] / (out[3] * sources) measures lane utilisation. */
int nf_stats_read(void *ws, int64_t *out, void *stream);

/* Stages of the pair kernel in the last force, adjoint or density call that
 * used `ws` (a measurement aid; no counterpart in the paper), host array
 * out[3], after a stream synchronisation:
 *   out[0] = stages (a warp's pass over one batch of staged sources);
 *   out[1] = stages computed on the exact path from the start (the sources of
 *            the work item's own cell: self pairs and the closest neighbours);
 *   out[2] = stages computed on the fast path (f = r^-3) and computed again on
 *            the exact path because a pair closer than eps_s met there
 *            (Eq. (spline)).
 * Returns NF_ERR_ARG for NULL pointers, NF_ERR_CUDA if a CUDA call fails. */
int nf_stage_stats_read(void *ws, int64_t *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* Device time of the stages of a recent nf_forces / nf_forces_adjoint /
 * batched call, from CUDA events recorded on the caller's stream around each
 * stage while profiling is on (milliseconds):
 *   bin_ms       cell ids, offsets, radix sort, cell-centred offsets;
 *   worklist_ms  pencil sizes, cost order, work items (and the gather of g);
 *   pair_ms      the persistent force or adjoint kernel alone;
 *   combine_ms   combine of the partial sums (error-free FP32 TwoSum, one row
 *                per particle in input order) and the FP64 net force;
 *   total_ms     first event to last. */
typedef struct {
    double bin_ms;
    double worklist_ms;
    double pair_ms;
    double combine_ms;
    double total_ms;
} nf_profile;

#define NF_PROFILE_RING 8

/* Turns per-stage event recording on (1) or off (0), process-wide, and
 * forgets earlier records.  While it is on, calls must not be captured into a
 * CUDA graph.  Not thread-safe against concurrent calls. */
int nf_profile_enable(int on);

/* Synchronises on the events of a profiled call and fills *out (host).
 * back = 0 is the most recent profiled call, 1 the one before, and so on up
 * to NF_PROFILE_RING - 1.  Returns NF_ERR_ARG if there is no such call. */
int nf_profile_read(int back, nf_profile *out);

/* Device time of the stages of a recent nf_far_forces call (same event ring
 * and the same rules as nf_profile_read; read a far call with this function):
 *   bin_ms          cell ids, offsets, radix sort, cell-centred offsets;
 *   multipoles_ms   the cell multipoles;
 *   convolution_ms  forward FFT, k-space product with the derivatives, inverse FFT;
 *   taylor_ms       the Taylor-series evaluation at every particle;
 *   total_ms        first event to last. */
typedef struct {
    double bin_ms;
    double multipoles_ms;
    double convolution_ms;
    double taylor_ms;
    double total_ms;
} nf_far_profile;

int nf_far_profile_read(int back, nf_far_profile *out);

/* Number of kernels libnf has launched in this process (all entry points). */
int64_t nf_kernel_launches(void);


#ifdef __cplusplus
}
#endif

#endif /* NF_H */
