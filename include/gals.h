/*
 * gals.h -- C ABI of the GB300 gradient-augmented level set (GALS) library.
 *
 * The library advances a level set function phi together with its gradient
 * psi = grad phi on a uniform grid with the gradient-augmented CIR scheme of Nave,
 * Rosales and Seibold (arXiv 0905.3409): for every grid node the characteristic is
 * traced back one time step with the superconsistent Shu-Osher RK3 scheme and the
 * Jacobian of that backward map (Sec. 5.1, Ex. "superconsistent Shu-Osher"); the
 * bi-/tri-cubic Hermite interpolant of the cell containing the foot point
 * (Sec. 2.3, eq. p-cubic_interpolant) gives phi+ = H(foot) and psi+ = J^T grad H(foot)
 * (eq. superconsistency); the mixed derivatives the interpolant needs are rebuilt
 * from the new gradients by central differences (Sec. 2.3, approach A).
 *
 * All arithmetic of a step runs in hand-written CUDA kernels for sm_103a, in FP32;
 * diagnostics accumulate in FP64 or exact integers.  There is no CPU fallback.
 *
 * Conventions for every call:
 *   - Every function returns gals_status: GALS_OK (0) or a negative error code.
 *     No exception or signal crosses the ABI.  gals_last_error() gives a message.
 *   - Grid data are SoA FP32 planes, x fastest: node (i,j,k) of a plane is element
 *     (k*n[1] + j)*n[0] + i of a dense array of n[0]*n[1]*n[2] floats (n[2] = 1 in 2D).
 *   - Plane order: 2D  phi, phi_x, phi_y, phi_xy
 *                  3D  phi, phi_x, phi_y, phi_z, phi_xy, phi_xz, phi_yz, phi_xyz.
 *   - Device pointers must be memory of the current CUDA device, 4-byte aligned.
 *   - Work is ordered on the grid's CUDA stream.  gals_step returns before the GPU
 *     has finished; errors of asynchronous work surface at the next synchronising
 *     call (gals_read_state, gals_diagnostics, gals_synchronize).
 *   - Handles are not thread-safe: use one handle per host thread.
 *   - libgals_checked.so, built from the same sources with -DGALS_CHECKED, exports the
 *     same ABI; there the step kernels test every data-dependent index against its
 *     buffer, and an index outside it fails the next synchronising call with
 *     GALS_ERR_CUDA (the message names the source line).  The normal build has no tests.
 *   - The step, state, diagnostics and point-evaluation calls are NVTX ranges named after
 *     the call.
 */
#ifndef GALS_H
#define GALS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GALS_OK = 0,
    GALS_ERR_ARG = -1,         /* invalid argument (null, size, range, non-finite) */
    GALS_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    GALS_ERR_NOMEM = -3,       /* device allocation failed */
    GALS_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out */
    GALS_ERR_NONFINITE = -5,   /* non-finite values found where finite ones are required */
    GALS_ERR_STATE = -6,       /* call out of order (e.g. step before set_state) */
    GALS_ERR_UNSUPPORTED = -7  /* combination of options not implemented */
} gals_status;

enum { GALS_MEM_HOST = 0, GALS_MEM_DEVICE = 1 };

/* Storage of the mixed derivatives between steps.
 *   FULL     all 4 (2D) / 8 (3D) planes are written every step (the paper's stored
 *            representation, Sec. 5.2: the projection keeps per-node cross derivatives).
 *   COMPACT  only phi and psi are kept in memory between steps; the mixed derivatives
 *            are rebuilt from psi by the same central differences each time they are
 *            needed.  Results are bit-identical to FULL; it moves 24 instead of 32 bytes
 *            per 2D node update (32 instead of 64 in 3D). */
enum { GALS_LAYOUT_FULL = 0, GALS_LAYOUT_COMPACT = 1 };

typedef struct {
    int dim;            /* 2 or 3 */
    int n[3];           /* nodes per axis including both ends, each >= 4 (n[2] ignored in 2D) */
    double lo[3];       /* domain [lo, hi] per axis; node spacing h = (hi - lo)/(n - 1) */
    double hi[3];
    int layout;         /* GALS_LAYOUT_FULL (default 0) or GALS_LAYOUT_COMPACT */
    int cross_scheme;   /* GALS_CROSS_CENTRAL (default 0) or GALS_CROSS_CELL */
    void *cuda_stream;  /* cudaStream_t to order work on, or NULL for a library-owned stream */
} gals_grid_desc;

/* Mixed derivatives of the interpolation data (Sec. 2.3).  CENTRAL, approach (A): node
 * values by central differences of the gradients (one-sided at the box edges), rebuilt
 * after every step.  CELL, approach (B): computed inside each cell from the gradients at
 * its vertices (edge-centre differences, vertex weights 3/4, 3/4, -1/4, -1/4; in 3D
 * within each vertex's facet, phi_xyz from the double difference of psi_z over the
 * vertex's x-y facet); a node has no single value, so the state's mixed-derivative planes
 * are zero (set_state ignores given ones) and the step reads and writes phi and psi only.
 * The diagnostics sample the interpolant of the grid's scheme. */
enum { GALS_CROSS_CENTRAL = 0, GALS_CROSS_CELL = 1 };

/* Analytic velocity fields v(x, t) with exactly known Jacobian (Sec. 4 assumes both
 * "exactly accessible everywhere").  Coordinates are physical (not index) units. */
enum {
    GALS_VEL_CONST = 0,     /* v = c */
    GALS_VEL_ROTATION = 1,  /* rigid rotation about center with angular speed omega, w = 0 */
    GALS_VEL_VORTEX2D = 2,  /* v = (-Psi_y, Psi_x), Psi = (1/pi)cos(pi t/T) sin^2(pi x) sin^2(pi y) (Sec. 6.1.2) */
    GALS_VEL_DEFORM3D = 3,  /* u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z), v = -sin(2 pi x) sin^2(pi y) sin(2 pi z),
                               w = -sin(2 pi x) sin(2 pi y) sin^2(pi z), all times cos(pi t/T) (Sec. 6.2.4) */
    GALS_VEL_PSEUDO1D = 4,  /* eq. velocity_1 (Sec. 6.1.1) */
    GALS_VEL_FOURIER2D = 5, /* v = (-Psi_y, Psi_x), Psi = sum_m a_m sin(k_m pi x) sin(l_m pi y) cos(2 pi n_m t + chi_m) */
    GALS_VEL_WAVES2D = 6    /* v = (-Psi_y, Psi_x), Psi = sum_m a_m sin(kx_m x + ky_m y + phase_m) cos(2 pi n_m t + chi_m):
                               plane waves of any wave vector, a field with no separable form
                               whose every evaluation costs one sine and cosine per mode (a costly
                               velocity; not in the paper) */
};

/* Backward trace of one step. */
enum {
    GALS_TRACE_EULER = 0,     /* superconsistent forward Euler (Sec. 5.1, first order) */
    GALS_TRACE_RK3 = 1,       /* superconsistent Shu-Osher RK3 (Sec. 5.1), the default of Sec. 6 */
    GALS_TRACE_SURROGATE = 2, /* learned flow map (gals_surrogate_*), RK3 fallback; 2D FOURIER2D */
    GALS_TRACE_HEUN_PSI = 3   /* CIR form of Sec. 4: foot by Shu-Osher RK3, psi(foot) = grad H,
                                 then d psi/d tau = -(grad v) . psi along the characteristic
                                 by one step of Heun's method (not superconsistent) */
};

typedef struct gals_surrogate gals_surrogate;   /* opaque, owned by the library */

#define GALS_MAX_MODES 64
#define GALS_MAX_WAVES 1024

typedef struct {
    int kind;               /* GALS_VEL_* */
    int trace;              /* GALS_TRACE_* */
    double T;               /* modulation period of VORTEX2D / DEFORM3D */
    double omega;           /* ROTATION angular speed (counter-clockwise) */
    double center[3];       /* ROTATION center */
    double c[3];            /* CONST velocity */
    int nmodes;             /* FOURIER2D: number of modes, 1..GALS_MAX_MODES; WAVES2D: 1..GALS_MAX_WAVES */
    const double *modes;    /* FOURIER2D: host array of nmodes rows (a, k, l, n, chi); k, l integers
                               in 1..4, n >= 0.  WAVES2D: rows (a, kx, ky, phase, n, chi), n >= 0.
                               Copied during the call. */
    const gals_surrogate *surrogate;  /* GALS_TRACE_SURROGATE: the trained flow map (else NULL) */
} gals_velocity;

typedef struct gals_grid gals_grid;   /* opaque, owned by the library */

/* Create a grid and allocate its double-buffered device state on the current device.
 * Size limits: 2D at most 2^31 - 1 elements per plane (row pitch = n[0] rounded up to a
 * multiple of 4, times n[1]) and n[1] <= 917490; 3D n[1], n[2] <= 262140.
 * Errors: GALS_ERR_ARG (dim not 2/3, n < 4 or above the limits, hi <= lo, bad layout),
 * GALS_ERR_NOMEM, GALS_ERR_CUDA.  On error *out is set to NULL. */
gals_status gals_create_grid(const gals_grid_desc *desc, gals_grid **out);

/* Free the grid's device memory and stream (if library-owned).  NULL is accepted. */
gals_status gals_destroy_grid(gals_grid *grid);

/* Flags of gals_set_state. */
enum { GALS_SET_RECON_CROSS = 1 };  /* rebuild the mixed derivatives from the given gradients */

/* Load the state at time t0.  fields[p] points to plane p (layout above) in host or
 * device memory (memspace); the data are copied and the caller keeps ownership.
 * nfields = 1 + dim (phi and gradient; the mixed derivatives are then rebuilt from the
 * gradients, Sec. 2.3 approach A) or all planes (4 in 2D, 8 in 3D), whose mixed
 * derivatives are used as given unless flags has GALS_SET_RECON_CROSS.
 * The copy is stream-ordered; host sources are read before the call returns.
 * Errors: GALS_ERR_ARG (null pointers, wrong nfields, memspace), GALS_ERR_CUDA. */
gals_status gals_set_state(gals_grid *grid, const float *const *fields, int nfields,
                           int memspace, double t0, int flags);

/* Advance nsteps steps of size dt from the grid's current time (Sec. 4 steps 1-3 in the
 * superconsistent form of Sec. 5.1; M = P A of Sec. 5.2).  Step s uses the velocity at
 * the stage times of the step from t0 + s*dt.  Feet outside the box are clamped into it
 * (outflow or tangential boundaries need no data, Sec. 4.1).  nsteps > 1 is replayed
 * from cached CUDA graphs of at most 256 steps each (of one launch per step, or of one
 * persistent launch, see gals_set_time_loop); each graph reads the grid clock on the
 * device and advances it, so longer calls replay the same graph.  In 2D the graph splits each step into up to 4 bands of whole tile
 * rows, at least 2 tiles and the velocity's reach plus 4 rows high; a band of step s
 * depends only on itself and its two neighbouring bands at step s - 1, so the next step's
 * bands start while the current one drains (same results bit for bit).  Asynchronous on
 * the grid stream.
 * Errors: GALS_ERR_ARG (dt <= 0 or non-finite, nsteps < 0, bad velocity descriptor),
 * GALS_ERR_STATE (no state loaded), GALS_ERR_UNSUPPORTED (velocity kind not available in
 * this dimension), GALS_ERR_CUDA (launch failure). */
gals_status gals_step(gals_grid *grid, const gals_velocity *vel, double dt, int nsteps);

/* Time loop of gals_step calls with nsteps > 1.
 *   LAUNCHES    one launch per step, replayed from a cached CUDA graph (the default).
 *   PERSISTENT  where it applies (2D, FULL layout, approach A, the Euler / RK3 / Heun-psi
 *               traces, and feet at most 126 columns and 12 rows from their node by the
 *               velocity's speed bound) each run of up to 256 steps of a call (see
 *               gals_step) is one persistent launch: blocks take
 *               (step, tile) items in order and a tile of step s starts once the 3 x 3 tiles
 *               around it have finished step s - 1, so no step waits for the last tiles of
 *               the previous one to drain; elsewhere one launch per step.  On a GB300 it
 *               runs slower than LAUNCHES on the 4096^2 single vortex (0.148 ms per step
 *               against 0.128 ms for the banded graph): the per-tile flag fence and acquire
 *               cost more than the drained tails it saves.
 * Both give the same results bit for bit. */
enum { GALS_LOOP_LAUNCHES = 0, GALS_LOOP_PERSISTENT = 1 };

/* Select the time loop of later gals_step calls (default LAUNCHES); synchronises when it
 * changes.  Errors: GALS_ERR_ARG. */
gals_status gals_set_time_loop(gals_grid *grid, int mode);

/* The number of kernel launches the last gals_step call on the grid issued (its step
 * kernels, per band where the step is banded, and its coefficient-table and clock
 * kernels; 0 after nsteps = 0), for profiling.  Errors: GALS_ERR_ARG (NULL pointer). */
gals_status gals_last_step_launches(const gals_grid *grid, int64_t *launches);

/* Copy the current state out (all planes, or the first nfields).  In the COMPACT layout
 * the mixed derivatives are rebuilt first.  Synchronises the grid stream.
 * Errors: GALS_ERR_ARG, GALS_ERR_STATE, GALS_ERR_CUDA. */
gals_status gals_read_state(gals_grid *grid, float *const *fields, int nfields, int memspace);

/* Diagnostics of the current state (Sec. 6: e_max of eq. maximum_norm, volume loss
 * tables).  The interpolant is sampled at q^p cell-centred points per cell
 * (xi = (s + 1/2)/q); counts are exact integers, norms accumulate in FP64. */
typedef struct {
    int q;                         /* samples per cell and axis, 1..16 (0: no sampling) */
    const gals_grid *reference;    /* optional grid of the same shape: symmetric difference of
                                      {H < 0} and error norms against it */
} gals_diag_request;

typedef struct {
    double t;                      /* grid time */
    int64_t steps;                 /* steps taken since the last set_state */
    int64_t samples;               /* number of sample points (cells * q^p) */
    int64_t n_negative;            /* samples with H < 0 */
    double measure_negative;       /* area (2D) / volume (3D) of {H < 0} = n_negative * cell / q^p */
    int64_t n_symdiff;             /* samples where sign(H < 0) differs from the reference */
    double measure_symdiff;        /* its area / volume (interface-location error numerator) */
    double emax_phi;               /* max |phi - phi_ref| over nodes (eq. maximum_norm) */
    double emax_psi;               /* max over nodes of max_i |psi_i - psi_ref_i| */
    double l2_phi;                 /* sqrt(sum (phi - phi_ref)^2 * cell) in FP64 */
    int64_t nonfinite;             /* nodes with a non-finite value in any plane */
} gals_diag;

/* Errors: GALS_ERR_ARG (q out of range, reference of another shape), GALS_ERR_STATE,
 * GALS_ERR_NOMEM, GALS_ERR_CUDA.  Synchronises the grid stream. */
gals_status gals_diagnostics(gals_grid *grid, const gals_diag_request *req, gals_diag *out);

/* One step from a state in host memory to a state in host memory, for callers that keep
 * the field on the host.  in[p] (all planes, the layout of gals_set_state, mixed
 * derivatives used as given) is the state at time t0; it is advanced one step of dt
 * (as gals_step) and written to out[p] (all planes), and the grid keeps the new state
 * at t0 + dt for later calls.  The same result as gals_set_state, gals_step and
 * gals_read_state, bit for bit, but the grid is cut into bands of nodes along its last
 * axis (rows in 2D, z-levels in 3D): band b is copied in on one stream, stepped on the
 * grid stream once every band its feet can reach is in (from a bound of the velocity's
 * speed), and copied out on a third stream, so that with page-locked host buffers the
 * host-to-device copy of later bands, the device-to-host copy of earlier ones and the
 * step overlap.  in and out may be the same buffers.  Synchronises.
 * Errors: GALS_ERR_ARG (null pointers, dt <= 0, non-finite t0, bad velocity),
 * GALS_ERR_UNSUPPORTED (COMPACT layout, approach B, the surrogate trace, a velocity kind
 * not available in this dimension), GALS_ERR_CUDA, GALS_ERR_TIMEOUT. */
gals_status gals_step_host(gals_grid *grid, const gals_velocity *vel, double dt, double t0,
                           const float *const *in, float *const *out);

/* gals_step_host without the final wait: returns once the copies and the step are queued,
 * for callers that step a host-resident field repeatedly.  in[p] must stay valid and
 * unchanged, and out[p] must not be read, until gals_synchronize (or a synchronous host
 * step) returns.  Consecutive calls overlap: the copy-in of a band of the next call waits
 * only for the copy-out of the same band of this one, so out may be the next call's in (a
 * host-side time loop).  Other calls on the grid (gals_step, gals_set_state,
 * gals_read_state, ...) wait for the pending copies before they touch the state.  Errors
 * of the queued work surface at gals_synchronize.  Bit-identical to gals_step_host.
 * Errors: as gals_step_host. */
gals_status gals_step_host_async(gals_grid *grid, const gals_velocity *vel, double dt, double t0,
                                 const float *const *in, float *const *out);

/* Value, unit normal and curvature of the current state's interpolant at npoints points
 * (Sec. 3.4: every first and second derivative inside a cell from the p-cubic interpolant
 * of that cell; eq. surface_normal n = grad H / |grad H|; eq. curvature in 2D,
 * kappa = (H_xx H_y^2 - 2 H_x H_y H_xy + H_yy H_x^2) / |grad H|^3, and in 3D its extension
 * kappa = div(grad H / |grad H|), the sum of the principal curvatures).  points: npoints
 * rows of dim FP64 coordinates (x first); a point outside the box is clamped into it.
 * Outputs, any of which may be NULL: H[npoints], normal[npoints * dim], kappa[npoints]
 * (FP32; n = 0 and kappa = 0 where grad H = 0).  memspace applies to points and outputs
 * alike; host arrays are staged through a device buffer the grid keeps.  The mixed
 * derivatives come from the planes (approach A; rebuilt first in the COMPACT layout) or
 * per cell (approach B).  Synchronises.
 * Errors: GALS_ERR_ARG, GALS_ERR_STATE, GALS_ERR_NOMEM, GALS_ERR_CUDA. */
gals_status gals_eval_points(gals_grid *grid, const double *points, int64_t npoints, int memspace,
                             float *H, float *normal, float *kappa);

/* Wait for the grid's stream and any pending host-step copies; returns the first
 * asynchronous error, if any. */
gals_status gals_synchronize(gals_grid *grid);

/* Current grid time (host copy; advanced by gals_step at issue). */
double gals_time(const gals_grid *grid);

/* Device pointers of the current state planes (for zero-copy consumers); valid until
 * the next gals_step.  In the COMPACT layout the mixed-derivative planes are only valid
 * after gals_read_state.  Errors: GALS_ERR_ARG. */
gals_status gals_state_planes(gals_grid *grid, float **planes, int nplanes, int64_t *row_pitch);

/* Message of the last error on this grid (or of the last failed create if grid is NULL).
 * The pointer stays valid until the next call on the same grid. */
const char *gals_last_error(const gals_grid *grid);

/* Library version string. */
const char *gals_version(void);

/* Test hook for the failure path of the bounded device waits (not in the paper).  In the
 * checked build (libgals_checked.so) it sets, for grids created afterwards, how many
 * polls a step kernel's wait for its staged tile makes before the wait counts as lost
 * (default 2^24), and with skip_copy != 0 the tile copy that completes the wait is not
 * issued, so every wait runs out: the kernel records GALS_ERR_TIMEOUT's code in the
 * grid's error word and returns, and the next synchronising call on that grid returns
 * GALS_ERR_TIMEOUT.  gals_checked_wait_test(1u << 24, 0) restores the defaults.  The
 * normal build returns GALS_ERR_UNSUPPORTED and changes nothing.
 * Errors: GALS_ERR_ARG (polls < 1), GALS_ERR_UNSUPPORTED. */
gals_status gals_checked_wait_test(uint32_t polls, int skip_copy);

/* ------------------------------------------------------------------------------------
 * Batched 2D mode: many independent problems of uneven size advanced together, one
 * kernel launch per step over a work list of (problem, tile) items; runs of steps are
 * replayed from a cached CUDA graph.  Each problem evolves exactly as it would on its own
 * grid (same per-node arithmetic, Sec. 4 / Sec. 5.1), with its own velocity and time
 * step.  This mode is not in the paper: it batches the paper's step for throughput.
 * ------------------------------------------------------------------------------------ */
typedef struct gals_batch gals_batch;   /* opaque, owned by the library */

/* Create a batch of `count` 2D problems.  All descriptors must have dim 2 and the same
 * layout; the stream of descs[0] (or a library stream if NULL) orders all work.
 * Errors: GALS_ERR_ARG (count < 1, a descriptor invalid as for gals_create_grid),
 * GALS_ERR_NOMEM, GALS_ERR_CUDA. */
gals_status gals_create_batch(const gals_grid_desc *descs, int count, gals_batch **out);
gals_status gals_destroy_batch(gals_batch *batch);

/* Load problem `index` (0-based); arguments as gals_set_state.  In the COMPACT layout the
 * mixed derivatives are always rebuilt from the gradients. */
gals_status gals_batch_set_state(gals_batch *batch, int index, const float *const *fields,
                                 int nfields, int memspace, double t0, int flags);

/* Advance every problem nsteps steps: vels[p] and dt[p] for problem p (host arrays of
 * count entries).  All velocities must have the same kind (FOURIER2D, VORTEX2D or
 * ROTATION) and the RK3 trace.  Asynchronous.  Errors: GALS_ERR_ARG, GALS_ERR_STATE (a
 * problem without state), GALS_ERR_UNSUPPORTED (kind or trace), GALS_ERR_CUDA. */
gals_status gals_batch_step(gals_batch *batch, const gals_velocity *vels, const double *dt,
                            int nsteps);

/* Copy problem `index`'s state out (synchronises); arguments as gals_read_state. */
gals_status gals_batch_read_state(gals_batch *batch, int index, float *const *fields,
                                  int nfields, int memspace);

gals_status gals_batch_synchronize(gals_batch *batch);

/* Launch shape and time loop of the batched step. */
typedef struct {
    int variant;          /* 0: tiles of 128 x 8 nodes, 1: 128 x 16 */
    int blocks;           /* blocks per launch; 0 = one per tile, else persistent blocks */
    double ms_per_step;   /* measured by gals_batch_autotune (0 if set by hand) */
    int loop;             /* GALS_LOOP_LAUNCHES: one launch per step (graph replay);
                             GALS_LOOP_PERSISTENT: all steps of a call in one launch, a tile of
                             step s waiting for the 3 x 3 tiles of its problem around it to finish
                             step s - 1 (used where every problem's feet stay within the tile
                             height minus 2 rows of their node; else one launch per step) */
} gals_batch_tuning;

/* Time every candidate (tile variant x {one block per tile, persistent grids of
 * 1..occupancy blocks per SM} one launch per step, and per tile variant the persistent
 * multi-step loop over trial_steps + 1 steps from a copy of the states) on the current
 * states (which are left unchanged) and keep the fastest; out (optional) receives it.
 * Synchronises.  Errors as gals_batch_step. */
gals_status gals_batch_autotune(gals_batch *batch, const gals_velocity *vels, const double *dt,
                                int trial_steps, gals_batch_tuning *out);
gals_status gals_batch_set_tuning(gals_batch *batch, const gals_batch_tuning *tuning);
gals_status gals_batch_get_tuning(const gals_batch *batch, gals_batch_tuning *tuning);

/* Total number of grid nodes over all problems (node updates per batched step). */
int64_t gals_batch_nodes(const gals_batch *batch);

const char *gals_batch_last_error(const gals_batch *batch);

/* ------------------------------------------------------------------------------------
 * Learned flow-map surrogate of the backward trace.  Not in the paper: a small MLP
 * (x, y, t mod 1) -> (foot displacement / h, (J - I) / dt) of one step of a fixed dt for one
 * 2D FOURIER2D velocity field of period 1, layers 3 -> 128 -> 128 -> 128 -> 128 -> 6 with
 * SiLU, trained on the GPU on targets of a 32-sub-step RK4 backward flow map with its
 * variational Jacobian (BF16 operands, FP32 accumulation, Adam).  gals_step with
 * trace = GALS_TRACE_SURROGATE evaluates it on the tensor cores and feeds the usual Hermite
 * stage; every 128-node tile checks `samples` nodes against the exact RK3 trace (Sec. 5.1)
 * and falls back to RK3 for the whole tile when |delta diff| > tol_x cells or
 * |J diff| > tol_J.  Parameters: flat FP32, per layer W (out x in, row-major) then b.
 * ------------------------------------------------------------------------------------ */
#define GALS_MLP_PARAMS 50822

typedef struct {
    uint64_t seed;          /* initialisation seed: first layer weights and biases uniform in
                               [-4, 4], other weights Glorot uniform, other biases 0 */
    void *cuda_stream;      /* stream for training and inference; NULL: library-owned */
} gals_mlp_desc;

typedef struct {
    int steps;              /* optimizer steps (>= 1) */
    int batch;              /* samples per step, 128..65536 (fresh random samples each step) */
    double lr, lr_min;      /* Adam learning rate, cosine-decayed from lr to lr_min */
    int substeps;           /* RK4 sub-steps of the targets (32) */
    uint64_t seed;          /* sample stream */
} gals_train_opts;

typedef struct {
    double initial_loss, final_loss;  /* MSE of the normalised outputs, first and last batch */
    double seconds;                   /* wall time of the training call */
    int steps;
} gals_train_report;

gals_status gals_surrogate_create(const gals_mlp_desc *desc, gals_surrogate **out);
gals_status gals_surrogate_destroy(gals_surrogate *s);
/* Train for velocity `vel` (FOURIER2D), step dt and grid spacing h (the surrogate is then
 * bound to them: gals_step checks dt, h and the field).  Synchronises. */
gals_status gals_surrogate_train(gals_surrogate *s, const gals_velocity *vel, double dt, double h,
                                 const gals_train_opts *opts, gals_train_report *report);
/* Residual check of gals_step (defaults: 4 samples, tol_x = 0.05 cells, tol_J = 0.05). */
gals_status gals_surrogate_set_check(gals_surrogate *s, double tol_x, double tol_J, int samples);
/* Tiles evaluated and tiles that fell back to RK3 since the last reset; synchronises. */
gals_status gals_surrogate_stats(gals_surrogate *s, int64_t *tiles, int64_t *fallbacks, int reset);
/* FP32 parameters (GALS_MLP_PARAMS floats) and output scales (6) to / from host memory.
 * set_params binds no field: call gals_surrogate_bind before gals_step. */
gals_status gals_surrogate_get_params(const gals_surrogate *s, float *params, float *scales);
gals_status gals_surrogate_set_params(gals_surrogate *s, const float *params, const float *scales);
gals_status gals_surrogate_bind(gals_surrogate *s, const gals_velocity *vel, double dt, double h);
/* Write / read a trained surrogate to / from a file: the FP32 parameters, the output
 * scales, the residual-check settings and, if bound, the field (FOURIER2D modes as the
 * library holds them), dt and h, so that a loaded surrogate serves gals_step at once.
 * Format (host byte order): "GALSMLP" 0x01, int32 version 1, int32 GALS_MLP_PARAMS,
 * int32 6, float params[], float scales[6], float tol_x, float tol_J, int32 samples,
 * int32 bound, then if bound: double dt, double h, int32 kind, int32 nmodes,
 * float a[nmodes], int32 k | l << 8 [nmodes], double n[nmodes], double chi / (2 pi) [nmodes].
 * Errors: GALS_ERR_ARG (NULL, unreadable / unwritable file, wrong magic, version or sizes,
 * truncated), GALS_ERR_CUDA.  save synchronises the surrogate's stream. */
gals_status gals_surrogate_save(const gals_surrogate *s, const char *path);
gals_status gals_surrogate_load(gals_surrogate *s, const char *path);
/* Network outputs (normalised, n x 6, host) for inputs in [-1,1] (n x 3, host), evaluated by
 * the tensor-core inference kernel; synchronises. */
gals_status gals_surrogate_forward(gals_surrogate *s, const float *inputs, int n, float *outputs);
/* The same evaluation on device memory: inputs (n x 3 floats) and outputs (n x 6 floats)
 * are device pointers owned by the caller, 1 <= n <= 2^26; enqueued on the surrogate's
 * stream and not synchronised (launch errors are returned, others surface at the next
 * synchronising call). */
gals_status gals_surrogate_forward_device(gals_surrogate *s, const float *inputs, int64_t n,
                                          float *outputs);
/* Loss and gradient (GALS_MLP_PARAMS floats, host) of the mean squared error against
 * `targets` (n x 6) for `inputs` (n x 3), by the training kernels; synchronises. */
gals_status gals_surrogate_gradient(gals_surrogate *s, const float *inputs, const float *targets,
                                    int n, float *grad, double *loss);
/* Training targets (dx/h, dy/h, (J-I)/dt; n x 6, host) at physical points (x, y, t mod 1)
 * (n x 3, host) for velocity vel: the 32-sub-step RK4 flow map kernel; synchronises. */
gals_status gals_surrogate_targets(gals_surrogate *s, const gals_velocity *vel, double dt, double h,
                                   int substeps, const float *points, int n, float *targets);
const char *gals_surrogate_last_error(const gals_surrogate *s);

/* ------------------------------------------------------------------------------------
 * Diagnostics without device allocation.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they need diagnostics --
 * a loop whose device memory was reserved up front by another allocator, code that must
 * not let cudaMalloc/cudaFree synchronise the device, or a service that accounts for
 * every byte it holds.  It computes what gals_diagnostics computes (same kernels), for
 * a state in caller memory, using a fixed scratch area inside the library (a
 * __device__ array of about 128 KB that each device holding the library keeps until
 * the process exits) instead of allocating.
 *
 *   state       device pointer of plane 0 (plane order as above, all 4 / 8 planes with
 *               valid mixed derivatives; plane p starts at state + p*plane_stride, node
 *               (i,j,k) of a plane at (k*n[1] + j)*row_pitch + i.  gals_state_planes gives
 *               these for a grid; for a COMPACT grid its mixed-derivative planes hold valid
 *               data only after gals_read_state, and the call cannot tell stale ones apart).
 *   reference   NULL, or another state of the same shape and layout.
 *   row_pitch   floats per row, n[0] <= row_pitch <= 2^31 - 1.
 *   plane_stride floats per plane, at least row_pitch * n[1] (* n[2] in 3D).
 *   q           samples per cell and axis, 0..16.
 *   cuda_stream stream to order the work on (NULL: the legacy default stream).
 *   out         host struct; t and steps are 0 (the state has no clock here).
 * Limits and rules:
 *   - grids of more than gals_noalloc_max_nodes() nodes (268,435,456) are rejected
 *     with GALS_ERR_ARG: the scratch holds one partial sum per 16384 nodes;
 *   - set-up: the first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress), and so does the first call after that device's context
 *     changed (cudaDeviceReset, another current context); make that first call before
 *     any stream capture;
 *   - every call on a device shares the one scratch area, which keeps the last call's
 *     contents (each call clears what must start at zero): calls whose GPU work
 *     overlaps -- on different streams or host threads -- race and give wrong results;
 *   - synchronises `cuda_stream` before returning.
 * Errors: GALS_ERR_ARG (dims, pointers, q, strides, size limit), GALS_ERR_CUDA; the
 * message is in gals_noalloc_last_error(), which is per host thread. */
gals_status gals_diagnostics_noalloc(int dim, const int *n, const double *lo, const double *hi,
                                     const float *state, const float *reference,
                                     int64_t row_pitch, int64_t plane_stride, int q,
                                     void *cuda_stream, gals_diag *out);
int64_t gals_noalloc_max_nodes(void);
const char *gals_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GALS_H */
