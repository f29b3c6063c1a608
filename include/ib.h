/*
 * ib.h -- C ABI of the GB300-native first-order immersed-boundary (IB) time
 * step (Givelberg & Bunn, "A Comprehensive Three-Dimensional Model of the
 * Cochlea", Section 3.2, "The Numerical Method").
 *
 * One context drives one fluid grid and one set of Lagrangian markers on one
 * GPU.  Every stage runs as a CUDA kernel of this library; there is no CPU
 * fallback: on a machine without a usable sm_103a device ib_create fails
 * with IB_ERR_CUDA.
 *
 * Conventions (all entry points)
 *  - Layouts.  A grid field component is [z][y][x] with x fastest; a vector
 *    field is [3][z][y][x] (component-major).  Marker arrays are [3][m].
 *    Lattice node (i, j, k) sits at x = h (i, j, k), the summation lattice
 *    of Eq. (discreteX); the box is periodic with edge L_j = n_j h.
 *  - Types.  Grid fields and marker forces are float for IB_FP32 contexts
 *    and double for IB_FP64 contexts ("real" below).  Marker positions are
 *    always double at the ABI; inside, an IB_FP32 context keeps each
 *    position as its FP64 reference point plus an FP32 displacement.
 *  - Pointers.  With IB_PTR_DEVICE in ib_grid_desc.flags every field and
 *    marker pointer passed to a call is a device pointer on the context's
 *    device; otherwise it is a host pointer.  Pointers are borrowed for the
 *    duration of the call only; structure arrays are copied.  Host marker
 *    arrays of ib_set_state / ib_get_state / ib_set_displacement /
 *    ib_get_displacement that are page-locked (cudaHostAlloc or
 *    cudaHostRegister) are read or written by the device in place; pageable
 *    ones are staged through device memory.  Either way the call has
 *    finished with them when it returns.
 *  - Ownership.  The context owns all device memory it allocates; ib_destroy
 *    frees it.
 *  - Asynchrony.  With device pointers, calls enqueue work on the context's
 *    stream and return; with host pointers they also wait for the copies back.
 *    Errors raised on the device (non-finite values) are reported by the
 *    next ib_sync or ib_get_state.
 *  - Errors.  Every call returns an ib_status; the message of the last
 *    failure on the calling thread is available from ib_last_error().  A
 *    call that fails on its arguments leaves the context unchanged.
 */
#ifndef IB_H
#define IB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IB_OK = 0,
    IB_ERR_ARG = 1,          /* invalid argument (null, size, index out of range) */
    IB_ERR_STATE = 2,        /* call out of order (e.g. ib_step before ib_set_structure) */
    IB_ERR_CUDA = 3,         /* CUDA runtime error, including "no usable device" */
    IB_ERR_NOMEM = 4,        /* device allocation failed */
    IB_ERR_NONFINITE = 5,    /* a NaN or Inf appeared in the marker velocities or positions, or a
                                position lies 2^30 or more cells from the origin */
    IB_ERR_TIMEOUT = 6,      /* a kernel's bounded wait for its own asynchronous copies ran out
                                (the kernel skipped its work and returned) */
    IB_ERR_UNSUPPORTED = 7   /* grid size or mode not supported by the library */
} ib_status;

/* IB_FP32_TCFFT: as IB_FP32, with the y passes of the fluid solve's FFT
 * (ny = 256) run as radix-16 DFT matrix products on the tensor cores, the
 * operands split into two BF16 parts and accumulated in FP32 (a precision
 * option, off by default: its rounding is about 2^-16 of the FP32 FFT's,
 * see k_tcfft.cu); other grid shapes take the FP32 y passes. */
typedef enum { IB_FP64 = 0, IB_FP32 = 1, IB_FP32_TCFFT = 2 } ib_precision;

#define IB_PTR_DEVICE 0x1u     /* caller pointers are device pointers */
#define IB_NO_ADVECTION 0x2u   /* drop the advection term of Eq. (discreteNS1) (Stokes) */

/* Fluid grid and time step.  n[j] must each be one of 32, 64, 96, 128, 256
 * (the FFT lengths the library implements).  One mesh width h for
 * all three axes (Section 3.2: the fluid lattice has one mesh width h). */
typedef struct {
    int32_t n[3];         /* grid points along x, y, z */
    double h;             /* mesh width (cm) */
    double rho;           /* fluid density (g/cm^3) */
    double mu;            /* viscosity (g/(cm s)) */
    double dt;            /* time step (s) */
    ib_precision prec;    /* arithmetic of grid fields, forces and FFTs */
    void *stream;         /* cudaStream_t to enqueue on; NULL = legacy default stream */
    uint32_t flags;       /* IB_PTR_DEVICE | IB_NO_ADVECTION */
} ib_grid_desc;

/* A rectangular membrane lattice: marker (i, a) is index first + i*n2 + a;
 * i runs along the length (n1 rows), a across the width (n2 columns).
 * ds is the length-wise spacing, dw[i] the width-wise spacing of row i and
 * seg_of_row[i] in [0, n_seg) the stiffness segment of row i. */
typedef struct {
    int64_t first;
    int32_t n1, n2;
    double ds;
    const double *dw;            /* [n1] (host) */
    const int32_t *seg_of_row;   /* [n1] (host) */
} ib_sheet;

/* Body force on the cells within `radius` of the axis through `center`
 * along the unit vector `direction` and within `half_len` of `center` along
 * it: density rho*amp*omega*cos(omega t) * direction.  amp = 0: none. */
typedef struct {
    double center[3];
    double direction[3];
    double radius;
    double half_len;
    double amp;
    double omega;
} ib_forcing;

/* Immersed material (Section 3.2, step 1; all arrays are host arrays).
 * Springs (fiber links, Peskin 1994): f_i += k (r - L0) d / r with
 * d = X_j - X_i, r = |d|, f_j -= the same.  Tethers: f_i += -k (X_i - X0_i).
 * Membrane bending on the length-wise lattice lines of each sheet,
 * measured from the rest shape X0: energy sum 1/2 c_i |v_i - v0_i|^2 with
 * v_i = X_{i+1} - 2 X_i + X_{i-1} and c_i = bend_b[seg_of_row[i]] dw_i / ds^3
 * (the paper defers the shell law to Givelberg's thesis; this discrete beam
 * law is this library's reading).  Markers carry f(q) dq (dyn) directly.
 * External marker force (the stapes load on the oval window, Section 4: a
 * force orthogonal to the window whose magnitude varies sinusoidally):
 * f_i += mforce_amp cos(mforce_omega t) mforce_dir[:, j] for i = mforce_i[j],
 * at the step's start time t; n_mforce = 0 for none. */
typedef struct {
    int64_t m;                   /* number of markers */
    const double *X0;            /* [3][m] reference positions (cm) */
    int64_t n_spring;
    const int32_t *spring_ij;    /* [n_spring][2] */
    const double *spring_k;      /* [n_spring] dyn/cm */
    const double *spring_L0;     /* [n_spring] cm */
    int64_t n_tether;
    const int32_t *tether_i;     /* [n_tether] */
    const double *tether_k;      /* [n_tether] dyn/cm */
    int32_t n_sheet;
    const ib_sheet *sheets;      /* [n_sheet] */
    int32_t n_seg;
    const double *bend_b;        /* [n_seg] dyn cm */
    ib_forcing forcing;
    int64_t n_mforce;
    const int32_t *mforce_i;     /* [n_mforce] marker ids (each at most once) */
    const double *mforce_dir;    /* [3][n_mforce] */
    double mforce_amp;           /* dyn */
    double mforce_omega;         /* rad/s */
} ib_structure_desc;

typedef struct ib_ctx ib_ctx;

/* Create a context on the current CUDA device.  Allocates the grid fields,
 * the spectral work space and the FFT/symbol tables.  Velocity starts at 0,
 * time at 0.  Fails with IB_ERR_UNSUPPORTED for grid sizes outside the list
 * above and IB_ERR_CUDA when no sm_103a device is usable. */
ib_status ib_create(const ib_grid_desc *desc, ib_ctx **out);

/* Set (or replace) the immersed material: copies the description, builds the
 * per-marker link tables and allocates the marker work space.  Positions are
 * reset to X0 (zero displacement).  Indices out of [0, m), or more than
 * (2^31 - 1)/3 markers (the marker kernels address [3][m] arrays with 32-bit
 * offsets) -> IB_ERR_ARG. */
ib_status ib_set_structure(ib_ctx *ctx, const ib_structure_desc *s);

/* Replace the state.  u: [3][G] real (NULL keeps the velocity); X: [3][m]
 * double positions (NULL keeps them); t: the time of the state. */
ib_status ib_set_state(ib_ctx *ctx, const void *u, const double *X, double t);

/* Read the state back: u [3][G] real, X [3][m] double, *t (each may be
 * NULL).  Synchronises the stream; reports pending device errors. */
ib_status ib_get_state(ib_ctx *ctx, void *u, double *X, double *t);

/* Displacement I/O: D = X - X0, [3][m] double (host or device per flags).
 * Exact: unlike ib_set_state/ib_get_state, whose absolute positions round
 * nanometre displacements against centimetre coordinates, these move the
 * displacement itself (rounded to float in IB_FP32 contexts on set). */
ib_status ib_set_displacement(ib_ctx *ctx, const double *D);
ib_status ib_get_displacement(ib_ctx *ctx, double *D);

/* Advance nsteps first-order IB time steps (Section 3.2, steps 1-4):
 * f^n from X^n; F^n by Eq. (discreteF) plus the body force at t^n;
 * u^{n+1} from Eqs. (discreteNS1)-(discreteNS2); X^{n+1} by Eq. (discreteX)
 * with u^{n+1} interpolated at X^n.  Enqueued as a captured CUDA graph. */
ib_status ib_step(ib_ctx *ctx, int64_t nsteps);

/* Eq. (discreteF) alone: F = sum_l f_l delta_h(x - X_l) for the context's m
 * markers at positions X [3][m] (double) with forces f [3][m] (real);
 * F [3][G] (real) is overwritten on every node.  Markers are radix-sorted
 * by 8^3 tile (bit-exact, stable, as ib_bin_sort), each work item of a bin
 * (at most 512 of its markers) is summed into its own partial box of nodes,
 * and each touched tile gathers the partial boxes of the bins covering it;
 * every sum has a fixed order, so repeated calls are bitwise identical. */
ib_status ib_spread(ib_ctx *ctx, const double *X, const void *f, void *F);

/* Eq. (discreteX), velocity part: U_l = sum_x u(x) delta_h(x - X_l) h^3 for
 * the context's m markers; X [3][m] double, u [3][G] real, U [3][m] real. */
ib_status ib_interp(ib_ctx *ctx, const double *X, const void *u, void *U);

/* Step 3 alone: solve Eqs. (discreteNS1)-(discreteNS2) for u^{n+1} (and
 * p^{n+1} when p is not NULL) given u^n and F^n, all [3][G] real (p: [G]).
 * Does not touch the context's state. */
ib_status ib_fluid_solve(ib_ctx *ctx, const void *u_n, const void *F, void *u_np1, void *p);

/* The marker bins of positions X [3][m]: key[l] is the tile-major index of
 * cell floor(X_l / h) (indices wrapped, X * (1/h) in FP64): with 8^3 tiles,
 * key = tile * 512 + (lz*8 + ly)*8 + lx, tile = (tz*nty + ty)*ntx + tx,
 * (t, l) = (cell / 8, cell % 8) per axis and nt = n/8; perm = marker ids
 * sorted stably by tile (key / 512), i.e. by (tile, id) (int32, [m]).  This
 * is the sort that ib_spread, ib_interp and ib_step use. */
ib_status ib_bin_sort(ib_ctx *ctx, const double *X, int32_t *key, int32_t *perm);

/* Mean velocity of the state (the zero-wavenumber mode of Eqs.
 * discreteNS1-2; it changes by (dt/rho) times the mean of F - rho A(u) plus
 * the body force each step).  FP32 contexts carry it in FP64 through the
 * steps (the grid field holds it rounded to FP32); FP64 contexts return the
 * field's mean.  mean: 3 doubles, HOST memory.  Synchronises the stream. */
ib_status ib_get_mean_velocity(ib_ctx *ctx, double *mean);

/* The bin sort that the last ib_step made from the context's own state
 * (X = X0 + D at the start of that step), in the caller's marker numbering:
 * key [m] = cell key of each caller marker (as ib_bin_sort defines it),
 * perm [m] = caller marker id at each sorted position, internal [m] = caller
 * marker id of each internal index.  The context numbers markers internally
 * by their initial cell; perm is sorted stably by tile in that numbering,
 * i.e. by (tile, internal index).  Each output may be NULL; int32, host or
 * device per IB_PTR_DEVICE.  IB_ERR_STATE if an explicit-position call
 * (ib_bin_sort, ib_spread, ib_interp) has sorted since the last step.
 * Parity aid for the step's bin sort (Section 3.3's partitioning of the
 * markers); host outputs synchronise the stream. */
ib_status ib_get_bin_order(ib_ctx *ctx, int32_t *key, int32_t *perm, int32_t *internal);

/* Allocation-free bin sort (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running
 * inside a CUDA graph capture in global mode, or a host runtime that owns
 * all device memory through its own pool).  Same keys and stable order as
 * ib_bin_sort, without a context: n[3] grid points, mesh width h, m markers,
 * X [3][m] double positions, key [m] and perm [m] int32 outputs, all device
 * pointers owned by the caller (grid sizes multiples of 8); work is enqueued on `stream` (NULL: legacy
 * default stream).  It calls no allocator: the radix sort's work space is
 * one fixed device array of IB_NOALLOC_MAX_MARKERS markers (about 12.9 MB),
 * set up on the first call on each device -- make that first call before
 * any stream capture -- and kept by that GPU until the process exits.  m
 * above the maximum, or a grid of 2^31 cells or more, returns IB_ERR_ARG
 * with a message.  Every call on a device shares the array, so calls whose
 * work overlaps on the GPU (different streams, no ordering between them)
 * race; serialise them. */
#define IB_NOALLOC_MAX_MARKERS 1048576
ib_status ib_bin_sort_noalloc(const int32_t n[3], double h, int64_t m, const double *X, int32_t *key,
                              int32_t *perm, void *stream);

/* Reverse of one forward step (Section 3.2, steps 1-4): the transpose of the
 * step's linearisation about the context's current state (u^n, D^n, t^n),
 * for the gradient of a scalar J of later states.  The state is not changed;
 * set it (ib_set_state, ib_set_displacement) to step n first.
 *   lam_u     [3][G] dJ/du^{n+1}, context precision;
 *   lam_D     [3][m] double, dJ/dD^{n+1} in the caller's marker numbering;
 *   u_np1     [3][G] u^{n+1} as ib_step computes it from this state, or NULL:
 *             then it is recomputed here (one more spread and fluid solve,
 *             body force at t^n);
 *   lam_u_out [3][G] receives dJ/du^n (may alias lam_u);
 *   lam_D_out [3][m] receives dJ/dD^n (may alias lam_D);
 *   grad_b    [n_seg] double, dJ/db_seg of the bending stiffness is ADDED
 *             (NULL: not wanted; accumulated per segment in FP64 in a fixed
 *             order, so repeated runs give identical sums).
 * With dJ/dX^{n+1} = lam_D: lam_U = dt lam_D, the interpolation's transpose
 * spreads it (Eq. discreteF with the roles swapped), the solve of Eqs.
 * discreteNS1-2 is applied unchanged (it is real symmetric), the upwind
 * term's transpose and the delta kernel's derivative phi' give the state and
 * position terms, and the elastic forces' Jacobian (springs, tethers,
 * bending) carries the force sensitivity back to D.  The sign switch of the
 * upwind difference and the cell of each marker are held fixed (the
 * derivative where it exists).  Pointers are host or device per
 * IB_PTR_DEVICE; u_np1 must not alias an output.  Work space is allocated on
 * the first call.  Errors: IB_ERR_ARG (null required pointer), IB_ERR_STATE
 * (no structure), IB_ERR_NOMEM, IB_ERR_CUDA. */
ib_status ib_adjoint_step(ib_ctx *ctx, const void *u_np1, const void *lam_u, const double *lam_D,
                          void *lam_u_out, double *lam_D_out, double *grad_b);

/* Replace the per-segment bending stiffness b [n_seg] (dyn cm, double; host
 * or device per IB_PTR_DEVICE) of the structure set last, keeping all other
 * structure data and the state (the basilar-membrane stiffness is the
 * parameter the gradient of ib_adjoint_step is taken in).  Synchronises the
 * context's stream.  Errors: IB_ERR_ARG (null or non-finite b), IB_ERR_STATE
 * (no structure). */
ib_status ib_set_bend_stiffness(ib_ctx *ctx, const double *bend_b);

/* State snapshots for checkpointing (the paper stores the material
 * positions every 10th step, Section 5; the reverse sweep replays segments
 * from snapshots).  A
 * snapshot is an opaque DEVICE buffer of ib_snapshot_bytes(ctx) bytes, owned
 * by the caller, that holds the velocity u ([3][G] in the context's
 * precision, at offset 0, so it can be passed as ib_adjoint_step's u_np1),
 * the marker displacement, the time and (FP32 contexts) the FP64 mean
 * velocity that the step carries for the zero-wavenumber mode of Eqs.
 * discreteNS1-2.  Save and load are device-to-device
 * copies enqueued on the context's stream, without synchronisation; a
 * snapshot is valid only for the context (structure) that wrote it.
 * ib_snapshot_bytes returns -1 for a null context. */
int64_t ib_snapshot_bytes(const ib_ctx *ctx);
ib_status ib_snapshot_save(ib_ctx *ctx, void *buf);
ib_status ib_snapshot_load(ib_ctx *ctx, const void *buf);

/* Tile shapes of one context: the parameters of the autotuner.  The FFT
 * passes are compiled in two tile variants for FP32 contexts (one for FP64),
 * the x forward pass in three:
 *   fft_x: x passes, 0 = 4 grid rows per block, 1 = 8 rows, 2 = 4 rows of
 *          16 planes per block marching along z, the planes staged in
 *          shared memory by bulk asynchronous copies (the inverse x pass
 *          takes 4 rows for 0 and 2);
 *   fft_y: y passes, 0 = 16 columns per block (FP64: 8), 1 = 8 columns;
 *   fft_z: z pass (with the projection), 0 = 8 columns (FP64: 4), 1 = 4;
 *   marker_blocks: blocks of the persistent spreading and interpolation
 *   kernels, 0 = every SM at full occupancy (a smaller grid leaves SMs to
 *   other instances of a batch).
 * The paper has no counterpart (its tuning was its data partitioning for the
 * shared-memory machines of Section 3.3). */
typedef struct {
    int32_t fft_x, fft_y, fft_z;
    int32_t marker_blocks;
} ib_tuning;

/* Set / read the tile shapes.  Setting synchronises the context's stream and
 * invalidates its captured step.  Errors: IB_ERR_ARG (null pointer, variant
 * out of range for the context's precision, negative marker_blocks). */
ib_status ib_set_tuning(ib_ctx *ctx, const ib_tuning *t);
ib_status ib_get_tuning(const ib_ctx *ctx, ib_tuning *t);

/* Choose the tile shapes of ctx by timing: coordinate descent over the FFT
 * variants and marker_blocks in {0, 2, 1, 1/2, 1/4 blocks per SM}, each
 * trial 2 warm-up steps plus `reps` timed steps (CUDA events, the captured
 * step graph).  The state is saved to a device snapshot first and restored
 * after every trial and at the end, so the simulation continues from where
 * it was; the best shapes are applied and, if best is not NULL, returned.
 * Allocates one snapshot for the duration of the call.  Errors: IB_ERR_ARG,
 * IB_ERR_STATE (no structure), IB_ERR_NOMEM, IB_ERR_CUDA. */
ib_status ib_autotune(ib_ctx *ctx, int32_t reps, ib_tuning *best);

/* Batched stepping of independent instances (a tone sweep over grids and
 * membranes of different sizes): the steps of n contexts, all on one
 * device, captured as parallel branches of one CUDA graph, steps_per_launch
 * steps per branch; every ib_batch_step launch of the graph on `stream`
 * (NULL: the legacy default stream) advances every instance.  The contexts
 * are borrowed (they must outlive the batch) and keep their own state:
 * read it with ib_get_state after ib_batch_sync.  The graph is recaptured
 * when a member's structure or tuning changes.  The paper runs one
 * experiment at a time (Section 5); instances here share nothing.
 * Errors: IB_ERR_ARG (null or repeated context, contexts on different
 * devices, nsteps not a multiple of steps_per_launch), IB_ERR_STATE (a
 * context without structure), IB_ERR_CUDA. */
typedef struct ib_batch ib_batch;
ib_status ib_batch_create(ib_ctx *const *ctxs, int32_t n, int32_t steps_per_launch, void *stream, ib_batch **out);
ib_status ib_batch_step(ib_batch *batch, int64_t nsteps);
/* The same tile shapes for every member, chosen by coordinate descent on
 * the whole batch's graph time (reps timed launches per trial); members'
 * states are saved and restored as in ib_autotune. */
ib_status ib_batch_autotune(ib_batch *batch, int32_t reps);
/* Wait for the batch and report the first member's device error, if any. */
ib_status ib_batch_sync(ib_batch *batch);
ib_status ib_batch_destroy(ib_batch *batch);

/* Marker probe: the normal displacement eta_i = (X_i - X0_i) . dir_i of n
 * chosen markers (the paper follows the travelling wave through the normal
 * displacement of the basilar membrane's centre line and its envelope over
 * time, Section 5).  After ib_set_probe every `every`-th step (counted from
 * this call) appends one record of n doubles, and the step's end time, to a
 * device ring of `capacity` records and raises the running envelope
 * max |eta_i|; the recording kernel is part of the captured step, so long
 * runs need no host involvement.  markers [n] are caller marker ids, dir
 * [3][n] double (host arrays, copied).  n = 0 removes the probe.  Setting
 * synchronises the stream and invalidates the captured step.
 * ib_read_probe synchronises and drains the ring: *count = records produced
 * since the last read; the newest min(*count, capacity) of them are written
 * in time order to eta [.][n] and times [.] (each may be NULL), and the
 * envelope [n] (may be NULL) since ib_set_probe.  The paper has no
 * counterpart interface (it wrote positions to files every 10th step).
 * Errors: IB_ERR_ARG, IB_ERR_STATE (no structure / no probe), IB_ERR_NOMEM. */
ib_status ib_set_probe(ib_ctx *ctx, int32_t n, const int32_t *markers, const double *dir, int32_t every,
                       int32_t capacity);
ib_status ib_read_probe(ib_ctx *ctx, double *eta, double *times, double *envelope, int64_t *count);

/* Stages of one step, in order, as timed by ib_profile. */
#define IB_NSTAGES 10
/* Name of stage i (0 <= i < IB_NSTAGES): keys, sort, records, spread,
 * fft_x_fwd, fft_y_fwd, fft_z_proj, fft_y_inv, fft_x_inv, interp. */
const char *ib_stage_name(int32_t i);

/* Advance nsteps steps (same arithmetic as ib_step) launched one by one
 * with CUDA events recorded on the context's stream between stages;
 * stage_ms[i] receives the mean device time of stage i per step and
 * *active_tiles (may be NULL) the number of grid tiles some marker's
 * stencil reached in the last step.  Synchronises. */
ib_status ib_profile(ib_ctx *ctx, int64_t nsteps, double *stage_ms, int64_t *active_tiles);

/* Wait for all work enqueued by the context; reports device errors. */
ib_status ib_sync(ib_ctx *ctx);

/* Self-check of the failure path for bounded waits (no counterpart in the
 * paper).  Enqueues on the context's stream one block that waits, for at
 * most `polls` polls (1 .. 2^20; each poll suspends for a bounded,
 * hardware-defined time), on a fresh mbarrier that nothing arrives on, by
 * the same bounded wait the staged kernels use for their copies: the wait
 * runs out and sets the context's timeout flag, so the next ib_sync or
 * ib_get_state returns IB_ERR_TIMEOUT and clears the flag.  Nothing else is
 * touched; the context stays usable.  Errors: IB_ERR_ARG (null context,
 * polls out of range), IB_ERR_CUDA (launch failure). */
ib_status ib_check_bounded_wait(ib_ctx *ctx, int32_t polls);

/* Free the context and everything it owns.  NULL is a no-op. */
ib_status ib_destroy(ib_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *ib_last_error(void);

/* Marker count, grid size and precision of a context (for bindings). */
ib_status ib_info(const ib_ctx *ctx, int64_t *m, int64_t *G, int32_t *prec);

#ifdef __cplusplus
}
#endif

#endif /* IB_H */
