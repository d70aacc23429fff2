/*
 * wlb.h - C ABI of the GB300 wave lattice Boltzmann acoustic-radiation-force
 * library (sm_103a).
 *
 * The library computes the time-averaged acoustic radiation force on a
 * density-matched compressible object held in a standing acoustic wave, by the
 * method of Castro-Avila, Malgaretti, Harting and Munoz, "A lattice Boltzmann
 * approach for acoustic manipulation":
 *
 *   1. a wave lattice Boltzmann model (D2Q5 or D3Q7, BGK with tau = 1/2,
 *      Sec. V, Eqs. 62-64 and 71) marches the first-order fields p1 and u1 on a
 *      lattice whose sound speed c(x) carries the object (Sec. VI, Eq. 79);
 *   2. p1 and u1 are interpolated onto N surface points with the three-point
 *      kernel of Eq. (82) (Eqs. 80-81) and time-averaged as <p1^2>, <u1.u1> and
 *      <u1 (u1.n)> over the last n_avg_periods periods (Sec. VII);
 *   3. King's surface integral, Eq. (14) (Eq. 77 in lattice variables), gives
 *      the force in FP64.
 *
 * All lattice quantities are in lattice units (dx = dt = 1).  The lattice is
 * periodic on every axis.  The initial condition is the standing wave
 * p1 = p_a cos(2 pi (s - antinode) / wavelength), u1 = 0, imposed through the
 * equilibrium as Eq. (72) describes for initial conditions.
 *
 * Conventions
 *   - Every call returns a wlb_status and never aborts the process.
 *   - Host pointers are owned by the caller.  Device memory is owned by the
 *     handle: either one caller-provided device workspace (see
 *     wlb_workspace_bytes) or, when none is given, memory the library allocates
 *     with cudaMalloc in wlb_create and frees in wlb_destroy.
 *   - Work is issued asynchronously on the CUDA stream given to wlb_create;
 *     calls that return host data (wlb_force, wlb_fields, wlb_surface,
 *     wlb_mask, wlb_run, wlb_force_history, wlb_save_state) and
 *     wlb_load_state synchronise that stream before returning.
 *   - A handle is not thread safe; distinct handles are independent.
 *   - Population layout in device memory: structure of arrays f[i][z][y][x],
 *     x fastest, velocity order i = 0 (rest), +x, -x, +y, -y, +z, -z.
 */
#ifndef WLB_H
#define WLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WLB_OK = 0,
    WLB_ERR_ARG = 1,       /* invalid parameter or argument                    */
    WLB_ERR_UNSTABLE = 2,  /* non-finite time-average accumulators              */
    WLB_ERR_CUDA = 3,      /* a CUDA runtime call or kernel launch failed       */
    WLB_ERR_OOM = 4,       /* device or host allocation failed, or workspace too small */
    WLB_ERR_STATE = 5,     /* call out of order (e.g. wlb_step before wlb_init) */
    WLB_ERR_TIMEOUT = 6    /* a bounded device-side wait gave up (reported, never a hang),
                              or wlb_run's host-clock deadline passed            */
} wlb_status;

typedef enum { WLB_D2Q5 = 0, WLB_D3Q7 = 1 } wlb_lattice;          /* Fig. 8   */
/* Geometry along the wave axis: fully periodic with the standing wave as the
 * initial state, or the driven cavity of Sec. VII (see wlb_params). */
typedef enum { WLB_BOUNDARY_PERIODIC = 0, WLB_BOUNDARY_DRIVEN = 1 } wlb_boundary;
/* Storage and arithmetic of the populations: FP32, FP64, or FP16 storage of
 * f / p_a (the deviation from the rest state f = 0, scaled to O(1)) with FP32
 * arithmetic, running sums and sound-speed field. */
typedef enum { WLB_POP_F32 = 0, WLB_POP_F64 = 1, WLB_POP_F16 = 2 } wlb_precision;

/*
 * Problem statement (Sec. VII and Table I; Eq. 79 for the object).
 *
 *   lattice        WLB_D2Q5 (2D, nz must be 1) or WLB_D3Q7.
 *   nx, ny, nz     lattice extents; all axes periodic.
 *   wave_axis      0, 1 or 2: axis s of the standing wave.
 *   c0, cp         sound speed of fluid and object; stability needs
 *                  D c^2 < 1 for both (D = 2 or 3; it keeps f_0^eq >= 0).
 *   rho0           mean density (the object is density matched).
 *   p_a            pressure amplitude of the standing wave.
 *   wavelength     lambda in cells; the box along wave_axis must hold a whole
 *                  number of wavelengths and T = lambda / c0 must be a whole
 *                  number of steps.
 *   antinode       coordinate of a pressure antinode along wave_axis.
 *   center         object centre r0 (the z entry is ignored in 2D).  Exact
 *                  integer classification of cells needs |x - r0|^2 exact in
 *                  double precision: use multiples of 2^-10.
 *   radius         R_p.
 *   interface_d    "square thickness" d of Eq. (79) (the paper uses 4).
 *   surface_radius radius of the integration surface (R_p in the paper).
 *   n_surface      N surface elements: equal arcs in 2D, Fibonacci points in 3D.
 *   n_periods      total run length in periods T.
 *   n_avg_periods  the last n_avg_periods periods are averaged (<= n_periods).
 *   precision      WLB_POP_F32, WLB_POP_F64 or WLB_POP_F16 (p_a != 0; p_a
 *                  sets the FP16 storage scale).
 *   boundary       WLB_BOUNDARY_PERIODIC, or WLB_BOUNDARY_DRIVEN: the driven
 *                  cavity of Sec. VII along wave_axis, starting from rest:
 *                  the planes s = 0 and s = n-1 are partially absorbing walls
 *                  (bounce-back damped by wall_damping, Eq. 73; the value that
 *                  would leave the domain is dropped), the plane s = 1 is a
 *                  source sheet where the fields are imposed after collision
 *                  (Eq. 72): rho1 = source_amplitude sin(2 pi (t mod T)/T),
 *                  J1 from Eq. (62).  The box length along wave_axis is free
 *                  (the paper uses lambda/2 + 3); the object, its band and
 *                  stencil must lie in 2 <= s <= n-2; antinode is ignored.
 *   wall_damping   Phi in [0, 1] (the paper uses 0.99).
 *   source_amplitude  rho_a of the source sheet.
 *
 * The object, its interface band and the interpolation stencil must fit in
 * half the box along every axis (minimum-image distances must be unique).
 */
typedef struct {
    int lattice;
    int nx, ny, nz;
    int wave_axis;
    double c0, cp, rho0;
    double p_a, wavelength, antinode;
    double center[3];
    double radius, interface_d, surface_radius;
    int n_surface;
    int n_periods, n_avg_periods;
    int precision;
    int boundary;
    double wall_damping, source_amplitude;
} wlb_params;

typedef struct wlb_handle wlb_handle;

/* Sizes derived from a parameter set. */
typedef struct {
    int dim, q;                 /* 2 or 3; 5 or 7 populations                   */
    long long cells;            /* nx * ny * nz                                 */
    long long period;           /* T = wavelength / c0 steps                    */
    long long n_steps;          /* n_periods * T                                */
    long long n_window;         /* n_avg_periods * T                            */
    long long steps_done;       /* steps since the last wlb_init (0 if none)    */
    long long samples_done;     /* steps sampled since the last wlb_init        */
    double bytes_per_update;    /* algorithmic HBM bytes of one cell update:
                                   2 q pop_bytes + 1 (class byte); pop_bytes is
                                   4, 8 or 2                                   */
    int vector_path;            /* 1 if the row-vectorised update kernel is used */
    int steps_per_launch;       /* steps per update launch: 1, or 2 with
                                   wlb_set_two_step (the default for 3D
                                   lattices where it applies)                   */
    int two_step_rows;          /* slab height of the two-step kernel, 0 off    */
    int two_step_segments;      /* warps per lattice row (per x-tile) in it, 0 off */
    int two_step_tiles;         /* x-tiles per row in it (1: whole rows), 0 off */
    int two_step_staging_warp;  /* 1: a dedicated warp stages its planes        */
    int two_step_c2_staged;     /* 3D whole rows: 1 band rows' c^2 staged in
                                   shared memory, 0 read from L2               */
} wlb_info;

/* Check a parameter set.  WLB_ERR_ARG for: unknown lattice or precision,
 * non-positive sizes, nz != 1 in 2D, bad wave_axis, D c0^2 >= 1 or
 * D cp^2 >= 1, c0 <= 0, cp <= 0, rho0 <= 0, non-integral T = wavelength/c0,
 * a box length along wave_axis that is not a whole number of wavelengths,
 * radius <= 0, interface_d <= 0, an object + band + stencil wider than half
 * the box, n_surface < 0, n_periods < 1, n_avg_periods outside [0, n_periods]. */
wlb_status wlb_validate(const wlb_params *p);

/* Device workspace, in bytes, that wlb_create needs for these parameters. */
wlb_status wlb_workspace_bytes(const wlb_params *p, size_t *bytes);

/* Create a handle.  device_workspace: NULL to let the library cudaMalloc its
 * own memory, else a device pointer (256-byte aligned) to at least
 * wlb_workspace_bytes bytes that stays valid until wlb_destroy.  stream: a
 * cudaStream_t (NULL = legacy default stream) on which all work is issued.
 * Captures nothing and launches nothing.  *out is set only on WLB_OK. */
wlb_status wlb_create(const wlb_params *p, void *device_workspace, size_t workspace_bytes,
                      void *stream, wlb_handle **out);

/* Setup and initial condition (asynchronous): cell classes and sound-speed
 * field (Eq. 79), surface elements and interpolation weights (Sec. VI,
 * Eqs. 80-82), the standing wave imposed through the equilibrium (Eq. 72),
 * and zeroed time averages.  Resets the step and sample counters and the
 * force history. */
wlb_status wlb_init(wlb_handle *h);

/* Advance n_steps >= 0 lattice steps (asynchronous).  Each step streams and
 * collides every cell (Eqs. 62-64, 71).  sample != 0 adds, at each step and
 * before its collision, the surface interpolation and the running sums of
 * p1^2, u1.u1 and (n.u1) u1 (Eqs. 80-82); FP32 running sums (FP64 with
 * WLB_POP_F64) are folded into FP64 once per period.  Whole periods are
 * replayed as CUDA graphs captured on first use.  WLB_ERR_STATE before
 * wlb_init. */
wlb_status wlb_step(wlb_handle *h, long long n_steps, int sample);

/* Time-averaged force from the samples taken since wlb_init, Eq. (14) in
 * FP64:  F_i = - sum_k dS_k [ (<p1^2>/(2 rho0 c0^2) - rho0 <u1.u1>/2) n_ki
 *                              + rho0 <u1_i (u1.n_k)> ].
 * Writes 3 doubles to force_out (host; the third is 0 in 2D) and
 * synchronises.  All zero if nothing was sampled.  WLB_ERR_UNSTABLE if any
 * accumulator is not finite. */
wlb_status wlb_force(wlb_handle *h, double force_out[3]);

/* The whole protocol: wlb_init, (n_periods - n_avg_periods) T unsampled steps,
 * n_avg_periods T sampled steps, wlb_force.  With a deadline set (below) and
 * passed: WLB_ERR_TIMEOUT (see wlb_set_deadline). */
wlb_status wlb_run(wlb_handle *h, double force_out[3]);

/* Host-clock watchdog of wlb_run (the paper has no counterpart).  seconds > 0:
 * wlb_run then issues its steps one period at a time with at most two periods
 * queued, and between periods compares the host clock since the call with
 * the limit; past it, it waits for the queued periods to finish (their
 * device work cannot be recalled) and returns WLB_ERR_TIMEOUT with the handle
 * consistent: wlb_get_info's steps_done counts the steps that ran, and
 * wlb_step / wlb_force / wlb_init may follow.  Results within the limit are
 * bit-identical to a run without it.  seconds = 0 (the default) turns it off;
 * WLB_ERR_ARG for a negative or non-finite value. */
wlb_status wlb_set_deadline(wlb_handle *h, double seconds);

/* Fields at the current time: p1 = c^2 rho1 and u1 = J1 / rho0 (Eq. 62).
 * p1_out: nx*ny*nz doubles, u1_out: dim*nx*ny*nz doubles laid out
 * [a][z][y][x]; either may be NULL.  Host buffers; synchronises. */
wlb_status wlb_fields(wlb_handle *h, double *p1_out, double *u1_out);

/* Surface elements after wlb_init: n_surface rows of
 * (x, y, z, n_x, n_y, n_z, dS) doubles (host buffer); synchronises. */
wlb_status wlb_surface(wlb_handle *h, double *pts_out);

/* Cell classes after wlb_init: nx*ny*nz bytes [z][y][x] (host buffer):
 * 0 fluid (c = c0), 1 object (c = cp), 2 interface band (c from Eq. 79);
 * with WLB_BOUNDARY_DRIVEN also 3 low wall, 4 high wall, 5 source sheet.
 * A cell is fluid when (|x - r0|^2 - R_p^2) >= 20 d, object when it is
 * <= -20 d, band otherwise (minimum-image distance); beyond the band the tanh
 * of Eq. (79) is +-1 in double precision.  Synchronises. */
wlb_status wlb_mask(wlb_handle *h, unsigned char *mask_out);

/* Checkpoint and resume.  The paper has no counterpart: a long run can stop
 * and continue in another handle or process.  The state after wlb_init and
 * any steps is the current populations, the running surface sums of the
 * current period, the folded FP64 sums, the force history, the non-finite
 * flag and the step counters; everything else follows from the parameters
 * and is rebuilt by the setup.  The buffer is host memory owned by the
 * caller: a fixed-size header (format tag, version, the parameters as
 * doubles, the counters and array sizes), then the arrays in that order,
 * each padded to 8 bytes.
 *
 *   wlb_state_bytes  *bytes: the buffer size the two calls below need.
 *   wlb_save_state   waits for the handle's stream, then copies the state
 *                    into host[0 .. wlb_state_bytes).  WLB_ERR_STATE before
 *                    wlb_init; WLB_ERR_ARG if bytes is too small.
 *   wlb_load_state   restores a state written by wlb_save_state for a handle
 *                    with the same parameters (runs the setup first if the
 *                    handle has not been initialised).  Steps issued after it
 *                    continue exactly where the saved handle stopped: forces
 *                    and fields are bit-identical.  WLB_ERR_ARG for a short
 *                    buffer, a foreign format or version, other parameters,
 *                    or counters out of range (nothing is changed then).
 * Both synchronise. */
wlb_status wlb_state_bytes(const wlb_handle *h, size_t *bytes);
wlb_status wlb_save_state(wlb_handle *h, void *host, size_t bytes);
wlb_status wlb_load_state(wlb_handle *h, const void *host, size_t bytes);

/* Force history (Sec. VII follows the force over time to see it settle).
 * Every fold of the running surface sums is recorded on the device (graph
 * replays included): each full sampled period, and the partial period that
 * wlb_force folds when called inside one.  Up to n_periods + 1 entries are
 * kept since wlb_init (later ones are counted, not kept).
 *   out          host, max_entries x 3 doubles: per entry, Eq. (14) over the
 *                samples that fold added alone (a sampled period's force).
 *   samples_out  host, max_entries long longs (may be NULL): those sample
 *                counts (T for a full period).  The mean of the rows weighted
 *                by their counts is the wlb_force result.
 *   *count       entries recorded (may exceed max_entries; only
 *                min(count, max_entries, n_periods + 1) rows are written).
 * WLB_ERR_STATE before wlb_init.  Synchronises. */
wlb_status wlb_force_history(wlb_handle *h, double *out, long long *samples_out, int max_entries, int *count);

/*
 * Allocation-free averaging (the paper has no counterpart of this call).
 *
 * For callers that cannot allocate device memory when they need a force:
 * processes whose device memory is a fixed pool owned by someone else (a
 * framework's caching allocator that has reserved the whole budget, or an
 * arena handed to a plugin that is given no allocator of its own), and loops
 * that cannot afford cudaMalloc / cudaFree, which may synchronise the whole
 * device.  Starting from the handle's current state, advances n_steps >= 0
 * sampled steps exactly as wlb_step(h, n_steps, 1) does (interpolation,
 * running sums folded to FP64 once per period, fused stream+collide, one
 * step per launch) and then returns the time-averaged force over those
 * n_steps, as wlb_force would for them, in force_out (3 host doubles; zeros
 * when n_steps == 0 or n_surface == 0).  The result equals wlb_step +
 * wlb_force over the same steps bit for bit.  Synchronises the handle's
 * stream.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine and
 * instantiates no graph: kernels are launched directly, and the running
 * sums, FP64 totals, force and error flag live in one file-scope device array
 * of 640 KiB, sized for WLB_NOALLOC_MAX_SURFACE points, that every GPU
 * loading the library holds until the process exits.  The handle's own
 * accumulators and sample counters are left untouched.
 *
 *   - The first call on a device (and the first after the device's context
 *     was reset) looks up that array's device address (cudaGetSymbolAddress,
 *     with that device current); make this first call before any stream
 *     capture.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call clears what it accumulates before use.  Calls whose work overlaps
 *     on the GPU (other streams, other threads, other handles) race on it:
 *     serialise them.
 *   - WLB_ERR_ARG if n_surface > WLB_NOALLOC_MAX_SURFACE or n_steps < 0;
 *     WLB_ERR_STATE before wlb_init; WLB_ERR_UNSTABLE on non-finite sums.
 */
#define WLB_NOALLOC_MAX_SURFACE 8192
wlb_status wlb_average_noalloc(wlb_handle *h, long long n_steps, double force_out[3]);

/*
 * Batched ensembles (Secs. V-VII protocol, run for many independent problems).
 *
 * count lattices of uneven size, one parameter set each (same lattice type and
 * precision; nx a multiple of 16 bytes of populations and at most 512 FP32 /
 * 256 FP64 / 1024 FP16 cells), stepped together: one launch per step updates
 * every row of every lattice still running, one launch samples every surface
 * point of every lattice inside its averaging window, and the step index lives
 * in device memory, so chunks of 64 steps replay as one CUDA graph.  Each
 * lattice follows exactly the protocol of wlb_run (its own period, n_periods
 * and n_avg_periods; a lattice stops at its own last step).
 *
 *   wlb_batch_workspace_bytes  device bytes for the batch (per-lattice regions
 *                              as in wlb_workspace_bytes, plus tables).
 *   wlb_batch_create           ws: NULL (library cudaMalloc) or a 256-byte
 *                              aligned device pointer of at least that size;
 *                              stream: cudaStream_t for all work.
 *   wlb_batch_autotune         times candidates on the actual batch for
 *                              steps_per_trial steps each (after a fresh setup)
 *                              and keeps the fastest, returned in *best (may be
 *                              NULL).  Two steps per launch (3D): every plan of
 *                              z-chunk length {16, 24, 32, 48, 64, 96, whole}
 *                              x slab-height cap {tallest, 8, 5} x lane
 *                              layout {one or two
 *                              16-byte chunks per lane for wide rows, one for
 *                              all} x staging {warp 0, a dedicated warp per
 *                              CTA}; 2D two steps: rows per warp chunk {the
 *                              height filling whole waves, 32, 24, 20, 16}; one
 *                              step per launch: threads per block {128, 256} x
 *                              blocks per SM {2, 4, 8, 16}.  Leaves the
 *                              lattices in an advanced state; wlb_batch_run
 *                              starts from setup.
 *   wlb_batch_run              setup, all steps, forces: forces_out is count x 3
 *                              host doubles (lattice order).  Synchronises.
 *                              WLB_ERR_UNSTABLE if any lattice's sums are not
 *                              finite.
 * WLB_ERR_ARG for count < 1, an invalid parameter set, mixed lattice types or
 * precisions, a row length the batched update does not cover, or a driven
 * geometry (batches are periodic only).
 */
typedef struct wlb_batch wlb_batch;
typedef struct {
    int threads_per_block, blocks_per_sm;
    float ms_per_step;
    int z_chunk;             /* two steps per launch: z-chunk length target (3D),
                                rows per warp chunk (2D)                       */
    int slab_rows_cap;       /* ... slab-height cap (0: the tallest that fits)  */
    int one_chunk_per_lane;  /* ... 1: one 16-byte chunk per lane everywhere   */
    int plans_tried;         /* launch shapes or plans timed                    */
    int staging_warp;        /* two steps per launch (3D): 1 = a dedicated warp
                                per CTA stages the planes                       */
} wlb_batch_tuning;
typedef struct {
    int count;
    long long total_rows, total_points, max_steps;
    long long lattice_updates;      /* sum over lattices of cells x steps */
    int threads_per_block, blocks_per_sm, row_chunks;
    int steps_per_launch;           /* 2: every launch advances all lattices two
                                       steps (wlb_set_two_step's kernel, one
                                       launch over every lattice's slabs)      */
    int total_ctas;                 /* work units of that launch: blocks (3D)
                                       or warps, one per row chunk (2D); 0 if
                                       one step per launch                    */
} wlb_batch_info;

wlb_status wlb_batch_workspace_bytes(const wlb_params *ps, int count, size_t *bytes);
wlb_status wlb_batch_create(const wlb_params *ps, int count, void *ws, size_t ws_bytes, void *stream,
                            wlb_batch **out);
wlb_status wlb_batch_autotune(wlb_batch *b, int steps_per_trial, wlb_batch_tuning *best);
wlb_status wlb_batch_run(wlb_batch *b, double *forces_out);
wlb_status wlb_batch_get_info(const wlb_batch *b, wlb_batch_info *out);
/* Steps two per launch for the whole batch: on by default when all run
 * lengths, windows and periods are even and every lattice is periodic and
 * either 3D with FP32/FP16 rows the two-step slab kernel takes (then one
 * launch of it per lane layout covers every lattice, each with its own slab
 * plan; with two lane layouts the two launches run side by side, the second
 * on a stream the batch creates and joins back into its own) or 2D with
 * rows of at most 64 sixteen-byte vectors and 8 values per lane (then each
 * warp sweeps a chunk of 32 rows of one lattice, both steps in registers).
 * A batched sampling launch adds the sums of both steps.  Bit-identical to
 * one step per launch.  enable = 0 returns to one step per launch;
 * enable != 0 where the batch does not qualify gives WLB_ERR_ARG. */
wlb_status wlb_batch_set_two_step(wlb_batch *b, int enable);
const char *wlb_batch_last_error(const wlb_batch *b);
wlb_status wlb_batch_destroy(wlb_batch *b);

/*
 * Learned surrogate of the force (not part of the paper's method; the lattice
 * runs above generate its training data and judge its error).
 *
 * MLP 4 -> 256 -> 256 -> 256 -> 1, GELU(z) = z Phi(z) on the hidden layers,
 * linear output, mean-squared-error loss.  Inputs are the four features
 * (k R_p, k z0, kappa~ = kappa_p/kappa_0, c~ = c_p/c_0), normalised to [-1, 1]
 * by the box [x_lo, x_hi] given at creation, which is also the "training hull"
 * reported by wlb_mlp_predict.  Every matrix product runs on the tensor cores
 * (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory); weights and
 * activations are BF16, the Adam masters FP32.
 *
 * Packed parameter vector (FP32, wlb_mlp_param_count() values): W1 [256][4],
 * b1 [256], W2 [256][256], b2, W3 [256][256], b3, W4 [1][256], b4 [1].
 *
 *   wlb_mlp_create       batch_max: multiple of 128 (<= 4 Mi); allocates its
 *                        device buffers with cudaMalloc; weights all zero.
 *   wlb_mlp_init_weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed).
 *   wlb_mlp_set_weights / wlb_mlp_get_weights   host FP32 packed vector;
 *                        set resets the Adam state.
 *   wlb_mlp_loss_grad    x: device n x 4 FP32, t: device n FP32 (n <= batch_max);
 *                        loss (host float, may be NULL) and gradient (host
 *                        packed FP32, may be NULL); no update.
 *   wlb_mlp_train        epochs over n device samples in shuffled whole
 *                        batches (SplitMix64(seed) Fisher-Yates), Adam
 *                        (0.9, 0.999, 1e-8) with the learning rate decayed
 *                        geometrically from lr to lr_final; loss_history
 *                        (host, epochs floats, may be NULL) gets each epoch's
 *                        mean batch loss.
 *   wlb_mlp_predict      x: device n x 4, y: device n FP32, inside: device n
 *                        bytes (may be NULL): 1 if the query lies in the box.
 *                        Any n >= 0 (not bounded by batch_max; x and y may be
 *                        NULL when n = 0).  By default
 *                        one persistent kernel runs the whole network per
 *                        128-query tile with the activations in shared and
 *                        tensor memory and the weights streamed from L2.
 *   wlb_mlp_set_fused    fused = 1 (default): predict as above; 0: one
 *                        tensor-core GEMM launch per layer through device
 *                        memory in batch_max chunks (the training forward).
 *                        Both give the same bits.  WLB_ERR_ARG otherwise.
 * All calls synchronise the stream before returning.  WLB_ERR_TIMEOUT if a
 * tensor-core completion wait gave up (the kernel returns instead of hanging).
 */
typedef struct wlb_mlp wlb_mlp;
int wlb_mlp_param_count(void);
wlb_status wlb_mlp_create(int batch_max, const float x_lo[4], const float x_hi[4], void *stream, wlb_mlp **out);
wlb_status wlb_mlp_init_weights(wlb_mlp *m, unsigned long long seed);
wlb_status wlb_mlp_set_weights(wlb_mlp *m, const float *w);
wlb_status wlb_mlp_get_weights(wlb_mlp *m, float *w);
wlb_status wlb_mlp_loss_grad(wlb_mlp *m, const float *x, const float *t, int n, float *loss, float *grad);
wlb_status wlb_mlp_train(wlb_mlp *m, const float *x, const float *t, long long n, int epochs, int batch, float lr,
                         float lr_final, unsigned long long seed, float *loss_history);
wlb_status wlb_mlp_predict(wlb_mlp *m, const float *x, long long n, float *y, unsigned char *inside);
wlb_status wlb_mlp_set_fused(wlb_mlp *m, int fused);
const char *wlb_mlp_last_error(const wlb_mlp *m);
wlb_status wlb_mlp_destroy(wlb_mlp *m);

/* Sizes and counters of a handle. */
wlb_status wlb_get_info(const wlb_handle *h, wlb_info *out);

/* Steps two per launch: the update of Eqs. (62)-(64), (71) applied twice in
 * one kernel, bit-identical to two single steps.  Each block owns a slab of
 * slab_rows rows (y) of a range of planes (z); it computes the first step on
 * its rows plus one halo row on either side and keeps that state on the SM,
 * so the populations cross HBM about once per two steps.  No block waits for
 * another.  In sampled steps a small kernel before it adds the surface sums
 * of both steps (t from the stored state, t+1 recomputed from it by the same
 * arithmetic), in the order two single steps add them.  On by default (set
 * up by wlb_create with an automatic slab height) wherever it is supported:
 * 3D, periodic boundaries, FP32 or FP16 storage, nx a multiple of 16 cells
 * (each row split into warp-wide segments, the last one possibly shorter),
 * and rows that fit the shared memory whole (nx up to about 1500 FP32
 * cells) or split into x-tiles (wlb_set_two_step_tiles).
 * 2D lattices (periodic, any storage, rows of at most two 16-byte chunks
 * per lane and 8 values per lane) take it on request (off by default: a
 * single lattice of such short rows has too few row chunks to fill the SMs
 * and one step per launch is faster; 2D batches use it by default): each
 * warp sweeps a chunk of rows, both steps in its registers (slab_rows must
 * be 0).
 * Elsewhere, or with enable = 0, every step is one launch.  enable: 0 off;
 * 1 on, lane layout chosen by the library; 2 on with one 16-byte chunk per
 * lane (more, lighter warps); 3 on with two (WLB_ERR_ARG if unsupported).
 * slab_rows: 0 lets the library choose (by estimated time: slab height and
 * z chunks that fill the SMs, the tallest among near-equal estimates), else
 * that height (WLB_ERR_ARG if it does not fit; the setting is then
 * unchanged).  A stalled staging copy (bounded
 * wait) makes wlb_force return WLB_ERR_TIMEOUT.  The paper has no counterpart:
 * it is a memory-traffic optimisation of the same update. */
wlb_status wlb_set_two_step(wlb_handle *h, int enable, int slab_rows);

/* x-tiles of the two-step kernel (3D).  A slab's rows are staged in shared
 * memory, so long rows leave room only for short slabs, and every slab
 * recomputes two halo rows: 512-cell FP32 rows allow 3-row slabs.  Splitting
 * each row into tiles of tx cells (a multiple of 16; the last tile may be
 * narrower) lets a CTA hold a taller slab of one tile; it stages 16 bytes of
 * every array on either side of its tile and also computes the first step on
 * the two cells just outside it, so no CTA waits for another.  Bit-identical
 * to whole rows.  The tiles' rows are staged by per-thread copies, which
 * cost instructions that whole rows do not: measured slower wherever a
 * whole-row slab fits (512^3 FP32: 1410 us per launch with 4 tiles of 14-row
 * slabs against 1254 us with 3-row whole-row slabs).  tiles: 0 lets the
 * library choose (whole rows where a whole-row slab fits the shared memory,
 * else the cheapest estimate of 2 .. 16 tiles: rows of more than about 1500
 * FP32 cells), 1 whole rows, n >= 2 n tiles of ceil(nx / n) cells rounded up
 * to 16, each at most one warp of 16-byte vectors (two per lane for FP32).  Applies to the current and
 * later wlb_set_two_step settings.  WLB_ERR_STATE while two steps per launch
 * is off; WLB_ERR_ARG if the tiling does not fit (setting unchanged) or on a
 * 2D lattice (tiles > 1).  The paper has no counterpart: it changes how the
 * same update is scheduled, not what it computes. */
wlb_status wlb_set_two_step_tiles(wlb_handle *h, int tiles);

/* Who stages the planes of the two-step kernel with whole rows (3D): the
 * bulk copies of a plane are issued once the plane barrier has passed, by
 * one warp.  staging: 0 lets the library choose, 1 warp 0 (which also
 * computes its row, so the next barrier waits for both), 2 a dedicated
 * extra warp that only stages (one fewer slab row may fit the thread
 * limit).  Bit-identical either way.  Applies to the current and later
 * wlb_set_two_step settings; x-tiles stage per warp and ignore it.
 * WLB_ERR_STATE while two steps per launch is off; WLB_ERR_ARG if the plan
 * does not fit (setting unchanged) or on a 2D lattice (staging 2). */
wlb_status wlb_set_two_step_staging(wlb_handle *h, int staging);

/* Where the two-step kernel with whole rows (3D) reads c^2 of rows that hold
 * interface-band cells (Eq. 79's smooth profile; elsewhere c^2 follows from
 * the cell class).  Staged in shared memory beside the populations, c^2
 * takes slab height from long rows (512-cell FP32 rows: 3-row slabs with it,
 * 4 without); otherwise the first step reads it from global memory, where
 * the staging warp has prefetched the row into L2 two planes ahead.  c2: 0
 * lets the library choose (staged, unless reading from L2 fits a slab plan
 * of lower estimated time than every staged one), 1 staged, 2 read from L2.  Bit-identical either way.  Applies to the current
 * and later wlb_set_two_step settings; x-tiles always stage it.
 * WLB_ERR_STATE while two steps per launch is off; WLB_ERR_ARG if the plan
 * does not fit (setting unchanged) or on a 2D lattice (c2 != 0).  The paper
 * has no counterpart: it moves the same values through another memory. */
wlb_status wlb_set_two_step_c2(wlb_handle *h, int c2);

/* Release the handle, its graphs, streams and any memory it allocated. */
wlb_status wlb_destroy(wlb_handle *h);

/* Static description of a status code. */
const char *wlb_status_str(wlb_status s);

/* Detail of the last error on this handle ("" if none). */
const char *wlb_last_error(const wlb_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* WLB_H */
