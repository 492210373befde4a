/*
 * celeris_gb.h -- C ABI of the GB300 time-step library for the extended
 * Boussinesq equations of Madsen & Sorensen in the conservative form used by
 * Celeris (Tavakkol & Lynett, arXiv 1611.05984).
 *
 * One step advances U = [h, P, Q] (unknowns [w, P, Q], w = h + z) by:
 *   KP07 generalized-minmod reconstruction, positivity fix and desingularised
 *   velocities (Sec. 2.2, Eq. 14); central-upwind fluxes; bed-slope, friction
 *   (Sec. 2.6, Eq. 31-32) and dispersive terms (Eq. 10-13); the AB3 predictor
 *   (Eq. 15-17) with K iterations of the AM4 corrector (Eq. 18-20), Euler for
 *   the first two steps; the tridiagonal solves of Eq. 21-23 per x-row and
 *   per y-column; boundaries (Sec. 2.4, Eq. 24-30).
 *
 * Conventions (every call):
 *   - SI units.  Cell (i,j) has its centre at ((i+1/2) dx, (j+1/2) dy).
 *   - Field arrays passed in or out are interior only, dense, row-major
 *     [ny][nx], of the grid's real type (real_bytes = 4: float, 8: double),
 *     in DEVICE memory unless a parameter says "host".
 *   - Memory ownership: the caller owns all device memory (workspace, arrays,
 *     checkpoints, gauge buffers).  The library never allocates device memory;
 *     the handle holds host metadata and pointers into caller memory only.
 *   - Streams: calls are asynchronous on the handle's stream unless marked
 *     "synchronises".  A handle must not be used from two threads at once.
 *   - Errors: every call returns a cel_status; nothing throws across the ABI.
 *     NULL pointers and bad sizes give CEL_ERR_INVALID_ARG; a CUDA error gives
 *     CEL_ERR_CUDA and its text is kept for cel_last_error().
 */
#ifndef CELERIS_GB_H
#define CELERIS_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cel_solver cel_solver; /* opaque, owned by the library (host) */

typedef enum {
    CEL_OK = 0,
    CEL_ERR_INVALID_ARG = 1,
    CEL_ERR_WORKSPACE_TOO_SMALL = 2,
    CEL_ERR_CUDA = 3,
    CEL_ERR_NONFINITE = 4,
    CEL_ERR_TIMEOUT = 5,
    CEL_ERR_NOT_IMPLEMENTED = 6
} cel_status;

enum { CEL_BSNQ = 0, CEL_NLSW = 1 };                 /* model, Sec. 3.2       */
enum { CEL_FRIC_NONE = 0, CEL_FRIC_QUADRATIC = 1, CEL_FRIC_MANNING = 2 }; /* Sec. 2.6 */
enum { CEL_SOLID = 0, CEL_SPONGE = 1, CEL_SINE = 2 }; /* boundary, Sec. 2.4    */
enum { CEL_WEST = 0, CEL_EAST = 1, CEL_SOUTH = 2, CEL_NORTH = 3 };
enum { CEL_FIELD_BBAR = 0, CEL_FIELD_D = 1, CEL_FIELD_USTAR = 2, CEL_FIELD_VSTAR = 3 };

/* Maximum line lengths of the tridiagonal solves (one thread block per line). */
#define CEL_MAX_LINE_F32 16384
#define CEL_MAX_LINE_F64 8192

typedef struct {
    int32_t nx, ny;       /* interior cells, 2 <= n <= CEL_MAX_LINE_*          */
    double dx, dy;        /* cell sizes [m]                                    */
    int32_t real_bytes;   /* 4 (FP32) or 8 (FP64): type of state and arithmetic */
} cel_grid;

typedef struct {
    int32_t model;        /* CEL_BSNQ or CEL_NLSW (Sec. 3.2)                   */
    double g;             /* gravity, 9.81                                     */
    double Bdisp;         /* dispersion calibration B of Eq. 2, 1/15           */
    double theta;         /* generalized-minmod parameter of KP07, in [1, 2]   */
    double eps;           /* desingularisation tolerance of Eq. 14 (5e-12)     */
    double dt;            /* fixed time step [s]                               */
    int32_t corrector_iters; /* K >= 0 AM4 iterations per step (Sec. 2.3)      */
    double still_water;   /* w_s                                               */
    int32_t friction;     /* CEL_FRIC_*                                        */
    double fric_coef;     /* f (quadratic, Eq. 31) or Manning n (Eq. 32)       */
} cel_params;

typedef struct {
    int32_t type;         /* CEL_SOLID | CEL_SPONGE | CEL_SINE (Sec. 2.4)       */
    int32_t width_cells;  /* sponge width L_s in cells (Eq. 30)                */
    int32_t ncomp;        /* sine components summed, 0..8 (Eq. 25-28)          */
    double amp[8];        /* a [m]                                             */
    double period[8];     /* T [s]                                             */
    double theta[8];      /* direction [rad] from +x                           */
    double phase[8];      /* phase added inside the sine [rad]                 */
} cel_bc;

/* Bytes of device workspace a solver of this grid/params needs.  Host only;
 * INVALID_ARG on bad sizes (n < 2, n above the line limit, real_bytes). */
cel_status cel_workspace_bytes(const cel_grid *grid, const cel_params *params,
                               size_t *bytes);

/* Create a solver.  z_dev: bed elevation at cell centres (Sec. 3.2 "bathymetry
 * file"), [ny][nx] real, device, read during the call only.  workspace_dev:
 * caller-owned device memory of at least cel_workspace_bytes, 256-byte
 * aligned, kept until cel_destroy.  cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream).  The state starts at rest: w = max(w_s, Bbar),
 * P = Q = 0, all sides CEL_SOLID, t = 0.  Asynchronous on the stream. */
cel_status cel_create(const cel_grid *grid, const cel_params *params,
                      const void *z_dev, void *workspace_dev, size_t ws_bytes,
                      void *cuda_stream, cel_solver **out);

/* Boundary of one side (CEL_WEST..CEL_NORTH), Sec. 2.4: solid wall (Eq. 24),
 * sponge layer (Eq. 30; the ghosts behind it are solid) or sine-wave maker
 * (Eq. 25-29, components summed).  Host only; takes effect at the next step. */
cel_status cel_set_boundary(cel_solver *s, int32_t side, const cel_bc *bc);

/* Hot start (Sec. 3.2): copy w, P, Q ([ny][nx] real, device).  w is raised to
 * the cell bed where below it and P = Q = 0 where the depth is zero.  Restarts
 * the AB3 history (the next two steps are Euler, Sec. 2.3).  Asynchronous. */
cel_status cel_set_state(cel_solver *s, const void *w, const void *P,
                         const void *Q);

/* Superpose a solitary wave (Sec. 2.7, Eq. 33-36) of height H [m] (negative:
 * depression), direction theta [rad], crest at (x0, y0) [m], where the still
 * water depth d > 0.  d in Eq. 35-36 is that of the cell holding the crest;
 * INVALID_ARG if it is dry or H + d <= 0.  Restarts the AB3 history.
 * Synchronises (reads the crest depth). */
cel_status cel_add_solitary(cel_solver *s, double H, double theta, double x0,
                            double y0);

/* Replace the bed (runtime terrain edit, Sec. 1) and re-derive the static
 * fields; w is raised to the new bed; restarts the AB3 history.  Async. */
cel_status cel_set_bathymetry(cel_solver *s, const void *z_dev);

/* Advance nsteps >= 0 time steps.  Asynchronous on the handle's stream. */
cel_status cel_step(cel_solver *s, int32_t nsteps);

/* Copy the current w, P, Q into [ny][nx] device arrays (any may be NULL).
 * Asynchronous. */
cel_status cel_get_state(cel_solver *s, void *w, void *P, void *Q);

/* Diagnostic fields into a [ny][nx] device array: CEL_FIELD_BBAR (cell bed),
 * CEL_FIELD_D (still-water depth), CEL_FIELD_USTAR / _VSTAR (the increments
 * of U*, V* of Eq. 7-8 over the last stage, the right sides of the last line
 * solves, which are solved for P^{n+1} - P^n).  Asynchronous. */
cel_status cel_get_field(cel_solver *s, int32_t which, void *dst);

/* Gauges (Sec. 3.2 "logData"): record eta = w - w_s at n cells (ij_host =
 * [i0,j0,i1,j1,...], host) every log_every steps into a ring of `capacity`
 * records kept in gauge_buf_dev (caller device memory of cel_gauge_bytes).
 * When full, the oldest record is overwritten.  Host + one async copy. */
cel_status cel_gauge_bytes(int32_t n, int32_t capacity, int32_t real_bytes,
                           size_t *bytes);
cel_status cel_set_gauges(cel_solver *s, const int32_t *ij_host, int32_t n,
                          int32_t log_every, int32_t capacity,
                          void *gauge_buf_dev, size_t buf_bytes);
/* Move up to max_rec oldest records into eta_host ([rec][n] real, host) and
 * drop them from the ring; *n_rec = records written.  Synchronises. */
cel_status cel_read_gauges(cel_solver *s, void *eta_host, int32_t max_rec,
                           int32_t *n_rec);
/* The same without synchronising: the copies are queued on the handle's
 * stream (asynchronous where eta_host is pinned), so the next steps can be
 * queued behind them; *n_rec is known at once, the values are in eta_host
 * once the stream has reached the copies (cudaStreamSynchronize or an event
 * recorded after this call).  eta_host must stay valid until then. */
cel_status cel_read_gauges_async(cel_solver *s, void *eta_host, int32_t max_rec,
                                 int32_t *n_rec);

/* Simulated time t = step * dt and the step count since create.  Host only. */
cel_status cel_get_time(cel_solver *s, double *t, int64_t *step);

/* Device reduction over w, P, Q: CEL_ERR_NONFINITE if any value is NaN/Inf
 * (the first offending cell index goes into cel_last_error).  Synchronises. */
cel_status cel_check_finite(cel_solver *s);

/* Diagnostics of the present state (device reduction over the interior):
 * mass = sum of (w - Bbar) dx dy [m^3]; max_speed = the largest |(P, Q)|
 * k(h) [m/s] with k the velocity factor of Eq. 14 (h = max(w - Bbar, 0));
 * wet_cells = the cells with w > Bbar.  The mass is summed in double, in no
 * fixed order.  Synchronises. */
typedef struct {
    double mass;
    double max_speed;
    int64_t wet_cells;
} cel_stats;
cel_status cel_get_stats(cel_solver *s, cel_stats *out);

/* Checkpoint: state, AB3/AM4 history, step count and time, enough for a
 * bit-exact resume.  Device buffer of cel_checkpoint_bytes.  Asynchronous
 * (save) / synchronises (load reads the header). */
cel_status cel_checkpoint_bytes(const cel_solver *s, size_t *bytes);
cel_status cel_save_checkpoint(cel_solver *s, void *dst_dev, size_t bytes);
cel_status cel_load_checkpoint(cel_solver *s, const void *src_dev, size_t bytes);

/* Run-up tracking (Sec. 4.1 and 4.3 read the run-up off the wet extent,
 * with a depth threshold delta = s dx / 3).  maxw_dev: [ny][nx] real,
 * device, owned by the caller; after every step maxw[j][i] becomes the
 * highest w seen so far while the cell's depth w - Bbar exceeded delta, and
 * stays -inf where it never did.  Enabling sets the field from the present
 * state (asynchronous); maxw_dev = NULL disables.  The field must stay
 * allocated while enabled.  CEL_ERR_INVALID_ARG for delta < 0. */
cel_status cel_runup_enable(cel_solver *s, void *maxw_dev, double delta);

/* Headless rendering of the present state into an RGBA image, for the
 * visualisation options of Sec. 3: a colormap of eta, u, v or the velocity
 * magnitude, or the water surface shaded photorealistically (reflection of a
 * sky gradient and refraction of the bed, weighted by the Fresnel equations
 * for air -> water); land (depth <= dry_h) is the terrain colormap of the bed
 * elevation with a hillshade; optional grid lines every `grid` metres.  No
 * graphics API is involved: the image is written to device memory.
 *
 * rgba_dev: [ny][nx][4] bytes (R, G, B, 255), device, owned by the caller;
 * row j of the image is grid row j (south first), one pixel per cell.
 * Velocities are u = P / max(h, h_min), v = Q / max(h, h_min).  The shading
 * is single precision, each operation rounded on its own (no fused
 * multiply-add, no transcendental functions), so the bytes are reproducible.
 * Asynchronous on the handle's stream.  CEL_ERR_INVALID_ARG for a bad mode,
 * vmax <= vmin, zmax <= zmin, grid < 0, dry_h < 0, h_min <= 0, absorb < 0,
 * a zero view or sun vector or non-finite values. */
enum { CEL_RENDER_ETA = 0, CEL_RENDER_U = 1, CEL_RENDER_V = 2, CEL_RENDER_SPEED = 3,
       CEL_RENDER_FRESNEL = 4 };
typedef struct {
    int32_t mode;          /* CEL_RENDER_*                                         */
    float vmin, vmax;      /* colormap range of the shown value (modes 0-3)        */
    float dry_h;           /* land where w - Bbar <= dry_h                         */
    float h_min;           /* floor of the depth in the velocities                 */
    float zmin, zmax;      /* terrain colormap range of the bed elevation          */
    float grid;            /* grid line spacing [m], 0 for none                    */
    float exaggeration;    /* vertical scale of the surface and bed normals        */
    float view[3];         /* direction of view, towards the surface               */
    float sun[3];          /* direction towards the light (terrain hillshade)      */
    float absorb;          /* refraction: the bed colour weighs 1 / (1 + absorb h) */
} cel_render_params;
cel_status cel_render(cel_solver *s, const cel_render_params *params, void *rgba_dev);

/* Discrete adjoint: the gradient of the gauge misfit
 *   L = 1/2 sum_{n=1..N} sum_g (eta_g^n - obs_g^n)^2,
 * eta_g^n = w - w_s at gauge g after step n, with respect to w at the start
 * and (optionally) to the cell-centre bed z, by the exact reverse of every
 * step: the KP07 flux with the limiter and positivity branches taken in the
 * forward run, the dry clamp and dry masks, the sponge, friction, the
 * dispersive and mixed terms (Eq. 10-13), the line solves transposed
 * (Eq. 21-23), the AB3 predictor with its history and Euler start-up, and
 * the AM4 corrector iterations (Eq. 15-20), for both models (Sec. 3.2).
 * The gradient is the derivative along the branches the forward run took
 * (the step is piecewise smooth).  The solver must hold a fresh history
 * (cel_set_state just before); it runs N steps forward keeping a checkpoint
 * every ckpt_every steps, then the reverse sweep, recomputing one segment of
 * states at a time from its checkpoint; it ends holding the state after
 * step N.  ckpt_every = 0 keeps every step's states, corrector iterates and
 * line solutions from the forward run instead, with no recomputation
 * (the scratch then grows with N: 3 (K + 1) values per cell and step, plus
 * 2 (K + 1) with the bed on the Boussinesq model); a negative ckpt_every is
 * CEL_ERR_INVALID_ARG.
 *
 * gij_host: ngauges (i, j) pairs; obs_dev: [N][ngauges] real, device;
 * scratch_dev: cel_adjoint_bytes(..., with_bed = grad_z_dev != NULL) bytes
 * of device memory (256-byte aligned), owned by the caller; eta_dev (may be
 * NULL): [N][ngauges] real, the recorded eta; grad_w_dev: [ny][nx] real,
 * dL/dw(t = 0) (w after cel_set_state's clamp to the bed); grad_z_dev (may
 * be NULL): [ny][nx] real, dL/dz for the bed z of cel_create or
 * cel_set_bathymetry, with the initial w held where the cell is wet and
 * equal to the cell bed where it is dry (the clamp), as when cel_set_state
 * is called again after a change of bed; the sine makers' ghost values
 * follow the depth beside them (Eckart wave number, celerity) and are
 * differentiated too.  *loss (may be NULL): L in double.  Synchronises.  The
 * adjoint sums reach a cell from several faces in no fixed order, so
 * repeated runs agree to rounding, not bit for bit. */
cel_status cel_adjoint_bytes(const cel_solver *s, int32_t nsteps, int32_t ckpt_every, int32_t ngauges,
                             int32_t with_bed, size_t *bytes);
cel_status cel_adjoint_gauge_misfit(cel_solver *s, int32_t nsteps, int32_t ckpt_every, const int32_t *gij_host,
                                    int32_t ngauges, const void *obs_dev, void *scratch_dev,
                                    size_t scratch_bytes, void *eta_dev, void *grad_w_dev, void *grad_z_dev,
                                    double *loss);

/* dL/dw_in from the dL/dw0 that cel_adjoint_gauge_misfit returns, for the
 * caller's w_in before cel_set_state clamped it to the bed (w0 = max(w_in,
 * Bbar), the reading of Sec. 2.2's dry cells used by cel_set_state): the
 * derivative is 1 where w_in lies above the cell bed Bbar and 0 where the
 * clamp holds w0 at the bed (the one-sided derivative at a tie).  w_in_dev:
 * [ny][nx] real, device, the values passed to cel_set_state; grad_w_dev:
 * [ny][nx] real, device, dL/dw0 on entry and dL/dw_in on return (in place).
 * Uses the solver's present bed.  Asynchronous on the handle's stream;
 * CEL_ERR_INVALID_ARG for a NULL argument, CEL_ERR_CUDA on a launch error. */
cel_status cel_adjoint_input_gradient(cel_solver *s, const void *w_in_dev, void *grad_w_dev);

/* Self-check of the adjoint's face-flux derivative (Sec. 2.2, Eq. 14): the
 * reverse sweep uses a hand-written vector-Jacobian product of the KP07
 * reconstruction and central-upwind flux; this evaluates it beside the
 * dual-number product of the forward's own flux code on caller-chosen
 * faces.  in_dev: [n][22] real, device (real_bytes 4 or 8), per face, in
 * order: the 4 cells' w[4], P[4], Q[4] (cells f-2..f+1), the face beds Bm,
 * Bf, Bp, the flux adjoints lH[3] (mass, normal, tangential momentum),
 * theta, g, eps and dir (0: x-face, P normal; 1: y-face, Q normal).  out_dev:
 * [n][30] real, device: the adjoints of (w[4], P[4], Q[4], Bm, Bf, Bp) by
 * dual numbers, then by hand.  cuda_stream as in cel_create.  Synchronises;
 * CEL_ERR_CUDA on a CUDA error, CEL_ERR_INVALID_ARG on bad arguments. */
cel_status cel_adjoint_face_selfcheck(int32_t real_bytes, const void *in_dev, int32_t n, void *out_dev,
                                      void *cuda_stream);

/* Line-solver splits (the per-line tridiagonal solves of Eq. 21-23).  A
 * line of up to 8192 rows (FP32) or 4096 (FP64) is cut into segments of 2, 4
 * or 8 rows, one per thread: the built-in rule takes 2 rows on lines of at
 * most 64, 4 up to 128 and 8 above.  cel_set_line_split(real_bytes,
 * max_rows, rows_per_thread) sets the rows per thread for the class of line
 * lengths up to max_rows (above the next smaller class's bound), where the
 * block of ceil(n / rows) threads, rounded up to 32, fits (1024 FP32, 512
 * FP64); rows_per_thread 0 removes the class.  It is meant for an autotuner:
 * the results of a line solve depend on its split at rounding level, so
 * cel_step and ensembles that are to agree bit for bit must run under the
 * same table.  The table is process-wide and applies to every later launch;
 * an ensemble created before a change refuses to step (create it again).
 * cel_reset_line_splits returns to the built-in rule.  cel_line_config
 * reports the rows per thread and the block size a line of `rows` rows gets.
 * CEL_ERR_INVALID_ARG for sizes or rows out of range.  The paper has one
 * line solver (a cyclic reduction on the GPU, Sec. 3.3); the splits are this
 * library's own. */
cel_status cel_set_line_split(int32_t real_bytes, int32_t max_rows, int32_t rows_per_thread);
cel_status cel_reset_line_splits(void);
cel_status cel_line_config(int32_t real_bytes, int32_t rows, int32_t *rows_per_thread, int32_t *threads);

/* Programmatic dependent launch of the step's kernels (ghost tables,
 * stencil, line solves, gauges, state captures; single grids and the
 * adjoint's reverse; the ensembles' batched launches stay plain),
 * process-wide, on by default: each is launched so that it
 * may start while the kernel before it on the stream drains its last
 * blocks, and waits on the device for that kernel's completion before it
 * touches memory.  The results do not depend on the setting; 0 launches
 * every kernel after the previous one has completed. */
cel_status cel_set_dependent_launch(int32_t enable);
cel_status cel_get_dependent_launch(int32_t *enabled);

/* Kernel launches issued by the most recent cel_step call. */
cel_status cel_last_launch_count(const cel_solver *s, int64_t *launches);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * each launch of the step kernels (0: stencil + update, 1: line solves, x-rows
 * and y-columns in one launch, 2: sine-maker ghost table).  cel_profile_enable creates `capacity` event
 * pairs (host-side CUDA resources; no device memory) and starts recording;
 * launches beyond capacity are not timed.  cel_profile_read synchronises and
 * returns the summed milliseconds and launch counts per kernel, then resets
 * the counters.  cel_profile_disable destroys the events. */
cel_status cel_profile_enable(cel_solver *s, int32_t capacity);
cel_status cel_profile_read(cel_solver *s, double ms[3], int64_t count[3]);
cel_status cel_profile_disable(cel_solver *s);

/* Ensembles: many solvers stepped in lockstep, each kernel kind launched once
 * per stage over all of them.  The paper steps one simulation at a time (the
 * time integration of Sec. 3.3 with the solves of Eq. 21-23); an ensemble
 * takes the same step for every member, so that a set of small grids (a few
 * tiles each, far fewer than the GPU's SMs) fills the GPU in one launch
 * instead of many.  Each member evolves bit for bit as it would under
 * cel_step: the kernels, the per-member arguments and the order of every sum
 * are the same.
 *
 * members: n >= 1 handles from cel_create, all of one precision and one
 * corrector_iters, on disjoint workspaces (CEL_ERR_INVALID_ARG otherwise);
 * they may differ in size, bed, boundaries, model, friction and dt.  The
 * ensemble keeps the handle pointers: members must outlive it.
 * cel_ensemble_table_bytes gives the device memory the ensemble needs for its
 * argument tables (tens of KB per member); table_dev (256-byte aligned, owned
 * by the caller) must stay allocated until cel_ensemble_destroy.  Every
 * launch of the ensemble goes to cuda_stream; work the caller queued on the
 * members' own streams must be finished (or ordered before it by the caller).
 * cel_ensemble_create copies a few small tables (asynchronous); a one-line
 * reason for a failure goes to msg (msg_len bytes, may be NULL).
 *
 * cel_ensemble_step advances every member by nsteps steps (asynchronous).
 * The members must be in lockstep: the same number of steps since their
 * last cel_set_state / cel_set_bathymetry / cel_add_solitary / checkpoint
 * load (CEL_ERR_INVALID_ARG otherwise, reason in cel_ensemble_last_error).
 * Members may be used alone between ensemble steps (cel_get_state, gauges,
 * checkpoints, cel_set_boundary: the ensemble rebuilds its tables when a
 * boundary or bed changed).  Gauges of members are logged as under cel_step.
 * Two ensembles (or an ensemble and cel_step) that share a member must not
 * overlap on the GPU.
 *
 * Captured cycles: once the members' history is full (two steps after the
 * state was set), the argument blocks of a step repeat every 6 steps.  Where
 * no member logs gauges or tracks run-up and profiling is off,
 * cel_ensemble_step records 6 steps as one CUDA graph (on a stream of the
 * library's own, the first time a cycle starts at a given phase; every
 * argument block of the cycle uploaded beforehand) and replays it on
 * cuda_stream for each further 6 steps: the same kernels with the same
 * arguments, so the results are bit for bit those of launching them one by
 * one.  The ghost tables' step index then comes from a counter in the table
 * that the graph advances.  A change of boundary or bed, or a new argument
 * block, discards the graphs.  cel_ensemble_use_graphs(e, 0) launches every
 * step one kernel at a time (the default is 1). */
typedef struct cel_ensemble cel_ensemble;     /* opaque, owned by the library (host) */
cel_status cel_ensemble_table_bytes(cel_solver *const *members, int32_t n, size_t *bytes);
cel_status cel_ensemble_create(cel_solver *const *members, int32_t n, void *table_dev,
                               size_t table_bytes, void *cuda_stream,
                               cel_ensemble **out, char *msg, size_t msg_len);
cel_status cel_ensemble_step(cel_ensemble *e, int32_t nsteps);
cel_status cel_ensemble_use_graphs(cel_ensemble *e, int32_t enable);
/* Steps taken by replaying a captured cycle since cel_ensemble_create. */
cel_status cel_ensemble_graph_steps(const cel_ensemble *e, int64_t *steps);
/* Persistent launch.  With enable != 0, where a captured cycle could be used
 * (above) and every line family takes the register solver in blocks of at
 * most 256 threads, cel_ensemble_step takes all its remaining steps in ONE
 * cooperative launch (as many 256-thread blocks as fit the GPU at once):
 * the blocks work through the ghost tables, then per stage the stencil
 * tiles and the line solves (several short lines side by side per block),
 * with a grid-wide barrier where a batched launch would end.  The arguments
 * are the batched launches' argument blocks, so the results are bit for bit
 * the same.  Every barrier wait is bounded by timeout_ms (in (0, 60000];
 * CEL_ERR_INVALID_ARG otherwise): a block whose wait runs out sets a status
 * word and the launch ends at the next barrier, leaving the members' states
 * undefined.  cel_ensemble_check synchronises the ensemble's stream and
 * returns CEL_ERR_TIMEOUT if that happened (the words are cleared).
 * CEL_ERR_CUDA if no block of the launch fits an SM.  Off by default. */
cel_status cel_ensemble_use_persistent(cel_ensemble *e, int32_t enable, double timeout_ms);
/* Steps taken by persistent launches since cel_ensemble_create. */
cel_status cel_ensemble_persistent_steps(const cel_ensemble *e, int64_t *steps);
cel_status cel_ensemble_check(cel_ensemble *e);
/* A check of the barrier's bound: one persistent launch that takes a single
 * barrier expecting `missing` more arrivals than it has blocks (0..1024),
 * waits at most timeout_ms, synchronises, and sets *timed_out to 1 if the
 * wait ran out (it must, for missing > 0) or 0 if the barrier completed.
 * The members are not touched. */
cel_status cel_ensemble_barrier_check(cel_ensemble *e, int32_t missing, double timeout_ms, int32_t *timed_out);
/* Kernel launches issued by the most recent cel_ensemble_step call. */
cel_status cel_ensemble_last_launch_count(const cel_ensemble *e, int64_t *launches);
/* Per-kernel event timing of the ensemble's launches, as cel_profile_* for a
 * solver (0: stencil, 1: line solves, one entry per line launch, 2: ghost
 * tables). */
cel_status cel_ensemble_profile_enable(cel_ensemble *e, int32_t capacity);
cel_status cel_ensemble_profile_read(cel_ensemble *e, double ms[3], int64_t count[3]);
cel_status cel_ensemble_profile_disable(cel_ensemble *e);
const char *cel_ensemble_last_error(const cel_ensemble *e);  /* never NULL */
/* Release the handle (not the members, not the table).  Does not synchronise. */
void cel_ensemble_destroy(cel_ensemble *e);

/* Fixed-scratch variant of the step, for callers that cannot allocate device
 * memory.  Some callers run inside a host application that owns the GPU's
 * memory (a rendering or visualisation engine with its own pool, where a
 * stray cudaMalloc is forbidden or breaks the engine's accounting); some run
 * real-time loops that must not allocate after start-up, because cudaMalloc
 * and cudaFree can synchronise the device and stall a frame; some are thin
 * bindings that can hand over a stream and a few existing buffers but have no
 * way to allocate or free device memory.  They cannot provide the workspace
 * that cel_create needs.  This call needs none: it keeps all its scratch (the
 * AB3 and AM4 carries, the increments of U* and V*, bed corners, depths and
 * dry-cell masks)
 * in one fixed array of CEL_NOALLOC_SCRATCH_BYTES that the library defines in
 * device memory; every GPU that loads the library holds that array until the
 * process exits.  The paper has no counterpart to this entry point.
 *
 * It advances the state (w_in, P_in, Q_in: [ny][nx] real, device) by nsteps
 * steps exactly as cel_create + cel_set_boundary + cel_set_state + cel_step
 * would, starting at time first_step * dt with a fresh AB3 history (the first
 * two steps are Euler), and writes the result to w_out, P_out, Q_out ([ny][nx]
 * real, device; may alias the inputs).  bcs: the four sides (CEL_WEST..
 * CEL_NORTH), or NULL for solid walls.  Asynchronous on cuda_stream.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  A grid whose
 * scratch would exceed CEL_NOALLOC_SCRATCH_BYTES is rejected with
 * CEL_ERR_WORKSPACE_TOO_SMALL (about 512 x 512 cells in FP32 with
 * corrector_iters >= 1, 256 x 256 in FP64); bad arguments give
 * CEL_ERR_INVALID_ARG.  A one-line reason is copied into msg (msg_len bytes,
 * may be NULL).  The first call on each device looks up the array's device
 * address (with that device current), and so does the first call after the
 * device's CUDA context changed (cudaDeviceReset, or another context made
 * current): the address is kept per device together with the context's unique
 * id.  Make that first call before any stream capture.  All calls share the one array and each call clears what must
 * start at zero, so calls that overlap on the GPU (on different streams, or
 * from different threads) race and give wrong results: serialise them. */
#define CEL_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
cel_status cel_advance_noalloc(const cel_grid *grid, const cel_params *params,
                               const cel_bc *bcs, const void *z_dev,
                               const void *w_in, const void *P_in,
                               const void *Q_in, void *w_out, void *P_out,
                               void *Q_out, int32_t nsteps, int64_t first_step,
                               void *cuda_stream, char *msg, size_t msg_len);

const char *cel_status_string(cel_status st);
const char *cel_last_error(const cel_solver *s);  /* "" if none; never NULL */
/* Release the handle (not the caller's memory).  Does not synchronise. */
void cel_destroy(cel_solver *s);

#ifdef __cplusplus
}
#endif
#endif
