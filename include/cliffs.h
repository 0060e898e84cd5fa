/*
 * cliffs.h - C ABI of the GB300 (sm_103a) shallow-water step library libcliffs.so.
 *
 * The library advances the nonlinear shallow-water equations of the Cliffs model
 * (E. Tolkova, "Cliffs User Manual", arXiv 1410.0753) on one structured grid: an x-sweep
 * over every row, then a y-sweep over every column (dimensional splitting, section
 * "Numerics", eqs. (eq2A), (eq2B)), each sweep the VTCS-2 update (solver2) on Riemann
 * invariants with the "moving cliff" inundation steps (a)-(e) (section "Inundation
 * algorithm"), in Cartesian or geographic-spherical metrics. It records max-wave, gauges
 * and boundary series for enclosed grids (section "Running Options", fields maxout, gout,
 * bndout). The state is FP32 on the device; bathymetry filtering runs in FP64.
 *
 * Conventions for every entry point:
 *  - Return value: CLIFFS_OK (0) or a negative CLIFFS_ERR_* code; the message of the last
 *    error on the calling thread is returned by cliffs_last_error().
 *  - Arrays passed in are owned by the caller and copied before the call returns; they may
 *    be host or device (CUDA unified addressing) pointers. Arrays passed out are filled
 *    before the call returns (the grid's stream is synchronised).
 *  - 2D fields are dense row-major [ny][nx], x (longitude) fastest, as the paper's output
 *    variables ha(time, lat, lon). Batched fields are [batch][ny][nx].
 *  - Indices are 0-based (the paper's parameter file is 1-based).
 *  - Depth d is positive down; negative values are land elevation (section "Running
 *    Options", "Bathymetry data").
 *  - A grid handle is not thread-safe; distinct handles may be used from distinct threads.
 */
#ifndef CLIFFS_H
#define CLIFFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLIFFS_OK            0
#define CLIFFS_ERR_ARG      -1   /* invalid argument (sizes, indices, CFL, nest outside grid) */
#define CLIFFS_ERR_STATE    -2   /* wrong call order (e.g. step before set_bathy) */
#define CLIFFS_ERR_CUDA     -3   /* a CUDA runtime call failed */
#define CLIFFS_ERR_UNSTABLE -4   /* a non-finite or runaway value appeared in the state */
#define CLIFFS_ERR_TIMEOUT  -5   /* a bounded device wait gave up */
#define CLIFFS_ERR_NOMEM    -6   /* device allocation failed */

#define CLIFFS_EDGE_WEST  0
#define CLIFFS_EDGE_EAST  1
#define CLIFFS_EDGE_SOUTH 2
#define CLIFFS_EDGE_NORTH 3

typedef struct cliffs_grid cliffs_grid;

/* An enclosed (nested) grid in master coordinates (parameter-file fields 3-4): nodes at
 * (x0 + i dx, y0 + j dy), i < nx, j < ny. Its boundary series are the master solution
 * interpolated bilinearly at its boundary nodes. */
typedef struct cliffs_nest {
    double  x0, y0, dx, dy;
    int32_t nx, ny;
} cliffs_nest;

/* Computational parameters (parameter-file fields 1, 6-10, 17-21). */
typedef struct cliffs_config {
    int32_t nx, ny;             /* nodes; nx == 1 or ny == 1 is a 1D grid; a 2D grid needs
                                   at least 3 nodes each way (section "Bathymetry data") */
    int32_t batch;              /* scenarios sharing the bathymetry (>= 1) */
    int32_t coords;             /* 1: Cartesian (m); otherwise geographic (degrees) */
    double  h_min;              /* 'ground': minimal flow depth, > 0; dry when h < h_min */
    double  manning_n2;         /* 'crough' read as Manning n^2; 0 disables friction */
    int32_t itopo;              /* 0: vertical wall at depth dwall; otherwise inundation */
    double  dwall;
    double  dt;                 /* time step, s; the CFL number |lambda| dt/dx must be <= 1 */
    int32_t transverse;         /* 1: advect the transverse velocity, eq. (pq3) */
    int32_t solver;             /* 2 (or 0): eq. (solver2); 1: eq. (solver1) */
    int32_t alternate;          /* 0: x then y every step; 1: y first on the odd steps
                                   (counted from 0 at set_initial), the alternating reading of
                                   section "Numerics"; every stepping path and the
                                   adjoint take it */
    int32_t maxout;             /* steps between max-wave updates (> 0) */
    int32_t gout;               /* steps between gauge records (> 0) */
    int32_t bndout;             /* steps between boundary-series records (> 0) */
    int32_t n_gauges;
    const int32_t* gauge_ixiy;  /* [2 * n_gauges]: (ix, iy) pairs; copied at create */
    int32_t n_nests;
    const cliffs_nest* nests;   /* [n_nests]; copied at create; 2D grids, batch == 1 only */
    void*   stream;             /* cudaStream_t for all work, or NULL (default stream) */
    int32_t open_edges;         /* open (radiating) outer edges, bits W 1, E 2, S 4, N 8;
                                   the others are reflecting walls. The paper gives no
                                   condition for an open edge; the reading taken: the ghost
                                   beyond a wet edge node carries the node's outgoing Riemann
                                   invariant and the incoming invariant of still water at the
                                   node's depth (sqrt(g max(d, 0))), the node's depth and
                                   transverse velocity; the adjoint takes the ghost as a
                                   function of the edge node. */
} cliffs_config;

/* Create a grid with the given parameters. Allocates the device state ([batch][ny][nx] of
 * eta, u, v, double-buffered), the max-wave fields and the record buffers. The handle is
 * owned by the library; release it with cliffs_destroy.
 * Errors: ERR_ARG for bad sizes, h_min <= 0, dt <= 0, out-of-range gauges, cadences < 1,
 * nests on a 1D or batched grid; ERR_NOMEM; ERR_CUDA. */
int cliffs_grid_create(const cliffs_config* cfg, cliffs_grid** out);

/* Set the bathymetry (section "Running Options", "Bathymetry data"): x[nx] and y[ny] node
 * coordinates (m, or degrees for geographic grids; strictly increasing), depth[ny][nx] in
 * FP64, positive down. With apply_filter != 0, the depth-jump filter of section "Numerical
 * stability" (eqs. (dstab), (newdw), (newdc); program depth_ssl) runs first on the device in
 * FP64 with limit alpha (1 < alpha < 3; 2 is typical) and minimal wet depth min_depth,
 * until a pass changes nothing (at most 100 passes). Checks that the nests lie inside the
 * grid and that the still-water Courant number sqrt(g d) dt / dx <= 1 in both directions
 * (section "Difference Scheme").
 * Errors: ERR_ARG (non-increasing coordinates, CFL > 1, nest outside), ERR_CUDA. */
int cliffs_set_bathy(cliffs_grid* g, const double* x, const double* y, const double* depth,
                     int apply_filter, double alpha, double min_depth);

/* Read back the FP64 depth in use (after the filter and any quake deformation), [ny][nx]
 * (host or device array). Errors: ERR_ARG (NULL argument); ERR_STATE before set_bathy. */
int cliffs_read_depth(cliffs_grid* g, double* depth);

/* Set the initial state of one scenario (scenario in [0, batch)) or of all (scenario = -1,
 * then eta/u/v hold [batch][ny][nx]) (section "Running Options", "input to the
 * computations"): free surface eta (m) and velocities u, v (m/s; NULL means zero). With
 * quake = 1 eta is a sea-floor deformation zeta (parameter-file field 12): the depth becomes
 * d - zeta and the free surface zeta on nodes that were wet (d >= h_min, and with itopo = 0
 * d >= dwall), 0 on the others; quake needs
 * batch == 1. Resets the step counter and the records, initialises max-wave from this state
 * and records step 0 (gauges, boundary series).
 * Errors: ERR_STATE before set_bathy; ERR_ARG; ERR_CUDA. */
int cliffs_set_initial(cliffs_grid* g, int scenario, const float* eta, const float* u,
                       const float* v, int quake);

/* Initial state interpolated from a source grid (section "Running Options", "The input to
 * the computations": the initial conditions need not cover the master grid nor share its
 * nodes; they are interpolated onto the part of the master grid inside the source grid and
 * set to zero outside it). sx[snx], sy[sny]: the source nodes, increasing, in the master's
 * units; eta, u, v: [sny][snx] FP32 (u, v may be NULL for zero). Master nodes inside the
 * source extent take the bilinear interpolation of the four surrounding source nodes (FP64
 * weights in coordinate space, rounded once to FP32); a source dimension of one node covers
 * only master nodes at exactly that coordinate. Then as cliffs_set_initial (scenario >= 0,
 * or -1 when batch == 1; quake as there). Errors: ERR_STATE before set_bathy; ERR_ARG. */
int cliffs_set_initial_interp(cliffs_grid* g, int scenario, const double* sx, int32_t snx, const double* sy,
                              int32_t sny, const float* eta, const float* u, const float* v, int quake);

/* Per-scenario step limits for a batched grid: scenario b stops after steps[b] steps
 * (its state, max-wave and records then stay as they were). steps[batch] is copied (host or
 * device); NULL removes the limits. Default: unlimited. Errors: ERR_ARG (no grid, a
 * negative duration). */
int cliffs_set_durations(cliffs_grid* g, const int64_t* steps);

/* Boundary input (section "Running Options", "The input to the computations": one series
 * per edge, vals(tim, uvq, pnt) of (u, v, eta) at times time(tim); parameter-file fields 5
 * and 13). edge: 0 W, 1 E, 2 S, 3 N; times[nt] in seconds, increasing; vals[nt][3][np] with
 * np = ny for W and E, nx for S and N (host or device arrays, copied). A 1D grid along x
 * takes W and E (one node each), along y S and N. The paper does not say how the input enters
 * the scheme; the reading taken here: before each step the edge nodes take the input's
 * values at the current model time, linearly interpolated between records (the first or last
 * record outside their span), edges in the order W, E, S, N (S and N own the corners); an
 * edge without input stays a reflecting wall. nt = 0 removes the edge's input. batch == 1
 * only; cliffs_step_n and the persistent run take it; the adjoint takes the input as fixed
 * (the imposed edge values carry no sensitivity). Errors: ERR_ARG (edge, sizes, times not increasing, batch > 1). */
int cliffs_set_boundary_input(cliffs_grid* g, int edge, const double* times, int64_t nt, const double* vals);

/* Model clock under boundary input (parameter-file fields 5, cuke, and 13). The run starts at
 * t_start: the first record time at which |eta| exceeds cuke anywhere on an input edge, or,
 * with cuke <= 0 (or no such record), the earliest record time. The state after k steps since
 * set_initial is at t_start + k dt, and the input for the step from it is taken at that time.
 * With stop_at_end != 0, cliffs_step_n ends early (returning CLIFFS_OK) before a step whose
 * result would lie past the end of the shortest record; cliffs_steps_done tells how far it
 * went. Writes t_start when the pointer is not NULL. Errors: ERR_STATE without input. */
int cliffs_set_boundary_clock(cliffs_grid* g, double cuke, int stop_at_end, double* t_start);

/* Advance n time steps. One step is an x-sweep over every row then a y-sweep over every
 * column (order alternates when cfg.alternate), each with the inundation steps (a)-(e) and
 * eq. (solver2); then max-wave (every maxout steps), gauges (every gout) and boundary
 * series (every bndout) are recorded. Kernels are launched on the grid's stream; the call
 * synchronises once at the end to check the device error flag.
 * Errors: ERR_STATE before set_initial; ERR_UNSTABLE when a non-finite value appeared
 * (the state is left as computed); ERR_CUDA. */
int cliffs_step_n(cliffs_grid* g, int64_t n);

/* Advance n time steps like cliffs_step_n, with the same results bit for bit, in ONE kernel
 * launch (no counterpart in the paper, which runs one scenario at a time): a persistent,
 * cooperatively launched kernel whose warps take (scenario, tile) work items of the
 * scenarios still running at each step and meet at a grid-wide barrier between steps.
 * Scenarios are visited in decreasing order of their cliffs_set_durations limit, so a
 * batch of uneven durations keeps every SM busy until the longest ends. The launch is
 * captured once into a CUDA graph (a copy of the step range into a device control block,
 * then the kernel) and replayed by later calls; it is captured again when a launch argument
 * changes (tile shape, record buffers, durations). 2D grids only; the alternating order, open
 * edges and boundary input are taken (the input is imposed by the kernel before each step
 * from the interpolation cliffs_step_n would use, computed on the host; the run stops where
 * cliffs_step_n would stop), a recorded run is not (cliffs_step_n). The grid barrier waits
 * at most about a second per step before it sets the timeout flag.
 * Errors: ERR_STATE before set_initial; ERR_ARG (1D grid, n < 0, a recorded run);
 * ERR_UNSTABLE as for
 * cliffs_step_n; ERR_TIMEOUT when a bounded wait gave up; ERR_CUDA (including a device
 * that cannot launch cooperatively). */
int cliffs_run_persistent(cliffs_grid* g, int64_t n);

/* Gradient of a gauge misfit with respect to the initial free surface (no counterpart in
 * the paper, which has no adjoint). Let X_0 be the grid's current state and X_1..X_n the
 * states of the next n steps; dL_dgauges[r][g] (row-major, r = 0 .. n/gout) is dL/d eta at
 * gauge g after r*gout of those steps. Writes dL/d eta(X_0) to dL_deta0 ([ny][nx], host or
 * device). The forward run is recomputed on the device: a state is kept every
 * checkpoint_every steps, and each segment is run again with all its states stored before
 * the adjoint steps go back through it. Each adjoint step is the transpose of the Jacobian
 * of the y-sweep, then of the x-sweep (eqs. (eqQ), (solver2), (stateu), (stateh), (pq3)),
 * with every branch of the inundation steps (a)-(e), the mirror walls and the friction
 * clamp taken as in the forward run. The grid's state, records and maxima are unchanged.
 * Under boundary input each adjoint step zeroes the input edges of the adjoint state (the
 * edge values were overwritten before the step) before the gauge records of that state are
 * added. dL_dgauges may be NULL (the gradient is then zero). 2D grids; on a batched grid
 * this is scenario 0 (cliffs_adjoint_scenario takes any). With the alternating order the
 * steps keep the forward's parity (steps counted from set_initial).
 * With checkpoint_every == 1 every state is kept and read in place: no recomputation, at
 * n states of 12 bytes per node (25 GB for 2000 steps of a 1024^2 grid).
 * Segments are recomputed several at a time, as one batched launch per step, when neither
 * boundary input nor the alternating order is set: as many segments NG as fit in 16 GiB of
 * recomputed states, at least one and at most 16. The checkpoint pass keeps every state of
 * the last NG segments (1 with boundary input or the alternating order) in that space, so
 * those are not recomputed.
 * Memory: (NG checkpoint_every + ceil(n / checkpoint_every) + 6) states of 12 bytes per
 * node, kept for later calls; if the NG segments do not fit, fewer are tried.
 * Errors: ERR_STATE before set_initial; ERR_ARG (1D grid, n < 1, checkpoint_every < 1,
 * NULL output); ERR_UNSTABLE, ERR_TIMEOUT from the forward
 * recomputation; ERR_CUDA. */
int cliffs_adjoint_n(cliffs_grid* g, int64_t n, int32_t checkpoint_every, const float* dL_dgauges,
                     float* dL_deta0);

/* cliffs_adjoint_n for scenario `scenario` of a batched grid (cliffs_adjoint_n is scenario 0):
 * X_0 is that scenario's current state, dL_dgauges its gauge records' adjoint. With
 * per-scenario durations (cliffs_set_durations) the scenario must still run n more steps.
 * The other scenarios are untouched. Errors: as cliffs_adjoint_n, and ERR_ARG for a
 * scenario outside 0..batch-1 or a run that stops before n steps. */
int cliffs_adjoint_scenario(cliffs_grid* g, int32_t scenario, int64_t n, int32_t checkpoint_every,
                            const float* dL_dgauges, float* dL_deta0);

/* cliffs_adjoint_scenario for a loss on the whole gauge records: dL_drecords[r][g][3] holds
 * dL/d (eta, u, v) at gauge g after r*gout steps (the layout cliffs_read_gauges writes), so
 * misfits of the recorded velocities differentiate too. Errors: as cliffs_adjoint_scenario. */
int cliffs_adjoint_records(cliffs_grid* g, int32_t scenario, int64_t n, int32_t checkpoint_every,
                           const float* dL_drecords, float* dL_deta0);

/* cliffs_adjoint_recorded with dL/d (eta, u, v) of the records, [nrec][G][3].
 * Errors: as cliffs_adjoint_recorded. */
int cliffs_adjoint_recorded_records(cliffs_grid* g, const float* dL_drecords, float* dL_deta0);

/* cliffs_adjoint_recorded for scenario `scenario` of a recorded batched run, with
 * components 1 (dL/d eta of the records, [nrec][G]) or 3 (dL/d (eta, u, v), [nrec][G][3]).
 * The scenario must have run every recorded step (its duration at least the record's
 * length). Errors: ERR_STATE without a record; ERR_ARG (scenario outside 0..batch-1, a
 * scenario that stopped earlier, components not 1 or 3); as cliffs_adjoint_n. */
int cliffs_adjoint_recorded_scenario(cliffs_grid* g, int32_t scenario, int32_t components, const float* dL,
                                     float* dL_deta0);

/* Record the forward run for the adjoint (no counterpart in the paper). With
 * checkpoint_every = K > 0, called right after cliffs_set_initial, the initial state and then
 * every K-th state produced by cliffs_step_n are kept (12 bytes per node and scenario each,
 * the store grows as the run does), so that cliffs_adjoint_recorded needs no checkpoint pass
 * of its own. A later cliffs_set_initial starts a new record with the same spacing; K = 0
 * stops recording and frees the store. A recording grid runs through cliffs_step_n only (the
 * persistent run rejects it). On a batched grid every scenario is recorded
 * (cliffs_adjoint_recorded_scenario). Errors: ERR_STATE before set_initial or after steps
 * since it; ERR_ARG (K < 0, 1D grid). */
int cliffs_adjoint_record(cliffs_grid* g, int32_t checkpoint_every);

/* cliffs_adjoint_n for the run recorded since the last cliffs_set_initial: n = the steps
 * done since, X_0 = the recorded initial state, checkpoints = the recorded ones. Each segment
 * is recomputed once from its checkpoint and the adjoint steps go back through it; the grid's
 * current state is not used and not changed. Errors: ERR_STATE without a recorded run of at
 * least one step; otherwise as cliffs_adjoint_n. */
int cliffs_adjoint_recorded(cliffs_grid* g, const float* dL_dgauges, float* dL_deta0);

/* The rest of the last adjoint's result: dL/du and dL/dv of the initial state ([ny][nx] each,
 * host or device; either may be NULL), for the loss whose gauge-eta derivative the last
 * successful cliffs_adjoint_n or cliffs_adjoint_recorded call was given. Errors: ERR_STATE
 * when no adjoint has run. */
int cliffs_adjoint_velocity(cliffs_grid* g, float* dL_du0, float* dL_dv0);

/* Choose the tile shape of the 2D step kernel by measurement (the rows S each warp of the
 * fused step owns: a warp walks S + 6 rows, so larger S means less halo work but fewer,
 * longer warps, and the count of warps against the resident slots decides the tail). Each
 * candidate S is timed over `trials` launches (after one warm-up) that read the current
 * state and write scratch planes, with max-wave and records off, each after a 192 MiB write
 * that evicts the inputs from L2; the fastest is kept for later steps. The grid's state, maxima and records are unchanged.
 * Optional outputs: cand[] and us[] (capacity 16) receive the candidates and their best
 * times in microseconds, *ncand their count (0 for 1D grids, which have no tile shape).
 * Errors: ERR_STATE before set_initial; ERR_NOMEM; ERR_CUDA; ERR_TIMEOUT. */
int cliffs_autotune(cliffs_grid* g, int trials, int32_t* cand, double* us, int32_t* ncand);

/* Set the tile shape of the 2D step kernel directly: `rows` output rows per warp (what
 * cliffs_autotune chooses by measurement), e.g. to repeat a measured configuration. Call it
 * after cliffs_set_bathy, which chooses a default shape. Results do not depend on the shape.
 * Errors: ERR_STATE before set_bathy; ERR_ARG (1D grid, rows outside 1..8192); ERR_NOMEM;
 * ERR_CUDA. */
int cliffs_set_rows_per_warp(cliffs_grid* g, int32_t rows);

/* Fault injection for tests of the bounded waits (no counterpart in the paper): the next
 * step launch of a 2D grid makes every shared-memory ring slot expect 16 bytes more than
 * its copies deliver, with waits limited to `cycles` clock cycles. Each wait then expires,
 * the kernel drains its copies (bounded), sets the timeout flag and returns; later launches
 * of the same call return at once; cliffs_step_n returns CLIFFS_ERR_TIMEOUT and the grid
 * stays usable (its state is whatever the interrupted step left). The injection applies to
 * the next cliffs_step_n or cliffs_run_persistent call, whichever comes first. No GPU fault
 * or hang is involved. Errors: ERR_ARG (no grid, cycles <= 0, 1D grid). */
int cliffs_inject_wait_expiry(cliffs_grid* g, int64_t cycles);

/* Steps completed since set_initial (for a batched grid, by the longest scenario).
 * Errors: ERR_ARG (NULL argument). */
int cliffs_steps_done(cliffs_grid* g, int64_t* steps);

/* Gauge records of one scenario (section "Running Options", the _gages output): writes
 * out[nrec][n_gauges][3] as (eta, u, v) at steps 0, gout, 2 gout, ... (host or device) and
 * sets *nrec. With out == NULL only *nrec is set. Errors: ERR_ARG (NULL grid or nrec, a
 * scenario outside 0..batch-1). */
int cliffs_read_gauges(cliffs_grid* g, int scenario, float* out, int64_t* nrec);

/* Max-wave of one scenario (the _maxwave output): maximal eta and maximal current
 * sqrt(u^2 + v^2) over wet nodes at the steps multiple of maxout and at the current
 * (last) step, [ny][nx] each (host or device); never-wet nodes hold -FLT_MAX and 0. Either
 * pointer may be NULL. Errors: ERR_ARG (no grid, scenario out of range); ERR_STATE before
 * set_initial. */
int cliffs_read_maxwave(cliffs_grid* g, int scenario, float* eta_max, float* speed_max);

/* Boundary series for one edge of one enclosed grid (the _west/_east/_south/_north
 * outputs): vals[nt][3][np] as (u, v, eta) in FP64 at steps 0, bndout, 2 bndout, ..., with
 * np = nest ny (west, east) or nx (south, north), the master state interpolated bilinearly
 * in the master grid's index space. With vals == NULL only *nt is set. Errors: ERR_ARG
 * (NULL grid or nt, nest or edge out of range). */
int cliffs_read_boundary(cliffs_grid* g, int nest, int edge, double* vals, int64_t* nt);

/* Current state of one scenario, [ny][nx] each (host or device); any pointer may be NULL.
 * Errors: ERR_ARG (no grid, scenario out of range). */
int cliffs_read_state(cliffs_grid* g, int scenario, float* eta, float* u, float* v);

/* The current state of one scenario as library-owned device memory, for zero-copy views
 * (section "Running Options": the wave state the screenshots hold): eta, u, v point to
 * [ny] rows of *pitch floats (the first nx of each row are the nodes). The grid alternates
 * two state buffers, so the pointers are valid until the next call that steps or sets the
 * state; writing through them changes the state the next step starts from. Any output
 * pointer may be NULL. Errors: ERR_ARG (scenario out of range). */
int cliffs_state_ptrs(cliffs_grid* g, int scenario, float** eta, float** u, float** v, int64_t* pitch);

/* Diagnostics of the current state of one scenario (a monitor beside the status codes; the
 * paper's program logs to a text file instead, section "Running Options"). Over wet nodes
 * (eta + d >= h_min, and with itopo = 0 d >= dwall, the max-wave test) out[4] (host)
 * receives: out[0] the displaced volume sum eta * A (m^3; A the node's area from its control
 * widths, half the distance to each neighbour and the full spacing at an end node, in
 * geographic metrics R^2 cos(phi) dlambda dphi; a one-node axis counts 1 m), out[1] the
 * number of wet nodes, out[2] max |eta| (m), out[3] the maximum speed sqrt(u^2 + v^2)
 * (m/s). The call synchronises. Errors: ERR_ARG (NULL argument, scenario out of range);
 * ERR_STATE before set_initial; ERR_CUDA. */
int cliffs_diagnostics(cliffs_grid* g, int scenario, double* out);


/* Kernel timing: enable != 0 records CUDA events around every sweep kernel launch (on the
 * grid's stream) from now on; *ms and *launches (either may be NULL) receive the total
 * device time and count of those launches since timing was enabled or last reset; the call
 * synchronises. enable < 0 resets the totals. Errors: ERR_ARG (no grid); ERR_CUDA. */
int cliffs_kernel_time(cliffs_grid* g, int enable, double* ms, int64_t* launches);

/* The depth-jump filter of cliffs_set_bathy for callers that cannot allocate device
 * memory. The paper has no counterpart of this entry point. It serves callers that must not
 * call cudaMalloc or cudaFree: applications whose own memory pool owns the whole device and
 * forbids allocations behind its back (a hidden allocation can fail, or fragment the pool),
 * and callers that cannot afford cudaFree's device-wide synchronisation, which stalls every
 * stream on the device. It allocates nothing: its scratch (a second FP64 Jacobi buffer and
 * a flag) is one static device array of CLIFFS_NOALLOC_MAX_CELLS doubles (8 MiB) that every
 * GPU loading the library holds until the process exits.
 *   depth   [ny][nx] FP64 input depth, positive down (host or device memory)
 *   out     [ny][nx] FP64 filtered depth, DEVICE (or managed) memory owned by the caller;
 *           it may be the same array as depth, but may not partly overlap it
 *   alpha, min_depth  as in cliffs_set_bathy; stream: cudaStream_t or NULL
 *   passes  receives the passes made (-1: stopped at the 100-pass cap); may be NULL
 * The result is bit-identical to the filter cliffs_set_bathy applies (both launch the same
 * per-node code). Errors: CLIFFS_ERR_ARG, with nothing launched, for a NULL pointer, an
 * empty grid, alpha outside (1, 3), an out that is not device memory, arrays that partly
 * overlap, or nx * ny larger than CLIFFS_NOALLOC_MAX_CELLS (the limit is in
 * cliffs_last_error()); CLIFFS_ERR_CUDA for a failed runtime call.
 * The first call on each device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current and keeps it; make that first call before
 * any stream capture. The kept address does not survive cudaDeviceReset. Every call on a
 * device shares the one array and leaves its last contents there (the flag is cleared
 * before each pass): calls that overlap on the GPU (other streams or threads) race and give
 * wrong results. The call synchronises the stream once per pass to read the flag. */
#define CLIFFS_NOALLOC_MAX_CELLS (1 << 20)
int cliffs_depth_filter_noalloc(const double* depth, double* out, int32_t nx, int32_t ny,
                                double alpha, double min_depth, void* stream, int32_t* passes);

/* Release every device buffer of the grid. NULL is allowed. */
void cliffs_destroy(cliffs_grid* g);

/* Message of the last error on the calling thread ("" if none). */
const char* cliffs_last_error(void);

/* ABI version of this header (2: cliffs_config gained open_edges). */
int cliffs_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CLIFFS_H */
