/*
 * adi.h -- C ABI of libadi, a GB300 (sm_103a) engine for the Peaceman-Rachford ADI time
 * step of the two 2-D acoustic schemes of Otero, Rojas, Moya and Castillo (arXiv
 * 2006.07583):
 *   ADI_CFD  fourth-order compact finite differences on the nodal mesh (Sec. 2.1, Eq. 4,
 *            App. A), one coupled line system per grid line (Eq. 8, Eq. 10);
 *   ADI_MFD  fourth-order mimetic divergence/gradient on the staggered mesh (Sec. 2.2,
 *            Eq. 12, App. B).
 * One time step is stage 1 (Eq. 6: implicit along every x-line) followed by stage 2
 * (Eq. 7: implicit along every y-line).  The line systems are solved exactly, i.e. the
 * library returns the fixed point of the paper's ADI iteration (Eq. 9).
 *
 * Conventions shared by every entry point
 *   - Grids have nx cells along x and ny along y, square cells of side h.  Arrays are
 *     row-major with i (row) the y index and j (column) the x index.
 *       CFD: U, V, W are (ny+1) x (nx+1) node arrays.
 *       MFD: U is (ny+2) x (nx+2) (cell centres plus the four edges), V is
 *            (ny+2) x (nx+1) (x-nodes), W is (ny+1) x (nx+2) (y-nodes); U's corners are
 *            unused.
 *     The wave speed c is given where U lives; density is 1 and kappa = c^2.
 *   - Dirichlet data: the pressure values on U's outer rows and columns (as given to
 *     adi_create or adi_set_fields) are held fixed while stepping (time-independent walls;
 *     zero for a free surface).
 *   - nx, ny >= 16 (ADI_MIN_CELLS) and <= ADI_MAX_CELLS.
 *   - Every function returns an adi_status (0 = ADI_OK).  Errors from device work are
 *     sticky per handle: once a kernel fails, later calls on that handle return the same
 *     code until the handle is destroyed.
 *   - Input arrays are copied; the library owns all device memory it allocates; output
 *     buffers belong to the caller.  A handle is not thread-safe; distinct handles are.
 */
#ifndef ADI_H
#define ADI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADI_MIN_CELLS 16
#define ADI_MAX_CELLS 16384

typedef enum { ADI_CFD = 0, ADI_MFD = 1 } adi_method;
typedef enum { ADI_FP32 = 0, ADI_FP64 = 1 } adi_precision;
/* Line solvers:
 *   ADI_SOLVER_LINE      one thread per grid line, factorisation on the fly (the plain path);
 *   ADI_SOLVER_CHUNKED   lines split into chunks joined by a separator system, factorisation
 *                        on the fly;
 *   ADI_SOLVER_FACTORED  per-chunk block-LU records built once in FP64 and kept on the
 *                        device, line inputs staged by bulk asynchronous copies, chunks in
 *                        registers joined by scans (the default where the line length allows
 *                        it, else CHUNKED, else LINE). */
typedef enum { ADI_SOLVER_LINE = 0, ADI_SOLVER_CHUNKED = 1, ADI_SOLVER_FACTORED = 2 } adi_solver;

typedef enum {
    ADI_OK = 0,
    ADI_EINVAL = 1,      /* bad argument: sizes, h/dt <= 0, c <= 0, NaN input, bad index */
    ADI_ENOMEM = 2,      /* device allocation failed or the request exceeds a budget     */
    ADI_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed                  */
    ADI_ENONFINITE = 4,  /* a field became NaN/Inf (checked by adi_check_finite)         */
    ADI_ETIMEOUT = 5,    /* a bounded wait ran out                                       */
    ADI_EBUSY = 6,       /* the object is in use (e.g. a member of a live batch)         */
    ADI_ENOTSUP = 7,     /* no usable CUDA device / unsupported configuration            */
    ADI_ESINGULAR = 8    /* a line system's precomputed pivot block was singular         */
} adi_status;

typedef struct adi_sim *adi_handle;
typedef struct adi_batch_t *adi_batch;

/* Version of this ABI (bumped on incompatible change). */
int adi_abi_version(void);
const char *adi_strerror(int code);

/*
 * adi_create -- one simulation resident on the current CUDA device: the velocity-pressure
 * system of Sec. 2, Eq. 1 (u_t = -kappa div(v,w) + f, rho (v,w)_t = -grad u) on nx x ny
 * cells with Dirichlet pressure on the walls, discretised by Eq. 4 (CFD, nodal mesh of
 * Sec. 2.1) or Eq. 12 (MFD, staggered mesh of Sec. 2.2; field placement as in Sec. 2.2).
 *   method     ADI_CFD or ADI_MFD.
 *   nx, ny     cells along x and y (16 .. 16384).
 *   h, dt      cell side and time step, both > 0 and finite.
 *   c_field    host, wave speed at U's points (shape as U), every value > 0; copied.
 *   u0,v0,w0   host initial fields (shapes above) or NULL for zeros; u0's outer rows and
 *              columns are the Dirichlet data.  Copied.
 *   precision  ADI_FP32 (bulk arithmetic FP32, per-line factors precomputed in FP64) or
 *              ADI_FP64.
 * The simulation clock starts at t = 0.  On failure *out is NULL.
 * Device memory: the carried state in both line layouts, two velocity copies each, alpha
 * in both layouts, the natural outputs and the solver's per-line records (about 15 fields'
 * worth at 4096^2 in FP32); adi_state_bytes() reports the exact figure.
 */
int adi_create(adi_handle *out, int method, int nx, int ny, double h, double dt,
               const double *c_field, const double *u0, const double *v0, const double *w0,
               int precision);

/*
 * adi_set_solver -- choose the line solver of a handle (adi_solver); rebuilds its per-line
 * factors.  ADI_ENOTSUP if the requested solver cannot take lines this long; ADI_EBUSY
 * inside a batch.  Lines longer than one CTA's chunks run as split lines in the factored
 * solver; where a split line's scan reach exceeds what a sub-line's halo takes, the handle
 * falls back to the chunked solver.  adi_get_solver returns the current one (-1 for a NULL
 * handle).
 */
int adi_set_solver(adi_handle sim, int solver);
int adi_get_solver(adi_handle sim);

/*
 * adi_get_scan_reach -- the factored solver's chunk-joining reach (a property of the solver,
 * not of the paper): the largest number of consecutive chunks, over the handle's lines, whose
 * transfer product still exceeds the neglect threshold (2^-40 for FP32 records, 2^-70 for
 * FP64).  Lines of a handle whose reach is above 32 join their chunks with full log-depth scans
 * instead of windowed ones.  *reach = 0 for the other solvers.  Errors: ADI_EINVAL (NULL).
 */
int adi_get_scan_reach(adi_handle sim, int *reach);

/*
 * adi_autotune -- picks the line solver of a handle by measurement.  Every solver the
 * configuration supports (ADI_SOLVER_FACTORED, _CHUNKED, _LINE: the chunk-parallel solves and
 * the thread-per-line Thomas-style elimination) runs `trials` steps (rounded up to an even
 * count, after as many untimed ones) on the handle's own state, timed with CUDA events on its
 * stream, and the fastest is kept.  The carried state, the natural fields, the step clock and
 * the parity are saved on the device first and restored afterwards, so the fields read
 * exactly as before the call.  ms_per_step (NULL, or 3 entries indexed by adi_solver)
 * receives each solver's time per step, -1 for one the configuration cannot use; *chosen
 * (may be NULL) the winner.  Results are cached per (method, nx, ny, precision) for the
 * process: a cached configuration is switched to its solver without timing unless force != 0.
 * Errors: ADI_EINVAL (trials < 1), ADI_EBUSY inside a batch, ADI_ENOMEM if the save buffer
 * (the size of the simulation's fields) cannot be allocated -- the handle is then unchanged.
 */
int adi_autotune(adi_handle sim, int trials, int force, int *chosen, double *ms_per_step);

/*
 * adi_set_launch / adi_get_launch -- launch parameters of the factored line solver (the paper
 * has no counterpart: GPU launch shape).  lines_per_cta caps the lines one CTA solves together
 * (0: as many as its threads and shared memory take); ring_depth caps the staged groups in
 * flight per CTA (0: as many as shared memory takes, at most 3; 1: no prefetch; 2: prefetch
 * the next group while solving one; 3: the next two).  The results do not change (every line
 * is solved by the same arithmetic), only the time.  When the factored solver is the fastest,
 * adi_autotune also times every lines_per_cta from the automatic count halved down to 1 with
 * the ring depths 0, 1 and 2, keeps the fastest and caches it with the solver choice;
 * adi_get_launch reports the current caps (0 = automatic).
 * Errors: ADI_EINVAL (ring_depth outside 0..3), ADI_EBUSY inside a batch.
 */
int adi_set_launch(adi_handle sim, int lines_per_cta, int ring_depth);
int adi_get_launch(adi_handle sim, int *lines_per_cta, int *ring_depth);

/* Device bytes adi_create allocates for this configuration with its default solver (0 if
 * invalid); transient staging buffers are not included. */
size_t adi_state_bytes(int method, int nx, int ny, int precision);

/*
 * adi_set_source -- Ricker point source s(t) = amp (1 - 2 pi^2 f0^2 tau^2)
 * exp(-pi^2 f0^2 tau^2), tau = t - tdelay, added as the forcing f = s(t)/h^2 of Eq. 1 at
 * the interior pressure point U[is][js] (Eq. 5-7 source terms A_F at t_m and t_{m+1}).
 * is, js must index an interior pressure point.  Replaces any previous source.
 */
int adi_set_source(adi_handle sim, int is, int js, double amp, double f0, double tdelay);

/*
 * adi_set_harmonic -- time-harmonic Dirichlet walls and a distributed forcing, the data of the
 * manufactured problem of Sec. 4 (Eq. 11: u = Psi(x, y) cos(2 pi t / T) with its forcing):
 *     u(t) = B cos(omega t + phase_b)   on U's outer rows and columns,
 *     f(t) = F cos(omega t + phase_f)   at U's interior points (Eq. 1's forcing term),
 * added to the carried state as Eqs. 6-7 add the source (dt/2 f(t_m) in stage 1, dt/2
 * f(t_{m+1}) in stage 2), t = steps * dt.  The intermediate pressure u* on the ends of the
 * x-lines (west and east walls) is taken at the half step, u(t_m + dt/2); the y-lines' ends
 * (south and north walls) take u(t_{m+1}).  The paper does not state u*'s wall value; this
 * reading gives the second-order convergence that Tables 4-5 report for Gamma != 0.
 *   B   host, U's shape; only its outer rows and columns are read.  NULL: back to
 *       time-independent walls (the values the fields hold at the call).
 *   F   host, U's shape, or NULL for no forcing; only interior points are read.
 * The current fields' walls are replaced by B cos(omega t_now + phase_b) and the carried state
 * is rebuilt at the current time.  A point source (adi_set_source) may be combined with it.
 * Velocities on the walls' own lines (v on the south/north rows, w on the west/east columns)
 * are not advanced, as in the paper's algorithms (they never enter the pressure).
 * Not used by adi_step_static or adi_fixed_point.  Device memory: the wall amplitudes and,
 * with F, two copies of F in the carried layouts (not counted by adi_state_bytes).
 * Errors: ADI_EINVAL (non-finite values, F without B), ADI_EBUSY in a batch, ADI_ENOMEM,
 * ADI_ECUDA.
 */
int adi_set_harmonic(adi_handle sim, const double *B, const double *F, double omega,
                     double phase_b, double phase_f);

/*
 * adi_set_sponge -- absorbing layers along every wall: Cerjan's damping, the technique Sec. 2.1
 * names for absorbing boundaries.  After every full step each field value at a point whose
 * distance to the nearest wall is delta cells, delta < width, is multiplied by
 *     g = exp(-(a (width - delta))^2)
 * (Cerjan's classic choice is width 20, a = 0.015); the pressure's wall values (the Dirichlet
 * data) are not damped.  Distances use the mesh of each field: nodes (CFD), cell centres and
 * faces (MFD).  width = 0 or a = 0 removes the layers.
 * A simulation with layers writes its natural fields every step and rebuilds its carried state
 * from the damped fields (the work of adi_set_fields' prologue), about one more stage's worth
 * of memory traffic per step.  Works with batches, graphs, sources and adi_set_harmonic.
 * Device memory: the y-line descriptors of both parities and the prologue's scratch.
 * Errors: ADI_EINVAL (negative or non-finite values), ADI_EBUSY in a batch, ADI_ENOMEM,
 * ADI_ECUDA.
 */
int adi_set_sponge(adi_handle sim, double width, double a);

/* adi_set_stream -- CUDA stream (cudaStream_t, NULL = legacy default) for later calls. */
int adi_set_stream(adi_handle sim, void *cuda_stream);

/*
 * adi_step -- enqueue nsteps >= 0 full time steps on the handle's stream.  Each step is the
 * Peaceman-Rachford split of Eq. 5: stage 1 (Eq. 6) solves the coupled line system of Eq. 8
 * on every interior x-line, stage 2 (Eq. 7) the system of Eq. 10 on every interior y-line,
 * each exactly (the fixed point of Eq. 9).  Asynchronous: returns after launching.  For
 * nsteps >= 2 the step loop is captured once into a CUDA graph and replayed.  The stream is
 * the one set by adi_set_stream (the handle's own stream by default).
 * Errors: ADI_EINVAL (nsteps < 0), ADI_EBUSY (member of a live batch or ticket), ADI_ECUDA,
 * or the handle's sticky error.
 */
int adi_step(adi_handle sim, int nsteps);

/* adi_sync -- wait for the handle's stream; returns the first sticky error. */
int adi_sync(adi_handle sim);

/*
 * adi_read_fields -- synchronise and copy the current (U, V, W) into caller-owned host
 * buffers with the shapes above (any pointer may be NULL to skip that field): pressure and
 * the two velocity components of Eq. 1 at the mesh points of Sec. 2.1 (CFD: all on nodes) or
 * Sec. 2.2 (MFD: pressure at cell centres and edges, v on x-faces, w on y-faces), at the
 * handle's current time.  Fields that need converting or packing (FP64 arrays, a padded
 * velocity array) pass through a device staging buffer of three fields in FP64, allocated on
 * its first use and kept until adi_destroy.  Errors: the handle's sticky error, ADI_ENOMEM (the
 * staging buffer), ADI_ECUDA.
 */
int adi_read_fields(adi_handle sim, double *u, double *v, double *w);

/*
 * adi_set_fields -- replace the current (U, V, W) by host arrays (shapes above; NULL keeps
 * that field) and rebuild the carried stage-1 state (Eq. 8's A and W* of Alg. 1/2) at the
 * current simulation time.  U's outer rows/columns become the new Dirichlet data.  Allowed
 * for a member of a batch (the batch's stream is synchronised first).
 */
int adi_set_fields(adi_handle sim, const double *u, const double *v, const double *w);

/*
 * adi_set_fields_f32 / adi_read_fields_f32 -- adi_set_fields and adi_read_fields with FP32
 * host arrays (same shapes), for callers whose fields live in single precision: an FP32
 * simulation's fields then cross the host link at half the bytes, without conversion on the
 * host.  An FP64 simulation converts them on the device (reading rounds to FP32).  The same
 * finite check, errors and batch behaviour as the FP64 calls.
 */
int adi_set_fields_f32(adi_handle sim, const float *u, const float *v, const float *w);
int adi_read_fields_f32(adi_handle sim, float *u, float *v, float *w);

/* adi_check_finite -- scans U, V, W on the device; ADI_ENONFINITE if any is NaN/Inf. */
int adi_check_finite(adi_handle sim);

/* Completed steps and the simulation time t = steps * dt. */
int adi_get_time(adi_handle sim, long long *steps, double *t);

/* adi_destroy -- frees everything the handle owns (NULL is accepted); ADI_EBUSY, freeing
 * nothing, while the handle is a member of a batch or of an unfinished ticket. */
int adi_destroy(adi_handle sim);

/*
 * Batching.  adi_batch_create groups n >= 1 simulations of one precision (any mix of
 * methods and sizes) so that every half step of all of them runs as ONE kernel launch
 * over a table of line descriptors (uneven lines from many simulations).  Members stay
 * valid handles but must not be stepped individually while the batch lives (ADI_EBUSY).
 * adi_batch_step(b, k) advances every member by k steps on the batch's stream, captured
 * as a CUDA graph.
 */
int adi_batch_create(adi_batch *out, const adi_handle *sims, int n);
int adi_batch_set_stream(adi_batch b, void *cuda_stream);
int adi_batch_step(adi_batch b, int nsteps);
int adi_batch_sync(adi_batch b);
/*
 * adi_batch_half_step -- enqueue ONE stage for every member: stage 1 (Eq. 6, all x-lines)
 * or stage 2 (Eq. 7, all y-lines); write_natural != 0 makes stage 2 also refresh the
 * natural u, w that adi_read_fields returns.  A full step is stage 1 then stage 2; the
 * caller must issue them in that order (used to time each kernel separately).
 */
int adi_batch_half_step(adi_batch b, int stage, int write_natural);
/*
 * adi_batch_set_timing -- enable != 0: every later adi_batch_half_step also records CUDA
 * events on the batch's stream around its line-solve launches (the transpose of the carried
 * pressure that follows them is outside).  adi_batch_solve_time synchronises the stream and
 * returns, for stage 1 or 2, the summed milliseconds and the number of half steps recorded
 * since the previous query, then clears the record.  Timing does not change the work done.
 */
int adi_batch_set_timing(adi_batch b, int enable);
int adi_batch_solve_time(adi_batch b, int stage, double *total_ms, int *count);
int adi_batch_destroy(adi_batch b);

/*
 * Serving.  A server runs simulations requested at any time on the current device:
 * requests wait in a FIFO queue and are admitted, in order, while the device memory their
 * state needs (adi_server_bytes) fits in the server's HBM budget and fewer than max_active
 * are running.  Admitted simulations stay resident and advance together: adi_server_tick
 * advances every running simulation by the same number of steps -- the server's quantum, or
 * fewer so that none passes its requested step count -- as one batch (one kernel launch per
 * half step and kernel variant over all their lines, adi_batch_*), then retires the finished
 * ones (their fields are copied to host memory and their device memory is freed) and admits
 * waiting requests into the freed budget.  The batch is re-formed whenever its membership
 * changes.  Requests arriving while others run are thus admitted at the next tick (continuous
 * batching).  The paper has no counterpart; the simulations themselves are the library's.
 * A server is not thread-safe.
 */
typedef struct adi_server_t *adi_server;
typedef struct {
    int method, nx, ny;          /* as adi_create */
    double h, dt;
    const double *c_field;       /* host, shape of U; copied by adi_server_submit */
    const double *u0, *v0, *w0;  /* host initial fields or NULL (zeros); copied */
    int nsteps;                  /* steps to run, >= 0 */
    int has_source;              /* nonzero: Ricker source (adi_set_source) below */
    int src_i, src_j;
    double src_amp, src_f0, src_tdelay;
} adi_request;
enum { ADI_REQ_PENDING = 0, ADI_REQ_RUNNING = 1, ADI_REQ_DONE = 2, ADI_REQ_FAILED = 3 };

/* Device bytes the server reserves for one request: adi_state_bytes plus its share of the
 * batch's line descriptors (0 if the configuration is invalid). */
size_t adi_server_bytes(int method, int nx, int ny, int precision);
/* hbm_budget: bytes the server's simulations may hold; precision: of every simulation;
 * quantum >= 1: steps per tick at most; max_active >= 1: simultaneously running simulations. */
int adi_server_create(adi_server *out, size_t hbm_budget, int precision, int quantum, int max_active);
/* Queues a request (arrays are copied); *ticket identifies it.  ADI_EINVAL for an invalid
 * request, ADI_ENOMEM if it could never fit the budget. */
int adi_server_submit(adi_server s, const adi_request *req, int *ticket);
/* One scheduling round (admit, advance, retire, admit); returns after the device work of the
 * round has finished.  *n_running, *n_pending (may be NULL) report the state afterwards. */
int adi_server_tick(adi_server s, int *n_running, int *n_pending);
/* State of a request (ADI_REQ_*) and its times in seconds since the server was created:
 * submission, admission and completion (negative while not reached).  Any pointer may be
 * NULL. */
int adi_server_status(adi_server s, int ticket, int *state, double *t_submit, double *t_start,
                      double *t_done);
/* Fields of a finished request (shapes as adi_read_fields; NULL skips a field). */
int adi_server_result(adi_server s, int ticket, double *u, double *v, double *w);
/* Device bytes currently reserved by running simulations. */
size_t adi_server_used_bytes(adi_server s);
int adi_server_destroy(adi_server s);

/*
 * adi_step_static -- one time step (stage 1 then stage 2, no source term) of a small
 * simulation whose fields the caller keeps in device memory, computed without allocating
 * anything.  The paper has no counterpart: this is a library service for callers that must
 * not allocate, e.g. a process whose device memory is wholly pre-reserved by its own pool,
 * or a latency-bound loop that cannot afford the device-wide synchronisation a cudaFree
 * implies.  The result equals adi_create + adi_step(1) + adi_read_fields with
 * ADI_SOLVER_LINE on the same inputs.
 *   method, nx, ny, h, dt, precision   as for adi_create; nx, ny <= ADI_STATIC_MAX_CELLS.
 *   c, u, v, w            device arrays of the precision's type (float or double), row-major
 *                         with the shapes of adi_create (c at U's points, every value > 0,
 *                         not checked); u's outer rows/columns are the Dirichlet data.  Each
 *                         of the seven pointers must be device or managed memory of the
 *                         current device (checked with cudaPointerGetAttributes: host memory
 *                         gives ADI_EINVAL before any work is enqueued); their sizes are
 *                         not checked.
 *   u_out, v_out, w_out   device arrays with the same shapes, each distinct from every
 *                         input and from each other; they receive the fields one step later.
 *   cuda_stream           the work runs on this stream (NULL = legacy default); the call
 *                         returns after it has finished.
 * Every temporary (line descriptors, tables, carried state, per-line solver scratch) lives in
 * one fixed-size array of device memory inside libadi (4 MiB, held by every device that loads
 * the library until the process exits).  The first call on a device looks up that array's
 * address with the device current and keeps it; make that first call before any stream
 * capture begins.  A cudaDeviceReset, or a driver context other than the device's primary
 * one, invalidates the kept address: use the entry point only in processes that keep the
 * primary context.  The call is synchronous: it returns once the step has finished on the
 * stream.  Calls that overlap in time (several host threads, or several streams of one
 * device) share the array and race: serialise them.
 * Errors: ADI_EINVAL (bad method/precision, sizes below ADI_MIN_CELLS, h or dt not > 0,
 * a NULL, aliased, host or other-device pointer); ADI_ENOMEM when nx or ny exceeds
 * ADI_STATIC_MAX_CELLS (the
 * array's capacity); ADI_ESINGULAR, ADI_ECUDA, ADI_ENOTSUP as elsewhere.
 */
#define ADI_STATIC_MAX_CELLS 128
int adi_step_static(int method, int nx, int ny, double h, double dt, int precision,
                    const void *c, const void *u, const void *v, const void *w,
                    void *u_out, void *v_out, void *w_out, void *cuda_stream);

/*
 * adi_batch_submit -- runs simulations with their own step counts as one asynchronous batch
 * and returns at once with a ticket.  Each member advances by the Peaceman-Rachford steps of
 * Eqs. 6-7 exactly as adi_step would; the paper notes that the line systems of one stage are
 * independent of each other (Sec. 2.1, after Alg. 1), which is what lets one launch serve
 * the lines of every member.  Every member with steps left advances together (one
 * persistent, graph-launched plan per phase over all their lines); a member whose count is
 * reached leaves and the others go on.  Until adi_batch_poll reports the ticket done, the
 * members are busy: adi_step, adi_set_solver, adi_set_source, adi_autotune, adi_batch_create,
 * adi_batch_submit and adi_destroy return ADI_EBUSY; adi_read_fields and adi_set_fields wait
 * for the ticket's work first.
 *   sims[n], nsteps[n]   distinct handles of one precision, none in a batch or ticket;
 *                        nsteps[k] >= 0.
 * Errors: ADI_EINVAL, ADI_EBUSY, ADI_ENOMEM, ADI_ECUDA (nothing is run then).
 *
 * adi_batch_poll -- *done = 1 once every step of the ticket has finished (the members are
 * released and the ticket retired), else 0; never blocks.  The poll that retires a ticket
 * returns the run's error, if any (also made sticky on its members).  ADI_EINVAL for an
 * unknown or retired ticket.
 */
int adi_batch_submit(const adi_handle *sims, const int *nsteps, int n, int *ticket);
int adi_batch_poll(int ticket, int *done);

/*
 * adi_fixed_point -- the paper's own stage solver, for comparison with the exact line solves
 * of adi_step: nsteps Peaceman-Rachford steps (Eqs. 6-7) from time t0 in which each stage's
 * coupled line systems (Eq. 8 / Eq. 10) are solved by the fixed-point iteration of Eq. 9
 * (Algorithms 3-4): u_{k+1} = a - alpha (Dv v_k), v_{k+1} = v^m - beta (Du u_{k+1}), from
 * (u_0, v_0) = (u^m, v^m) for the x-lines and (u*, w^m) for the y-lines, until the sum of the
 * Frobenius norms of the two updates over the whole grid is at most eps or kmax sweeps have
 * run.  The test runs on the device (no host round trip between sweeps).
 *   method, nx, ny, h, dt, c_field, precision   as for adi_create.
 *   u, v, w       host arrays (shapes of adi_create), read as the fields at t0 and overwritten
 *                 with the fields at t0 + nsteps dt.
 *   source        NULL, or 5 values (is, js, amp, f0, tdelay): a Ricker point source at U's
 *                 point (is, js) as in adi_set_source.
 *   kmax >= 1, eps >= 0   sweep limit and stopping threshold per stage.
 *   sweeps        (may be NULL) receives the sweeps run over all stages of the call.
 *   device_ms     (may be NULL) receives the device time of the steps (CUDA events; the
 *                 host <-> device copies of the fields are outside it).
 * Device memory (about 14 fields) is allocated for the call and freed before it returns.
 * Errors: ADI_EINVAL (arguments), ADI_ENOMEM, ADI_ECUDA, ADI_ENOTSUP (no device).
 */
int adi_fixed_point(int method, int nx, int ny, double h, double dt, const double *c_field,
                    double *u, double *v, double *w, int nsteps, double t0, const double *source,
                    int kmax, double eps, int precision, long long *sweeps, double *device_ms);

/*
 * adi_fma_peak -- measured fused multiply-add throughput of the current device in FP64 or FP32
 * (flop/s, counting an FMA as two), the denominator of the ALU roofline of the line solvers in
 * that precision.  The paper has no counterpart: a measurement service.  A grid of 8 CTAs per
 * SM, each thread 16 independent FMA chains; the best of three timed launches after a warm-up
 * one, CUDA events on a stream of its own.  Allocates a small output buffer for the call.
 * Changes no setting of the GPU.  Errors: ADI_EINVAL, ADI_ECUDA, ADI_ENOTSUP.
 */
int adi_fma_peak(int precision, double *flops_per_s);

/*
 * adi_selftest_wait_timeout -- runs the failure path of the kernels' bounded waits on
 * purpose: one GPU thread waits on an mbarrier that nothing arrives at, polling at most
 * `polls` times (1 .. 2^22; the line kernels use 2^22), then gives up as a line kernel does
 * when its staged inputs never land.  *gave_up = 1 when the wait ran out (the expected
 * result), 0 if it completed; *cycles (may be NULL) the SM clock cycles it took.  The kernel
 * always ends; nothing else waits on it.  Errors: ADI_EINVAL, ADI_ECUDA, ADI_ENOTSUP.
 */
int adi_selftest_wait_timeout(int polls, int *gave_up, long long *cycles);

#ifdef __cplusplus
}
#endif
#endif /* ADI_H */
