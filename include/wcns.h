/*
 * wcns.h -- C ABI of the GB300 TCNS library (libwcns.so).
 *
 * The library evaluates the semi-discrete right-hand side of the
 * fifth-order weighted compact nonlinear scheme with TENO-style stencil
 * selection ("TCNS") of Zhang, Zhang & Xu (arXiv 1810.07806) for the
 * compressible Euler equations of an ideal gas, dimension by dimension, and
 * advances it with third-order SSP Runge-Kutta under a CFL rule.
 *
 * Conventions shared by every call:
 *  - Every call returns a wcns_status and never aborts the process.  On
 *    failure wcns_last_error() gives a message (thread-local).
 *  - State arrays are caller-owned DEVICE pointers in structure-of-arrays
 *    layout U[var][z][y][x] (x fastest, no padding), with the conserved
 *    variables (rho, rho*u_1 .. rho*u_ndim, E), nv = ndim + 2.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is stream-ordered; calls do not synchronise
 *    unless they return a host value (stated per call).
 *  - Asynchronous CUDA errors surface as WCNS_ERR_CUDA on a later call.
 *  - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef WCNS_H
#define WCNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WCNS_OK = 0,
    WCNS_ERR_INVALID = 1,     /* bad argument or unsupported combination        */
    WCNS_ERR_NOMEM = 2,       /* device or host allocation failed / over budget */
    WCNS_ERR_NONPHYSICAL = 3, /* rho <= 0 or p <= 0 met (first-order fallback)  */
    WCNS_ERR_TIMEOUT = 4,     /* a bounded wait gave up                          */
    WCNS_ERR_BUSY = 5,        /* no free slot / queue full                       */
    WCNS_ERR_CUDA = 6         /* a CUDA runtime call failed                      */
} wcns_status;

/* Boundary kinds: zero-gradient copy of the boundary node (Sec. 3.4),
 * periodic wrap, reflecting wall, fixed (Dirichlet) state; the last two are
 * the Rayleigh-Taylor boundaries of Sec. 3.9. */
enum { WCNS_BC_TRANSMISSIVE = 0, WCNS_BC_PERIODIC = 1, WCNS_BC_REFLECTING = 2, WCNS_BC_FIXED = 3 };
/* Midpoint flux (Sec. 1 names all three): Roe flux-difference splitting,
 * van Leer flux-vector splitting, Liou-Steffen AUSM. */
enum { WCNS_FLUX_ROE = 0, WCNS_FLUX_VANLEER = 1, WCNS_FLUX_AUSM = 2 };
/* Midpoint-to-node difference: Eq. 3 (MD, a = 75/64, -25/384, 3/640), Eq. 4
 * (HWCNS, b = 64/45, -2/9, 1/180 on midpoints i+-1/2 and the physical fluxes
 * of nodes i+-1, i+-2) or Eq. 5 (MND, c = 3/2, -3/10, 1/30 on midpoints
 * i+-1/2, i+-3/2 and nodes i+-1); all sixth order. */
enum { WCNS_DIFF_MD6 = 0, WCNS_DIFF_HWCNS = 1, WCNS_DIFF_MND = 2 };
/* Interpolation weights: TENO selection (Eq. 16-19, the paper's scheme),
 * WCNS-JS (Eq. 14), linear (the optimal weights d_k of Eq. 13, i.e. Eq. 7)
 * and WCNS-Z (the weights of Borges et al. that the paper compares with,
 * alpha_k = d_k (1 + tau_5 / (beta_k + eps)) with the tau_5 of Eq. 16).
 * All four run in FP64 and FP32 everywhere (single grids, batches, the
 * server); in FP32 the comparison weights are rescaled like the TENO
 * indicators and use tile configuration 0. */
enum { WCNS_W_TENO = 0, WCNS_W_JS = 1, WCNS_W_LINEAR = 2, WCNS_W_Z = 3 };
enum { WCNS_FP64 = 0, WCNS_FP32 = 1 };

/* Uniform grid.  Axis a has n[a] nodes on [lo[a], hi[a]].  An axis whose
 * two sides are transmissive places nodes on both end points,
 * h = (hi - lo)/(n - 1); any other axis has h = (hi - lo)/n: a periodic axis
 * has n unique nodes, and an axis with a reflecting wall or a fixed state
 * places its nodes at cell centres lo + (i + 1/2) h, the walls on the outer
 * faces.  bc[a][0] / bc[a][1] are the low / high side; periodic must be set
 * on both sides.  A reflecting side mirrors the nodes about the wall face
 * with the normal momentum negated (needs n[a] >= 5); a fixed side fills
 * its 5 ghost nodes with bc_state[a][side] (conserved variables rho,
 * rho u_1 .. rho u_ndim, E; rho > 0, p > 0).  gravity is a body force per
 * unit mass: the RHS gains (0, rho g, rho u.g) (Sec. 3.9: g = (0, 1)).
 * Axes >= ndim are ignored.  n[a] >= 2 (transmissive) or >= 1 (periodic).
 * Single grids, batches and the server take every boundary kind and the
 * body force; the allocation-free step takes transmissive and periodic
 * sides without a body force. */
typedef struct {
    int ndim;
    int n[3];
    double lo[3], hi[3];
    int bc[3][2];
    double bc_state[3][2][5];
    double gravity[3];
} wcns_grid;

/* Scheme parameters (Sec. 2 of the paper).  wcns_default_params() fills the
 * paper's values: TENO weights with C = 1, eps = 1e-40, q = 6 (Eq. 16) and
 * C_T = 1e-5 (Sec. 2.3), characteristic interpolation (Sec. 3), sixth-order
 * MD differencing (Eq. 3), Roe flux, FP64, CFL 0.5. */
typedef struct {
    int flux;            /* WCNS_FLUX_ROE | WCNS_FLUX_VANLEER | WCNS_FLUX_AUSM */
    int diff;            /* WCNS_DIFF_MD6 | WCNS_DIFF_HWCNS | WCNS_DIFF_MND    */
    int weights;         /* WCNS_W_TENO | _JS | _LINEAR | _Z                  */
    double C, eps, CT;   /* Eq. 16 and Eq. 18 constants (eps also serves Z)   */
    int q;               /* Eq. 16 power, 1..16                               */
    int characteristic;  /* must be 1: interpolate characteristic variables   */
    int precision;       /* WCNS_FP64 | WCNS_FP32                             */
    double cfl;          /* CFL number of the time-step rule                  */
    int entropy_fix;     /* must be 0 (the paper uses none)                   */
    double eps_js;       /* epsilon of Eq. 14 (WCNS-JS), default 1e-6         */
} wcns_scheme_params;

typedef struct wcns_handle wcns_handle;

void wcns_default_params(wcns_scheme_params* p);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* wcns_last_error(void);

/* Library version string. */
const char* wcns_version(void);

/* Create a solver for one grid.  Allocates the handle's device scratch on
 * the current CUDA device (two state-sized arrays plus small reduction
 * buffers; FP32 mode adds three single-precision state-sized arrays).
 * gamma > 1.  The handle owns its scratch; free it with wcns_destroy. */
wcns_status wcns_create(const wcns_grid* grid, double gamma, const wcns_scheme_params* params,
                        wcns_handle** out);
wcns_status wcns_destroy(wcns_handle* h);

/* Bytes of device scratch the handle holds (for admission budgets). */
size_t wcns_handle_bytes(const wcns_handle* h);

/* Semi-discrete RHS, Eq. 2: L = -sum_d dF_d/dx_d with each derivative from
 * Eq. 3 over midpoint fluxes of the TCNS characteristic interpolation
 * (Eq. 8-19) and the chosen flux.  U and L are device arrays in the handle's
 * precision (double for WCNS_FP64, float for WCNS_FP32), nv * N elements.
 * flags (nullable, device, wcns_flags_bytes bytes) receives per direction d,
 * characteristic field k, grid line and face j + 1/2 (j = -3 .. n_d + 1)
 * one byte: bits 0-2 = delta_1..3 of the left-biased value, bits 3-5 = the
 * same for the right-biased value; layout [d][k][line][j + 3], where lines
 * of direction d enumerate the other axes in (z, y, x) order, x fastest.
 * Faces whose interpolated state had rho <= 0 or p <= 0 use first-order
 * values and are counted (wcns_fallback_count).  Stream-ordered: the call
 * does not wait for the device, so it cannot report such faces itself and
 * returns WCNS_OK; read the count with wcns_fallback_count. */
wcns_status wcns_rhs(wcns_handle* h, const void* U, void* L, uint8_t* flags, void* stream);

/* Size in bytes of the flags array of wcns_rhs. */
size_t wcns_flags_bytes(const wcns_handle* h);

/* One SSP-RK3 step (Shu-Osher form) in place on the FP64 device state U
 * (double, nv * N).  In FP32 mode the right-hand sides run in single
 * precision and each stage value is the FP64 base state U^n plus an FP32
 * increment (D1 = dt L, D2 = (D1 + dt L)/4, U^(n+1) = U^n + 2/3 (D2 + dt L),
 * the last sum accumulated in FP64).  dt > 0 uses that step; dt <= 0
 * computes dt = cfl / max_i sum_d (|u_d| + c)/h_d on the device (FP64
 * maximum).  If dt_used is non-NULL the call copies the step to the host,
 * synchronises the stream and returns WCNS_ERR_NONPHYSICAL (with the step
 * completed) when faces fell back to first-order values during it;
 * otherwise nothing is synchronised and the status does not report such
 * faces (see wcns_fallback_count).  With dt <= 0 (and profiling
 * off) the step's launches are captured once per state pointer U as a CUDA
 * graph on an internal stream and replayed on `stream` afterwards; passing
 * another U, or changing the tile configuration, captures again. */
wcns_status wcns_step_rk3(wcns_handle* h, void* U, double dt, double* dt_used, void* stream);

/* nsteps SSP-RK3 steps with the CFL rule (as wcns_step_rk3 with dt <= 0) on
 * a HOST FP64 state U (nv * N doubles, SoA, updated in place; pinned memory
 * copies fastest, pageable memory works).  The call copies U to a device
 * state the handle owns (allocated on the first call, freed by
 * wcns_destroy; WCNS_ERR_NOMEM if that fails), steps it, copies it back and
 * synchronises the stream.  Returns WCNS_ERR_NONPHYSICAL, with the steps
 * done and U written, when faces fell back to first-order values. */
wcns_status wcns_step_rk3_host(wcns_handle* h, double* U, int nsteps, void* stream);

/* Advance U (FP64 device state) from t = 0 to t_end with CFL steps, the
 * last one clipped to land on t_end, or until max_steps.  The time and step
 * size stay on the device; the host loop checks completion every `check`
 * steps (one small device-to-host read).  Writes the reached time and the
 * number of steps.  Synchronises the stream before returning.  Returns
 * WCNS_ERR_NONPHYSICAL, with the run completed and the outputs written, when
 * faces had rho <= 0 or p <= 0 and used first-order values during the call
 * (wcns_fallback_count gives the number).  Each step
 * replays a captured CUDA graph (per state pointer, as for wcns_step_rk3). */
wcns_status wcns_advance(wcns_handle* h, void* U, double t_end, int max_steps, int check,
                         double* t_out, int* steps_out, void* stream);

/* FP64 conserved totals sum_i U_v,i * prod_d h_d for each variable (host
 * array of nv doubles), from an FP64 device state.  Deterministic order.
 * Synchronises the stream. */
wcns_status wcns_conserved(wcns_handle* h, const void* U, double* out, void* stream);

/* The CFL time step of an FP64 device state (host result; synchronises). */
wcns_status wcns_cfl_dt(wcns_handle* h, const void* U, double* dt, void* stream);

/* Number of first-order fallback faces since creation or the last reset
 * (synchronises the stream). */
wcns_status wcns_fallback_count(wcns_handle* h, long long* count, int reset, void* stream);

/* Tile-shape autotuner (no counterpart in the paper).  For FP32 handles of
 * 2D/3D grids, times every compiled pencil-tile configuration of each
 * direction's sweep (lines per tile x nodes per line; the halo depth is fixed
 * at 5 by the stencil) on the FP64 device state U, and keeps the fastest for
 * this handle.  chosen (nullable) receives the configuration per direction
 * (0 = default).  FP64 and 1D handles, and FP32 handles with the JS, linear
 * or Z weights (one compiled configuration), keep configuration 0.  Results
 * do not depend on the configuration.  Synchronises the stream. */
wcns_status wcns_autotune(wcns_handle* h, const void* U, int* chosen, void* stream);

/* Set (set non-NULL: one configuration 0..2 per direction; ignored by FP64
 * and 1D handles) and/or read (get non-NULL, 3 ints) the handle's tile
 * configurations.  No device work. */
wcns_status wcns_tile_config(wcns_handle* h, const int* set, int* get);

/* Kernel timing for measurement (no counterpart in the paper).  While
 * enabled, the sweep launches of each right-hand side of this handle (one
 * per direction) are bracketed by a pair of CUDA events recorded on the
 * launch stream: in FP32 the sweeps after the first of a right-hand side
 * start as programmatic dependents of the previous one and overlap its last
 * wave, so the right-hand side, not the single sweep, is what events can
 * time.  wcns_profile_read synchronises those events and returns the summed
 * duration (ms) and the number of sweep launches they cover since the last
 * read (so the ratio is the average sweep launch), then clears them.
 * Enabling costs two event records per right-hand side and disables the
 * CUDA-graph form of steps; disabled by default. */
wcns_status wcns_profile(wcns_handle* h, int enable);
wcns_status wcns_profile_read(wcns_handle* h, double* sweep_ms, long long* sweep_launches);

/* One FP64 SSP-RK3 step that allocates no device memory.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, for example
 * an application whose device memory is all reserved up front by another
 * allocator, or a time-critical loop that must make no allocation calls.
 * It needs no handle: grid, gamma and params are as for wcns_create
 * (params->precision must be WCNS_FP64), U is the caller's FP64 device
 * state (nv * N doubles, updated in place) and dt / dt_used are as for
 * wcns_step_rk3, with the same results.  The stage state and right-hand
 * side live in one library-owned static device buffer of
 * WCNS_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  The buffer holds a 512-byte header and
 * two state-sized parts, each rounded up to 256 bytes, so a grid of N nodes
 * fits when 512 + 2 * round_up(8 * nv * N, 256) <= WCNS_NOALLOC_SCRATCH_BYTES:
 * at most 349,514 nodes in 1D, 262,136 in 2D and 209,708 in 3D.  Larger
 * grids are rejected with WCNS_ERR_INVALID before any device work (the
 * node count is checked axis by axis, so no product can overflow).
 * The first call on each device performs a one-time set-up there (the
 * buffer's device address, kernel attributes, a constant table); make that
 * first call before any stream capture.  All calls on one device share
 * its buffer, which keeps the last call's contents: calls on the same
 * device whose GPU work overlaps (different streams or host threads) race
 * on it and must be serialised by the caller. */
#define WCNS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
wcns_status wcns_step_rk3_noalloc(const wcns_grid* grid, double gamma,
                                  const wcns_scheme_params* params, void* U, double dt,
                                  double* dt_used, void* stream);

/* ---------------------------------------------------------------------
 * Batches (no counterpart in the paper; the method is applied unchanged to
 * every instance).  A batch advances many independent grids of one
 * dimension, precision and scheme together: each instance has its own node
 * counts, boundary rules (every kind, with the fixed states and the body
 * force), CFL time step, end time and, in FP32, reference state.  One
 * launch per sweep direction covers the tiles of all instances; one SSP-RK3
 * step of the whole batch is captured as a CUDA graph and replayed.  An
 * instance gives the same result in a batch as alone, bit for bit, in FP64
 * and in FP32 (the batched and single-grid kernels round identically).
 * --------------------------------------------------------------------- */
typedef struct wcns_batch wcns_batch;

/* Create a batch for up to max_instances instances holding max_nodes nodes
 * in total (device arenas are allocated here: state, stage and RHS arrays,
 * plus per-instance clocks).  params as for wcns_create. */
wcns_status wcns_batch_create(int ndim, double gamma, const wcns_scheme_params* params,
                              long long max_nodes, int max_instances, wcns_batch** out);
wcns_status wcns_batch_destroy(wcns_batch* b);
size_t wcns_batch_bytes(const wcns_batch* b);

/* Add an instance with FP64 initial state U0 (nv * N doubles, SoA; a host
 * pointer, or a device pointer when u0_on_device) to be advanced from t = 0
 * to t_end.  Returns its slot.  WCNS_ERR_BUSY: no free slot; WCNS_ERR_NOMEM:
 * not enough free arena.  The copy is queued on `stream`; it joins at the
 * next wcns_batch_step. */
wcns_status wcns_batch_add(wcns_batch* b, const wcns_grid* grid, const double* U0, int u0_on_device,
                           double t_end, int* slot, void* stream);

/* Free an instance's slot and arena range (after its result was read). */
wcns_status wcns_batch_remove(wcns_batch* b, int slot);

/* Advance every instance by nsteps RK3 steps (finished instances do no
 * work).  If active is non-NULL, synchronises and returns how many
 * instances advanced in the last step (0: all have reached t_end). */
wcns_status wcns_batch_step(wcns_batch* b, int nsteps, int* active, void* stream);

/* Sweep launch form of the batch (no counterpart in the paper): 0 = one CTA
 * per tile of the tile table (default), 1 = persistent: as many CTAs as are
 * resident on the device, each taking tiles from a device counter until the
 * table is done (no CTA waits on another).  Results do not depend on the
 * form.  No device work; the next step captures its graph again. */
wcns_status wcns_batch_launch_mode(wcns_batch* b, int mode);

/* Autotuner of the batch's launch form (no counterpart in the paper): times
 * `steps` graph-replayed RK3 steps of the current instances in each form,
 * keeps the faster, and restores the batch's states, clocks and counters, so
 * the results are unchanged.  mode_out (nullable) receives the form kept,
 * ms_per_step (nullable, 2 doubles) the time per step of each form (0 when
 * the batch is empty).  Allocates a temporary copy of the state arena
 * (WCNS_ERR_NOMEM if it does not fit).  Synchronises the stream. */
wcns_status wcns_batch_autotune(wcns_batch* b, int steps, int* mode_out, double* ms_per_step, void* stream);

/* Step until every instance has finished or max_steps, checking every
 * `check` steps.  Returns the steps taken.  Synchronises. */
wcns_status wcns_batch_run(wcns_batch* b, int max_steps, int check, int* steps, void* stream);

/* Copy an instance's FP64 state (host pointer, or device when out_on_device;
 * nullable) and return its time and step count.  Synchronises the stream.
 * Returns WCNS_ERR_NONPHYSICAL, with every output written, when faces of
 * this instance had rho <= 0 or p <= 0 and used first-order values since
 * it was added (each instance has its own counter). */
wcns_status wcns_batch_read(wcns_batch* b, int slot, double* U_out, int out_on_device, double* t,
                            int* steps, void* stream);

/* ---------------------------------------------------------------------
 * Serving (no counterpart in the paper).  A server accepts solve requests
 * at any time and runs them with continuous batching: a worker thread
 * admits queued requests (in arrival order) into resident batches, one per
 * scheme class, as the HBM budget, a slot and arena space allow; everything
 * admitted advances together, a fixed number of RK3 steps per tick;
 * requests join and leave at step boundaries; finished states are copied
 * to the host and returned by wcns_serve_poll.  A result equals the same
 * problem solved alone (bit for bit, either precision).  The server uses the
 * CUDA device that is current when it is created.
 * --------------------------------------------------------------------- */
typedef struct wcns_server wcns_server;

typedef struct {
    size_t hbm_budget_bytes;      /* device memory the server may reserve      */
    int max_instances_per_class;  /* slots of each class's batch               */
    long long max_nodes_per_class;/* arena cap per class (0: budget share)     */
    int steps_per_tick;           /* RK3 steps of the most expensive class per
                                     tick (admission and retirement happen
                                     between ticks); cheaper classes take as
                                     many more steps as fit in the same GPU
                                     time, at most 64 times as many           */
} wcns_server_config;

typedef struct {
    wcns_grid grid;
    double gamma;
    wcns_scheme_params params;    /* precision selects the FP32 or FP64 path   */
    const double* U0;             /* host FP64 initial state, copied on submit */
    double t_end;
    uint64_t tag;                 /* returned unchanged in the result          */
} wcns_request;

typedef struct {
    uint64_t ticket, tag;
    wcns_status status;           /* WCNS_OK; WCNS_ERR_NONPHYSICAL when faces of
                                     this request fell back to first-order values
                                     (the state is still returned); otherwise
                                     why the request failed                    */
    int ndim, n[3], precision;
    double t;                     /* time reached (t_end)                      */
    int steps;                    /* RK3 steps taken                           */
    double* U;                    /* host FP64 final state, owned by the result */
    double t_submit, t_admit, t_done;   /* seconds since server creation       */
} wcns_result;

typedef struct {
    int queued, max_queue, max_running;
    long long admitted, completed, ticks, steps;
    size_t bytes_reserved;
} wcns_server_stats_t;

void wcns_server_default_config(wcns_server_config* cfg);
wcns_status wcns_server_create(const wcns_server_config* cfg, wcns_server** out);
/* Stops the worker; requests still queued complete with WCNS_ERR_BUSY. */
wcns_status wcns_server_destroy(wcns_server* sv);

/* Queue a request (thread-safe; copies U0).  Returns a ticket. */
wcns_status wcns_batch_submit(wcns_server* sv, const wcns_request* req, uint64_t* ticket);

/* Up to `max` finished results, waiting up to timeout_us for the first
 * (0: no wait).  WCNS_ERR_TIMEOUT if none arrived in time.  Each result's U
 * must be released with wcns_result_free. */
wcns_status wcns_serve_poll(wcns_server* sv, wcns_result* out, int max, int* n_out, int timeout_us);
void wcns_result_free(wcns_result* r);
wcns_status wcns_server_stats(wcns_server* sv, wcns_server_stats_t* stats);

/* ---------------------------------------------------------------------
 * Scalar conservation laws u_t + f(u)_x = 0 on periodic 1D grids, the
 * paper's accuracy tests (Sec. 3.2: linear advection, f = u; Sec. 3.3:
 * inviscid Burgers, f = u^2 / 2).  The midpoint flux is Eq. 6 with the
 * approximate eigenvalue a = 1 (advection) or a = (u_L + u_R) / 2
 * (Burgers); u_L and u_R come from the node-to-midpoint interpolation of
 * Sec. 2.2 with the weights params->weights selects (no characteristic
 * projection: there is one field); the derivative is Eq. 3, 4 or 5 as
 * params->diff selects (node fluxes f(u_i)).  params->flux is not used.
 * FP64 only.
 *
 * `count` independent lines of n unique nodes each (periodic: node n is
 * node 0; h is the node spacing) sit in device memory at u + i * ld,
 * i = 0 .. count-1, ld >= n doubles.  Each line is solved by one
 * thread-block cluster that keeps it resident in distributed shared memory
 * for the whole call.  1 <= n <= wcns_scalar_max_nodes(); count >= 1.
 * Stream-ordered; no allocation; no host synchronisation.
 * --------------------------------------------------------------------- */
enum { WCNS_SCALAR_ADVECTION = 0, WCNS_SCALAR_BURGERS = 1 };

/* Largest n the scalar solver accepts on the current device. */
int wcns_scalar_max_nodes(void);

/* L = -f'(u) by Eq. 3 for every line (L has the same layout as u). */
wcns_status wcns_scalar_rhs(int kind, const wcns_scheme_params* params, int n, double h, int count,
                            const double* u, long long ld, double* L, void* stream);

/* nsteps SSP-RK3 steps of equal size dt = t_end / nsteps, in place, in one
 * kernel launch (the lines stay on chip between steps). */
wcns_status wcns_scalar_run(int kind, const wcns_scheme_params* params, int n, double h,
                            double t_end, int nsteps, int count, double* u, long long ld,
                            void* stream);

/* Arithmetic-throughput probe (a measurement utility, no counterpart in the
 * paper): runs independent fused multiply-add chains on every SM of the
 * current device and writes the rate reached in TFLOP/s (an FMA counts 2
 * flops).  kind 0: FP32 fmaf; 1: packed FP32 (__ffma2_rn, two FMAs per
 * instruction); 2: FP64 fma.  Allocates a small device buffer; synchronises
 * the stream. */
wcns_status wcns_alu_probe(int kind, double* tflops, void* stream);

/* Number of kernel launches one wcns_step_rk3 call issues (for accounting). */
int wcns_launches_per_step(const wcns_handle* h, int cfl_step);

#ifdef __cplusplus
}
#endif
#endif /* WCNS_H */
