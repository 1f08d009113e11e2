/*
 * dgx.h -- C ABI of the GB300 (sm_103a) modal Discontinuous Galerkin hot path of
 * Cernetic, Springel, Guillet & Pakmor, "High-order Discontinuous Galerkin
 * hydrodynamics with sub-cell shock capturing on GPUs" (arXiv 2208.11131).
 *
 * One handle = one simulation on one GPU: a Cartesian grid of equal cells
 * (Sec. 2.2), a tensor-product scaled-Legendre basis of degree n per axis
 * (Sec. 2.3), n+1 Gauss points per axis (Sec. 2.4), the conserved fields
 * (rho, rho v, e) of Eq. euler plus, when artificial viscosity is on, the
 * viscosity field alpha of Sec. 4.1 as one more expanded field.
 *
 * State layout (host and device, all entry points): float64
 *   w[field][cell][mode],  cell = ix + Nx*(iy + Ny*iz),
 *   mode l = lx + (n+1)*(ly + (n+1)*lz) (tensor basis; with the total-degree
 *   basis the same order with the modes lx + ly + lz > n left out),
 *   fields (rho, rho vx, rho vy, [rho vz], e, [rho c], [alpha]) -- rho c with the tracer on.
 * w[f][K][0] is the cell mean (basis normalised so that (1/|K|) int phi_l phi_m = delta).
 *
 * Ownership: the library owns every device buffer of a handle (allocated in
 * dg_create / dg_set_params, freed in dg_destroy).  Host and device pointers
 * passed in are borrowed for the duration of the call only.
 *
 * Streams: all work of a handle is issued on its stream (default: the legacy
 * default stream; see dg_set_stream).  Entry points that return data to the
 * host (dg_get_state, dg_rhs, dg_max_dt, dg_conserved_sums, dg_get_aux,
 * dg_sync) synchronise that stream; dg_step and dg_steps only enqueue work.
 *
 * Errors: every int-returning call returns DG_OK (0) or one of the codes
 * below; the message of the last failure of a handle is in dg_last_error().
 * Device-side problems (a non-positive density or pressure at a quadrature
 * point, a non-finite time step) set a status word on the device; it is read
 * and cleared by dg_sync / dg_get_state and reported as DG_ENONPHYS.
 * Nothing in the library traps or asserts on the device.
 */
#ifndef DGX_H
#define DGX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_handle dg_t;

enum {
    DG_OK = 0,
    DG_EINVAL = 1,       /* bad argument                                    */
    DG_ENOMEM = 2,       /* device allocation failed                         */
    DG_ECUDA = 3,        /* a CUDA runtime call failed                       */
    DG_ENONPHYS = 4,     /* rho <= 0 or p <= 0 at a quadrature point (Sec. 4.2) */
    DG_ETIMEOUT = 5,     /* reserved: no kernel of this build waits on the
                            device (no spins, no cross-CTA flags), so no
                            call returns it                                  */
    DG_EUNSUPPORTED = 6  /* valid request this build does not implement      */
};

enum { DG_BC_PERIODIC = 0, DG_BC_OUTFLOW = 1 };
enum { DG_FP64 = 0, DG_FP32_BULK = 1 };
enum { DG_BASIS_TENSOR = 0, DG_BASIS_TOTAL = 1 };

/* Cartesian grid: dim = 2 or 3; n[a] cells along axis a on [lo[a], hi[a]];
 * bc[a] = DG_BC_PERIODIC or DG_BC_OUTFLOW (the ghost trace equals the
 * interior trace; no dissipative flux crosses an outflow boundary). */
typedef struct dg_grid {
    int dim;
    int n[3];
    double lo[3];
    double hi[3];
    int bc[3];
} dg_grid;

/* Run-time parameters.  Defaults (dg_default_params) are the paper's:
 * cfl 0.5 (Sec. 2.5, Eq. timestep), av_scale 1, f_v 2.5, f_tau 0.5, f_w 0.2,
 * s_onset 1e-4 (Sec. 4.1; the threshold applied is s_onset / (n+1)^2).
 *  precision: DG_FP64 (all arithmetic in FP64) or DG_FP32_BULK (quadrature,
 *             flux and contraction arithmetic in FP32; the state u^n, the
 *             Runge-Kutta accumulation u^{n+1} = u^n + delta, the time step
 *             and the conservation sums in FP64).
 *  rk_stages: 0 = the paper's choice (n+1 stages for n+1 <= 3: forward Euler,
 *             SSP-RK2, SSP-RK3; else the 5-stage 4th-order SSP scheme), or
 *             1, 2, 3, 5 explicitly.
 *  av_on:     1 adds the alpha field and artificial viscosity (Sec. 4.1).
 *  positivity_on: 1 applies the positivity limiter of Sec. 4.2 after every
 *             stage (rho_bottom = 1e-6 mean rho, p_bottom = 1e-6 p(mean state),
 *             at most 60 pressure halvings; a cell that still fails, or whose
 *             mean state is non-physical, sets the status word).
 *  forcing_on: 1 adds the turbulence driving of Sec. 7.1: an acceleration s(x)
 *             of Fourier modes 2pi/L <= |k| <= 2 (2pi/L) (one of each +-k
 *             pair: 6 in 2-D, 16 in 3-D), amplitude force_amp |k|^(-5/3) with
 *             |k| in units of 2pi/L, complex vector coefficients that follow
 *             Ornstein-Uhlenbeck processes of correlation time force_ts > 0,
 *             advanced exactly at times j * force_dt (force_dt > 0) from
 *             counter-based SplitMix64 + Box-Muller draws of force_seed, and
 *             projected onto the plane normal to k (solenoidal).  The source
 *             rho s enters the momentum and s.(rho v) the energy, integrated
 *             with the volume Gauss rule.  Each step applies the updates due at
 *             its start time and keeps that field for all of its stages.
 *             Defaults: off, force_amp 0, force_ts 1, force_dt 0.01, seed 0.
 *  tracer_on: 1 adds a passive tracer (Sec. 3.4): the conserved field rho c
 *             right after the energy (before alpha), advected with flux
 *             c rho v and diffused with flux tracer_eta rho grad c through the
 *             recovered gradients of Sec. 3.2; it has no effect on the flow.
 *             Changing it reallocates the state (one more field).  Not
 *             supported in batches.
 *  basis:     DG_BASIS_TENSOR (default): all products Pt_lx Pt_ly Pt_lz with
 *             every l_a <= n, (n+1)^d modes; DG_BASIS_TOTAL: the paper's
 *             truncation l_x + l_y + l_z <= n (Sec. 2.3; (n+1)(n+2)/2 modes in
 *             2-D, (n+1)(n+2)(n+3)/6 in 3-D), in the same order with the other
 *             modes left out.  States passed in and out hold those modes only.
 *             3-D FP32-bulk handles of degree 1 or 3 without a tracer store
 *             only those modes on the device too ((n+1)(n+2)(n+3)/6 instead
 *             of (n+1)^3 values per cell and field; such handles cannot join
 *             a batch); the others keep the tensor layout with the other modes
 *             at zero.  The arithmetic per step is the tensor arithmetic.  The
 *             oscillation sensor's high modes become l_x + l_y + l_z = n.
 *             Changing it reallocates the state.  dg_max_dt_noalloc reads
 *             tensor-layout states only. */
typedef struct dg_params {
    int precision;
    int rk_stages;
    double cfl;
    int av_on;
    double av_scale, f_v, f_tau, f_w, s_onset;
    int positivity_on;
    int forcing_on;
    double force_amp, force_ts, force_dt;
    unsigned long long force_seed;
    int tracer_on;
    double tracer_eta;
    int basis;
} dg_params;

/* Fill p with the defaults listed above (DG_FP64, automatic RK, AV off). */
int dg_default_params(dg_params *p);

/* Create a simulation: grid, polynomial degree n (0..5; the paper's order is
 * p = n+1, Sec. 2.3), adiabatic index gamma > 1 (Eq. 3), kinematic viscosity
 * nu >= 0 and thermal diffusivity kappa >= 0 of the Navier-Stokes flux
 * (Sec. 3.3; both 0 gives the Euler equations).  Uses the current CUDA device.
 * The state is zero until dg_set_state*.  *out receives the handle. */
int dg_create(const dg_grid *grid, int degree, double gamma, double nu, double kappa, dg_t **out);
void dg_destroy(dg_t *h);

/* Change run-time parameters; (re)allocates device buffers when the field
 * count or the precision changes, which resets the state to zero. */
int dg_set_params(dg_t *h, const dg_params *p);
int dg_get_params(const dg_t *h, dg_params *p);

/* Sizes of the state array: fields (d+2, +1 with AV), modes per cell, cells. */
int dg_sizes(const dg_t *h, int *nfields, int *nmodes, long long *ncells);

/* Issue all further work of the handle on `stream` (a cudaStream_t). */
int dg_set_stream(dg_t *h, void *stream);

/* State in/out, layout above.  *_device variants take device pointers
 * (float64, same layout) and copy on the handle's stream without a host sync. */
int dg_set_state(dg_t *h, const double *host_w);
int dg_get_state(dg_t *h, double *host_w);
int dg_set_state_device(dg_t *h, const double *dev_w);
int dg_get_state_device(dg_t *h, double *dev_w);

/* Right-hand side L(w) = dw/dt of Eq. weight_evolution (volume integral,
 * HLLC surface flux, recovered-gradient viscous and artificial-viscosity
 * fluxes of Sec. 3, alpha source of Eq. timedependentviscosity) of the
 * current state, with the per-cell wiggle term as stored (dg_set_aux) and,
 * with forcing on, the driving field of the current forcing state (no update).
 * No time advance.  Output in the state layout, float64. */
int dg_rhs(dg_t *h, double *host_out);
int dg_rhs_device(dg_t *h, double *dev_out);

/* One SSP Runge-Kutta step (Sec. 2.5).  dt > 0: that step size; dt <= 0: the
 * CFL step of Eq. timestep from the state at the start of the step.  With AV
 * on, the oscillation sensor (Eq. discontinuity_sensor2) and its wiggle
 * source are updated at the start of the step.  Enqueues only. */
int dg_step(dg_t *h, double dt);
/* nsteps such steps, replayed from a captured CUDA graph.  Enqueues only. */
int dg_steps(dg_t *h, int nsteps, double dt);

/* One step as dg_step, timed: CUDA events are recorded on the handle's stream
 * around each launch of the step and the call waits for the last one.
 * ms[0] = step prologue (oscillation sensor + CFL speeds), ms[1] = time-step
 * reduction, ms[2 + i] = fused right-hand-side / Runge-Kutta stage i.  With
 * two or more stages and the limiter off, the prologue work is done inside
 * stage 0 (ms[0] = 0, ms[2] includes it) and the reduction runs after it.
 * nms must be at least 2 + the stage count (at most 7).  For profiling and
 * benchmarks; the arithmetic is identical to dg_step. */
int dg_step_timed(dg_t *h, double dt, float *ms, int nms);

/* Wait for the handle's stream and report the device status word. */
int dg_sync(dg_t *h);

/* CFL step of Eq. timestep for the current state (FP64), no time advance.
 * The CFL factor is the handle's dg_params.cfl (set with dg_set_params), so
 * the call takes no cfl argument; dg_max_dt_noalloc, which has no handle,
 * takes it explicitly. */
int dg_max_dt(dg_t *h, double *dt);

/* FP64 totals sum_K |K| w[f][K][0] for the conserved fields (d+2 values). */
int dg_conserved_sums(dg_t *h, double *out);

/* Auxiliary per-cell and scalar data of the time stepper (for checkpoints
 * and tests).  S_prev, wig: one double per cell (previous sensor value and
 * the current wiggle source of Sec. 4.1); scal: {dt of the last step, step
 * count, time}.  Any pointer may be NULL to skip it. */
int dg_get_aux(dg_t *h, double *S_prev, double *wig, double *scal);
int dg_set_aux(dg_t *h, const double *S_prev, const double *wig, const double *scal);

/* Driving (forcing) state, DG_FORCING_STATE doubles: [0] index of the last OU update
 * applied (-1: none yet; the first step draws the stationary state), then for each of the
 * 16 mode slots (6 used in 2-D, in the order: kz outer, ky, kx inner over the integer vectors
 * with 1 <= |k|^2 <= 4 whose first non-zero component is positive) the real and imaginary
 * parts of the OU vector, x y z each (components beyond d are zero).  For checkpoints and
 * for restarting a run bit for bit; a state set with dg_set_forcing takes effect at the next
 * dg_step or dg_rhs.  DG_EINVAL when forcing is off. */
#define DG_FORCING_STATE 97
int dg_get_forcing(dg_t *h, double *host_state);
int dg_set_forcing(dg_t *h, const double *host_state);

/* The CFL time step dt = cfl * h_min / (2 (n+1) (max c_s + max |v|)), the
 * maxima taken over the volume Gauss points of the state -- the same value as
 * dg_max_dt -- for callers that cannot let a library allocate device memory:
 * code that hands all device memory to its own pool at start-up and forbids
 * later allocations, or time-stepping loops that cannot take the device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this
 * is a service of this library.
 *
 * Needs no handle and allocates nothing.  dev_state: device pointer to the
 * FP64 state in the layout above (its first d+2 fields are read; an alpha
 * field may follow).  dev_dt: device pointer to one double that receives the
 * step, or NaN if a Gauss point has rho <= 0 or p <= 0.  grid->bc is unused.
 * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream)
 * without a host synchronisation; the arithmetic is that of dg_max_dt in FP64.
 *
 * Scratch: a 4 MiB file-scope device array (2^18 per-tile slots + a status
 * word) that every GPU which loads the library keeps until the process exits.
 * Grids that need more than 2^18 tiles of the time-step kernel (e.g. more than
 * 4.19 M cells in 3-D at degree 3, 16.7 M cells in 2-D at degree 3) return
 * DG_EUNSUPPORTED.  All calls share that array: calls whose work overlaps on
 * the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  The first call on each device does set-up work
 * on the host: it looks up the array's device address (cudaGetSymbolAddress),
 * and with lazy module loading it is also the call that loads the library's
 * kernels onto that device (the array becomes resident there then) and sets
 * the time-step kernel's shared-memory attribute.  Make that first call on a
 * device before any stream capture on it.  Returns DG_OK, DG_EINVAL,
 * DG_EUNSUPPORTED or DG_ECUDA. */
int dg_max_dt_noalloc(const dg_grid *grid, int degree, double gamma, double cfl, const double *dev_state,
                      double *dev_dt, void *stream);

/* Batched ensembles: many independent simulations advanced together.
 * Members are grouped by (dim, degree, precision, AV, NS, limiter); each group
 * runs one persistent stage kernel per Runge-Kutta stage over the work list of
 * all its members' tiles, with each member's own time step (CFL of its own
 * state, or the fixed dt) computed on the device.  Members with the positivity
 * limiter (Sec. 4.2) form groups of their own: each member's step prologue and
 * limiter launches run on the group's stream around the batched stage launches.
 * Groups run concurrently; dg_batch_step replays two whole steps at a time from
 * one captured CUDA graph.  Members keep their own state and may be read with
 * dg_get_state after dg_batch_sync.  All members must share the device, the
 * stream and the step parity (same number of steps taken so far modulo 2) and
 * have at least two Runge-Kutta stages; driving and tracer members are not
 * available in batches (DG_EUNSUPPORTED).  The batch does not own the members:
 * destroy it before them.  The arithmetic of every member is the same as with
 * dg_step. */
typedef struct dg_batch dg_batch_t;
int dg_batch_create(dg_t *const *sims, int count, dg_batch_t **out);
int dg_batch_step(dg_batch_t *b, int nsteps, double dt); /* enqueues only */
int dg_batch_sync(dg_batch_t *b);                        /* waits; first member error */
const char *dg_batch_last_error(const dg_batch_t *b);
void dg_batch_destroy(dg_batch_t *b);

const char *dg_last_error(const dg_t *h);
const char *dg_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* DGX_H */
