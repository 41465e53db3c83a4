/*
 * lbms.h -- C ABI of the GB300 solver for ternary (H2-H2O-Ar) diffusion in a
 * porous SOFC anode: an advection-diffusion lattice Boltzmann model (one
 * distribution per species, BGK collision, bounce-back on a voxel mask)
 * coupled cell by cell to the Maxwell-Stefan equations through a local
 * relaxation time (Huang, Bao, Jiang, Zhang, arXiv:1809.01600, Section 3).
 *
 * Conventions shared by every entry point
 *  - Every call returns an lbms_status and never aborts; on failure
 *    lbms_last_error(ctx) holds a one-line message for that handle.
 *  - Host arrays passed in are read during the call only (copied); output
 *    arrays are caller-owned host buffers of the stated size.
 *  - Dense fields are indexed [species][z][y][x], x fastest; N = nx*ny*nz.
 *  - Species order is (H2, H2O, Ar) = (1, 2, n) of the paper; the last one is
 *    the reference species n of Eqs. 31-34.
 *  - Units are SI except the current density (A/cm^2, as in Eq. 39's use).
 *  - All device work is issued on options.stream; calls that return host
 *    data synchronise that stream.  A handle is not thread-safe.
 */
#ifndef LBMS_H
#define LBMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbms_ctx lbms_ctx;

typedef enum {
    LBMS_OK = 0,
    LBMS_EINVAL = 1,          /* invalid argument (message says which) */
    LBMS_ENOMEM = 2,          /* device or host allocation failed */
    LBMS_ECUDA = 3,           /* a CUDA call failed (message has the CUDA error) */
    LBMS_ENOTCONVERGED = 4,   /* run_to_residual hit max_steps above tol */
    LBMS_EUNSTABLE = 5,       /* NaN/Inf found in the mole fractions */
    LBMS_EDEPLETED = 6,       /* outlet H2 (or inlet H2O) <= 0: Eq. 43 undefined */
    LBMS_ESTATE = 7           /* call out of order (e.g. step before set_bc) */
} lbms_status;

enum { LBMS_FP64 = 0, LBMS_FP32 = 1, LBMS_FP16 = 2 };
enum { LBMS_COUPLING_MS = 0, LBMS_COUPLING_TAU_ONLY = 1 };
enum { LBMS_INIT_UNIFORM = 0, LBMS_INIT_PROFILE_1D = 1 };
enum { LBMS_OUTLET_FLUX = 0, LBMS_OUTLET_EXTRAPOLATED = 1 };
enum { LBMS_GRAD_CENTRAL = 0, LBMS_GRAD_FORWARD = 1 };

/* Geometry.  dim = 2 uses D2Q9 (Eq. 2, weights Eq. 9); dim = 3 uses D3Q19.
 * solid: N bytes, nonzero = solid voxel (half-way bounce-back, Section 3.3).
 * periodic_x = 0: inlet nodes at x = 0 (Dirichlet, Eq. 36) and reacting
 *   outlet nodes at x = nx-1 (flux of Eq. 39); both columns must be fluid;
 *   grid spacing dx = length_x_m / (nx - 1).
 * periodic_x = 1: closed box periodic in x, dx = length_x_m / nx.
 * y and z are always periodic. */
typedef struct {
    int dim;
    int nx, ny, nz;
    const uint8_t *solid;
    double length_x_m;
    int periodic_x;
} lbms_geometry;

/* Species data (Table 1, Eq. 38): n must be 3. */
typedef struct {
    int n;
    const double *molar_mass;     /* kg/kmol, n entries */
    const double *fuller_volume;  /* Fuller diffusion volume, n entries */
    const int *stoich;            /* nu_i of Eq. 38, n entries */
    int electrons;                /* n of Eqs. 39 and 43 */
} lbms_species;

/* Binary diffusivities.  D_binary_m2s: n*n row-major (diagonal ignored), or
 * NULL for the Fuller correlation of Eq. 40.  pore_diameter_m > 0 adds the
 * Knudsen term of Eq. 42 through Eq. 41; <= 0 leaves it out.  eps_over_tau
 * is the porosity/tortuosity prefactor of Eq. 41 (1.0 for resolved pores). */
typedef struct {
    const double *D_binary_m2s;
    double pore_diameter_m;
    double eps_over_tau;
} lbms_diffusivities;

/* Options; lbms_default_options fills the defaults in brackets.
 *  precision  LBMS_FP64: state and arithmetic in FP64.  LBMS_FP32: FP32
 *             arithmetic, non-equilibrium populations in FP32 and mole
 *             fractions as double-float pairs (two FP32 words), which keeps
 *             steady states free of FP32 stagnation.  LBMS_FP16: as FP32
 *             with the non-equilibrium populations stored in FP16 [FP32]
 *  coupling   LBMS_COUPLING_MS: clamped tau plus drift velocity (exact
 *             Maxwell-Stefan flux); LBMS_COUPLING_TAU_ONLY: tau alone,
 *             Eqs. 28-29 literally [MS]
 *  tau_min, tau_max  clamp of Eq. 25 [1, 5]
 *  dt_s       time step; 0 picks dt = dx^2 / (6 min D_ij,eff) [0]
 *  check_every residual interval K of run_to_residual [100]
 *  extrapolate_every  W > 0: run_to_residual extrapolates the slowest decay
 *             mode every W steps (Aitken: with rho the ratio of successive
 *             W-step changes of X, X += rho / (1 - rho) * (last change) when
 *             two successive ratios agree within 2 % and 0.05 < rho < 0.98).
 *             The fixed point is unchanged; only the approach is shortened.
 *             With W > 0, a case that meets tol is not done yet: a final
 *             extrapolation is taken at its next W-step check (from the
 *             last two W-step changes, or from the snapshots of the current
 *             reduced-rank cycle, see extrapolate_modes), repeated (at most
 *             three times) while the single-mode jump moved X by more than
 *             1e-5 of |X|, and the case is done when it meets tol again
 *             after the last one.  The residual measures
 *             the rate of change, so the error it leaves is largest along
 *             the slowest mode; the final extrapolation removes most of it.
 *             0 = off [0]
 *  extrapolate_modes  how the extrapolation every W steps works: 0 or 1:
 *             the single-mode jump above; M in 2..6: reduced-rank
 *             extrapolation (RRE) over M + 1 snapshots of X taken W steps
 *             apart (the first W / 8 steps after the start or the last jump,
 *             past the fast transient), X = sum_j gamma_j x_j with gamma minimising
 *             || sum_j gamma_j (x_{j+1} - x_j) || subject to sum_j gamma_j = 1
 *             (per case, FP64), which removes up to M - 1 decay modes at once;
 *             a case whose snapshot differences do not shrink is left alone.
 *             Holds (M + 1) x 3 x cells doubles of snapshots [1]
 *  step_variant  0: the autotuner picks the step kernel's tile, thread
 *             mapping (a thread per cell and species, or per cell) and
 *             neighbour lookup by timing; k in 1..10 forces variant k - 1
 *             (for tests).  Variants 0-5 and 6-7 read a table of 32-bit
 *             fluid indices (or 16-bit offsets, 3-5) per cell and link;
 *             8-9 decode the neighbours from per-row fluid bitmasks and a
 *             4-byte coordinate per cell (built when no case is periodic in
 *             x and nx <= 2048, ny <= 1024, nz <= 2048).  An unavailable
 *             variant is an error [0]
 *  init_mode  state a case starts from at its first set_bc:
 *             LBMS_INIT_UNIFORM: the inlet composition everywhere, f = w X_in;
 *             LBMS_INIT_PROFILE_1D: the initial state of Section 4.1, every
 *             column x at the 1-D profile of Eq. 19 integrated from the
 *             inlet with the fluxes held at their outlet values (Eq. 39),
 *             N_i(x) = N_i|A/E, and the handle's D_ij,eff (Eq. 41);
 *             LBMS_EDEPLETED from set_bc if that profile drives a mole
 *             fraction below zero.  Boxes periodic in x start uniform [UNIFORM]
 *  outlet_bc  LBMS_OUTLET_FLUX: the Eq. 39 flux imposed link-wise at x =
 *             nx-1, f_k = f*_opp - (w_opp / W) q (exactly q leaves per node
 *             and step; Ar sees bounce-back); LBMS_OUTLET_EXTRAPOLATED: Eq. 37
 *             read as a wet node, X_out = X^{t-1}(nx-2) + dX with dX from
 *             Eq. 19 over one spacing at the Eq. 39 fluxes, applied with the
 *             Eq. 36 rule (first order: the delivered flux approaches q as
 *             dx -> 0); computed by the per-cell step kernel only, so the
 *             autotuner then picks among the per-cell variants 6-9 [FLUX]
 *  grad_stencil  LBMS_GRAD_CENTRAL: central differences of the previous
 *             step's X on every axis (one-sided at x = 0, nx-1);
 *             LBMS_GRAD_FORWARD: Eq. 35 as printed, the forward difference
 *             along x only [CENTRAL]
 *  stream     cudaStream_t for all device work, NULL = legacy default [NULL]
 *  alloc/free device allocator callbacks (e.g. a framework's caching
 *             allocator); NULL = cudaMalloc/cudaFree [NULL] */
typedef struct {
    int precision;
    int coupling;
    double tau_min, tau_max;
    double dt_s;
    int check_every;
    int extrapolate_every;
    int step_variant;
    int init_mode;
    int outlet_bc;
    int grad_stencil;
    void *stream;
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *alloc_user;
    int extrapolate_modes;
} lbms_options;

typedef struct {
    int64_t n_cells, n_fluid;
    int q;                      /* 9 or 19 */
    int precision;
    double dx_m, dt_s, C_t;     /* C_t = p / RT (Section 4.1) */
    double D_eff_m2s[9];        /* Eq. 41, row-major 3x3 */
    double D_lat[9];            /* D_eff dt / dx^2 */
    double q_lat[3];            /* outlet flux per node per step, Eq. 39 */
    double x_in[3];
    double current_A_cm2;
    int64_t steps;              /* time steps taken since the last reset */
    size_t device_bytes;        /* device memory held by the handle */
    uint64_t h2d_bytes;         /* host-to-device bytes copied so far */
    uint64_t d2h_bytes;         /* device-to-host bytes copied so far */
    int n_cases;                /* cases in the handle (1 unless made by lbms_create_batch) */
    int tile_cells;             /* step-kernel tile picked by the autotuner: cells per block */
    int tile_min_blocks;        /*   and its register budget (resident blocks per SM) */
    int neighbour_bits;         /*   and its neighbour lookup: 32 (indices), 16 (offsets) or 1 (row bitmasks) */
    int threads_per_cell;       /*   and its thread mapping: 3 (one per species) or 1 */
} lbms_info;
/* n_cells and n_fluid sum over all cases; dx_m, dt_s, q_lat, x_in and
 * current_A_cm2 describe case 0. */

void lbms_default_options(lbms_options *opt);

/* Builds the solver: host properties (Eqs. 40-42, C_t, dx, dt), the fluid
 * cell list and its neighbour table, and the device state.  Nothing runs
 * until lbms_set_bc.  *out receives the handle, or NULL on failure, when
 * lbms_last_error(NULL) gives the reason (per thread).  Same as
 * lbms_create_batch with one case. */
lbms_status lbms_create(const lbms_geometry *geom, const lbms_species *species,
                        const lbms_diffusivities *diff, double T_K, double p_Pa,
                        const lbms_options *opt, lbms_ctx **out);

/* Batch of n_cases >= 1 independent anodes (geoms[n_cases], all with the
 * same dim; sizes, masks and lengths may differ) sharing the gas data and the
 * options.  Every lbms_step advances all cases with one kernel launch per
 * step (graph-replayed); the step kernel's tile shape is picked by timing
 * the compiled candidates on the first full initialisation (lbms_info).  The
 * paper runs one anode at a time; the batch is the sweep of Section 4.2
 * (several currents and dilutions) made one launch.  An explicit dt_s needs
 * the same grid spacing in every case. */
lbms_status lbms_create_batch(int n_cases, const lbms_geometry *geoms, const lbms_species *species,
                              const lbms_diffusivities *diff, double T_K, double p_Pa,
                              const lbms_options *opt, lbms_ctx **out);

/* Boundary data: inlet mole fractions (3, each >= 0, sum 1 within 1e-9;
 * Eq. 36) and current density (A/cm^2, >= 0; Eq. 39), for every case of the
 * handle.  The first call for a case initialises its fluid cells to
 * f = w X_in (Eq. 29); later calls change the boundary data and keep the
 * state. */
lbms_status lbms_set_bc(lbms_ctx *ctx, const double *x_inlet, double current_A_cm2);

/* As lbms_set_bc for case k only (0 <= k < n_cases).  Stepping needs every
 * case to have boundary data. */
lbms_status lbms_batch_set_bc(lbms_ctx *ctx, int k, const double *x_inlet, double current_A_cm2);

/* Restarts from a given field: X is host, 3*N dense (solid entries ignored),
 * f = w X (Eq. 29).  Resets the step counter and the residual snapshot.
 * Needs a prior lbms_set_bc (the boundary data).  Acts on case 0. */
lbms_status lbms_set_fields(lbms_ctx *ctx, const double *X);

/* As lbms_set_fields for case k, X being 3*N_k dense for that case's grid. */
lbms_status lbms_batch_set_fields(lbms_ctx *ctx, int k, const double *X);

/* Advances nsteps >= 0 time steps (Eq. 28 with the coupling of Eqs. 19-35
 * and the boundaries of Eqs. 36, 39).  Asynchronous: returns once the work is
 * queued on the stream. */
lbms_status lbms_step(lbms_ctx *ctx, int64_t nsteps);

/* Residual r = max_i ||X_i - X_i,snap||_2 / (K ||X_i||_2) over fluid cells
 * (FP64), where the snapshot is the state at the previous residual call (or
 * the last reset); refreshes the snapshot.  K >= 1 is the number of steps
 * since then.  LBMS_EUNSTABLE if NaN/Inf is present (residual set to inf).
 * With several cases, the maximum over cases. */
lbms_status lbms_residual(lbms_ctx *ctx, int K, double *residual);

/* Per-case residuals (residuals[n_cases]); refreshes every snapshot. */
lbms_status lbms_batch_residuals(lbms_ctx *ctx, int K, double *residuals);

/* Steps until the residual (checked every check_every steps) is <= tol or
 * max_steps are taken.  LBMS_ENOTCONVERGED in the latter case;
 * LBMS_EUNSTABLE on NaN/Inf.  steps_taken / final_residual may be NULL. */
lbms_status lbms_run_to_residual(lbms_ctx *ctx, double tol, int64_t max_steps,
                                 int64_t *steps_taken, double *final_residual);

/* Batch form: steps every case until all residuals are <= tol (or
 * max_steps).  case_steps[n_cases] receives the step count at which each case
 * first met tol (-1 if never) and final_residuals[n_cases] the last
 * residuals; either may be NULL.  LBMS_ENOTCONVERGED if a case missed tol. */
lbms_status lbms_batch_run_to_residual(lbms_ctx *ctx, double tol, int64_t max_steps,
                                       int64_t *steps_taken, int64_t *case_steps,
                                       double *final_residuals);

/* Fields of the last step on the dense grid, solid voxels zero (case 0).
 * X: 3*N mole fractions.  u: 3*dim*N component velocities (m/s,
 * [species][axis][z][y][x], Eq. 20) or NULL.  tau: 3*N relaxation times
 * (Eq. 25) or NULL. */
lbms_status lbms_get_fields(lbms_ctx *ctx, double *X, double *u, double *tau);

/* As lbms_get_fields for case k (arrays sized for that case's grid). */
lbms_status lbms_batch_get_fields(lbms_ctx *ctx, int k, double *X, double *u, double *tau);

/* Concentration overpotential (V) by Eq. 43 with X_out the mean over the
 * outlet column (FP64) and X_in the boundary values; x_out_mean (3 doubles)
 * may be NULL.  LBMS_EDEPLETED when a logarithm argument is <= 0.  Case 0. */
lbms_status lbms_overpotential(lbms_ctx *ctx, double *eta_V, double *x_out_mean);

/* Eq. 43 for every case: eta_V[n_cases], x_out_mean[3*n_cases] (or NULL).
 * A case whose logarithm is undefined gets NaN and the call returns
 * LBMS_EDEPLETED after filling the others. */
lbms_status lbms_batch_overpotentials(lbms_ctx *ctx, double *eta_V, double *x_out_mean);

/* Mass balance in FP64: inlet_flux[3] = net mole-fraction units per step
 * that cross the plane between x = 0 and x = 1 toward +x (carried by the
 * last post-collision populations); totals[3] = sum of X over fluid cells.
 * Either pointer may be NULL.  Case 0. */
lbms_status lbms_boundary_flux(lbms_ctx *ctx, double *inlet_flux, double *totals);

lbms_status lbms_get_info(const lbms_ctx *ctx, lbms_info *info);

/* Waits for all queued work of the handle. */
lbms_status lbms_synchronize(lbms_ctx *ctx);

/* Allocation-free residual sums, for callers that cannot allocate device
 * memory: code inside a CUDA graph being captured, hosts whose memory pool
 * owns every device allocation, loops that must not call cudaMalloc (it
 * synchronises the device).  The paper has no counterpart; this is an
 * integration helper that runs the residual reduction of lbms_residual on
 * caller-owned FP64 fields.
 *   X, snapshot  device, 3*n doubles each, species-major ([species][cell]);
 *                1 <= n <= INT32_MAX (larger n: LBMS_EINVAL).
 *   update       nonzero: the snapshot takes X after the sums are read.
 *   out          device, 10 doubles: out[0..2] = sum (X - snapshot)^2 per
 *                species, out[3..5] = sum X^2, out[6..8] = sum X,
 *                out[9] = number of non-finite X.  The residual of
 *                lbms_residual is max_i sqrt(out[i]) / (K sqrt(out[3+i])).
 *   stream       cudaStream_t (NULL = legacy default); the call only queues
 *                work and does not synchronise.
 * Scratch: a fixed 40 KiB device array (512 blocks x 10 partial sums) plus a
 * counter, held by every GPU that loads this library until the process
 * exits; the grid is capped at 512 blocks and the kernel walks the cells with
 * a 64-bit index, so any n in range fits.  The first call on a device looks
 * up the scratch address (once per device, with that device current) and
 * keeps it for the life of the process: make that first call before any
 * stream capture, and do not use this entry point after cudaDeviceReset on
 * that device (the module, and with it the scratch, may move).  All calls
 * share the scratch, so calls that overlap on the GPU (other streams, other
 * threads) race; serialise them.  Nothing is allocated or freed.
 * LBMS_EINVAL on NULL pointers or n out of range, LBMS_ECUDA on a CUDA error. */
lbms_status lbms_residual_sums_noalloc(const double *X, double *snapshot, int64_t n, int update,
                                       double *out, void *stream);

void lbms_destroy(lbms_ctx *ctx);
const char *lbms_last_error(const lbms_ctx *ctx);
const char *lbms_status_string(lbms_status s);

#ifdef __cplusplus
}
#endif

#endif /* LBMS_H */
