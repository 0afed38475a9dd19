/*
 * sph.h -- C ABI of libsph, a GB300 (sm_103a) implementation of the time step of
 * the weakly compressible SPH method of Dominguez, Crespo & Gomez-Gesteira,
 * "Optimization strategies for parallel CPU and GPU implementations of a
 * meshfree particle method" (DualSPHysics).
 *
 * One time step is the paper's three stages (Section 2, Fig. 1), each a call:
 *   sph_neighbour_list  NL  cell-linked list: cell of every fluid particle, a
 *                           sort by (cell, id), reordering of all particle data,
 *                           first particle of every cell (Sections 2, 4.1,
 *                           Fig. 8);
 *   sph_interact        PI  fluid-fluid + fluid-boundary interactions of fluid
 *                           targets and boundary-fluid interactions of boundary
 *                           targets (Section 4.5): momentum and continuity with
 *                           the cubic spline, Tait pressure and artificial
 *                           viscosity (Table 1);
 *   sph_update          SU  variable time step from the largest force, sound
 *                           speed and viscous term (Section 4.1, Table 1) and
 *                           the Verlet scheme with a periodic Euler step (Table 1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units are SI.  Particle arrays exchanged with the caller are float64 in
 *   persistent-id order: fluid particles first (ids 0 .. n_f-1), then boundary
 *   particles (ids n_f .. n_f+n_b-1); vectors are [n][3] row-major.
 * - Every pointer argument may be host memory or device memory of the
 *   context's GPU (the library copies with cudaMemcpyDefault).
 * - Ownership: the caller owns all memory, including the device workspace given
 *   to sph_create; the library never allocates or frees device memory and keeps
 *   pointers into the workspace until sph_destroy.  The context itself is a
 *   small host allocation freed by sph_destroy.
 * - Work is enqueued on the caller's CUDA stream (`stream`, may be NULL for the
 *   legacy default stream).  Calls that return data to a host pointer
 *   synchronise that stream; the other calls are asynchronous.
 * - Errors: every int-returning call returns SPH_OK (0) or a negative
 *   SPH_ERR_* code; nothing is thrown across the ABI.  Conditions found on the
 *   device (a particle leaving the cell grid, a NaN, a vanishing time step) set
 *   bits of a device status word (SPH_FLAG_*) that sph_status reads; a call
 *   that synchronises returns SPH_ERR_DEVICE_FLAG when a flag is set.
 * - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* precision forms */
#define SPH_FP64       0  /* every stage in float64 */
#define SPH_FP32_SPLIT 1  /* PI in float32 on cell-relative float32 offsets; float64
                             position accumulation and time-step reduction */

/* PI kernel designs (same arithmetic, different mapping; see pi_kernel below) */
#define SPH_PI_WARP              0  /* one warp per cell: lockstep candidate tests in
                                       shared memory, per-lane hit walks (default) */
#define SPH_PI_THREAD            1  /* the paper's design: one thread per particle, 27
                                       cells from CellBeginEnd (Section 4.4, Fig. 11 top) */
#define SPH_PI_THREAD_FASTCELLS  2  /* one thread per particle, 9 ranges per cell
                                       precomputed after NL (Fig. 11 bottom) */
#define SPH_PI_WARP_SYM          3  /* the warp design with symmetric pairs (Section
                                       3.1, optimisation A, taken to the GPU): pairs
                                       between different cells evaluated once for
                                       both particles, both sides added with float
                                       atomics, so results are not bit-reproducible
                                       from run to run (float32 rounding only);
                                       cells >= 2h, no tensile correction */

/* return codes */
#define SPH_OK                 0
#define SPH_ERR_INVALID_ARG   -1
#define SPH_ERR_WORKSPACE     -2
#define SPH_ERR_CUDA          -3
#define SPH_ERR_DEVICE_FLAG   -4
#define SPH_ERR_TOO_LARGE     -5
#define SPH_ERR_SEQUENCE      -6  /* stage called out of order (NL -> PI -> SU) */

/* device status bits */
#define SPH_FLAG_OUT_OF_GRID   1u  /* a fluid particle left the cell grid; it is frozen */
#define SPH_FLAG_NAN           2u  /* NaN/Inf in a density, velocity or force */
#define SPH_FLAG_DT_TOO_SMALL  4u  /* variable dt fell below 1e-12 s */

/* Run constants (Table 1 formulation; see the oracle for every formula).
 * cell_size must be >= 2h (the support of the cubic spline); the cell grid
 * spans [dom_min, dom_max) with ceil((max-min)/cell_size) cells per axis. */
typedef struct sph_params {
    double dp;            /* particle spacing (m) */
    double h;             /* smoothing length (m); support radius 2h */
    double cell_size;     /* cell edge (m): >= 2h searches the 27 surrounding cells (9
                             x-runs, Fig. 10); an edge in [h, 2h) the 125 surrounding
                             cells (25 x-runs; the finer cells of Section 4.6,
                             optimisation F), supported by SPH_FP64 and by
                             SPH_PI_THREAD only; below h: SPH_ERR_INVALID_ARG */
    double rho0;          /* reference density (kg/m^3) */
    double gamma;         /* Tait exponent (SPH_FP32_SPLIT: 7 only, as in Table 1;
                             other values give SPH_ERR_INVALID_ARG) */
    double c0;            /* speed of sound at rho0 (m/s) */
    double alpha;         /* artificial viscosity coefficient */
    double eta2_coef;     /* eta^2 = eta2_coef * h^2 */
    double cfl;           /* Courant number of the variable time step */
    double mass;          /* particle mass (kg), the same for every particle */
    double g[3];          /* gravity (m/s^2) */
    double dom_min[3];    /* cell grid origin (m) */
    double dom_max[3];    /* cell grid end (m) */
    int64_t verlet_euler_every; /* N_s: an Euler step when (step+1) % N_s == 0 */
    double fixed_dt;      /* > 0: constant time step; <= 0: variable */
    int64_t clamp_boundary_rho; /* 1: boundary density never drops below rho0 */
    int32_t precision;    /* SPH_FP64 or SPH_FP32_SPLIT */
    int32_t pi_kernel;    /* SPH_PI_*.  SPH_FP64: SPH_PI_WARP (default: the warp-per-item
                             kernel with float32 lockstep tests and float64 pairs when
                             cell_size >= 2h, one thread per particle for finer cells)
                             or SPH_PI_THREAD (one thread per particle); the other
                             designs give SPH_ERR_INVALID_ARG */
    /* Tensile correction (Monaghan 2000; the "tensil" term of Table 3), off when
     * both coefficients are 0: the momentum term P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab
     * gains R_ab (W(r)/W(dp))^n with R_ab = tensile_pos (P_a/rho_a^2 + P_b/rho_b^2)
     * if both pressures are positive, else the sum of tensile_eps |P|/rho^2 over
     * the negative ones.  Supported by SPH_FP64 and by SPH_PI_WARP; not by the
     * thread-per-particle kernels or the adjoint (SPH_ERR_INVALID_ARG). */
    double tensile_eps;
    double tensile_pos;
    int64_t tensile_n;    /* exponent n >= 1 (4 in Monaghan 2000) */
} sph_params;

typedef struct sph_ctx sph_ctx;

/* Device workspace (bytes, 256-byte aligned start required) that sph_create
 * needs for n_f fluid and n_b boundary particles.  Returns SPH_ERR_INVALID_ARG
 * for inconsistent parameters and SPH_ERR_TOO_LARGE when a count or the cell
 * grid exceeds the 32-bit indices the kernels use (2^31 - 1). */
int sph_workspace_bytes(const sph_params *p, int64_t n_f, int64_t n_b, size_t *bytes);

/* Create a context on the current CUDA device: copies the initial state
 * (pos [n][3], vel [n][3], rho [n]; host or device; the previous Verlet level
 * is set equal to it), builds the boundary cell list once (boundaries never
 * move, Section 2) and leaves the context ready for sph_neighbour_list.
 * `workspace` is caller-owned device memory of at least sph_workspace_bytes.
 * Synchronises `stream` once. */
int sph_create(const sph_params *p, int64_t n_f, int64_t n_b,
               const double *pos, const double *vel, const double *rho,
               void *workspace, size_t ws_bytes, void *stream, sph_ctx **out);

/* NL (Section 4.1): cell of every fluid particle, sort by (cell, id) (a
 * counting sort by cell, then the rank by id inside each cell), all fluid
 * arrays copied into that order, packed PI inputs (Section 4.3), the first
 * index of every cell and the PI work items.  Asynchronous. */
int sph_neighbour_list(sph_ctx *ctx);

/* PI (Sections 4.3-4.5): forces and density rates of every particle from its
 * 27 neighbouring cells (9 x-runs), plus the maxima the time step needs.
 * Requires sph_neighbour_list since the last update.  Asynchronous. */
int sph_interact(sph_ctx *ctx);

/* SU (Section 4.1): time step dt = CFL * min(sqrt(h/max|f|), h/(max c + max
 * visc)) (or the fixed dt), then the Verlet / Euler update.  When dt_out is
 * not NULL the stream is synchronised and the dt used is written there.
 * Requires sph_interact since the last update. */
int sph_update(sph_ctx *ctx, double *dt_out);

/* n_steps repetitions of NL, PI, SU.  Asynchronous. */
int sph_run(sph_ctx *ctx, int64_t n_steps);

/* The same steps replayed from a CUDA graph: two consecutive steps (the
 * particle buffers swap every step, so that pair repeats) are captured once
 * per context and launched n_steps / 2 times, an odd last step runs as
 * ordinary launches.  Results are identical to sph_run.  Needs a stream created
 * by the caller (not the legacy or per-thread default stream; else
 * SPH_ERR_INVALID_ARG).  The executable graphs are driver resources released by
 * sph_destroy.  Asynchronous. */
int sph_run_graph(sph_ctx *ctx, int64_t n_steps);

/* Copy the state out in persistent-id order (any pointer may be NULL).
 * vel_prev / rho_prev are the previous Verlet level.  Synchronises. */
int sph_get_state(sph_ctx *ctx, double *pos, double *vel, double *rho,
                  double *vel_prev, double *rho_prev);

/* Replace the state (persistent-id order).  pos, vel and rho are required;
 * vel_prev / rho_prev may be NULL (then equal to vel / rho).  Boundary
 * positions are taken as given and their cell list is rebuilt.  The step
 * counter and time are kept.  Synchronises. */
int sph_set_state(sph_ctx *ctx, const double *pos, const double *vel, const double *rho,
                  const double *vel_prev, const double *rho_prev);

/* Simulated time, last dt and number of completed steps.  Synchronises. */
int sph_get_time(sph_ctx *ctx, double *time, double *last_dt, int64_t *steps);

/* Device status bits (SPH_FLAG_*), cleared when clear != 0.  Synchronises. */
int sph_status(sph_ctx *ctx, uint32_t *flags, int clear);

/* The fluid neighbour list of the last sph_neighbour_list: for sorted position
 * k, sorted_id[k] is the persistent id and cell[k] the cell id (n_cells for a
 * particle outside the grid); cell_start[c] for c = 0 .. n_cells+1 is the
 * number of fluid particles with cell < c (the CellBeginEnd array of Fig. 8:
 * cell c holds [cell_start[c], cell_start[c+1])).  Any pointer may be NULL;
 * sizes are n_f, n_f and n_cells+2.  Synchronises. */
int sph_get_neighbour_list(sph_ctx *ctx, uint32_t *sorted_id, uint32_t *cell,
                           int32_t *cell_start);

/* Grid dimensions (cells per axis) of the context. */
int sph_get_grid(sph_ctx *ctx, int64_t dims[3]);

/* PI outputs of the last sph_interact in persistent-id order: ace [n_f][3]
 * (acceleration, gravity included), ar [n_f+n_b] (density rate) and the three
 * time-step maxima {max|f|, max c, max visc}.  Any pointer may be NULL.
 * Synchronises. */
int sph_get_forces(sph_ctx *ctx, double *ace, double *ar, double *maxima);

/* Exact work counts of the current neighbour list and state (a validation
 * pass, not part of a step): counts[0] candidates tested by fluid targets
 * (members of their 27 cells, fluid and boundary lists, self excluded),
 * counts[1] fluid-target pairs (F-F + F-B), counts[2] candidates of boundary
 * targets, counts[3] boundary-target pairs (B-F).  A pair is an ordered (a, b),
 * a != b, |x_a - x_b| < 2h.  Requires sph_neighbour_list.  Synchronises. */
int sph_count_work(sph_ctx *ctx, int64_t counts[4]);

/* Number of kernels this context has launched so far. */
int64_t sph_launch_count(const sph_ctx *ctx);

/* Size in bytes of one checkpoint of the full state (for sph_save_state). */
int sph_checkpoint_bytes(const sph_ctx *ctx, size_t *bytes);

/* Copy the full internal state (all arrays, step counter, time) into the
 * caller's device buffer `dst` / back from it.  Asynchronous. */
int sph_save_state(sph_ctx *ctx, void *dst);
int sph_load_state(sph_ctx *ctx, const void *src);

/* ---- objective and adjoint (differentiable form) -------------------------
 * An adjoint vector lam is float64 in persistent-id order with the layout of
 * sph_get_state: [x: 3N][v: 3N][rho: N][v_prev: 3N][rho_prev: N], N = n_f + n_b
 * (boundary rows of x, v and v_prev are unused).  It holds dJ/d(state) for a
 * scalar objective J. */

/* Maximum number of sensor points per call. */
#define SPH_MAX_SENSORS 4096

/* Pressure at sensor points (device [S][3] float64) for the current state,
 * Shepard-normalised over the fluid particles within 2h:
 *   P_s = sum_b (m/rho_b) P_b W_sb / sum_b (m/rho_b) W_sb   (0 with no particle),
 * with the Tait pressure and cubic spline of Table 1.  Output: device [S].
 * Requires sph_neighbour_list for the current state.  Asynchronous. */
int sph_sensor_pressure(sph_ctx *ctx, const double *sensors, int64_t n_sensors,
                        double *pressure);

/* Adds to lam (device, layout above) the derivative of J = sum_s dj_dp[s] P_s
 * with respect to the current state's positions and densities.  SPH_FP64 only;
 * requires sph_neighbour_list for the current state.  Asynchronous. */
int sph_sensor_adjoint(sph_ctx *ctx, const double *sensors, int64_t n_sensors,
                       const double *dj_dp, double *lam);

/* Front position of the fluid: the smooth maximum J = tau log sum_a exp(x_a / tau)
 * of the x coordinates of all fluid particles of the current state (between
 * max x and max x + tau log n_f; tau > 0, e.g. dp), as a differentiable
 * measure of how far the collapsing column has run.  The paper defines no
 * objective: this one and the sensor pressures serve the differentiable form.
 * Output: device double *J.  SPH_ERR_INVALID_ARG without fluid particles or
 * for tau <= 0.  Asynchronous. */
int sph_front_position(sph_ctx *ctx, double tau, double *J);

/* Adds to lam (device, layout above) the derivative of dj * J_front with
 * respect to the current positions: dj exp((x_a - max x) / tau) /
 * sum_b exp((x_b - max x) / tau) on the x component of fluid particle a.
 * dj is a host value.  SPH_FP64 only.  Asynchronous. */
int sph_front_adjoint(sph_ctx *ctx, double tau, double dj, double *lam);

/* Adjoint of one time step at fixed dt (PI + SU, Table 1 formulation; the
 * neighbour relation of the step is a constant of the step).  The context must
 * hold the state at the start of the step (e.g. after sph_load_state of a
 * snapshot taken then); the call rebuilds that step's neighbour list and PI
 * (left valid, so sph_sensor_adjoint may follow), then writes to lam the adjoint
 * of the state at the start of the step given lam_next, the adjoint of the state
 * after it, and adds dJ/dalpha to *dalpha.  lam, lam_next and dalpha are device
 * memory and must not alias.  SPH_FP64 with fixed_dt > 0 and no tensile
 * correction only (else SPH_ERR_INVALID_ARG).  Asynchronous. */
int sph_adjoint_step(sph_ctx *ctx, const double *lam_next, double *lam, double *dalpha);

/* Limits of sph_neighbour_list_static (points, cells of the grid). */
#define SPH_STATIC_MAX_POINTS 524288
#define SPH_STATIC_MAX_CELLS  16777216

/* The neighbour list of one point set, computed without any device
 * allocation.  The paper has no counterpart: this call is for callers that
 * cannot call cudaMalloc -- a solver embedded in a host program whose own
 * allocator owns all of the GPU's memory, or a loop that must not stall on
 * cudaMalloc/cudaFree, which can synchronise the whole device.
 *   p           run constants; only the cell grid (h, cell_size, dom_min,
 *               dom_max) and the parameter checks of sph_workspace_bytes matter
 *   n           number of points, at most SPH_STATIC_MAX_POINTS; the grid may
 *               have at most SPH_STATIC_MAX_CELLS cells (else SPH_ERR_TOO_LARGE)
 *   pos         [n][3] float64 positions in device memory of the current GPU
 *   sorted_id   out, [n] uint32: the points in (cell, index) order
 *   cell        out, [n] uint32: cell id of sorted_id[k] (n_cells if outside)
 *   cell_start  out, [n_cells + 2] int32: number of points in cells below c
 *               (the CellBeginEnd array of sph_get_neighbour_list)
 *   stream      CUDA stream (NULL: legacy default stream); asynchronous.
 * Every output is device memory the caller owns.  The same outputs as the fluid
 * part of sph_neighbour_list for the same positions, bit for bit.
 * Scratch: one fixed device array inside the library (about 8.7 MB), held by
 * every GPU that loads the library until the process exits.  Every call looks
 * up that array's device address on the current device (cudaGetSymbolAddress);
 * the first call on a device may also load the library's device code there, so
 * make that first call before any stream capture.
 * Every call shares the array and leaves its contents behind, so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise them. */
int sph_neighbour_list_static(const sph_params *p, int64_t n, const double *pos,
                              uint32_t *sorted_id, uint32_t *cell, int32_t *cell_start,
                              void *stream);

/* Measurement helper, not part of the method: the rate of independent fused
 * multiply-adds on the current device, i.e. the arithmetic roofline of PI
 * (float32 FMAs for SPH_FP32_SPLIT, float64 FMAs for SPH_FP64).  One warm-up
 * and one timed launch of a kernel of 8 independent FMA chains per thread and
 * 2048 threads per SM, timed with CUDA events on `stream` (about 10 ms).
 *   precision  SPH_FP32_SPLIT or SPH_FP64, else SPH_ERR_INVALID_ARG
 *   scratch    device memory of at least 8 bytes that the caller owns (written
 *              only if the chains reached a value they cannot reach)
 *   stream     CUDA stream (NULL: legacy default stream)
 *   flops      out: 2 x FMAs per second (host)
 * Synchronises the stream. */
int sph_fma_rate(int precision, void *scratch, void *stream, double *flops);

/* Human-readable text of a return code (static storage). */
const char *sph_error_string(int code);

/* Free the host-side context (the workspace stays the caller's). */
void sph_destroy(sph_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
