/*
 * wrffire.h -- C ABI of the GB300 (sm_103a) fire-model step of WRF-Fire
 * (Mandel, Beezley & Kochanski, "Coupled atmosphere-wildland fire modeling
 * with WRF-Fire version 3.3", arXiv:1102.1343).
 *
 * One call of fire_step is the fire model's time step of Sect. 5 ("Coupling
 * of the fire and the atmospheric models", the six-item list):
 *   1. active ignitions update the level-set function     (Sect. 3.4)
 *   2. Heun / Godunov advance of the level-set equation   (eqs. Heun, F-disc, Godunov)
 *   3. ignition time of newly ignited nodes               (eq. set-ignition-time)
 *   4. fuel fraction by submesh quadrature                (Sect. 3.3)
 *   5. sensible and latent heat flux per fire cell        (eqs. sensible-/latent-heat-flux)
 *   6. average of the fluxes over each atmospheric cell   (Sect. 5, item 6)
 * The surface wind (already at the 6.1 m height of Sect. 5) is the input, on
 * the staggered atmospheric grid of Sect. 3 ("Domain, grids, and nodes");
 * the averaged heat fluxes are the output.
 *
 * Conventions for every entry point:
 *  - Grids.  The atmospheric mesh has nx_atm x ny_atm cells of dx_atm x dy_atm
 *    metres.  The fire mesh refines it sr_x x sr_y times: NX = sr_x*nx_atm,
 *    NY = sr_y*ny_atm nodes at the cell centres ((i+1/2) dx, (j+1/2) dy),
 *    dx = dx_atm/sr_x.  Fire-mesh arrays are row-major [NY][NX]; the wind u is
 *    [ny_atm][nx_atm+1] at the x-faces (I dx_atm, (J+1/2) dy_atm), v is
 *    [ny_atm+1][nx_atm] at the y-faces; heat outputs are [ny_atm][nx_atm].
 *    NX, NY >= 2.
 *  - Precision.  FIRE_FP64 keeps every field in double.  FIRE_FP32 keeps the
 *    level-set function, fuel fraction, terrain gradient, multiplier and wind
 *    in float and the ignition time, the time and the heat reduction in
 *    double.  Pointers typed "const void*" point to elements of the context's
 *    precision (double for FIRE_FP64, float for FIRE_FP32).
 *  - Memory.  Pointers named *_dev are device pointers on the context's
 *    device; pointers named *_host are host pointers (pinned memory gives the
 *    fastest copies).  The caller owns every buffer it passes; fire_init
 *    copies what it needs, so its inputs may be freed after it returns.  The
 *    library owns the fire state (level set, ignition time, fuel fraction).
 *  - Streams.  All device work of a context is enqueued on the stream given
 *    to fire_init (a cudaStream_t; NULL = legacy default stream), in call
 *    order.  No call synchronises except fire_status, fire_get_state's time
 *    read-back, fire_kernel_time_ms and the *_host variants.
 *  - Errors.  Every call returns FIRE_OK (0) or a negative FIRE_ERR_* code and
 *    never aborts.  Faults detected on the device (fire reaching the boundary
 *    band, a non-finite level set or wind) are recorded in a sticky status
 *    word that fire_status reads.
 *  - Threads.  A context may be used by one host thread at a time.
 *  - Devices.  A context (or an ensemble) lives on the device current at its
 *    fire_init (fire_ensemble_create); every later call on it switches the
 *    calling thread to that device for its duration and back on return, so
 *    contexts of several GPUs may be used from one thread.
 */
#ifndef WRFFIRE_H
#define WRFFIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fire_ctx fire_ctx; /* opaque; created by fire_init, freed by fire_destroy */

enum fire_precision { FIRE_FP64 = 0, FIRE_FP32 = 1 };

enum fire_error {
    FIRE_OK = 0,
    FIRE_ERR_ARG = -1,       /* invalid argument or size */
    FIRE_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    FIRE_ERR_OOM = -3,       /* device or pinned host memory exhausted */
    FIRE_ERR_BOUNDARY = -4,  /* fire reached the boundary band (Sect. 3.1, last paragraph) */
    FIRE_ERR_NONFINITE = -5, /* non-finite wind or level-set value */
    FIRE_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
    FIRE_ERR_STATE = -7,     /* call not valid in the context's state */
    FIRE_ERR_BOUNDS = -8     /* a kernel formed an index outside its buffer (reported
                              * only by libraries built with FIRE_BOUNDS_CHECK,
                              * whose kernels check every global index; the
                              * access then goes to the buffer's first element) */
};

/* 1 if this library was built with FIRE_BOUNDS_CHECK (every global index of
 * the step kernels checked, FIRE_ERR_BOUNDS on a bad one; slower, for
 * testing), else 0.  No counterpart in the paper. */
int fire_bounds_checked(void);

/* Test of the index check itself (FIRE_BOUNDS_CHECK builds): one device
 * thread checks the indices -1, 0, 9 and 10 of a 10-element buffer, touching
 * no memory through them, and flags_host[4] receives whether each was
 * flagged (1 0 0 1 when the check works).  FIRE_ERR_STATE in other builds;
 * FIRE_ERR_ARG for a NULL pointer.  No counterpart in the paper. */
int fire_bounds_selftest(int *flags_host);

/* Grid and numerical parameters.
 *   eps_visc       artificial viscosity eps of eq. (F-disc), 0.4 in the paper.
 *                  The term is applied as eps * S * (scaled 5-point Laplacian),
 *                  the reading that makes it a speed.
 *   boundary_band  width (nodes) of the outer ring in which psi < 0 is reported
 *                  as FIRE_ERR_BOUNDARY; >= 1.
 *   psi_far        initial level-set value ("const > 0", Sect. 3.4); <= 0
 *                  selects the domain diagonal. */
typedef struct {
    int nx_atm, ny_atm;
    int sr_x, sr_y;
    double dx_atm, dy_atm;
    int precision;
    int boundary_band;
    double eps_visc;
    double psi_far;
} fire_grid_desc;

/* One fuel category: the properties of Table 1, in the units of Table 1.
 * Setting chaparral != 0 selects the chaparral rate of eq. (chapparal).
 * weight is the fuel weight w (s) of Table 1, from which the burn time is
 * T_f = -600 w / (1000 ln 0.6); with weight_is_tf != 0 it is T_f itself. */
typedef struct {
    double windrf;      /* a, wind reduction from 6.1 m to midflame height */
    double weight;      /* w (s), or T_f (s) when weight_is_tf */
    int weight_is_tf;
    int chaparral;
    double fgi;         /* w_l, total fuel load (kg m^-2) */
    double fueldepthm;  /* delta_m, fuel depth (m) */
    double savr;        /* sigma, surface-area-to-volume ratio (1/m) */
    double fuelmce;     /* M_x, moisture content of extinction */
    double fueldens;    /* rho_P, ovendry particle density (kg m^-3) */
    double st;          /* S_T, total mineral content */
    double se;          /* S_E, effective mineral content */
    double cmbcnst;     /* h, heat content of dry fuel (J kg^-1) */
    double fuelmc_g;    /* M_f, fuel particle moisture content */
} fire_fuel_class;

/* One ignition (Sect. 3.4): the segment from (ax, ay) to (bx, by) in metres
 * (a == b is a point).
 *   speed > 0: from time t_start the fire spreads from the segment at this
 *     speed S_g until the distance radius r_g is reached (eqs. ignition-lfn,
 *     ignition-min); applied at the start of every step with
 *     t_start <= t <= t_start + radius/speed; newly ignited nodes get the
 *     arrival time t_start + dist/speed.
 *   speed <= 0: instantaneous ignition of every node within radius of the
 *     segment, applied once at the first step start t >= t_start (at fire_init
 *     when t_start <= 0), with ignition time t_start.
 *   (vx, vy) != 0 (needs speed > 0 and t_end >= t_start): a drip torch (the
 *     paragraph after eq. ignition-min).  The torch leaves a at t_start with
 *     velocity (vx, vy) m/s until t_end; at a step start t the ignition line
 *     is the segment from a to a + v (min{t, t_end} - t_start) (bx, by are
 *     not used) and the fire around it has the radius min{radius, speed (t -
 *     t_start)}; applied at every step start with t_start <= t <= t_end +
 *     radius/speed.  A newly ignited node gets the time the fire, starting
 *     at the nearest point of the line when the torch laid it, reaches it at
 *     this speed, or t if that is later.
 * Zero-initialise unused fields (vx = vy = t_end = 0 for the other forms). */
typedef struct {
    double ax, ay, bx, by;
    double t_start;
    double radius;
    double speed;
    double vx, vy;  /* drip-torch velocity (m/s); 0, 0 for a fixed segment */
    double t_end;   /* drip torch: time the torch stops */
} fire_ignition;

#define FIRE_MAX_CLASSES 64
#define FIRE_MAX_IGNITIONS 256

/* Create a context: validates the grid, allocates the state on the current
 * device, evaluates the spread-rate coefficients of eq. (spread-WRF-Fire) per
 * fuel class from Table 2 (on the device, in double), and initialises the
 * state: psi = psi_far, no ignition time, fuel fraction 1, then the
 * instantaneous ignitions with t_start <= 0 (Sect. 3.4, "initialized with no
 * fire"; Sect. 5 "terrain gradient ... interpolated to the fire mesh in
 * preprocessing").
 *   classes[n_classes]    host array, 1 <= n_classes <= FIRE_MAX_CLASSES
 *   fuel_class_dev        uint8 [NY][NX] device, class index per node (< n_classes)
 *   moisture_dev          [NY][NX] device per-node fuel moisture M_f (>= 0,
 *                         context precision), or NULL (the class moisture
 *                         fuelmc_g).  The coefficients of eq.
 *                         (spread-WRF-Fire) are kept per grid point: with a
 *                         per-node M_f, R0, c, d and the heat factors H_s,
 *                         H_q of each node are evaluated from Table 2 at
 *                         that node's class and moisture (in double, stored
 *                         in the context precision, 5 values per node);
 *                         S0, b, e and T_f do not depend on M_f
 *   spread_mult_dev       [NY][NX] device per-node multiplier of S, or NULL (= 1)
 *   dzdx_dev, dzdy_dev    [NY][NX] device terrain gradient at the nodes
 *   ignitions[n_ign]      host array, 0 <= n_ign <= FIRE_MAX_IGNITIONS
 *   cuda_stream           cudaStream_t for all work of this context
 * On success *out receives the context; on failure *out is NULL. */
int fire_init(fire_ctx **out, const fire_grid_desc *grid,
              const fire_fuel_class *classes, int n_classes,
              const uint8_t *fuel_class_dev, const void *moisture_dev,
              const void *spread_mult_dev, const void *dzdx_dev, const void *dzdy_dev,
              const fire_ignition *ignitions, int n_ign, void *cuda_stream);

/* One fire time step t -> t + dt with the given wind (Sect. 5, items 1-6).
 *   wind_u_dev [ny_atm][nx_atm+1], wind_v_dev [ny_atm+1][nx_atm]: device,
 *     context precision, m/s at 6.1 m; constant within the step.
 *   dt > 0 (s).
 *   heat_sens_dev, heat_lat_dev: device double [ny_atm][nx_atm], receive the
 *     sensible and latent heat flux densities (W m^-2) averaged over each
 *     atmospheric cell for this step; either may be NULL to skip it.
 * Returns FIRE_OK once the step is enqueued (device faults show up in
 * fire_status). */
int fire_step(fire_ctx *ctx, const void *wind_u_dev, const void *wind_v_dev, double dt,
              double *heat_sens_dev, double *heat_lat_dev);

/* fire_step with host buffers: copies the wind to the device, runs the step,
 * copies the heat fluxes back and waits for them.  Buffers as in fire_step
 * but on the host; heat outputs may be NULL.  Heat outputs in page-locked
 * host memory that the device can address (cudaHostAlloc / cudaHostRegister,
 * e.g. torch's pin_memory) are written by the step kernel directly, with no
 * separate copy; pageable ones go through a device buffer and a copy. */
int fire_step_host(fire_ctx *ctx, const void *wind_u_host, const void *wind_v_host,
                   double dt, double *heat_sens_host, double *heat_lat_host);

/* nsteps fire steps with a wind held constant over all of them; the heat
 * outputs (nullable) receive the fluxes of the last step.  Steps without an
 * active ignition are replayed from a CUDA graph captured on first use. */
int fire_run(fire_ctx *ctx, int nsteps, double dt, const void *wind_u_dev,
             const void *wind_v_dev, double *heat_sens_dev, double *heat_lat_dev);

/* Copy the state out (checkpoint): psi and frac in the context precision,
 * tign double, each [NY][NX] device; any pointer may be NULL.  *t_host (if
 * not NULL) receives the model time. */
int fire_get_state(fire_ctx *ctx, void *psi_dev, double *tign_dev, void *frac_dev,
                   double *t_host);

/* Replace the state (resume): psi, frac in the context precision, tign double
 * (+inf = not ignited), each [NY][NX] device and all required; t the model
 * time.  Ignitions keep their applied/pending record. */
int fire_set_state(fire_ctx *ctx, const void *psi_dev, const double *tign_dev,
                   const void *frac_dev, double t);

/* Replace the per-node spread multiplier m (S := m S, [NY][NX] device,
 * context precision) by a copy of mult_dev; NULL removes it (m = 1).  Waits
 * for the copy.  Not for the context of an ensemble member. */
int fire_set_spread_mult(fire_ctx *ctx, const void *mult_dev);

/* Replace the fuel-class table (Table 1 properties, e.g. other moisture
 * values) by n_classes host records; n_classes must equal fire_init's.  The
 * per-class coefficients of eq. (spread-WRF-Fire) are recomputed (and the
 * per-node ones, where a per-node moisture is set); waits. */
int fire_set_fuel_classes(fire_ctx *ctx, const fire_fuel_class *classes, int n_classes);

/* Replace the per-node fuel moisture M_f by a copy of moisture_dev ([NY][NX]
 * device, context precision, >= 0) and recompute the per-node coefficients
 * (as fire_init does with a moisture); NULL returns to the class moisture.
 * Waits.  Not for the context of an ensemble member. */
int fire_set_moisture(fire_ctx *ctx, const void *moisture_dev);

/* Adjoint of the arrival-time misfit (data assimilation, the use the paper
 * gives for the level-set formulation in Sect. 7):
 *
 *     J = 1/2 sum over nodes with finite t_i and finite t_obs of (t_i - t_obs)^2
 *
 * after nsteps steps of dt from the current state with the wind held constant
 * (wind_u_dev, wind_v_dev as in fire_step).  No ignition may be active or
 * pending in those steps (else FIRE_ERR_STATE).  The context advances exactly
 * as fire_run would (same kernels, same state afterwards); its psi is saved
 * every ckpt_every steps and the states in between are recomputed during the
 * reverse sweep.  ckpt_every = 1 keeps every state (nsteps + 1 of them) and
 * recomputes nothing: the fastest form where they fit in device memory
 * (FIRE_ERR_OOM where they do not; a larger ckpt_every then trades memory
 * for the recomputation).
 *
 *   t_obs_dev    [NY][NX] double device; NaN or +-inf where not observed
 *   J_host       receives J (host double)
 *   g_mult_dev   dJ/dm per node, [NY][NX] double device, at the context's
 *                multiplier (1 where none was given)
 *   g_moist_dev  dJ/dM_f per node, [NY][NX] double device: the derivative for
 *                a change of the fuel moisture of that node alone, at the
 *                node's moisture (the per-node M_f where one is set, else
 *                the class moisture)
 *   g_u_dev      dJ/du on the x-faces [ny_atm][nx_atm + 1], double device
 *   g_v_dev      dJ/dv on the y-faces [ny_atm + 1][nx_atm], double device
 * Gradient pointers may be NULL; with all four NULL only J is computed.
 * Derivatives follow the branches the forward values take (upwind
 * selection, limits of the spread rate, boundary extrapolation), so they are
 * one-sided at switch points.  Workspace, kept by the context: the
 * checkpoints (nsteps/ckpt_every states, nsteps + 1 with ckpt_every = 1),
 * with ckpt_every > 1 a ring of ckpt_every + 1 recomputed states, and per
 * node about 6 path-precision values and 6 doubles (13 path-precision values
 * more in FP64, for its unfused reverse step).
 * Synchronous: returns after J and the gradients are written. */
int fire_adjoint(fire_ctx *ctx, int nsteps, double dt, const void *wind_u_dev,
                 const void *wind_v_dev, const double *t_obs_dev, int ckpt_every,
                 double *J_host, double *g_mult_dev, double *g_moist_dev, double *g_u_dev,
                 double *g_v_dev);

/* The same for a heat misfit (a data-assimilation objective for observed
 * fire heat release):
 *
 *     J = 1/2 sum over atmospheric cells with a finite q_obs of (Q - q_obs)^2,
 *     Q = sensible heat released per unit area of the cell over the nsteps
 *         steps = sum over its fire cells of (F_start - F_end) H_s / (sr_x sr_y)
 *
 * (J m^-2; the time integral of the heat_sens output of fire_step, whose sum
 * over steps telescopes).  The gradient also carries the moisture dependence
 * of H_s and, through the fuel-fraction quadrature of Sect. 3.3, the
 * dependence of F_end on psi and on the ignition times.
 *   q_obs_dev    [ny_atm][nx_atm] double device; NaN or +-inf where not observed
 * Everything else as fire_adjoint (the mesh needs at least 2 x 2 fire nodes);
 * the workspace also holds F at the start of the run (one path-precision
 * value per node) and three doubles per node for the seeds. */
int fire_adjoint_heat(fire_ctx *ctx, int nsteps, double dt, const void *wind_u_dev,
                      const void *wind_v_dev, const double *q_obs_dev, int ckpt_every,
                      double *J_host, double *g_mult_dev, double *g_moist_dev, double *g_u_dev,
                      double *g_v_dev);

/* Waits for the context's stream and returns the first sticky device fault
 * (FIRE_ERR_BOUNDARY, FIRE_ERR_NONFINITE, FIRE_ERR_TIMEOUT) or FIRE_OK;
 * FIRE_ERR_CUDA if the stream reports a CUDA error. */
int fire_status(fire_ctx *ctx);

/* Clears the sticky device status word (enqueued on the stream). */
int fire_clear_status(fire_ctx *ctx);

/* Fire-mesh size and the model time (host value, no synchronisation). */
int fire_mesh_size(const fire_ctx *ctx, int *nx, int *ny);
double fire_time(const fire_ctx *ctx);

/* Step-kernel variant and its tile shape, in atmospheric cells per CTA
 * (chosen by fire_init's defaults or the autotuner, settable for sweeps):
 *   FIRE_KERNEL_MARCH  two fire columns per thread marching down a strip of
 *                      kx*sr_x columns (an even number <= 248) and ky*sr_y
 *                      rows;
 *   FIRE_KERNEL_TILE   a 2-D tile of kx*sr_x by ky*sr_y nodes staged with
 *                      a 3-node halo in shared memory (any refinement);
 *   FIRE_KERNEL_WARP   each warp marches alone down a strip of kx*sr_x
 *                      columns (an even number <= 60) and ky*sr_y rows, rows
 *                      held in registers, neighbours exchanged by shuffles;
 *   FIRE_KERNEL_WARP4  (FIRE_FP32 only) the same with four columns per lane:
 *                      strips of kx*sr_x <= 120 columns, the per-row control
 *                      shared by four columns;
 *   FIRE_KERNEL_WARP_DENSE  (FIRE_FP32 only) FIRE_KERNEL_WARP's strips
 *                      with t_i read a row ahead where psi <= 0 and the two
 *                      cells of a lane in one packed fuel-fraction
 *                      evaluation: the same results bit for bit, faster
 *                      where much of the mesh burns, slower where little
 *                      does (with a per-node moisture it runs as
 *                      FIRE_KERNEL_WARP).
 * FIRE_ERR_ARG if the shape does not fit the variant or the device. */
enum fire_kernel_variant {
    FIRE_KERNEL_TILE = 0,
    FIRE_KERNEL_MARCH = 1,
    FIRE_KERNEL_WARP = 2,
    FIRE_KERNEL_WARP4 = 3,
    FIRE_KERNEL_WARP_DENSE = 4
};
int fire_set_kernel(fire_ctx *ctx, int variant, int kx, int ky);

/* Adaptive choice between FIRE_KERNEL_WARP and FIRE_KERNEL_WARP_DENSE (same
 * results bit for bit, so the choice changes no value): on from fire_init
 * when its default is FIRE_KERNEL_WARP (FIRE_FP32); off after fire_set_kernel,
 * fire_autotune or FIRE_FRACTION_LINEAR, and for ensemble members.  Every 64
 * steps (and at fire_init, and after fire_set_state) a small kernel counts
 * the nodes with psi <= 0 on the context's stream; the count is read on a
 * later step without waiting (a host that runs ahead of the device sees it,
 * and changes the kernel, that much later).  From a burnt fraction of 0.5 %
 * the steps run FIRE_KERNEL_WARP_DENSE with strips of ky = min(ky, 60/sr_y)
 * atmospheric rows; below 0.25 % the default strips come back.
 *   fire_set_adaptive(ctx, 1) turns it on with the current warp strips as
 *     the default shape (FIRE_ERR_ARG unless the context is FIRE_FP32 on
 *     FIRE_KERNEL_WARP or FIRE_KERNEL_WARP_DENSE with the subcell scheme);
 *     fire_set_adaptive(ctx, 0) turns it off and keeps the current kernel.
 *   fire_adaptive_info reports whether it is on, how many counts were
 *     launched so far and the last burnt fraction read (-1 before the
 *     first); outputs nullable. */
int fire_set_adaptive(fire_ctx *ctx, int on);
int fire_adaptive_info(const fire_ctx *ctx, int *on, long long *counts, double *burnt_fraction);

/* Fuel-fraction scheme of the context's steps:
 *   FIRE_FRACTION_SUBCELL (default)  the 4-subcell scheme of Sect. 3.3,
 *                 eqs. (approx-area), (approx-fraction);
 *   FIRE_FRACTION_LINEAR  the alternative the Discussion describes, exact
 *                 when psi and the time from ignition are linear in space.
 *                 Each subcell is split along its centre-corner diagonal;
 *                 on each triangle psi and t - t_i are the linear
 *                 interpolants of the same vertex values, the triangle is
 *                 clipped to psi <= 0 (t_i = t on the cut) and
 *                 1 - exp(-(t - t_i)/T_f) is integrated exactly; nodes not
 *                 ignited extend t - t_i as -lambda psi, lambda fitted on the
 *                 3x3 neighbourhood's burning nodes (exact for linear data).
 *                 Runs on the 2-D tile kernel only: selecting it switches the
 *                 context to tiles, and fire_set_kernel then refuses other
 *                 variants; fire_adjoint and fire_adjoint_heat refuse it
 *                 (FIRE_ERR_STATE).  More expensive per burning cell.
 * Not for the context of an ensemble member.  FIRE_ERR_ARG for an unknown
 * scheme. */
enum fire_fraction_scheme { FIRE_FRACTION_SUBCELL = 0, FIRE_FRACTION_LINEAR = 1 };
int fire_set_fraction_scheme(fire_ctx *ctx, int scheme);
int fire_get_kernel(const fire_ctx *ctx, int *variant, int *kx, int *ky);

/* Autotuner of the step kernel: times candidate shapes (the marching strip
 * with widths of about 16..248 columns and heights of about 8..512 rows; the
 * 2-D tile at a few shapes) for probe_steps launches each on a scratch copy
 * of the current state with the given wind and dt, keeps the fastest
 * (fire_set_kernel) and reports it (outputs nullable).  The state and the
 * model time are unchanged; the scratch is the context's workspace.
 * Synchronous. */
int fire_autotune(fire_ctx *ctx, const void *wind_u_dev, const void *wind_v_dev, double dt,
                  int probe_steps, int *variant, int *kx, int *ky);

/* The launch shape fire_init (and fire_step_noalloc) takes by default for a
 * mesh of nx_atm x ny_atm atmospheric cells refined sr_x x sr_y, in the given
 * precision, on a device with n_sm SMs: strips (warp strips in FP32 when
 * sr_x <= 30, else marching strips) as tall as the large-mesh shapes (~160 /
 * ~60 rows) while that still gives 3.5 / 2.5 waves of resident CTAs, else
 * shorter, down to one atmospheric cell; 2-D tiles of one atmospheric cell
 * where even those fill under a quarter of one wave.  A pure host
 * computation (no device needed); fire_init falls back to smaller tiles if
 * the shape's shared memory does not fit.  Returns FIRE_ERR_ARG for
 * non-positive sizes or an unknown precision. */
int fire_default_kernel(int precision, int nx_atm, int ny_atm, int sr_x, int sr_y, int n_sm,
                        int *variant, int *kx, int *ky);

/* Kernel timing: when enabled, CUDA events bracket every launch of the fused
 * step kernel on the context's stream; fire_kernel_time_ms waits for them and
 * returns the summed device time and the launch count since the last reset. */
int fire_enable_timing(fire_ctx *ctx, int on);
int fire_kernel_time_ms(fire_ctx *ctx, double *ms, long *launches);

/* One fire step on caller-owned state that allocates no memory: no
 * cudaMalloc, cudaFree or allocating library call, and no context.  For
 * callers that cannot allocate device memory while they run: applications
 * whose device memory comes from their own pool or from a host framework
 * that forbids driver allocations after start-up, coupled models that must
 * not touch the allocator inside their time loop (an allocation there can
 * synchronise the device, or fail once the pool holds the memory).  The
 * paper has no counterpart: it is a way of calling the same step as
 * fire_step (same kernels, same results) without a fire_ctx.
 *   grid, classes[n_classes]  as for fire_init; 1 <= n_classes <= 64
 *                             (FIRE_MAX_CLASSES), more is FIRE_ERR_ARG
 *   psi_in/out, frac_in/out   [NY][NX] device, context precision; in and out
 *                             must be different buffers
 *   tign_dev                  [NY][NX] device double, updated in place
 *   fuel_class_dev, spread_mult_dev (nullable), dzdx_dev, dzdy_dev,
 *   wind_u_dev, wind_v_dev    as for fire_init / fire_step
 *   t, dt                     model time at the step start, time step (s)
 *   heat_sens_dev, heat_lat_dev  [ny_atm][nx_atm] device double, nullable
 *   status_dev                device int that faults are OR-ed into
 *                             (bit 1 boundary, 2 non-finite, 8 an index
 *                             outside its buffer in a FIRE_BOUNDS_CHECK
 *                             build), nullable; with
 *                             NULL the faults go to a status word inside the
 *                             library's fixed array that no call reads back,
 *                             so they cannot be seen: pass status_dev to
 *                             detect fire at the boundary or non-finite input
 *   cuda_stream               stream for all work of the call
 * Ignitions are not applied: the state passed in already holds them.
 * Fuel classes are checked as fire_init checks them (FIRE_ERR_ARG).
 * Intermediate values (the class table, its coefficients, the start and end
 * time, and the status word when status_dev is NULL) live in one file-scope
 * device array of about 11 KB per device, held until the process exits.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make it before any stream
 * capture.  Every call shares the array and it keeps the last call's
 * contents, so calls that overlap on the GPU (other streams, other host
 * threads) race with each other: serialise them. */
int fire_step_noalloc(const fire_grid_desc *grid, const fire_fuel_class *classes, int n_classes,
                      const void *psi_in_dev, void *psi_out_dev, const void *frac_in_dev,
                      void *frac_out_dev, double *tign_dev, const uint8_t *fuel_class_dev,
                      const void *spread_mult_dev, const void *dzdx_dev, const void *dzdy_dev,
                      const void *wind_u_dev, const void *wind_v_dev, double t, double dt,
                      double *heat_sens_dev, double *heat_lat_dev, int *status_dev,
                      void *cuda_stream);

/* ---------------------------------------------------------------------
 * Batched ensemble: independent fire runs (different mesh sizes, fuels,
 * terrain, winds) advanced together.  Each fire_ensemble_step call runs all
 * members for nsteps steps in ONE persistent cooperative kernel launch (a
 * work list of member strips per step, a bounded grid-wide barrier between
 * steps), captured in a CUDA graph and replayed while its shape is
 * unchanged.  A member advanced here matches the same member advanced alone
 * by fire_step with the same kernel configuration.  Motivation: ensemble
 * data assimilation (Sect. 7, "Data assimilation"); not part of the paper's
 * fire step itself.
 * --------------------------------------------------------------------- */
typedef struct fire_ensemble fire_ensemble;
#define FIRE_MAX_MEMBERS 1024

/* One member: the arguments of fire_init (device arrays as there; moisture_dev
 * is the member's per-node fuel moisture or NULL).  All members must share
 * the precision.  When any member has a per-node moisture, every member's
 * step reads per-node coefficients (members without one get them from their
 * class moisture, 5 more values per node). */
typedef struct {
    fire_grid_desc grid;
    const fire_fuel_class *classes;
    int n_classes;
    const uint8_t *fuel_class_dev;
    const void *moisture_dev;
    const void *spread_mult_dev;
    const void *dzdx_dev;
    const void *dzdy_dev;
    const fire_ignition *ignitions;
    int n_ign;
} fire_member_desc;

/* Creates the members (fire_init each, on cuda_stream) and the work list.
 * Members need refinements that the marching kernel supports (sr_x <= 124). */
int fire_ensemble_create(fire_ensemble **out, int n_members, const fire_member_desc *members,
                         void *cuda_stream);

/* nsteps steps of every member with member winds wind_u_dev[m],
 * wind_v_dev[m] (host arrays of device pointers, context precision, held
 * constant over the call); heat_sens_dev / heat_lat_dev: host arrays of device
 * pointers (the arrays and their entries may be NULL) receiving each member's
 * last-step fluxes.  Steps in which a member has an active ignition window run
 * one by one through fire_step; the others in one persistent launch. */
int fire_ensemble_step(fire_ensemble *ens, int nsteps, double dt, const void *const *wind_u_dev,
                       const void *const *wind_v_dev, double *const *heat_sens_dev,
                       double *const *heat_lat_dev);

/* The member's context (owned by the ensemble: use it for fire_get_state,
 * fire_set_state, fire_status; do not destroy it). */
int fire_ensemble_member(fire_ensemble *ens, int member, fire_ctx **ctx);

/* Waits; returns FIRE_ERR_TIMEOUT if a barrier wait gave up, else the worst
 * member status; member_status (nullable host array [n]) receives each. */
int fire_ensemble_status(fire_ensemble *ens, int *member_status);
int fire_ensemble_clear_status(fire_ensemble *ens);

/* Strip shape of the persistent kernel in fire nodes (rounded to whole
 * atmospheric cells and an even width per member); the launch grid is sized
 * to the CTAs that fit on the device at once.  fire_ensemble_get_kernel
 * reports the grid and the number of work items per step. */
int fire_ensemble_set_kernel(fire_ensemble *ens, int strip_columns, int strip_rows);
int fire_ensemble_get_kernel(const fire_ensemble *ens, int *grid_ctas, int *work_items);

/* Autotuner of the strip shape: times candidate shapes (40..240 columns x
 * 20..320 rows) on probe_steps steps of the members with the given winds,
 * each from the members' current states, keeps the fastest and puts the
 * states back.  No ignition may be active or pending within 2 probe_steps
 * steps (else FIRE_ERR_STATE).  Outputs nullable.  Synchronous. */
int fire_ensemble_autotune(fire_ensemble *ens, int probe_steps, double dt,
                           const void *const *wind_u_dev, const void *const *wind_v_dev,
                           int *strip_columns, int *strip_rows);

/* Test hook for the bounded barrier: CTA skip_block (-1: none) never
 * arrives at the barriers, and waits give up after spin_limit polls (about
 * 100 ns each), setting FIRE_ERR_TIMEOUT and ending the launch. */
int fire_ensemble_set_barrier_test(fire_ensemble *ens, int skip_block, long long spin_limit);

void fire_ensemble_destroy(fire_ensemble *ens);

/* ---------------------------------------------------------------------
 * Coupling with the atmospheric model (Sect. "Coupling of the fire and the
 * atmospheric models"): the steps before and after the fire step.
 * --------------------------------------------------------------------- */

/* The wind at the height z_f above the terrain (6.1 m in the paper, after
 * BEHAVE) by vertical log-linear interpolation: at each of npts horizontal
 * points (e.g. the u-points [ny_atm][nx_atm+1] or the v-points
 * [ny_atm+1][nx_atm] of the staggered grid) the piecewise linear interpolant
 * in ln z of the values u(z0) = 0, u(z_1), u(z_2), ... at ln z0, ln z_1, ...,
 * evaluated at ln z_f; 0 where z_f <= z0.  Levels at or below z0 are not
 * used; above the highest level the top value is returned.
 *   precision        FIRE_FP32 or FIRE_FP64: the element type of all arrays
 *   u3d_dev, z3d_dev [nz][npts] device: the wind component and the height
 *                    above the terrain of the cell centres, level k of point
 *                    p at k*npts + p, heights increasing with k
 *   z0_dev           [npts] device roughness heights (m)
 *   out_dev          [npts] device: the wind at z_f (the input of fire_step)
 * Enqueued on cuda_stream; FIRE_ERR_ARG for bad sizes or null arrays. */
int fire_wind_at_height(int precision, int nz, long long npts, const void *u3d_dev,
                        const void *z3d_dev, const void *z0_dev, double z_f, void *out_dev,
                        void *cuda_stream);

/* Insertion of the fire's heat fluxes into the atmospheric tendencies, as
 * forcing in a layer above the surface with exponential decay in height:
 *   d(mu theta)/dt += mu phi_h / (cp rho) S_k,  d(mu q_m)/dt += mu phi_q / (L rho) S_k
 * in the model layer k between the face heights zw_k < zw_{k+1}, where S_k
 * is the layer average of the convergence of the flux phi exp(-z/z_ext),
 *   S_k = (exp(-zw_k/z_ext) - exp(-zw_{k+1}/z_ext)) / (zw_{k+1} - zw_k)
 * (reading: the paper's d/dz exp(-z/z_ext) with the sign of a heating; the
 * column integral of cp rho S_k dz is phi (1 - exp(-zw_top/z_ext))).
 *   ncols                 horizontal columns (the atmospheric cells, ny_atm*nx_atm)
 *   heat_sens_dev, heat_lat_dev [ncols] device double: phi_h, phi_q (W m^-2),
 *                         e.g. fire_step's outputs
 *   zw_dev                [nz+1][ncols] device double: face heights above the
 *                         terrain (m), zw_0 = 0, increasing
 *   rho_dev               [nz][ncols] device double: air density (kg m^-3)
 *   mu_dev                [ncols] device double: dry-air column mass mu (Pa)
 *   z_ext                 heat extinction depth (m, fire_ext_grnd), > 0
 *   cp, latent            specific heat of air (J kg^-1 K^-1) and L (J kg^-1)
 *   rth_dev, rqv_dev      [nz][ncols] device double: the sources are ADDED to
 *                         these tendencies; either may be NULL (skipped, and
 *                         then its flux array may be NULL too)
 * Enqueued on cuda_stream. */
int fire_heat_insertion(int nz, long long ncols, const double *heat_sens_dev,
                        const double *heat_lat_dev, const double *zw_dev, const double *rho_dev,
                        const double *mu_dev, double z_ext, double cp, double latent,
                        double *rth_dev, double *rqv_dev, void *cuda_stream);

const char *fire_strerror(int code);

/* Name and message of the last CUDA error an entry point saw on the calling
 * host thread, with the call that returned it ("no error" if none): detail
 * behind FIRE_ERR_CUDA / FIRE_ERR_OOM.  The string is owned by the library. */
const char *fire_last_cuda_error(void);

void fire_destroy(fire_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* WRFFIRE_H */
