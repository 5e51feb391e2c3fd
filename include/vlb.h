/*
 * vlb.h -- C ABI of a GB300 (sm_103a) implementation of the volumetric
 * lattice Boltzmann method for thermal particulate flows with conjugate heat
 * transfer (Zhang, Wang, Li & Huang, arXiv 2410.23802).
 *
 * One time step (Sec. 2 of the paper) consists of
 *   - the particle update (Eqs. 26, 29, 30; forward Euler) with contact forces,
 *   - the solid fraction f_s of every cell from the particle positions (Sec. 2),
 *   - collision and streaming of the flow populations f (Eqs. 3-7) followed by
 *     the volumetric nonslip correction (Eq. 8) and the macroscopic rho, u (Eq. 9),
 *   - the momentum-exchange force and torque on each particle (Eq. 28),
 *   - collision and streaming of the internal-energy populations g (Eqs. 17-20)
 *     with the convection term as a source (Eq. 16), variable c_v and lambda
 *     (Eq. 11), the local temperature gradient (Eq. 23), the df_s/dt recursion
 *     (Eq. 24) and the implicit temperature (Eq. 25).
 *
 * Units are lattice units (dx = dt = c = 1, rho_f = c_vf = 1).  The lattice has
 * nx * ny cells; cell (i, j) covers [i, i+1] x [j, j+1] and its node sits at
 * the cell centre.  Field arrays exchanged with the caller are row-major with
 * y as the slow index: element (j, i) is at j * nx + i.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a vlb_status; no C++ exception crosses the ABI.
 *   - All pointers are HOST pointers owned by the caller unless stated.  The
 *     library owns all device memory of a handle and frees it in vlb_destroy.
 *   - Work is queued on the handle's CUDA stream; vlb_step returns before the
 *     GPU finishes.  The vlb_get_* calls synchronise that stream first.
 *   - A handle is not thread-safe; separate handles are independent.
 *   - On failure the call returns a negative status and vlb_last_error()
 *     describes it; the handle stays usable unless the status is VLB_ECUDA.
 *   - Device-side failures (list overflows, a particle leaving the domain or
 *     moving faster than 0.5 lu per step, NaN) set a flag that the next call
 *     returns as VLB_EOVERFLOW or VLB_EUNSTABLE; no kernel traps or spins.
 */
#ifndef VLB_H
#define VLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VLB_ABI_VERSION 1u

typedef struct vlb_handle vlb_handle;

typedef enum {
  VLB_OK = 0,
  VLB_EINVAL = -1,     /* bad argument or parameter */
  VLB_ENOMEM = -2,     /* device or host allocation failed */
  VLB_ECUDA = -3,      /* a CUDA call failed; the handle should be destroyed */
  VLB_ESTATE = -4,     /* call not allowed in the handle's current state */
  VLB_EUNSTABLE = -5,  /* NaN, a particle too fast, or a particle out of the domain */
  VLB_EOVERFLOW = -6,  /* a fixed-capacity list (owners, tile lists, contacts) overflowed */
  VLB_ETIMEOUT = -7    /* a bounded device-side wait ran out (vlb_step_batch) */
} vlb_status;

/* Arithmetic and storage precision of the lattice populations. */
typedef enum {
  VLB_FP64 = 0,        /* FP64 storage and arithmetic */
  VLB_FP32 = 1,        /* FP32 storage and arithmetic */
  VLB_FP16_STORE = 2,  /* FP16 storage of the populations (as deviations from the rest
                          equilibrium), FP32 arithmetic; FP64 particle sums and integration */
  VLB_BF16_STORE = 3   /* the same with BF16 storage */
} vlb_precision;

typedef enum { VLB_WALL_ADIABATIC = 0, VLB_WALL_DIRICHLET = 1 } vlb_thermal_wall;

/* Field selection bits of vlb_get_fields. */
enum {
  VLB_FIELD_RHO = 1,
  VLB_FIELD_UX = 2,
  VLB_FIELD_UY = 4,
  VLB_FIELD_T = 8,
  VLB_FIELD_FS = 16
};

/*
 * Problem statement (Sec. 3 of the paper; rho_f = c_vf = 1).  Fill it with
 * vlb_params_default() and override fields.  Walls sit on the cell faces of
 * every non-periodic side; they are no-slip (halfway bounce-back of f) and
 * either adiabatic (bounce-back of g) or held at wall_T (anti-bounce-back).
 * A side whose bit is set in outflow_mask is open instead: the fully
 * developed condition of Sec. 3.2 (zero normal derivative), read as a
 * population entering there taking the value the same population has one
 * cell further in, for f and g; no wall contact there.
 * Side order in the [4] arrays and the mask bits: x-, x+, y-, y+.
 */
typedef struct {
  uint32_t abi_version;       /* must equal VLB_ABI_VERSION */
  int32_t nx, ny;             /* lattice cells, >= 2 each */
  int32_t periodic[2];        /* 1 = periodic in x / y instead of walls */
  int32_t thermal_wall[4];    /* vlb_thermal_wall per side */
  int32_t thermal_rates_mode; /* 0: (1/s_j-1/2)(1/s_e-1/2)=1/4 (Sec. 3); 1: s_0=s_e=s_eps=1 (Sec. 3.5) */
  int32_t precision;          /* vlb_precision */
  int32_t max_particles;      /* capacity of the particle arrays */
  int32_t outflow_mask;       /* bit k set: side k is open (outflow); 0: every side is a wall */
  int32_t reserved1;          /* zero */
  double tau_f;               /* flow relaxation time, s_p = 1/tau_f (Sec. 2.1) */
  double lambda_q_flow;       /* (1/s_p-1/2)(1/s_q-1/2); the paper uses 1/12 (Sec. 3) */
  double s_e;                 /* s_e = s_eps; the paper uses 1.25 (Sec. 3) */
  double prandtl;             /* Pr = nu / alpha_f; sets lambda_f = nu / Pr */
  double rho_ratio;           /* rho_s / rho_f, all particles */
  double cv_ratio;            /* R_cv = c_vs / c_vf (pseudo specific heat, Sec. 2.2) */
  double k_ratio_default;     /* R_lambda = lambda_s / lambda_f when none is given per particle */
  double gravity[2];          /* gravitational acceleration g (lattice units) */
  double beta;                /* volume expansivity; buoyancy -rho_f beta g (T - T_ref) on the fluid */
  double T_ref;               /* buoyancy reference temperature */
  double T_fluid_init;        /* initial fluid temperature */
  double wall_T[4];           /* wall temperatures of Dirichlet sides */
  double contact_range;       /* zeta of the short-range contact force (lu) */
  double contact_eps_p;       /* stiffness parameter between particles */
  double contact_eps_w;       /* stiffness parameter between a particle and a wall */
} vlb_params;

/* sizeof(vlb_params), for bindings that re-declare the struct. */
size_t vlb_params_size(void);

/* Fill *p with the paper's defaults: tau_f = 0.8, lambda_q_flow = 1/12,
 * s_e = 1.25, Pr = 0.7, rho_ratio = 1.5, R_cv = R_lambda = 1, no gravity,
 * beta = 0, T_ref = T_fluid_init = 1, adiabatic walls on four sides,
 * mode 0, zeta = 2, eps_p = 0.01, eps_w = 0.005, FP32, 1024 particles.
 * Returns VLB_EINVAL if p is NULL. */
vlb_status vlb_params_default(vlb_params* p);

/* Allocate a lattice of p->nx * p->ny cells on the current CUDA device and
 * its particle arrays.  *out receives the handle (NULL on failure).  Errors:
 * VLB_EINVAL for inconsistent parameters (tau_f <= 1/2, ratios <= 0, bad
 * sizes, unknown precision), VLB_ENOMEM, VLB_ECUDA. */
vlb_status vlb_create(const vlb_params* p, vlb_handle** out);

/* Hold particles [first, first + n) at their temperature T0 (held[k] != 0)
 * or let them conduct (held[k] == 0, the default): in the held-temperature
 * sedimentation case of Sec. 3.3 the particle stays at T_c; the paper does
 * not say how.  held[k] == 1 (reading R11): in the part of a cell such a
 * particle covers, the thermal populations are replaced by the equilibrium
 * at T0 in the volumetric form of Eq. 8,
 * g = (1 - f_fix) g + sum_p f_s,p g^eq(c_vs T0_p, T0_p).  held[k] == 2
 * (reading R11b): every cell the particle owns takes that equilibrium whole
 * (weight 1 in place of f_s,p; several such owners share the cell equally).
 * Other non-zero values mean 1.  Only before the first vlb_step (VLB_ESTATE
 * afterwards); VLB_EINVAL for a range outside the particles added so far. */
vlb_status vlb_set_fixed_temperature(vlb_handle* h, int32_t first, int32_t n, const int32_t* held);

/* Queue all further work of h on cuda_stream (a cudaStream_t; NULL selects
 * the legacy default stream).  Pending work on the previous stream is
 * synchronised first. */
vlb_status vlb_set_stream(vlb_handle* h, void* cuda_stream);

/* Append n disks (Sec. 2.3) before the first step.  xy[2n] centres, radius[n]
 * (>= 1 lu), T0[n] initial temperatures; k_ratio[n] per-particle
 * lambda_s/lambda_f, uv[2n] and omega[n] initial velocities may be NULL
 * (defaults: k_ratio_default, 0, 0).  Host arrays, copied.  Errors:
 * VLB_ESTATE after the first step, VLB_EINVAL if a disk leaves the domain,
 * overlaps another or crosses a periodic boundary, VLB_EOVERFLOW beyond
 * max_particles. */
vlb_status vlb_add_particles(vlb_handle* h, int32_t n, const double* xy, const double* radius,
                             const double* T0, const double* k_ratio, const double* uv,
                             const double* omega);

/* Append n elliptical particles (Sec. 3.2) before the first step: centres
 * xy[2n], semi-axes semi_a[n] >= semi_b[n] >= 1 lu, theta[n] the angle of
 * the major axis from the x axis (radians), then as vlb_add_particles.
 * Reading of the paper (silent on all of it): the solid fraction is the
 * exact area of ellipse and cell; a cell is solid when its four corners lie
 * in the ellipse and fluid when the ellipse's quadratic form stays >= 1
 * over it, both decided in FP64; the orientation advances with the angular
 * velocity (theta + Omega per step, forward Euler) and sets the raster; mass
 * rho_s pi a b, moment of inertia M (a^2 + b^2) / 4; between particles the
 * contact force acts on the circumscribed disks (radius semi_a), at a wall
 * on the ellipse's extent along the wall's normal.  A particle with
 * semi_a == semi_b is a disk.  Errors as vlb_add_particles (the domain and
 * overlap tests use the circumscribed disks), VLB_EINVAL for semi-axes out
 * of order or below 1. */
vlb_status vlb_add_ellipses(vlb_handle* h, int32_t n, const double* xy, const double* semi_a,
                            const double* semi_b, const double* theta, const double* T0,
                            const double* k_ratio, const double* uv, const double* omega);

/* Add n disks between two steps (mid-run insertion; before the first step
 * the same as vlb_add_particles).  Reading (the paper has no insertion): a
 * disk inserted at the current level n joins the particle set with the given
 * centre and velocity and first appears in the solid fraction of level n+1;
 * from there the paper's own equations act on it -- the volumetric
 * correction (Eq. 8) imposes its velocity in the cells it covers, and the
 * change of f_s enters the energy equation through df_s/dt (Eq. 24), so a
 * conducting disk starts at the temperature of the fluid it displaces (T0
 * is kept for vlb_set_fixed_temperature-style holding and inspection).  Its
 * first update has no exchange or particle contact force.  Arguments as for
 * vlb_add_particles.  Errors: VLB_EINVAL for a disk outside the domain,
 * overlapping a disk where that disk is now, or larger than the largest disk
 * present at the first step (the band tables' size); VLB_EOVERFLOW beyond
 * max_particles.  Synchronises the handle's stream. */
vlb_status vlb_insert_particles(vlb_handle* h, int32_t n, const double* xy, const double* radius, const double* T0,
                                const double* k_ratio, const double* uv, const double* omega);

/* Advance nsteps >= 0 time steps (asynchronous).  The first call builds the
 * initial state (f at rest, corrected by f_s^0; g at equilibrium with the
 * volume-weighted initial temperature).  Returns a device-side failure of
 * earlier steps if one has been recorded. */
vlb_status vlb_step(vlb_handle* h, int32_t nsteps);

/* nsteps time steps of each of n handles (independent cases of any sizes,
 * e.g. many small channels), in one of two forms (vlb_set_batch_form):
 *   0  per step, one launch of the particle step over every particle of every
 *      case and one lattice launch of one CTA per tile of any case (one per
 *      distinct precision / storage / held-path combination);
 *   1  per step, one persistent launch per such combination: a grid of the
 *      GPU's resident capacity whose CTAs take, in order from a device
 *      counter, the lattice tiles of every case and then the particle steps
 *      of the next level, each particle after a bounded wait for the last
 *      tile of its own case.  The launches of one step are the same every
 *      step: up to 64 steps of them are captured into a CUDA graph (its
 *      executable form kept per host thread and updated) and replayed
 *      (plain launches on the legacy default stream, which cannot be
 *      captured).  A wait that runs out (VLB_ETIMEOUT on that handle) leaves
 *      the context usable.
 * Each handle advances exactly as vlb_step(h, nsteps) would, in either form,
 * bit for bit, and single steps and batch calls may alternate.  The work is
 * queued on hs[0]'s stream after the work already queued on every handle's
 * stream; every handle's stream then waits for it, so later calls on any
 * handle are ordered after the batch.  Batch steps are not recorded by
 * vlb_profile_begin / vlb_profile_end.
 *   hs      host array of n distinct handles (borrowed)
 *   failed  NULL, or receives -1 on success and else the index of the handle
 *           whose failure is returned; vlb_last_error(hs[*failed]) describes
 *           it (vlb_last_error(NULL) for a NULL handle or a bad argument).
 * Errors: VLB_EINVAL for n < 0, nsteps < 0, a NULL or repeated handle; a
 * handle's pending device flags (as vlb_step would return them); VLB_ECUDA.
 * No handle advances unless every handle passes the checks.  Device flags
 * raised during the call surface on each handle's next call, as with
 * vlb_step.  Not part of the paper: it batches the paper's time step over
 * cases. */
vlb_status vlb_step_batch(vlb_handle* const* hs, int32_t n, int32_t nsteps, int32_t* failed);

/* The form of later vlb_step_batch calls and served rounds, process-wide:
 * 0 or 1 as above.  The default is the build's (0 unless built with
 * VLB_BATCH_PERSISTENT=1; on GB300 the two forms measured equal on 256
 * channels and form 0 faster in served rounds of a few small cases).
 * VLB_EINVAL for another value. */
vlb_status vlb_set_batch_form(int32_t form);
int32_t vlb_get_batch_form(void);

/* Test hook of the bounded waits of vlb_step_batch (form 1): wait_ns is the limit of
 * each device-side wait (<= 0: the default, one second; a normal wait lasts
 * less than one lattice pass).  stuck_handle >= 0 names a position in the
 * handle array of later vlb_step_batch calls whose particle steps then wait
 * for a tile count that is never reached, so that those waits run out: the
 * handle's next call returns VLB_ETIMEOUT (its state is no longer valid), the
 * other handles and the context are unaffected.  -1 turns it off.
 * Process-wide.  VLB_EINVAL for stuck_handle < -1. */
vlb_status vlb_debug_batch_wait(int64_t wait_ns, int32_t stuck_handle);

/* Block until the handle's queued work is done; returns the first recorded
 * device-side failure, else VLB_OK. */
vlb_status vlb_synchronize(vlb_handle* h);

/* Number of completed time steps in *n (after the queued work finishes). */
vlb_status vlb_get_step(vlb_handle* h, int64_t* n);

/* Copy macroscopic fields of the current time level into caller-owned host
 * arrays of nx*ny doubles (row-major, y slow): rho, u_x, u_y, T (Eqs. 9, 25)
 * and the solid fraction f_s.  Only arrays whose VLB_FIELD_* bit is set in
 * mask are written; the others may be NULL. */
vlb_status vlb_get_fields(vlb_handle* h, uint32_t mask, double* rho, double* ux, double* uy,
                          double* T, double* fs);

/* Copy the state of the first n particles (n <= count): centres xy[2n],
 * orientation theta[n], velocity uv[2n], angular velocity omega[n], and the
 * total force force[2n] and torque torque[n] (F_c, T_c of Eq. 26) that
 * produced the current velocities.  Any pointer may be NULL. */
vlb_status vlb_get_particle_state(vlb_handle* h, int32_t n, double* xy, double* theta, double* uv,
                                  double* omega, double* force, double* torque);

/* The same read without waiting for the GPU: vlb_particle_state_async queues
 * a copy of the first n particles' state at the current level (after the
 * work already queued on the handle's stream) into one of two
 * library-owned pinned buffers and returns; vlb_particle_state_wait blocks
 * until the oldest queued copy has arrived and writes it out like
 * vlb_get_particle_state (any array may be NULL; n must equal the queued
 * copy's), with the step number of its level in *step (may be NULL).  A
 * caller that queues a copy after each vlb_step and collects it after the
 * next one reads every step's result while the GPU runs the next step.
 * VLB_ESTATE when two copies are pending (async) or none is (wait);
 * VLB_EINVAL for a bad n; device flags as vlb_step returns them. */
vlb_status vlb_particle_state_async(vlb_handle* h, int32_t n);
vlb_status vlb_particle_state_wait(vlb_handle* h, int32_t n, double* xy, double* theta, double* uv, double* omega,
                                   double* force, double* torque, int64_t* step);

/* Number of particles in *n. */
vlb_status vlb_get_particle_count(vlb_handle* h, int32_t* n);

/* FP64 audits of the stored post-collision state: total mass sum_x sum_i f_i,
 * total internal energy sum_x eps of the current level, and sum_x sum_i g_i.
 * Any pointer may be NULL.  Sets VLB_EUNSTABLE if a population is NaN. */
vlb_status vlb_get_audit(vlb_handle* h, double* total_mass, double* total_eps, double* total_g);

/* Solid-fraction ownership of the current level (Sec. 2; integer part exact):
 * count[nx*ny] owners per cell; owner[4*nx*ny] particle ids in ascending
 * order, -1 padded; flag[4*nx*ny] 1 = interface, 2 = solid, 0 padded;
 * fsp[4*nx*ny] per-owner fractions.  Arrays may be NULL. */
vlb_status vlb_get_solid_fraction(vlb_handle* h, uint8_t* count, int32_t* owner, uint8_t* flag,
                                  double* fsp);

/* Allocation-free variant of vlb_get_solid_fraction (the paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory during a run -- e.g. while a caching allocator or memory pool owns
 * the device, or where cudaMalloc/cudaFree would synchronise the device).
 * Same outputs as vlb_get_solid_fraction, but the dump's scratch lives in one
 * static device array of the library instead of cudaMalloc'd buffers.
 *   - At most VLB_NOALLOC_MAX_CELLS cells; a larger lattice gives VLB_EINVAL.
 *   - The handle must already hold its initial state (vlb_step(h, 0) or any
 *     step), because building it allocates: otherwise VLB_ESTATE.
 *   - Every GPU that loads the library holds the array (about 3.5 MB) until
 *     the process exits; all calls share it and it keeps the last call's
 *     contents (each call overwrites everything it reads back).
 *   - Calls that overlap on the GPU race on the array: serialise them.
 *   - The first call on a device looks the array up with
 *     cudaGetSymbolAddress; make it before any stream capture.
 *   - The device that was current at vlb_create must be current at the call
 *     (the array's address is per device): otherwise VLB_EINVAL. */
#define VLB_NOALLOC_MAX_CELLS 65536
vlb_status vlb_get_solid_fraction_noalloc(vlb_handle* h, uint8_t* count, int32_t* owner, uint8_t* flag,
                                          double* fsp);

/* Contact pair list of the current level: pairs (i, j), i < j, with
 * |X_i - X_j| < R_i + R_j + zeta, in ascending (i, j) order, written as
 * pairs[2k], pairs[2k+1] for k < min(*npairs, capacity).  *npairs receives
 * the total number of pairs. */
vlb_status vlb_get_contact_pairs(vlb_handle* h, int32_t capacity, int32_t* pairs, int32_t* npairs);

/* Checkpoint and resume.  The state of a run after time step n (Sec. 2: the
 * post-collision populations f-bar and g-bar, the S plane of Eq. 24, and the
 * particle state of Sec. 2.3 with the exchange sums, contact lists and tile
 * lists of that level) as one host image that continues the run bit for bit.
 *   vlb_state_size: *bytes receives the image size of h (initialising h if
 *     it has not stepped yet).
 *   vlb_save_state: writes the image into the caller's host buffer of at
 *     least that many bytes (synchronises the handle's stream).
 *   vlb_load_state: restores an image into h, which must have been created
 *     with the same parameters and given the same number of particles (their
 *     positions and properties come from the image); afterwards vlb_step,
 *     vlb_get_fields and the other calls continue from the saved level.
 *     VLB_EINVAL if the image is not one of this library version or belongs
 *     to a handle of other sizes, precision or particle count.
 * The image holds device data of this build (storage type, tile height); it
 * is not a portable file format. */
vlb_status vlb_state_size(vlb_handle* h, uint64_t* bytes);
vlb_status vlb_save_state(vlb_handle* h, void* buf, uint64_t bytes);
vlb_status vlb_load_state(vlb_handle* h, const void* buf, uint64_t bytes);

/* Measurement hooks.  Between begin and end, each step records CUDA events
 * around its lattice kernel on the handle's stream.  end() returns the summed
 * lattice-kernel time in ms, the number of timed launches, and the number of
 * kernel launches each step issues. */
vlb_status vlb_profile_begin(vlb_handle* h, int32_t max_steps);
vlb_status vlb_profile_end(vlb_handle* h, double* lattice_ms, int32_t* lattice_launches,
                           int32_t* launches_per_step);

/* Description of the last failure on h (or of a failed vlb_create when h is
 * NULL).  The string stays valid until the next call on the same handle. */
const char* vlb_last_error(const vlb_handle* h);

/* Free every resource of h (NULL is ignored). */
void vlb_destroy(vlb_handle* h);

/* Device bytes that a handle of parameters p allocates for n particles of
 * the given radii (create, particles and first step; rows padded to 32 B,
 * band tables sized by the largest radius).  VLB_EINVAL for inconsistent
 * parameters, as vlb_create would return it. */
vlb_status vlb_device_bytes(const vlb_params* p, int32_t n, const double* radius, uint64_t* bytes);

/* ---- Served mode ----------------------------------------------------------
 * Independent cases (each a vlb_params block, its particles and a number of
 * steps) are submitted as they arrive.  Each vlb_serve_poll call is one
 * round: every resident case advances by the same number of steps with one
 * vlb_step_batch call (at most steps_per_round, and at most what the nearest
 * case still needs); while the GPU runs it, queued cases are admitted first
 * come first served while their vlb_device_bytes fit in the HBM budget (and
 * under max_active) and join the next round; then the cases that have done
 * their steps are read back (fields and particle state into host memory),
 * freed, and their time to result recorded.  A case advances bit for bit as it would alone with
 * vlb_step.  All resident cases run on the server's own CUDA stream.  One
 * host thread per server.  Not part of the paper: it serves the paper's
 * time step to a stream of cases. */
typedef struct vlb_server vlb_server;

typedef struct {
  uint64_t hbm_budget;      /* device bytes for resident cases (0: half of the free device memory at creation) */
  int32_t steps_per_round;  /* most steps between two admission points (0: 100) */
  int32_t max_active;       /* most resident cases (0: no limit) */
} vlb_serve_params;

typedef enum { VLB_CASE_QUEUED = 0, VLB_CASE_ACTIVE = 1, VLB_CASE_DONE = 2, VLB_CASE_FAILED = 3 } vlb_case_state;

/* Defaults: budget 0 (half of free memory), 100 steps per round, no limit on resident cases. */
vlb_status vlb_serve_params_default(vlb_serve_params* sp);

/* A server (no device memory yet beyond its stream).  VLB_EINVAL for
 * negative fields, VLB_ENOMEM, VLB_ECUDA. */
vlb_status vlb_serve_create(const vlb_serve_params* sp, vlb_server** out);

/* Queue a case: parameters p (copied), n particles as in vlb_add_particles
 * (xy[2n], radius[n], T0[n], k_ratio[n] or NULL; copied), nsteps time
 * steps.  *id receives the case id.  VLB_EINVAL for bad arguments or
 * parameters (n > p->max_particles included), VLB_ENOMEM when the case alone
 * exceeds the HBM budget.  Disk placement errors surface at admission, as a
 * failed case. */
vlb_status vlb_serve_submit(vlb_server* s, const vlb_params* p, int32_t n, const double* xy, const double* radius,
                            const double* T0, const double* k_ratio, int64_t nsteps, int64_t* id);

/* One round (see above); afterwards the numbers of queued, resident and
 * finished (done or failed, not yet taken) cases, each pointer may be NULL.
 * A case whose step fails (VLB_EUNSTABLE, VLB_EOVERFLOW) becomes
 * VLB_CASE_FAILED and the others go on; VLB_ECUDA ends the round with the
 * server's error. */
vlb_status vlb_serve_poll(vlb_server* s, int32_t* nqueued, int32_t* nactive, int32_t* ndone);

/* State (vlb_case_state), lattice size, particle count and times (seconds
 * since the server's creation: times[0] submitted, [1] admitted, [2]
 * finished with its result in host memory) of a case not yet taken. */
vlb_status vlb_serve_case_info(vlb_server* s, int64_t id, int32_t* state, int32_t* nx, int32_t* ny, int32_t* n,
                               double* times);

/* The result of a finished case, then forgotten: the five fields as
 * vlb_get_fields writes them (nx*ny each, any may be NULL) and the particle
 * state [n][9] = x, y, theta, ux, uy, omega, F_x, F_y, T (may be NULL).  A
 * failed case returns its failure (vlb_serve_last_error describes it) and is
 * forgotten too; VLB_ESTATE for a case still queued or running. */
vlb_status vlb_serve_take(vlb_server* s, int64_t id, double* rho, double* ux, double* uy, double* T, double* fs,
                          double* pstate);

/* Description of the server's last failure (of a failed vlb_serve_create when s is NULL). */
const char* vlb_serve_last_error(const vlb_server* s);

/* Free the server and every resident case (NULL is ignored). */
void vlb_serve_destroy(vlb_server* s);

#ifdef __cplusplus
}
#endif

#endif /* VLB_H */
