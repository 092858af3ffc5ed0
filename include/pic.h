/*
 * pic.h -- C ABI of the GB300 (sm_103a) explicit electromagnetic particle-in-cell step in
 * a Lorentz-boosted frame (Vay, Fawley, Geddes, Cormier-Michel, Grote, "Speeding up
 * simulations of relativistic systems using an optimal boosted frame", arXiv:0909.5603).
 *
 * The calls follow the paper's statement of the problem (Sec. 2): inputs are given in
 * the laboratory frame and transformed into the boosted frame (pic_load_lab_frame); the
 * relativistic PIC loop -- field gather, Vay (or Boris) push, charge-conserving current
 * deposit, low-pass binomial filtering of the current, Yee Maxwell update -- evolves the
 * system in the boosted frame (pic_step); results are read back (pic_get_*).
 *
 * Conventions, for every call:
 *  - Normalised units: c = eps0 = 1.  The species charge q and mass m are options
 *    (default electrons, q = -1, m = 1).  Boost along +z.
 *  - Every call returns pic_status; no C++ exception crosses the ABI.  After a non-OK
 *    status, pic_last_error() describes it.
 *  - The library owns all device memory of a context (obtained through the allocator
 *    given in pic_options, or cudaMalloc).  The caller owns every host buffer passed in;
 *    getters copy into it and check its size (count / cap) first (PIC_ERR_ARG if short).
 *  - Getters return FP64 whatever the storage precision (widening is exact).
 *  - Work is issued on the context's stream (pic_options.stream).  pic_step is
 *    asynchronous; getters synchronise the stream.  A device-side error word (e.g. a
 *    bounded wait that timed out, a particle faster than one cell per step) is sticky and
 *    reported by the next synchronising call.
 *  - A context is thread-compatible, not thread-safe.
 *  - Grid arrays exchanged with the host are n0 * n1 * n2 doubles, x fastest, with the
 *    Yee staggering: Ex[i,j,k] at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2),
 *    Bx at (i, j+1/2, k+1/2), By at (i+1/2, j, k+1/2), Bz at (i+1/2, j+1/2, k), J like E,
 *    rho and div E on nodes (i, j, k).
 *  - 2D3V (ndim = 2) is the x-z plane: n[1] must be 1, y is invariant, all three field
 *    and momentum components are kept.
 *  - Particles: int32 linear cell index c = i + n0 (j + n1 k) and in-cell offsets in
 *    [0, 1) per axis (3 doubles per particle, the y offset is 0 in 2D), momenta
 *    u = gamma v (3 doubles), weight w (physical particles per macro-particle), optional
 *    int32 id carried along unchanged.
 *  - Particle order: after every load and every step the particles are kept in the
 *    canonical order -- a stable sort by tile id (tile coordinates lexicographic, z
 *    slowest) of the previous order; getters return them in that order.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,            /* invalid argument, size or pointer */
    PIC_ERR_CFL = 2,            /* dt above the field solver's Courant limit */
    PIC_ERR_CUDA = 3,           /* a CUDA runtime or driver call failed */
    PIC_ERR_OOM = 4,            /* the allocator returned no memory */
    PIC_ERR_STATE = 5,          /* call not valid in this state (e.g. step before load) */
    PIC_ERR_PARTICLE_SPEED = 6, /* device: a particle moved a cell or more, or became NaN */
    PIC_ERR_TIMEOUT = 7,        /* device: a bounded wait gave up */
    PIC_ERR_NAN = 8,            /* non-finite value in a host input */
    PIC_ERR_UNSUPPORTED = 9,    /* valid request this build does not implement */
    PIC_ERR_INTERNAL = 10       /* device: an internal consistency check failed */
} pic_status;

enum { PIC_PERIODIC = 0, PIC_ABSORBING = 1 };
enum { PIC_PREC_FP32 = 0, PIC_PREC_FP64 = 1 };
enum { PIC_PUSHER_VAY = 0, PIC_PUSHER_BORIS = 1 };
enum { PIC_SOLVER_YEE = 0, PIC_SOLVER_CK = 1 };
enum {
    PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ,
    PIC_RHO = 9, /* charge density on the nodes: particles + ion background (getter only) */
    PIC_DIVE = 10 /* discrete divergence of E on nodes (getter only) */
};
enum { PIC_PHASE_PARTICLES = 1, PIC_PHASE_FILTER = 2, PIC_PHASE_MAXWELL = 4, PIC_PHASE_ALL = 7 };

typedef struct {
    int ndim;  /* 2 (x-z plane, n[1] = 1) or 3 */
    int n[3];  /* cells per axis */
    int bc[3]; /* PIC_PERIODIC or PIC_ABSORBING per axis (fields and particles) */
} pic_grid;

/* Device allocator hooks: return a device pointer of at least `bytes` bytes aligned to
 * 256 bytes, or NULL; free it.  Both are called only from pic_create, pic_load_* and
 * pic_destroy / pic_batch_*. */
typedef void *(*pic_alloc_fn)(size_t bytes, void *user);
typedef void (*pic_free_fn)(void *ptr, void *user);

typedef struct {
    int precision;          /* PIC_PREC_FP32: FP32 particles, fields and deposits, FP64
                               only in the Vay gamma solve and the diagnostics sums;
                               PIC_PREC_FP64: everything FP64 */
    int pusher;             /* PIC_PUSHER_VAY (default) or PIC_PUSHER_BORIS */
    int filter_passes;      /* binomial 1-2-1 passes on J per step, 0..8 (0 = none) */
    int tile[3];            /* particle tile in cells; 0 = default (8^3 in 3D, 16x1x16 in
                               2D); tile[0] must be a multiple of 4 */
    int threads;            /* threads per particle CTA: 0 = this build's size (256), or
                               that size given explicitly (others: PIC_ERR_UNSUPPORTED) */
    int absorb_cells;       /* width L of the absorbing layer (default 16) */
    double absorb_strength; /* per-step damping 1 - s (d/L)^2 at depth d (default 0.1) */
    double charge, mass;    /* species charge and mass (default -1, 1) */
    int track_ids;          /* carry an int32 id per particle (default 1) */
    pic_alloc_fn alloc;     /* NULL: cudaMalloc */
    pic_free_fn free;       /* NULL: cudaFree */
    void *alloc_user;
    void *stream;           /* cudaStream_t used for all work; NULL = legacy stream */
    int device;             /* CUDA device ordinal (default: the current device) */
    int solver;             /* PIC_SOLVER_YEE (default): the Yee scheme, Courant limit
                               1 / sqrt(sum_a 1/dx_a^2).  PIC_SOLVER_CK: the low-dispersion
                               solver Sec. 2 uses against the boosted-frame instability
                               (after Karkkainen et al.): every difference of the Faraday
                               update averaged over its transverse neighbours, 7/12 on
                               itself, 1/12 on the four edge and 1/48 on the four corner
                               neighbours (3/4, 1/8 in 2D3V); dispersion-free along the axis
                               of the smallest cell at dt equal to it, Courant limit
                               min_a dx_a.  Ampere's law keeps the Yee differences. */
    int absorb_faces;       /* which faces of absorbing axes carry the damping layer: bit 2a
                               the lower face of axis a, bit 2a+1 the upper one (default
                               0x3F, all).  A face without its bit stays absorbing for
                               particles and zero beyond, undamped: the inner face of a slab
                               whose neighbour slab supplies the field (pic_put_planes). */
} pic_options;

typedef struct {
    int64_t step;          /* steps taken since the last load */
    double t;              /* boosted-frame time step * dt */
    double field_energy;   /* (1/2) sum (E^2 + B^2) dV over the cells, FP64 sum */
    double kinetic_energy; /* sum w m (gamma - 1) over particles, FP64 sum */
    double total_charge;   /* sum q w over particles (ion background excluded), FP64 sum */
    int64_t n_particles;   /* live macro-particles */
    int64_t n_lost;        /* macro-particles removed at absorbing boundaries */
    int32_t error_flags;   /* sticky device error word (0 = none) */
} pic_diag;

/* Per-phase device time accumulated while profiling is on (CUDA events on the
 * context's stream around each kernel; see pic_set_profiling). */
typedef struct {
    int64_t steps;
    double ms_particles; /* fused gather + push + deposit + reorder kernel */
    double ms_scan;      /* tile population scan */
    double ms_filter;    /* current filter */
    double ms_maxwell;   /* Yee B/E/B (+ absorbing layer, ghost exchange) */
    double ms_other;     /* J clear and step bookkeeping */
    int64_t launches;    /* kernels launched by the profiled steps */
} pic_timings;

/* Fills *o with the defaults listed above. */
void pic_default_options(pic_options *o);

/* Creates a simulation instance on a boosted-frame grid.
 *  grid: dimensions and boundaries; dx: cell sizes (> 0); dt: time step, at most the
 *  field solver's Courant limit over the active axes, 1 / sqrt(sum_a 1/dx_a^2) for Yee,
 *  min_a dx_a for PIC_SOLVER_CK (else PIC_ERR_CFL);
 *  gamma_boost >= 1: Lorentz factor of the boosted frame relative to the lab (Sec. 2),
 *  used by pic_load_lab_frame; shape_order: 1 (linear) or 2 (quadratic) particle shape
 *  for gather and deposit; opt: NULL for defaults.  Periodic axes need at least 3 tiles
 *  unless they hold a single tile.  On success *out owns the instance (free with
 *  pic_destroy).  Fields start at zero, no particles. */
pic_status pic_create(const pic_grid *grid, const double dx[3], double dt, double gamma_boost,
                      int shape_order, const pic_options *opt, pic_ctx **out);

/* Frees the instance (or a batch, which does not free its members).  NULL is a no-op. */
void pic_destroy(pic_ctx *ctx);

/* Human-readable description of the last non-OK status on ctx (or of the last failed
 * pic_create when ctx is NULL).  Valid until the next call on ctx. */
const char *pic_last_error(const pic_ctx *ctx);

/* Laboratory-frame inputs (Sec. 2).  Box coordinates: x in [0, n0 dx0), y in [0, n1 dx1),
 * z' in [0, n2 dx2) at boosted time t' = 0; lab z = 0 coincides with z' = 0 at t = t' = 0. */
typedef struct {
    double a0;       /* normalised peak vector potential (invariant) */
    double lambda0;  /* lab wavelength */
    double waist;    /* 1/e field radius (invariant), centred on the box axis */
    double duration; /* 1/e half-length of the field envelope, lab (c tau) */
    double z_center; /* lab position of the envelope centre at lab time 0 */
} pic_laser_lab;     /* linearly polarised along x, propagating along +z, no curvature */

typedef struct {
    double n0;       /* lab electron density for z >= z_start + ramp_len */
    double z_start;  /* lab position where the density starts */
    double ramp_len; /* lab length of the linear up-ramp (0 = step) */
    int ppc;         /* macro-particles per cell */
    double u_th[3];  /* lab thermal momentum spread per axis (0 = cold) */
    uint64_t seed;
} pic_plasma_lab;

typedef struct {
    int64_t n;           /* macro-particles */
    double gamma;        /* lab Lorentz factor of the beam centroid (> 1) */
    double rel_spread;   /* isotropic momentum spread / (gamma beta) */
    double sigma_r;      /* lab rms transverse size, centred on the box axis */
    double sigma_z;      /* lab rms length */
    double z0;           /* lab centroid position at lab time 0 */
    double total_weight; /* physical particles in the beam */
    uint64_t seed;
} pic_beam_lab;

/* Replaces the state with lab-frame inputs transformed to the boosted frame (Sec. 2):
 * laser Doppler-shifted (wavelength and length x gamma(1+beta), a0 and waist invariant,
 * E'x = B'y), plasma at lab rest drifting at -beta with density gamma n0, beam
 * particles boosted then drifted ballistically to t' = 0.  Host FP64, seeded with
 * SplitMix64 (counter-based); particles falling outside the box are dropped.  Any of
 * the three may be NULL.  Resets step count, J and the lost counter.
 * Ion background: the plasma's ions are at rest in the lab frame, so they are not
 * macro-particles but a rigid charge density of the opposite charge, the lab profile
 * contracted by gamma_b, filling the loaded box at t' = 0 and streaming at -beta_b
 * (wrapping when z is periodic, leaving through the -z face when absorbing).  Every
 * step adds their current on the Jz faces -- the charge of the profile crossing each
 * face during the step, over dt -- and PIC_RHO adds their charge on each node's dual
 * cell, so div E - rho stays constant for the ions too.
 * Beam self-field: a beam enters with the field of its own charge moving rigidly at its
 * centroid velocity in this frame (beta', gamma'), the field whose action on the beam
 * itself Sec. 2 discusses: phi from phi_xx + phi_yy + phi_zz / gamma'^2 = -rho (rho on
 * the nodes with the particle shape; phi = 0 one node beyond absorbing faces, periodic
 * axes wrap; on an all-periodic grid the mean charge is dropped), solved exactly on the
 * host in FP64; E = -(phi_x, phi_y, phi_z / gamma'^2) at the Yee positions and
 * B = beta' z x E (E averaged over the two z nodes around B's half-integer z). */
pic_status pic_load_lab_frame(pic_ctx *ctx, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                              const pic_beam_lab *beam);

/* Replaces the particles with n host particles (exact-input path).  cell[n]; off3[3n]
 * in [0,1) (PIC_ERR_ARG otherwise); u3[3n]; w[n]; id[n] or NULL (ids 0..n-1).  The
 * library sorts them into the canonical order.  Clears any ion background. */
pic_status pic_load_particles(pic_ctx *ctx, int64_t n, const int32_t *cell, const double *off3,
                              const double *u3, const double *w, const int32_t *id);

/* pic_load_particles with the values in the context's storage precision: off3, u3 and w
 * are float arrays for a PIC_PREC_FP32 context and double arrays for PIC_PREC_FP64 (then
 * the call is pic_load_particles).  The particles of Sec. 2 as the step stores them, so
 * an FP32 run moves and checks half the bytes on the host and places the values as they
 * are (an offset must lie in [0,1) as a float).  Same layout, validation and errors as
 * pic_load_particles; the arrays stay the caller's (page-locked host memory, e.g. from
 * cudaHostAlloc, copies at the link's full rate). */
pic_status pic_load_particles_stored(pic_ctx *ctx, int64_t n, const int32_t *cell, const void *off3,
                                     const void *u3, const void *w, const int32_t *id);

/* Overwrites one field component (PIC_EX .. PIC_JZ) with count = n0 n1 n2 host values. */
pic_status pic_set_field(pic_ctx *ctx, int comp, const double *host, size_t count);

/* Advances n >= 0 steps of the relativistic PIC loop in the boosted frame (Sec. 2: field
 * gather, Vay or Boris push, charge-conserving current deposit, binomial filtering of the
 * current, Yee Maxwell update; plus the ion background's current, the stations, the
 * antenna and the injection plane when set).  Asynchronous; the step is replayed from a
 * CUDA graph captured on first use unless profiling is on.  A device error of a step
 * (PIC_ERR_PARTICLE_SPEED, PIC_ERR_TIMEOUT, ...) is reported by the next synchronising
 * call.  PIC_ERR_STATE before any load; PIC_ERR_ARG for n < 0. */
pic_status pic_step(pic_ctx *ctx, int n);

/* Runs the selected phases (PIC_PHASE_* mask) of one step, for unit testing a phase in
 * isolation; a full step is PIC_PHASE_ALL. */
pic_status pic_run_phases(pic_ctx *ctx, int phase_mask);

/* Copies one component (PIC_EX .. PIC_JZ, PIC_RHO, PIC_DIVE) of the boosted-frame grid
 * (Sec. 2: the fields the boosted-frame PIC loop evolves, before any transform back to
 * the lab, which the stations do) into host_out[count], count >= n0 n1 n2, FP64, in the
 * staggered layout above.  J is the current used by the last Maxwell update (after the
 * filter).  PIC_RHO deposits the particles' charge with their shape (plus the ion
 * background) into per-context FP64 memory; PIC_DIVE is the node divergence of E.
 * Synchronises; PIC_ERR_ARG for an unknown component or a short buffer. */
pic_status pic_get_field(pic_ctx *ctx, int comp, double *host_out, size_t count);

/* Copies ncomp components (as for pic_get_field, Sec. 2) into
 * host_out[ncomp][n2][n1][n0], count >= ncomp n0 n1 n2; comps[i] as pic_get_field.
 * Synchronises; PIC_ERR_ARG for an unknown component, ncomp < 1 or a short buffer. */
pic_status pic_get_fields(pic_ctx *ctx, const int *comps, int ncomp, double *host_out, size_t count);

/* Gauss-law residual on the nodes: *max_abs = max |div E - rho| and, when rms is not NULL,
 * *rms = sqrt(mean (div E - rho)^2), with div E and rho (particles and ion background)
 * as PIC_DIVE and PIC_RHO, in FP64 on the device.  The Esirkepov deposit keeps div E - rho
 * constant in time when the current is not filtered (with the binomial filter on, div E -
 * F rho is the constant one, F the same passes on the nodes).  Synchronises; device
 * memory for one n0 n1 n2 array of doubles during the call. */
pic_status pic_get_gauss_residual(pic_ctx *ctx, double *max_abs, double *rms);

/* Number of live particles (synchronises). */
pic_status pic_num_particles(pic_ctx *ctx, int64_t *n_out);

/* Copies the live macro-particles of the boosted frame (Sec. 2: the plasma and beam
 * particles the PIC loop pushes), in canonical order, into host arrays with room for cap
 * particles (any pointer may be NULL to skip that array); *n_out = count.  Layout as in
 * the conventions above (cell int32, off3/u3 3 doubles per particle, w, id int32 -- ids
 * are int32 like the cell index: a context holds fewer than 2^31 particles).
 * Synchronises; PIC_ERR_ARG when cap is below the count (*n_out still set).  The first
 * call allocates a device staging buffer (9 values per particle of capacity) that the
 * context keeps. */
pic_status pic_get_particles(pic_ctx *ctx, int32_t *cell, double *off3, double *u3, double *w,
                             int32_t *id, int64_t cap, int64_t *n_out);

/* pic_get_particles (the Sec. 2 macro-particles, canonical order) with the values in the
 * storage precision: off3, u3 and w receive floats for a PIC_PREC_FP32 context (no
 * widening on the host; the FP64 values pic_get_particles returns are exactly these
 * widened) and doubles for PIC_PREC_FP64.  Same layout, cap rule, errors and staging
 * buffer as pic_get_particles; into page-locked host memory the copies run at the
 * link's full rate. */
pic_status pic_get_particles_stored(pic_ctx *ctx, int32_t *cell, void *off3, void *u3, void *w, int32_t *id,
                                    int64_t cap, int64_t *n_out);

/* FP64 global diagnostics of the boosted frame, computed on the device and copied to
 * *out: field energy sum (E^2 + B^2) dV / 2, particles' kinetic energy sum w (gamma - 1)
 * m, total charge, live and removed particle counts, step and time.  The paper judges
 * its runs by the energy they reach (Sec. 3.1) and the boosted-frame instability by the
 * growth of the field (Sec. 2); error_flags holds the sticky device error word.
 * Synchronises. */
pic_status pic_get_diagnostics(pic_ctx *ctx, pic_diag *out);

/* Profiling: when on, pic_step launches each kernel directly (no graph) between CUDA
 * events on the context's stream and accumulates per-phase device time; reset clears the
 * sums.  pic_get_timings synchronises and returns the sums. */
pic_status pic_set_profiling(pic_ctx *ctx, int on, int reset);
pic_status pic_get_timings(pic_ctx *ctx, pic_timings *out);

/* Waits for all work of ctx; reports a sticky device error. */
pic_status pic_synchronize(pic_ctx *ctx);

/* Batching of independent boosted-frame instances (the paper has no counterpart; it
 * serves scans over the boost, the parameter Sec. 1 ties the speed-up to).  Groups n >= 1
 * instances created with identical ndim, shape order, precision, pusher, field solver,
 * tile, threads and device into a batch whose pic_step advances all of them in one
 * launch per phase (one flattened tile list over all instances), captured in one graph.
 * The members keep their own memory and stay readable with the getters; destroy the
 * batch before its members.  Only pic_step, pic_run_phases, pic_synchronize,
 * pic_set_profiling, pic_get_timings and pic_destroy accept a batch. */
pic_status pic_batch_create(int n, pic_ctx *const *instances, pic_ctx **batch);

/* Persistent batched step (the paper has no counterpart; it serves the batch above).
 * With on = 1, every later pic_step(batch, n) runs its n steps in ONE launch of a
 * persistent kernel: CTAs pull (step, phase, instance, item) work items from a device
 * list and each item waits only until its own instance has completed its previous phase,
 * so the instances of an uneven batch do not wait for one another at phase boundaries.
 * Each wait is bounded by spin_limit polls (<= 0: 2^21, about a second); a wait that
 * gives up sets PIC_ERR_TIMEOUT on its instance (reported by the next synchronising
 * call) and ends the launch.  test_stall >= 0 makes that instance's J set-up wait for an
 * item that never runs, to exercise the timeout (-1: off).  Members must be FP32, Vay,
 * Yee, with one filter pass count <= 4 and no antenna, injection plane or stations (else
 * PIC_ERR_UNSUPPORTED); pic_run_phases and profiled steps keep the per-phase launches.
 * on = 0 returns to the per-phase CUDA graph.  Not valid on a member (PIC_ERR_ARG). */
pic_status pic_batch_set_persistent(pic_ctx *batch, int on, long long spin_limit, int test_stall);

/* Online choice of the batch's launch form (the paper has no counterpart): runs one
 * untimed and `steps` >= 1 timed steps with the per-phase CUDA graph, then the same with
 * the persistent step when the batch admits it (pic_batch_set_persistent), and leaves
 * the faster form on.  The 2 (steps + 1) steps are real steps of the run.  Reports the
 * choice (*persistent, may be NULL) and the milliseconds per step of each form (-1 for
 * a form not run; may be NULL).  Not valid on a member (PIC_ERR_ARG) or with profiling
 * on (PIC_ERR_STATE); a device error of a step is returned as pic_step's would be. */
pic_status pic_batch_autotune(pic_ctx *batch, int steps, int *persistent, double *ms_graph, double *ms_persistent);

/* Lab-frame stations (Sec. 2: the results are recorded at planes immobile in the
 * laboratory frame and transformed back to it).  Replaces the stations with `count`
 * planes z = z_lab[i] (lab coordinates; lab and boosted frames share their origin at
 * t = t' = 0, boost along +z), each holding up to max_records records (count = 0 removes
 * them).  At boosted time t' a plane sits at z' = z_lab / gamma_b - beta_b t'; after the
 * load or pic_set_stations, and after every full step (pic_step, or pic_run_phases with
 * PIC_PHASE_ALL), every station whose plane lies in the box records: each field
 * component at its own transverse Yee position, interpolated linearly in z' between the
 * two planes of its z stagger (zero beyond an absorbing face, wrapped on a periodic
 * axis), transformed back to the lab frame (E_x = g (E'_x + b B'_y), E_y = g (E'_y -
 * b B'_x), B_x = g (B'_x - b E'_y), B_y = g (B'_y + b E'_x), z components unchanged), with
 * its lab time t'/gamma_b + beta_b z_lab.  FP64 arithmetic, stored in the working
 * precision.  A new load restarts every station's history.  Device memory: 6 n0 n1
 * values per record.  Not valid on a batch (PIC_ERR_ARG). */
pic_status pic_set_stations(pic_ctx *ctx, int count, const double *z_lab, int max_records);

/* Copies station `station`'s history: *n_records; t_lab[n_records] (may be NULL, else
 * t_count >= n_records); fields[n_records][6][n1][n0] as Ex Ey Ez Bx By Bz (may be NULL,
 * else f_count >= n_records 6 n0 n1).  Synchronises. */
pic_status pic_get_station(pic_ctx *ctx, int station, int *n_records, double *t_lab, size_t t_count, double *fields,
                           size_t f_count);

/* Laser antenna on a plane fixed in the laboratory (Sec. 2: the laser enters through a
 * plane fixed in the lab frame that drifts in the boosted frame).
 *  laser: the lab pulse (as for pic_load_lab_frame; z_center = where its envelope centre
 *    would be at lab time 0 had it always propagated freely), or NULL to remove the
 *    antenna.  z_lab: the plane's lab position; at boosted time t' it sits at
 *    z' = z_lab / gamma_b - beta_b t' (t' = dt x Maxwell phases since the load).
 * The plane emits the pulse forward: downstream of it the field includes the free pulse,
 * upstream it does not.  The grid is split at the plane into a total-field region (z
 * positions above the plane's position at the time of the fields) and a scattered-field
 * region (the field minus the incident pulse); the incident pulse E'_x = B'_y =
 * exp(-(x^2 + y^2) / w0^2) g(z', t') is carried on a 1D lattice aligned with the grid's z
 * lattice and advanced by the same leapfrog, so a plane wave crosses the moving boundary
 * without reflection.  Each Maxwell phase adds the incident term to the B_y and E_x
 * differences that straddle the plane (7 small launches) and moves the values the
 * receding plane passed into the total field; under the low-dispersion solver
 * (PIC_SOLVER_CK) the averaged Faraday differences spread the B_y term over the
 * neighbouring columns and add a B_z term at the nodes on either side of the plane (3D).
 * The call adds the incident field downstream of the plane now.  Needs a loaded state
 * (else PIC_ERR_STATE) and an absorbing z axis (else PIC_ERR_ARG); not valid on a batch
 * (PIC_ERR_ARG), but a batch steps its members' antennas.  A load removes the antenna.  Device memory: two
 * doubles per lattice node (the box, the pulse's extent upstream and the distance light
 * covers while the plane crosses the box). */
pic_status pic_set_laser_antenna(pic_ctx *ctx, const pic_laser_lab *laser, double z_lab);

/* Beam injection through a plane fixed in the laboratory (Sec. 2: the beam enters the
 * boosted frame through a transverse lab-fixed plane that drifts in this frame; the beam
 * still upstream of it is carried by frozen, drifting macro-particles).
 *  enable: 1 sets the plane, 0 removes it (z_lab and first_id ignored).
 *  z_lab: lab position of the plane (finite); at boosted time t' it sits at
 *    z' = z_lab / gamma_b - beta_b t'.
 *  first_id: particles with id >= first_id are beam particles; first_id < 0 selects the
 *    beam of the last pic_load_lab_frame (its ids follow the plasma's; no beam there:
 *    no particle is frozen).
 * At each particle phase (push time t^n = n dt, n = particle phases since the load), a
 * beam particle whose z position in cells, k + offset, is below (z_lab / gamma_b -
 * beta_b t^n) / dz (both in FP64) is frozen for that phase: no field acts on it (its
 * momentum stays bit for bit), it moves at its own velocity and deposits its current like
 * any particle, so the space charge of the beam upstream of the plane is present.
 * Downstream of the plane it is pushed as usual.  With a lab beam drifting freely
 * upstream of z_lab this reproduces the lab history: the frozen worldline is the lab one.
 * The setting persists across loads.  Needs particle ids (track_ids; else
 * PIC_ERR_STATE); not valid on a batch (PIC_ERR_ARG); z_lab not finite: PIC_ERR_ARG. */
pic_status pic_set_injection(pic_ctx *ctx, int enable, double z_lab, int32_t first_id);

/* Autotuner: picks the particle tile shape for a workload by measurement (the paper has
 * no counterpart; it tunes this implementation).  For every candidate tile (3D: 8^3,
 * 16x8x8, 8x8x16, 8x16x8, 16x16x4, 16x8x4, 8x8x4, 4x8x8, 16x16x8, 32x8x4; 2D: 16x16,
 * 32x8, 8x32, 32x16, 16x32, 32x32, 64x8) it creates a context with `base` (NULL =
 * defaults) and that tile, loads the lab-frame inputs, runs 2 warm-up steps, times
 * `steps` >= 1 steps with the library's per-phase CUDA events and destroys it.  The
 * fastest candidate's options go to *best (its tile set, everything else from base) and
 * its time per step (ms, all phases) to *ms_per_step (may be NULL).  Candidates that
 * pic_create rejects are skipped; if none runs, the last error is returned.  Device
 * memory for one candidate at a time; a slab of the workload (fewer z cells) gives the
 * same per-particle ranking at a fraction of the cost. */
pic_status pic_autotune(const pic_grid *grid, const double dx[3], double dt, double gamma_boost, int shape_order,
                        const pic_options *base, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                        const pic_beam_lab *beam, int steps, pic_options *best, double *ms_per_step);

/* Domain decomposition along z (the paper needs no change of the PIC code's parallelism
 * in the boosted frame, Sec. 3.2): a slab of a larger grid runs as its own context whose
 * inner z faces are absorbing without a damping layer (pic_options.absorb_faces), carrying
 * ghost planes that a neighbour slab owns.  These calls move z planes of the fields and
 * the particles that left a slab; the exchange schedule is the caller's (the Python
 * module paper_0909_5603_gb300.slab).  The paper has no counterpart for the calls
 * themselves; they are how its unchanged parallel PIC loop maps onto several GPUs.
 *
 * pic_get_planes copies the nk z planes k0 .. k0 + nk - 1 of component comp (PIC_EX ..
 * PIC_BZ, or PIC_JX .. PIC_JZ: the current as pic_get_field reads it, i.e. the deposit
 * after a particle phase, the filtered current once the filter has run) into
 * host_out[nk][n1][n0] (count >= nk n0 n1), FP64.  pic_put_planes overwrites (add = 0) or
 * adds to (add = 1) those planes from host_in; for J it writes the deposit the coming
 * filter phase reads (meaningful between pic_run_phases(PIC_PHASE_PARTICLES) and the
 * filter).  0 <= k0,
 * k0 + nk <= n2, nk >= 1 (else PIC_ERR_ARG).  Both synchronise ctx's stream; device
 * memory: none beyond the context's. */
pic_status pic_get_planes(pic_ctx *ctx, int comp, int k0, int nk, double *host_out, size_t count);
pic_status pic_put_planes(pic_ctx *ctx, int comp, int k0, int nk, const double *host_in, size_t count, int add);
/* The same for ncomp >= 1 components comps[i] at once, host arrays [ncomp][nk][n1][n0]
 * (count >= ncomp nk n0 n1): one copy and one synchronisation per call (per group of
 * components that fit the context's dense scratch of n0 n1 n2 values). */
pic_status pic_get_planes_n(pic_ctx *ctx, const int *comps, int ncomp, int k0, int nk, double *host_out, size_t count);
pic_status pic_put_planes_n(pic_ctx *ctx, const int *comps, int ncomp, int k0, int nk, const double *host_in,
                            size_t count, int add);

/* pic_extract_particles removes the live particles whose z cell index lies outside
 * [k_lo, k_hi) and copies them, in canonical order, into the caller's arrays (layout as
 * pic_get_particles; id may be NULL; room for cap particles, else PIC_ERR_ARG with *n_out
 * set and nothing removed).  pic_add_particles appends n particles (layout as
 * pic_load_particles; id may be NULL when ids are not tracked).  Unlike a load, both keep
 * the step count, the ion background, the antenna, the injection plane and the stations:
 * the particle set changes, the state of the run does not.  Both read the particles out
 * on the device, copy their cells to the host for the canonical order (a stable counting
 * sort by tile) and place the set again on the device; only the particles taken out or
 * added cross to the host in full.  Device memory: a read-out staging copy of the
 * particles (kept for later read-outs) and a map of one int per particle. */
pic_status pic_extract_particles(pic_ctx *ctx, int k_lo, int k_hi, int32_t *cell, double *off3, double *u3, double *w,
                                 int32_t *id, int64_t cap, int64_t *n_out);
pic_status pic_add_particles(pic_ctx *ctx, int64_t n, const int32_t *cell, const double *off3, const double *u3,
                             const double *w, const int32_t *id);

/* pic_adopt_slab makes slab (loaded with its particles) continue the run of whole as the z
 * slab whose plane 0 is plane k_origin of whole (k_origin may be negative or run past
 * whole's planes: positions there are taken in whole's box, wrapped when its z is
 * periodic) and which owns its planes k_lo .. k_hi - 1 (0 <= k_lo < k_hi <= n2; the
 * others are ghosts): it takes over the ion background of whole's lab-frame plasma, in
 * whole's box, with the ions' current deposited on the owned planes only (a ghost plane
 * receives it from its owner), the step count and the phase counter.  Both are 3D
 * members of the same x-y grid, cell size, time step, boost, shape order and precision
 * (else PIC_ERR_ARG); neither carries an antenna, an injection plane or stations
 * (PIC_ERR_STATE).  Fields and particles are moved with the calls above.  Synchronises
 * both streams. */
pic_status pic_adopt_slab(pic_ctx *slab, pic_ctx *whole, int k_origin, int k_lo, int k_hi);

/* Charge density read-out that allocates no device memory.  The paper has no counterpart:
 * this is a service of the library, not a step of the method.
 *
 * Same result as pic_get_field(ctx, PIC_RHO, host_out, count) -- rho on the nodes,
 * n0 n1 n2 doubles, x fastest -- but the deposit goes into a fixed work grid that the
 * library owns (a device array of PIC_NOALLOC_RHO_MAX_CELLS doubles, 8 MiB, present on
 * every GPU on which a context was created, until the process exits) instead of
 * per-context memory.  It is for callers that must not enter a device allocator when they read the
 * density: code running under a device-memory budget that is already fully committed,
 * code called back from inside another library's memory pool, or a tight loop that has
 * to stay out of allocator locks.  The call itself allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine).
 *  - Grids of more than PIC_NOALLOC_RHO_MAX_CELLS cells are rejected with PIC_ERR_ARG.
 *  - CUDA loads the library's code lazily, and loading the part that holds the work grid
 *    allocates it; pic_create does that load on its device, so this call never does.
 *    Each call looks the grid's device address up afresh (cudaGetSymbolAddress, with
 *    ctx's device current).
 *  - Every call shares the one work grid, which keeps the last call's contents; each call
 *    clears the part it uses first.  Calls that overlap on the GPU (several threads or
 *    streams at once) race on it: serialise them.
 *  - Synchronises ctx's stream; host_out as in pic_get_field (count >= n0 n1 n2).
 *  - Not valid on a batch (PIC_ERR_ARG). */
#define PIC_NOALLOC_RHO_MAX_CELLS (1 << 20)
pic_status pic_get_rho_noalloc(pic_ctx *ctx, double *host_out, size_t count);

#ifdef __cplusplus
}
#endif
#endif
