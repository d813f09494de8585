/*
 * qed.h -- C ABI of the GB300 QED particle-step library.
 *
 * The library advances macro-particles (electrons, positrons, photons, ions)
 * through one or more particle-in-cell time steps of the extended PIC scheme
 * of Gonoskov et al. (arXiv:1412.6426):
 *   field gather (analytic test fields or CIC on a Yee mesh),
 *   Boris push (Appendix A),
 *   the adaptive event generator (Sec. IV.H) around the modified event
 *   generator for photon emission (Sec. IV.G, Eq. (25)) and the pair
 *   generator (Sec. V.A, Eq. (30)),
 *   creation of photons and pairs,
 *   Esirkepov current deposit and the Yee FDTD field update (Appendix C).
 * The calls follow the paper's statement of a PIC module (Appendix A): a
 * module is initialised with the grid, the species and the rate tables,
 * run once per step with the fields, the particles and the time step, and
 * queried for diagnostics.
 *
 * Units ("Compton units"): momentum m c, energy m c^2, time hbar/(m c^2),
 * length hbar/(m c), fields E_S = m^2 c^3/(e hbar).  Charges in e, masses in
 * the electron mass.  Photons carry their momentum hbar k in m c.
 *
 * Conventions shared by every call:
 *  - Every function returns a qed_status; 0 (QED_OK) is success.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work is ordered on it; qed_step is asynchronous.
 *  - Pointers documented as "host or device" may be ordinary host memory,
 *    page-locked host memory or device memory of the context's GPU; the
 *    library detects which.
 *  - The library never traps or aborts on the device.  Device-side failures
 *    (capacity overflow, non-finite values, a bounded wait that timed out,
 *    a probability above one under the strict flag, a particle moving a
 *    cell or more in one step) set a device status word that the next
 *    synchronising call (qed_diagnostics, qed_particles_get) returns.
 *    After such a failure the context refuses qed_step with QED_ERR_STATE
 *    until it is destroyed.
 *  - The library is not thread-safe per context; distinct contexts are
 *    independent.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QED_ABI_VERSION 3

typedef enum qed_status {
    QED_OK = 0,
    QED_ERR_ARG = 1,        /* invalid argument; nothing was changed */
    QED_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    QED_ERR_CAPACITY = 3,   /* a particle or product buffer overflowed */
    QED_ERR_NONFINITE = 4,  /* a non-finite field or momentum was seen */
    QED_ERR_TIMEOUT = 5,    /* a bounded device wait gave up, or the
                               products of one step nested too deeply */
    QED_ERR_PMGT1 = 6,      /* P_m or P_p exceeded 1 with pm_strict set */
    QED_ERR_STATE = 7,      /* the context holds an earlier device error */
    QED_ERR_COURANT = 8     /* a charged particle moved >= 1 cell in a step
                               with the deposit on */
} qed_status;

typedef enum qed_species {
    QED_ELECTRON = 0,
    QED_POSITRON = 1,
    QED_PHOTON = 2,
    QED_ION = 3,
    QED_NSPECIES = 4
} qed_species;

typedef enum qed_field_mode {
    /* E, B gathered by CIC from caller-owned Yee arrays (all axes periodic;
     * n[2] <= 65535 and n[1] <= 524280, the FDTD launch shape) */
    QED_FIELD_GRID = 0,
    /* constant fields: fp = {Ex, Ey, Ez, Bx, By, Bz} */
    QED_FIELD_UNIFORM = 1,
    /* linearly polarised paraxial Gaussian pulse moving along -x, E along
     * y, B = -E along z, Gaussian temporal envelope:
     * fp = {E0, omega, w0, tau_fwhm_of_intensity, x_focus, y_focus,
     *       z_focus, t_focus, phase0} */
    QED_FIELD_GAUSSIAN_LP = 2,
    /* E = E0 (cos(omega t), sin(omega t), 0), B = 0: fp = {E0, omega} */
    QED_FIELD_ROTATING_E = 3,
    /* independent ensembles (batched test-particle runs): the top ens_bits
     * bits of a particle's id name its ensemble e, whose row of the table
     * given to qed_ensembles_set defines a uniform field plus a rotating E:
     *   E = Eu + E0 (cos(omega t + phase), sin(omega t + phase), 0),  B = Bu,
     *   row = {E0, omega, phase, Eu_x, Eu_y, Eu_z, Bu_x, Bu_y, Bu_z, thin_scale}.
     * Products keep their parent's ensemble bits.  A particle whose ensemble
     * has no row sees no field.  A 10th entry thin_scale > 0 scales the
     * ensemble's thinning limits (floor(thin_limit[sp] * thin_scale)), so an
     * instance keeps a budget in proportion to its size. */
    QED_FIELD_ENSEMBLE = 4,
    /* plane standing wave along x (the avalanche cascade of Sec. V):
     * E_y = E0 sin(omega x) cos(omega t), B_z = -E0 cos(omega x) sin(omega t),
     * x the absolute position (lattice origin included): fp = {E0, omega} */
    QED_FIELD_STANDING_WAVE = 5
} qed_field_mode;

#define QED_ENS_STRIDE 10    /* doubles per row of the ensemble table */
#define QED_MAX_ENS_BITS 16

/* Position lattice (and Yee mesh in QED_FIELD_GRID).  Particles are stored
 * as a cell index plus an offset in [0,1) cell units; node (i,j,k) sits at
 * x0 + (i,j,k)*d.  Yee staggering in cell units:
 *   Ex (i+1/2,j,k)  Ey (i,j+1/2,k)  Ez (i,j,k+1/2)   (J likewise)
 *   Bx (i,j+1/2,k+1/2)  By (i+1/2,j,k+1/2)  Bz (i+1/2,j+1/2,k)
 * Field arrays hold n[0]*n[1]*n[2] elements, x fastest. */
typedef struct qed_grid_desc {
    int32_t n[3];          /* cells per axis, >= 1, product < 2^31 */
    int32_t periodic[3];   /* per axis: 1 periodic, 0 open (particles that
                              leave are removed and counted as absorbed) */
    double d[3];           /* cell size, > 0 */
    double x0[3];          /* position of node (0,0,0) */
    int32_t field_mode;    /* qed_field_mode */
    int32_t reserved;      /* must be 0 */
    double fp[16];         /* analytic field parameters, see qed_field_mode */
} qed_grid_desc;

typedef struct qed_species_desc {
    int64_t capacity[4];   /* particles each species store can hold (>= 0) */
    double charge[4];      /* in e; normally -1, +1, 0, Z */
    double mass[4];        /* in m_e; normally 1, 1, 0, M (photon mass ignored) */
} qed_species_desc;

typedef struct qed_params {
    int32_t precision;          /* 32: FP32 push/gather/deposit; 64: FP64 */
    int32_t nsub_max;           /* cap on sub-intervals of one step, >= 1 */
    int32_t emission_on;        /* photon emission by e-/e+ (Sec. IV.G) */
    int32_t pairs_on;           /* Breit-Wheeler pairs (Sec. V.A) */
    int32_t same_step_children; /* 1: products evolve for the rest of the
                                   step in which they are born; 0: they
                                   start at the next step */
    int32_t deposit_on;         /* grid mode: Esirkepov deposit + Yee update */
    int32_t pm_strict;          /* 1: P_m > 1 or P_p > 1 is an error */
    uint32_t seed;              /* enters every random stream */
    int32_t nbins;              /* photon spectrum bins (0 = none), <= 4096 */
    int32_t compact_interval;   /* steps between removals of dead particles
                                   (0 = only on qed_particles_get) */
    double kappa;               /* dt_q = kappa * bound of Eq. (28) / (33) */
    double lg_lo, lg_hi;        /* log10 range of the spectra */
    int64_t pending_capacity;   /* products per step that evolve within the
                                   step (0 = 1/8 of the total capacity,
                                   at least 65536) */
    /* --- independent ensembles (QED_FIELD_ENSEMBLE) --- */
    int32_t ens_bits;           /* top id bits naming the ensemble, 0..16;
                                   products keep their parent's top bits.
                                   In the other field modes the bits only
                                   record lineage (which seed a product
                                   descends from) and thinning treats each
                                   species as one group */
    /* --- controlling the particle count (Sec. VI) --- */
    int32_t thin_interval;      /* thin after every step whose index s has
                                   (s + 1) % thin_interval == 0 (0 = never) */
    int64_t thin_limit[4];      /* per species: the most particles a group
                                   (one ensemble, or the whole species
                                   without ensembles) keeps; 0 = not thinned.
                                   A group of N > L particles keeps each with
                                   probability L/N and multiplies the
                                   survivors' weights by (its total weight) /
                                   (the survivors' weight): global even
                                   redistribution */
    double emit_fg, pair_fg;    /* generator factors f_g (values <= 1 mean 1):
                                   a product of an accepted draw is kept with
                                   probability 1/f_g and weight x f_g; the
                                   parent's own event is unchanged */
    int32_t emit_ng, pair_ng;   /* N_g samples of the generator per occasion
                                   for the products (values <= 1 mean 1),
                                   weight x 1/N_g; sample 0 is the parent's */
    /* --- the photon-emission event generator (Sec. IV.F-G) --- */
    int32_t generator;          /* qed_generator; the generator factors above
                                   apply to the modified generator only */
    int32_t reserved_gen;       /* must be 0 */
    /* --- pairs from the vacuum (Sec. V.B) --- */
    int32_t schwinger_on;       /* 1: once per step, in every cell, an electron
                                   and a positron at rest are created at a
                                   uniform point of the cell with probability
                                   P_S = E^2 exp(-pi/E) V_cell dt / (4 pi^3)
                                   (Compton units; E = |E| at the cell centre,
                                   B neglected as in the paper); not with
                                   QED_FIELD_ENSEMBLE */
    int32_t reserved_s;         /* must be 0 */
    double schwinger_weight;    /* their statistical weight, > 0 */
} qed_params;

typedef enum qed_generator {
    /* modified event generator, Eq. (25) with f_m = r1^3 (the default):
     * emit delta = r1^3 when r2 < P_m(r1) */
    QED_GEN_MODIFIED = 0,
    /* alternative event generator (Sec. IV.F): emit delta = r1 when
     * r2 < P(r1); under-samples low energies where P > 1 */
    QED_GEN_ALTERNATIVE = 1,
    /* standard event generator (Sec. IV.F) with delta_min -> 0: emit when
     * r1 < W(1), delta the root of W(delta)/W(1) = r2, from inverse-CDF
     * tables built in FP64 at init (chi 1e-6 .. 1e4, 4097 x 1025 values;
     * relative accuracy of delta about 1e-5) */
    QED_GEN_STANDARD = 2
} qed_generator;

/* Launch shapes and schedules; they change the speed, never the results
 * (every particle's random stream is keyed by its id). */
typedef struct qed_tuning {
    int32_t photon_blocks_per_sm;  /* resident 256-thread blocks of the photon
                                      pass per SM (1 .. its occupancy limit) */
    int32_t massive_blocks_per_sm; /* likewise for electrons, positrons, ions */
    int32_t work_chunk;            /* particles a block of the e-/e+/ion pass
                                      takes per grab of the shared work
                                      counter (multiple of 256); 0 = a static
                                      grid-stride loop.  Ensembles and the
                                      mesh's unsorted records only: in the
                                      other analytic modes warps take 32
                                      particles per grab and refill each
                                      lane as its particle finishes */
    int32_t compact_interval;      /* steps between removals of dead records
                                      (and re-sorts), >= 1 */
    int32_t sort_massive;          /* QED_FIELD_ENSEMBLE: at each compaction,
                                      order e-, e+ and ions by the number of
                                      sub-intervals (Eq. (28)) their next step
                                      is estimated to take, so that warps run
                                      loops of about equal length */
    int32_t concurrent;            /* 1: the photon pass and the e-/e+/ion
                                      pass run at the same time on two
                                      streams (the second one the library's
                                      own), so the latency-bound lepton work
                                      fills the photon pass's idle issue
                                      slots; give the two passes at most the
                                      SM's blocks between them */
    int32_t deposit_halo;          /* QED_FIELD_GRID: the current of a cell
                                      block's e-, e+, ions is summed in a
                                      shared-memory tile covering the block
                                      and H cells each side, 0 .. 4 (Appendix
                                      C: the current reduced per block in
                                      shared memory); a particle that has
                                      drifted farther since the last sort, and
                                      every particle with H = 0, adds its
                                      current to J with global atomics */
    int32_t refill_lanes;          /* QED_FIELD_GRID, e-/e+ in cell-block
                                      order: a warp takes new particles for
                                      its idle lanes together once at least
                                      this many lanes have finished their
                                      sub-interval loops (Sec. IV.H: the
                                      loops differ in length), 1 .. 32; 0 =
                                      whole batches of 32, taken when every
                                      lane has finished */
} qed_tuning;

/* Caller-owned Yee arrays (device memory, context precision). */
typedef struct qed_fields {
    void *E[3];
    void *B[3];
    void *J[3];   /* overwritten each step with the deposited current
                     (number-current density: charge in e, velocity in c,
                     per (hbar/mc)^3); Maxwell: dE/dt = curl B - 4 pi alpha J */
} qed_fields;

typedef struct qed_diag {
    int64_t count[4];           /* live particles per species */
    int64_t particle_steps;     /* sum over steps of the live particles at the
                                   start of each step (all species) */
    int64_t species_steps[4];   /* the same sum per species */
    int64_t emissions, pairs;   /* events since qed_init */
    int64_t substeps_lepton, substeps_photon;
    int64_t pm_gt1, pp_gt1;     /* draws where P_m > 1 or P_p > 1 */
    int64_t capped;             /* intervals that hit nsub_max */
    int64_t absorbed;           /* particles removed at open boundaries */
    int64_t overflow;           /* products lost to a full buffer */
    int64_t nonfinite;          /* particles with non-finite field/momentum */
    int64_t photons_created;    /* photons made (equals emissions unless the
                                   generator factors are set) */
    int64_t pairs_created;      /* pairs made (likewise) */
    int64_t thinned;            /* particles removed by thinning */
    int64_t schwinger_pairs;    /* pairs created from the vacuum */
    int64_t schwinger_gt1;      /* cell-steps with P_S > 1 (one pair made) */
    int64_t kernel_launches;    /* CUDA kernels this context has launched */
    int64_t step;               /* steps taken */
    double time;                /* current time */
    int32_t status;             /* device status (qed_status) */
    int32_t nbins;              /* in: length of the arrays below */
    double *spectrum;           /* in: host array of nbins or NULL; out:
                                   weighted counts of emitted photons over
                                   log10(delta) in [lg_lo, lg_hi) */
    double *spectrum_energy;    /* same over log10(photon energy / m c^2) */
    int64_t block_steps;        /* QED_FIELD_GRID: the part of particle_steps
                                   that the cell-block pass advanced and
                                   deposited (e-, e+, ions in cell-block
                                   order; the rest go through the other
                                   passes) */
    int64_t tile_deposits;      /* QED_FIELD_GRID: of block_steps, the
                                   deposits made through the shared-memory
                                   current tile of their cell block (the
                                   others, which drifted out of the tile's
                                   reach since the last sort, add to J
                                   directly) */
} qed_diag;

typedef struct qed_ctx qed_ctx;

/* Create a context on the current CUDA device.
 *  grid, species, params: host structs, copied.
 *  tables: NULL to build the FP64 rate tables of F1(z), F2(z) (Sec. IV.E,
 *    Eq. (20)-(21)) on the device, or a host buffer of tables_bytes
 *    previously filled by qed_tables_export (any precision).
 *  Allocates the particle stores (capacity per species, library-owned) and
 *  the product buffer.  Returns QED_ERR_ARG for invalid descriptors,
 *  QED_ERR_CUDA if an allocation or launch fails; *out is NULL then. */
int qed_init(qed_ctx **out, const qed_grid_desc *grid, const qed_species_desc *species,
             const void *tables, size_t tables_bytes, const qed_params *params, void *stream);

/* Copy the context's rate tables to host memory.  With host_buf == NULL
 * only *needed is written.  QED_ERR_ARG if bytes < *needed. */
int qed_tables_export(qed_ctx *ctx, void *host_buf, size_t bytes, size_t *needed);

/* Replace the particles of one species (host or device pointers):
 *  x: n x 3 absolute positions, p: n x 3 momenta (m c), w: n weights,
 *  id: n unique 64-bit ids (they key the random streams, Sec. IV.G).
 * Positions outside an open lattice are removed (absorbed).  QED_ERR_ARG if
 * n exceeds the capacity or species is invalid. */
int qed_particles_set(qed_ctx *ctx, int species, const double *x, const double *p,
                      const double *w, const uint64_t *id, int64_t n, void *stream);

/* Remove dead particles of one species and copy the live ones out (host or
 * device pointers; layout as in qed_particles_set, FP64).  This is the
 * particle ensemble of the module interface (Appendix A: the Ensemble
 * object the Controller exposes, with its iterator over a domain's
 * particles); the records hold what Sec. IV.F and V.A give a super-particle:
 * position, momentum, statistical weight, plus the id that keys its random
 * streams.  *n_out receives the live count; at most max_n are written
 * (QED_ERR_ARG if more are live, and nothing is written then).  Host
 * buffers are filled by copies from a device staging buffer of 64 B per
 * particle, allocated on first use and kept by the context.
 * Synchronises the stream and returns the device status (a failure latches
 * the context). */
int qed_particles_get(qed_ctx *ctx, int species, double *x, double *p, double *w,
                      uint64_t *id, int64_t max_n, int64_t *n_out, void *stream);

/* Read the live particles of one species, like qed_particles_get, without
 * allocating any memory.  The paper has no counterpart; this call exists for
 * callers that cannot call cudaMalloc when they want the results: hosts
 * whose device memory all belongs to their own pool allocator (an
 * allocation behind the pool's back can fail or fragment it), and real-time
 * loops that forbid allocation after start-up (an allocation can block on
 * the driver for an unbounded time).
 *  x, p, w, id: device or page-locked host buffers (layout as in
 *    qed_particles_set); pageable host memory is refused with QED_ERR_ARG,
 *    since it would need a staging buffer.  With max_n == 0 they may be NULL.
 *  The current device must be the context's (else QED_ERR_ARG).
 *  At most max_n particles are written, in store order (the order
 *  qed_particles_get would give); *n_out receives the live count, and
 *  QED_ERR_ARG is returned when it exceeds max_n (the first max_n are
 *  written all the same).
 *  Unlike qed_particles_get the store is not compacted.
 *  Scratch: a fixed device array of 65536 tile counters inside the library
 *  (512 KiB, held by every GPU that loads the library until exit), enough
 *  for stores of up to 134,217,728 records (live plus not yet removed);
 *  larger stores are refused with QED_ERR_CAPACITY.  The first call on a
 *  device looks up the array's device address (cudaGetSymbolAddress), so
 *  make that first call before any stream capture.  All calls share the
 *  array: calls that overlap on the GPU race and must be ordered by the
 *  caller.
 * Synchronises the stream and returns the device status; a failure latches
 * the context as in qed_particles_get. */
int qed_particles_read_static(qed_ctx *ctx, int species, double *x, double *p, double *w,
                              uint64_t *id, int64_t max_n, int64_t *n_out, void *stream);

/* Advance all species by nsteps steps of dt: the module's run at the port
 * points of one PIC iteration (Appendix A), fused into one launch sequence.
 * Each step is, per particle, the field held fixed over the step (Sec. IV.H),
 * the adaptive event generator (Sec. IV.H: N = ceil(dt/dt_q) sub-intervals,
 * dt_q from Eq. (28) for e-/e+ and Eq. (33) for photons) around the Boris
 * push (Appendix A) and the modified emission generator (Sec. IV.G,
 * Eq. (25)) or the pair generator (Sec. V.A, Eq. (30)), creation of the
 * products, and, in QED_FIELD_GRID, the Esirkepov deposit and the Yee FDTD
 * update (Appendix C); then thinning (Sec. VI) and pairs from the vacuum
 * (Sec. V.B) when enabled.
 *  fields: NULL unless field_mode is QED_FIELD_GRID, where the E, B arrays
 *    are read (gather), J is overwritten by the deposit and E, B are advanced
 *    by one symmetrised FDTD step after the particles (deposit_on).  The
 *    first step of a call reads the largest |E|, |B| components off the
 *    arrays (the bound behind the photons' early exit); later steps of the
 *    same call take them from the field update before, so the caller
 *    changes the arrays only between calls.
 *  Asynchronous; allocates nothing, so it may be captured in a CUDA graph.
 *  QED_ERR_STATE after a device error, QED_ERR_ARG for dt <= 0 or missing
 *  fields. */
int qed_step(qed_ctx *ctx, const qed_fields *fields, double dt, int32_t nsteps, void *stream);

/* Set the field table of QED_FIELD_ENSEMBLE: n_ens rows of QED_ENS_STRIDE
 * doubles (host memory, copied; see QED_FIELD_ENSEMBLE).  n_ens must be in
 * 1 .. 2^ens_bits (1 when ens_bits is 0) and every entry finite, else
 * QED_ERR_ARG.  May be called between steps to change the fields.
 * qed_step in this mode returns QED_ERR_ARG until a table is set. */
int qed_ensembles_set(qed_ctx *ctx, int32_t n_ens, const double *table, void *stream);

/* Read or replace the launch shapes and schedules (host struct).
 * QED_ERR_ARG for values outside the documented ranges.  After
 * qed_set_tuning the next compaction comes compact_interval steps later, so
 * a captured sequence of steps that starts there and covers an even number
 * of compactions (and a whole number of thinning intervals) replays
 * correctly. */
int qed_get_tuning(qed_ctx *ctx, qed_tuning *out);
int qed_set_tuning(qed_ctx *ctx, const qed_tuning *tuning);

/* Pick the tuning by measurement: advances the simulation by real steps of
 * dt (the results are the ones untuned steps would give), trying the
 * candidates of each field of qed_tuning in turn, each for
 * max(steps_per_trial, its compaction interval) steps timed with CUDA
 * events on the stream, in the order listed and then reversed, so that a
 * workload that grows during the search does not favour the later
 * candidates.  The cost of a candidate is its time per particle-step.
 * Candidates: 1 .. 4 blocks per SM for each pass (up to the occupancy
 * limit), work chunks {0, 256, 1024, 4096, 16384}, compaction intervals
 * {c, c/2, c/4} below the current interval c (the capacities were sized
 * for c), with ensembles sorting on or off, and on the Yee mesh the deposit's
 * tile halo {4, 3, 2, 1} or global atomics only (0) and the lane refill of
 * the cell-block pass {0, 24, 16}.  The search stops before a
 * trial that would take more than max_steps steps in all; the fields not
 * reached keep their values.  Applies the best tuning found, writes it to
 * *out (may be NULL) and the number of steps taken to *steps_taken (may be
 * NULL).  Synchronises the stream. */
int qed_autotune(qed_ctx *ctx, const qed_fields *fields, double dt, int32_t steps_per_trial,
                 int64_t max_steps, void *stream, qed_tuning *out, int64_t *steps_taken);

/* Set the step counter and time used by the next qed_step (the random
 * streams are keyed by the step, so a restart reproduces a run exactly). */
int qed_set_clock(qed_ctx *ctx, int64_t step, double time);

/* Profiling aid: record CUDA events (cudaEvent_t passed as void*, created by
 * the caller on the context's device) around the kernels of every following
 * step, on the stream of that step: start before the first step kernel,
 * photon_done after the photon kernel (may be NULL), stop after the last
 * step kernel (compaction excluded).  All NULL stops recording.  The events
 * are not owned by the library. */
int qed_profile_events(qed_ctx *ctx, void *start, void *photon_done, void *stop);

/* Points of a step at which qed_profile_stages records its events, in the
 * order the step reaches them on its stream.  A stage a step does not run
 * (no mesh, no vacuum pairs, ...) is recorded right after the previous one,
 * so the time between two consecutive events is the time of the kernels in
 * between (zero when there are none). */
typedef enum qed_stage {
    QED_STAGE_BEGIN = 0,     /* before the step's first kernel */
    QED_STAGE_CONSTANTS,     /* after the mesh maxima (read off the fields at the
                                first step of a qed_step call; later steps take
                                them from the field update) and the step constants */
    QED_STAGE_PHOTONS,       /* after the photon pass */
    QED_STAGE_BLOCKS,        /* after the cell-block pass of e-, e+, ions (mesh) */
    QED_STAGE_DEPOSIT,       /* after the cell-block current deposit (mesh) */
    QED_STAGE_MASSIVE,       /* after the e-/e+/ion pass of the other records */
    QED_STAGE_PRODUCTS,      /* after the in-step products */
    QED_STAGE_SCHWINGER,     /* after the pairs from the vacuum */
    QED_STAGE_FIELD,         /* after the Yee field update (mesh) */
    QED_STAGE_END,           /* after thinning, compaction and sorting */
    QED_NSTAGES
} qed_stage;

/* Profiling aid: record the caller's CUDA events (cudaEvent_t passed as
 * void*, created on the context's device) at the stages of the following
 * steps, on the stream of each step.  n <= QED_NSTAGES: entry k for stage
 * k, recorded by every step (give a fresh array before each step to keep
 * every step's times).  n = m QED_NSTAGES with m > 1: entries j QED_NSTAGES
 * + k for stage k of step j of every following qed_step call (steps from m
 * on record nothing), so one call of m steps keeps every step's times.
 * NULL entries are skipped; n == 0 stops recording.  QED_ERR_ARG for any
 * other n.  The events are not owned by the library; the array itself is
 * copied. */
int qed_profile_stages(qed_ctx *ctx, void *const *events, int32_t n);

/* Self-test of the failure detection of the bounded device waits: the grid
 * barrier between the passes of the in-step products, in a cooperative
 * launch of one block per SM of which block absent_block (-1: none) never
 * arrives.  The others give up after spin_limit polls of about 64 ns each
 * (the step itself allows 2^24, about a second).  Returns QED_ERR_TIMEOUT
 * when the wait ran out, QED_OK when every block got through; uses spare
 * device words of the context and leaves its status as it was.  The paper
 * has no counterpart; the call exists to test that a wait that cannot end
 * ends with an error instead of a hang.  Synchronises the stream. */
int qed_selftest_barrier(qed_ctx *ctx, int32_t absent_block, int64_t spin_limit, void *stream);

/* Synchronise the stream and read counters, live counts, spectra and the
 * device status into *out (host struct).  The quantities are the ones the
 * paper's tests read off a run: the emitted-photon spectrum over log10(delta)
 * that Sec. IV.G compares with Eq. (21), the particle numbers per species
 * (the distribution functions of Sec. VII.B integrated over energy) and the
 * event and sub-interval counts of the adaptive generator (Sec. IV.H).
 * Returns the device status (a failure latches the context). */
int qed_diagnostics(qed_ctx *ctx, qed_diag *out, void *stream);

/* Free every resource of the context.  NULL is accepted. */
int qed_destroy(qed_ctx *ctx);

/* Static description of a status code. */
const char *qed_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* QED_H */
