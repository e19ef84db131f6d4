/*
 * pic.h -- C ABI of the GB300 (sm_103a) particle-in-cell Monte Carlo time step.
 *
 * The library advances a batch of independent 1D3V bounded-plasma instances through
 * the PIC cycle of Williams et al., arXiv 2404.10270, Section 2 (density deposit,
 * field solve, collisions and plasma-wall interaction, particle mover), with the
 * linear field gather and the position update of the moveb() mover (Listing 7).
 * One call of pic_step() runs, for every particle of every instance:
 *   gather -> push (leapfrog, or Boris rotation when B != 0) -> move -> wall ->
 *   null-collision Monte Carlo collision -> cloud-in-cell deposit,
 * then, per instance, the Poisson solve with E = -grad(phi) (Section 2, "Field
 * Solver"), and every `sort_interval` steps a counting sort of the particles by cell
 * (the locality the paper's "natural sorting" layout provides, Section 2, Fig.
 * "BIT1_sorting").
 *
 * Units are normalised: eps0 = e = m_e = n0 = lambda_D = omega_pe = 1 (T_e = 1).
 * A position is the BIT1 pair (cell j, in-cell offset f in [0,1)), Section 2 and
 * Listing 7.  Velocities cross this interface in units of lambda_D * omega_pe.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status (PIC_OK or a negative pic_status).  No C++
 *    exception, abort or exit crosses the interface.
 *  - Input pointers are borrowed for the duration of the call; data is copied in.
 *    Output buffers belong to the caller.  `flags` of the particle calls: PIC_DEVICE
 *    means the pointers are CUDA device pointers valid on the handle's device (else
 *    host memory, pinned or pageable); PIC_CELL_UNITS means velocities are in the
 *    library's internal unit, cells per time step (u = v dt/dx), which makes a
 *    get/load round trip exact (checkpoints); otherwise they are physical.
 *  - The handle owns all device memory it allocates and releases it in pic_destroy.
 *  - A handle is used by one host thread at a time.  Work is ordered on the handle's
 *    stream (the borrowed `cuda_stream` of pic_config, or a stream the library owns).
 *  - pic_step only enqueues work.  Errors detected on the device (capacity
 *    overflow, non-finite state, invalid loaded particles) are latched in a device
 *    status word and reported by the next synchronising call (pic_sync, pic_moments,
 *    pic_get_particles, pic_charge_raw); from then on every call except pic_destroy
 *    and pic_last_error returns PIC_ESTATE.
 */
#ifndef PIC_H
#define PIC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#define PIC_MAX_SPECIES 4
#define PIC_MAX_PROC 8

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,     /* invalid argument or configuration */
    PIC_ENOMEM = -2,     /* device or host allocation failed */
    PIC_ECUDA = -3,      /* a CUDA runtime call failed */
    PIC_ECAPACITY = -4,  /* a species segment or the event buffer overflowed */
    PIC_ENONFINITE = -5, /* a particle velocity became Inf/NaN */
    PIC_ETIMEOUT = -6,   /* a bounded device wait ran out */
    PIC_ESTATE = -7      /* the handle is in the error state */
} pic_status;

enum { PIC_FP32 = 0, PIC_FP64 = 1 };                          /* particle state precision */
enum { PIC_DEVICE = 1, PIC_CELL_UNITS = 2 };                  /* flags of load/get */
enum { PIC_BC_ABSORB = 0, PIC_BC_PERIODIC = 1, PIC_BC_SOURCE = 2 };
enum { PIC_FIELD_POISSON = 0, PIC_FIELD_NONE = 1, PIC_FIELD_EXTERNAL = 2 };
enum { PIC_PROC_ELASTIC = 0, PIC_PROC_CX = 1, PIC_PROC_IONIZE = 2, PIC_PROC_EXCITE = 3 };

/* One species of one instance. */
typedef struct {
    double charge;      /* q_s in units of e */
    double mass;        /* m_s in units of m_e */
    double weight;      /* w_s, physical particles per unit area per macro-particle */
    double temperature; /* T_s of the volume source's Maxwellian (PIC_BC_SOURCE) */
    int64_t capacity;   /* particle slots reserved (>= largest load + creations) */
    int32_t nstep;      /* subcycling (Listing 7's x += nstep*vx): the species is advanced
                           with time step nstep*dt on the steps n (counted from 0) with
                           (n+1) mod nstep = 0, so that every species is at the same time
                           at the multiples of nstep*dt, and deposited every step; 0 or
                           1 = every step (at most 4096) */
    int32_t sn2d;       /* 1: a 2-D species that also drifts in y (Listing 1's
                           yp += nstep*vy): a coordinate yp parallel to the walls, in cell
                           units, advanced with the velocity after the push on the steps
                           the species moves and used by nothing else (the field, walls and
                           collisions are 1D); a re-injected particle restarts at yp = 0,
                           ionization products start at their parent's yp.  Set and read
                           with pic_load_yp / pic_get_yp.  0: no y coordinate */
} pic_species;

/* One collision process against the uniform neutral background (null-collision
 * Monte Carlo; the paper's collision phase, Section 2).  The collision frequency is
 * `nu` for projectile energies at or above `threshold` and 0 below. */
typedef struct {
    int32_t kind;      /* PIC_PROC_*; PIC_PROC_EXCITE: energy loss of `threshold`, new
                          direction uniform on the sphere */
    int32_t species;   /* projectile species */
    int32_t product;   /* PIC_PROC_IONIZE: species of the created ion, else -1 */
    int32_t pad;
    double nu;         /* units of omega_pe */
    double threshold;  /* units of T_e */
} pic_process;

/* One bounded-plasma instance: cells 0..ncells-1, nodes 0..ncells, walls at the
 * first and last node. */
typedef struct {
    int32_t ncells;
    int32_t bc;        /* PIC_BC_* */
    int32_t field;     /* PIC_FIELD_* (PIC_FIELD_POISSON needs a non-periodic bc) */
    int32_t nspecies;  /* 1..PIC_MAX_SPECIES */
    double dx, dt, eps0;
    double E_ext;      /* uniform field for PIC_FIELD_EXTERNAL */
    double B[3];       /* uniform magnetic field; x is the wall normal */
    double T_neutral;  /* neutral background temperature (units of T_e) */
    double m_neutral;  /* neutral background mass (units of m_e) */
    pic_species sp[PIC_MAX_SPECIES];
    int32_t nproc;
    int32_t smooth;    /* 1: the density smoother (Section 2's "Density Smoother" phase):
                          a 1-2-1 binomial filter of the interior node charge densities
                          before the field solve, wall nodes unfiltered; 0: off */
    pic_process proc[PIC_MAX_PROC];
    uint64_t seed;     /* Philox4x32-10 key of this instance */
    /* Neutral target species (the paper's test case, Section 3 Table 1: electrons, D+ and
       D neutrals as particles): 0 = every process collides with the uniform background;
       k+1 = species k (charge 0) is the target of every process: a candidate in cell j is
       kept with probability min(1, n_j / nref), n_j the live target particles whose cell
       was j at the start of the step, and an ionization turns the live target particle of
       cell j with the smallest id into the product ion (same id, position and velocity),
       creating one electron.  The target species must move only on the sort steps: its
       nstep equals the sort interval. */
    int32_t target;
    int32_t nref;      /* target particles per cell at which the processes' nu apply */
} pic_instance;

typedef struct {
    int32_t n_instances;        /* >= 1 */
    int32_t precision;          /* PIC_FP32 or PIC_FP64 */
    int32_t sort_interval;      /* sort by cell every this many steps; 0 = never;
                                   -1 = autotune (10, 20, 40 or 80) */
    int32_t block;              /* mover threads per block (128, 256, 512); 0 = autotune.
                                   The step that ends a sort cycle has its own block size,
                                   128 ($BITPIC_SORT_BLOCK: 128, 256 or 512).
                                   The autotuner times one sort cycle per candidate on the
                                   first steps of the run (results do not depend on either
                                   choice) and caches the choice per GPU and size bucket
                                   in $BITPIC_TUNE_CACHE (default
                                   $HOME/.cache/bitpic/autotune.json).  An FP32 batch
                                   without magnetic field, whose colliding species move
                                   on every step, with at least $BITPIC_PAIR_MIN_SLOTS
                                   particle slots (default 2^24) moves its particles
                                   with a mover variant that leaves most collision-clock
                                   draws to the event kernel; this too changes no
                                   result. */
    const pic_instance* inst;   /* n_instances entries, copied */
    void* cuda_stream;          /* borrowed cudaStream_t; NULL = library-owned stream */
} pic_config;

typedef struct pic_handle pic_handle;

/* Per-instance diagnostics of the current step. */
typedef struct {
    int64_t step;                              /* steps taken since creation */
    int64_t live[PIC_MAX_SPECIES];             /* particles alive */
    int64_t wall_count[PIC_MAX_SPECIES][2];    /* absorbed at [left, right] wall */
    double wall_energy[PIC_MAX_SPECIES][2];    /* sum of w m v^2/2 of absorbed particles */
    int64_t collisions[PIC_MAX_PROC];          /* real collision events per process */
    double kinetic[PIC_MAX_SPECIES];           /* sum of w m v^2/2 over live particles */
    int64_t next_id;                           /* id the next created particle gets */
} pic_moments_out;

/* Create a handle: validates the configuration, allocates the particle store
 * (structure of arrays, capacity per species segment), the grid arrays and the
 * counters on the current CUDA device.  *out is set only on success. */
PIC_API int pic_create(const pic_config* cfg, pic_handle** out);

/* Replace the particles of (instance, species) with n particles: cell[k] in
 * [0, ncells), off[k] in [0, 1), physical velocities.  id == NULL numbers them after
 * the largest id of the instance so far.  state == NULL starts every particle's
 * collision clock at 0 (its next step draws); otherwise state[k] is the clock that
 * pic_get_particles returned (bits 0-6: steps to skip before the particle's next
 * collision event step; bit 7: that event step is a collision candidate), which makes
 * a checkpoint/restart continue bit-identically.  n must not exceed the species
 * capacity (else PIC_ECAPACITY).  Invalid cell/offset values are reported as
 * PIC_EINVAL by the next synchronising call.  Marks the fields stale: the next
 * pic_step first deposits all particles and solves the field. */
PIC_API int pic_load_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                               const int32_t* cell, const double* off, const double* vx,
                               const double* vy, const double* vz, const uint32_t* id,
                               const uint8_t* state, int32_t flags);

/* pic_load_particles with offsets and velocities in float: the same call with 24
 * instead of 40 bytes per particle through the host link, for callers whose data is
 * single precision (the FP32 form keeps its state in float anyway).  Each offset must
 * be below 1 as a float; the FP64 form widens the values exactly. */
PIC_API int pic_load_particles_f32(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                                   const int32_t* cell, const float* off, const float* vx,
                                   const float* vy, const float* vz, const uint32_t* id,
                                   const uint8_t* state, int32_t flags);

/* The y coordinates (cell units) of an sn2d species (see pic_species.sn2d), for the n
 * particles of the last pic_load_particles(_f32) call of (instance, species) and in the
 * same order; that call sets them to 0.  Only between that call and the next pic_step
 * (else PIC_ESTATE for this call, the handle stays usable), n equal to that call's n
 * (else PIC_EINVAL), a species with sn2d = 1 (else PIC_EINVAL).  flags: PIC_DEVICE when
 * yp is device memory (else host memory, copied in before the call returns). */
PIC_API int pic_load_yp(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                        const double* yp, int32_t flags);

/* The y coordinates (cell units) of the live particles of (instance, species) in the
 * order of pic_get_particles (storage order); *n_out receives their number, which must
 * not exceed `capacity` (else PIC_ECAPACITY).  A species without sn2d gets zeros.
 * flags: PIC_DEVICE when yp is device memory.  Synchronises. */
PIC_API int pic_get_yp(pic_handle* h, int32_t inst, int32_t species, int64_t capacity,
                       double* yp, int32_t flags, int64_t* n_out);

/* Enqueue nsteps time steps of every instance on the handle's stream. */
PIC_API int pic_step(pic_handle* h, int64_t nsteps);

/* Wait for the handle's stream and report latched device errors. */
PIC_API int pic_sync(pic_handle* h);

/* Diagnostics of instance `inst` (synchronises).  Optional host arrays (NULL to skip),
 * each indexed by node 0..ncells: `density` nspecies*(ncells+1) number densities
 * (species-major; the wall nodes are normalised by the half cell next to the wall),
 * `phi` the potential and `E` the field of the current step. */
PIC_API int pic_moments(pic_handle* h, int32_t inst, pic_moments_out* out, double* density,
                double* phi, double* E);

/* Number of live particles of (inst, species) (synchronises). */
PIC_API int pic_count(pic_handle* h, int32_t inst, int32_t species, int64_t* n);

/* Copy out the live particles of (inst, species) in storage order: *n_out receives
 * their number, which must not exceed `capacity` (else PIC_ECAPACITY, nothing
 * written).  Any output pointer may be NULL.  Velocities are physical; `state`
 * receives each particle's collision clock (see pic_load_particles). */
PIC_API int pic_get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t capacity,
                              int32_t* cell, double* off, double* vx, double* vy, double* vz,
                              uint32_t* id, uint8_t* state, int32_t flags, int64_t* n_out);

/* pic_get_particles into float offsets and velocities (each value formed in double, as
 * pic_get_particles returns it, and rounded once to float).  An FP64-form offset so
 * close to 1 that it would round to 1.0f is returned as the largest float below 1
 * (1 - 2^-24) in the same cell, so every read-back loads again.  Same arguments and
 * errors otherwise. */
PIC_API int pic_get_particles_f32(pic_handle* h, int32_t inst, int32_t species,
                                  int64_t capacity, int32_t* cell, float* off, float* vx,
                                  float* vy, float* vz, uint32_t* id, uint8_t* state,
                                  int32_t flags, int64_t* n_out);

/* Restore the counters a checkpoint needs besides the particles: the step count of
 * the handle (it keys every random draw) and, when next_id is not NULL, the next
 * particle id of each of the n_instances instances (ids given to ionization
 * products).  Together with pic_load_particles(..., state, ...) of every species this
 * continues a run bit-identically. */
PIC_API int pic_restore_counters(pic_handle* h, int64_t step, const uint64_t* next_id);

/* The fixed-point charge deposit of the last step for instance `inst`: host array of
 * nspecies*(ncells+1) int64 node sums, in units where every live particle adds
 * exactly *unit (2^24 in the FP32 form, 2^48 in the FP64 form) split over the two
 * nodes of its cell (synchronises). */
PIC_API int pic_charge_raw(pic_handle* h, int32_t inst, int64_t* out, int64_t* unit);

/* Kernel timing: when enabled, every kernel launch of pic_step is bracketed by CUDA
 * events on the handle's stream.  pic_kernel_time returns, for kernel class `which`
 * (0 mover, 1 field, 2 sort, 3 other, 5 the mover of a step that also sorts the store),
 * the number of timed launch groups and their total milliseconds since the last
 * pic_profile call (synchronises); `which` = 4 returns the number of kernels the
 * library launched since then (total_ms = 0). */
PIC_API int pic_profile(pic_handle* h, int32_t enable);
PIC_API int pic_kernel_time(pic_handle* h, int32_t which, int64_t* launches, double* total_ms);

/* Destroy the handle and release its memory.  NULL-safe; always returns PIC_OK. */
PIC_API int pic_destroy(pic_handle* h);

/* Text of the last error on this handle (or of the last failed pic_create when h is
 * NULL).  The string lives until the next call on the handle. */
PIC_API const char* pic_last_error(const pic_handle* h);

/* The library's Philox4x32-10 generator (Salmon et al., SC'11), run on the GPU:
 * out[4k..4k+3] = Philox4x32-10(ctr[4k..4k+3], key) for k < n.  Exposes the exact
 * generator that keys every random draw of the time step by (seed, particle id,
 * step, purpose), so that it can be checked on its own.  `stream` is a borrowed
 * cudaStream_t (NULL = default stream); the call synchronises it. */
PIC_API int pic_philox(uint64_t key, const uint32_t* ctr, uint32_t* out, int64_t n,
               int32_t on_device, void* stream);

/* Self-test of the bounds-checked device build (the library compiled with PIC_CHECKED,
 * in which every index a kernel computes into a particle store, node array, queue or
 * staging buffer is checked and a violation latches a status bit that the next
 * synchronising call reports as PIC_ECUDA, the access skipped; the paper has no
 * counterpart).  One thread asks for an index one past a range through that check; the
 * check must refuse it (no access is made) and latch the bit.  Returns PIC_OK when it
 * did, PIC_ECUDA when it did not or a launch failed, PIC_EINVAL in the normal build
 * (which has no checks).  `stream`: borrowed cudaStream_t (NULL = default stream); the
 * call synchronises it.  Message from pic_last_error(NULL). */
PIC_API int pic_bounds_probe(void* stream);

/* Allocation-free field solve (the paper has no counterpart; it exists for callers
 * that cannot allocate device memory: code running while a CUDA graph is being
 * captured, latency-critical loops in which an allocation could block or fragment,
 * and host frameworks that own all device memory through their own pools).
 * Computes, for one instance of `ncells` cells (at most 65536), the field E on nodes
 * 0..ncells from its fixed-point charge deposits with the same arithmetic as the
 * handle's field phase: the grounded Dirichlet Poisson problem solved in 128-bit
 * integers, E = -grad phi with Gauss's law over the wall half cells.  The deposits are
 * used as given: no density smoother is applied, so for an instance created with
 * smooth = 1 the result is the field of the unfiltered charge, not the handle's E.
 *   charge  device array, nspecies x (ncells+1) int64, species-major: the per-node
 *           deposits in units where one particle adds `unit` (the layout and unit
 *           pic_charge_raw returns);
 *   z       host array of nspecies integers: species charge q_s w_s = z_s * delta;
 *   eps0    vacuum permittivity;  E  device array of ncells+1 doubles (output);
 *   stream  borrowed cudaStream_t (NULL = default stream); the call only enqueues.
 * Allocates nothing: its scratch (one 128-bit sum per node) is a static device array
 * of the library, 1 MB on every GPU that loads it, held until the process exits.  A
 * call whose stream is not capturing looks up that array's device address for the
 * current device (so a device reset between calls is harmless); a call made while its
 * stream is being captured reuses the address of the last such lookup on the device,
 * so make the first call on a device before any stream capture.  Every call on a device
 * shares the array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  Returns PIC_EINVAL for ncells outside
 * [1, 65536] or bad arguments, PIC_ECUDA if a launch fails; the message is available
 * from pic_last_error(NULL). */
PIC_API int pic_field_solve_noalloc(int32_t ncells, int32_t nspecies, const int64_t* charge,
                                    const int32_t* z, double delta, int64_t unit, double eps0,
                                    double* E, void* stream);

#ifdef __cplusplus
}
#endif
#endif
