/*
 * oracle.h -- plain FP64 CPU oracle of the 1D3V PIC Monte Carlo time step
 * (Williams et al., "Accelerating Particle-in-Cell Monte Carlo Simulations with
 * MPI, OpenMP/OpenACC and Asynchronous Multi-GPU Programming", arXiv 2404.10270).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is the slow, obviously correct reference
 * that the GPU library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table
 * or helper with the GPU library: everything below is written independently from
 * the paper (Section 2, the PIC cycle; Listing 7, the moveb() gather/update) and
 * from the textbook methods named at each function.
 *
 * Units are normalised: eps0 = e = m_e = n0 = lambda_D = omega_pe = 1, so the
 * electron thermal speed and the electron temperature T_e are 1.  As in BIT1
 * (Section 2, "natural sorting"; Listing 7), a particle position is the pair
 * (cell index j, in-cell offset f in [0,1)), and inside the oracle velocities are
 * carried in cells per time step (u = v dt/dx), so that the paper's position
 * update "x += nstep*vx" applies literally.  Velocities cross the API in physical
 * units (lambda_D * omega_pe).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_ABSORB = 0, ORC_BC_PERIODIC = 1, ORC_BC_SOURCE = 2 };
enum { ORC_FIELD_POISSON = 0, ORC_FIELD_NONE = 1, ORC_FIELD_EXTERNAL = 2 };
enum { ORC_PROC_ELASTIC = 0, ORC_PROC_CX = 1, ORC_PROC_IONIZE = 2, ORC_PROC_EXCITE = 3 };
/* Philox counter word 3 ("purpose") of every draw the step makes. */
enum { ORC_RNG_COLLIDE = 0, ORC_RNG_SCATTER = 1, ORC_RNG_MAXWELL = 2,
       ORC_RNG_INJECT_A = 3, ORC_RNG_INJECT_B = 4, ORC_RNG_IONIZE_E = 5,
       ORC_RNG_IONIZE_I = 6 };

#define ORC_MAX_SPECIES 4
#define ORC_MAX_PROC 8

typedef struct {
    double charge;      /* q_s in units of e */
    double mass;        /* m_s in units of m_e */
    double weight;      /* w_s: physical particles per unit area per macro-particle */
    double temperature; /* T_s (units of T_e) of the volume source's Maxwellian */
    int32_t nstep;      /* subcycling (Listing 7's x += nstep*vx): advanced with time step
                           nstep*dt on the steps n with (n+1) mod nstep = 0; 0 or 1 =
                           every step */
    int32_t sn2d;       /* 1: the species also drifts in y (Listing 1: yp += nstep*vy), a
                           coordinate in cell units parallel to the walls that nothing
                           else depends on */
} orc_species;

typedef struct {
    int32_t kind;       /* ORC_PROC_* */
    int32_t species;    /* projectile species */
    int32_t product;    /* ionization: species index of the created ion (else -1) */
    int32_t pad;
    double nu;          /* collision frequency above threshold, units of omega_pe */
    double threshold;   /* energy threshold, units of T_e */
} orc_process;

typedef struct {
    int32_t ncells;     /* N: cells; nodes 0..N */
    int32_t bc;         /* ORC_BC_* */
    int32_t field;      /* ORC_FIELD_* */
    int32_t nspecies;
    double dx, dt, eps0;
    double E_ext;       /* uniform field for ORC_FIELD_EXTERNAL */
    double B[3];        /* uniform magnetic field; x is the wall normal */
    double T_neutral;   /* neutral background temperature */
    double m_neutral;   /* neutral background mass */
    orc_species sp[ORC_MAX_SPECIES];
    int32_t nproc;
    int32_t smooth;     /* 1: 1-2-1 filter of the interior charge density before Poisson */
    orc_process proc[ORC_MAX_PROC];
    uint64_t seed;      /* Philox key */
    int32_t target;     /* 0: uniform neutral background; k+1: species k (charge 0) is the
                           particle target of every process (see orc_step) */
    int32_t nref;       /* target particles per cell at which the processes' nu apply */
} orc_params;

typedef struct orc_sim orc_sim;

/* Returns NULL on invalid parameters or allocation failure. */
orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);

/* Replace species `sp` with n particles.  cell/off are the BIT1 (j, f) pair,
 * velocities are physical.  id == NULL assigns consecutive ids after all ids
 * loaded so far.  mcc: per-particle collision clock (bits 0-6 steps to skip, bit 7
 * candidate pending), NULL = 0 (the next step draws).  yp: the y coordinate (cell
 * units) of an sn2d species, NULL = 0.  Returns 0 or a negative error. */
int orc_load(orc_sim* s, int32_t sp, int64_t n, const int32_t* cell, const double* off,
             const double* vx, const double* vy, const double* vz, const uint32_t* id,
             const uint8_t* mcc, const double* yp);

/* Advance nsteps time steps.  Returns 0 or a negative error. */
int orc_step(orc_sim* s, int64_t nsteps);

/* Use E (N+1 node values) as the field of the next step instead of the one formed from
 * this instance's own particles (a run split into subdomains solves it jointly). */
int orc_set_field(orc_sim* s, const double* E);

/* Continue a saved run: set the step counter (the next step is `step`, which keys its
 * draws and places it on the collision clock's grid) and raise the next id for created
 * particles to at least next_id.  Counters of walls and collisions are not touched. */
int orc_set_step(orc_sim* s, int64_t step, uint32_t next_id);

/* One time step in two halves, for a run split into subdomains: orc_step_loop moves
 * every particle (gather, push, move, walls, collisions) and records the step's
 * ionizations; orc_step_finish creates their products (converting neutral particle
 * targets), deposits and solves the field.  orc_step is the two in order.  In between,
 * orc_births_take removes the ionizations recorded in cells outside [lo, hi) and
 * copies them to out (at most cap; returns how many, -2 if cap is too small), and
 * orc_births_add appends ionizations recorded by another subdomain's loop in this
 * subdomain's cells: their products are made here, with the step's own, in the order
 * of their parents' ids. */
typedef struct {
    uint32_t parent;          /* the ionizing particle's id */
    int32_t esp, isp, psp;    /* species of the new electron, of the new ion (-1: a
                                 converted target), of the process's product ion */
    int32_t cell;             /* where the products appear */
    double off, yp;
    double e[3], i[3];        /* their velocities (cells per own step) */
} orc_birth_rec;
int orc_step_loop(orc_sim* s);
int orc_step_finish(orc_sim* s);
int64_t orc_births_take(orc_sim* s, int32_t lo, int32_t hi, orc_birth_rec* out, int64_t cap);
int orc_births_add(orc_sim* s, const orc_birth_rec* in, int64_t n);

/* The parent ids of the last step's ionizations in ascending order (the order in which
 * their children were numbered: the r-th parent's children have the r-th ids after the
 * step's first new id).  Writes at most cap of them (parents may be NULL) and returns
 * how many there were, or -1.  A run split into subdomains renumbers its children by
 * the rank of their parent among every subdomain's parents. */
int64_t orc_last_parents(const orc_sim* s, uint32_t* parents, int64_t cap);

int64_t orc_count(const orc_sim* s, int32_t sp);
/* Copy out species sp sorted by ascending id (capacity = orc_count); yp (cell units)
 * is 0 for a species without sn2d. */
int orc_get(const orc_sim* s, int32_t sp, int32_t* cell, double* off, double* vx,
            double* vy, double* vz, uint32_t* id, uint8_t* mcc, double* yp);

typedef struct {
    int64_t step;
    int64_t live[ORC_MAX_SPECIES];
    int64_t wall_count[ORC_MAX_SPECIES][2];   /* [species][left,right] */
    double wall_energy[ORC_MAX_SPECIES][2];   /* sum of w * m v^2 / 2 */
    int64_t collisions[ORC_MAX_PROC];         /* real (non-null) events per process */
    double kinetic[ORC_MAX_SPECIES];          /* sum of w * m v^2 / 2 */
} orc_moments;

/* Scalars, plus (when non-NULL) node arrays of length N+1: per-species number
 * density (species-major, nspecies*(N+1)), potential and field of the current step. */
int orc_moments_get(orc_sim* s, orc_moments* m, double* density, double* phi, double* E);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the published
 * round function. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Density smoother: 1-2-1 binomial filter of rho[1..N-1] in place (N+1 entries; the
 * wall entries rho[0], rho[N] are kept), formed in binary128 and rounded once. */
void orc_smooth(int32_t N, double* rho);

/* Dirichlet Poisson problem of the field phase: -phi[j-1]+2phi[j]-phi[j+1] =
 * dx^2 rho[j]/eps0 for 1<=j<=N-1, phi[0]=phi[N]=0, by the Thomas algorithm, then
 * E = -grad(phi) (centred inside, Gauss half cell at the walls).  The recurrences and
 * E are carried in IEEE binary128 and rounded to FP64 once.  rho has N+1 entries;
 * rho[0], rho[N] are half-cell (wall) densities.  Returns 0 or < 0. */
int orc_poisson(int32_t N, double dx, double eps0, const double* rho, double* phi, double* E);

#ifdef __cplusplus
}
#endif
#endif
