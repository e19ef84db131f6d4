/*
 * oracle.c -- plain FP64 CPU oracle of the 1D3V PIC Monte Carlo time step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline timing).  Independent of
 * the GPU library: no shared code, headers, tables or helpers.
 *
 * What one time step computes, in the order this oracle takes it (the paper's PIC
 * cycle, Section 2 and Fig. "diagram"; the gather/update of Listing 7):
 *   for every live particle, species by species, in ascending id order:
 *     1. gather   a = A[j] + f*(A[j+1]-A[j])        (Listing 7, moveb(): linear gather
 *                                                    of the pre-scaled acceleration A;
 *                                                    f*(...) + A[j] is one fma)
 *     2. push     u += a (B = 0), or the Boris rotation (B != 0)   (Section 2, mover)
 *     3. move     f += u; the integer part of f moves the particle across cells
 *                 (Listing 7: x += nstep*vx with x the in-cell offset); a 2-D species
 *                 also drifts in y (Listing 1: yp += nstep*vy)
 *     4. wall     absorbing walls with flux counters, periodic, or absorption followed
 *                 by volume re-injection                 (Section 2, plasma-wall phase)
 *     5. MCC      null-collision Monte Carlo against a uniform neutral background
 *                                                        (Section 2, collision phase)
 *   then the particles created by ionization are appended,
 *   then the cloud-in-cell charge deposit (Section 2, density phase),
 *   then the Poisson solve by the Thomas algorithm and E = -grad(phi) (Section 2, field
 *   solver: "in 1D ... a tridiagonal matrix").
 *
 * The paper gives neither the push in a magnetic field, nor the collision model,
 * nor the interpolation weights, nor the wall treatment; the readings taken here are:
 * Boris (1970) rotation; null-collision MCC (Skullerud 1968, Vahedi & Surendra 1995)
 * whose candidate steps are drawn as geometric runs from Philox4x32-10 words with
 * integer thresholds, and whose process selection uses fixed integer slots; linear
 * (CIC) weights;
 * Gauss's law over the half cell at the wall nodes.  All particle arithmetic is FP64
 * and the file is compiled without floating-point contraction; the fused operations
 * are the explicit fma() calls of the gather and the Boris cross products (the paper
 * does not fix how a product-sum rounds; a C compiler on FMA hardware contracts it to
 * one rounding).  The density and field phases run in binary128 (the node sums of the
 * CIC weights, the charge density, the Poisson solve and E) and round E and phi to
 * FP64 once, so the field is the exact solution of the discrete problem for the
 * particles' positions to within that rounding (see deposit() and orc_poisson).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* IEEE binary128 for the density and field phases: long double where it is binary128
 * (aarch64 Linux), else GCC's _Float128 (x86_64; +, -, *, / in libgcc's soft float). */
#if defined(__LDBL_MANT_DIG__) && __LDBL_MANT_DIG__ == 113
typedef long double quad;
#else
typedef _Float128 quad;
#endif
_Static_assert(sizeof(quad) == 16, "binary128 expected");

#define TWO_PI 6.283185307179586476925286766559
#define ORC_GAP_MAX 127
#define TWO32 4294967296.0

/* ------------------------------------------------------------------------- */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11, Section 4.  One round: two 32x32->64 multiplications of counter
 * words 0 and 2 by the round multipliers; the new words are
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
 * and the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = M0 * (uint64_t)c0;
        uint64_t p1 = M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw of one purpose for one particle in one step: counter (id, step_hi, step_lo,
 * purpose), key = seed. */
static void draw(const orc_sim* s, uint32_t id, int64_t step, uint32_t purpose, uint32_t w[4]);

/* 32-bit word -> uniform double on the open interval (0,1): (w + 1/2) / 2^32. */
static double uniform(uint32_t w) { return ((double)w + 0.5) / TWO32; }

/* Box-Muller (1958): two uniforms -> two standard normals. */
static void box_muller(uint32_t wa, uint32_t wb, double* z0, double* z1)
{
    double r = sqrt(-2.0 * log(uniform(wa)));
    double th = TWO_PI * uniform(wb);
    *z0 = r * cos(th);
    *z1 = r * sin(th);
}

/* Unit vector uniform on the sphere: cos(theta) = 1 - 2 u0 about the x axis (the wall
 * normal), azimuth 2 pi u1. */
static void iso_dir(uint32_t w0, uint32_t w1, double n[3])
{
    double ct = 1.0 - 2.0 * uniform(w0);
    double st = sqrt(1.0 - ct * ct);
    double ph = TWO_PI * uniform(w1);
    n[0] = ct;
    n[1] = st * cos(ph);
    n[2] = st * sin(ph);
}

/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n, cap;
    int32_t* cell;
    double* off;
    double *ux, *uy, *uz; /* cells per step */
    uint32_t* id;
    unsigned char* alive;
    uint8_t* mcc;  /* collision clock: bits 0-6 steps to skip, bit 7 candidate pending */
    double* yp;    /* y coordinate in cell units (Listing 1's yp; 0 unless sn2d) */
} orc_store;

typedef struct {
    uint32_t parent;    /* parent id: children are numbered by the rank of this id */
    int32_t esp, isp;   /* species of the new electron and of the new ion (-1: the ion is
                           a converted target particle) */
    int32_t psp;        /* product ion species of the process */
    int32_t cell;
    double off;
    double yp;          /* the parent's y coordinate */
    double e[3], i[3];  /* velocities (cells per step) */
} orc_birth;

struct orc_sim {
    orc_params p;
    int32_t N;
    int64_t step;
    uint32_t next_id;
    orc_store st[ORC_MAX_SPECIES];
    /* per-species constants, derived once from the parameters */
    double accel[ORC_MAX_SPECIES];   /* c_s: A = c_s * E (cells/step^2 per unit E) */
    double tvec[ORC_MAX_SPECIES][3]; /* Boris t = (q/m) B dt/2 */
    double svec[ORC_MAX_SPECIES][3]; /* Boris s = 2 t / (1 + t.t) */
    double kefac[ORC_MAX_SPECIES];   /* w m (dx/dt)^2 / 2: energy per (cells/step)^2 */
    double vinj[ORC_MAX_SPECIES];    /* sqrt(T_s/m_s) in cells/step */
    /* (with subcycling every "step" of a species above is its own step K dt) */
    int collides[ORC_MAX_SPECIES];   /* species has collision processes */
    uint32_t gapT[ORC_MAX_SPECIES][ORC_GAP_MAX + 1]; /* floor((1-P)^g 2^32), g = 1..127 */
    uint64_t slot_end[ORC_MAX_PROC]; /* cumulative slot bound of each process */
    double thr_u2[ORC_MAX_PROC];     /* energy threshold as |u|^2 */
    double vneutral[ORC_MAX_SPECIES]; /* sqrt(T_n/m_n) in cells per step of the species */
    int64_t nstep[ORC_MAX_SPECIES];  /* subcycling factor K >= 1 */
    double vs[ORC_MAX_SPECIES];      /* physical velocity -> cells per step of the species */
    int has_B;
    /* neutral target species (p.target = k+1): per cell j, the live target particles
     * whose cell was j at the start of the step, as positions in the target store in
     * ascending id order (tfirst[j] .. tfirst[j+1]-1 of tlist) */
    int64_t* tlist;
    int64_t* tfirst;
    int64_t tcap;
    /* grid */
    quad* dens;     /* nspecies * (N+1): summed CIC weights per node (binary128) */
    double* A;      /* nspecies * (N+1): pre-scaled acceleration on nodes */
    double *phi, *E;
    quad* rho;      /* N+1: charge density of the field phase (binary128) */
    int fields_ready;
    /* counters */
    int64_t wall_count[ORC_MAX_SPECIES][2];
    double wall_energy[ORC_MAX_SPECIES][2];
    int64_t collisions[ORC_MAX_PROC];
    /* births of the current step */
    orc_birth* births;
    int64_t nbirths, capbirths;
    int in_step;  /* between orc_step_loop and orc_step_finish */
};

static void draw(const orc_sim* s, uint32_t id, int64_t step, uint32_t purpose, uint32_t w[4])
{
    uint32_t ctr[4] = {id, (uint32_t)((uint64_t)step >> 32), (uint32_t)step, purpose};
    uint32_t key[2] = {(uint32_t)s->p.seed, (uint32_t)(s->p.seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

static int store_reserve(orc_store* a, int64_t cap)
{
    if (cap <= a->cap) return 0;
    int64_t nc = a->cap ? a->cap : 16;
    while (nc < cap) nc *= 2;
    void* p;
#define GROW(f, T) p = realloc(a->f, (size_t)nc * sizeof(T)); if (!p) return -2; a->f = (T*)p;
    GROW(cell, int32_t) GROW(off, double) GROW(ux, double) GROW(uy, double)
    GROW(uz, double) GROW(id, uint32_t) GROW(alive, unsigned char) GROW(mcc, uint8_t)
    GROW(yp, double)
#undef GROW
    a->cap = nc;
    return 0;
}

static void store_free(orc_store* a)
{
    free(a->cell); free(a->off); free(a->ux); free(a->uy); free(a->uz);
    free(a->id); free(a->alive); free(a->mcc); free(a->yp);
    memset(a, 0, sizeof(*a));
}

orc_sim* orc_create(const orc_params* p)
{
    if (!p || p->ncells < 1 || p->nspecies < 1 || p->nspecies > ORC_MAX_SPECIES ||
        p->nproc < 0 || p->nproc > ORC_MAX_PROC || !(p->dx > 0) || !(p->dt > 0) ||
        !(p->eps0 > 0) || p->bc < 0 || p->bc > 2 || p->field < 0 || p->field > 2)
        return NULL;
    if (p->bc == ORC_BC_PERIODIC && p->field == ORC_FIELD_POISSON) return NULL;
    for (int k = 0; k < p->nproc; ++k) {
        const orc_process* q = &p->proc[k];
        if (q->species < 0 || q->species >= p->nspecies || !(q->nu >= 0)) return NULL;
        if (q->kind == ORC_PROC_ELASTIC && !(p->sp[q->species].mass <= 0.25 * p->m_neutral))
            return NULL;
        if (q->kind == ORC_PROC_IONIZE && (q->product < 0 || q->product >= p->nspecies))
            return NULL;
        if (q->kind < 0 || q->kind > 3) return NULL;
    }
    if (p->target < 0 || p->target > p->nspecies) return NULL;
    if (p->target > 0 && (p->sp[p->target - 1].charge != 0.0 || p->nref < 1)) return NULL;
    for (int i = 0; i < p->nspecies; ++i)
        if (!(p->sp[i].mass > 0) || p->sp[i].nstep < 0 || p->sp[i].nstep > 4096 ||
            p->sp[i].sn2d < 0 || p->sp[i].sn2d > 1)
            return NULL;

    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = p->ncells;
    const int N = s->N, S = p->nspecies;
    s->dens = (quad*)calloc((size_t)S * (N + 1), sizeof(quad));
    s->A = (double*)calloc((size_t)S * (N + 1), sizeof(double));
    s->phi = (double*)calloc((size_t)(N + 1), sizeof(double));
    s->E = (double*)calloc((size_t)(N + 1), sizeof(double));
    s->rho = (quad*)calloc((size_t)(N + 1), sizeof(quad));
    if (!s->dens || !s->A || !s->phi || !s->E || !s->rho) {
        orc_destroy(s);
        return NULL;
    }

    const double Bsq = p->B[0] * p->B[0] + p->B[1] * p->B[1] + p->B[2] * p->B[2];
    s->has_B = Bsq > 0.0;
    for (int i = 0; i < S; ++i) {
        const orc_species* q = &p->sp[i];
        /* subcycling: the species' own time step is K dt (Listing 7's nstep) */
        s->nstep[i] = q->nstep > 1 ? q->nstep : 1;
        const double dt = (double)s->nstep[i] * p->dt;
        const double vs = dt / p->dx; /* physical velocity -> cells per step */
        s->vs[i] = vs;
        const double qm = q->charge / q->mass;
        s->accel[i] = qm * (dt * dt / p->dx);
        const double qmh = qm * (0.5 * dt);
        for (int k = 0; k < 3; ++k) s->tvec[i][k] = qmh * p->B[k];
        const double tt = s->tvec[i][0] * s->tvec[i][0] + s->tvec[i][1] * s->tvec[i][1] +
                          s->tvec[i][2] * s->tvec[i][2];
        const double sf = 2.0 / (1.0 + tt);
        for (int k = 0; k < 3; ++k) s->svec[i][k] = sf * s->tvec[i][k];
        const double dxdt = p->dx / dt;
        s->kefac[i] = 0.5 * q->mass * q->weight * (dxdt * dxdt);
        s->vinj[i] = sqrt(q->temperature / q->mass) * vs;
        /* null-collision candidate probability over one step: 1 - exp(-nu_max dt) */
        double numax = 0.0;
        for (int k = 0; k < p->nproc; ++k)
            if (p->proc[k].species == i) numax += p->proc[k].nu;
        /* candidate steps form a Bernoulli sequence with P = 1 - exp(-nu_max dt); the
         * probability of g candidate-free steps in a row is (1-P)^g = exp(-g nu_max dt) */
        s->collides[i] = numax > 0.0;
        const double x = numax * dt;
        for (int g = 1; g <= ORC_GAP_MAX; ++g) {
            const double T = floor(exp(-(double)g * x) * TWO32);
            s->gapT[i][g] = T >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)T;
        }
        s->gapT[i][0] = 0xFFFFFFFFu;
        /* fixed slots of [0, 2^32) for the processes of this species, in list order */
        double cum = 0.0;
        int last = -1;
        for (int k = 0; k < p->nproc; ++k) {
            if (p->proc[k].species != i) continue;
            cum += p->proc[k].nu;
            s->slot_end[k] = (uint64_t)floor(cum / numax * TWO32);
            last = k;
        }
        if (last >= 0) s->slot_end[last] = (uint64_t)1 << 32;
    }
    for (int k = 0; k < p->nproc; ++k) {
        const int sp = p->proc[k].species;
        const double m = p->sp[sp].mass;
        s->thr_u2[k] = (2.0 * p->proc[k].threshold / m) * (s->vs[sp] * s->vs[sp]);
    }
    for (int i = 0; i < S; ++i)
        s->vneutral[i] = p->m_neutral > 0 ? sqrt(p->T_neutral / p->m_neutral) * s->vs[i] : 0.0;
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int i = 0; i < ORC_MAX_SPECIES; ++i) store_free(&s->st[i]);
    free(s->dens); free(s->A); free(s->phi); free(s->E); free(s->rho); free(s->births);
    free(s->tlist); free(s->tfirst);
    free(s);
}

typedef struct { uint32_t id; int64_t at; } id_at;
static int cmp_id_at(const void* a, const void* b)
{
    const id_at *x = (const id_at*)a, *y = (const id_at*)b;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return x->at < y->at ? -1 : (x->at > y->at);
}

int orc_load(orc_sim* s, int32_t sp, int64_t n, const int32_t* cell, const double* off,
             const double* vx, const double* vy, const double* vz, const uint32_t* id,
             const uint8_t* mcc, const double* yp)
{
    if (!s || sp < 0 || sp >= s->p.nspecies || n < 0) return -1;
    if (n > 0 && (!cell || !off || !vx || !vy || !vz)) return -1;
    for (int64_t k = 0; k < n; ++k)
        if (cell[k] < 0 || cell[k] >= s->N || !(off[k] >= 0.0 && off[k] < 1.0)) return -1;
    orc_store* a = &s->st[sp];
    a->n = 0;
    if (store_reserve(a, n > 0 ? n : 1)) return -2;
    id_at* order = (id_at*)malloc((size_t)(n > 0 ? n : 1) * sizeof(id_at));
    if (!order) return -2;
    for (int64_t k = 0; k < n; ++k) {
        order[k].id = id ? id[k] : s->next_id + (uint32_t)k;
        order[k].at = k;
    }
    qsort(order, (size_t)n, sizeof(id_at), cmp_id_at);
    const double vs = s->vs[sp];
    for (int64_t r = 0; r < n; ++r) {
        int64_t k = order[r].at;
        a->cell[r] = cell[k];
        a->off[r] = off[k];
        a->ux[r] = vx[k] * vs;
        a->uy[r] = vy[k] * vs;
        a->uz[r] = vz[k] * vs;
        a->id[r] = order[r].id;
        a->alive[r] = 1;
        a->mcc[r] = mcc ? mcc[k] : 0;
        a->yp[r] = (yp && s->p.sp[sp].sn2d) ? yp[k] : 0.0;
        if (order[r].id >= s->next_id) s->next_id = order[r].id + 1;
    }
    a->n = n;
    free(order);
    s->fields_ready = 0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Density phase: cloud-in-cell weights, (1-f) to node j and f to node j+1, summed in
 * ascending id order per species.  The weights and their sums are carried in binary128:
 * 1 - f is exact there, and a node's sum of a few thousand weights of 53 bits stays
 * within the 113-bit significand, so the node densities are the exact sums (an FP64
 * sum of n weights errs by ~sqrt(n) ulp per node, which the field integrates over the
 * N nodes). */
static void deposit(orc_sim* s)
{
    const int N = s->N;
    for (int sp = 0; sp < s->p.nspecies; ++sp) {
        quad* d = s->dens + (size_t)sp * (N + 1);
        for (int j = 0; j <= N; ++j) d[j] = 0;
        const orc_store* a = &s->st[sp];
        for (int64_t k = 0; k < a->n; ++k) {
            if (!a->alive[k]) continue;
            const int j = a->cell[k];
            const quad f = (quad)a->off[k];
            d[j] += (quad)1 - f;
            d[j + 1] += f;
        }
        if (s->p.bc == ORC_BC_PERIODIC) { /* node N is node 0 */
            d[0] += d[N];
            d[N] = d[0];
        }
    }
}

/* The Poisson solve and E of the field phase for a binary128 charge density (see
 * orc_poisson). */
static int poisson_q(int32_t N, double dx, double eps0, const quad* rho, double* phi, double* E)
{
    const int M = N - 1; /* interior unknowns phi[1..N-1] */
    /* The Thomas algorithm is backward stable, but its forward error in phi grows with
     * the condition number of the tridiagonal matrix (~N^2): in FP64 it reaches ~1e-11
     * of the field at N = 8192.  The recurrences are therefore carried in binary128
     * (113-bit significand; the same error bound is then ~1e-26 at N = 65536) and every
     * result is rounded to FP64 once, at the end: phi and E are the exact solution of
     * the discrete problem for this rho, to within the final rounding. */
    quad* q = (quad*)malloc((size_t)(N + 1) * sizeof(quad));   /* phi in binary128 */
    quad* cp = (quad*)malloc((size_t)(N + 1) * sizeof(quad));
    quad* dp = (quad*)malloc((size_t)(N + 1) * sizeof(quad));
    if (!q || !cp || !dp) { free(q); free(cp); free(dp); return -2; }
    q[0] = 0;
    q[N] = 0;
    if (M >= 1) {
        /* Thomas algorithm on a_i = -1, b_i = 2, c_i = -1, d_i = dx^2 rho_i / eps0 */
        const quad a = -1, b = 2, c = -1;
        const quad h2 = (quad)dx * (quad)dx / (quad)eps0;
        cp[1] = c / b;
        dp[1] = h2 * rho[1] / b;
        for (int i = 2; i <= M; ++i) {
            const quad di = h2 * rho[i];
            const quad m = b - a * cp[i - 1];
            cp[i] = c / m;
            dp[i] = (di - a * dp[i - 1]) / m;
        }
        q[M] = dp[M];
        for (int i = M - 1; i >= 1; --i) q[i] = dp[i] - cp[i] * q[i + 1];
    }
    /* E = -dphi/dx: centred inside; at a wall node Gauss's law over the half cell
     * next to the wall, whose charge per area is rho_wall * dx/2. */
    const quad qdx = (quad)dx, half = (quad)dx / (2 * (quad)eps0);
    for (int j = 1; j < N; ++j) E[j] = (double)((q[j - 1] - q[j + 1]) / (2 * qdx));
    E[0] = (double)(-(q[1] - q[0]) / qdx - rho[0] * half);
    E[N] = (double)(-(q[N] - q[N - 1]) / qdx + rho[N] * half);
    for (int j = 0; j <= N; ++j) phi[j] = (double)q[j];
    free(q);
    free(cp);
    free(dp);
    return 0;
}

int orc_poisson(int32_t N, double dx, double eps0, const double* rho, double* phi, double* E)
{
    if (N < 1 || !rho || !phi || !E || !(dx > 0) || !(eps0 > 0)) return -1;
    quad* r = (quad*)malloc((size_t)(N + 1) * sizeof(quad));
    if (!r) return -2;
    for (int j = 0; j <= N; ++j) r[j] = (quad)rho[j];
    const int rc = poisson_q(N, dx, eps0, r, phi, E);
    free(r);
    return rc;
}

/* Density smoother (Section 2's "Density Smoother" phase): a 1-2-1 binomial filter
 * of the interior node densities rho[1..N-1], the wall nodes (half cells) kept. */
static void smooth_q(int32_t N, quad* rho)
{
    if (N < 2) return;
    const quad quarter = (quad)0.25, halfq = (quad)0.5;
    quad prev = rho[0];
    for (int j = 1; j < N; ++j) {
        const quad cur = rho[j];
        rho[j] = quarter * prev + halfq * cur + quarter * rho[j + 1];
        prev = cur;
    }
}

void orc_smooth(int32_t N, double* rho)
{
    if (N < 2) return;
    quad* r = (quad*)malloc((size_t)(N + 1) * sizeof(quad));
    if (!r) return;
    for (int j = 0; j <= N; ++j) r[j] = (quad)rho[j];
    smooth_q(N, r);
    for (int j = 0; j <= N; ++j) rho[j] = (double)r[j];
    free(r);
}

/* Field phase: charge density from the deposit, Poisson solve, then the pre-scaled
 * accelerations A_s = c_s E used by the gather. */

static int solve_fields(orc_sim* s)
{
    const int N = s->N, S = s->p.nspecies;
    const double dx = s->p.dx;
    if (s->p.field == ORC_FIELD_POISSON) {
        for (int j = 0; j <= N; ++j) {
            quad q = 0;
            for (int sp = 0; sp < S; ++sp)
                q += (quad)s->p.sp[sp].charge * (quad)s->p.sp[sp].weight *
                     s->dens[(size_t)sp * (N + 1) + j];
            /* interior node: cell volume dx; wall node: half cell */
            s->rho[j] = (j == 0 || j == N) ? q / ((quad)0.5 * (quad)dx) : q / (quad)dx;
        }
        if (s->p.smooth) smooth_q(N, s->rho);
        int rc = poisson_q(N, dx, s->p.eps0, s->rho, s->phi, s->E);
        if (rc) return rc;
    } else {
        const double e = s->p.field == ORC_FIELD_EXTERNAL ? s->p.E_ext : 0.0;
        for (int j = 0; j <= N; ++j) {
            s->E[j] = e;
            s->phi[j] = -e * ((double)j * dx);
            s->rho[j] = 0;
        }
    }
    for (int sp = 0; sp < S; ++sp)
        for (int j = 0; j <= N; ++j) s->A[(size_t)sp * (N + 1) + j] = s->accel[sp] * s->E[j];
    s->fields_ready = 1;
    return 0;
}

static int ensure_fields(orc_sim* s)
{
    if (s->fields_ready) return 0;
    deposit(s);
    return solve_fields(s);
}

static int add_birth(orc_sim* s, const orc_birth* b)
{
    if (s->nbirths == s->capbirths) {
        int64_t nc = s->capbirths ? 2 * s->capbirths : 64;
        void* p = realloc(s->births, (size_t)nc * sizeof(orc_birth));
        if (!p) return -2;
        s->births = (orc_birth*)p;
        s->capbirths = nc;
    }
    s->births[s->nbirths++] = *b;
    return 0;
}

static int cmp_birth(const void* a, const void* b)
{
    const orc_birth *x = (const orc_birth*)a, *y = (const orc_birth*)b;
    return x->parent < y->parent ? -1 : (x->parent > y->parent);
}

/* Number of candidate-free steps, counted from the current one, that the word w
 * encodes: g = #{k in 1..127 : w < floor((1-P)^k 2^32)}, so P(g >= k) = (1-P)^k
 * (geometric, truncated at 127). */
static int gap_steps(const orc_sim* s, int sp, uint32_t w)
{
    int g = 0;
    for (int k = 1; k <= ORC_GAP_MAX; ++k) {
        if (w < s->gapT[sp][k]) g = k;
        else break;
    }
    return g;
}

static int candidate(orc_sim* s, int sp, orc_store* a, int64_t k, uint32_t wsel,
                     uint32_t wdens);

/* The clock of a particle whose next event step is a test on its own step m1 (after a
 * candidate, a re-injection or a conversion into an ion): that test taken now, from
 * the draw of its own step, since its outcome depends on the id and the step alone —
 * the count from m1 to the event it schedules (a candidate g steps on, g < D, or the
 * test at the next multiple of 127, g = D), exactly as the test on m1 would set it,
 * one step earlier.  A species without collisions keeps clock 0. */
static uint8_t clock_after(orc_sim* s, int sp, uint32_t id, int64_t m1)
{
    if (!s->collides[sp]) return 0;
    const int64_t n1 = (m1 + 1) * s->nstep[sp] - 1;  /* the global step of own step m1 */
    uint32_t w[4];
    draw(s, id, n1, ORC_RNG_COLLIDE, w);
    const int D = ORC_GAP_MAX - (int)(m1 % ORC_GAP_MAX);
    int g = gap_steps(s, sp, w[0]);
    if (g > D) g = D;
    return (uint8_t)(g | (g < D ? 0x80 : 0));
}

/* own index of the first step >= n on which species sp moves */
static int64_t own_from(const orc_sim* s, int sp, int64_t n)
{
    const int64_t K = s->nstep[sp];
    return (n + K) / K - 1;
}

/* Collision phase for one particle (null-collision MCC).  Whether a step holds a
 * collision candidate is a Bernoulli(P) sequence per particle; instead of one draw per
 * step the particle carries its clock: C steps to skip, and whether the next event
 * step is a candidate.  At an event step without a pending candidate (a test) the
 * draw COLLIDE(id, step) word 0 gives the candidate-free run g starting at this step,
 * cut at the next step that is a multiple of 127 (D steps away): g = 0 is a candidate
 * now, 0 < g < D a candidate g steps later, g = D none before that step, which then
 * tests again.  (The cut keeps the tests of all particles on the same steps, and by
 * the memorylessness of the sequence changes nothing in its distribution.)  A
 * candidate selects its process with word 1 of COLLIDE(id, step) of its own step; the
 * step after a candidate is a test.  Returns 0 or < 0. */
static int collide(orc_sim* s, int sp, orc_store* a, int64_t k)
{
    if (!s->collides[sp]) return 0;
    const uint8_t m = a->mcc[k];
    const int C = m & 0x7F, pending = m >> 7;
    if (C > 0) {
        a->mcc[k] = (uint8_t)((C - 1) | (pending << 7));
        return 0;
    }
    uint32_t w[4];
    draw(s, a->id[k], s->step, ORC_RNG_COLLIDE, w);
    if (!pending) {
        /* the grid of test steps counts the species' own steps ((step+1)/K - 1) */
        const int64_t own = (s->step + 1) / s->nstep[sp] - 1;
        const int D = ORC_GAP_MAX - (int)(own % ORC_GAP_MAX);
        int g = gap_steps(s, sp, w[0]);
        if (g > D) g = D;
        if (g == D) {
            a->mcc[k] = (uint8_t)(D - 1);
            return 0;
        }
        if (g > 0) {
            a->mcc[k] = (uint8_t)((g - 1) | 0x80);
            return 0;
        }
    }
    /* the step after a candidate is a test */
    a->mcc[k] = clock_after(s, sp, a->id[k], own_from(s, sp, s->step + 1));
    return candidate(s, sp, a, k, w[1], w[2]);
}

/* A collision candidate: with a particle target, first the target density: kept with
 * probability min(1, n_j / nref) by the word wdens against floor(n_j 2^32 / nref) (n_j
 * the live target particles whose cell was j at the start of the step, j the
 * candidate's cell); then the process slot from the selection word, the energy
 * threshold (below it the event is a null collision), kinematics. */
static int candidate(orc_sim* s, int sp, orc_store* a, int64_t k, uint32_t wsel,
                     uint32_t wdens)
{
    const uint32_t id = a->id[k];
    if (s->p.target) {
        const int j = a->cell[k];
        const uint64_t nj = (uint64_t)(s->tfirst[j + 1] - s->tfirst[j]);
        const uint64_t nr = (uint64_t)s->p.nref;
        if (nj < nr && (uint64_t)wdens >= (nj << 32) / nr) return 0;
    }
    int proc = -1;
    for (int q = 0; q < s->p.nproc; ++q) {
        if (s->p.proc[q].species != sp) continue;
        if ((uint64_t)wsel < s->slot_end[q]) { proc = q; break; }
    }
    if (proc < 0) return 0;
    double ux = a->ux[k], uy = a->uy[k], uz = a->uz[k];
    const double u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 >= s->thr_u2[proc])) return 0; /* below threshold: null collision */
    const orc_process* P = &s->p.proc[proc];
    uint32_t r[4];
    if (P->kind == ORC_PROC_ELASTIC) {
        /* isotropic new direction n; speed loss for the scattering angle chi between
         * the old and the new direction: |u'| = |u| sqrt(1 - 2 (m/M)(1 - cos chi)) */
        draw(s, id, s->step, ORC_RNG_SCATTER, r);
        double n[3];
        iso_dir(r[0], r[1], n);
        const double speed = sqrt(u2);
        if (speed > 0.0) {
            const double cchi = (ux * n[0] + uy * n[1] + uz * n[2]) / speed;
            const double mr = s->p.sp[sp].mass / s->p.m_neutral;
            const double fac = sqrt(1.0 - 2.0 * mr * (1.0 - cchi));
            const double sp2 = speed * fac;
            a->ux[k] = sp2 * n[0];
            a->uy[k] = sp2 * n[1];
            a->uz[k] = sp2 * n[2];
        }
    } else if (P->kind == ORC_PROC_CX) {
        /* charge exchange: the ion takes the velocity of a background neutral */
        draw(s, id, s->step, ORC_RNG_MAXWELL, r);
        double z0, z1, z2, z3;
        box_muller(r[0], r[1], &z0, &z1);
        box_muller(r[2], r[3], &z2, &z3);
        a->ux[k] = z0 * s->vneutral[sp];
        a->uy[k] = z1 * s->vneutral[sp];
        a->uz[k] = z2 * s->vneutral[sp];
    } else if (P->kind == ORC_PROC_EXCITE) {
        /* excitation: the electron loses the threshold energy and leaves in a direction
         * uniform on the sphere */
        draw(s, id, s->step, ORC_RNG_SCATTER, r);
        double n[3];
        iso_dir(r[0], r[1], n);
        const double sp2 = sqrt(u2 - s->thr_u2[proc]);
        a->ux[k] = sp2 * n[0];
        a->uy[k] = sp2 * n[1];
        a->uz[k] = sp2 * n[2];
    } else { /* ORC_PROC_IONIZE */
        /* the incident electron pays the threshold; the rest is shared equally by the
         * two outgoing electrons, both isotropic; the ion is a background neutral */
        const double us = sqrt(0.5 * (u2 - s->thr_u2[proc]));
        double n1[3], n2[3];
        draw(s, id, s->step, ORC_RNG_SCATTER, r);
        iso_dir(r[0], r[1], n1);
        draw(s, id, s->step, ORC_RNG_IONIZE_E, r);
        iso_dir(r[0], r[1], n2);
        uint32_t ri[4];
        draw(s, id, s->step, ORC_RNG_IONIZE_I, ri);
        double z0, z1, z2, z3;
        box_muller(ri[0], ri[1], &z0, &z1);
        box_muller(ri[2], ri[3], &z2, &z3);
        a->ux[k] = us * n1[0];
        a->uy[k] = us * n1[1];
        a->uz[k] = us * n1[2];
        orc_birth b;
        b.parent = id;
        b.esp = sp;
        /* with a particle target the ion is the converted target particle (after the
         * particle loop), not a new particle */
        b.isp = s->p.target ? -1 : P->product;
        b.psp = P->product;
        b.cell = a->cell[k];
        b.off = a->off[k];
        b.yp = a->yp[k];
        b.e[0] = us * n2[0]; b.e[1] = us * n2[1]; b.e[2] = us * n2[2];
        /* the ion's velocity in its own species' units */
        const double vn = s->vneutral[P->product];
        b.i[0] = z0 * vn; b.i[1] = z1 * vn; b.i[2] = z2 * vn;
        int rc = add_birth(s, &b);
        if (rc) return rc;
    }
    s->collisions[proc] += 1;
    return 0;
}

/* Volume source: the absorbed particle re-enters at a uniform position with a
 * Maxwellian velocity of its species' source temperature. */
static void reinject(orc_sim* s, int sp, orc_store* a, int64_t k)
{
    uint32_t r[4], q[4];
    draw(s, a->id[k], s->step, ORC_RNG_INJECT_A, r);
    draw(s, a->id[k], s->step, ORC_RNG_INJECT_B, q);
    const double x = uniform(r[0]) * (double)s->N;
    double fl = floor(x);
    int j = (int)fl;
    double f = x - fl;
    if (j >= s->N) { j = s->N - 1; f = 0.0; }
    double z0, z1, z2, z3;
    box_muller(r[1], r[2], &z0, &z1);
    box_muller(q[0], q[1], &z2, &z3);
    a->cell[k] = j;
    a->off[k] = f;
    a->mcc[k] = clock_after(s, sp, a->id[k], own_from(s, sp, s->step + 1));
    a->yp[k] = 0.0; /* a re-injected particle starts its y coordinate anew */
    a->ux[k] = z0 * s->vinj[sp];
    a->uy[k] = z1 * s->vinj[sp];
    a->uz[k] = z2 * s->vinj[sp];
}

/* The live target particles by their cell at the start of the step, ascending ids
 * within a cell (the target store is kept in ascending id order). */
static int index_targets(orc_sim* s)
{
    const int N = s->N;
    const orc_store* a = &s->st[s->p.target - 1];
    if (a->n + 1 > s->tcap) {
        void* q = realloc(s->tlist, (size_t)(a->n + 1) * sizeof(int64_t));
        if (!q) return -2;
        s->tlist = (int64_t*)q;
        s->tcap = a->n + 1;
    }
    if (!s->tfirst) {
        s->tfirst = (int64_t*)calloc((size_t)N + 2, sizeof(int64_t));
        if (!s->tfirst) return -2;
    }
    memset(s->tfirst, 0, ((size_t)N + 2) * sizeof(int64_t));
    for (int64_t k = 0; k < a->n; ++k)
        if (a->alive[k]) s->tfirst[a->cell[k] + 1] += 1;
    for (int j = 0; j < N; ++j) s->tfirst[j + 1] += s->tfirst[j];
    int64_t* cur = (int64_t*)malloc(((size_t)N + 1) * sizeof(int64_t));
    if (!cur) return -2;
    memcpy(cur, s->tfirst, ((size_t)N + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < a->n; ++k)
        if (a->alive[k]) s->tlist[cur[a->cell[k]]++] = k;
    free(cur);
    return 0;
}

/* Reorder a store by ascending id (after target particles joined it as ions). */
static int store_sort_by_id(orc_store* a)
{
    if (a->n < 2) return 0;
    id_at* order = (id_at*)malloc((size_t)a->n * sizeof(id_at));
    orc_store b;
    memset(&b, 0, sizeof(b));
    if (!order || store_reserve(&b, a->n)) {
        free(order);
        store_free(&b);
        return -2;
    }
    for (int64_t k = 0; k < a->n; ++k) {
        order[k].id = a->id[k];
        order[k].at = k;
    }
    qsort(order, (size_t)a->n, sizeof(id_at), cmp_id_at);
    for (int64_t r = 0; r < a->n; ++r) {
        const int64_t k = order[r].at;
        b.cell[r] = a->cell[k]; b.off[r] = a->off[k];
        b.ux[r] = a->ux[k]; b.uy[r] = a->uy[k]; b.uz[r] = a->uz[k];
        b.id[r] = a->id[k]; b.alive[r] = a->alive[k]; b.mcc[r] = a->mcc[k];
        b.yp[r] = a->yp[k];
    }
    b.n = a->n;
    free(order);
    store_free(a);
    *a = b;
    return 0;
}

/* Ionization against the particle target: in each cell j, the r_j ionizations of the
 * step (r_j electrons of cell j) turn the first r_j live target particles of cell j
 * (as of the start of the step, smallest ids first) into product ions: same id,
 * position and physical velocity, collision clock 0.  A cell with fewer targets than
 * ionizations converts what it has. */
static int convert_targets(orc_sim* s)
{
    const int t = s->p.target - 1, N = s->N;
    orc_store* a = &s->st[t];
    int64_t* taken = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    if (!taken) return -2;
    int touched[ORC_MAX_SPECIES] = {0};
    for (int64_t r = 0; r < s->nbirths; ++r) {
        const orc_birth* b = &s->births[r];
        if (b->isp >= 0) continue;
        const int j = b->cell;
        if (taken[j] >= s->tfirst[j + 1] - s->tfirst[j]) continue;
        const int64_t v = s->tlist[s->tfirst[j] + taken[j]++];
        orc_store* ion = &s->st[b->psp];
        if (store_reserve(ion, ion->n + 1)) { free(taken); return -2; }
        const int64_t m = ion->n++;
        const double ratio = (double)s->nstep[b->psp] / (double)s->nstep[t];
        ion->cell[m] = a->cell[v];
        ion->off[m] = a->off[v];
        ion->ux[m] = a->ux[v] * ratio;
        ion->uy[m] = a->uy[v] * ratio;
        ion->uz[m] = a->uz[v] * ratio;
        ion->id[m] = a->id[v];
        ion->alive[m] = 1;
        ion->mcc[m] = clock_after(s, b->psp, a->id[v], own_from(s, b->psp, s->step + 1));
        ion->yp[m] = s->p.sp[b->psp].sn2d ? a->yp[v] : 0.0;
        a->alive[v] = 0;
        touched[b->psp] = 1;
    }
    free(taken);
    for (int sp = 0; sp < s->p.nspecies; ++sp)
        if (touched[sp] && store_sort_by_id(&s->st[sp])) return -2;
    return 0;
}

/* A time step in two halves: the particle loop (gather, push, move, walls, collisions;
 * the ionizations recorded as births), then creation, the target conversions, the
 * deposit and the field.  One step is the two in order; a run split into subdomains
 * hands births between them in the middle (orc_births_take / orc_births_add). */
static int step_loop(orc_sim* s)
{
    const int N = s->N, S = s->p.nspecies;
    int rc = ensure_fields(s);
    if (rc) return rc;
    s->nbirths = 0;
    if (s->p.target && (rc = index_targets(s))) return rc;
    for (int sp = 0; sp < S; ++sp) {
        /* subcycling: a species with factor K moves on the steps n with (n+1) mod K = 0,
         * so that all species meet at the multiples of K dt */
        if ((s->step + 1) % s->nstep[sp] != 0) continue;
        orc_store* a = &s->st[sp];
        const double* A = s->A + (size_t)sp * (N + 1);
        const double* t = s->tvec[sp];
        const double* sv = s->svec[sp];
        for (int64_t k = 0; k < a->n; ++k) {
            if (!a->alive[k]) continue;
            int j = a->cell[k];
            double f = a->off[k];
            /* 1. gather (Listing 7): A[j] + f (A[j+1] - A[j]), the product and the sum
             *    rounded once (fused multiply-add) */
            const double acc = fma(f, A[j + 1] - A[j], A[j]);
            /* 2. push */
            if (!s->has_B) {
                a->ux[k] = a->ux[k] + acc;
            } else {
                const double half = 0.5 * acc;
                const double mx = a->ux[k] + half, my = a->uy[k], mz = a->uz[k];
                /* v' = v + v x t, then v+ = v + v' x s, each component as two fused
                 * multiply-adds: m_x + m_y t_z - m_z t_y = fma(m_y, t_z, fma(-m_z, t_y, m_x)) */
                const double px = fma(my, t[2], fma(-mz, t[1], mx));
                const double py = fma(mz, t[0], fma(-mx, t[2], my));
                const double pz = fma(mx, t[1], fma(-my, t[0], mz));
                const double qx = fma(py, sv[2], fma(-pz, sv[1], mx));
                const double qy = fma(pz, sv[0], fma(-px, sv[2], my));
                const double qz = fma(px, sv[1], fma(-py, sv[0], mz));
                a->ux[k] = qx + half;
                a->uy[k] = qy;
                a->uz[k] = qz;
            }
            /* 3. move (Listing 7: x += nstep*vx, x the in-cell offset) */
            const double xn = f + a->ux[k];
            const double fl = floor(xn);
            f = xn - fl;
            j += (int)fl;
            if (f >= 1.0) { /* xn a tiny negative number: f rounded up to 1 */
                f = 0.0;
                j += 1;
            }
            a->cell[k] = j;
            a->off[k] = f;
            /* the y drift of a 2-D species (Listing 1: yp += nstep*vy, with the velocity
             * in cells per own step) */
            if (s->p.sp[sp].sn2d) a->yp[k] += a->uy[k];
            /* 4. walls */
            int reinjected = 0;
            if (j < 0 || j >= N) {
                if (s->p.bc == ORC_BC_PERIODIC) {
                    while (j < 0) j += N;
                    while (j >= N) j -= N;
                    a->cell[k] = j;
                } else {
                    const int wall = j < 0 ? 0 : 1;
                    const double u2 = a->ux[k] * a->ux[k] + a->uy[k] * a->uy[k] +
                                      a->uz[k] * a->uz[k];
                    s->wall_count[sp][wall] += 1;
                    s->wall_energy[sp][wall] += s->kefac[sp] * u2;
                    if (s->p.bc == ORC_BC_SOURCE) {
                        reinject(s, sp, a, k);
                        reinjected = 1;
                    } else {
                        a->alive[k] = 0;
                        continue;
                    }
                }
            }
            /* 5. Monte Carlo collisions */
            if (!reinjected) {
                rc = collide(s, sp, a, k);
                if (rc) return rc;
            }
        }
    }
    return 0;
}

static int step_finish(orc_sim* s)
{
    const int S = s->p.nspecies;
    int rc;
    /* creation: children numbered by the rank of the parent id among this step's
     * ionizing parents; electron 2r, ion 2r+1 after the largest id so far (with a
     * particle target only the electron is new: id r; the ion is a converted target) */
    if (s->nbirths > 0) {
        qsort(s->births, (size_t)s->nbirths, sizeof(orc_birth), cmp_birth);
        if (s->p.target && (rc = convert_targets(s))) return rc;
        const uint32_t base = s->next_id;
        const int per = s->p.target ? 1 : 2;
        for (int64_t r = 0; r < s->nbirths; ++r) {
            const orc_birth* b = &s->births[r];
            for (int c = 0; c < per; ++c) {
                const int sp = c == 0 ? b->esp : b->isp;
                const double* u = c == 0 ? b->e : b->i;
                orc_store* a = &s->st[sp];
                if (store_reserve(a, a->n + 1)) return -2;
                const int64_t k = a->n++;
                a->cell[k] = b->cell;
                a->off[k] = b->off;
                a->ux[k] = u[0];
                a->uy[k] = u[1];
                a->uz[k] = u[2];
                a->id[k] = base + (uint32_t)(per * r + c);
                a->alive[k] = 1;
                a->mcc[k] = 0;
                a->yp[k] = s->p.sp[sp].sn2d ? b->yp : 0.0;
            }
        }
        s->next_id = base + (uint32_t)(per * s->nbirths);
    }
    /* drop absorbed particles (ids stay ascending) */
    for (int sp = 0; sp < S; ++sp) {
        orc_store* a = &s->st[sp];
        int64_t m = 0;
        for (int64_t k = 0; k < a->n; ++k) {
            if (!a->alive[k]) continue;
            if (m != k) {
                a->cell[m] = a->cell[k]; a->off[m] = a->off[k];
                a->ux[m] = a->ux[k]; a->uy[m] = a->uy[k]; a->uz[m] = a->uz[k];
                a->id[m] = a->id[k]; a->alive[m] = 1; a->mcc[m] = a->mcc[k];
                a->yp[m] = a->yp[k];
            }
            ++m;
        }
        a->n = m;
    }
    deposit(s);
    rc = solve_fields(s);
    if (rc) return rc;
    s->step += 1;
    return 0;
}

static int one_step(orc_sim* s)
{
    int rc = step_loop(s);
    return rc ? rc : step_finish(s);
}

/* The field of the next step supplied by the caller (E on the N+1 nodes) in place of
 * the one the field phase formed: the gather then uses A_s = c_s E as usual.  A run split
 * into subdomains solves the field jointly and hands each part the result. */
int orc_set_field(orc_sim* s, const double* E)
{
    if (!s || !E) return -1;
    const int N = s->N, S = s->p.nspecies;
    for (int j = 0; j <= N; ++j) s->E[j] = E[j];
    for (int sp = 0; sp < S; ++sp)
        for (int j = 0; j <= N; ++j) s->A[(size_t)sp * (N + 1) + j] = s->accel[sp] * s->E[j];
    s->fields_ready = 1;
    return 0;
}

int orc_step(orc_sim* s, int64_t nsteps)
{
    if (!s || nsteps < 0 || s->in_step) return -1;
    for (int64_t n = 0; n < nsteps; ++n) {
        int rc = one_step(s);
        if (rc) return rc;
    }
    return 0;
}

int orc_set_step(orc_sim* s, int64_t step, uint32_t next_id)
{
    if (!s || step < 0) return -1;
    s->step = step;
    if (next_id > s->next_id) s->next_id = next_id;
    return 0;
}

int orc_step_loop(orc_sim* s)
{
    if (!s || s->in_step) return -1;
    int rc = step_loop(s);
    if (!rc) s->in_step = 1;
    return rc;
}

int orc_step_finish(orc_sim* s)
{
    if (!s || !s->in_step) return -1;
    s->in_step = 0;
    return step_finish(s);
}

int64_t orc_births_take(orc_sim* s, int32_t lo, int32_t hi, orc_birth_rec* out, int64_t cap)
{
    if (!s || !s->in_step || lo < 0 || hi > s->N || lo > hi || cap < 0) return -1;
    int64_t m = 0, k = 0;
    for (int64_t r = 0; r < s->nbirths; ++r) {
        const orc_birth* b = &s->births[r];
        if (b->cell >= lo && b->cell < hi) {
            s->births[m++] = *b;
            continue;
        }
        if (k >= cap) return -2;  /* (ask with cap large enough: at most nbirths) */
        orc_birth_rec* o = &out[k++];
        o->parent = b->parent;
        o->esp = b->esp; o->isp = b->isp; o->psp = b->psp; o->cell = b->cell;
        o->off = b->off; o->yp = b->yp;
        for (int c = 0; c < 3; ++c) { o->e[c] = b->e[c]; o->i[c] = b->i[c]; }
    }
    s->nbirths = m;
    return k;
}

int orc_births_add(orc_sim* s, const orc_birth_rec* in, int64_t n)
{
    if (!s || !s->in_step || n < 0 || (n > 0 && !in)) return -1;
    for (int64_t k = 0; k < n; ++k) {
        if (in[k].cell < 0 || in[k].cell >= s->N) return -1;
        orc_birth b;
        b.parent = in[k].parent;
        b.esp = in[k].esp; b.isp = in[k].isp; b.psp = in[k].psp; b.cell = in[k].cell;
        b.off = in[k].off; b.yp = in[k].yp;
        for (int c = 0; c < 3; ++c) { b.e[c] = in[k].e[c]; b.i[c] = in[k].i[c]; }
        int rc = add_birth(s, &b);
        if (rc) return rc;
    }
    return 0;
}

int64_t orc_last_parents(const orc_sim* s, uint32_t* parents, int64_t cap)
{
    if (!s || cap < 0) return -1;
    /* the births of the last step, sorted by parent id when their children were numbered */
    for (int64_t r = 0; parents && r < s->nbirths && r < cap; ++r) parents[r] = s->births[r].parent;
    return s->nbirths;
}

int64_t orc_count(const orc_sim* s, int32_t sp)
{
    if (!s || sp < 0 || sp >= s->p.nspecies) return -1;
    return s->st[sp].n;
}

int orc_get(const orc_sim* s, int32_t sp, int32_t* cell, double* off, double* vx,
            double* vy, double* vz, uint32_t* id, uint8_t* mcc, double* yp)
{
    if (!s || sp < 0 || sp >= s->p.nspecies) return -1;
    const orc_store* a = &s->st[sp];
    const double iv = s->p.dx / ((double)s->nstep[sp] * s->p.dt); /* cells per step -> physical */
    for (int64_t k = 0; k < a->n; ++k) {
        if (cell) cell[k] = a->cell[k];
        if (off) off[k] = a->off[k];
        if (vx) vx[k] = a->ux[k] * iv;
        if (vy) vy[k] = a->uy[k] * iv;
        if (vz) vz[k] = a->uz[k] * iv;
        if (id) id[k] = a->id[k];
        if (mcc) mcc[k] = a->mcc[k];
        if (yp) yp[k] = a->yp[k];
    }
    return 0;
}

int orc_moments_get(orc_sim* s, orc_moments* m, double* density, double* phi, double* E)
{
    if (!s || !m) return -1;
    int rc = ensure_fields(s);
    if (rc) return rc;
    const int N = s->N, S = s->p.nspecies;
    memset(m, 0, sizeof(*m));
    m->step = s->step;
    for (int sp = 0; sp < S; ++sp) {
        const orc_store* a = &s->st[sp];
        double ke = 0.0;
        int64_t live = 0;
        for (int64_t k = 0; k < a->n; ++k) {
            if (!a->alive[k]) continue;
            ++live;
            ke += s->kefac[sp] * (a->ux[k] * a->ux[k] + a->uy[k] * a->uy[k] + a->uz[k] * a->uz[k]);
        }
        m->live[sp] = live;
        m->kinetic[sp] = ke;
        for (int w = 0; w < 2; ++w) {
            m->wall_count[sp][w] = s->wall_count[sp][w];
            m->wall_energy[sp][w] = s->wall_energy[sp][w];
        }
        if (density) {
            const quad* d = s->dens + (size_t)sp * (N + 1);
            const quad wdx = (quad)s->p.sp[sp].weight / (quad)s->p.dx;
            for (int j = 0; j <= N; ++j) {
                const int wall = (j == 0 || j == N) && s->p.bc != ORC_BC_PERIODIC;
                density[(size_t)sp * (N + 1) + j] = (double)(wall ? 2 * wdx * d[j] : wdx * d[j]);
            }
        }
    }
    for (int q = 0; q < s->p.nproc; ++q) m->collisions[q] = s->collisions[q];
    if (phi) memcpy(phi, s->phi, (size_t)(N + 1) * sizeof(double));
    if (E) memcpy(E, s->E, (size_t)(N + 1) * sizeof(double));
    return 0;
}
