// engine.cu -- the handle behind the C ABI (include/pic.h): validation, memory
// layout, the per-step launch sequence and the synchronising queries.
//
// Launch sequence of one time step (all on the handle's stream):
//   k_tiles     snapshot each segment's slot count (rounded to a whole quad), build the
//               tile list, empty the rare-event queue
//   k_move      gather, push, move, periodic wrap, collision clock, fixed-point deposit;
//               walls and collision candidates are queued (mover.cuh)
//   k_events    the queued walls and candidates: counters, re-injection, kinematics,
//               creations (events.cuh)
//   k_victims   neutral particle targets: the ionized targets become ions (events.cuh)
//   k_births    number this step's ionization products (only with ionization)
//   k_field     exact integer Poisson solve (optional smoother) -> E -> node pairs of
//               pre-scaled accelerations, and hand-over of the deposit (field.cu)
//   the sort, every `sort_interval` steps: the step before counts the particles per cell
//   at its end (k_move's deposit, k_events); the sort step scans the counts
//   (k_cell_partial, k_cell_scan), its mover writes every particle into its cell-ordered
//   slot of the other store copy, and k_sort_finish adopts the new counts before
//   k_events.  Otherwise (neutral targets, sort interval 1, no counts from the step
//   before) the separate sort follows the step: k_tiles, histogram, scan, scatter.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include <sys/stat.h>

#include "kernels.h"
#include "mover.cuh"

using namespace bitpic;

namespace {

thread_local std::string g_create_error;

void mkdir_if_missing(const std::string& dir);

struct Store {
    int32_t* cell = nullptr;
    void* off = nullptr;
    void* ux = nullptr;
    void* uy = nullptr;
    void* uz = nullptr;
    uint32_t* id = nullptr;
    void* yp = nullptr;  // y coordinates of 2-D species (allocated only when some species has one)
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

void mkdir_if_missing(const std::string& dir)
{
    if (!dir.empty()) mkdir(dir.c_str(), 0755);  // fails harmlessly when it exists
}

}  // namespace

namespace bitpic {
// The message pic_last_error(NULL) returns (failed pic_create, pic_philox,
// pic_field_solve_noalloc).
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace bitpic

struct pic_handle {
    int precision = PIC_FP32;
    int ninst = 0, nseg = 0, sort_interval = 0, nt = 256, grid_move = 0, sms = 0;
    size_t tsize = 4;
    std::vector<pic_instance> inst;
    std::vector<SegParams> segh;
    std::vector<InstParams> insth;
    int64_t total_cap = 0, seg_nodes = 0, inst_nodes = 0, max_cap = 0, ev_total = 0;
    int64_t rare_cap = 0;  // entries of the per-step rare-event queue
    int max_nodes = 0;
    bool any_poisson = false, any_mag = false, any_ionize = false, any_subcycle = false;
    bool any_target = false;       // some instance collides with neutral particles
    bool any_unmag = false;        // some instance has no magnetic field
    bool any_sn2d = false;         // some species drifts in y (pic_species.sn2d)
    std::vector<int64_t> fresh_n;  // per segment: n of its last load while no step or field
                                   // phase has run since (-1 otherwise), for pic_load_yp
    unsigned *tcount = nullptr, *treq = nullptr;  // target segment node arrays
    int64_t* vlist = nullptr;                     // target nodes with requests this step
    int grid_victims = 0;

    SegParams* segd = nullptr;
    InstParams* instd = nullptr;
    Store st[2];
    int cur = 0;
    void* accel = nullptr;
    unsigned long long *dep = nullptr, *dep_last = nullptr;
    double* E = nullptr;
    int nchunks = 0;
    int* chunk_inst = nullptr;
    i128 *part_sum = nullptr, *part_w = nullptr, *zfirst = nullptr;
    i128* zs = nullptr;  // smoothed node charges (instances with the density smoother)
    bool any_smooth = false;
    unsigned* hist = nullptr;
    unsigned long long *newn = nullptr, *seg_n = nullptr, *seg_live = nullptr, *hwm_alt = nullptr;
    int64_t *seg_nmove = nullptr, *tile_start = nullptr;
    unsigned long long *wall_count = nullptr, *collisions = nullptr, *ev_count = nullptr,
                       *next_id = nullptr;
    uint32_t *birth_keys_a = nullptr, *birth_keys_b = nullptr;  // k_births: parent ids being sorted
    unsigned long long* cell_part = nullptr;  // sort: per segment and 4096-cell chunk
    int cell_chunks = 1;
    double* wall_energy = nullptr;
    Event* events = nullptr;
    uint64_t* rare = nullptr;
    unsigned long long* rare_count = nullptr;
    int grid_events = 0;
    unsigned* err = nullptr;
    // the step count: [0] the step the kernels of a step read (set from [1] by k_tiles,
    // the first kernel of every step), [1] the steps completed (the field phase of a
    // step writes [0] + 1), so that the field phase may run beside the event kernels
    int64_t* step_d = nullptr;
    int* test_all = nullptr;  // nonzero: every clock may need a test in the next step (after a load)
    int64_t pair_min = (int64_t)1 << 24;  // particle slots from which plain FP32 steps use the mover pair
    bool pair_ok = true;                  // every colliding species moves on every step
    double *kin = nullptr, *phi_d = nullptr;
    std::vector<void*> allocs;
    char* io = nullptr;       // staging of pic_load_particles / pic_get_particles host data
    size_t io_bytes = 0;

    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // read-back: device-to-host copies beside the writes
    // a step's event kernels run on side_stream beside its field phase when neither
    // touches what the other reads or writes (no deposit from the event kernels:
    // no volume source, no ionization, no neutral particle target); fork and join events
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool any_source = false;  // some instance re-injects through its walls (volume source)
    int64_t step_h = 0;
    bool stale = true;
    // the sort folded into the time step: the last step before a sort counted the
    // particles per cell into `hist` (cleared by anything that changes the store from
    // the host, and by the sort that used it); grid of the sorting mover
    bool hist_ready = false;
    int grid_sort = 0;
    int grid_test = 0;  // grid of the mover pair's inline-test partner (FP32, no subcycling)
    // threads per block of the step that ends a sort cycle, apart from the other steps':
    // its four block-wide barriers a chunk cost less in small blocks, while the plain
    // mover gains from large ones (196.6 M particles, FP32: the sort step 2.22 / 2.31 /
    // 2.57 ms at 128 / 256 / 512 threads, the plain mover 0.783 / 0.771 / 0.754 ms);
    // `$BITPIC_SORT_BLOCK` (128, 256 or 512) overrides it
    int nt_sort = 128;
    int state = PIC_OK;
    std::string last_error;

    // autotuning of the mover block size and the sort interval (see tune_step)
    bool tune_block = false, tune_sort = false;
    int tune_phase = 0;        // 0 idle/done, 1 block sizes, 2 sort intervals
    int tune_idx = 0;          // candidate being measured
    double tune_best = 1e300;  // best cost per particle-step so far (ms)
    int tune_best_val = 0;
    std::string tune_key;
    char gpu_name[256] = {0};

    // CUDA graphs of the step windows pic_step has run: a window is a run of steps
    // inside one sort cycle (at most to its sort step), keyed by the store copy it
    // starts from, its first step's place in the cycle, its length and whether the step
    // before it counted cells for the sort; each records the host state it ends in
    struct Window {
        cudaGraphExec_t exec = nullptr;
        int end_cur = 0;
        bool end_hist = false;
        int64_t kernels = 0;
    };
    bool graphs = true;
    std::map<std::tuple<int, int64_t, int64_t, bool>, Window> windows;
    bool profiling = false;
    struct Timed { int cls; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
    // per kernel class: 0 mover, 1 field, 2 sort, 3 other, 5 the mover of a sort step
    // (index 4 is unused: pic_kernel_time(4) reports the kernel count)
    int64_t launches[6] = {0, 0, 0, 0, 0, 0};
    double ms[6] = {0, 0, 0, 0, 0, 0};
    int64_t kernels = 0;  // kernel launches since the last pic_profile call
};

namespace {

int fail(pic_handle* h, int code, const std::string& msg);

// The handle's staging buffer for host transfers, grown on demand and kept (a fresh
// allocation of gigabytes per call costs more than the copy).  The stream is drained
// before a smaller buffer is given back.
cudaError_t io_buffer(pic_handle* h, size_t bytes, char** out)
{
    if (bytes > h->io_bytes) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess && h->io) e = cudaFree(h->io);
        h->io = nullptr;
        h->io_bytes = 0;
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->io, bytes);
        if (e != cudaSuccess) {
            h->io = nullptr;
            return e;
        }
        h->io_bytes = bytes;
    }
    *out = h->io;
    return cudaSuccess;
}

// The device address of a host array when it is pinned and mapped (page-locked host
// memory: the load kernel then reads it over the host link itself, the conversion in
// the same pass as the transfer, at the link's rate); null for pageable memory.
const void* mapped_host(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return at.devicePointer;
}

int fail(pic_handle* h, int code, const std::string& msg)
{
    if (h) {
        h->last_error = msg;
        if (code == PIC_ECUDA) h->state = PIC_ECUDA;
    } else {
        g_create_error = msg;
    }
    return code;
}

#define CUDA_TRY(h, expr)                                                            \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail((h), PIC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int check_state(pic_handle* h)
{
    if (!h) return PIC_EINVAL;
    if (h->state != PIC_OK) {
        if (h->last_error.empty()) h->last_error = "handle is in the error state";
        return PIC_ESTATE;
    }
    return PIC_OK;
}

template <typename T>
int dalloc(pic_handle* h, T** p, size_t count)
{
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, PIC_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PIC_OK;
}

cudaEvent_t take_event(pic_handle* h)
{
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Span {
    pic_handle* h;
    int cls;
    cudaEvent_t a = nullptr;
    Span(pic_handle* hh, int c) : h(hh), cls(c)
    {
        if (h->profiling) {
            a = take_event(h);
            cudaEventRecord(a, h->stream);
        }
    }
    ~Span()
    {
        if (a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, h->stream);
            h->timed.push_back({cls, a, b});
        }
    }
};

// --- validation -------------------------------------------------------------------
int validate_instance(const pic_instance& I, int idx, std::string* why)
{
    auto bad = [&](const std::string& m) {
        *why = "instance " + std::to_string(idx) + ": " + m;
        return PIC_EINVAL;
    };
    if (I.ncells < 1 || I.ncells > kMaxCells) return bad("ncells must be in [1, 2^23 - 1]");
    if (I.nspecies < 1 || I.nspecies > PIC_MAX_SPECIES) return bad("nspecies must be 1..4");
    if (!(I.dx > 0) || !(I.dt > 0) || !(I.eps0 > 0)) return bad("dx, dt, eps0 must be > 0");
    if (I.bc < 0 || I.bc > 2) return bad("invalid bc");
    if (I.field < 0 || I.field > 2) return bad("invalid field mode");
    if (I.field == PIC_FIELD_POISSON && I.bc == PIC_BC_PERIODIC)
        return bad("the grounded Poisson solve needs walls (bc != PERIODIC)");
    for (int s = 0; s < I.nspecies; ++s) {
        if (!(I.sp[s].mass > 0) || !std::isfinite(I.sp[s].charge) || !(I.sp[s].weight >= 0))
            return bad("species " + std::to_string(s) + ": mass > 0, finite charge, weight >= 0");
        if (I.sp[s].capacity < 0) return bad("negative capacity");
        if (!(I.sp[s].temperature >= 0)) return bad("temperature must be >= 0");
        if (I.sp[s].nstep < 0 || I.sp[s].nstep > 4096) return bad("nstep must be 0..4096");
        if (I.sp[s].sn2d != 0 && I.sp[s].sn2d != 1) return bad("sn2d must be 0 or 1");
    }
    if (I.nproc < 0 || I.nproc > PIC_MAX_PROC) return bad("nproc must be 0..8");
    if (I.smooth != 0 && I.smooth != 1) return bad("smooth must be 0 or 1");
    if (I.target < 0 || I.target > I.nspecies) return bad("target must be 0..nspecies");
    if (I.target > 0) {
        if (I.sp[I.target - 1].charge != 0.0) return bad("the neutral target species must have charge 0");
        if (I.nref < 1) return bad("nref must be >= 1 with a neutral target");
    }
    for (int k = 0; k < I.nproc; ++k) {
        const pic_process& P = I.proc[k];
        if (P.kind < 0 || P.kind > 3) return bad("process kind");
        if (I.target > 0 && P.species == I.target - 1)
            return bad("the neutral target species cannot be a projectile");
        if (P.species < 0 || P.species >= I.nspecies) return bad("process species");
        if (!(P.nu >= 0) || !(P.threshold >= 0)) return bad("process nu/threshold must be >= 0");
        if (P.kind == PIC_PROC_ELASTIC && !(I.sp[P.species].mass <= 0.25 * I.m_neutral))
            return bad("elastic scattering needs m_s <= m_neutral / 4");
        if (P.kind == PIC_PROC_IONIZE &&
            (P.product < 0 || P.product >= I.nspecies || P.product == P.species))
            return bad("ionization needs a product species other than the projectile");
        if ((P.kind == PIC_PROC_CX || P.kind == PIC_PROC_IONIZE) && !(I.m_neutral > 0))
            return bad("charge exchange / ionization need m_neutral > 0");
    }
    return PIC_OK;
}

// Subcycling factor of species s (>= 1).
int species_nstep(const pic_instance& I, int s)
{
    return I.sp[s].nstep > 1 ? I.sp[s].nstep : 1;
}

// Derive the per-segment constants.  The expressions mirror the definitions in the
// mover: A = c_s E with c_s = (q/m) dt^2/dx; Boris t = (q/m) B dt/2, s = 2t/(1+t.t);
// candidate probability P = 1 - exp(-nu_max dt) as floor(P 2^32).
void seg_constants(const pic_instance& I, int s, SegParams* P)
{
    const pic_species& S = I.sp[s];
    // subcycling: the species' own time step is nstep * dt (Listing 7's x += nstep*vx);
    // every per-step constant below is for that step
    P->nstep = species_nstep(I, s);
    const double dt = (double)P->nstep * I.dt;
    const double vs = dt / I.dx;
    const double qm = S.charge / S.mass;
    P->accel = qm * (dt * dt / I.dx);
    const double qmh = qm * (0.5 * dt);
    for (int k = 0; k < 3; ++k) P->t[k] = qmh * I.B[k];
    const double tt = P->t[0] * P->t[0] + P->t[1] * P->t[1] + P->t[2] * P->t[2];
    const double sf = 2.0 / (1.0 + tt);
    for (int k = 0; k < 3; ++k) P->s[k] = sf * P->t[k];
    for (int k = 0; k < 3; ++k) {
        P->tf[k] = (float)P->t[k];
        P->sf[k] = (float)P->s[k];
    }
    const double dxdt = I.dx / dt;
    P->kefac = 0.5 * S.mass * S.weight * (dxdt * dxdt);
    P->vinj = std::sqrt(S.temperature / S.mass) * vs;
    P->vneutral = I.m_neutral > 0 ? std::sqrt(I.T_neutral / I.m_neutral) * vs : 0.0;
    P->mratio = I.m_neutral > 0 ? S.mass / I.m_neutral : 0.0;
    double numax = 0.0;
    for (int k = 0; k < I.nproc; ++k)
        if (I.proc[k].species == s) numax += I.proc[k].nu;
    // candidate steps: Bernoulli(P), P = 1 - exp(-nu_max dt); a run of g candidate-free
    // steps has probability (1-P)^g = exp(-g nu_max dt)
    const double x = numax * dt;
    P->gap[0] = 0xFFFFFFFFu;
    for (int g = 1; g <= kGapMax; ++g) {
        const double T = std::floor(std::exp(-(double)g * x) * 4294967296.0);
        P->gap[g] = T >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)T;
    }
    // log2(1-P) = -x / ln 2
    P->glog = x > 0.0 ? (float)(-0.69314718055994530942 / x) : 0.0f;
    P->nproc = 0;
    double cum = 0.0;
    for (int k = 0; k < I.nproc; ++k) {
        if (I.proc[k].species != s) continue;
        const int q = P->nproc++;
        cum += I.proc[k].nu;
        P->proc[q] = k;
        P->kind[q] = I.proc[k].kind;
        P->product[q] = I.proc[k].product;  // species index; remapped to a segment later
        P->slot_end[q] = (uint64_t)std::floor(cum / numax * 4294967296.0);
        P->thr_u2[q] = (2.0 * I.proc[k].threshold / S.mass) * (vs * vs);
    }
    if (P->nproc > 0) P->slot_end[P->nproc - 1] = (uint64_t)1 << 32;
    P->collide = (P->nproc > 0 && numax > 0.0) ? 1 : 0;
    P->key0 = (uint32_t)I.seed;
    P->key1 = (uint32_t)(I.seed >> 32);
    P->sn2d = S.sn2d;
}

// Charge of each species as an exact integer multiple of a common unit delta
// (needed by the integer field solve).
int charge_units(const pic_instance& I, double* delta, int32_t z[PIC_MAX_SPECIES], std::string* why)
{
    double d = 0.0;
    for (int s = 0; s < I.nspecies; ++s) {
        const double qw = std::fabs(I.sp[s].charge * I.sp[s].weight);
        if (qw > 0 && (d == 0.0 || qw < d)) d = qw;
    }
    if (d == 0.0) d = 1.0;
    for (int s = 0; s < I.nspecies; ++s) {
        const double qw = I.sp[s].charge * I.sp[s].weight;
        const double r = std::nearbyint(qw / d);
        if (std::fabs(r) > 1048576.0 || r * d != qw) {
            *why = "Poisson field: species charges q*w must be integer multiples of a common unit";
            return PIC_EINVAL;
        }
        z[s] = (int32_t)r;
    }
    *delta = d;
    return PIC_OK;
}

MoveArgs move_args(pic_handle* h)
{
    MoveArgs a;
    const Store& S = h->st[h->cur];
    a.cell = S.cell;
    a.off = S.off;
    a.ux = S.ux;
    a.uy = S.uy;
    a.uz = S.uz;
    a.id = S.id;
    a.seg = h->segd;
    a.inst = h->instd;
    a.nseg = h->nseg;
    a.tile_start = h->tile_start;
    a.seg_nmove = h->seg_nmove;
    a.seg_n = h->seg_n;
    a.seg_live = h->seg_live;
    a.accel = h->accel;
    a.dep = h->dep;
    a.wall_count = h->wall_count;
    a.wall_energy = h->wall_energy;
    a.collisions = h->collisions;
    a.events = h->events;
    a.ev_count = h->ev_count;
    a.err = h->err;
    a.step = h->step_d;
    a.rare = h->rare;
    a.rare_count = h->rare_count;
    a.rare_cap = h->rare_cap;
    a.tcount = h->tcount;
    a.treq = h->treq;
    a.vlist = h->vlist;
    a.vcap = h->any_target ? std::max<int64_t>(h->ev_total, 1) : 0;
    a.hist = h->hist;
    a.hist_out = nullptr;
    a.cursor = nullptr;
    a.dcell = nullptr;
    a.doff = a.dux = a.duy = a.duz = nullptr;
    a.did = nullptr;
    a.yp = S.yp;
    a.dyp = nullptr;
    a.test_all = h->test_all;
    a.pair = 0;
    return a;
}

SortArgs sort_args(pic_handle* h)
{
    SortArgs a;
    a.seg = h->segd;
    a.nseg = h->nseg;
    a.precision = h->precision;
    a.tile_start = h->tile_start;
    a.seg_nmove = h->seg_nmove;
    a.seg_n = h->seg_n;
    a.seg_live = h->seg_live;
    a.hwm_alt = h->hwm_alt;
    a.hist = h->hist;
    a.tcount = h->any_target ? h->tcount : nullptr;
    a.cell_part = h->cell_part;
    a.cell_chunks = h->cell_chunks;
    a.seg_nodes = h->seg_nodes;
    a.newn = h->newn;
    for (int b = 0; b < 2; ++b) {
        a.cell[b] = h->st[b].cell;
        a.off[b] = h->st[b].off;
        a.ux[b] = h->st[b].ux;
        a.uy[b] = h->st[b].uy;
        a.uz[b] = h->st[b].uz;
        a.id[b] = h->st[b].id;
        a.yp[b] = h->st[b].yp;
    }
    a.src = h->cur;
    a.max_cap = h->max_cap;
    a.max_cells = h->max_nodes - 1;
    a.err = h->err;
    return a;
}

FieldArgs field_args(pic_handle* h)
{
    FieldArgs f;
    f.seg = h->segd;
    f.inst = h->instd;
    f.ninst = h->ninst;
    f.max_nodes = h->max_nodes;
    f.dep = h->dep;
    f.dep_last = h->dep_last;
    f.accel = h->accel;
    f.seg_nodes = h->seg_nodes;
    f.precision = h->precision;
    f.E = h->E;
    f.chunk_inst = h->chunk_inst;
    f.nchunks = h->nchunks;
    f.part_sum = h->part_sum;
    f.part_w = h->part_w;
    f.zfirst = h->zfirst;
    f.step = h->step_d;
    f.any_poisson = h->any_poisson ? 1 : 0;
    f.zs = h->zs;
    return f;
}

// Phases of a time step with respect to the sort folded into it.
enum StepPhase { kPlain = 0, kCount = 1, kSortStep = 2 };

// The mover (and, for a time step, the event kernels).  kCount: the step also counts the
// particles per cell at its end into `hist`; kSortStep: the step scans those counts,
// moves every particle into its sorted slot of the other store copy, adopts the new
// counts and makes that copy current before the event kernels run on it.
int launch_move(pic_handle* h, bool move, int phase = kPlain)
{
    MoveArgs a = move_args(h);
    const bool mag = move && h->any_mag;
    const bool sort = move && phase == kSortStep;
    SortArgs sa;
    if (move && phase == kCount) {
        CUDA_TRY(h, cudaMemsetAsync(h->hist, 0, sizeof(unsigned) * (size_t)h->seg_nodes, h->stream));
        a.hist_out = h->hist;
    }
    if (sort) {
        sa = sort_args(h);
        Span sp(h, 2);
        h->kernels += 2;
        CUDA_TRY(h, launch_sort_scan(sa, h->stream));
        const Store& D = h->st[1 - h->cur];
        a.cursor = h->hist;
        a.dcell = D.cell;
        a.doff = D.off;
        a.dux = D.ux;
        a.duy = D.uy;
        a.duz = D.uz;
        a.did = D.id;
        a.dyp = D.yp;
    }
    {
        Span sp(h, sort ? 5 : 0);
        const int grid = sort ? h->grid_sort : h->grid_move;
        // a plain FP32 step of a batch without magnetic field launches the mover with the
        // clock test inline and the one that queues the tests (the draw's code and
        // registers cost the common path of this variant 6 %; the FP64 form is bound by
        // its FP64 pipe and the Boris variant holds its registers anyway, so they keep the
        // test inline).  The step count (and a load since the last step) decides on the
        // device which of the two runs, so one captured sort cycle serves every cycle.
        // The partner that returns at once costs about 3 us, more than the 6 % saves
        // below some 16 M particle slots.  A batch with a subcycled colliding species
        // (its candidates and tests bunched on its moving steps) keeps the test inline;
        // subcycled species that never collide, like neutral targets, do not matter.
        const bool pair = move && !sort && !h->any_mag && h->precision == PIC_FP32 &&
                          h->total_cap >= h->pair_min && h->pair_ok;
        a.pair = pair ? 1 : 0;
        // the step on which the neutral particle targets move (they all have the sort
        // interval as their subcycling factor): the variant that updates their kept
        // deposit; on the other steps their tiles are skipped
        const bool kept = move && h->any_target && h->sort_interval > 1 &&
                          (h->step_h + 1) % h->sort_interval == 0;
        for (int v = 0; v < (pair ? 2 : 1); ++v) {
            h->kernels += 1;
            const bool lean = v == 1;
            // the pair's inline-test partner without subcycling: its own variant and grid
            const bool gridv = pair && !lean && !h->any_subcycle;
            const cudaError_t e =
                h->precision == PIC_FP64
                    ? launch_move_f64(a, mag, move, h->any_subcycle, h->any_unmag, sort, kept,
                                      sort ? h->nt_sort : h->nt, grid, h->stream)
                    : launch_move_f32(a, mag, move, h->any_subcycle, h->any_unmag, sort, lean,
                                      gridv, kept, sort ? h->nt_sort : h->nt,
                                      gridv ? h->grid_test : grid, h->stream);
            CUDA_TRY(h, e);
        }
    }
    if (sort) {
        Span sp(h, 2);
        h->kernels += 1;
        CUDA_TRY(h, launch_sort_finish(sa, h->stream));
        h->cur = 1 - h->cur;  // the event kernels work on the sorted copy
    }
    return PIC_OK;
}

// The event kernels of a time step, after its mover, on stream s: the y drift of 2-D
// species (with the velocities after the push, before collisions change them) and the
// rare events.  kCount: a re-injected particle or an ionization product is counted in
// the cell histogram of the coming sort.
int launch_step_events(pic_handle* h, int phase, cudaStream_t s)
{
    MoveArgs a = move_args(h);
    if (phase == kCount) a.hist_out = h->hist;
    if (h->any_sn2d) {
        Span sd(h, 3);
        h->kernels += 1;
        CUDA_TRY(h, launch_drift_y(a, h->precision, 4 * h->sms, s));
    }
    Span se(h, 3);
    h->kernels += 1;
    CUDA_TRY(h, launch_events(a, h->precision, h->grid_events, s));
    return PIC_OK;
}

// The conversions of neutral particle targets into ions requested by the event kernel.
int launch_victims_h(pic_handle* h, cudaStream_t s)
{
    const MoveArgs a = move_args(h);
    Span se(h, 3);
    h->kernels += 1;
    CUDA_TRY(h, launch_victims(a, h->precision, h->grid_victims, s));
    return PIC_OK;
}

// The numbering of this step's ionization products (their ids).
int launch_births_h(pic_handle* h, cudaStream_t s)
{
    Span sp(h, 3);
    h->kernels += 1;
    CUDA_TRY(h, launch_births(h->instd, h->ninst, h->events, h->ev_count, h->next_id,
                              h->st[h->cur].id, h->birth_keys_a, h->birth_keys_b, h->err, s));
    return PIC_OK;
}

int launch_tiles_h(pic_handle* h)
{
    Span sp(h, 3);
    h->kernels += 1;
    CUDA_TRY(h, launch_tiles(h->segd, h->seg_n, h->seg_nmove, h->tile_start, h->nseg, 32,
                             h->rare_count, h->step_d, h->stream));
    return PIC_OK;
}

int do_sort(pic_handle* h);

int ensure_fields(pic_handle* h)
{
    if (!h->stale) return PIC_OK;
    int rc;
    // the field phase (with neutral targets a sort) may reorder the store: the order of
    // the last loads is gone
    std::fill(h->fresh_n.begin(), h->fresh_n.end(), (int64_t)-1);
    h->hist_ready = false;
    // a neutral particle target needs the cell ranges of a sorted store
    if (h->any_target && (rc = do_sort(h))) return rc;
    rc = launch_tiles_h(h);
    if (rc) return rc;
    // a fresh deposit of every particle (kept deposits start over too)
    CUDA_TRY(h, cudaMemsetAsync(h->dep, 0, sizeof(unsigned long long) * (size_t)h->seg_nodes, h->stream));
    if ((rc = launch_move(h, false))) return rc;
    {
        Span sp(h, 1);
        h->kernels += h->any_poisson ? 2 : 1;
        CUDA_TRY(h, launch_field(field_args(h), false, h->stream));
    }
    h->stale = false;
    return PIC_OK;
}

// The separate sort (histogram, scan, scatter, finish): neutral targets, sort interval
// 1, and a sort due with no histogram counted by the step before.
int do_sort(pic_handle* h)
{
    int rc = launch_tiles_h(h);
    if (rc) return rc;
    Span sp(h, 2);
    CUDA_TRY(h, cudaMemsetAsync(h->hist, 0, sizeof(unsigned) * (size_t)h->seg_nodes, h->stream));
    const SortArgs a = sort_args(h);
    h->hist_ready = false;
    h->kernels += h->any_target ? 6 : 5;
    CUDA_TRY(h, launch_sort(a, h->nt, h->sms, h->stream));
    h->cur = 1 - h->cur;
    return PIC_OK;
}

// Synchronise and translate a latched device error.
int sync_check(pic_handle* h)
{
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    unsigned e = 0;
    CUDA_TRY(h, cudaMemcpy(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (e == 0) return PIC_OK;
    int code = PIC_ECUDA;
    std::string msg;
    if (e & kErrInput) { code = PIC_EINVAL; msg = "loaded particle with cell outside [0, ncells) or offset outside [0, 1)"; }
    else if (e & kErrCapacity) { code = PIC_ECAPACITY; msg = "particle creation overflowed a species segment, the event buffer or the 32-bit ids"; }
    else if (e & kErrNonFinite) { code = PIC_ENONFINITE; msg = "a particle velocity became non-finite"; }
    else if (e & kErrEvents) { code = PIC_ECAPACITY; msg = "the rare-event queue of a step (wall hits and collision candidates) overflowed"; }
    else if (e & kErrTimeout) { code = PIC_ETIMEOUT; msg = "a bounded device wait ran out"; }
    else if (e & kErrBounds) { code = PIC_ECUDA; msg = "the bounds-checked build refused a device index"; }
    h->state = code;
    h->last_error = msg;
    return code;
}

int collect_times(pic_handle* h)
{
    if (h->timed.empty()) return PIC_OK;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (auto& t : h->timed) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        h->ms[t.cls] += ms;
        h->launches[t.cls] += 1;
        h->event_pool.push_back(t.a);
        h->event_pool.push_back(t.b);
    }
    h->timed.clear();
    return PIC_OK;
}

void set_block(pic_handle* h, int nt)
{
    h->nt = nt;
    // (FP32: plain steps of a batch with subcycling that the mover pair does not serve run
    // the variant with subcycling and the inline clock test, built for fewer warps)
    const bool subtest = h->any_subcycle && !(h->total_cap >= h->pair_min && h->pair_ok);
    const int bps = h->precision == PIC_FP64 ? move_blocks_per_sm_f64(h->any_mag, false, false, nt)
                                             : move_blocks_per_sm_f32(h->any_mag, false, false, subtest, false, nt);
    h->grid_move = h->sms * std::max(bps, 1);
    const int bts = h->precision == PIC_FP64 ? bps : move_blocks_per_sm_f32(false, false, false, false, true, nt);
    h->grid_test = h->sms * std::max(bts, 1);
    // (the sort step's variant with the y coordinates of 2-D species holds more shared
    // memory a block; its block size is its own)
    const int bss = h->precision == PIC_FP64
                        ? move_blocks_per_sm_f64(h->any_mag, true, h->any_sn2d, h->nt_sort)
                        : move_blocks_per_sm_f32(h->any_mag, true, h->any_sn2d, false, false, h->nt_sort);
    h->grid_sort = h->sms * std::max(bss, 1);
}

void drop_graphs(pic_handle* h)
{
    for (auto& kv : h->windows)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    h->windows.clear();
}

// ---- autotuner ----------------------------------------------------------------------
// Live particles of the whole handle (synchronises the stream).
int live_total(pic_handle* h, double* out)
{
    std::vector<unsigned long long> live((size_t)h->nseg);
    CUDA_TRY(h, cudaMemcpyAsync(live.data(), h->seg_live, 8 * (size_t)h->nseg, cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    double t = 0.0;
    for (unsigned long long v : live) t += (double)v;
    *out = t;
    return PIC_OK;
}

// The time step's results do not depend on the mover block size or on the sort interval
// (deposits are integer, random draws are keyed by particle id, the sort only permutes),
// so the tuner measures candidates on the first steps of the real run: one sort cycle
// per candidate, block sizes first (at sort interval 20), then sort intervals.  The
// choice is cached per GPU and size bucket (precision, magnetised or not, log2 of the
// particle count and of the mean cell count) in a JSON file: $BITPIC_TUNE_CACHE, else
// $HOME/.cache/bitpic/autotune.json.
const int kTuneBlocks[] = {128, 256, 512};
const int kTuneSorts[] = {10, 20, 40, 80};
std::mutex g_tune_mutex;

std::string tune_cache_path()
{
    if (const char* p = std::getenv("BITPIC_TUNE_CACHE")) return p;
    if (const char* home = std::getenv("HOME")) return std::string(home) + "/.cache/bitpic/autotune.json";
    return "";
}

// The cache is a flat JSON object {"key": [block, sort_interval], ...}.
std::map<std::string, std::pair<int, int>> tune_cache_read()
{
    std::map<std::string, std::pair<int, int>> m;
    const std::string path = tune_cache_path();
    if (path.empty()) return m;
    std::ifstream in(path);
    if (!in) return m;
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string t = ss.str();
    size_t i = 0;
    while ((i = t.find('"', i)) != std::string::npos) {
        const size_t j = t.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = t.substr(i + 1, j - i - 1);
        int b = 0, k = 0;
        const size_t lb = t.find('[', j);
        if (lb == std::string::npos || std::sscanf(t.c_str() + lb, "[%d , %d]", &b, &k) != 2) break;
        m[key] = {b, k};
        i = t.find(']', lb);
        if (i == std::string::npos) break;
    }
    return m;
}

void tune_cache_write(const std::map<std::string, std::pair<int, int>>& m)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        std::string cur;
        for (size_t k = 1; k <= dir.size(); ++k)  // mkdir -p, errors ignored
            if (k == dir.size() || dir[k] == '/') {
                cur = dir.substr(0, k);
                mkdir_if_missing(cur);
            }
    }
    const std::string tmp = path + ".tmp";
    std::ofstream out(tmp);
    if (!out) return;
    out << "{\n";
    size_t n = 0;
    for (const auto& kv : m)
        out << "  \"" << kv.first << "\": [" << kv.second.first << ", " << kv.second.second << "]"
            << (++n < m.size() ? ",\n" : "\n");
    out << "}\n";
    out.close();
    std::rename(tmp.c_str(), path.c_str());
}

void tune_begin(pic_handle* h)
{
    int64_t np = 0, cells = 0;
    for (const auto& I : h->inst) {
        cells += I.ncells;
        for (int s = 0; s < I.nspecies; ++s) np += I.sp[s].capacity;
    }
    const int lp = (int)std::floor(std::log2((double)std::max<int64_t>(np, 1)));
    const int lc = (int)std::floor(std::log2((double)std::max<int64_t>(cells / h->ninst, 1)));
    char key[400];
    std::snprintf(key, sizeof(key), "%s|%s|%s|p%d|c%d", h->gpu_name,
                  h->precision == PIC_FP64 ? "fp64" : "fp32", h->any_mag ? "mag" : "nomag", lp, lc);
    h->tune_key = key;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const auto m = tune_cache_read();
    const auto it = m.find(h->tune_key);
    if (it != m.end()) {
        if (h->tune_block && (it->second.first == 128 || it->second.first == 256 || it->second.first == 512))
            set_block(h, it->second.first);
        if (h->tune_sort && it->second.second > 0) h->sort_interval = it->second.second;
        h->tune_block = h->tune_sort = false;
        return;
    }
    h->tune_phase = h->tune_block ? 1 : 2;
    h->tune_idx = 0;
    h->tune_best = 1e300;
    if (h->tune_phase == 1) set_block(h, kTuneBlocks[0]);
    else h->sort_interval = kTuneSorts[0];
}

void tune_finish(pic_handle* h)
{
    h->tune_phase = 0;
    h->tune_block = h->tune_sort = false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto m = tune_cache_read();
    m[h->tune_key] = {h->nt, h->sort_interval};
    tune_cache_write(m);
}

}  // namespace

extern "C" {

int pic_create(const pic_config* cfg, pic_handle** out)
{
    g_create_error.clear();
    if (!cfg || !out || !cfg->inst || cfg->n_instances < 1)
        return fail(nullptr, PIC_EINVAL, "pic_create: null config/out/instances or n_instances < 1");
    if (cfg->precision != PIC_FP32 && cfg->precision != PIC_FP64)
        return fail(nullptr, PIC_EINVAL, "precision must be PIC_FP32 or PIC_FP64");
    if (cfg->sort_interval < -1) return fail(nullptr, PIC_EINVAL, "sort_interval must be >= -1");
    if (cfg->block != 0 && cfg->block != 128 && cfg->block != 256 && cfg->block != 512)
        return fail(nullptr, PIC_EINVAL, "block must be 0, 128, 256 or 512");
    for (int i = 0; i < cfg->n_instances; ++i) {
        std::string why;
        if (validate_instance(cfg->inst[i], i, &why)) return fail(nullptr, PIC_EINVAL, why);
    }
    pic_handle* h = new (std::nothrow) pic_handle();
    if (!h) return fail(nullptr, PIC_ENOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        g_create_error = h->last_error;
        pic_destroy(h);
        return rc;
    };
    h->precision = cfg->precision;
    h->tsize = cfg->precision == PIC_FP64 ? 8 : 4;
    h->tune_sort = cfg->sort_interval < 0;
    h->tune_block = cfg->block == 0;
    h->sort_interval = h->tune_sort ? 20 : cfg->sort_interval;
    h->nt = cfg->block ? cfg->block : 256;
    if (const char* sb = std::getenv("BITPIC_SORT_BLOCK")) {
        const int v = std::atoi(sb);
        if (v == 128 || v == 256 || v == 512) h->nt_sort = v;
    }
    h->ninst = cfg->n_instances;
    h->inst.assign(cfg->inst, cfg->inst + cfg->n_instances);
    const double S = cfg->precision == PIC_FP64 ? 281474976710656.0 : 16777216.0;

    // segment and node layout
    int64_t slot = 0, snode = 0, inode = 0, ev = 0;
    for (int i = 0; i < h->ninst; ++i) {
        const pic_instance& I = h->inst[i];
        InstParams ip;
        std::memset(&ip, 0, sizeof(ip));
        ip.ncells = I.ncells;
        ip.field = I.field;
        ip.seg0 = (int32_t)h->segh.size();
        ip.nseg = I.nspecies;
        ip.inode = inode;
        ip.chunk0 = h->nchunks;
        ip.nchunk = (I.ncells + 1 + kChunk - 1) / kChunk;
        h->nchunks += ip.nchunk;
        double delta = 1.0;
        if (I.field == PIC_FIELD_POISSON) {
            std::string why;
            if (charge_units(I, &delta, ip.z, &why)) {
                h->last_error = "instance " + std::to_string(i) + ": " + why;
                return bail(PIC_EINVAL);
            }
            h->any_poisson = true;
        }
        ip.lambda = delta / (2.0 * (double)I.ncells * S * I.eps0);
        // the smoother's integer charges are 4x the filtered ones (exact power of two)
        ip.smooth = (I.field == PIC_FIELD_POISSON && I.smooth) ? 1 : 0;
        ip.tseg = -1;
        ip.iseg = -1;
        if (I.target > 0) {
            ip.tseg = ip.seg0 + I.target - 1;
            ip.nref = I.nref;
            h->any_target = true;
            for (int k = 0; k < I.nproc; ++k)
                if (I.proc[k].kind == PIC_PROC_IONIZE) {
                    ip.iseg = ip.seg0 + I.proc[k].product;
                    ip.tratio = (double)species_nstep(I, I.proc[k].product) /
                                (double)species_nstep(I, I.target - 1);
                    break;
                }
        }
        if (ip.smooth) {
            ip.lambda *= 0.25;
            h->any_smooth = true;
        }
        // ionization events per step are at most the candidates of the projectile
        // species: about capacity x P per step; reserve 4x that, at least 4096
        bool ionize = false;
        int64_t evcap = 0;
        for (int k = 0; k < I.nproc; ++k)
            if (I.proc[k].kind == PIC_PROC_IONIZE) {
                ionize = true;
                const int sp = I.proc[k].species;
                double numax = 0.0;
                for (int q = 0; q < I.nproc; ++q)
                    if (I.proc[q].species == sp) numax += I.proc[q].nu;
                const double P = -std::expm1(-numax * I.dt * species_nstep(I, sp));
                const double cap = (double)std::max<int64_t>(I.sp[sp].capacity, 1);
                const int64_t want = (int64_t)std::ceil(cap * std::min(1.0, 4.0 * P));
                evcap = std::max<int64_t>(evcap, std::max<int64_t>(4096, want));
            }
        ip.ev_base = ev;
        ip.ev_cap = ionize ? evcap : 0;
        ev += ip.ev_cap;
        h->any_ionize |= ionize;
        if (I.B[0] != 0.0 || I.B[1] != 0.0 || I.B[2] != 0.0) h->any_mag = true;
        else h->any_unmag = true;
        if (I.bc == PIC_BC_SOURCE) h->any_source = true;
        for (int s = 0; s < I.nspecies; ++s) {
            if (species_nstep(I, s) > 1) h->any_subcycle = true;
            if (I.sp[s].sn2d) h->any_sn2d = true;
        }
        for (int s = 0; s < I.nspecies; ++s) {
            SegParams P;
            std::memset(&P, 0, sizeof(P));
            P.inst = i;
            P.species = s;
            P.ncells = I.ncells;
            P.bc = I.bc;
            P.base = slot;
            P.cap = round_up(std::max<int64_t>(I.sp[s].capacity, 4), kSegAlign);
            P.node = snode;
            P.inode = inode;
            seg_constants(I, s, &P);
            P.is_target = (I.target == s + 1) ? 1 : 0;
            P.mag = (I.B[0] != 0.0 || I.B[1] != 0.0 || I.B[2] != 0.0) ? 1 : 0;
            for (int q = 0; q < P.nproc; ++q)
                if (P.kind[q] == PIC_PROC_IONIZE) P.product[q] = ip.seg0 + P.product[q];
            slot += P.cap;
            snode += round_up(I.ncells + 1, 4);
            h->max_cap = std::max(h->max_cap, P.cap);
            // rare-event queue: the collision candidates of a step and the clock tests
            // that follow them and ionization (about cap x P each; 4x P is reserved),
            // and the wall hits (a sixteenth of the segment; twice that with a volume
            // source, whose re-injected particles may have their clock tests queued on
            // the next step)
            {
                double numax = 0.0;
                for (int q = 0; q < I.nproc; ++q)
                    if (I.proc[q].species == s) numax += I.proc[q].nu;
                const double Pc = -std::expm1(-numax * I.dt * species_nstep(I, s));
                const double wall = I.bc == PIC_BC_PERIODIC ? 0.0 : (I.bc == PIC_BC_SOURCE ? 2.0 : 1.0) / 16.0;
                const double frac = std::min(1.0, 4.0 * Pc + wall);
                h->rare_cap += (int64_t)std::ceil((double)P.cap * frac);
            }
            h->segh.push_back(P);
        }
        inode += I.ncells + 1;
        h->max_nodes = std::max(h->max_nodes, I.ncells + 1);
        h->insth.push_back(ip);
    }
    h->nseg = (int)h->segh.size();
    h->fresh_n.assign((size_t)h->nseg, (int64_t)-1);
    if (h->nseg >= kMaxSegments) {
        h->last_error = "too many (instance, species) segments: at most " + std::to_string(kMaxSegments - 1);
        return bail(PIC_EINVAL);
    }
    if (h->any_target) {
        // the targets' cell ranges come from the sort, and hold between sorts only if the
        // target species moves on the sort steps alone
        if (h->tune_sort || h->sort_interval <= 0) {
            h->last_error = "a neutral particle target needs a fixed sort interval equal to the target's nstep";
            return bail(PIC_EINVAL);
        }
        for (int i = 0; i < h->ninst; ++i) {
            const pic_instance& I = h->inst[i];
            if (I.target > 0 && species_nstep(I, I.target - 1) != h->sort_interval) {
                h->last_error = "instance " + std::to_string(i) +
                                ": the neutral target's nstep must equal the sort interval";
                return bail(PIC_EINVAL);
            }
        }
    }
    h->rare_cap = std::min<int64_t>(h->rare_cap + 65536, std::max<int64_t>(slot, 65536));
    h->total_cap = slot;
    if (const char* pm = std::getenv("BITPIC_PAIR_MIN_SLOTS")) h->pair_min = std::atoll(pm);
    for (int i = 0; i < h->ninst; ++i)
        for (int q = 0; q < h->inst[i].nproc; ++q)
            if (species_nstep(h->inst[i], h->inst[i].proc[q].species) > 1) h->pair_ok = false;
    h->seg_nodes = snode;
    h->inst_nodes = inode;
    h->ev_total = ev;

    if (cfg->cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            h->last_error = "cudaStreamCreate failed";
            return bail(PIC_ECUDA);
        }
        h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        h->last_error = "cudaStreamCreate / cudaEventCreate failed";
        return bail(PIC_ECUDA);
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        h->last_error = "no CUDA device";
        return bail(PIC_ECUDA);
    }
    h->sms = prop.multiProcessorCount;
    h->grid_events = (int)std::min<int64_t>((h->rare_cap + 127) / 128, (int64_t)16 * h->sms);
    // one warp per requested target cell: at most the ionization events of a step
    h->grid_victims = (int)std::min<int64_t>((std::max<int64_t>(h->ev_total, 1) + 3) / 4, (int64_t)4 * h->sms);
    std::snprintf(h->gpu_name, sizeof(h->gpu_name), "%s", prop.name);
    set_block(h, h->nt);
    if (h->tune_block || h->tune_sort) tune_begin(h);

    // device memory
    int rc = PIC_OK;
    const size_t T = h->tsize;
    for (int b = 0; b < 2 && rc == PIC_OK; ++b) {
        Store& st = h->st[b];
        char *o = nullptr, *x = nullptr, *y = nullptr, *z = nullptr;
        if ((rc = dalloc(h, &st.cell, (size_t)slot))) break;
        if ((rc = dalloc(h, &o, (size_t)slot * T))) break;
        if ((rc = dalloc(h, &x, (size_t)slot * T))) break;
        if ((rc = dalloc(h, &y, (size_t)slot * T))) break;
        if ((rc = dalloc(h, &z, (size_t)slot * T))) break;
        if ((rc = dalloc(h, &st.id, (size_t)slot))) break;
        st.off = o; st.ux = x; st.uy = y; st.uz = z;
        if (h->any_sn2d) {
            char* q = nullptr;
            if ((rc = dalloc(h, &q, (size_t)slot * T))) break;
            st.yp = q;
        }
    }
    char* acc = nullptr;
    if (rc == PIC_OK) rc = dalloc(h, &acc, (size_t)snode * 2 * T);  // (A_j, A_{j+1} - A_j) pairs
    h->accel = acc;
    if (rc == PIC_OK) rc = dalloc(h, &h->dep, (size_t)snode);
    if (rc == PIC_OK) rc = dalloc(h, &h->dep_last, (size_t)snode);
    if (rc == PIC_OK) rc = dalloc(h, &h->hist, (size_t)snode);
    if (rc == PIC_OK) rc = dalloc(h, &h->E, (size_t)inode);
    if (rc == PIC_OK) rc = dalloc(h, &h->chunk_inst, (size_t)h->nchunks);
    if (rc == PIC_OK) rc = dalloc(h, &h->part_sum, (size_t)h->nchunks);
    if (rc == PIC_OK) rc = dalloc(h, &h->part_w, (size_t)h->nchunks);
    if (rc == PIC_OK) rc = dalloc(h, &h->zfirst, (size_t)h->nchunks);
    if (rc == PIC_OK && h->any_smooth) rc = dalloc(h, &h->zs, (size_t)inode);
    if (rc == PIC_OK && h->any_target) rc = dalloc(h, &h->tcount, (size_t)snode);
    if (rc == PIC_OK && h->any_target) rc = dalloc(h, &h->treq, (size_t)snode);
    if (rc == PIC_OK && h->any_target) rc = dalloc(h, &h->vlist, (size_t)std::max<int64_t>(ev, 1));
    if (rc == PIC_OK) rc = dalloc(h, &h->phi_d, (size_t)h->max_nodes);
    if (rc == PIC_OK) rc = dalloc(h, &h->segd, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->instd, (size_t)h->ninst);
    if (rc == PIC_OK) rc = dalloc(h, &h->newn, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->seg_n, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->seg_live, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->hwm_alt, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->seg_nmove, (size_t)h->nseg);
    if (rc == PIC_OK) rc = dalloc(h, &h->tile_start, (size_t)h->nseg + 1);
    if (rc == PIC_OK) rc = dalloc(h, &h->wall_count, (size_t)h->nseg * 2);
    if (rc == PIC_OK) rc = dalloc(h, &h->wall_energy, (size_t)h->nseg * 2);
    if (rc == PIC_OK) rc = dalloc(h, &h->collisions, (size_t)h->ninst * kMaxProc);
    if (rc == PIC_OK) rc = dalloc(h, &h->events, (size_t)std::max<int64_t>(ev, 1));
    if (rc == PIC_OK) rc = dalloc(h, &h->ev_count, (size_t)h->ninst);
    if (rc == PIC_OK) rc = dalloc(h, &h->rare, (size_t)h->rare_cap);
    if (rc == PIC_OK) rc = dalloc(h, &h->rare_count, 2);
    if (rc == PIC_OK) rc = dalloc(h, &h->next_id, (size_t)h->ninst);
    if (rc == PIC_OK) rc = dalloc(h, &h->birth_keys_a, (size_t)std::max<int64_t>(h->ev_total, 1));
    if (rc == PIC_OK) rc = dalloc(h, &h->birth_keys_b, (size_t)std::max<int64_t>(h->ev_total, 1));
    h->cell_chunks = (h->max_nodes + 4095) / 4096;
    if (rc == PIC_OK) rc = dalloc(h, &h->cell_part, (size_t)h->nseg * h->cell_chunks);
    if (rc == PIC_OK) rc = dalloc(h, &h->err, 1);
    if (rc == PIC_OK) rc = dalloc(h, &h->step_d, 2);
    if (rc == PIC_OK) rc = dalloc(h, &h->test_all, 1);
    if (rc == PIC_OK) rc = dalloc(h, &h->kin, (size_t)PIC_MAX_SPECIES);
    if (rc) return bail(rc);

    cudaStream_t s = h->stream;
    auto z = [&](void* p, size_t bytes) { return cudaMemsetAsync(p, 0, bytes, s); };
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = z(h->st[b].off, (size_t)slot * T);
        if (e == cudaSuccess) e = z(h->st[b].ux, (size_t)slot * T);
        if (e == cudaSuccess) e = z(h->st[b].uy, (size_t)slot * T);
        if (e == cudaSuccess) e = z(h->st[b].uz, (size_t)slot * T);
        if (e == cudaSuccess) e = z(h->st[b].id, (size_t)slot * 4);
        if (e == cudaSuccess && h->st[b].yp) e = z(h->st[b].yp, (size_t)slot * T);
        if (e == cudaSuccess) e = launch_fill_i32(h->st[b].cell, 0, slot, -1, s);
    }
    if (e == cudaSuccess) e = z(h->accel, (size_t)snode * 2 * T);
    if (e == cudaSuccess) e = z(h->rare_count, 16);
    if (e == cudaSuccess) e = z(h->dep, (size_t)snode * 8);
    if (e == cudaSuccess) e = z(h->dep_last, (size_t)snode * 8);
    if (e == cudaSuccess && h->any_target) e = z(h->tcount, (size_t)snode * 4);
    if (e == cudaSuccess && h->any_target) e = z(h->treq, (size_t)snode * 4);
    if (e == cudaSuccess) e = z(h->E, (size_t)inode * 8);
    if (e == cudaSuccess) e = z(h->part_sum, (size_t)h->nchunks * 16);
    if (e == cudaSuccess) e = z(h->part_w, (size_t)h->nchunks * 16);
    if (e == cudaSuccess) e = z(h->zfirst, (size_t)h->nchunks * 16);
    std::vector<int> ci((size_t)h->nchunks);
    for (int i = 0; i < h->ninst; ++i)
        for (int c = 0; c < h->insth[i].nchunk; ++c) ci[(size_t)h->insth[i].chunk0 + c] = i;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->chunk_inst, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = z(h->seg_n, (size_t)h->nseg * 8);
    if (e == cudaSuccess) e = z(h->seg_live, (size_t)h->nseg * 8);
    if (e == cudaSuccess) e = z(h->hwm_alt, (size_t)h->nseg * 8);
    if (e == cudaSuccess) e = z(h->wall_count, (size_t)h->nseg * 16);
    if (e == cudaSuccess) e = z(h->wall_energy, (size_t)h->nseg * 16);
    if (e == cudaSuccess) e = z(h->collisions, (size_t)h->ninst * kMaxProc * 8);
    if (e == cudaSuccess) e = z(h->ev_count, (size_t)h->ninst * 8);
    if (e == cudaSuccess) e = z(h->next_id, (size_t)h->ninst * 8);
    if (e == cudaSuccess) e = z(h->err, 4);
    if (e == cudaSuccess) e = z(h->step_d, 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->test_all, 1, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->segd, h->segh.data(), sizeof(SegParams) * h->segh.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->instd, h->insth.data(), sizeof(InstParams) * h->insth.size(),
                            cudaMemcpyHostToDevice, s);
    // constant fields: none (A = 0) or a uniform external field
    if (e == cudaSuccess) {
        std::vector<double> Eh((size_t)inode, 0.0);
        std::vector<char> Ah((size_t)snode * 2 * T, 0);  // pairs (A, 0): a uniform field
        for (int i = 0; i < h->ninst; ++i) {
            const pic_instance& I = h->inst[i];
            if (I.field != PIC_FIELD_EXTERNAL) continue;
            for (int j = 0; j <= I.ncells; ++j) Eh[h->insth[i].inode + j] = I.E_ext;
            for (int k = 0; k < I.nspecies; ++k) {
                const SegParams& P = h->segh[h->insth[i].seg0 + k];
                for (int j = 0; j <= I.ncells; ++j) {
                    const double a = P.accel * I.E_ext;
                    if (T == 8) reinterpret_cast<double*>(Ah.data())[2 * (P.node + j)] = a;
                    else reinterpret_cast<float*>(Ah.data())[2 * (P.node + j)] = (float)a;
                }
            }
        }
        e = cudaMemcpyAsync(h->E, Eh.data(), Eh.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->accel, Ah.data(), Ah.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        h->last_error = std::string("initialisation failed: ") + cudaGetErrorString(e);
        return bail(PIC_ECUDA);
    }
    *out = h;
    return PIC_OK;
}

namespace {
// pic_load_particles and pic_load_particles_f32: offsets and velocities in double, or in
// float with host_f32 (hb bytes per value).
int load_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                   const int32_t* cell, const void* off, const void* vx, const void* vy,
                   const void* vz, const uint32_t* id, const uint8_t* state, int32_t flags,
                   bool host_f32)
{
    const bool on_device = (flags & PIC_DEVICE) != 0;
    const size_t hb = host_f32 ? 4 : 8;
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || species < 0 || species >= h->inst[inst].nspecies || n < 0)
        return fail(h, PIC_EINVAL, "pic_load_particles: bad instance/species/count");
    if (n > 0 && (!cell || !off || !vx || !vy || !vz))
        return fail(h, PIC_EINVAL, "pic_load_particles: null input array");
    const int si = h->insth[inst].seg0 + species;
    const SegParams& P = h->segh[si];
    if (n > P.cap) return fail(h, PIC_ECAPACITY, "pic_load_particles: n exceeds the species capacity");
    cudaStream_t s = h->stream;
    // staging of host input
    void* stage = nullptr;
    const int32_t* dc = cell;
    const void *doff = off, *dvx = vx, *dvy = vy, *dvz = vz;
    const uint32_t* did = id;
    const uint8_t* dstate = state;
    bool direct = false;  // every host array pinned: k_load reads them itself
    if (!on_device && n > 0) {
        const void* m[7] = {mapped_host(cell), mapped_host(off), mapped_host(vx), mapped_host(vy),
                            mapped_host(vz), mapped_host(id), mapped_host(state)};
        direct = m[0] && m[1] && m[2] && m[3] && m[4] && (!id || m[5]) && (!state || m[6]);
        if (direct) {
            dc = static_cast<const int32_t*>(m[0]);
            doff = m[1];
            dvx = m[2];
            dvy = m[3];
            dvz = m[4];
            did = static_cast<const uint32_t*>(m[5]);
            dstate = static_cast<const uint8_t*>(m[6]);
        }
    }
    if (!on_device && n > 0 && !direct) {
        const size_t bytes = (size_t)n * (4 + hb * 4) + (id ? (size_t)n * 4 : 0) +
                             (state ? (size_t)n : 0) + 128;
        char* p = nullptr;
        CUDA_TRY(h, io_buffer(h, bytes, &p));
        stage = p;
        auto put = [&](const void* src, size_t b) {
            char* d = p;
            p += (b + 15) / 16 * 16;
            return cudaMemcpyAsync(d, src, b, cudaMemcpyHostToDevice, s) == cudaSuccess ? d : nullptr;
        };
        const size_t nbh = (size_t)n * hb;
        dc = (const int32_t*)put(cell, (size_t)n * 4);
        doff = put(off, nbh);
        dvx = put(vx, nbh);
        dvy = put(vy, nbh);
        dvz = put(vz, nbh);
        did = id ? (const uint32_t*)put(id, (size_t)n * 4) : nullptr;
        dstate = state ? (const uint8_t*)put(state, (size_t)n) : nullptr;
        if (!dc || !doff || !dvx || !dvy || !dvz || (id && !did) || (state && !dstate))
            return fail(h, PIC_ECUDA, "pic_load_particles: host-to-device copy failed");
    }
    // automatic ids continue after the largest id of the instance
    unsigned long long id0 = 0;
    if (!id) {
        CUDA_TRY(h, cudaMemcpyAsync(&id0, h->next_id + inst, 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
        if (id0 + (unsigned long long)n > 0xFFFFFFFFull)
            return fail(h, PIC_ECAPACITY, "pic_load_particles: 32-bit particle ids exhausted");
    }
    LoadArgs l;
    l.cell = dc;
    l.off = doff;
    l.vx = dvx;
    l.vy = dvy;
    l.vz = dvz;
    l.host_f32 = host_f32 ? 1 : 0;
    l.id = did;
    l.state = dstate;
    l.own0 = clock_origin(P, h->step_h);
    l.n = n;
    l.id0 = (uint32_t)id0;
    l.vscale = (flags & PIC_CELL_UNITS)
                   ? 1.0
                   : (double)species_nstep(h->inst[inst], species) * h->inst[inst].dt / h->inst[inst].dx;
    l.base = P.base;
    l.cap = P.cap;
    l.ncells = P.ncells;
    const Store& S = h->st[h->cur];
    l.s_cell = S.cell;
    l.s_off = S.off;
    l.s_ux = S.ux;
    l.s_uy = S.uy;
    l.s_uz = S.uz;
    l.s_id = S.id;
    l.s_yp = S.yp;
    l.err = h->err;
    l.precision = h->precision;
    l.next_id = h->next_id + inst;
    CUDA_TRY(h, launch_load(l, s));
    // a loaded clock may need its test at any step: the next step draws them all inline
    CUDA_TRY(h, cudaMemsetAsync(h->test_all, 1, sizeof(int), s));
    // the other copy of the segment holds nothing
    CUDA_TRY(h, launch_fill_i32(h->st[1 - h->cur].cell, P.base, P.base + P.cap, -1, s));
    // counts and the next automatic id
    std::vector<unsigned long long> nn(1, (unsigned long long)n);
    CUDA_TRY(h, cudaMemcpyAsync(h->seg_n + si, nn.data(), 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->seg_live + si, nn.data(), 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemsetAsync(h->hwm_alt + si, 0, 8, s));
    (void)stage;
    if (!id) {
        // with explicit ids k_load has raised the next id to max(id) + 1 itself
        const unsigned long long nid = id0 + (unsigned long long)n;
        CUDA_TRY(h, cudaMemcpyAsync(h->next_id + inst, &nid, 8, cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->stale = true;
    h->hist_ready = false;
    h->fresh_n[si] = n;
    return PIC_OK;
}

}  // namespace

int pic_load_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                       const int32_t* cell, const double* off, const double* vx,
                       const double* vy, const double* vz, const uint32_t* id,
                       const uint8_t* state, int32_t flags)
{
    return load_particles(h, inst, species, n, cell, off, vx, vy, vz, id, state, flags, false);
}

int pic_load_particles_f32(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                           const int32_t* cell, const float* off, const float* vx,
                           const float* vy, const float* vz, const uint32_t* id,
                           const uint8_t* state, int32_t flags)
{
    return load_particles(h, inst, species, n, cell, off, vx, vy, vz, id, state, flags, true);
}

namespace {

// Enqueue one time step (and the sort when it falls due).  A sort falls due at the end of
// every step n with (n+1) mod sort_interval = 0.  It is folded into that step (the
// mover writes the particles in cell order into the other copy) when the step before
// counted the particles per cell; else (neutral targets, which need their cell ranges
// from the sort at the end of the step; sort interval 1; a run that starts on the
// sort step) the separate sort follows the step.
int enqueue_step(pic_handle* h)
{
    int rc;
    const int64_t K = h->sort_interval;
    const bool fold = K >= 2 && !h->any_target;
    int phase = kPlain;
    bool sort_after = false;
    if (K > 0 && (h->step_h + 1) % K == 0) {
        if (fold && h->hist_ready) phase = kSortStep;
        else sort_after = true;
    } else if (fold && (h->step_h + 2) % K == 0) {
        phase = kCount;
    }
    if ((rc = launch_tiles_h(h))) return rc;
    if ((rc = launch_move(h, true, phase))) return rc;
    h->hist_ready = phase == kCount;
    // Work that shares no word with the rest of the step runs on the side stream, forked
    // after the mover or the event kernel and joined before the next step (not when
    // kernels are timed one by one): the event kernels when they deposit nothing (no
    // volume source, no ionization, no neutral particle target; the field phase reads
    // and writes only the deposit, the field and its own scratch), else the numbering
    // of ionization products (it writes only the products' ids and the next free id,
    // which neither the target conversions nor the field phase read)
    const bool side = !h->profiling;
    const bool quiet = !h->any_source && !h->any_ionize && !h->any_target;
    auto fork = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
        return e == cudaSuccess ? cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0) : e;
    };
    bool joined = false;
    if (quiet && side) {
        CUDA_TRY(h, fork());
        if ((rc = launch_step_events(h, phase, h->side_stream))) return rc;
        CUDA_TRY(h, cudaEventRecord(h->ev_join, h->side_stream));
        joined = true;
    } else {
        if ((rc = launch_step_events(h, phase, h->stream))) return rc;
        if (h->any_ionize && side) {
            CUDA_TRY(h, fork());
            if ((rc = launch_births_h(h, h->side_stream))) return rc;
            CUDA_TRY(h, cudaEventRecord(h->ev_join, h->side_stream));
            joined = true;
        }
        if (h->any_target && (rc = launch_victims_h(h, h->stream))) return rc;
        if (h->any_ionize && !side && (rc = launch_births_h(h, h->stream))) return rc;
    }
    {
        Span sp(h, 1);
        h->kernels += h->any_poisson ? 2 : 1;
        CUDA_TRY(h, launch_field(field_args(h), true, h->stream));
    }
    if (joined) CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    h->step_h += 1;
    if (sort_after && (rc = do_sort(h))) return rc;
    return PIC_OK;
}

// Capture `len` steps from the current state (store copy h->cur, step h->step_h,
// hist_ready) as one graph.  Every kernel reads the step count and segment sizes from
// device memory, so the same graph replays every window that starts from the same copy
// at the same place of a sort cycle.  The host state is put back; the window records
// the state its steps end in.
int capture_window(pic_handle* h, int64_t len, pic_handle::Window* w)
{
    const int c0 = h->cur;
    const bool hr0 = h->hist_ready;
    const int64_t step0 = h->step_h, k0 = h->kernels;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = PIC_OK;
    for (int64_t n = 0; n < len && rc == PIC_OK; ++n) rc = enqueue_step(h);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    w->end_cur = h->cur;
    w->end_hist = h->hist_ready;
    w->kernels = h->kernels - k0;
    h->step_h = step0;
    h->cur = c0;
    h->hist_ready = hr0;
    h->kernels = k0;
    if (rc != PIC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, PIC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(h, PIC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    w->exec = ex;
    return PIC_OK;
}

}  // namespace

int pic_step(pic_handle* h, int64_t nsteps)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(h, PIC_EINVAL, "pic_step: nsteps < 0");
    if ((rc = ensure_fields(h))) return rc;
    std::fill(h->fresh_n.begin(), h->fresh_n.end(), (int64_t)-1);
    int64_t n = 0;
    while (n < nsteps) {
        const int64_t K = h->sort_interval;
        // autotuning: time one whole sort cycle per candidate on the real run
        if (h->tune_phase && K > 0 && h->step_h % K == 0 && nsteps - n >= K) {
            // the cost per particle-step: sources and ionization change the particle
            // count from one candidate's cycle to the next
            double live0 = 0.0, live1 = 0.0;
            if ((rc = live_total(h, &live0))) return rc;
            cudaEvent_t ea = take_event(h), eb = take_event(h);
            CUDA_TRY(h, cudaEventRecord(ea, h->stream));
            for (int64_t k = 0; k < K; ++k)
                if ((rc = enqueue_step(h))) return rc;
            CUDA_TRY(h, cudaEventRecord(eb, h->stream));
            CUDA_TRY(h, cudaEventSynchronize(eb));
            float ms = 0.f;
            CUDA_TRY(h, cudaEventElapsedTime(&ms, ea, eb));
            h->event_pool.push_back(ea);
            h->event_pool.push_back(eb);
            n += K;
            if ((rc = live_total(h, &live1))) return rc;
            const double per = ms / ((double)K * std::max(0.5 * (live0 + live1), 1.0));
            if (h->tune_phase == 1) {
                if (per < h->tune_best) { h->tune_best = per; h->tune_best_val = h->nt; }
                if (++h->tune_idx < 3) {
                    set_block(h, kTuneBlocks[h->tune_idx]);
                } else {
                    set_block(h, h->tune_best_val);
                    if (h->tune_sort) {
                        h->tune_phase = 2;
                        h->tune_idx = 0;
                        h->tune_best = 1e300;
                        h->sort_interval = kTuneSorts[0];
                    } else {
                        tune_finish(h);
                    }
                }
            } else {
                if (per < h->tune_best) { h->tune_best = per; h->tune_best_val = (int)K; }
                if (++h->tune_idx < 4) {
                    h->sort_interval = kTuneSorts[h->tune_idx];
                } else {
                    h->sort_interval = h->tune_best_val;
                    tune_finish(h);
                }
            }
            drop_graphs(h);
            h->hist_ready = false;
            continue;
        }
        const bool graphs = h->graphs && !h->profiling && !h->tune_phase && K > 0 &&
                            h->stream != nullptr;
        if (graphs) {
            // the steps up to the end of this sort cycle (or of the call) as one graph
            const int64_t p = h->step_h % K;
            const int64_t len = std::min<int64_t>(K - p, nsteps - n);
            const auto key = std::make_tuple(h->cur, p, len, h->hist_ready);
            auto it = h->windows.find(key);
            if (it == h->windows.end()) {
                // a call pattern that keeps creating new windows (several sort
                // intervals' worth of lengths) starts the cache over
                if (h->windows.size() >= 256) drop_graphs(h);
                pic_handle::Window w;
                if ((rc = capture_window(h, len, &w))) return rc;
                it = h->windows.emplace(key, w).first;
            }
            CUDA_TRY(h, cudaGraphLaunch(it->second.exec, h->stream));
            h->kernels += it->second.kernels;
            h->step_h += len;
            h->cur = it->second.end_cur;
            h->hist_ready = it->second.end_hist;
            n += len;
            continue;
        }
        if ((rc = enqueue_step(h))) return rc;
        ++n;
    }
    return PIC_OK;
}

int pic_sync(pic_handle* h)
{
    int rc = check_state(h);
    if (rc) return rc;
    return sync_check(h);
}

int pic_moments(pic_handle* h, int32_t inst, pic_moments_out* out, double* density,
                double* phi, double* E)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || !out) return fail(h, PIC_EINVAL, "pic_moments: bad arguments");
    if ((rc = ensure_fields(h))) return rc;
    const pic_instance& I = h->inst[inst];
    const InstParams& ip = h->insth[inst];
    const int ns = I.nspecies, N = I.ncells;
    cudaStream_t s = h->stream;
    CUDA_TRY(h, cudaMemsetAsync(h->kin, 0, sizeof(double) * PIC_MAX_SPECIES, s));
    const Store& S = h->st[h->cur];
    int64_t maxslots = 0;
    for (int k = 0; k < ns; ++k) maxslots = std::max(maxslots, h->segh[ip.seg0 + k].cap);
    CUDA_TRY(h, launch_kinetic(h->segd, ip.seg0, ns, maxslots, S.cell, S.ux, S.uy, S.uz,
                               h->precision, h->kin, s));
    if (phi && I.field == PIC_FIELD_POISSON)
        CUDA_TRY(h, launch_potential(field_args(h), inst, I.dx, h->phi_d, s));
    if ((rc = sync_check(h))) return rc;

    std::memset(out, 0, sizeof(*out));
    int64_t step = 0;
    std::vector<unsigned long long> live(ns), wc(2 * ns), col(kMaxProc);
    std::vector<double> we(2 * ns), kin(ns);
    CUDA_TRY(h, cudaMemcpy(&step, h->step_d + 1, 8, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(live.data(), h->seg_live + ip.seg0, 8 * ns, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(wc.data(), h->wall_count + 2 * ip.seg0, 16 * ns, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(we.data(), h->wall_energy + 2 * ip.seg0, 16 * ns, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(col.data(), h->collisions + (size_t)inst * kMaxProc, 8 * kMaxProc, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(kin.data(), h->kin, 8 * ns, cudaMemcpyDeviceToHost));
    unsigned long long nid = 0;
    CUDA_TRY(h, cudaMemcpy(&nid, h->next_id + inst, 8, cudaMemcpyDeviceToHost));
    out->step = step;
    out->next_id = (int64_t)nid;
    for (int k = 0; k < ns; ++k) {
        out->live[k] = (int64_t)live[k];
        out->wall_count[k][0] = (int64_t)wc[2 * k];
        out->wall_count[k][1] = (int64_t)wc[2 * k + 1];
        out->wall_energy[k][0] = we[2 * k];
        out->wall_energy[k][1] = we[2 * k + 1];
        out->kinetic[k] = kin[k];
    }
    for (int q = 0; q < I.nproc; ++q) out->collisions[q] = (int64_t)col[q];
    if (density) {
        const double Sunit = h->precision == PIC_FP64 ? 281474976710656.0 : 16777216.0;
        std::vector<unsigned long long> d((size_t)(N + 1));
        for (int k = 0; k < ns; ++k) {
            const SegParams& P = h->segh[ip.seg0 + k];
            CUDA_TRY(h, cudaMemcpy(d.data(), h->dep_last + P.node, 8 * (size_t)(N + 1), cudaMemcpyDeviceToHost));
            const double wdx = I.sp[k].weight / I.dx;
            double* o = density + (size_t)k * (N + 1);
            for (int j = 0; j <= N; ++j) o[j] = wdx * ((double)d[j] / Sunit);
            if (I.bc == PIC_BC_PERIODIC) {
                const double v = wdx * ((double)(d[0] + d[N]) / Sunit);
                o[0] = v;
                o[N] = v;
            } else {
                o[0] *= 2.0;
                o[N] *= 2.0;
            }
        }
    }
    if (E) CUDA_TRY(h, cudaMemcpy(E, h->E + ip.inode, 8 * (size_t)(N + 1), cudaMemcpyDeviceToHost));
    if (phi) {
        if (I.field == PIC_FIELD_POISSON) {
            CUDA_TRY(h, cudaMemcpy(phi, h->phi_d, 8 * (size_t)(N + 1), cudaMemcpyDeviceToHost));
        } else {
            const double e0 = I.field == PIC_FIELD_EXTERNAL ? I.E_ext : 0.0;
            for (int j = 0; j <= N; ++j) phi[j] = -e0 * ((double)j * I.dx);
        }
    }
    return PIC_OK;
}

int pic_count(pic_handle* h, int32_t inst, int32_t species, int64_t* n)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || species < 0 || species >= h->inst[inst].nspecies || !n)
        return fail(h, PIC_EINVAL, "pic_count: bad arguments");
    if ((rc = sync_check(h))) return rc;
    unsigned long long v = 0;
    CUDA_TRY(h, cudaMemcpy(&v, h->seg_live + h->insth[inst].seg0 + species, 8, cudaMemcpyDeviceToHost));
    *n = (int64_t)v;
    return PIC_OK;
}

namespace {
// pic_get_particles and pic_get_particles_f32: offsets and velocities in double, or in
// float with host_f32 (hb bytes per value).
constexpr int64_t kGetChunks = 8;  // read-back: write/copy overlap granularity

int get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t capacity,
                  int32_t* cell, void* off, void* vx, void* vy, void* vz, uint32_t* id,
                  uint8_t* state, int32_t flags, int64_t* n_out, bool host_f32,
                  double* yp = nullptr)
{
    const bool on_device = (flags & PIC_DEVICE) != 0;
    const size_t hb = host_f32 ? 4 : 8;
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || species < 0 || species >= h->inst[inst].nspecies || !n_out)
        return fail(h, PIC_EINVAL, "pic_get_particles: bad arguments");
    if ((rc = sync_check(h))) return rc;
    const int si = h->insth[inst].seg0 + species;
    const SegParams& P = h->segh[si];
    unsigned long long live = 0, nslots = 0;
    CUDA_TRY(h, cudaMemcpy(&live, h->seg_live + si, 8, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(&nslots, h->seg_n + si, 8, cudaMemcpyDeviceToHost));
    *n_out = (int64_t)live;
    if ((int64_t)live > capacity) return fail(h, PIC_ECAPACITY, "pic_get_particles: capacity too small");
    nslots = std::min<unsigned long long>(((nslots + 3) & ~3ull), (unsigned long long)P.cap);
    cudaStream_t s = h->stream;
    const int64_t nb = ((int64_t)nslots + 1023) / 1024;
    const size_t n = (size_t)std::max<unsigned long long>(live, 1);
    char* tmp = nullptr;
    const size_t scratch = (size_t)(nb + 1) * 8;
    // (host outputs are staged on the device and copied: measured on the GB300, the copy
    // engine moves them at 193 GB/s, the get kernel's compacted 4-byte stores straight
    // into pinned host memory at about 120 GB/s)
    const size_t outb = on_device ? 0 : n * (4 + hb * 4 + 4 + 1 + 8) + 9 * 16;
    CUDA_TRY(h, io_buffer(h, scratch + outb + 16, &tmp));
    GetArgs g;
    const Store& S = h->st[h->cur];
    g.s_cell = S.cell;
    g.s_off = S.off;
    g.s_ux = S.ux;
    g.s_uy = S.uy;
    g.s_uz = S.uz;
    g.s_id = S.id;
    g.s_yp = S.yp;
    g.base = P.base;
    g.nslots = (int64_t)nslots;
    g.own0 = clock_origin(P, h->step_h);
    g.vscale_inv = (flags & PIC_CELL_UNITS)
                       ? 1.0
                       : h->inst[inst].dx / ((double)species_nstep(h->inst[inst], species) * h->inst[inst].dt);
    g.precision = h->precision;
    g.block_count = reinterpret_cast<unsigned long long*>(tmp);
    g.capacity = (int64_t)live;
    g.host_f32 = host_f32 ? 1 : 0;
    if (on_device) {
        g.cell = cell; g.off = off; g.vx = vx; g.vy = vy; g.vz = vz; g.id = id; g.state = state;
        g.yp = yp;
    } else {
        char* p = tmp + (scratch + 15) / 16 * 16;
        auto take = [&](size_t b) { char* d = p; p += (b + 15) / 16 * 16; return d; };
        g.cell = cell ? (int32_t*)take(n * 4) : nullptr;
        g.off = off ? take(n * hb) : nullptr;
        g.vx = vx ? take(n * hb) : nullptr;
        g.vy = vy ? take(n * hb) : nullptr;
        g.vz = vz ? take(n * hb) : nullptr;
        g.id = id ? (uint32_t*)take(n * 4) : nullptr;
        g.state = state ? (uint8_t*)take(n) : nullptr;
        g.yp = yp ? (double*)take(n * 8) : nullptr;
    }
    CUDA_TRY(h, launch_get_scan(g, s));
    if (on_device || live == 0) {
        CUDA_TRY(h, launch_get_write(g, 0, nb, s));
    } else {
        // the output offsets of the blocks on the host, then the writes in chunks: the
        // copy stream moves each chunk's outputs to the host while the next is written
        std::vector<unsigned long long> bc((size_t)nb + 1);
        CUDA_TRY(h, cudaMemcpyAsync(bc.data(), g.block_count, 8 * (size_t)(nb + 1),
                                    cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
        const int64_t chunks = std::min<int64_t>(nb, kGetChunks);
        std::vector<cudaEvent_t> evs;
        auto span = [&](void* dst, const void* src, size_t elem, size_t o0, size_t o1) {
            return cudaMemcpyAsync(static_cast<char*>(dst) + o0 * elem,
                                   static_cast<const char*>(src) + o0 * elem, (o1 - o0) * elem,
                                   cudaMemcpyDeviceToHost, h->copy_stream);
        };
        for (int64_t c = 0; c < chunks; ++c) {
            const int64_t b0 = nb * c / chunks, b1 = nb * (c + 1) / chunks;
            CUDA_TRY(h, launch_get_write(g, b0, b1 - b0, s));
            cudaEvent_t ev = take_event(h);
            evs.push_back(ev);
            CUDA_TRY(h, cudaEventRecord(ev, s));
            CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, ev, 0));
            const size_t o0 = (size_t)std::min<unsigned long long>(bc[b0], live);
            const size_t o1 = (size_t)std::min<unsigned long long>(bc[b1], live);
            if (o1 <= o0) continue;
            if (cell) CUDA_TRY(h, span(cell, g.cell, 4, o0, o1));
            if (off) CUDA_TRY(h, span(off, g.off, hb, o0, o1));
            if (vx) CUDA_TRY(h, span(vx, g.vx, hb, o0, o1));
            if (vy) CUDA_TRY(h, span(vy, g.vy, hb, o0, o1));
            if (vz) CUDA_TRY(h, span(vz, g.vz, hb, o0, o1));
            if (id) CUDA_TRY(h, span(id, g.id, 4, o0, o1));
            if (state) CUDA_TRY(h, span(state, g.state, 1, o0, o1));
            if (yp) CUDA_TRY(h, span(yp, g.yp, 8, o0, o1));
        }
        CUDA_TRY(h, cudaStreamSynchronize(h->copy_stream));
        for (cudaEvent_t ev : evs) h->event_pool.push_back(ev);
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return PIC_OK;
}
}  // namespace

int pic_get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t capacity,
                      int32_t* cell, double* off, double* vx, double* vy, double* vz,
                      uint32_t* id, uint8_t* state, int32_t flags, int64_t* n_out)
{
    return get_particles(h, inst, species, capacity, cell, off, vx, vy, vz, id, state, flags,
                         n_out, false);
}

int pic_get_particles_f32(pic_handle* h, int32_t inst, int32_t species, int64_t capacity,
                          int32_t* cell, float* off, float* vx, float* vy, float* vz,
                          uint32_t* id, uint8_t* state, int32_t flags, int64_t* n_out)
{
    return get_particles(h, inst, species, capacity, cell, off, vx, vy, vz, id, state, flags,
                         n_out, true);
}

int pic_load_yp(pic_handle* h, int32_t inst, int32_t species, int64_t n, const double* yp,
                int32_t flags)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || species < 0 || species >= h->inst[inst].nspecies || n < 0 ||
        (n > 0 && !yp))
        return fail(h, PIC_EINVAL, "pic_load_yp: bad arguments");
    if (!h->inst[inst].sp[species].sn2d)
        return fail(h, PIC_EINVAL, "pic_load_yp: the species has no y coordinate (sn2d = 0)");
    const int si = h->insth[inst].seg0 + species;
    if (h->fresh_n[si] < 0) {
        h->last_error = "pic_load_yp: only after pic_load_particles of the species, before the next "
                        "pic_step, pic_moments or pic_charge_raw";
        return PIC_ESTATE;  // the handle stays usable
    }
    if (n != h->fresh_n[si]) return fail(h, PIC_EINVAL, "pic_load_yp: n differs from the load's");
    cudaStream_t s = h->stream;
    const double* d = yp;
    if (!(flags & PIC_DEVICE) && n > 0) {
        char* p = nullptr;
        CUDA_TRY(h, io_buffer(h, (size_t)n * 8, &p));
        CUDA_TRY(h, cudaMemcpyAsync(p, yp, (size_t)n * 8, cudaMemcpyHostToDevice, s));
        d = reinterpret_cast<const double*>(p);
    }
    CUDA_TRY(h, launch_set_yp(h->st[h->cur].yp, h->segh[si].base, d, n, h->precision, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return PIC_OK;
}

int pic_get_yp(pic_handle* h, int32_t inst, int32_t species, int64_t capacity, double* yp,
               int32_t flags, int64_t* n_out)
{
    if (!yp) return fail(h, PIC_EINVAL, "pic_get_yp: null output");
    return get_particles(h, inst, species, capacity, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, flags & PIC_DEVICE, n_out, false, yp);
}

int pic_restore_counters(pic_handle* h, int64_t step, const uint64_t* next_id)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (step < 0) return fail(h, PIC_EINVAL, "pic_restore_counters: step < 0");
    if ((rc = sync_check(h))) return rc;
    const int64_t both[2] = {step, step};
    CUDA_TRY(h, cudaMemcpy(h->step_d, both, 16, cudaMemcpyHostToDevice));
    if (step != h->step_h) {
        CUDA_TRY(h, launch_rebase_clocks(h->segd, h->nseg, h->st[h->cur].cell, h->step_h, step, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    if (next_id) {
        for (int i = 0; i < h->ninst; ++i)
            if (next_id[i] > 0xFFFFFFFFull) return fail(h, PIC_EINVAL, "pic_restore_counters: next_id >= 2^32");
        CUDA_TRY(h, cudaMemcpy(h->next_id, next_id, 8 * (size_t)h->ninst, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(h, cudaMemset(h->test_all, 1, sizeof(int)));
    h->step_h = step;
    h->hist_ready = false;
    return PIC_OK;
}

int pic_charge_raw(pic_handle* h, int32_t inst, int64_t* out, int64_t* unit)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (inst < 0 || inst >= h->ninst || !out || !unit) return fail(h, PIC_EINVAL, "pic_charge_raw: bad arguments");
    if ((rc = ensure_fields(h))) return rc;
    if ((rc = sync_check(h))) return rc;
    const InstParams& ip = h->insth[inst];
    const int N = h->inst[inst].ncells;
    for (int k = 0; k < ip.nseg; ++k) {
        const SegParams& P = h->segh[ip.seg0 + k];
        CUDA_TRY(h, cudaMemcpy(out + (size_t)k * (N + 1), h->dep_last + P.node, 8 * (size_t)(N + 1),
                               cudaMemcpyDeviceToHost));
    }
    *unit = h->precision == PIC_FP64 ? (int64_t)1 << 48 : (int64_t)1 << 24;
    return PIC_OK;
}

int pic_profile(pic_handle* h, int32_t enable)
{
    int rc = check_state(h);
    if (rc) return rc;
    if ((rc = collect_times(h))) return rc;
    h->profiling = enable != 0;
    for (int k = 0; k < 6; ++k) {
        h->launches[k] = 0;
        h->ms[k] = 0.0;
    }
    h->kernels = 0;
    return PIC_OK;
}

int pic_kernel_time(pic_handle* h, int32_t which, int64_t* launches, double* total_ms)
{
    int rc = check_state(h);
    if (rc) return rc;
    if (which < 0 || which > 5 || !launches || !total_ms) return fail(h, PIC_EINVAL, "pic_kernel_time: bad arguments");
    if ((rc = collect_times(h))) return rc;
    if (which == 4) {
        *launches = h->kernels;
        *total_ms = 0.0;
        return PIC_OK;
    }
    *launches = h->launches[which];
    *total_ms = h->ms[which];
    return PIC_OK;
}

int pic_destroy(pic_handle* h)
{
    if (!h) return PIC_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& t : h->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    drop_graphs(h);
    for (void* p : h->allocs) cudaFree(p);
    if (h->io) cudaFree(h->io);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    cudaGetLastError();
    delete h;
    return PIC_OK;
}

const char* pic_last_error(const pic_handle* h)
{
    return h ? h->last_error.c_str() : g_create_error.c_str();
}

int pic_philox(uint64_t key, const uint32_t* ctr, uint32_t* out, int64_t n, int32_t on_device,
               void* stream)
{
    g_create_error.clear();
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(nullptr, PIC_EINVAL, "pic_philox: bad arguments");
    if (n == 0) return PIC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t* dc = ctr;
    uint32_t* dout = out;
    void* tmp = nullptr;
    const size_t b = (size_t)n * 16;
    if (!on_device) {
        if (cudaMallocAsync(&tmp, 2 * b, s) != cudaSuccess) return fail(nullptr, PIC_ENOMEM, "pic_philox: allocation failed");
        dc = static_cast<uint32_t*>(tmp);
        dout = static_cast<uint32_t*>(tmp) + 4 * n;
        if (cudaMemcpyAsync((void*)dc, ctr, b, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(nullptr, PIC_ECUDA, "pic_philox: copy failed");
    }
    cudaError_t e = launch_philox(key, dc, dout, n, s);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dout, b, cudaMemcpyDeviceToHost, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, std::string("pic_philox: ") + cudaGetErrorString(e));
    return PIC_OK;
}

}  // extern "C"
