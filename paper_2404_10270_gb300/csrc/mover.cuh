// mover.cuh -- the fused per-particle time step ("particle mover" of the paper,
// Section 2 and Listing 7) for one precision T:
//
//   gather   a = A[j] + f (A[j+1] - A[j]), one fused multiply-add on the node pair
//            (A_j, A_{j+1} - A_j)                   (Listing 7, moveb())
//   push     u += a, or the Boris rotation when B != 0 (Boris 1970)
//   move     f += u_x; the integer part moves the particle across cells
//   wall     periodic wrap inline; a particle that leaves through an absorbing or
//            source wall is queued for the event kernel and leaves the store
//   MCC      null collision: the collision clock in the cell word says when the
//            particle's next candidate step is; at a test step Philox(id, step,
//            COLLIDE) word 0 sets the clock; a candidate is queued for the event
//            kernel, which selects the process and does the kinematics
//   deposit  cloud-in-cell in fixed point: node j gets S - Q, node j+1 gets
//            Q = rint(f S), so every particle adds exactly S (S = 2^24 FP32,
//            2^48 FP64); reduced per node across the warp in registers, then one
//            64-bit reduction per node and warp into HBM.
//
// Work decomposition: a tile is 32 quads of four consecutive particles of one
// segment (instance, species), owned by one warp; each lane loads its quad with
// 128-bit accesses.  The particle id is not streamed: it is read only at clock test
// steps (once per 127 steps per particle) and by the event kernel.  Warps walk the
// tiles of all segments independently, with no block-level barrier, so an SM keeps
// the loads of many tiles in flight.  The loop has no calls: the rare events
// (collision candidates, wall hits) go to a queue that the event kernel
// (events.cuh) works through after the mover, so the common path keeps its whole
// state in registers.  Velocity changes do not move a particle, so a candidate is
// deposited here; a wall particle is deposited by the event kernel if it is
// re-injected.
#pragma once
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace bitpic {

#ifndef BITPIC_MOVE_MIN_WARPS
#define BITPIC_MOVE_MIN_WARPS 48
#endif
constexpr int kMoveMinWarps = BITPIC_MOVE_MIN_WARPS;  // resident warps per SM the mover is built for
#ifndef BITPIC_MOVE_MIN_WARPS_SUBTEST
#define BITPIC_MOVE_MIN_WARPS_SUBTEST 40
#endif
// the FP32 variant with subcycling and the inline clock test, which runs every step of a
// batch with a subcycled colliding species: 48 resident warps leave it 40 registers and
// ~100 B of spills, 40 leave it 48 (measured 2.5 % faster a step on 196.6 M particles)
constexpr int kMoveMinWarpsSubTest = BITPIC_MOVE_MIN_WARPS_SUBTEST;
#ifndef BITPIC_MOVE_MIN_WARPS_GRID
#define BITPIC_MOVE_MIN_WARPS_GRID 32
#endif
// the FP32 variant for the steps on which every clock without a candidate tests (GRID):
// four draws in flight per lane want registers more than warps
constexpr int kMoveMinWarpsGrid = BITPIC_MOVE_MIN_WARPS_GRID;
#ifndef BITPIC_MOVE_MIN_WARPS64
#define BITPIC_MOVE_MIN_WARPS64 32
#endif
constexpr int kMoveMinWarps64 = BITPIC_MOVE_MIN_WARPS64;  // the same for the FP64 form
#ifndef BITPIC_MOVE_MIN_WARPS_MAG
#define BITPIC_MOVE_MIN_WARPS_MAG 32
#endif
constexpr int kMoveMinWarpsMag = BITPIC_MOVE_MIN_WARPS_MAG;  // the Boris (3V) variant, FP32
#ifndef BITPIC_MOVE_MIN_WARPS64_MAG
#define BITPIC_MOVE_MIN_WARPS64_MAG 24
#endif
constexpr int kMoveMinWarps64Mag = BITPIC_MOVE_MIN_WARPS64_MAG;  // the Boris variant, FP64

struct MoveArgs {
    int32_t* cell;
    void* off;
    void* ux;
    void* uy;
    void* uz;
    uint32_t* id;
    const SegParams* seg;
    const InstParams* inst;
    int nseg;
    const int64_t* tile_start;          // nseg+1 prefix of tiles
    const int64_t* seg_nmove;           // slots of each segment moved this step
    unsigned long long* seg_n;          // slots in use (appends for created particles)
    unsigned long long* seg_live;       // live particles
    const void* accel;                  // T pairs (A_j, A_{j+1} - A_j), segment node arrays
    unsigned long long* dep;            // fixed-point deposit, segment node arrays
    unsigned long long* wall_count;     // [nseg][2]
    double* wall_energy;                // [nseg][2]
    unsigned long long* collisions;     // [ninst][kMaxProc]
    Event* events;
    unsigned long long* ev_count;       // [ninst]
    unsigned* err;
    const int64_t* step;
    uint64_t* rare;                     // queue of rare events of this step (rare_pack)
    unsigned long long* rare_count;     // [0]: entries queued this step, [1]: entries of vlist
    int64_t rare_cap;                   // queue entries
    // neutral particle targets (segment node arrays of the target segments): live
    // targets per cell as of the start of the step, ionization requests of the step,
    // and the sort histogram, which holds each cell's end position after a sort
    unsigned* tcount;
    unsigned* treq;
    // the target nodes with ionization requests this step (each once), for k_victims
    int64_t* vlist;
    int64_t vcap;
    const unsigned* hist;
    // the sort folded into the time step: the step before a sort counts each cell's
    // particles at the end of the step into `hist_out` (null: no counting); the sort
    // step reserves each particle's slot in the other store copy from `cursor` (the
    // scanned counts, by the cell at the start of the step) and writes it there
    unsigned* hist_out;
    unsigned* cursor;
    // the collision-clock test: on the steps that are multiples of kGapMax every clock
    // without a candidate tests, and after a load (`test_all` set) any clock may.  With
    // `pair` set both variants are launched for the step: the one with the test inline
    // runs on those steps, the one that queues the few other tests for the event kernel
    // on the rest, and each returns at once on the steps that are not its own (0: the
    // variant launched runs).
    int* test_all;
    int pair;
    int32_t* dcell;
    void* doff;
    void* dux;
    void* duy;
    void* duz;
    uint32_t* did;
    // y coordinates of 2-D species (null when no species has one): this store copy's,
    // and the sort destination's
    void* yp;
    void* dyp;
};

template <typename T> struct Prec;
template <> struct Prec<float> {
    using Q = uint32_t;  // fixed-point charge of one particle (< 2^25)
    using T2 = float2;
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // Boris vectors t, s of the segment in this precision
    static __device__ __forceinline__ float bt(const SegParams& P, int k) { return P.tf[k]; }
    static __device__ __forceinline__ float bs(const SegParams& P, int k) { return P.sf[k]; }
    static constexpr int min_warps = kMoveMinWarps;  // memory bound: as many warps as fit
    static constexpr int min_warps_mag = kMoveMinWarpsMag;
    static constexpr int min_warps_subtest = kMoveMinWarpsSubTest;
    static constexpr int min_warps_grid = kMoveMinWarpsGrid;
    static __device__ __forceinline__ uint64_t qright(float f)
    {
        return (uint64_t)__float2uint_rn(f * 16777216.0f);
    }
    static constexpr uint64_t S = 1ull << 24;
    // (w + 1/2) 2^-32 rounded to float, kept below 1
    static __device__ __forceinline__ float uni(uint32_t w)
    {
        return fminf(__fmaf_rn(__uint2float_rn(w), 0x1p-32f, 0x1p-33f), 0x1.fffffep-1f);
    }
    static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c)
    {
        sincospif(2.0f * u, s, c);
    }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ bool finite(float x) { return isfinite(x); }
    // move (Listing 7: x += nstep*vx with x the in-cell offset): f' = f + u, the integer
    // part of f' moves the particle across cells; an f' - floor(f') that rounds up to 1
    // (f' a tiny negative number) is renormalised to the next cell
    static __device__ __forceinline__ void move(float& f, float u, int& j)
    {
        const float xn = f + u;
        const float fl = floorf(xn);
        f = xn - fl;
        j += (int)fl;
        if (f >= 1.0f) {
            f = 0.0f;
            j += 1;
        }
    }
};
template <> struct Prec<double> {
    using Q = uint64_t;  // fixed-point charge of one particle (< 2^49)
    using T2 = double2;
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double bt(const SegParams& P, int k) { return P.t[k]; }
    static __device__ __forceinline__ double bs(const SegParams& P, int k) { return P.s[k]; }
    static constexpr int min_warps = kMoveMinWarps64;  // FP64-pipe bound: registers first
    static constexpr int min_warps_mag = kMoveMinWarps64Mag;
    static constexpr int min_warps_subtest = kMoveMinWarps64;
    static constexpr int min_warps_grid = kMoveMinWarps64;
    // rint(f 2^48) for f in [0, 1), ties to even, from the bits: f = m 2^(e-1075), so
    // f 2^48 = m / 2^(1027-e) rounded to nearest even (integer ALU only).
    static __device__ __forceinline__ uint64_t qright(double f)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(f);
        const int e = (int)(b >> 52);
        const int sh = 1027 - e;
        if (b == 0ull || sh >= 64) return 0ull;
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        unsigned long long q = m >> sh;
        const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) q += 1ull;
        return q;
    }
    static constexpr uint64_t S = 1ull << 48;
    static __device__ __forceinline__ double uni(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
    static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c)
    {
        const double th = 6.283185307179586476925286766559 * u;
        *s = sin(th);
        *c = cos(th);
    }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    // Finiteness from the exponent bits of the high word (integer ALU; the FP64 pipe
    // is this form's limit, and a test on the whole 64-bit pattern may be turned back
    // into a floating-point comparison by the compiler).
    static __device__ __forceinline__ bool finite(double x)
    {
        return (__double2hiint(x) & 0x7FF00000) != 0x7FF00000;
    }
    // The same move as the float form with the same rounding: f' - floor(f') and the
    // truncation.  For the common -1 < f' < 2 the floor is read from the bits, and only
    // a particle that crossed a cell edge needs f' - floor(f'): the one IEEE addition
    // f' + c, c = +1 or -1 (identical to the subtraction of -1 or 1).  The FP64 pipe is
    // this form's limit, so the addition sits in a branch that a warp takes only when
    // one of its particles crossed (most ion warps do not).  A result that rounds up to
    // 1 (f' a tiny negative number) is renormalised to the next cell from its bits.
    static __device__ __forceinline__ void move(double& f, double u, int& j)
    {
        const double xn = f + u;
        const int hi = __double2hiint(xn);
        const int e = (hi >> 20) & 0x7FF;
        if (__builtin_expect(e < 1023 || (e == 1023 && hi >= 0), 1)) {
            const bool neg = hi < 0;   // -1 < f' < 0, or f' = -0
            const bool up = e == 1023; // 1 <= f' < 2
            double fk = xn;            // 0 <= f' < 1: f' itself
            if (__builtin_expect(neg || up, 0)) {
                fk = xn + __hiloint2double(neg ? 0x3FF00000 : (int)0xBFF00000u, 0);
                j += neg ? -1 : 1;
                if (__double2hiint(fk) == 0x3FF00000) {  // fk in [0, 1]: this is fk == 1
                    fk = 0.0;
                    j += 1;
                }
            }
            f = fk;
            return;
        }
        const double fl = floor(xn);
        double fk = xn - fl;
        j += (int)fl;
        if (fk >= 1.0) {
            fk = 0.0;
            j += 1;
        }
        f = fk;
    }
};

// Resident blocks per SM each mover variant is compiled for (its register budget).
// SUBTEST: the variant with subcycling and the inline clock test; GRID: the variant for
// the steps on which every clock tests.
template <typename T, bool MAG, int NT, bool SUBTEST = false, bool GRID = false>
struct MoveOccupancy {
    static constexpr int warps = MAG ? Prec<T>::min_warps_mag
                                 : GRID ? Prec<T>::min_warps_grid
                                 : SUBTEST ? Prec<T>::min_warps_subtest : Prec<T>::min_warps;
    static constexpr int blocks = warps / (NT / 32) > 0 ? warps / (NT / 32) : 1;
};

// The quad's four values of one array with one 128-bit access (two for double).  The
// particle arrays are streamed (each byte is read and written once per step, and the
// store is far larger than L2), so the accesses carry the evict-first hint and leave L2
// to the node arrays, the deposit and the rare-event queue.
__device__ __forceinline__ void ld4(const float* p, float v[4])
{
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4])
{
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4])
{
    __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st4(double* p, const double v[4])
{
    __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(v[2], v[3]));
}

// Warp-level deposit of four particles per lane.  With Q = rint(f S) the charge of
// one particle is S - Q on node j and Q on node j+1, so the total on node c is
//     S n_c - R_c + R_{c-1},   n_c = particles in cell c,  R_c = sum of their Q.
// The warp forms n_c and R_c for every cell of its range [wmin, wmax]; lane l then
// owns node wmin + l, takes R_{c-1} from lane l-1 by shuffle, and adds the node total
// to HBM with one 64-bit reduction (no return value, so nothing waits on it).  A warp
// whose particles sit in a few cells (the store was sorted recently) forms the sums by
// register reductions, one round per cell; one whose particles have spread over more
// cells (late in a sort cycle) adds each lane's runs of equal cells into a window of
// 32 cells in shared memory (`win`, the warp's own, zero outside this call), which
// costs the same few instructions whatever the spread; beyond 32 cells every particle
// goes to HBM on its own.
// jd = -1 marks an empty slot: as unsigned it is never the minimum of a live cell, as
// signed never the maximum, and it matches no cell.
// NEG: take the quad's charge away instead (two's complement sums; the counts are not
// touched), for a particle deposit that is kept from step to step and updated.
constexpr int kDepLoopCells = 6;  // register reductions up to this many cells

// Words of a warp's deposit window: 32 counts and 32 charge sums (FP64: the 48-bit
// charges as two 24-bit halves; a half summed over a tile of 128 stays below 2^31).
template <typename Q>
struct DepWin {
    static constexpr int words = sizeof(Q) == 4 ? 64 : 96;
};

// Clear the warp's window (once, before its first deposit).
template <typename Q>
__device__ __forceinline__ void dep_win_clear(uint32_t* win)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < DepWin<Q>::words / 32; ++i) win[32 * i + lane] = 0u;
    __syncwarp();
}

template <typename Q, bool NEG = false>
__device__ __forceinline__ void warp_deposit(const int jd[4], const Q qr[4],
                                             unsigned long long S,
                                             unsigned long long* __restrict__ gdep,
                                             unsigned* __restrict__ ghist,
                                             uint32_t* __restrict__ win)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned lmin = 0xFFFFFFFFu;
    int lmax = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lmin = min(lmin, (unsigned)jd[k]);
        lmax = max(lmax, jd[k]);
    }
    const unsigned wminu = __reduce_min_sync(FULL, lmin);
    if (wminu == 0xFFFFFFFFu) return;  // no live particle in the tile
    const int wmin = (int)wminu;
    const int wmax = __reduce_max_sync(FULL, lmax);
    const int ncell = wmax - wmin + 1;
    if (ncell < 32) {
        unsigned long long myR = 0;  // R_c of cell wmin + lane
        uint32_t myn = 0;            // n_c of cell wmin + lane
        if (ncell <= kDepLoopCells) {
            for (int i = 0; i < ncell; ++i) {
                const int cidx = wmin + i;
                uint32_t n = 0;
                if (sizeof(Q) == 4) {
                    uint32_t r = 0;  // at most 128 x 2^24 < 2^32
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool in = jd[k] == cidx;
                        r += in ? (uint32_t)qr[k] : 0u;
                        n += in ? 1u : 0u;
                    }
                    const uint32_t tr = __reduce_add_sync(FULL, r);
                    const uint32_t tn = __reduce_add_sync(FULL, n);
                    if (lane == i) {
                        myR = tr;
                        myn = tn;
                    }
                } else {
                    // 48-bit charges: reduce the high and low 24-bit halves separately
                    uint32_t lo = 0, hi = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool in = jd[k] == cidx;
                        const uint64_t q = in ? (uint64_t)qr[k] : 0ull;
                        lo += (uint32_t)(q & 0xFFFFFFu);
                        hi += (uint32_t)(q >> 24);
                        n += in ? 1u : 0u;
                    }
                    const uint32_t tl = __reduce_add_sync(FULL, lo);
                    const uint32_t th = __reduce_add_sync(FULL, hi);
                    const uint32_t tn = __reduce_add_sync(FULL, n);
                    if (lane == i) {
                        myR = ((unsigned long long)th << 24) + tl;
                        myn = tn;
                    }
                }
            }
        } else {
            // each run of equal cells among the lane's four (consecutive) particles is
            // added to the window once
            uint32_t n = 0, lo = 0, hi = 0;
            int cur = -1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (jd[k] != cur) {
                    if (cur >= 0) {
                        atomicAdd(win + (cur - wmin), n);
                        atomicAdd(win + 32 + (cur - wmin), lo);
                        if (sizeof(Q) == 8) atomicAdd(win + 64 + (cur - wmin), hi);
                    }
                    cur = jd[k];
                    n = lo = hi = 0u;
                }
                if (jd[k] >= 0) {
                    n += 1u;
                    if (sizeof(Q) == 4) {
                        lo += (uint32_t)qr[k];
                    } else {
                        lo += (uint32_t)((uint64_t)qr[k] & 0xFFFFFFu);
                        hi += (uint32_t)((uint64_t)qr[k] >> 24);
                    }
                }
            }
            if (cur >= 0) {
                atomicAdd(win + (cur - wmin), n);
                atomicAdd(win + 32 + (cur - wmin), lo);
                if (sizeof(Q) == 8) atomicAdd(win + 64 + (cur - wmin), hi);
            }
            __syncwarp();
            myn = win[lane];
            myR = win[32 + lane];
            if (sizeof(Q) == 8) myR += (unsigned long long)win[64 + lane] << 24;
            win[lane] = 0u;  // (lanes past the range read and write zeros)
            win[32 + lane] = 0u;
            if (sizeof(Q) == 8) win[64 + lane] = 0u;
            __syncwarp();
        }
        const unsigned long long prevR = __shfl_up_sync(FULL, myR, 1);
        if (lane <= ncell) {
            const unsigned long long tot =
                S * (unsigned long long)myn - myR + (lane > 0 ? prevR : 0ull);
            if (tot != 0) atomicAdd(gdep + wmin + lane, NEG ? 0ull - tot : tot);
        }
        // the particles per cell, for a sort in the next step
        if (ghist && lane < ncell && myn != 0u) atomicAdd(ghist + wmin + lane, myn);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jd[k] >= 0) {
                const unsigned long long l = S - (unsigned long long)qr[k], r = qr[k];
                atomicAdd(gdep + jd[k], NEG ? 0ull - l : l);
                atomicAdd(gdep + jd[k] + 1, NEG ? 0ull - r : r);
                if (ghist) atomicAdd(ghist + jd[k], 1u);
            }
    }
}

// Sort step: the slot of each particle that was in the quad at the start of the step
// (-1: none) from its group's reservation and its rank in the group; a reservation past
// the segment (a histogram that does not match the store, which no path produces) is
// refused and latched rather than written.
__device__ __forceinline__ void sort_destinations(const MoveArgs& a, const SegParams& P,
                                                  const unsigned grp[4], const unsigned rbase[4],
                                                  unsigned had, int64_t to[4])
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned b = __shfl_sync(0xffffffffu, rbase[k], __ffs(grp[k]) - 1);
        to[k] = -1;
        if (had & (1u << k)) {
            const int64_t r = (int64_t)b + __popc(grp[k] & lt);
            if (r < P.cap) to[k] = P.base + r;
            else set_error(a.err, kErrCapacity);
        }
    }
}

// Sort step: the quad's particles into their slots of the other store copy (a particle
// that left through a wall goes there as an empty slot with its velocity, for the event
// kernel).  Streaming stores: the next step reads the copy back from HBM anyway, and
// evict-first lines leave L2 to the partly written lines of other warps' runs.
template <typename T>
__device__ __forceinline__ void sort_write(const MoveArgs& a, const int64_t to[4], const int c[4],
                                           const T f[4], const T ux[4], const T uy[4],
                                           const T uz[4], const uint32_t id[4])
{
    T* const doff = static_cast<T*>(a.doff);
    T* const dux = static_cast<T*>(a.dux);
    T* const duy = static_cast<T*>(a.duy);
    T* const duz = static_cast<T*>(a.duz);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (to[k] < 0) continue;
        const int64_t g = to[k];
        __stcs(a.dcell + g, c[k]);
        __stcs(doff + g, f[k]);
        __stcs(dux + g, ux[k]);
        __stcs(duy + g, uy[k]);
        __stcs(duz + g, uz[k]);
        __stcs(a.did + g, id[k]);
    }
}

// Steps 1-5 of the time step for the four particles of one quad (a lane's share of
// a tile): gather, push, move, walls, collision clock.  c, f, u* hold the quad's
// state on entry and its new state on exit (cell word -1: left through a wall).  The
// masks get one bit per quad position: collision candidate (cand), absorbed at the
// low or high wall (wlo, whi), clock test left to the event kernel (tst), cell word
// changed (chg).  mown is the species' own index of this step (its clock's time),
// dgrid the own steps to its next multiple of kGapMax.  The id of a test draw comes
// from idq (SORT: already loaded) or from the store at `slot`; PRE: the test's
// candidate-free run (before the cut at dgrid) is already in gq.
template <typename T, bool MAG, bool SORT, bool TEST, bool PRE = false>
__device__ __forceinline__ void quad_physics(const MoveArgs& a, const SegParams& P, bool smag,
                                             int64_t step, int64_t mown, int dgrid, int64_t slot,
                                             const uint32_t idq[4], int c[4], T f[4], T ux[4],
                                             T uy[4], T uz[4], unsigned& cand, unsigned& wlo,
                                             unsigned& whi, unsigned& tst, unsigned& chg,
                                             const int* gq = nullptr)
{
    using T2 = typename Prec<T>::T2;
    const T2* const accp = static_cast<const T2*>(a.accel);
    const int N = P.ncells;
    const int bc = P.bc;
    const int collides = P.collide;
    const uint32_t key0 = P.key0, key1 = P.key1;
    const int64_t node0 = P.node;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (c[k] < 0) continue;
        const int cw = c[k];
        int j = (int)((uint32_t)c[k] & kCellMask);
        uint32_t clk = (uint32_t)c[k] >> kClockShift;
        if (!in_range(a.err, j, 0, N)) {  // (bounds-checked build only)
            c[k] = -1;
            chg |= 1u << k;
            continue;
        }
        // 1. gather (Listing 7) from the node pair (A_j, A_{j+1} - A_j)
        const T2 pr = __ldg(accp + node0 + j);
        T fk = f[k];
        const T acc = Prec<T>::fma_(fk, pr.y, pr.x);
        // 2. push
        if (!MAG || !smag) {
            ux[k] = ux[k] + acc;
        } else {
            const T half = T(0.5) * acc;
            const T t0 = Prec<T>::bt(P, 0), t1 = Prec<T>::bt(P, 1), t2 = Prec<T>::bt(P, 2);
            const T s0 = Prec<T>::bs(P, 0), s1 = Prec<T>::bs(P, 1), s2 = Prec<T>::bs(P, 2);
            const T mx = ux[k] + half, my = uy[k], mz = uz[k];
            // v' = v + v x t, v+ = v + v' x s, each component as two fused
            // multiply-adds (m_x + m_y t_z - m_z t_y = fma(m_y, t_z, fma(-m_z, t_y, m_x)))
            const T px = Prec<T>::fma_(my, t2, Prec<T>::fma_(-mz, t1, mx));
            const T py = Prec<T>::fma_(mz, t0, Prec<T>::fma_(-mx, t2, my));
            const T pz = Prec<T>::fma_(mx, t1, Prec<T>::fma_(-my, t0, mz));
            const T qx = Prec<T>::fma_(py, s2, Prec<T>::fma_(-pz, s1, mx));
            const T qy = Prec<T>::fma_(pz, s0, Prec<T>::fma_(-px, s2, my));
            const T qz = Prec<T>::fma_(px, s1, Prec<T>::fma_(-py, s0, mz));
            ux[k] = qx + half;
            uy[k] = qy;
            uz[k] = qz;
        }
        if (!Prec<T>::finite(ux[k])) set_error(a.err, kErrNonFinite);
        // 3. move (Listing 7: x += nstep*vx, x the in-cell offset)
        Prec<T>::move(fk, ux[k], j);
        f[k] = fk;
        // 4. walls: periodic wrap here; an absorbed or re-injected particle
        // leaves the store and the event kernel takes over
        if (j < 0 || j >= N) {
            if (bc == PIC_BC_PERIODIC) {
                j %= N;
                if (j < 0) j += N;
            } else {
                if (j < 0) wlo |= 1u << k; else whi |= 1u << k;
                c[k] = -1;
                chg |= 1u << k;
                continue;
            }
        }
        // 5. null collision.  The candidate steps of a particle form a
        // Bernoulli(P) sequence; its clock names the own step of its next event
        // step.  At an event step without a pending candidate (a test), Philox word
        // 0 gives the candidate-free run g from this step, cut at the next multiple
        // of 127 (D steps away): g = 0 candidate now, g < D a candidate g steps
        // later, g = D none before then.  The cut puts the tests of all particles on
        // the same steps, so a warp runs them together.  Candidates go to the event
        // kernel.  Between events the clock, and so the word, does not change.
        if (collides && (clk & kClockDue) == (uint32_t)(mown & (int64_t)kClockDue)) {
            if (clk & kClockPending) {
                cand |= 1u << k;
                // a test next step (the event kernel draws it when it takes the
                // candidate and puts its outcome in the clock)
                clk = (uint32_t)((mown + 1) & (int64_t)kClockDue);
            } else if (!TEST) {
                // a test off the common test steps (the first clock of an ionization
                // product, whose id the event kernel did not know yet, or of a loaded
                // particle): the event kernel draws it, with this step's counter, and
                // sets the clock
                tst |= 1u << k;
            } else {
                // a test step: the id is read only here
                int g;
                if (PRE) {
                    g = min(gq[k], dgrid);
                } else {
                    const uint32_t idk = SORT ? idq[k] : __ldg(a.id + slot + k);
                    const uint4 w = draw(idk, step, kRngCollide, key0, key1);
                    g = min(gap_steps(P.gap, P.glog, w.x), dgrid);
                }
                if (g == 0) cand |= 1u << k;
                const int64_t due = g == 0 ? mown + 1 : mown + g;
                clk = (uint32_t)(due & (int64_t)kClockDue) | (g > 0 && g < dgrid ? kClockPending : 0u);
            }
        }
        c[k] = (int)((uint32_t)j | (clk << kClockShift));
        if (c[k] != cw) chg |= 1u << k;
    }
}

// Queue the quad's rare events for the event kernel (a few lanes of a few tiles per
// step).  at[k]: the slot the particle occupies after this step (-1: none, nothing is
// queued for it).
__device__ __forceinline__ void queue_rare(const MoveArgs& a, int s, unsigned cand, unsigned wlo,
                                           unsigned whi, unsigned tst, const int64_t at[4])
{
    const unsigned ev = cand | wlo | whi | tst;
    if (!ev) return;
    unsigned long long e = atomicAdd(a.rare_count, (unsigned long long)__popc(ev));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned bit = 1u << k;
        if (!(ev & bit)) continue;
        const uint32_t kind = (cand & bit) ? kRareCandidate
                              : (tst & bit) ? kRareTest
                              : (wlo & bit) ? kRareWallLow : kRareWallHigh;
        if (at[k] < 0) {
            // refused destination (capacity error latched): nothing to queue
        } else if (e < (unsigned long long)a.rare_cap)
            a.rare[e] = rare_pack(at[k], s, kind);
        else
            set_error(a.err, kErrEvents);
        ++e;
    }
}

// The fused time step.  Work unit: a warp tile of 32 quads (128 consecutive particles
// of one segment); each lane owns one quad and moves it with 128-bit accesses.  Warps
// walk the tiles of all segments independently (no block-level barrier), so every SM
// keeps many tiles' loads in flight.  The gather reads each particle's node pair with
// one vector load (the node arrays are small and stay in L1/L2).  The loop is free of
// calls; walls and collision candidates are queued for the event kernel.
// SUB: some species of the batch is subcycled (else every segment moves every step and
// the clock grid is the global one, computed once).  MIXED (with MAG): the batch mixes
// magnetized and unmagnetized instances, so the push is chosen per segment.
// TEST: the collision-clock test (a Philox draw and a table search) runs inline;
// without it a particle whose clock needs a test is queued for the event kernel, which
// keeps the common path free of the draw's code and registers.  KEPT: the step on which
// the neutral particle targets (whose deposit is kept, deposit_kept()) move; on every
// other step their tiles are skipped (a separate variant, so that the update's
// registers do not burden the common steps).  (The step that ends a sort cycle runs
// k_move_sort below instead.)
template <typename T, int NT, bool MAG, bool MOVE, bool SUB, bool MIXED, bool TEST,
          bool KEPT = false, bool GRID = false>
__global__ void __launch_bounds__(NT, MoveOccupancy<T, MAG, NT, MOVE && SUB && TEST, GRID>::blocks)
k_move(const __grid_constant__ MoveArgs a)
{
    using Q = typename Prec<T>::Q;
    const int lane = threadIdx.x & 31;
    T* const offp = static_cast<T*>(a.off);
    T* const uxp = static_cast<T*>(a.ux);
    T* const uyp = static_cast<T*>(a.uy);
    T* const uzp = static_cast<T*>(a.uz);
    const int64_t step = MOVE ? *a.step : 0;
    if (MOVE && a.pair) {
        // every clock without a candidate tests on the multiples of kGapMax (a pair is
        // launched only when every colliding species moves on every step)
        const bool tstep = step % kGapMax == 0 || *a.test_all != 0;
        if (tstep != TEST) return;
    }
    __shared__ uint32_t s_dwin[NT / 32][DepWin<Q>::words];  // the warps' deposit windows
    uint32_t* const dwin = s_dwin[threadIdx.x >> 5];
    dep_win_clear<Q>(dwin);
    const int64_t total = a.tile_start[a.nseg];
    const int64_t wstride = (int64_t)gridDim.x * (NT / 32);
    int s = 0;                         // segment of the previous tile (tiles only increase)
    int64_t s_begin = 0, s_end = -1;   // its tiles
    bool moves = MOVE;                 // the segment moves this step (subcycling)
    bool smag = MAG;                   // the segment's instance is magnetized
    // steps (of the segment's species) to the next multiple of kGapMax
    int dgrid = kGapMax - (int)(step % kGapMax);
    int64_t mown = step;  // the segment's own index of this step (its clock's time)
    for (int64_t tile = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5); tile < total;
         tile += wstride) {
        if (tile >= s_end) {
            s = advance_segment(a.tile_start, a.nseg, s, tile);
            s_begin = __ldg(a.tile_start + s);
            s_end = __ldg(a.tile_start + s + 1);
            // in a batch that mixes magnetized and unmagnetized instances, the latter
            // keep the plain push (and never touch uy, uz), as they would alone
            if (MAG && MIXED) smag = a.seg[s].mag != 0;
            if (MOVE && SUB) {
                // a species with subcycling factor K moves on the steps n with
                // (n+1) mod K = 0 (all species meet at the multiples of K dt); its
                // collision clock counts its own steps, (n+1)/K - 1, and at the multiples
                // of kGapMax of those every clock without a candidate tests
                const int ks = a.seg[s].nstep;
                const int64_t q = ks == 1 ? step + 1 : (step + 1) / ks;
                moves = ks == 1 || q * ks == step + 1;
                dgrid = kGapMax - (int)((q - 1) % kGapMax);
                mown = q - 1;
                // a neutral particle target keeps its deposit from step to step (the
                // field phase does not clear it; conversions into ions take their share
                // away): between its moves nothing of it changes, so the warp goes on
                // with its first tile past the segment
                if (!moves && deposit_kept(a.seg[s])) {
                    tile += ((s_end - 1 - tile) / wstride) * wstride;
                    continue;
                }
            }
        }
        const SegParams& P = a.seg[s];
        const int64_t node0 = P.node;
        const int64_t quad = (tile - s_begin) * 32 + lane;
        const int64_t nq = a.seg_nmove[s] >> 2;
        const int64_t slot = P.base + 4 * quad;
        const bool act = quad < nq && in_range(a.err, slot + 3, P.base, P.base + P.cap);

        int c[4] = {-1, -1, -1, -1};
        T f[4] = {T(0), T(0), T(0), T(0)}, ux[4] = {T(0), T(0), T(0), T(0)};
        T uy[4] = {T(0), T(0), T(0), T(0)}, uz[4] = {T(0), T(0), T(0), T(0)};
        uint32_t idq[4] = {0u, 0u, 0u, 0u};
        if (act) {
            const int4 cc = __ldcs(reinterpret_cast<const int4*>(a.cell + slot));
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
            ld4(offp + slot, f);
            if (MOVE && (!SUB || moves)) ld4(uxp + slot, ux);
            if (MOVE && MAG && smag && (!SUB || moves)) {
                ld4(uyp + slot, uy);
                ld4(uzp + slot, uz);
            }
            if (GRID) {
                const uint4 ii = __ldcs(reinterpret_cast<const uint4*>(a.id + slot));
                idq[0] = ii.x; idq[1] = ii.y; idq[2] = ii.z; idq[3] = ii.w;
            }
        }
        // GRID: every clock without a candidate tests on this step, so the quad's four
        // draws (and their table lookups) go first, side by side, while the state loads
        // are in flight; a clock that does not test ignores its result
        int gq[4] = {0, 0, 0, 0};
        if (GRID && P.collide) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = draw(idq[k], step, kRngCollide, P.key0, P.key1).x;
#pragma unroll
            for (int k = 0; k < 4; ++k) gq[k] = gap_steps(P.gap, P.glog, w[k]);
        }
        if (KEPT && MOVE && SUB && moves && deposit_kept(P)) {
            // its move: the old positions' charge leaves the kept deposit (the new
            // positions' joins it below), exactly as a fresh deposit would come out
            int jd[4];
            Q qr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                jd[k] = (c[k] >> 31) | (int)((uint32_t)c[k] & kCellMask);
                if (jd[k] >= 0 && !in_range(a.err, jd[k], 0, P.ncells)) jd[k] = -1;
                qr[k] = c[k] >= 0 ? (Q)Prec<T>::qright(f[k]) : (Q)0;
            }
            warp_deposit<Q, true>(jd, qr, Prec<T>::S, a.dep + node0, nullptr, dwin);
        }
        if (MOVE && (!SUB || moves)) {
            unsigned cand = 0, wlo = 0, whi = 0, tst = 0, chg = 0;
            quad_physics<T, MAG, false, TEST, GRID>(a, P, smag, step, mown, dgrid, slot, idq, c, f,
                                                    ux, uy, uz, cand, wlo, whi, tst, chg, gq);
            // the cell words go back only where one of them changed (a cell crossing, a
            // wall, a collision event: a few per cent of the particles a step), decided
            // per 32-byte sector (two lanes) so that memory sees whole sectors
            const bool wcell = (chg | __shfl_xor_sync(0xffffffffu, chg, 1)) != 0u;
            if (act) {
                if (wcell)
                    __stcs(reinterpret_cast<int4*>(a.cell + slot), make_int4(c[0], c[1], c[2], c[3]));
                st4(offp + slot, f);
                st4(uxp + slot, ux);
                if (MAG && smag) {
                    st4(uyp + slot, uy);
                    st4(uzp + slot, uz);
                }
            }
            const int64_t at[4] = {slot, slot + 1, slot + 2, slot + 3};
            queue_rare(a, s, cand, wlo, whi, tst, at);
        }
        // 6. deposit of the (new) positions; an empty slot (cell word < 0) gets jd = -1
        int jd[4];
        Q qr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            jd[k] = (c[k] >> 31) | (int)((uint32_t)c[k] & kCellMask);
            if (jd[k] >= 0 && !in_range(a.err, jd[k], 0, P.ncells)) jd[k] = -1;
            qr[k] = c[k] >= 0 ? (Q)Prec<T>::qright(f[k]) : (Q)0;
        }
        warp_deposit<Q>(jd, qr, Prec<T>::S, a.dep + node0,
                        a.hist_out ? a.hist_out + node0 : nullptr, dwin);
    }
}

// ---- the step that ends a sort cycle -------------------------------------------------
// Every particle present at the start of the step goes to its slot of the other store
// copy, in the order of a counting sort by its cell at the start of the step (`cursor`:
// each cell's next free slot, from the counts the step before made).  A block works on
// NT/32 consecutive tiles at a time (a chunk of up to 128 NT/32 particles).  When the
// chunk lies in one segment and its particles' start cells span fewer than kSortSpan
// cells (the common case: the store was sorted one cycle ago), the block counts them
// per cell in shared memory, reserves each cell's run with one global atomic per cell,
// stages the moved particles in shared memory in that order and writes every run with
// consecutive threads, so the scattered writes of a sort become coalesced runs of
// about a cell's share of the chunk.  Otherwise (a chunk across two segments, or
// particles spread widely) each warp reserves per cell and quad position and writes
// its particles directly.
constexpr int kSortSpan = 128;

template <typename T, int NT, bool YP>
struct SortSmem {
    static constexpr int NW = NT / 32;
    static constexpr int C = NW * 128;  // particles of a chunk
    // staged particles (off, ux, uy, uz and with YP yp in T; cell word, id; destination
    // in the segment), then the per-cell counts, run offsets in the chunk, global run starts, and
    // the per-warp summaries (segment, lowest and highest start cell) of two consecutive
    // chunks
    static constexpr size_t bytes = (size_t)C * ((YP ? 5 : 4) * sizeof(T) + 4 + 4 + 4) +
                                    (size_t)3 * kSortSpan * 4 + (size_t)2 * 3 * NW * 4;
};

// YP: some species drifts in y (MoveArgs.yp): the y coordinates are sorted with the
// particles (a separate variant: carrying them costs the others registers).
template <typename T, int NT, bool MAG, bool SUB, bool MIXED, bool YP>
__global__ void __launch_bounds__(NT, MoveOccupancy<T, true, NT>::blocks)
k_move_sort(const __grid_constant__ MoveArgs a)
{
    using Q = typename Prec<T>::Q;
    constexpr int NW = NT / 32, C = NW * 128;
    const unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const s_off = reinterpret_cast<T*>(smem_raw);
    T* const s_ux = s_off + C;
    T* const s_uy = s_ux + C;
    T* const s_uz = s_uy + C;
    T* const s_yp = s_uz + C;  // (only with YP)
    int* const s_cell = reinterpret_cast<int*>(s_yp + (YP ? C : 0));
    uint32_t* const s_id = reinterpret_cast<uint32_t*>(s_cell + C);
    uint32_t* const s_dst = s_id + C;
    int* const cnt = reinterpret_cast<int*>(s_dst + C);
    int* const pre = cnt + kSortSpan;
    unsigned* const gb = reinterpret_cast<unsigned*>(pre + kSortSpan);
    // per-warp summaries, double-buffered by chunk parity: a warp may write the next
    // chunk's entry while another still reads this chunk's (the next chunk's first
    // barrier keeps it from getting further ahead)
    int* const wsum = reinterpret_cast<int*>(gb + kSortSpan);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    __shared__ uint32_t s_dwin[NW][DepWin<Q>::words];  // the warps' deposit windows
    uint32_t* const dwin = s_dwin[warp];
    dep_win_clear<Q>(dwin);
    T* const offp = static_cast<T*>(a.off);
    T* const uxp = static_cast<T*>(a.ux);
    T* const uyp = static_cast<T*>(a.uy);
    T* const uzp = static_cast<T*>(a.uz);
    const int64_t step = *a.step;
    const int64_t total = a.tile_start[a.nseg];
    int s = 0;
    int64_t s_begin = 0, s_end = -1;
    bool moves = true, smag = MAG;
    int dgrid = kGapMax - (int)(step % kGapMax);
    int64_t mown = step;  // the segment's own index of this step (its clock's time)
    // every warp of the block walks the same chunks, so the barriers below match
    int parity = 0;
    for (int64_t chunk = blockIdx.x; chunk * NW < total; chunk += gridDim.x, parity ^= 1) {
        int* const wseg = wsum + parity * 3 * NW;
        int* const wmin = wseg + NW;
        int* const wmax = wmin + NW;
        const int64_t tile = chunk * NW + warp;
        const bool have = tile < total;
        if (have && tile >= s_end) {
            s = advance_segment(a.tile_start, a.nseg, s, tile);
            s_begin = __ldg(a.tile_start + s);
            s_end = __ldg(a.tile_start + s + 1);
            if (MAG && MIXED) smag = a.seg[s].mag != 0;
            if (SUB) {
                const int ks = a.seg[s].nstep;
                const int64_t q = ks == 1 ? step + 1 : (step + 1) / ks;
                moves = ks == 1 || q * ks == step + 1;
                dgrid = kGapMax - (int)((q - 1) % kGapMax);
                mown = q - 1;
            }
        }
        const SegParams& P = a.seg[s];
        const int64_t quad = (tile - s_begin) * 32 + lane;
        const int64_t slot = P.base + 4 * quad;
        const bool act = have && quad < (a.seg_nmove[s] >> 2) &&
                         in_range(a.err, slot + 3, P.base, P.base + P.cap);

        int c[4] = {-1, -1, -1, -1};
        T f[4] = {T(0), T(0), T(0), T(0)}, ux[4] = {T(0), T(0), T(0), T(0)};
        T uy[4] = {T(0), T(0), T(0), T(0)}, uz[4] = {T(0), T(0), T(0), T(0)};
        uint32_t idq[4] = {0u, 0u, 0u, 0u};
        if (act) {
            const int4 cc = __ldcs(reinterpret_cast<const int4*>(a.cell + slot));
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
            ld4(offp + slot, f);
            ld4(uxp + slot, ux);
            ld4(uyp + slot, uy);
            ld4(uzp + slot, uz);
            const uint4 ii = __ldcs(reinterpret_cast<const uint4*>(a.id + slot));
            idq[0] = ii.x; idq[1] = ii.y; idq[2] = ii.z; idq[3] = ii.w;
        }
        // start cells of the quad (-1: empty slot); the chunk's span and segments
        int j0[4];
        unsigned lmin = 0xFFFFFFFFu;
        int lmax = -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            j0[k] = c[k] >= 0 ? (int)((uint32_t)c[k] & kCellMask) : -1;
            if (j0[k] >= 0 && !in_range(a.err, j0[k], 0, P.ncells)) {  // (checked build)
                j0[k] = -1;
                c[k] = -1;
            }
            if (j0[k] >= 0) {
                lmin = min(lmin, (unsigned)j0[k]);
                lmax = max(lmax, j0[k]);
            }
        }
        const unsigned wmn = __reduce_min_sync(FULL, lmin);
        const int wmx = __reduce_max_sync(FULL, lmax);
        if (lane == 0) {
            wseg[warp] = wmx >= 0 ? s : -1;
            wmin[warp] = (int)wmn;
            wmax[warp] = wmx;
        }
        for (int i = threadIdx.x; i < kSortSpan; i += NT) cnt[i] = 0;
        __syncthreads();
        // the chunk's segment (one if every warp's live particles are in the same one)
        // and its span of start cells, from the per-warp summaries
        int bseg, bmin, bmax;
        bool one;
        {
            const int ws = lane < NW ? wseg[lane] : -1;
            const int mn = ws >= 0 ? wmin[lane] : INT_MAX;
            const int mx = ws >= 0 ? wmax[lane] : -1;
            const int smax = __reduce_max_sync(FULL, ws);
            const int smin = __reduce_min_sync(FULL, ws >= 0 ? ws : INT_MAX);
            bseg = smax;
            one = smax < 0 || smin == smax;
            bmin = __reduce_min_sync(FULL, mn);
            bmax = __reduce_max_sync(FULL, mx);
        }
        const bool staged = one && bseg >= 0 && bmax - bmin < kSortSpan;
        unsigned cand = 0, wlo = 0, whi = 0, tst = 0, chg = 0;  // (the sort writes every word)
        int64_t to[4] = {-1, -1, -1, -1};
        if (staged) {
            const SegParams& B = a.seg[bseg];
            // rank of each particle among the chunk's particles of its start cell: equal
            // cells of a quad position grouped across the warp, one shared atomic a group
            int key[4], rank[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                key[k] = j0[k] >= 0 ? j0[k] - bmin : -1;
                const unsigned grp = __match_any_sync(FULL, key[k] >= 0 ? key[k] : kSortSpan + lane);
                const int leader = __ffs(grp) - 1;
                int base = 0;
                if (key[k] >= 0 && lane == leader) base = atomicAdd(cnt + key[k], __popc(grp));
                base = __shfl_sync(FULL, base, leader);
                rank[k] = base + __popc(grp & lt);
            }
            __syncthreads();
            // each cell's run: its offset in the chunk (scan of the counts) and its global
            // start (one reservation per cell, waited for only after the move)
            unsigned gres = 0;
            if (threadIdx.x < kSortSpan) {
                const int n = cnt[threadIdx.x];
                if (n > 0) gres = atomicAdd(a.cursor + B.node + bmin + threadIdx.x, (unsigned)n);
            }
            if (warp == 0) {
                int v[kSortSpan / 32], sum = 0;
#pragma unroll
                for (int i = 0; i < kSortSpan / 32; ++i) {
                    v[i] = cnt[lane * (kSortSpan / 32) + i];
                    sum += v[i];
                }
                int inc = sum;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int t = __shfl_up_sync(FULL, inc, d);
                    if (lane >= d) inc += t;
                }
                int run = inc - sum;
#pragma unroll
                for (int i = 0; i < kSortSpan / 32; ++i) {
                    pre[lane * (kSortSpan / 32) + i] = run;
                    run += v[i];
                }
            }
            if (!SUB || moves)
                quad_physics<T, MAG, true, true>(a, P, smag, step, mown, dgrid, slot, idq, c, f,
                                                 ux, uy, uz, cand, wlo, whi, tst, chg);
            if (threadIdx.x < kSortSpan) gb[threadIdx.x] = gres;
            __syncthreads();
            // stage every particle at its place in the chunk's cell order
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (key[k] < 0) continue;
                const int p = pre[key[k]] + rank[k];
                if (!in_range(a.err, p, 0, C)) continue;  // (bounds-checked build only)
                s_off[p] = f[k];
                s_ux[p] = ux[k];
                s_uy[p] = uy[k];
                s_uz[p] = uz[k];
                s_cell[p] = c[k];
                s_id[p] = idq[k];
                if (YP) s_yp[p] = static_cast<const T*>(a.yp)[slot + k];
                const int64_t r = (int64_t)gb[key[k]] + rank[k];
                to[k] = r < B.cap ? B.base + r : -1;
                s_dst[p] = r < B.cap ? (uint32_t)r : 0xFFFFFFFFu;
            }
            queue_rare(a, bseg, cand, wlo, whi, tst, to);
            // (read before the barrier: the next chunk clears the counts after it)
            const int ntot = pre[kSortSpan - 1] + cnt[kSortSpan - 1];
            __syncthreads();
            // write the runs: consecutive threads, consecutive slots of a cell's run
            T* const doff = static_cast<T*>(a.doff);
            T* const dux = static_cast<T*>(a.dux);
            T* const duy = static_cast<T*>(a.duy);
            T* const duz = static_cast<T*>(a.duz);
#pragma unroll 4
            for (int p = threadIdx.x; p < ntot; p += NT) {
                const uint32_t r = s_dst[p];
                if (r == 0xFFFFFFFFu) {  // a histogram that does not match the store: refused
                    set_error(a.err, kErrCapacity);
                    continue;
                }
                const int64_t g = B.base + (int64_t)r;
                __stcs(a.dcell + g, s_cell[p]);
                __stcs(doff + g, s_off[p]);
                __stcs(dux + g, s_ux[p]);
                __stcs(duy + g, s_uy[p]);
                __stcs(duz + g, s_uz[p]);
                __stcs(a.did + g, s_id[p]);
                if (YP) static_cast<T*>(a.dyp)[g] = s_yp[p];
            }
        } else {
            // per warp: reserve each particle's slot by its start cell (equal cells of a
            // quad position grouped across the warp, one counter update per group)
            unsigned grp[4] = {0u, 0u, 0u, 0u}, rbase[4] = {0u, 0u, 0u, 0u}, had = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int kk = j0[k] >= 0 ? j0[k] : -1 - lane;
                grp[k] = __match_any_sync(FULL, kk);
                if (j0[k] >= 0) had |= 1u << k;
                if (j0[k] >= 0 && lane == __ffs(grp[k]) - 1)
                    rbase[k] = atomicAdd(a.cursor + P.node + kk, (unsigned)__popc(grp[k]));
            }
            if (!SUB || moves)
                quad_physics<T, MAG, true, true>(a, P, smag, step, mown, dgrid, slot, idq, c, f,
                                                 ux, uy, uz, cand, wlo, whi, tst, chg);
            sort_destinations(a, P, grp, rbase, had, to);
            sort_write<T>(a, to, c, f, ux, uy, uz, idq);
            if (YP) {  // the y coordinates go along
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (to[k] >= 0)
                        static_cast<T*>(a.dyp)[to[k]] = static_cast<const T*>(a.yp)[slot + k];
            }
            queue_rare(a, s, cand, wlo, whi, tst, to);
        }
        // 6. deposit of the new positions
        int jd[4];
        Q qr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            jd[k] = (c[k] >> 31) | (int)((uint32_t)c[k] & kCellMask);
            if (jd[k] >= 0 && !in_range(a.err, jd[k], 0, P.ncells)) jd[k] = -1;
            qr[k] = c[k] >= 0 ? (Q)Prec<T>::qright(f[k]) : (Q)0;
        }
        warp_deposit<Q>(jd, qr, Prec<T>::S, a.dep + P.node, nullptr, dwin);
    }
}

// Host side of k_move_sort: the launch with its shared memory, and the set-up of every
// variant (the dynamic shared-memory limit, needed above 48 KB) with the occupancy the
// grid is sized by.  The set-up runs when the handle sizes its grids, outside any
// stream capture.
template <typename T, int NT, bool MAG, bool SUB, bool MIXED, bool YP>
inline cudaError_t launch_sort_variant(const MoveArgs& a, int grid, cudaStream_t st)
{
    k_move_sort<T, NT, MAG, SUB, MIXED, YP><<<grid, NT, SortSmem<T, NT, YP>::bytes, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int NT, bool YP>
inline cudaError_t launch_sort_step_yp(const MoveArgs& a, bool mag, bool sub, bool mixed,
                                       int grid, cudaStream_t st)
{
    if (!mag)
        return sub ? launch_sort_variant<T, NT, false, true, false, YP>(a, grid, st)
                   : launch_sort_variant<T, NT, false, false, false, YP>(a, grid, st);
    if (mixed)
        return sub ? launch_sort_variant<T, NT, true, true, true, YP>(a, grid, st)
                   : launch_sort_variant<T, NT, true, false, true, YP>(a, grid, st);
    return sub ? launch_sort_variant<T, NT, true, true, false, YP>(a, grid, st)
               : launch_sort_variant<T, NT, true, false, false, YP>(a, grid, st);
}

template <typename T, int NT>
inline cudaError_t launch_sort_step(const MoveArgs& a, bool mag, bool sub, bool mixed, int grid,
                                    cudaStream_t st)
{
    return a.yp ? launch_sort_step_yp<T, NT, true>(a, mag, sub, mixed, grid, st)
                : launch_sort_step_yp<T, NT, false>(a, mag, sub, mixed, grid, st);
}

template <typename T, int NT, bool YP>
inline cudaError_t sort_step_setup(int* blocks_mag, int* blocks_plain)
{
    const int sm = (int)SortSmem<T, NT, YP>::bytes;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_move_sort<T, NT, false, false, false, YP>, A, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_move_sort<T, NT, false, true, false, YP>, A, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_move_sort<T, NT, true, false, false, YP>, A, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_move_sort<T, NT, true, true, false, YP>, A, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_move_sort<T, NT, true, false, true, YP>, A, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_move_sort<T, NT, true, true, true, YP>, A, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_mag, k_move_sort<T, NT, true, false, false, YP>, NT, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_plain, k_move_sort<T, NT, false, false, false, YP>, NT, sm);
    return e;
}

// Blocks per SM the sort-step grid is sized by (YP: the variant with the y coordinates,
// launched when some species drifts in y; it holds more shared memory).
template <typename T, int NT>
inline int sort_step_blocks_per_sm(bool mag, bool yp)
{
    int m = 0, p = 0;
    const cudaError_t e = yp ? sort_step_setup<T, NT, true>(&m, &p) : sort_step_setup<T, NT, false>(&m, &p);
    if (e != cudaSuccess) return 0;
    return mag ? m : p;
}

}  // namespace bitpic
