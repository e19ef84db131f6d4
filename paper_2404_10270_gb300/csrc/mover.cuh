// mover.cuh -- the fused per-particle time step ("particle mover" of the paper,
// Section 2 and Listing 7) for one precision T:
//
//   gather   a = A[j] + f (A[j+1] - A[j])           (Listing 7, moveb())
//   push     u += a, or the Boris rotation when B != 0 (Boris 1970)
//   move     f += u_x; the integer part moves the particle across cells
//   wall     absorbing (flux counters), periodic, or absorb + volume re-injection
//   MCC      null collision: Philox(id, step, COLLIDE) word 0 < floor(P 2^32)
//            selects a candidate, word 1 a process slot; energy thresholds,
//            elastic / charge-exchange / ionization kinematics
//   deposit  cloud-in-cell in fixed point: node j gets S - Q, node j+1 gets
//            Q = rint(f S), so every particle adds exactly S (S = 2^24 FP32,
//            2^48 FP64); reduced per node across the warp in registers, then one
//            64-bit reduction per node and warp into HBM.
//
// Work decomposition: a tile is 32 quads of four consecutive particles of one
// segment (instance, species), owned by one warp; each lane loads its quad with
// 128-bit accesses.  The particle id is not streamed: the collision clock (bits
// 23-30 of the cell word) makes Philox draws happen about once per 127 steps per
// particle, and only then, or at a wall, is the id read.  Warps walk the tiles of all segments independently.  The
// acceleration of the nodes a warp touches is staged in registers and exchanged by
// warp shuffles; there is no block-level barrier anywhere in the step, so an SM keeps
// the loads of many tiles in flight (the kernel is bound by HBM, not by latency).
#pragma once
#include <climits>

#include "common.cuh"

namespace bitpic {

#ifndef BITPIC_MOVE_MIN_WARPS
#define BITPIC_MOVE_MIN_WARPS 48
#endif
constexpr int kMoveMinWarps = BITPIC_MOVE_MIN_WARPS;  // resident warps per SM the mover is built for
#ifndef BITPIC_MOVE_MIN_WARPS64
#define BITPIC_MOVE_MIN_WARPS64 24
#endif
constexpr int kMoveMinWarps64 = BITPIC_MOVE_MIN_WARPS64;  // the same for the FP64 form
#ifndef BITPIC_MOVE_MIN_WARPS_MAG
#define BITPIC_MOVE_MIN_WARPS_MAG 32
#endif
constexpr int kMoveMinWarpsMag = BITPIC_MOVE_MIN_WARPS_MAG;  // cap for the Boris (3V) variant
constexpr int kDeadCell = -(1 << 30);

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
    const void* accel;                  // T, segment node arrays
    unsigned long long* dep;            // fixed-point deposit, segment node arrays
    unsigned long long* wall_count;     // [nseg][2]
    double* wall_energy;                // [nseg][2]
    unsigned long long* collisions;     // [ninst][kMaxProc]
    Event* events;
    unsigned long long* ev_count;       // [ninst]
    unsigned* err;
    const int64_t* step;
};

template <typename T> struct Prec;
template <> struct Prec<float> {
    using Q = uint32_t;  // fixed-point charge of one particle (< 2^25)
    static constexpr int min_warps = kMoveMinWarps;  // memory bound: as many warps as fit
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
    static constexpr int min_warps = kMoveMinWarps64;  // FP64-pipe bound: registers first
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
    // Finiteness from the exponent bits (integer ALU; the FP64 pipe is this form's limit).
    static __device__ __forceinline__ bool finite(double x)
    {
        return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
    }
    // The same move as the float form with the same rounding: floor(f'), f' - floor(f')
    // and the truncation.  For the common -1 < f' < 2 the floor is read from the bits,
    // and the subtraction of 0 or -1 or 1 is done as the identical IEEE operation (or
    // skipped when it is exact), which saves three of this form's FP64 instructions.
    static __device__ __forceinline__ void move(double& f, double u, int& j)
    {
        const double xn = f + u;
        const long long b = __double_as_longlong(xn);
        const int e = (int)((b >> 52) & 0x7FF);
        if (e < 1023) {                                  // |f'| < 1
            if (b >= 0 || (b & 0x7FFFFFFFFFFFFFFFll) == 0) {
                f = __longlong_as_double(b & 0x7FFFFFFFFFFFFFFFll);  // f' - 0 (-0 -> +0)
                return;
            }
            double fk = xn + 1.0;                        // f' - (-1)
            j -= 1;
            if (fk >= 1.0) {
                fk = 0.0;
                j += 1;
            }
            f = fk;
            return;
        }
        if (e == 1023 && b >= 0) {                       // 1 <= f' < 2: exact f' - 1
            f = xn - 1.0;
            j += 1;
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
template <typename T, bool MAG, int NT>
struct MoveOccupancy {
    static constexpr int warps =
        MAG && kMoveMinWarpsMag < Prec<T>::min_warps ? kMoveMinWarpsMag : Prec<T>::min_warps;
    static constexpr int blocks = warps / (NT / 32) > 0 ? warps / (NT / 32) : 1;
};

__device__ __forceinline__ void ld4(const float* p, float v[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4])
{
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Unit vector uniform on the sphere, polar axis x (the wall normal).
template <typename T>
__device__ __forceinline__ void iso_dir(uint32_t w0, uint32_t w1, T n[3])
{
    const T ct = T(1) - T(2) * Prec<T>::uni(w0);
    const T st = Prec<T>::sqrt_(T(1) - ct * ct);
    T sp, cp;
    Prec<T>::sincos2pi(Prec<T>::uni(w1), &sp, &cp);
    n[0] = ct;
    n[1] = st * cp;
    n[2] = st * sp;
}

// Box-Muller (1958).
template <typename T>
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, T* z0, T* z1)
{
    const T r = Prec<T>::sqrt_(T(-2) * Prec<T>::log_(Prec<T>::uni(wa)));
    T s, c;
    Prec<T>::sincos2pi(Prec<T>::uni(wb), &s, &c);
    *z0 = r * c;
    *z1 = r * s;
}

// Warp-level deposit of four particles per lane.  With Q = rint(f S) the charge of
// one particle is S - Q on node j and Q on node j+1, so the total on node c is
//     S n_c - R_c + R_{c-1},   n_c = particles in cell c,  R_c = sum of their Q.
// The warp's particles usually sit in a few neighbouring cells (they are sorted by
// cell), so per occupied cell the warp forms n_c and R_c by register reductions; lane
// l then owns node wmin + l, takes R_{c-1} from lane l-1 by shuffle, and adds the node
// total to HBM with one 64-bit reduction (no return value, so nothing waits on it).
template <typename Q>
__device__ __forceinline__ void warp_deposit(const int jd[4], const Q qr[4],
                                             unsigned long long S,
                                             unsigned long long* __restrict__ gdep)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int lmin = INT_MAX, lmax = INT_MIN;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (jd[k] >= 0) {
            lmin = min(lmin, jd[k]);
            lmax = max(lmax, jd[k]);
        }
    const int wmin = __reduce_min_sync(FULL, lmin);
    if (wmin == INT_MAX) return;
    const int wmax = __reduce_max_sync(FULL, lmax);
    const int ncell = wmax - wmin + 1;
    if (ncell < 32) {
        unsigned long long myR = 0;  // R_c of cell wmin + lane
        uint32_t myn = 0;            // n_c of cell wmin + lane
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
        const unsigned long long prevR = __shfl_up_sync(FULL, myR, 1);
        if (lane <= ncell) {
            const unsigned long long tot =
                S * (unsigned long long)myn - myR + (lane > 0 ? prevR : 0ull);
            if (tot != 0) atomicAdd(gdep + wmin + lane, tot);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jd[k] >= 0) {
                atomicAdd(gdep + jd[k], S - (unsigned long long)qr[k]);
                atomicAdd(gdep + jd[k] + 1, (unsigned long long)qr[k]);
            }
    }
}

// A null-collision candidate of one particle (velocity u in cells/step, after the
// move): process slot from the selection word `wsel`, energy threshold (below it the
// event is a null collision), kinematics.  Returns true when u changed.  Ionization
// appends two particles.
template <typename T>
__device__ __noinline__ bool collide(const MoveArgs& a, const SegParams& P, int s,
                                     uint32_t id, int64_t step, int j, T f, T& ux, T& uy,
                                     T& uz, uint32_t wsel)
{
    int q = -1;
    for (int k = 0; k < P.nproc; ++k)
        if ((uint64_t)wsel < P.slot_end[k]) { q = k; break; }
    if (q < 0) return false;
    const T u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 >= (T)P.thr_u2[q])) return false;  // below threshold: null event
    const int kind = P.kind[q];
    if (kind == PIC_PROC_ELASTIC) {
        const uint4 r = draw(id, step, kRngScatter, P.key0, P.key1);
        T n[3];
        iso_dir<T>(r.x, r.y, n);
        const T speed = Prec<T>::sqrt_(u2);
        if (speed > T(0)) {
            const T cchi = (ux * n[0] + uy * n[1] + uz * n[2]) / speed;
            const T fac = Prec<T>::sqrt_(T(1) - T(2) * (T)P.mratio * (T(1) - cchi));
            const T sp2 = speed * fac;
            ux = sp2 * n[0];
            uy = sp2 * n[1];
            uz = sp2 * n[2];
        }
    } else if (kind == PIC_PROC_CX) {
        const uint4 r = draw(id, step, kRngMaxwell, P.key0, P.key1);
        T z0, z1, z2, z3;
        box_muller<T>(r.x, r.y, &z0, &z1);
        box_muller<T>(r.z, r.w, &z2, &z3);
        const T vn = (T)P.vneutral;
        ux = z0 * vn;
        uy = z1 * vn;
        uz = z2 * vn;
    } else {  // PIC_PROC_IONIZE
        const T us = Prec<T>::sqrt_(T(0.5) * (u2 - (T)P.thr_u2[q]));
        T n1[3], n2[3];
        const uint4 r1 = draw(id, step, kRngScatter, P.key0, P.key1);
        iso_dir<T>(r1.x, r1.y, n1);
        const uint4 r2 = draw(id, step, kRngIonizeE, P.key0, P.key1);
        iso_dir<T>(r2.x, r2.y, n2);
        const uint4 ri = draw(id, step, kRngIonizeI, P.key0, P.key1);
        T z0, z1, z2, z3;
        box_muller<T>(ri.x, ri.y, &z0, &z1);
        box_muller<T>(ri.z, ri.w, &z2, &z3);
        ux = us * n1[0];
        uy = us * n1[1];
        uz = us * n1[2];
        // append the new electron (this segment) and the new ion (product segment)
        const int si = P.product[q];
        const SegParams& Pi = a.seg[si];
        const unsigned long long ke = atomicAdd(a.seg_n + s, 1ull);
        const unsigned long long ki = atomicAdd(a.seg_n + si, 1ull);
        const InstParams& I = a.inst[P.inst];
        const unsigned long long ev = atomicAdd(a.ev_count + P.inst, 1ull);
        if (ke >= (unsigned long long)P.cap || ki >= (unsigned long long)Pi.cap ||
            ev >= (unsigned long long)I.ev_cap) {
            set_error(a.err, kErrCapacity);
        } else {
            const T vn = (T)P.vneutral;
            const int64_t ge = P.base + (int64_t)ke, gi = Pi.base + (int64_t)ki;
            T* off = static_cast<T*>(a.off);
            T* vx = static_cast<T*>(a.ux);
            T* vy = static_cast<T*>(a.uy);
            T* vz = static_cast<T*>(a.uz);
            a.cell[ge] = j; off[ge] = f;
            vx[ge] = us * n2[0]; vy[ge] = us * n2[1]; vz[ge] = us * n2[2];
            a.id[ge] = 0xFFFFFFFFu;
            a.cell[gi] = j; off[gi] = f;
            vx[gi] = z0 * vn; vy[gi] = z1 * vn; vz[gi] = z2 * vn;
            a.id[gi] = 0xFFFFFFFFu;
            Event e;
            e.parent = id;
            e.pad = 0;
            e.slot_e = ge;
            e.slot_i = gi;
            a.events[I.ev_base + (int64_t)ev] = e;
            atomicAdd(a.seg_live + s, 1ull);
            atomicAdd(a.seg_live + si, 1ull);
            // the children's charge joins this step's deposit
            const uint64_t qr = Prec<T>::qright(f), ql = Prec<T>::S - qr;
            atomicAdd(a.dep + P.node + j, (unsigned long long)ql);
            atomicAdd(a.dep + P.node + j + 1, (unsigned long long)qr);
            atomicAdd(a.dep + Pi.node + j, (unsigned long long)ql);
            atomicAdd(a.dep + Pi.node + j + 1, (unsigned long long)qr);
        }
    }
    atomicAdd(a.collisions + (int64_t)P.inst * kMaxProc + P.proc[q], 1ull);
    return true;
}

// Wall phase for a particle that left [0, N) (rare): counts and energy of the
// absorbed particle, then either absorption (returns 2), or volume re-injection with a
// new position and Maxwellian velocity (returns 1).  Periodic walls are handled inline.
template <typename T>
__device__ __noinline__ int wall_event(const MoveArgs& a, const SegParams& P, int s, uint32_t id,
                                       int64_t step, int& j, T& f, T& ux, T& uy, T& uz)
{
    const int wall = j < 0 ? 0 : 1;
    const double u2 = (double)ux * (double)ux + (double)uy * (double)uy + (double)uz * (double)uz;
    atomicAdd(a.wall_count + 2 * s + wall, 1ull);
    atomicAdd(a.wall_energy + 2 * s + wall, P.kefac * u2);
    if (P.bc != PIC_BC_SOURCE) {
        atomicAdd(a.seg_live + s, ~0ull);  // -1
        return 2;
    }
    const int N = P.ncells;
    const uint4 r = draw(id, step, kRngInjectA, P.key0, P.key1);
    const uint4 q2 = draw(id, step, kRngInjectB, P.key0, P.key1);
    const T x = Prec<T>::uni(r.x) * (T)N;
    const T fx = Prec<T>::floor_(x);
    j = (int)fx;
    f = x - fx;
    if (j >= N) {
        j = N - 1;
        f = T(0);
    }
    T z0, z1, z2, z3;
    box_muller<T>(r.y, r.z, &z0, &z1);
    box_muller<T>(q2.x, q2.y, &z2, &z3);
    const T vi = (T)P.vinj;
    ux = z0 * vi;
    uy = z1 * vi;
    uz = z2 * vi;
    return 1;
}

// The state of one lane's quad, copied out of registers only for the rare handler.
template <typename T>
struct Quad {
    int c[4];
    T f[4], ux[4], uy[4], uz[4];
};

// Rare events of one quad, in particle order: wall hits (bit k of `wall`) and
// null-collision candidates (bit k of `cand`; the selection word is word 1 of the
// step's COLLIDE draw).  Out of line so that the hot loop keeps its state in
// registers.  Returns the bits of particles whose uy/uz changed (non-MAG callers
// store those).  q->c holds cell words; a candidate or a re-injection restarts the
// particle's collision clock.
template <typename T, bool MAG>
__device__ __noinline__ unsigned rare_events(const MoveArgs& a, const SegParams& P, int s,
                                             int64_t step, int64_t slot, unsigned wall,
                                             unsigned cand, Quad<T>* q)
{
    const T* uyp = static_cast<const T*>(a.uy);
    const T* uzp = static_cast<const T*>(a.uz);
    unsigned dirty = 0;
    for (int k = 0; k < 4; ++k) {
        const unsigned bit = 1u << k;
        if (!((wall | cand) & bit)) continue;
        const uint32_t idk = a.id[slot + k];
        T vy = MAG ? q->uy[k] : uyp[slot + k];
        T vz = MAG ? q->uz[k] : uzp[slot + k];
        // a wall hit carries its raw (out of range) cell index; others a cell word
        int j = (wall & bit) ? q->c[k] : (int)((uint32_t)q->c[k] & kCellMask);
        T f = q->f[k];
        T vx = q->ux[k];
        if (wall & bit) {
            const int r = wall_event<T>(a, P, s, idk, step, j, f, vx, vy, vz);
            if (r == 2) {
                q->c[k] = -1;
                continue;
            }
        } else {
            q->c[k] = j;  // the step after a candidate draws again
            const uint4 w = draw(idk, step, kRngCollide, P.key0, P.key1);
            if (!collide<T>(a, P, s, idk, step, j, f, vx, vy, vz, w.y)) continue;
        }
        q->c[k] = j;
        q->f[k] = f;
        q->ux[k] = vx;
        q->uy[k] = vy;
        q->uz[k] = vz;
        dirty |= bit;
    }
    return dirty;
}

// The fused time step.  Work unit: a warp tile of 32 quads (128 consecutive particles
// of one segment); each lane owns one quad and moves it with 128-bit accesses.  Warps
// walk the tiles of all segments independently (no block-level barrier), so every SM
// keeps many tiles' loads in flight.  The acceleration of the nodes a warp's
// particles occupy is staged in registers: one coalesced load of the warp's node span,
// then each particle picks its two nodes by warp shuffle.  The loop over the quad is
// free of calls; walls and collision candidates are flagged and handled out of line.
template <typename T, int NT, bool MAG, bool MOVE>
__global__ void __launch_bounds__(NT, MoveOccupancy<T, MAG, NT>::blocks)
k_move(const __grid_constant__ MoveArgs a)
{
    using Q = typename Prec<T>::Q;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    T* const offp = static_cast<T*>(a.off);
    T* const uxp = static_cast<T*>(a.ux);
    T* const uyp = static_cast<T*>(a.uy);
    T* const uzp = static_cast<T*>(a.uz);
    const T* const accp = static_cast<const T*>(a.accel);
    const int64_t step = MOVE ? *a.step : 0;
    // steps to the next multiple of kGapMax, where every clock without a candidate tests
    const int dgrid = kGapMax - (int)(step % kGapMax);
    const int64_t total = a.tile_start[a.nseg];
    const int64_t wstride = (int64_t)gridDim.x * (NT / 32);

    for (int64_t tile = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5); tile < total;
         tile += wstride) {
        const int s = find_segment(a.tile_start, a.nseg, tile);
        const SegParams& P = a.seg[s];
        const int N = P.ncells;
        const int bc = P.bc;
        const int collides = P.collide;
        const uint32_t key0 = P.key0, key1 = P.key1;
        const int64_t node0 = P.node;
        const int64_t quad = (tile - a.tile_start[s]) * 32 + lane;
        const int64_t nq = a.seg_nmove[s] >> 2;
        const bool act = quad < nq;
        const int64_t slot = P.base + 4 * quad;

        int c[4] = {-1, -1, -1, -1};
        T f[4] = {T(0), T(0), T(0), T(0)}, ux[4] = {T(0), T(0), T(0), T(0)};
        T uy[4] = {T(0), T(0), T(0), T(0)}, uz[4] = {T(0), T(0), T(0), T(0)};
        if (act) {
            const int4 cc = __ldcs(reinterpret_cast<const int4*>(a.cell + slot));
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
            ld4(offp + slot, f);
            if (MOVE) ld4(uxp + slot, ux);
            if (MOVE && MAG) {
                ld4(uyp + slot, uy);
                ld4(uzp + slot, uz);
            }
        }

        if (MOVE) {
            // stage the acceleration of the warp's node span in registers
            int lmin = INT_MAX, lmax = INT_MIN;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c[k] >= 0) {
                    const int jj = (int)((uint32_t)c[k] & kCellMask);
                    lmin = min(lmin, jj);
                    lmax = max(lmax, jj);
                }
            const int wmin = __reduce_min_sync(FULL, lmin);
            const int wmax = __reduce_max_sync(FULL, lmax);
            const bool staged = wmin != INT_MAX && wmax - wmin + 2 <= 32;
            T av = T(0);
            if (staged && lane <= wmax - wmin + 1) av = __ldg(accp + node0 + wmin + lane);
            unsigned wallbits = 0, candbits = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // 1. gather (Listing 7)
                const bool live = c[k] >= 0;
                int j = (int)((uint32_t)c[k] & kCellMask);
                uint32_t clk = ((uint32_t)c[k] >> kClockShift) & 0xFFu;
                T a0, a1;
                if (staged) {
                    const int i = live ? j - wmin : 0;
                    a0 = __shfl_sync(FULL, av, i);
                    a1 = __shfl_sync(FULL, av, i + 1);
                } else if (live) {
                    a0 = __ldg(accp + node0 + j);
                    a1 = __ldg(accp + node0 + j + 1);
                } else {
                    a0 = T(0);
                    a1 = T(0);
                }
                if (!live) continue;
                T fk = f[k];
                const T acc = a0 + fk * (a1 - a0);
                // 2. push
                if (!MAG) {
                    ux[k] = ux[k] + acc;
                } else {
                    const T half = T(0.5) * acc;
                    const T t0 = (T)P.t[0], t1 = (T)P.t[1], t2 = (T)P.t[2];
                    const T s0 = (T)P.s[0], s1 = (T)P.s[1], s2 = (T)P.s[2];
                    const T mx = ux[k] + half, my = uy[k], mz = uz[k];
                    const T px = mx + (my * t2 - mz * t1);
                    const T py = my + (mz * t0 - mx * t2);
                    const T pz = mz + (mx * t1 - my * t0);
                    const T qx = mx + (py * s2 - pz * s1);
                    const T qy = my + (pz * s0 - px * s2);
                    const T qz = mz + (px * s1 - py * s0);
                    ux[k] = qx + half;
                    uy[k] = qy;
                    uz[k] = qz;
                }
                if (!Prec<T>::finite(ux[k])) set_error(a.err, kErrNonFinite);
                // 3. move (Listing 7: x += nstep*vx, x the in-cell offset)
                Prec<T>::move(fk, ux[k], j);
                f[k] = fk;
                // 4. walls (absorption and re-injection out of line)
                if (j < 0 || j >= N) {
                    if (bc == PIC_BC_PERIODIC) {
                        j %= N;
                        if (j < 0) j += N;
                    } else {
                        c[k] = j;  // out of range: the rare handler decides
                        wallbits |= 1u << k;
                        continue;
                    }
                }
                // 5. null collision.  The candidate steps of a particle form a
                // Bernoulli(P) sequence; its clock counts the steps to skip before the
                // next event step.  At an event step without a pending candidate (a
                // test), Philox word 0 gives the candidate-free run g from this step,
                // cut at the next multiple of 127 (D steps away): g = 0 candidate now,
                // g < D a candidate g steps later, g = D none before then.  The cut puts
                // the tests of all particles on the same steps, so a warp runs them
                // together.  Candidates continue out of line.
                if (collides) {
                    if (clk & kClockCount) {
                        clk -= 1u;
                    } else if (clk & kClockPending) {
                        candbits |= 1u << k;
                        clk = 0u;
                    } else {
                        // a test step: the id is read only here
                        const uint32_t idk = __ldg(a.id + slot + k);
                        const uint4 w = draw(idk, step, kRngCollide, key0, key1);
                        const int g = min(gap_steps(P.gap, w.x), dgrid);
                        if (g == 0) {
                            candbits |= 1u << k;
                            clk = 0u;
                        } else {
                            clk = g < dgrid ? ((uint32_t)(g - 1) | kClockPending)
                                            : (uint32_t)(dgrid - 1);
                        }
                    }
                }
                c[k] = (int)((uint32_t)j | (clk << kClockShift));
            }
            unsigned dirty = 0;
            if (wallbits | candbits) {
                Quad<T> q;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    q.c[k] = c[k]; q.f[k] = f[k]; q.ux[k] = ux[k]; q.uy[k] = uy[k]; q.uz[k] = uz[k];
                }
                dirty = rare_events<T, MAG>(a, P, s, step, slot, wallbits, candbits, &q);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    c[k] = q.c[k]; f[k] = q.f[k]; ux[k] = q.ux[k]; uy[k] = q.uy[k]; uz[k] = q.uz[k];
                }
            }
            if (act) {
                __stcs(reinterpret_cast<int4*>(a.cell + slot), make_int4(c[0], c[1], c[2], c[3]));
                st4(offp + slot, f);
                st4(uxp + slot, ux);
                if (MAG) {
                    st4(uyp + slot, uy);
                    st4(uzp + slot, uz);
                } else if (dirty) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (dirty & (1u << k)) {
                            uyp[slot + k] = uy[k];
                            uzp[slot + k] = uz[k];
                        }
                }
            }
        }
        // 6. deposit of the (new) positions
        int jd[4];
        Q qr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            jd[k] = c[k] >= 0 ? (int)((uint32_t)c[k] & kCellMask) : kDeadCell;
            qr[k] = c[k] >= 0 ? (Q)Prec<T>::qright(f[k]) : (Q)0;
        }
        warp_deposit<Q>(jd, qr, Prec<T>::S, a.dep + node0);
    }
}

}  // namespace bitpic
