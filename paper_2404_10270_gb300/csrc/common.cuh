// common.cuh -- device-side data structures and helpers of the PIC-MCC library.
//
// Layout in HBM (one handle):
//   * particle store, structure of arrays, two copies (the counting sort scatters
//     from one into the other and the roles swap):  cell int32, off T, ux/uy/uz T,
//     id uint32, T = float (FP32 form) or double (FP64 form).  Velocities are kept
//     in cells per step (u = v dt/dx) so that the move is the paper's
//     x += nstep*vx (Listing 7) with x the in-cell offset.  A slot with cell < 0 is
//     empty.  Every (instance, species) pair owns one contiguous segment whose base
//     and capacity are multiples of 64 slots, so 128-bit loads of four particles
//     never straddle segments.
//   * per segment, node arrays of ncells+1 entries: the pre-scaled acceleration as
//     pairs (A_j, A_{j+1} - A_j) of type T, A = c_s E, which the gather reads with one
//     vector load, and the fixed-point charge deposit (uint64, two copies: the one
//     being accumulated and the last complete one).
//   * per instance, E on the nodes (double) and scratch for the field solve.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace bitpic {

constexpr int kMaxSpecies = PIC_MAX_SPECIES;
constexpr int kMaxProc = PIC_MAX_PROC;
constexpr int kSegAlign = 64;  // slots

// The cell word of a particle: bits 0-22 the cell index j, bits 23-29 the collision
// clock: the species' own step (the index of its moving steps, modulo 128) of its next
// collision event step, bit 30 "that event step is a collision candidate", bit 31 set =
// empty slot (the word is -1).  The event is at most kGapMax own steps ahead, so seven
// bits name it; a step without an event or a cell change leaves the word as it is,
// and the mover does not write it back.  Outside the library (loads, reads, the
// oracle) the clock is the count of own steps to skip before that event step.
constexpr uint32_t kCellMask = (1u << 23) - 1u;
constexpr int kClockShift = 23;
constexpr uint32_t kClockDue = 0x7Fu;
constexpr uint32_t kClockPending = 0x80u;
constexpr int kGapMax = 127;
constexpr int kMaxCells = (1 << 23) - 1;

// The own-step index of the first step >= n on which a species with subcycling factor
// K moves (it moves on the steps n' with (n'+1) mod K = 0, own index (n'+1)/K - 1).
__host__ __device__ __forceinline__ int64_t own_step_from(int64_t n, int K)
{
    return (n + K) / K - 1;
}
// The clock bits of an event at own step `own` (pending: a candidate).
__host__ __device__ __forceinline__ uint32_t clock_bits(int64_t own, bool pending)
{
    return ((uint32_t)(own & (int64_t)kClockDue) | (pending ? kClockPending : 0u)) << kClockShift;
}

// Device status word bits (latched, reported by synchronising calls).
enum : unsigned {
    kErrCapacity = 1u,
    kErrNonFinite = 2u,
    kErrInput = 4u,
    kErrEvents = 8u,
    kErrTimeout = 16u,
    kErrBounds = 32u,  // the bounds-checked build refused an index (see in_range)
};

// Philox counter word 3: what a draw is for.
enum : uint32_t {
    kRngCollide = 0, kRngScatter = 1, kRngMaxwell = 2, kRngInjectA = 3, kRngInjectB = 4,
    kRngIonizeE = 5, kRngIonizeI = 6,
};

// Per-segment (instance, species) constants, derived on the host from pic_instance.
struct SegParams {
    int32_t inst;          // instance index
    int32_t species;       // species index within the instance
    int32_t ncells;        // N of the instance
    int32_t bc;            // PIC_BC_*
    int64_t base;          // first slot of the segment
    int64_t cap;           // slots (multiple of kSegAlign)
    int64_t node;          // first entry of this segment's node arrays
    int64_t inode;         // first entry of the instance's node arrays (E)
    uint32_t key0, key1;   // Philox key = instance seed
    double accel;          // c_s = (q/m) dt^2/dx: A = c_s E in cells/step^2
    double t[3], s[3];     // Boris: t = (q/m) B dt/2, s = 2t/(1+t.t)
    float tf[3], sf[3];    // the same rounded to float (the FP32 form's values)
    double kefac;          // w m (dx/dt)^2 / 2: energy of |u|^2 = 1 (cells/step)^2
    double vinj;           // sqrt(T_s/m_s) in cells/step (volume source)
    double vneutral;       // sqrt(T_n/m_n) in cells/step
    double mratio;         // m_s / m_neutral (elastic energy transfer)
    uint32_t gap[kGapMax + 1];     // gap[g] = floor((1-P)^g 2^32), P = 1 - exp(-nu_max dt)
    float glog;            // 1 / log2(1-P) (0 without collisions): first guess of gap_steps
    int32_t nproc;         // processes of this species (list order)
    int32_t proc[kMaxProc];        // instance-level index of each process
    int32_t kind[kMaxProc];        // PIC_PROC_*
    int32_t product[kMaxProc];     // ionization: segment index of the new ion
    uint64_t slot_end[kMaxProc];   // cumulative slot bounds in [0, 2^32]
    double thr_u2[kMaxProc];       // energy threshold as |u|^2 (cells/step)^2
    int32_t collide;       // any process
    int32_t nstep;         // subcycling: moved on the steps n with (n+1) mod nstep = 0
    int32_t is_target;     // the instance's neutral particle target
    int32_t mag;           // the instance has a magnetic field (Boris push)
    int32_t sn2d;          // the species also drifts in y (Listing 1: yp += nstep*vy)
    int32_t pad;
};

// A segment whose fixed-point deposit is kept from step to step instead of being formed
// anew: a neutral particle target that moves only on some steps (subcycled).  Its
// charge is 0, so the kept deposit serves the density diagnostic alone; the mover
// skips its tiles between its moves and, on a move, takes the old positions' share
// away and adds the new one; a conversion into an ion takes the particle's share away.
__host__ __device__ __forceinline__ bool deposit_kept(const SegParams& P)
{
    return P.is_target != 0 && P.nstep > 1;
}

// The origin of a segment's clocks at step n (loads and reads count from it): its own
// index of the next moving step.  A species without collisions never looks at its clock
// and keeps the one it was loaded with, unchanged (origin 0).
__host__ __device__ __forceinline__ int64_t clock_origin(const SegParams& P, int64_t n)
{
    return P.collide ? own_step_from(n, P.nstep) : 0;
}
// The cell word of a particle placed in cell j after the mover of step n (created,
// re-injected, converted): its clock tests on the species' next moving step.
__host__ __device__ __forceinline__ int fresh_word(const SegParams& P, int j, int64_t n)
{
    return (int)((uint32_t)j | clock_bits(clock_origin(P, n + 1), false));
}

constexpr int kChunk = 256;  // nodes per block of the field solve

struct InstParams {
    int32_t ncells;
    int32_t field;         // PIC_FIELD_*
    int32_t seg0;          // first segment
    int32_t nseg;          // segments (= nspecies)
    int32_t chunk0;        // first field-solve chunk of this instance
    int32_t nchunk;        // chunks of ncells+1 nodes
    int64_t inode;         // first entry of E
    int64_t ev_base;       // first entry in the ionization event buffer
    int64_t ev_cap;        // event buffer entries of this instance
    double lambda;         // E = lambda * G (integer field numerator G)
    int32_t z[kMaxSpecies]; // charge q_s w_s in integer multiples of the unit delta
    int32_t smooth;        // density smoother on: the field uses 4x the filtered charges
    // neutral particle target (-1: uniform background): its segment, the reference
    // count per cell, the product ion segment of ionizations and the factor K_ion /
    // K_target that turns a target velocity into the ion's cells per step
    int32_t tseg;
    int32_t nref;
    int32_t iseg;
    int32_t pad;
    double tratio;
};

// A particle the mover leaves to the event kernel (a null-collision candidate, a wall
// hit, or a collision-clock test that the mover variant without the test left over),
// packed in 64 bits: kind in bits 0-1, segment in bits 2-23, store slot in bits 24-63.
enum : uint32_t { kRareCandidate = 0, kRareWallLow = 1, kRareWallHigh = 2, kRareTest = 3 };
constexpr int kRareSegBits = 22;
constexpr int kMaxSegments = 1 << kRareSegBits;
__host__ __device__ __forceinline__ uint64_t rare_pack(int64_t slot, int seg, uint32_t kind)
{
    return ((uint64_t)slot << 24) | ((uint64_t)(uint32_t)seg << 2) | (uint64_t)kind;
}

struct Event {            // one ionization event awaiting child ids
    uint32_t parent;
    uint32_t pad;
    int64_t slot_e;       // global slot of the new electron
    int64_t slot_i;       // global slot of the new ion
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// products on counter words 0 and 2, mixed with words 1, 3 and the key; the key is
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // one 32x32->64 multiply-wide per product: hi and lo come out together
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// Number of candidate-free steps, counted from the current one, that the word w
// encodes: the largest g <= 127 with w < gap[g] (0 if none), so P(g >= k) = (1-P)^k.
// gap[g] ~ (1-P)^g 2^32, so g ~ log2(w 2^-32) / log2(1-P): that first guess (float
// logarithm) is off by at most a step or so, and the table, non-increasing with
// gap[0] = 2^32 - 1, then decides exactly in a read or two (instead of the seven
// dependent reads of a binary search, at addresses that differ across the warp).
__device__ __forceinline__ int gap_steps(const uint32_t* __restrict__ gap, float glog, uint32_t w)
{
    const float t = (__log2f(fmaxf((float)w, 1.0f)) - 32.0f) * glog;
    int g = (int)fminf(fmaxf(t, 0.0f), (float)kGapMax);
    while (g > 0 && w >= __ldg(gap + g)) --g;
    while (g < kGapMax && w < __ldg(gap + g + 1)) ++g;
    return g;
}

// Draw of one purpose for particle `id` in step `step`.
__device__ __forceinline__ uint4 draw(uint32_t id, int64_t step, uint32_t purpose,
                                      uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(id, (uint32_t)((uint64_t)step >> 32), (uint32_t)step, purpose),
                         k0, k1);
}

// ---------------------------------------------------------------------------
// 128-bit integers (the field solve is exact integer arithmetic).
typedef __int128 i128;

// Correctly rounded i128 -> double: keep the top 64 significant bits with a sticky
// bit for everything shifted out, convert with round-to-nearest, rescale exactly.
__device__ __forceinline__ double i128_to_double(i128 x)
{
    const bool neg = x < 0;
    unsigned __int128 m = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const uint64_t hi = (uint64_t)(m >> 64);
    double r;
    if (hi == 0) {
        r = __ull2double_rn((uint64_t)m);
    } else {
        const int sh = 64 - __clzll((long long)hi);  // 1..64 bits in the high word
        uint64_t t = (uint64_t)(m >> sh);
        const unsigned __int128 rest = m & (((unsigned __int128)1 << sh) - 1);
        if (rest != 0) t |= 1u;
        r = __ull2double_rn(t) * __longlong_as_double((long long)(1023 + sh) << 52);
    }
    return neg ? -r : r;
}

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int d)
{
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)((unsigned __int128)v >> 64);
    const uint64_t l2 = __shfl_up_sync(0xffffffffu, lo, d);
    const uint64_t h2 = __shfl_up_sync(0xffffffffu, hi, d);
    return (i128)(((unsigned __int128)h2 << 64) | l2);
}

__device__ __forceinline__ i128 shfl_i128(i128 v, int src)
{
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)((unsigned __int128)v >> 64);
    const uint64_t l2 = __shfl_sync(0xffffffffu, lo, src);
    const uint64_t h2 = __shfl_sync(0xffffffffu, hi, src);
    return (i128)(((unsigned __int128)h2 << 64) | l2);
}

__device__ __forceinline__ void set_error(unsigned* err, unsigned bit) { atomicOr(err, bit); }

// The bounds-checked device build (compiled with -DPIC_CHECKED): every index a kernel
// computes into a particle store, a node array, a queue or a staging buffer is checked
// against its range before it is used; a violation latches kErrBounds (reported by the
// next synchronising call) and the access is skipped, so nothing traps.  In the normal
// build the check is a constant true and costs nothing.
#ifdef PIC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool in_range(unsigned* err, int64_t i, int64_t lo, int64_t hi)
{
    if (!kChecked) return true;
    if (i >= lo && i < hi) return true;
    set_error(err, kErrBounds);
    return false;
}

// Segment of tile t: the last s with tile_start[s] <= t (tile_start has nseg+1 entries).
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ tile_start, int nseg,
                                            int64_t t)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The segment of tile t for a walker whose tiles only increase: from its previous
// segment s (tiles [tile_start[s], end) with end = tile_start[s+1] cached by the
// caller), a few steps forward, else a binary search over the rest.
__device__ __forceinline__ int advance_segment(const int64_t* __restrict__ tile_start, int nseg,
                                               int s, int64_t t)
{
#pragma unroll 1
    for (int it = 0; it < 3; ++it) {
        if (s + 1 >= nseg || __ldg(tile_start + s + 1) > t) return s;
        ++s;
    }
    int lo = s, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace bitpic
