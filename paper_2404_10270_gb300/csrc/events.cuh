// events.cuh -- the rare events of a time step, worked through after the mover:
// null-collision candidates (Section 2: the MCC step of the PIC cycle; elastic,
// charge-exchange and ionization kinematics), collision-clock tests that the mover
// variant without the inline test left (a candidate of this same step when the draw
// says so) and particles that left through an absorbing or source wall (flux and
// energy counters, re-injection of the volume source).  The mover queues them
// (rare_pack) so that its own loop stays call-free; here one thread takes one queued
// particle.  Collisions change only velocities, so the mover has already deposited a
// candidate; a re-injected particle and the children of an ionization are deposited
// here (and, on the step before a sort, counted in the cell histogram).  Everything
// this kernel adds is an integer sum or keyed by particle id and step, so the order
// of the queue does not change any result.
#pragma once

#include "mover.cuh"

namespace bitpic {

// The cell word of a particle in cell j whose next collision event is a clock test on
// its species' own step m1: the test is drawn here already (word 0 of its counter, the
// global step of own step m1), so the mover finds the outcome in the clock instead of
// queueing the test: a candidate g own steps on (g < D), or the next test at the
// species' next multiple of kGapMax (g = D).  Exactly what the test at m1 would set; a
// species without collisions keeps clock 0.
__device__ __forceinline__ int test_word(const SegParams& P, uint32_t id, int j, int64_t m1)
{
    if (!P.collide) return j;
    const int64_t n1 = (m1 + 1) * (int64_t)P.nstep - 1;
    const int dg = kGapMax - (int)(m1 % kGapMax);
    const uint4 w = draw(id, n1, kRngCollide, P.key0, P.key1);
    const int g = min(gap_steps(P.gap, P.glog, w.x), dg);
    return (int)((uint32_t)j | clock_bits(m1 + g, g < dg));
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

// A null-collision candidate of one particle (velocity u in cells/step, after the
// move): with a neutral particle target, first the target density (kept with
// probability min(1, n_j / nref) by the word `wdens`), then the process slot from the
// selection word `wsel`, energy threshold (below it the event is a null collision),
// kinematics.  Returns the instance-level index of the process that took place (u
// changed), or -1 for a null event.  Ionization appends two particles (the electron
// only with a particle target: the target particle itself becomes the ion, see
// k_victims).  The caller counts the collision.
template <typename T>
__device__ __forceinline__ int collide(const MoveArgs& a, const SegParams& P, int s,
                                    uint32_t id, int64_t step, int j, T f, T& ux, T& uy,
                                    T& uz, uint32_t wsel, uint32_t wdens, int64_t pslot)
{
    const InstParams& I = a.inst[P.inst];
    if (I.tseg >= 0) {
        const uint64_t nj = a.tcount[a.seg[I.tseg].node + j];
        const uint64_t nr = (uint64_t)I.nref;
        if (nj < nr && (uint64_t)wdens >= (nj << 32) / nr) return -1;
    }
    int q = -1;
    for (int k = 0; k < P.nproc; ++k)
        if ((uint64_t)wsel < P.slot_end[k]) { q = k; break; }
    if (q < 0) return -1;
    const T u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 >= (T)P.thr_u2[q])) return -1;  // below threshold: null event
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
    } else if (kind == PIC_PROC_EXCITE) {
        // the electron loses the threshold energy and leaves in a direction uniform
        // on the sphere
        const uint4 r = draw(id, step, kRngScatter, P.key0, P.key1);
        T n[3];
        iso_dir<T>(r.x, r.y, n);
        const T sp2 = Prec<T>::sqrt_(u2 - (T)P.thr_u2[q]);
        ux = sp2 * n[0];
        uy = sp2 * n[1];
        uz = sp2 * n[2];
    } else {  // PIC_PROC_IONIZE
        const T us = Prec<T>::sqrt_(T(0.5) * (u2 - (T)P.thr_u2[q]));
        T n1[3], n2[3];
        const uint4 r1 = draw(id, step, kRngScatter, P.key0, P.key1);
        iso_dir<T>(r1.x, r1.y, n1);
        const uint4 r2 = draw(id, step, kRngIonizeE, P.key0, P.key1);
        iso_dir<T>(r2.x, r2.y, n2);
        ux = us * n1[0];
        uy = us * n1[1];
        uz = us * n1[2];
        const InstParams& Ii = a.inst[P.inst];
        const unsigned long long ev = atomicAdd(a.ev_count + P.inst, 1ull);
        const unsigned long long ke = atomicAdd(a.seg_n + s, 1ull);
        const bool target = Ii.tseg >= 0;
        // the new ion: a new particle of the product segment, or (particle target) the
        // target particle that k_victims converts
        const int si = P.product[q];
        const SegParams& Pi = a.seg[si];
        const unsigned long long ki = target ? 0ull : atomicAdd(a.seg_n + si, 1ull);
        if (ke >= (unsigned long long)P.cap || ki >= (unsigned long long)Pi.cap ||
            ev >= (unsigned long long)Ii.ev_cap) {
            set_error(a.err, kErrCapacity);
            if (ev < (unsigned long long)Ii.ev_cap) {
                // the record k_births reads must exist: an empty one
                Event e;
                e.parent = id;
                e.pad = 0;
                e.slot_e = -1;
                e.slot_i = -1;
                a.events[Ii.ev_base + (int64_t)ev] = e;
            }
        } else {
            const int64_t ge = P.base + (int64_t)ke;
            T* off = static_cast<T*>(a.off);
            T* vx = static_cast<T*>(a.ux);
            T* vy = static_cast<T*>(a.uy);
            T* vz = static_cast<T*>(a.uz);
            // fresh clocks: a test on the species' next moving step
            a.cell[ge] = fresh_word(P, j, step);
            off[ge] = f;
            vx[ge] = us * n2[0]; vy[ge] = us * n2[1]; vz[ge] = us * n2[2];
            a.id[ge] = 0xFFFFFFFFu;
            // the products start at the parent's y coordinate (2-D species)
            T* const ypp = static_cast<T*>(a.yp);
            const T yparent = ypp ? ypp[pslot] : T(0);
            if (ypp) ypp[ge] = P.sn2d ? yparent : T(0);
            atomicAdd(a.seg_live + s, 1ull);
            // the children's charge joins this step's deposit
            const uint64_t qr = Prec<T>::qright(f), ql = Prec<T>::S - qr;
            atomicAdd(a.dep + P.node + j, (unsigned long long)ql);
            atomicAdd(a.dep + P.node + j + 1, (unsigned long long)qr);
            if (a.hist_out) atomicAdd(a.hist_out + P.node + j, 1u);
            Event e;
            e.parent = id;
            e.pad = 0;
            e.slot_e = ge;
            e.slot_i = -1;
            if (target) {
                // the first request of a target cell puts it on the step's list
                const int64_t tn = a.seg[Ii.tseg].node + j;
                if (atomicAdd(a.treq + tn, 1u) == 0u) {
                    const unsigned long long vi = atomicAdd(a.rare_count + 1, 1ull);
                    if (vi < (unsigned long long)a.vcap) a.vlist[vi] = tn;
                    else set_error(a.err, kErrCapacity);
                }
            } else {
                const uint4 ri = draw(id, step, kRngIonizeI, P.key0, P.key1);
                T z0, z1, z2, z3;
                box_muller<T>(ri.x, ri.y, &z0, &z1);
                box_muller<T>(ri.z, ri.w, &z2, &z3);
                const T vn = (T)Pi.vneutral;  // the ion's velocity in its own species' units
                const int64_t gi = Pi.base + (int64_t)ki;
                a.cell[gi] = fresh_word(Pi, j, step);
                off[gi] = f;
                vx[gi] = z0 * vn; vy[gi] = z1 * vn; vz[gi] = z2 * vn;
                a.id[gi] = 0xFFFFFFFFu;
                if (ypp) ypp[gi] = Pi.sn2d ? yparent : T(0);
                e.slot_i = gi;
                atomicAdd(a.seg_live + si, 1ull);
                atomicAdd(a.dep + Pi.node + j, (unsigned long long)ql);
                atomicAdd(a.dep + Pi.node + j + 1, (unsigned long long)qr);
                if (a.hist_out) atomicAdd(a.hist_out + Pi.node + j, 1u);
            }
            a.events[Ii.ev_base + (int64_t)ev] = e;
        }
    }
    return P.proc[q];
}

// Wall phase for a particle that left [0, N) (rare): energy of the absorbed particle
// (the caller counts it), then either absorption (returns 2), or volume re-injection
// with a new position and Maxwellian velocity (returns 1).  Periodic walls are handled
// in the mover.
template <typename T>
__device__ __forceinline__ int wall_event(const MoveArgs& a, const SegParams& P, int s, uint32_t id,
                                       int64_t step, int& j, T& f, T& ux, T& uy, T& uz)
{
    const int wall = j < 0 ? 0 : 1;
    const double u2 = (double)ux * (double)ux + (double)uy * (double)uy + (double)uz * (double)uz;
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

// Add `key`'s count once per group of lanes with the same key (key < 0: nothing).
// Same-address atomics from every event would queue behind each other in L2.
__device__ __forceinline__ void count_by_key(unsigned long long* counts, int key)
{
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1)
        atomicAdd(counts + key, (unsigned long long)__popc(grp));
}

// One thread per queued particle.  The loop is uniform across each warp (every lane
// takes the same iterations), so that the collision and wall counts can be combined
// per warp before they reach memory.
template <typename T>
__global__ void __launch_bounds__(128) k_events(const __grid_constant__ MoveArgs a)
{
    const unsigned long long n = min(*a.rare_count, (unsigned long long)a.rare_cap);
    const int64_t step = *a.step;
    // the movers of this step have read it: from the next step on, clocks that need a
    // test off the common test steps are queued again
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.test_all) *a.test_all = 0;
    T* const offp = static_cast<T*>(a.off);
    T* const uxp = static_cast<T*>(a.ux);
    T* const uyp = static_cast<T*>(a.uy);
    T* const uzp = static_cast<T*>(a.uz);
    const unsigned long long lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         w < n; w += stride) {
        const unsigned long long i = w + lane;
        int ckey = -1, wkey = -1;  // collision counter, wall counter
        bool ok = i < n;
        uint64_t e = 0;
        if (ok) {
            e = a.rare[i];
            // (bounds-checked build: the entry's segment and slot)
            const int s0 = (int)((e >> 2) & (uint64_t)(kMaxSegments - 1));
            ok = in_range(a.err, s0, 0, a.nseg) &&
                 in_range(a.err, (int64_t)(e >> 24), a.seg[s0].base, a.seg[s0].base + a.seg[s0].cap);
        }
        if (ok) {
            const uint32_t kind = (uint32_t)(e & 3u);
            const int s = (int)((e >> 2) & (uint64_t)(kMaxSegments - 1));
            const int64_t slot = (int64_t)(e >> 24);
            const SegParams& P = a.seg[s];
            const uint32_t id = a.id[slot];
            // a clock test needs only the id and the cell word; the state is read when the
            // particle collides or left through a wall (a candidate and a wall hit need it
            // in any case: read together with the id, one round trip to memory fewer)
            T f = T(0), vx = T(0), vy = T(0), vz = T(0);
            if (kind != kRareTest) {
                f = offp[slot];
                vx = uxp[slot];
                vy = uyp[slot];
                vz = uzp[slot];
            }
            if ((kind == kRareCandidate || kind == kRareTest) &&
                in_range(a.err, (int)((uint32_t)a.cell[slot] & kCellMask), 0, P.ncells)) {
                const int j = (int)((uint32_t)a.cell[slot] & kCellMask);
                const uint4 wd = draw(id, step, kRngCollide, P.key0, P.key1);
                bool now = kind == kRareCandidate;
                if (!now) {
                    // the clock test the mover left: word 0 gives the candidate-free run
                    // from this step, cut at the species' next multiple of kGapMax steps
                    const int ks = P.nstep;
                    const int64_t q = ks == 1 ? step + 1 : (step + 1) / ks;
                    const int dgrid = kGapMax - (int)((q - 1) % kGapMax);
                    const int g = min(gap_steps(P.gap, P.glog, wd.x), dgrid);
                    now = g == 0;
                    // the next event: a test next step after a candidate now, else the
                    // candidate g steps on, or the test at the grid step
                    const int64_t mown = q - 1;
                    a.cell[slot] = (int)((uint32_t)j | clock_bits(g == 0 ? mown + 1 : mown + g,
                                                                  g > 0 && g < dgrid));
                }
                if (now) {
                    if (kind == kRareTest) {
                        f = offp[slot];
                        vx = uxp[slot];
                        vy = uyp[slot];
                        vz = uzp[slot];
                    }
                    const int p = collide<T>(a, P, s, id, step, j, f, vx, vy, vz, wd.y, wd.z,
                                             slot);
                    if (p >= 0) {
                        uxp[slot] = vx;
                        uyp[slot] = vy;
                        uzp[slot] = vz;
                        ckey = P.inst * kMaxProc + p;
                    }
                    // a candidate is followed by a test on the next own step: drawn now
                    const int ks = P.nstep;
                    const int64_t q = ks == 1 ? step + 1 : (step + 1) / ks;  // own step q - 1
                    a.cell[slot] = test_word(P, id, j, q);
                }
            } else if (kind == kRareWallLow || kind == kRareWallHigh) {
                int j = kind == kRareWallLow ? -1 : P.ncells;
                wkey = 2 * s + (kind == kRareWallLow ? 0 : 1);
                if (wall_event<T>(a, P, s, id, step, j, f, vx, vy, vz) == 1) {
                    // re-injected: back in the store with a fresh clock (and y coordinate),
                    // deposited here
                    if (a.yp) static_cast<T*>(a.yp)[slot] = T(0);
                    a.cell[slot] = test_word(P, id, j, own_step_from(step + 1, P.nstep));
                    offp[slot] = f;
                    uxp[slot] = vx;
                    uyp[slot] = vy;
                    uzp[slot] = vz;
                    const uint64_t qr = Prec<T>::qright(f);
                    atomicAdd(a.dep + P.node + j, (unsigned long long)(Prec<T>::S - qr));
                    atomicAdd(a.dep + P.node + j + 1, (unsigned long long)qr);
                    if (a.hist_out) atomicAdd(a.hist_out + P.node + j, 1u);
                }
            }
        }
        count_by_key(a.collisions, ckey);
        count_by_key(a.wall_count, wkey);
    }
}

// Ionization against a neutral particle target: the r_j ionizations of cell j this step
// turn the r_j live target particles of cell j with the smallest ids (as of the start
// of the step: the cell's range of the target segment after the last sort, which the
// target has not left since, since it moves only on the sort steps) into product ions:
// same id, position and physical velocity (x K_ion / K_target in cells per step),
// collision clock 0.  The ion's charge joins this step's deposit and the target's
// (charge 0, but counted in its density) leaves it.  A cell with fewer targets than
// ionizations converts what it has.  One warp per target cell on the step's request
// list (k_events puts a cell there with its first request): it scans the cell's range
// together (32 entries per pass) for the next smallest live id.
template <typename T>
__global__ void __launch_bounds__(128) k_victims(const __grid_constant__ MoveArgs a)
{
    const unsigned FULL = 0xffffffffu;
    T* const offp = static_cast<T*>(a.off);
    T* const uxp = static_cast<T*>(a.ux);
    T* const uyp = static_cast<T*>(a.uy);
    T* const uzp = static_cast<T*>(a.uz);
    const int lane = threadIdx.x & 31;
    const int64_t step = *a.step;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nv = (int64_t)min(a.rare_count[1], (unsigned long long)a.vcap);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nv; w += nw) {
        const int64_t n = a.vlist[w];
        const unsigned r = a.treq[n];
        __syncwarp();
        if (lane == 0) a.treq[n] = 0u;
        {
            // the segment of node n (segments' node arrays are in increasing order)
            int lo = 0, hi = a.nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.seg[mid].node <= n) lo = mid; else hi = mid - 1;
            }
            const int ts = lo;
            const SegParams& P = a.seg[ts];
            const int j = (int)(n - P.node);
            const InstParams& I = a.inst[P.inst];
            const SegParams& Pi = a.seg[I.iseg];
            if (!in_range(a.err, j, 0, P.ncells)) continue;  // (bounds-checked build only)
            const int64_t begin = P.base + (j > 0 ? (int64_t)a.hist[n - 1] : 0);
            int64_t end = P.base + (int64_t)a.hist[n];
            if (!in_range(a.err, end - 1, begin - 1, P.base + P.cap)) end = begin;
            // a range of up to 128 targets (the usual ~nref) is read once, four entries per
            // lane with their cell and id loads issued together, and every selection below
            // works on registers; a longer range is scanned again for each conversion
            const bool held = end - begin <= 128;
            uint32_t hid[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t g = begin + lane + 32 * q;
                hid[q] = 0xFFFFFFFFu;  // not live (no live target has this id: ids < 2^32 - 1)
                if (held && g < end) {
                    const int cg = a.cell[g];
                    const uint32_t ig = a.id[g];
                    if (cg >= 0) hid[q] = ig;
                }
            }
            uint32_t last = 0;
            bool first = true;
            for (unsigned k = 0; k < r; ++k) {
                // the next smallest live id of the range
                uint32_t best = 0xFFFFFFFFu;
                int64_t v = -1;
                if (held) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (hid[q] != 0xFFFFFFFFu && (first || hid[q] > last) && hid[q] < best) {
                            best = hid[q];
                            v = begin + lane + 32 * q;
                        }
                } else {
                    for (int64_t g0 = begin; g0 < end; g0 += 32) {
                        const int64_t g = g0 + lane;
                        if (g < end && a.cell[g] >= 0) {
                            const uint32_t idg = a.id[g];
                            if ((first || idg > last) && idg < best) {
                                best = idg;
                                v = g;
                            }
                        }
                    }
                }
                const uint32_t wbest = __reduce_min_sync(FULL, best);
                const unsigned owner = __ballot_sync(FULL, v >= 0 && best == wbest);
                if (owner == 0u) break;  // no live target left in the cell
                first = false;
                last = wbest;
                if (lane == __ffs(owner) - 1) {
                    const unsigned long long ki = atomicAdd(a.seg_n + I.iseg, 1ull);
                    if (ki >= (unsigned long long)Pi.cap) {
                        set_error(a.err, kErrCapacity);
                    } else {
                        const int64_t gi = Pi.base + (int64_t)ki;
                        const int jv = (int)((uint32_t)a.cell[v] & kCellMask);
                        const T fv = offp[v];
                        const T ratio = (T)I.tratio;
                        a.cell[gi] = test_word(Pi, wbest, jv, own_step_from(step + 1, Pi.nstep));
                        offp[gi] = fv;
                        uxp[gi] = uxp[v] * ratio;
                        uyp[gi] = uyp[v] * ratio;
                        uzp[gi] = uzp[v] * ratio;
                        a.id[gi] = wbest;
                        if (a.yp) static_cast<T*>(a.yp)[gi] = Pi.sn2d ? static_cast<T*>(a.yp)[v] : T(0);
                        a.cell[v] = -1;
                        const uint64_t qr = Prec<T>::qright(fv), ql = Prec<T>::S - qr;
                        atomicAdd(a.dep + Pi.node + jv, (unsigned long long)ql);
                        atomicAdd(a.dep + Pi.node + jv + 1, (unsigned long long)qr);
                        atomicAdd(a.dep + P.node + jv, (unsigned long long)(0ull - ql));
                        atomicAdd(a.dep + P.node + jv + 1, (unsigned long long)(0ull - qr));
                        atomicAdd(a.seg_live + ts, ~0ull);
                        atomicAdd(a.seg_live + I.iseg, 1ull);
                        a.tcount[n] -= 1u;
                    }
                }
                __syncwarp();
            }
        }
    }
}

// The y drift of 2-D species (Listing 1: yp += nstep*vy), after the mover and before
// the event kernel: every particle of such a species that moved this step (the store
// copy the step leaves, its live particles), with its velocity after the push in cells
// per own step.  A particle that left through a wall (empty in the store until the event
// kernel re-injects it) gets no drift; re-injection starts its y coordinate anew.
template <typename T>
__global__ void __launch_bounds__(256) k_drift_y(const __grid_constant__ MoveArgs a)
{
    const int64_t step = *a.step;
    T* const yp = static_cast<T*>(a.yp);
    const T* const uy = static_cast<const T*>(a.uy);
    const int64_t total = a.tile_start[a.nseg] * 128;  // tiles of 32 quads
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int s = 0;
    int64_t s_begin = 0, s_end = -1;
    bool on = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t tile = t >> 7;
        if (tile >= s_end) {
            s = advance_segment(a.tile_start, a.nseg, s, tile);
            s_begin = __ldg(a.tile_start + s);
            s_end = __ldg(a.tile_start + s + 1);
            const int ks = a.seg[s].nstep;
            on = a.seg[s].sn2d != 0 && (ks == 1 || (step + 1) % ks == 0);
        }
        if (!on) {  // on to this thread's first slot past the segment
            t += ((s_end * 128 - 1 - t) / stride) * stride;
            continue;
        }
        const int64_t k = (tile - s_begin) * 128 + (t & 127);
        if (k >= a.seg_nmove[s]) continue;
        if (!in_range(a.err, k, 0, a.seg[s].cap)) continue;  // (bounds-checked build only)
        const int64_t g = a.seg[s].base + k;
        if (a.cell[g] >= 0) yp[g] = yp[g] + uy[g];
    }
}

}  // namespace bitpic