// sort.cu -- periodic counting sort of every segment by cell.
//
// The paper keeps particles in per-cell lists ("natural sorting", Section 2, Fig.
// "BIT1_sorting") so that particles near in space are near in memory.  Here the same
// locality comes from a compact structure-of-arrays store that is re-sorted by cell
// every few steps: histogram of cells -> exclusive scan per segment -> scatter into
// the second copy of the store, which drops the empty slots left by absorbed
// particles.  Results of the time step do not depend on particle order (deposits
// are integer, random draws are keyed by particle id), so the order inside a cell
// is free.  Usually the histogram comes from the step before the sort and the scatter
// is done by the sort step's mover (mover.cuh); this file then runs only the scan and
// the finish, and the whole sort below serves the remaining cases.
#include <algorithm>

#include "kernels.h"
#include "mover.cuh"

namespace bitpic {

namespace {

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_hist(const SortArgs a)
{
    const int32_t* cell = a.cell[a.src];
    const int64_t total = a.tile_start[a.nseg];
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * (NT / 32);
    for (int64_t tile = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5); tile < total;
         tile += wstride) {
        const int s = find_segment(a.tile_start, a.nseg, tile);
        const SegParams& P = a.seg[s];
        const int64_t quad = (tile - a.tile_start[s]) * 32 + lane;
        const int64_t nq = a.seg_nmove[s] >> 2;
        int c[4] = {-1, -1, -1, -1};
        if (quad < nq && in_range(a.err, 4 * quad + 3, 0, P.cap)) {
            const int4 cc = *reinterpret_cast<const int4*>(cell + P.base + 4 * quad);
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (c[k] >= 0 && !in_range(a.err, (int)((uint32_t)c[k] & kCellMask), 0, P.ncells))
                c[k] = -1;  // (bounds-checked build only)
            // sort key: the cell index (empty slots get distinct keys and never group)
            const int key = c[k] >= 0 ? (int)((uint32_t)c[k] & kCellMask) : -1 - lane;
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            if (c[k] >= 0 && lane == __ffs(grp) - 1)
                atomicAdd(a.hist + P.node + key, (unsigned)__popc(grp));
        }
    }
}

// Exclusive scan of the cell histogram of every segment in place, in chunks of
// kCellChunk cells (blocks (segment, chunk), coalesced): k_cell_partial sums each chunk,
// k_cell_scan adds the sums of the segment's earlier chunks and scans its own.
constexpr int kCellThreads = 1024;
constexpr int kCellRounds = 4;
constexpr int kCellChunk = kCellThreads * kCellRounds;

__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v,
                                                            unsigned long long* total,
                                                            unsigned long long* sh /* 33 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const unsigned long long w = lane < nw ? sh[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += t;
        }
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[32] = wi;
    }
    __syncthreads();
    const unsigned long long out = sh[warp] + inc - v;
    *total = sh[32];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(kCellThreads) k_cell_partial(const SortArgs a)
{
    __shared__ unsigned long long sh[33];
    const SegParams& P = a.seg[blockIdx.x];
    const int c = blockIdx.y;
    const int N = P.ncells;
    if ((int64_t)c * kCellChunk >= N) return;
    unsigned long long local = 0;
#pragma unroll
    for (int r = 0; r < kCellRounds; ++r) {
        const int j = c * kCellChunk + r * kCellThreads + threadIdx.x;
        if (j < N) local += a.hist[P.node + j];
    }
    unsigned long long tot;
    block_scan_u64(local, &tot, sh);
    if (threadIdx.x == 0) a.cell_part[(int64_t)blockIdx.x * a.cell_chunks + c] = tot;
}

__global__ void __launch_bounds__(kCellThreads) k_cell_scan(const SortArgs a)
{
    __shared__ unsigned long long sh[33];
    const SegParams& P = a.seg[blockIdx.x];
    const int c = blockIdx.y;
    const int N = P.ncells;
    const int nch = (N + kCellChunk - 1) / kCellChunk;
    if (c >= nch) return;
    const unsigned long long* part = a.cell_part + (int64_t)blockIdx.x * a.cell_chunks;
    unsigned long long run = 0;
    for (int k = threadIdx.x; k < c; k += blockDim.x) run += part[k];
    unsigned long long off;
    block_scan_u64(run, &off, sh);  // off = the sum of all earlier chunks
    for (int r = 0; r < kCellRounds; ++r) {
        const int j = c * kCellChunk + r * kCellThreads + threadIdx.x;
        const unsigned h = j < N ? a.hist[P.node + j] : 0u;
        unsigned long long tot;
        const unsigned long long ex = block_scan_u64(h, &tot, sh);
        if (j < N) a.hist[P.node + j] = (unsigned)(off + ex);
        off += tot;
    }
    if (c == nch - 1 && threadIdx.x == 0) a.newn[blockIdx.x] = off;
}

// One lane's quad in flight through the scatter.
template <typename T>
struct SortQuad {
    int c[4];
    T vo[4], vx[4], vy[4], vz[4];
    uint32_t vi[4];
    int s;
    int64_t slot;
};

// Scatter.  Each warp keeps the loads of its next tile in flight while it reserves the
// destinations of the current one (an atomic round trip through L2 per cell group),
// so the reservation latency does not stall the stream of loads.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_scatter(const SortArgs a)
{
    const int src = a.src, dst = 1 - a.src;
    const int32_t* cell = a.cell[src];
    const T* off = static_cast<const T*>(a.off[src]);
    const T* ux = static_cast<const T*>(a.ux[src]);
    const T* uy = static_cast<const T*>(a.uy[src]);
    const T* uz = static_cast<const T*>(a.uz[src]);
    const uint32_t* id = a.id[src];
    int32_t* dcell = a.cell[dst];
    T* doff = static_cast<T*>(a.off[dst]);
    T* dux = static_cast<T*>(a.ux[dst]);
    T* duy = static_cast<T*>(a.uy[dst]);
    T* duz = static_cast<T*>(a.uz[dst]);
    uint32_t* did = a.id[dst];
    const T* yps = static_cast<const T*>(a.yp[src]);
    T* ypd = static_cast<T*>(a.yp[dst]);
    const int64_t total = a.tile_start[a.nseg];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t wstride = (int64_t)gridDim.x * (NT / 32);
    int ls = 0;                            // segment walk of the loads (tiles only increase)
    int64_t ls_begin = 0, ls_end = -1;
    auto load = [&](int64_t tile, SortQuad<T>& q) {
        if (tile >= ls_end) {
            ls = advance_segment(a.tile_start, a.nseg, ls, tile);
            ls_begin = __ldg(a.tile_start + ls);
            ls_end = __ldg(a.tile_start + ls + 1);
        }
        q.s = ls;
        const int64_t quad = (tile - ls_begin) * 32 + lane;
        q.slot = a.seg[ls].base + 4 * quad;
        q.c[0] = q.c[1] = q.c[2] = q.c[3] = -1;
        if (quad < (a.seg_nmove[ls] >> 2) && in_range(a.err, 4 * quad + 3, 0, a.seg[ls].cap)) {
            // the whole quad with 128-bit loads (the mover's access pattern)
            const int4 cc = __ldcs(reinterpret_cast<const int4*>(cell + q.slot));
            q.c[0] = cc.x; q.c[1] = cc.y; q.c[2] = cc.z; q.c[3] = cc.w;
            ld4(off + q.slot, q.vo);
            ld4(ux + q.slot, q.vx);
            ld4(uy + q.slot, q.vy);
            ld4(uz + q.slot, q.vz);
            const uint4 ii = __ldcs(reinterpret_cast<const uint4*>(id + q.slot));
            q.vi[0] = ii.x; q.vi[1] = ii.y; q.vi[2] = ii.z; q.vi[3] = ii.w;
        }
    };
    int64_t tile = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    SortQuad<T> cur;
    if (tile < total) load(tile, cur);
    for (; tile < total; tile += wstride) {
        SortQuad<T> nxt;
        nxt.c[0] = nxt.c[1] = nxt.c[2] = nxt.c[3] = -1;
        if (tile + wstride < total) load(tile + wstride, nxt);
        const SegParams& P = a.seg[cur.s];
        // group equal cells of each slot across the warp; the four reservations are
        // independent, so they are all issued before the first one is waited for
        unsigned grp[4], base[4];
        int key[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (cur.c[k] >= 0 &&
                !in_range(a.err, (int)((uint32_t)cur.c[k] & kCellMask), 0, P.ncells))
                cur.c[k] = -1;  // (bounds-checked build only)
            key[k] = cur.c[k] >= 0 ? (int)((uint32_t)cur.c[k] & kCellMask) : -1 - lane;
            grp[k] = __match_any_sync(0xffffffffu, key[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            base[k] = 0;
            if (cur.c[k] >= 0 && lane == __ffs(grp[k]) - 1)
                base[k] = atomicAdd(a.hist + P.node + key[k], (unsigned)__popc(grp[k]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned b = __shfl_sync(0xffffffffu, base[k], __ffs(grp[k]) - 1);
            if (cur.c[k] >= 0 && in_range(a.err, (int64_t)b + __popc(grp[k] & lt), 0, P.cap)) {
                const int64_t to = P.base + (int64_t)b + __popc(grp[k] & lt);
                dcell[to] = cur.c[k];
                doff[to] = cur.vo[k];
                dux[to] = cur.vx[k];
                duy[to] = cur.vy[k];
                duz[to] = cur.vz[k];
                did[to] = cur.vi[k];
                if (yps) ypd[to] = yps[cur.slot + k];
            }
        }
        cur = nxt;
    }
}

// Per segment: mark the destination's slots past the new count empty, then adopt the
// new count.  The destination copy may still hold particles up to its own earlier
// high-water mark.
__global__ void k_sort_finish(const SortArgs a)
{
    const int s = blockIdx.x;
    const SegParams& P = a.seg[s];
    const unsigned long long nnew = a.newn[s];
    const unsigned long long old = a.seg_n[s];
    const unsigned long long hw = min(max(old, a.hwm_alt[s]), (unsigned long long)P.cap);
    int32_t* dcell = a.cell[1 - a.src];
    for (unsigned long long i = nnew + threadIdx.x; i < hw; i += blockDim.x) dcell[P.base + (int64_t)i] = -1;
    __syncthreads();
    if (threadIdx.x == 0) {
        a.hwm_alt[s] = old;
        a.seg_n[s] = nnew;
        a.seg_live[s] = nnew;
    }
}

// One resident wave of a grid-stride kernel: blocks per SM at full occupancy x SMs
// (a second, partial wave would run its share of the tiles at a fraction of the
// machine).
template <typename K>
int one_wave(K kernel, int nt, int sms)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, nt, 0) != cudaSuccess || nb < 1)
        nb = 1;
    return nb * sms;
}

// Neutral particle targets: the live particles of every cell, from the cell ends the
// scatter left in the histogram.  One thread per node of all segments.
__global__ void __launch_bounds__(256) k_target_counts(const SortArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < a.seg_nodes; n += stride) {
        int lo = 0, hi = a.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.seg[mid].node <= n) lo = mid; else hi = mid - 1;
        }
        const SegParams& P = a.seg[lo];
        const int j = (int)(n - P.node);
        if (!P.is_target || j >= P.ncells) continue;
        a.tcount[n] = a.hist[n] - (j > 0 ? a.hist[n - 1] : 0u);
    }
}

template <int NT>
cudaError_t run_sort(const SortArgs& a, int sms, cudaStream_t st)
{
    k_hist<NT><<<one_wave(k_hist<NT>, NT, sms), NT, 0, st>>>(a);
    const dim3 cg(a.nseg, a.cell_chunks);
    k_cell_partial<<<cg, kCellThreads, 0, st>>>(a);
    k_cell_scan<<<cg, kCellThreads, 0, st>>>(a);
    if (a.precision == PIC_FP64)
        k_scatter<double, NT><<<one_wave(k_scatter<double, NT>, NT, sms), NT, 0, st>>>(a);
    else
        k_scatter<float, NT><<<one_wave(k_scatter<float, NT>, NT, sms), NT, 0, st>>>(a);
    k_sort_finish<<<a.nseg, 256, 0, st>>>(a);
    if (a.tcount)
        k_target_counts<<<(int)std::min<int64_t>((a.seg_nodes + 255) / 256, 64 * sms), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sort_scan(const SortArgs& a, cudaStream_t st)
{
    const dim3 cg(a.nseg, a.cell_chunks);
    k_cell_partial<<<cg, kCellThreads, 0, st>>>(a);
    k_cell_scan<<<cg, kCellThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sort_finish(const SortArgs& a, cudaStream_t st)
{
    k_sort_finish<<<a.nseg, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sort(const SortArgs& a, int nt, int sms, cudaStream_t st)
{
    switch (nt) {
        case 128: return run_sort<128>(a, sms, st);
        case 512: return run_sort<512>(a, sms, st);
        default: return run_sort<256>(a, sms, st);
    }
}

}  // namespace bitpic
