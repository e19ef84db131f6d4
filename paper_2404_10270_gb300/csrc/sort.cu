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
// Scatter.  A block takes NT/32 consecutive tiles (a chunk of up to 128 NT/32
// particles).  When the chunk lies in one segment and its particles' cells span fewer
// than kSortSpan cells (the common case: the store was sorted one cycle ago), the block
// ranks them per cell in shared memory, reserves each cell's run with one global atomic
// per cell, stages the particles in shared memory in that order and writes every run
// with consecutive threads, so the scattered writes become coalesced runs of about a
// cell's share of the chunk (the same staging as the sort step's mover, without its
// physics).  Otherwise each warp reserves per cell and quad position and writes its
// particles directly.
template <typename T, int NT, bool YP>
__global__ void __launch_bounds__(NT) k_scatter(const SortArgs a)
{
    constexpr int NW = NT / 32, C = NW * 128;
    const unsigned FULL = 0xffffffffu;
    const int src = a.src, dst = 1 - a.src;
    const int32_t* cell = a.cell[src];
    const T* off = static_cast<const T*>(a.off[src]);
    const T* ux = static_cast<const T*>(a.ux[src]);
    const T* uy = static_cast<const T*>(a.uy[src]);
    const T* uz = static_cast<const T*>(a.uz[src]);
    const T* yps = static_cast<const T*>(a.yp[src]);
    const uint32_t* id = a.id[src];
    int32_t* dcell = a.cell[dst];
    T* doff = static_cast<T*>(a.off[dst]);
    T* dux = static_cast<T*>(a.ux[dst]);
    T* duy = static_cast<T*>(a.uy[dst]);
    T* duz = static_cast<T*>(a.uz[dst]);
    T* ypd = static_cast<T*>(a.yp[dst]);
    uint32_t* did = a.id[dst];
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
    // per-warp summaries (segment, lowest and highest cell), double-buffered by chunk
    // parity: a warp may write the next chunk's entry while another still reads these
    int* const wsum = reinterpret_cast<int*>(gb + kSortSpan);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t total = a.tile_start[a.nseg];
    int s = 0;
    int64_t s_begin = 0, s_end = -1;
    int parity = 0;
    // every warp of the block walks the same chunks, so the barriers below match
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
        }
        const SegParams& P = a.seg[s];
        const int64_t quad = (tile - s_begin) * 32 + lane;
        const int64_t slot = P.base + 4 * quad;
        int c[4] = {-1, -1, -1, -1};
        T vo[4], vx[4], vy[4], vz[4], vyp[4];
        uint32_t vi[4] = {0u, 0u, 0u, 0u};
        if (have && quad < (a.seg_nmove[s] >> 2) && in_range(a.err, 4 * quad + 3, 0, P.cap)) {
            // the whole quad with 128-bit loads (the mover's access pattern)
            const int4 cc = __ldcs(reinterpret_cast<const int4*>(cell + slot));
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
            ld4(off + slot, vo);
            ld4(ux + slot, vx);
            ld4(uy + slot, vy);
            ld4(uz + slot, vz);
            const uint4 ii = __ldcs(reinterpret_cast<const uint4*>(id + slot));
            vi[0] = ii.x; vi[1] = ii.y; vi[2] = ii.z; vi[3] = ii.w;
            if (YP) ld4(yps + slot, vyp);
        }
        // cells of the quad (-1: empty slot); the chunk's span and segments
        int j[4];
        unsigned lmin = 0xFFFFFFFFu;
        int lmax = -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            j[k] = c[k] >= 0 ? (int)((uint32_t)c[k] & kCellMask) : -1;
            if (j[k] >= 0 && !in_range(a.err, j[k], 0, P.ncells)) {  // (checked build)
                j[k] = -1;
                c[k] = -1;
            }
            if (j[k] >= 0) {
                lmin = min(lmin, (unsigned)j[k]);
                lmax = max(lmax, j[k]);
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
        if (staged) {
            const SegParams& B = a.seg[bseg];
            // rank of each particle among the chunk's particles of its cell: equal cells
            // of a quad position grouped across the warp, one shared atomic a group
            int key[4], rank[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                key[k] = j[k] >= 0 ? j[k] - bmin : -1;
                const unsigned grp = __match_any_sync(FULL, key[k] >= 0 ? key[k] : kSortSpan + lane);
                const int leader = __ffs(grp) - 1;
                int base = 0;
                if (key[k] >= 0 && lane == leader) base = atomicAdd(cnt + key[k], __popc(grp));
                base = __shfl_sync(FULL, base, leader);
                rank[k] = base + __popc(grp & lt);
            }
            __syncthreads();
            // each cell's run: its offset in the chunk (scan of the counts) and its global
            // start (one reservation per cell on the cell's cursor)
            if (threadIdx.x < kSortSpan) {
                const int n = cnt[threadIdx.x];
                gb[threadIdx.x] = n > 0 ? atomicAdd(a.hist + B.node + bmin + threadIdx.x, (unsigned)n) : 0u;
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
            __syncthreads();
            // stage every particle at its place in the chunk's cell order
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (key[k] < 0) continue;
                const int p = pre[key[k]] + rank[k];
                if (!in_range(a.err, p, 0, C)) continue;  // (bounds-checked build only)
                s_off[p] = vo[k];
                s_ux[p] = vx[k];
                s_uy[p] = vy[k];
                s_uz[p] = vz[k];
                s_cell[p] = c[k];
                s_id[p] = vi[k];
                if (YP) s_yp[p] = vyp[k];
                const int64_t r = (int64_t)gb[key[k]] + rank[k];
                s_dst[p] = r < B.cap ? (uint32_t)r : 0xFFFFFFFFu;
            }
            // (read before the barrier: the next chunk clears the counts after it)
            const int ntot = pre[kSortSpan - 1] + cnt[kSortSpan - 1];
            __syncthreads();
            // write the runs: consecutive threads, consecutive slots of a cell's run
#pragma unroll 4
            for (int p = threadIdx.x; p < ntot; p += NT) {
                const uint32_t r = s_dst[p];
                if (r == 0xFFFFFFFFu) {  // a histogram that does not match the store: refused
                    set_error(a.err, kErrCapacity);
                    continue;
                }
                const int64_t g = B.base + (int64_t)r;
                __stcs(dcell + g, s_cell[p]);
                __stcs(doff + g, s_off[p]);
                __stcs(dux + g, s_ux[p]);
                __stcs(duy + g, s_uy[p]);
                __stcs(duz + g, s_uz[p]);
                __stcs(did + g, s_id[p]);
                if (YP) ypd[g] = s_yp[p];
            }
        } else {
            // per warp: group equal cells of each quad position across the warp; the
            // four reservations are independent, so they are all issued before the first
            // one is waited for
            unsigned grp[4], base[4];
            int key[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                key[k] = j[k] >= 0 ? j[k] : -1 - lane;
                grp[k] = __match_any_sync(FULL, key[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                base[k] = 0;
                if (j[k] >= 0 && lane == __ffs(grp[k]) - 1)
                    base[k] = atomicAdd(a.hist + P.node + key[k], (unsigned)__popc(grp[k]));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned b = __shfl_sync(FULL, base[k], __ffs(grp[k]) - 1);
                const int64_t r = (int64_t)b + __popc(grp[k] & lt);
                if (j[k] < 0) continue;
                if (r >= P.cap) {  // a histogram that does not match the store: refused
                    set_error(a.err, kErrCapacity);
                    continue;
                }
                const int64_t to = P.base + r;
                dcell[to] = c[k];
                doff[to] = vo[k];
                dux[to] = vx[k];
                duy[to] = vy[k];
                duz[to] = vz[k];
                did[to] = vi[k];
                if (YP) ypd[to] = vyp[k];
            }
        }
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

// The scatter with its shared memory (staging of a chunk), on one resident wave.
template <typename T, int NT, bool YP>
cudaError_t launch_scatter(const SortArgs& a, int sms, cudaStream_t st)
{
    const int sm = (int)SortSmem<T, NT, YP>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_scatter<T, NT, YP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    int nb = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter<T, NT, YP>, NT, sm);
    if (e != cudaSuccess) return e;
    k_scatter<T, NT, YP><<<std::max(nb, 1) * sms, NT, sm, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t run_sort(const SortArgs& a, int sms, cudaStream_t st)
{
    k_hist<NT><<<one_wave(k_hist<NT>, NT, sms), NT, 0, st>>>(a);
    const dim3 cg(a.nseg, a.cell_chunks);
    k_cell_partial<<<cg, kCellThreads, 0, st>>>(a);
    k_cell_scan<<<cg, kCellThreads, 0, st>>>(a);
    const bool yp = a.yp[a.src] != nullptr;
    const cudaError_t e =
        a.precision == PIC_FP64
            ? (yp ? launch_scatter<double, NT, true>(a, sms, st) : launch_scatter<double, NT, false>(a, sms, st))
            : (yp ? launch_scatter<float, NT, true>(a, sms, st) : launch_scatter<float, NT, false>(a, sms, st));
    if (e != cudaSuccess) return e;
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
