// field.cu -- field phase (Poisson solve and E = -grad phi, Section 2 "Field Solver")
// plus the per-step bookkeeping kernels (tile list, ionization ids).
//
// Field solve.  The deposit gives, per instance and node j, the integer
// Z_j = sum_s z_s D_s[j], where D_s is species s's fixed-point deposit (unit S per
// particle) and z_s = q_s w_s / delta is an exact small integer.  The grounded
// Dirichlet problem
//     -phi[j-1] + 2 phi[j] - phi[j+1] = kappa Z_j  (1 <= j <= N-1),  phi[0] = phi[N] = 0,
// kappa = delta dx / (S eps0), has the exact solution phi[j+1] - phi[j] = kappa (U/N - R_j)
// with R_j = sum_{1<=k<=j} Z_k (R_0 = 0) and U = sum_{m=0}^{N-1} R_m = sum_k (N-k) Z_k.
// Hence, with lambda = delta / (2 N S eps0) and every numerator an exact 128-bit integer:
//     E_j = lambda (N (R_{j-1} + R_j) - 2U)             inside (centred difference),
//     E_0 = lambda (-2U - 2N Z_0),  E_N = lambda (2N R_{N-1} - 2U + 2N Z_N)
// (Gauss's law over the half cell at each wall).  This is the tridiagonal solve the
// paper names, carried out as one prefix sum and one weighted sum, so it is
// independent of launch geometry and rounds only once, at the conversion to FP64.
#include <algorithm>

#include "kernels.h"
#include "mover.cuh"

namespace bitpic {

namespace {

constexpr int kFieldThreads = 1024;

__device__ __forceinline__ i128 warp_incl_scan(i128 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const i128 t = shfl_up_i128(v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ i128 warp_sum(i128 v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const uint64_t lo = (uint64_t)v, hi = (uint64_t)((unsigned __int128)v >> 64);
        const uint64_t l2 = __shfl_xor_sync(0xffffffffu, lo, d);
        const uint64_t h2 = __shfl_xor_sync(0xffffffffu, hi, d);
        v += (i128)(((unsigned __int128)h2 << 64) | l2);
    }
    return v;
}

// Block-wide exclusive scan of one i128 per thread; returns the exclusive prefix and
// the block total.  All threads of the block must call it.
__device__ i128 block_excl_scan(i128 v, i128* total, i128* sh /* >= 33 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const i128 inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        i128 w = lane < nw ? sh[lane] : (i128)0;
        const i128 wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;  // exclusive warp offsets
        if (lane == nw - 1) sh[32] = wi;
    }
    __syncthreads();
    const i128 out = sh[warp] + inc - v;
    *total = sh[32];
    __syncthreads();
    return out;
}

__device__ i128 block_sum(i128 v, i128* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    i128 t = 0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : (i128)0;
        t = warp_sum(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    t = sh[32];
    __syncthreads();
    return t;
}

// Interior charge Z'_j of node j of instance I, from the deposit array `dep`
// (Z'_0 = Z'_N = 0: the wall nodes do not enter the Dirichlet system).
__device__ __forceinline__ i128 node_charge(const FieldArgs& f, const InstParams& I, int j,
                                           const unsigned long long* dep)
{
    i128 z = 0;
    for (int k = 0; k < I.nseg; ++k) {
        const SegParams& P = f.seg[I.seg0 + k];
        z += (i128)I.z[k] * (i128)(long long)dep[P.node + j];
    }
    return z;
}

// Density smoother (Section 2's "Density Smoother" phase), in the integer charges: the
// 1-2-1 filter of the interior node densities, wall nodes (half cells, density 2Z/dx)
// kept, times 4 so that it stays exact:
//     Z''_j = Z_{j-1} w_{j-1} + 2 Z_j + Z_{j+1} w_{j+1},  w = 2 at a wall node, else 1,
//     Z''_0 = 4 Z_0, Z''_N = 4 Z_N;
// lambda carries the 1/4.  Node charges of [0, N] only (dep is not being written).
__device__ __forceinline__ i128 smoothed_charge(const FieldArgs& f, const InstParams& I, int j,
                                                const unsigned long long* dep)
{
    const int N = I.ncells;
    const i128 zc = node_charge(f, I, j, dep);
    if (j == 0 || j == N) return 4 * zc;
    const i128 zl = node_charge(f, I, j - 1, dep), zr = node_charge(f, I, j + 1, dep);
    return (j - 1 == 0 ? 2 * zl : zl) + 2 * zc + (j + 1 == N ? 2 * zr : zr);
}

// The solve runs over chunks of kChunk nodes (one block each):
//   k_field_partial  per chunk: S_c = sum of Z' and W_c = sum of (N-j) Z' over the chunk,
//                    and the charge of its first node;
//   k_field_emit     per chunk: the chunk's prefix (sum of S over the instance's earlier
//                    chunks) and U = sum of W_c, an in-block scan of Z' + that prefix =
//                    R_j, then E_j and the accelerations as node pairs (A_j, A_{j+1} - A_j),
//                    A_{j+1} of the chunk's last node from the next chunk's first charge;
//                    also hands the deposit over for the next step.
constexpr int kChunkThreads = 256;
constexpr int kChunkPer = 1;  // nodes per thread
static_assert(kChunk == kChunkThreads * kChunkPer, "chunk layout");

__global__ void __launch_bounds__(kChunkThreads) k_field_partial(const FieldArgs f)
{
    __shared__ i128 sh[33];
    const int c = blockIdx.x;
    const int b = f.chunk_inst[c];
    const InstParams& I = f.inst[b];
    if (I.field != PIC_FIELD_POISSON) return;
    const int N = I.ncells;
    const int a = (c - I.chunk0) * kChunk;
    const int j0 = a + threadIdx.x * kChunkPer;
    i128 sum = 0, wsum = 0;
#pragma unroll
    for (int t = 0; t < kChunkPer; ++t) {
        const int j = j0 + t;
        if (j < 0 || j > N) continue;
        i128 z;
        if (I.smooth) {
            // the filtered charges of all nodes, walls included, for the emit phase
            z = smoothed_charge(f, I, j, f.dep);
            f.zs[I.inode + j] = z;
        } else {
            z = node_charge(f, I, j, f.dep);
        }
        if (j == 0 || j == N) continue;
        sum += z;
        wsum += (i128)(N - j) * z;
    }
    const i128 S = block_sum(sum, sh);
    const i128 Wt = block_sum(wsum, sh);
    if (threadIdx.x == 0) {
        f.part_sum[c] = S;
        f.part_w[c] = Wt;
        // the charge of the chunk's first node (the walls' too), for the emit of the
        // chunk before it
        f.zfirst[c] = j0 <= N ? (I.smooth ? f.zs[I.inode + j0] : node_charge(f, I, j0, f.dep))
                              : (i128)0;
    }
}

template <typename T>
__global__ void __launch_bounds__(kChunkThreads) k_field_emit(const FieldArgs f, int advance)
{
    __shared__ i128 sh[33];
    const int c = blockIdx.x;
    // the steps completed (the kernels of the next step read it once k_tiles has set it)
    if (advance && c == 0 && threadIdx.x == 0) f.step[1] = f.step[0] + 1;
    const int b = f.chunk_inst[c];
    const InstParams& I = f.inst[b];
    const int N = I.ncells;
    const int a = (c - I.chunk0) * kChunk;
    const int j0 = a + threadIdx.x * kChunkPer;
    const bool poisson = I.field == PIC_FIELD_POISSON;
    i128 z[kChunkPer];
    i128 run = 0;
#pragma unroll
    for (int t = 0; t < kChunkPer; ++t) {
        const int j = j0 + t;
        z[t] = 0;
        if (j > N) continue;
        // the deposit hand-over: keep the last complete deposit, clear for the next step
        // (a kept deposit, deposit_kept(), is updated in place instead)
        for (int k = 0; k < I.nseg; ++k) {
            const SegParams& P = f.seg[I.seg0 + k];
            const unsigned long long d = f.dep[P.node + j];
            f.dep_last[P.node + j] = d;
            if (!deposit_kept(P)) f.dep[P.node + j] = 0ull;
            z[t] += (i128)I.z[k] * (i128)(long long)d;
        }
        if (I.smooth && poisson) z[t] = f.zs[I.inode + j];
        if (j > 0 && j < N) run += z[t];
    }
    if (!poisson) return;  // uniform per block: one instance per chunk
    // the chunk's prefix of the interior charge and U, from the chunk partials
    i128 ps = 0, pw = 0;
    for (int k = threadIdx.x; k < I.nchunk; k += blockDim.x) {
        if (I.chunk0 + k < c) ps += f.part_sum[I.chunk0 + k];
        pw += f.part_w[I.chunk0 + k];
    }
    const i128 coff = block_sum(ps, sh);
    const i128 U = block_sum(pw, sh);
    i128 tot;
    const i128 off = coff + block_excl_scan(run, &tot, sh);
    const i128 NN = (i128)N;
    // G of node j from R_{j-1}, Z_j: E_j = lambda G
    auto numer = [&](int j, i128 Rprev, i128 zj) {
        if (j == 0) return -2 * U - 2 * NN * zj;
        if (j == N) return 2 * NN * Rprev - 2 * U + 2 * NN * zj;
        return NN * (2 * Rprev + zj) - 2 * U;
    };
    __shared__ double sE[kChunkThreads + 1];
    i128 Rprev = off;  // R_{j0-1}
    const int j = j0;  // one node per thread
    double E = 0.0;
    if (j <= N) {
        E = I.lambda * i128_to_double(numer(j, Rprev, z[0]));
        f.E[I.inode + j] = E;
        const i128 R = Rprev + ((j > 0 && j < N) ? z[0] : (i128)0);
        sE[threadIdx.x] = E;
        // the next chunk's first node (same instance), with the same integers as there
        if (threadIdx.x == kChunkThreads - 1 && j < N)
            sE[kChunkThreads] = I.lambda * i128_to_double(numer(j + 1, R, f.zfirst[c + 1]));
    }
    __syncthreads();
    if (j > N) return;
    T* acc = static_cast<T*>(f.accel);
    const double En = j < N ? sE[threadIdx.x + 1] : 0.0;
    for (int k = 0; k < I.nseg; ++k) {
        const SegParams& P = f.seg[I.seg0 + k];
        // the pair (A_j, A_{j+1} - A_j), the difference of the two rounded accelerations
        const T A = (T)(P.accel * E);
        acc[2 * (P.node + j)] = A;
        acc[2 * (P.node + j) + 1] = j < N ? (T)(P.accel * En) - A : T(0);
    }
}

// Potential for the diagnostics (one block, on demand), from the last complete
// deposit: R_j and U as in the solve, then phi_j = 2 dx lambda (j U - N U_j),
// U_j = sum_{m<j} R_m.
__global__ void __launch_bounds__(kFieldThreads) k_potential(const FieldArgs f, int b,
                                                             double dx, double* phi)
{
    __shared__ i128 sh[33];
    const InstParams I = f.inst[b];
    const int N = I.ncells;
    const int nn = N + 1;
    const int C = (nn + blockDim.x - 1) / blockDim.x;
    const int j0 = min(nn, (int)threadIdx.x * C), j1 = min(nn, j0 + C);
    // pass 1: R at the start of this thread's run, U
    i128 sum = 0, wsum = 0;
    auto charge = [&](int j) {
        return I.smooth ? smoothed_charge(f, I, j, f.dep_last) : node_charge(f, I, j, f.dep_last);
    };
    for (int j = j0; j < j1; ++j) {
        if (j == 0 || j == N) continue;
        const i128 z = charge(j);
        sum += z;
        wsum += (i128)(N - j) * z;
    }
    i128 tot;
    const i128 R0 = block_excl_scan(sum, &tot, sh);
    const i128 U = block_sum(wsum, sh);
    // pass 2: sum of R over this thread's run, then the exclusive prefix U_{j0}
    i128 R = R0, rsum = 0;
    for (int j = j0; j < j1; ++j) {
        if (j != 0 && j != N) R += charge(j);
        rsum += R;
    }
    i128 run = block_excl_scan(rsum, &tot, sh);
    R = R0;
    for (int j = j0; j < j1; ++j) {
        const i128 Phi = (i128)j * U - (i128)N * run;
        phi[j] = (2.0 * dx * I.lambda) * i128_to_double(Phi);
        if (j != 0 && j != N) R += charge(j);
        run += R;
    }
}

__global__ void __launch_bounds__(1024) k_tiles(const SegParams* seg, unsigned long long* seg_n,
                                                int64_t* seg_nmove, int64_t* tile_start, int nseg,
                                                int tile_quads, unsigned long long* rare_count,
                                                int64_t* step)
{
    if (threadIdx.x == 0) {
        rare_count[0] = 0ull;
        rare_count[1] = 0ull;
        step[0] = step[1];  // the step the kernels of this step read
    }
    __shared__ i128 sh[33];
    const int C = (nseg + blockDim.x - 1) / blockDim.x;
    const int s0 = min(nseg, (int)threadIdx.x * C), s1 = min(nseg, s0 + C);
    int64_t local = 0;
    for (int s = s0; s < s1; ++s) {
        // an overflowing creation (already latched as an error) may have pushed the
        // count past the capacity: never walk beyond the segment.  Only the count to
        // move is rounded up to a whole quad (the slots past the count are empty, and
        // creations append after the mover), so appends waste no slots.
        const unsigned long long cap = (unsigned long long)seg[s].cap;
        const unsigned long long nn = min(seg_n[s], cap);
        const unsigned long long n4 = min((nn + 3ull) & ~3ull, cap);
        seg_n[s] = nn;
        seg_nmove[s] = (int64_t)n4;
        const int64_t quads = (int64_t)(n4 >> 2);
        local += (quads + tile_quads - 1) / tile_quads;
    }
    i128 tot;
    int64_t run = (int64_t)block_excl_scan((i128)local, &tot, sh);
    for (int s = s0; s < s1; ++s) {
        tile_start[s] = run;
        const int64_t quads = seg_nmove[s] >> 2;
        run += (quads + tile_quads - 1) / tile_quads;
    }
    if (threadIdx.x == 0) tile_start[nseg] = (int64_t)tot;
}

// Children of this step's ionization events are numbered after the largest id so
// far: electron 2r, ion 2r+1, r = rank of the parent id among this step's events (with
// a neutral particle target only the electron is new: id r).  One block per instance
// sorts the parent ids (a stable least-significant-digit radix sort, 8 bits a pass,
// as many passes as the largest id so far needs; the ids of one step are distinct;
// in shared memory when they fit) and ranks every event by a binary search in the
// sorted ids, then advances the instance's next id: O(n) work per pass for n events.
constexpr int kBirthThreads = 1024;
constexpr int kBirthSmemKeys = 3072;

__global__ void __launch_bounds__(kBirthThreads) k_births(const InstParams* inst, Event* events,
                                                          unsigned long long* ev_count,
                                                          unsigned long long* next_id, uint32_t* id,
                                                          uint32_t* keys_a, uint32_t* keys_b,
                                                          unsigned* err)
{
    constexpr int NW = kBirthThreads / 32;
    __shared__ unsigned hist[256];     // digit counts of the pass
    __shared__ unsigned run[256];      // next slot of each digit in the pass's output
    __shared__ unsigned tot[256];      // digit counts of the tile
    __shared__ unsigned short wcnt[NW][256];  // digit counts of each warp in the tile
    __shared__ uint32_t skeys[2][kBirthSmemKeys];   // the keys of a small step
    const int b = blockIdx.x;
    const InstParams& I = inst[b];
    const unsigned long long cnt = ev_count[b];
    if (cnt == 0) return;
    const int64_t n = (int64_t)min(cnt, (unsigned long long)I.ev_cap);
    const Event* ev = events + I.ev_base;
    const unsigned long long base = next_id[b];
    const unsigned long long per = I.tseg >= 0 ? 1ull : 2ull;
    if (base + per * (unsigned long long)n > 0xFFFFFFFFull) {
        if (threadIdx.x == 0) set_error(err, kErrCapacity);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    // a step with few events sorts in shared memory, a larger one in its buffers
    const bool small = n <= kBirthSmemKeys;
    uint32_t* const buf0 = small ? skeys[0] : keys_a + I.ev_base;
    uint32_t* const buf1 = small ? skeys[1] : keys_b + I.ev_base;
    // every parent id is below the next id: passes for its significant bytes
    int passes = 0;
    for (unsigned long long m = base > 0 ? base - 1 : 0; m != 0; m >>= 8) ++passes;
    if (passes == 0) passes = 1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const uint32_t* src = (pass & 1) ? buf0 : buf1;
        uint32_t* dst = (pass & 1) ? buf1 : buf0;
        auto key = [&](int64_t i) -> uint32_t { return pass == 0 ? ev[i].parent : src[i]; };
        for (int d = threadIdx.x; d < 256; d += kBirthThreads) hist[d] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += kBirthThreads)
            atomicAdd(&hist[(key(i) >> shift) & 255u], 1u);
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the 256 counts, 8 a lane
            unsigned v[8], sum = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = hist[lane * 8 + k];
                sum += v[k];
            }
            unsigned inc = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, inc, d);
                if (lane >= d) inc += t;
            }
            unsigned r = inc - sum;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                run[lane * 8 + k] = r;
                r += v[k];
            }
        }
        // tiles of kBirthThreads keys in index order: a key's place is its digit's next
        // slot plus the keys of the same digit before it in the tile (earlier warps,
        // then lower lanes), so equal digits keep their order
        for (int64_t t0 = 0; t0 < n; t0 += kBirthThreads) {
            for (int e = threadIdx.x; e < NW * 256; e += kBirthThreads) (&wcnt[0][0])[e] = 0;
            __syncthreads();
            const int64_t i = t0 + threadIdx.x;
            const bool have = i < n;
            const uint32_t k = have ? key(i) : 0u;
            const int d = have ? (int)((k >> shift) & 255u) : 256 + lane;
            const unsigned grp = __match_any_sync(FULL, d);
            if (have && lane == __ffs(grp) - 1) wcnt[warp][d] = (unsigned short)__popc(grp);
            __syncthreads();
            if (threadIdx.x < 256) {  // per digit: the warps' counts become their offsets
                unsigned r = 0;
                for (int w = 0; w < NW; ++w) {
                    const unsigned c = wcnt[w][threadIdx.x];
                    wcnt[w][threadIdx.x] = (unsigned short)r;
                    r += c;
                }
                tot[threadIdx.x] = r;
            }
            __syncthreads();
            if (have) {
                const unsigned at = run[d] + wcnt[warp][d] + __popc(grp & lt);
                if (at < (unsigned)n) dst[at] = k;
            }
            __syncthreads();
            if (threadIdx.x < 256) run[threadIdx.x] += tot[threadIdx.x];
        }
        __syncthreads();
    }
    // rank of every event: its parent's place among the sorted ids
    const uint32_t* sorted = ((passes - 1) & 1) ? buf1 : buf0;
    for (int64_t i = threadIdx.x; i < n; i += kBirthThreads) {
        const uint32_t p = ev[i].parent;
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (sorted[mid] < p) lo = mid + 1; else hi = mid;
        }
        // an event whose creation overflowed (already latched) has no slots
        if (ev[i].slot_e >= 0) id[ev[i].slot_e] = (uint32_t)(base + per * (unsigned long long)lo);
        if (per == 2ull && ev[i].slot_i >= 0)
            id[ev[i].slot_i] = (uint32_t)(base + 2ull * (unsigned long long)lo + 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        next_id[b] = base + per * (unsigned long long)n;
        ev_count[b] = 0ull;
    }
}

}  // namespace

cudaError_t launch_field(const FieldArgs& f, bool advance_step, cudaStream_t st)
{
    if (f.any_poisson) k_field_partial<<<f.nchunks, kChunkThreads, 0, st>>>(f);
    if (f.precision == PIC_FP64)
        k_field_emit<double><<<f.nchunks, kChunkThreads, 0, st>>>(f, advance_step ? 1 : 0);
    else
        k_field_emit<float><<<f.nchunks, kChunkThreads, 0, st>>>(f, advance_step ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_potential(const FieldArgs& f, int inst, double dx, double* phi,
                             cudaStream_t st)
{
    k_potential<<<1, kFieldThreads, 0, st>>>(f, inst, dx, phi);
    return cudaGetLastError();
}

cudaError_t launch_tiles(const SegParams* seg, unsigned long long* seg_n, int64_t* seg_nmove,
                         int64_t* tile_start, int nseg, int tile_quads,
                         unsigned long long* rare_count, int64_t* step, cudaStream_t st)
{
    k_tiles<<<1, 1024, 0, st>>>(seg, seg_n, seg_nmove, tile_start, nseg, tile_quads, rare_count,
                                step);
    return cudaGetLastError();
}

cudaError_t launch_births(const InstParams* inst, int ninst, Event* events,
                          unsigned long long* ev_count, unsigned long long* next_id,
                          uint32_t* id, uint32_t* keys_a, uint32_t* keys_b, unsigned* err,
                          cudaStream_t st)
{
    k_births<<<ninst, kBirthThreads, 0, st>>>(inst, events, ev_count, next_id, id, keys_a, keys_b, err);
    return cudaGetLastError();
}

}  // namespace bitpic
