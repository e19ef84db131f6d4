// io.cu -- loading particles into the store, reading them back, diagnostics and the
// stand-alone Philox kernel.
#include <string>

#include "kernels.h"
#include "mover.cuh"

namespace bitpic {

namespace {

// Load: velocities physical -> cells per step (u = v dt/dx); invalid cells or
// offsets are latched as kErrInput.  Slots [n, cap) become empty.  T: the store's
// precision, H: the caller's (double, or float).
template <typename T, typename H>
__global__ void k_load(const LoadArgs l)
{
    const H* const in_off = static_cast<const H*>(l.off);
    const H* const in_vx = static_cast<const H*>(l.vx);
    const H* const in_vy = static_cast<const H*>(l.vy);
    const H* const in_vz = static_cast<const H*>(l.vz);
    T* off = static_cast<T*>(l.s_off);
    T* ux = static_cast<T*>(l.s_ux);
    T* uy = static_cast<T*>(l.s_uy);
    T* uz = static_cast<T*>(l.s_uz);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t idmax = 0;  // largest loaded id seen by this thread
    bool any = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < l.cap; k += stride) {
        const int64_t g = l.base + k;
        if (k < l.n) {
            const int c = l.cell[k];
            const double f = (double)in_off[k];
            const bool ok = c >= 0 && c < l.ncells && f >= 0.0 && f < 1.0;
            if (!ok) set_error(l.err, kErrInput);
            T ft = (T)f;
            int cc = c;
            if (ft >= T(1)) {  // an offset just below 1 that rounds up in FP32
                ft = T(0);
                cc = c + 1;
                if (cc >= l.ncells) {
                    cc = l.ncells - 1;
                    ft = (T)0.99999994f;
                }
            }
            // cell word: index | collision clock; the caller's clock counts the own
            // steps to skip (bits 0-6) before the event step, the word names that step
            const uint32_t clk = l.state ? (uint32_t)l.state[k] : 0u;
            const uint32_t cb = clock_bits(l.own0 + (int64_t)(clk & kClockDue), (clk & kClockPending) != 0u);
            l.s_cell[g] = ok ? (int)((uint32_t)cc | cb) : -1;
            off[g] = ft;
            const double vx = (double)in_vx[k], vy = (double)in_vy[k], vz = (double)in_vz[k];
            ux[g] = l.vscale == 1.0 ? (T)vx : (T)(vx * l.vscale);
            uy[g] = l.vscale == 1.0 ? (T)vy : (T)(vy * l.vscale);
            uz[g] = l.vscale == 1.0 ? (T)vz : (T)(vz * l.vscale);
            l.s_id[g] = l.id ? l.id[k] : l.id0 + (uint32_t)k;
            if (l.s_yp) static_cast<T*>(l.s_yp)[g] = T(0);
        } else {
            l.s_cell[g] = -1;
        }
        if (l.id && k < l.n) {
            idmax = max(idmax, l.id[k]);
            any = true;
        }
    }
    // the next automatic id follows the largest loaded one: one atomic per warp
    if (l.id) {
        const unsigned m = __reduce_max_sync(0xffffffffu, idmax);
        if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0)
            atomicMax(l.next_id, (unsigned long long)m + 1ull);
    }
}

// The step counter moves from `from` to `to` (a restored run): every clock keeps its
// distance from the species' next moving step, so its due step moves with it.
__global__ void k_rebase_clocks(const SegParams* seg, int nseg, int32_t* cell, int64_t from,
                                int64_t to)
{
    for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
        const SegParams& P = seg[s];
        const uint32_t delta = (uint32_t)(clock_origin(P, to) - clock_origin(P, from)) & kClockDue;
        if (delta == 0u) continue;
        for (int64_t k = threadIdx.x; k < P.cap; k += blockDim.x) {
            const int w = cell[P.base + k];
            if (w < 0) continue;
            const uint32_t u = (uint32_t)w;
            const uint32_t due = ((u >> kClockShift) + delta) & kClockDue;
            cell[P.base + k] = (int)((u & ~(kClockDue << kClockShift)) | (due << kClockShift));
        }
    }
}

__global__ void k_get_count(const int32_t* cell, int64_t base, int64_t nslots,
                            unsigned long long* block_count)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = k < nslots && cell[base + k] >= 0;
    const unsigned b = __ballot_sync(0xffffffffu, live);
    if ((threadIdx.x & 31) == 0) atomicAdd(&cnt, __popc(b));
    __syncthreads();
    if (threadIdx.x == 0) block_count[blockIdx.x] = (unsigned long long)cnt;
}

// exclusive scan of nb block counts (single block), total in block_count[nb]
__global__ void __launch_bounds__(1024) k_get_scan(unsigned long long* bc, int64_t nb)
{
    __shared__ unsigned long long sh[33];
    const int64_t C = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = min(nb, (int64_t)threadIdx.x * C), i1 = min(nb, i0 + C);
    unsigned long long local = 0;
    for (int64_t i = i0; i < i1; ++i) local += bc[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = local;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = sh[lane];
        unsigned long long wi = w;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += t;
        }
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    unsigned long long run = sh[warp] + inc - local;
    for (int64_t i = i0; i < i1; ++i) {
        const unsigned long long v = bc[i];
        bc[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) bc[nb] = sh[32];
}

template <typename T, typename H>
__global__ void k_get_write(const GetArgs g)
{
    const int64_t blk = g.block0 + blockIdx.x;  // this block's 1024 slots
    const int64_t k = blk * (int64_t)blockDim.x + threadIdx.x;
    const bool live = k < g.nslots && g.s_cell[g.base + k] >= 0;
    const unsigned b = __ballot_sync(0xffffffffu, live);
    __shared__ int woff[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) woff[warp] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int t = woff[w];
            woff[w] = r;
            r += t;
        }
    }
    __syncthreads();
    if (!live) return;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int64_t o = (int64_t)g.block_count[blk] + woff[warp] + __popc(b & lt);
    if (o >= g.capacity) return;
    const int64_t s = g.base + k;
    const uint32_t word = (uint32_t)g.s_cell[s];
    if (g.cell) g.cell[o] = (int)(word & kCellMask);
    if (g.state) {  // the event step's distance from the next own step (mod 128)
        const uint32_t clk = word >> kClockShift;
        const uint32_t skip = (uint32_t)((int64_t)(clk & kClockDue) - g.own0) & kClockDue;
        g.state[o] = (uint8_t)(skip | (clk & kClockPending));
    }
    // in double, then rounded once to the caller's type
    if (g.off) {
        H fo = (H)(double)static_cast<const T*>(g.s_off)[s];
        // a double offset that rounds up to 1 in float stays in its cell, just below 1
        if (fo >= H(1)) fo = (H)0.99999994f;
        static_cast<H*>(g.off)[o] = fo;
    }
    if (g.vx) static_cast<H*>(g.vx)[o] = (H)((double)static_cast<const T*>(g.s_ux)[s] * g.vscale_inv);
    if (g.vy) static_cast<H*>(g.vy)[o] = (H)((double)static_cast<const T*>(g.s_uy)[s] * g.vscale_inv);
    if (g.vz) static_cast<H*>(g.vz)[o] = (H)((double)static_cast<const T*>(g.s_uz)[s] * g.vscale_inv);
    if (g.id) g.id[o] = g.s_id[s];
    if (g.yp) g.yp[o] = g.s_yp ? (double)static_cast<const T*>(g.s_yp)[s] : 0.0;
}

template <typename T>
__global__ void k_set_yp(T* yp, int64_t base, const double* in, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
        yp[base + k] = (T)in[k];
}

template <typename T>
__global__ void k_kinetic(const SegParams* seg, int s0, const int32_t* cell, const T* ux,
                          const T* uy, const T* uz, double* out)
{
    const int s = s0 + blockIdx.y;
    const SegParams& P = seg[s];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.cap; k += stride) {
        const int64_t g = P.base + k;
        if (cell[g] < 0) continue;
        if (sizeof(T) == 4) {
            // |u|^2 of a float state in float (two fused multiply-adds), summed in double:
            // one FP64 operation per particle, the GB300's scarce pipe
            const float a = (float)ux[g], b = (float)uy[g], c = (float)uz[g];
            acc += (double)__fmaf_rn(a, a, __fmaf_rn(b, b, c * c));
        } else {
            const double a = ux[g], b = uy[g], c = uz[g];
            acc += a * a + b * b + c * c;
        }
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(out + blockIdx.y, P.kefac * t);
    }
}

__global__ void k_philox(uint64_t key, const uint4* ctr, uint4* out, int64_t n)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) out[k] = philox4x32_10(ctr[k], (uint32_t)key, (uint32_t)(key >> 32));
}

__global__ void k_fill_i32(int32_t* p, int64_t lo, int64_t hi, int32_t v)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < hi; k += stride) p[k] = v;
}

int grid_for(int64_t n, int nt, int cap = 152 * 32)
{
    const int64_t g = (n + nt - 1) / nt;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_rebase_clocks(const SegParams* seg, int nseg, int32_t* cell, int64_t from,
                                 int64_t to, cudaStream_t st)
{
    k_rebase_clocks<<<nseg < 1024 ? nseg : 1024, 256, 0, st>>>(seg, nseg, cell, from, to);
    return cudaGetLastError();
}

cudaError_t launch_load(const LoadArgs& l, cudaStream_t st)
{
    const int g = grid_for(l.cap, 256);
    if (l.precision == PIC_FP64) {
        if (l.host_f32) k_load<double, float><<<g, 256, 0, st>>>(l);
        else k_load<double, double><<<g, 256, 0, st>>>(l);
    } else {
        if (l.host_f32) k_load<float, float><<<g, 256, 0, st>>>(l);
        else k_load<float, double><<<g, 256, 0, st>>>(l);
    }
    return cudaGetLastError();
}

cudaError_t launch_get_scan(const GetArgs& g, cudaStream_t st)
{
    const int64_t nb = (g.nslots + 1023) / 1024;
    if (nb == 0) return cudaSuccess;
    k_get_count<<<(unsigned)nb, 1024, 0, st>>>(g.s_cell, g.base, g.nslots, g.block_count);
    k_get_scan<<<1, 1024, 0, st>>>(g.block_count, nb);
    return cudaGetLastError();
}

cudaError_t launch_get_write(GetArgs g, int64_t block0, int64_t nblocks, cudaStream_t st)
{
    if (nblocks <= 0) return cudaSuccess;
    g.block0 = block0;
    const unsigned nb = (unsigned)nblocks;
    if (g.precision == PIC_FP64) {
        if (g.host_f32) k_get_write<double, float><<<nb, 1024, 0, st>>>(g);
        else k_get_write<double, double><<<nb, 1024, 0, st>>>(g);
    } else {
        if (g.host_f32) k_get_write<float, float><<<nb, 1024, 0, st>>>(g);
        else k_get_write<float, double><<<nb, 1024, 0, st>>>(g);
    }
    return cudaGetLastError();
}

cudaError_t launch_set_yp(void* s_yp, int64_t base, const double* in, int64_t n, int precision,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (precision == PIC_FP64)
        k_set_yp<double><<<grid_for(n, 256), 256, 0, st>>>(static_cast<double*>(s_yp), base, in, n);
    else
        k_set_yp<float><<<grid_for(n, 256), 256, 0, st>>>(static_cast<float*>(s_yp), base, in, n);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const SegParams* seg, int s0, int ns, int64_t max_slots,
                           const int32_t* cell, const void* ux, const void* uy,
                           const void* uz, int precision, double* out, cudaStream_t st)
{
    dim3 grid((unsigned)grid_for(max_slots, 256, 1024), (unsigned)ns);
    if (precision == PIC_FP64)
        k_kinetic<double><<<grid, 256, 0, st>>>(seg, s0, cell, (const double*)ux,
                                                 (const double*)uy, (const double*)uz, out);
    else
        k_kinetic<float><<<grid, 256, 0, st>>>(seg, s0, cell, (const float*)ux,
                                                (const float*)uy, (const float*)uz, out);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t key, const uint32_t* ctr, uint32_t* out, int64_t n,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + 255) / 256);
    k_philox<<<g, 256, 0, st>>>(key, reinterpret_cast<const uint4*>(ctr),
                                reinterpret_cast<uint4*>(out), n);
    return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t* p, int64_t lo, int64_t hi, int32_t v, cudaStream_t st)
{
    if (hi <= lo) return cudaSuccess;
    k_fill_i32<<<grid_for(hi - lo, 256), 256, 0, st>>>(p, lo, hi, v);
    return cudaGetLastError();
}

// The bounds-checked build's self-test: one thread asks for entry kProbeN of a
// kProbeN-entry range of g_probe_buf through in_range, which must refuse it (the array
// has 2 kProbeN entries, so even an accepted index would stay inside it) and latch the
// bit in g_probe_err.
constexpr int kProbeN = 4;
__device__ int g_probe_buf[2 * kProbeN];
__device__ unsigned g_probe_err;

__global__ void k_bounds_probe()
{
    if (in_range(&g_probe_err, kProbeN, 0, kProbeN)) g_probe_buf[kProbeN] = 1;
}

void set_global_error(const std::string& msg);

}  // namespace bitpic

extern "C" PIC_API int pic_bounds_probe(void* stream)
{
    using namespace bitpic;
    set_global_error("");
    if (!kChecked) {
        set_global_error("pic_bounds_probe: not the bounds-checked build");
        return PIC_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned zero = 0;
    unsigned got = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_probe_err, &zero, sizeof(zero), 0,
                                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_bounds_probe<<<1, 1, 0, st>>>();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyFromSymbolAsync(&got, g_probe_err, sizeof(got), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_global_error(std::string("pic_bounds_probe: ") + cudaGetErrorString(e));
        return PIC_ECUDA;
    }
    if (!(got & kErrBounds)) {
        set_global_error("pic_bounds_probe: the check did not refuse the index");
        return PIC_ECUDA;
    }
    return PIC_OK;
}
