// noalloc.cu -- pic_field_solve_noalloc: the integer Poisson solve and E = -grad phi
// of one instance, computed without allocating any memory.
//
// Some callers cannot allocate device memory: code that runs while a CUDA graph is
// being captured, latency-critical loops in which an allocation could block or
// fragment the heap, and host frameworks that own every byte of device memory
// through their own pools.  This entry point serves them.  The caller passes the
// fixed-point charge deposits and the output array; the only scratch the solve
// needs (one 128-bit prefix sum per node and one 128-bit total) lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.  The math is the same as the handle's field phase (without
// its optional density smoother: the deposits are used as given):
//   Z_j = sum_s z_s D_s[j],  R_j = sum_{1<=k<=j, k<N} Z_k,  U = sum_{1<=k<N} (N-k) Z_k,
//   E_j = lambda (N (R_{j-1} + R_j) - 2U)      (0 < j < N),
//   E_0 = lambda (-2U - 2N Z_0),  E_N = lambda (2N R_{N-1} - 2U + 2N Z_N),
//   lambda = delta / (2 N S eps0).
#include <mutex>
#include <string>

#include "common.cuh"

namespace bitpic {
namespace {

constexpr int kNoAllocMaxCells = 65536;
constexpr int kNoAllocMaxNodes = kNoAllocMaxCells + 1;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: R_j for j = 0..N, then U.
static __device__ __align__(256) i128 g_scratch[kNoAllocMaxNodes + 1];

// Device address of g_scratch per device, from the last lookup made with that device
// current and no capture in progress on the call's stream.
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

struct NoAllocArgs {
    const long long* charge;  // nspecies x (N+1) deposits, species-major
    int ncells;
    int nspecies;
    int z[kMaxSpecies];
    double lambda;
    i128* scratch;            // R[0..N], U at [N+1]
    double* E;
};

__device__ __forceinline__ i128 incl_scan_warp(i128 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const i128 t = shfl_up_i128(v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ i128 sum_warp(i128 v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += shfl_i128(v, (threadIdx.x & 31) ^ d);
    return v;
}

__device__ __forceinline__ i128 charge_at(const NoAllocArgs& a, int j)
{
    i128 z = 0;
    for (int k = 0; k < a.nspecies; ++k)
        z += (i128)a.z[k] * (i128)a.charge[(int64_t)k * (a.ncells + 1) + j];
    return z;
}

// One block of 1024 threads: R (inclusive prefix of the interior charge) and U.  Each
// thread owns C consecutive nodes; their interior charges Z_j are formed once, kept in
// the scratch slots R_j until the prefix overwrites them.
__global__ void __launch_bounds__(1024) k_scan_noalloc(const NoAllocArgs a)
{
    __shared__ i128 sh[33];
    const int N = a.ncells, nn = N + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = (nn + blockDim.x - 1) / blockDim.x;
    const int j0 = min(nn, (int)threadIdx.x * C), j1 = min(nn, j0 + C);
    i128 sum = 0, wsum = 0;
    for (int j = j0; j < j1; ++j) {
        const i128 z = (j == 0 || j == N) ? (i128)0 : charge_at(a, j);
        a.scratch[j] = z;
        sum += z;
        wsum += (i128)(N - j) * z;
    }
    // block exclusive scan of `sum`
    const i128 inc = incl_scan_warp(sum);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const i128 w = sh[lane];
        const i128 wi = incl_scan_warp(w);
        sh[lane] = wi - w;
    }
    __syncthreads();
    i128 run = sh[warp] + inc - sum;
    __syncthreads();
    // block sum of `wsum`
    const i128 ws = sum_warp(wsum);
    if (lane == 0) sh[warp] = ws;
    __syncthreads();
    if (warp == 0) {
        const i128 t = sum_warp(sh[lane]);
        if (lane == 0) a.scratch[N + 1] = t;
    }
    for (int j = j0; j < j1; ++j) {
        run += a.scratch[j];
        a.scratch[j] = run;
    }
}

__global__ void k_emit_noalloc(const NoAllocArgs a)
{
    const int N = a.ncells;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > N) return;
    const i128 U = a.scratch[N + 1];
    const i128 NN = (i128)N;
    i128 G;
    if (j == 0)
        G = -2 * U - 2 * NN * charge_at(a, 0);
    else if (j == N)
        G = 2 * NN * a.scratch[N - 1] - 2 * U + 2 * NN * charge_at(a, N);
    else
        G = NN * (a.scratch[j - 1] + a.scratch[j]) - 2 * U;
    a.E[j] = a.lambda * i128_to_double(G);
}

// The device address of the scratch array for the current device.  Host code must not
// hand the symbol itself to a kernel.  Outside stream capture the address is looked up
// on every call (cheap; a device reset or a new context reloads the module at another
// address); during a capture the lookup could load the module inside it, so the address
// of the last lookup on this device is reused and a first call under capture fails.
int scratch_for_current_device(cudaStream_t st, void** out, std::string* why)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *why = "device index out of range";
        return PIC_EINVAL;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) {
        *why = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PIC_ECUDA;
        }
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        *why = "the first call on a device must not be made during stream capture";
        return PIC_EINVAL;
    }
    *out = g_scratch_addr[dev];
    return PIC_OK;
}

}  // namespace

// defined with pic_last_error: the message pic_last_error(NULL) returns
void set_global_error(const std::string& msg);

}  // namespace bitpic

using namespace bitpic;

extern "C" PIC_API int pic_field_solve_noalloc(int32_t ncells, int32_t nspecies,
                                               const int64_t* charge, const int32_t* z,
                                               double delta, int64_t unit, double eps0,
                                               double* E, void* stream)
{
    set_global_error("");
    if (ncells < 1 || ncells > kNoAllocMaxCells) {
        set_global_error("pic_field_solve_noalloc: ncells must be in [1, " +
                         std::to_string(kNoAllocMaxCells) + "] (the size of its static scratch)");
        return PIC_EINVAL;
    }
    if (nspecies < 1 || nspecies > kMaxSpecies || !charge || !z || !E || unit <= 0 ||
        !(delta > 0) || !(eps0 > 0)) {
        set_global_error("pic_field_solve_noalloc: bad arguments");
        return PIC_EINVAL;
    }
    void* scratch = nullptr;
    std::string why;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = scratch_for_current_device(st, &scratch, &why);
    if (rc != PIC_OK) {
        set_global_error("pic_field_solve_noalloc: " + why);
        return rc;
    }
    NoAllocArgs a;
    a.charge = reinterpret_cast<const long long*>(charge);
    a.ncells = ncells;
    a.nspecies = nspecies;
    for (int k = 0; k < kMaxSpecies; ++k) a.z[k] = k < nspecies ? z[k] : 0;
    a.lambda = delta / (2.0 * (double)ncells * (double)unit * eps0);
    a.scratch = static_cast<i128*>(scratch);
    a.E = E;
    k_scan_noalloc<<<1, 1024, 0, st>>>(a);
    k_emit_noalloc<<<(ncells + 1 + 255) / 256, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(std::string("pic_field_solve_noalloc: ") + cudaGetErrorString(e));
        return PIC_ECUDA;
    }
    return PIC_OK;
}
