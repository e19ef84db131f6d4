// mover_f64.cu -- instantiations of the fused mover for double particle state.
#include "kernels.h"
#include "mover.cuh"

namespace bitpic {

namespace {
template <int NT, bool SUB, bool KEPT>
cudaError_t go_sub(const MoveArgs& a, bool mag, bool mixed, int grid, cudaStream_t st)
{
    if (!mag)
        k_move<double, NT, false, true, SUB, false, true, KEPT><<<grid, NT, 0, st>>>(a);
    else if (mixed)
        k_move<double, NT, true, true, SUB, true, true, KEPT><<<grid, NT, 0, st>>>(a);
    else
        k_move<double, NT, true, true, SUB, false, true, KEPT><<<grid, NT, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t go(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed, bool sort,
               bool kept, int grid, cudaStream_t st)
{
    if (!move) {
        k_move<double, NT, false, false, false, false, true><<<grid, NT, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (sort) return launch_sort_step<double, NT>(a, mag, sub, mixed, grid, st);
    if (sub && kept) return go_sub<NT, true, true>(a, mag, mixed, grid, st);
    if (sub) return go_sub<NT, true, false>(a, mag, mixed, grid, st);
    return go_sub<NT, false, false>(a, mag, mixed, grid, st);
}

template <int NT>
int occupancy(bool mag, bool sort, bool yp)
{
    if (sort) return sort_step_blocks_per_sm<double, NT>(mag, yp);
    int n = 0;
    const cudaError_t e =
        mag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<double, NT, true, true, false, false, true>, NT, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<double, NT, false, true, false, false, true>, NT, 0);
    return e == cudaSuccess ? n : 0;
}
}  // namespace

cudaError_t launch_move_f64(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed,
                            bool sort, bool kept, int nt, int grid, cudaStream_t st)
{
    switch (nt) {
        case 128: return go<128>(a, mag, move, sub, mixed, sort, kept, grid, st);
        case 512: return go<512>(a, mag, move, sub, mixed, sort, kept, grid, st);
        default: return go<256>(a, mag, move, sub, mixed, sort, kept, grid, st);
    }
}

int move_blocks_per_sm_f64(bool mag, bool sort, bool yp, int nt)
{
    switch (nt) {
        case 128: return occupancy<128>(mag, sort, yp);
        case 512: return occupancy<512>(mag, sort, yp);
        default: return occupancy<256>(mag, sort, yp);
    }
}

}  // namespace bitpic
