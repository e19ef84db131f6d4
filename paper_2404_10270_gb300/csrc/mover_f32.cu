// mover_f32.cu -- instantiations of the fused mover for float particle state.
#include "kernels.h"
#include "mover.cuh"

namespace bitpic {

namespace {
template <int NT, bool SUB, bool TEST, bool KEPT>
cudaError_t go_sub(const MoveArgs& a, bool mag, bool mixed, int grid, cudaStream_t st)
{
    if (!mag)
        k_move<float, NT, false, true, SUB, false, TEST, KEPT><<<grid, NT, 0, st>>>(a);
    else if (mixed)
        k_move<float, NT, true, true, SUB, true, TEST, KEPT><<<grid, NT, 0, st>>>(a);
    else
        k_move<float, NT, true, true, SUB, false, TEST, KEPT><<<grid, NT, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t go(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed, bool sort,
               bool lean, bool gridv, bool kept, int grid, cudaStream_t st)
{
    if (!move) {
        k_move<float, NT, false, false, false, false, true><<<grid, NT, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (sort) return launch_sort_step<float, NT>(a, mag, sub, mixed, grid, st);
    if (gridv && !lean && !mag && !sub) {
        k_move<float, NT, false, true, false, false, true, false, true><<<grid, NT, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (lean && !mag) {
        if (sub && kept)
            k_move<float, NT, false, true, true, false, false, true><<<grid, NT, 0, st>>>(a);
        else if (sub)
            k_move<float, NT, false, true, true, false, false><<<grid, NT, 0, st>>>(a);
        else
            k_move<float, NT, false, true, false, false, false><<<grid, NT, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (sub && kept) return go_sub<NT, true, true, true>(a, mag, mixed, grid, st);
    if (sub) return go_sub<NT, true, true, false>(a, mag, mixed, grid, st);
    return go_sub<NT, false, true, false>(a, mag, mixed, grid, st);
}

template <int NT>
int occupancy(bool mag, bool sort, bool yp, bool subtest, bool gridv)
{
    if (sort) return sort_step_blocks_per_sm<float, NT>(mag, yp);
    int n = 0;
    const cudaError_t e =
        gridv ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<float, NT, false, true, false, false, true, false, true>, NT, 0)
        : mag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<float, NT, true, true, false, false, true>, NT, 0)
        : subtest ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<float, NT, false, true, true, false, true>, NT, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<float, NT, false, true, false, false, true>, NT, 0);
    return e == cudaSuccess ? n : 0;
}
}  // namespace

cudaError_t launch_move_f32(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed,
                            bool sort, bool lean, bool gridv, bool kept, int nt, int grid,
                            cudaStream_t st)
{
    switch (nt) {
        case 128: return go<128>(a, mag, move, sub, mixed, sort, lean, gridv, kept, grid, st);
        case 512: return go<512>(a, mag, move, sub, mixed, sort, lean, gridv, kept, grid, st);
        default: return go<256>(a, mag, move, sub, mixed, sort, lean, gridv, kept, grid, st);
    }
}

int move_blocks_per_sm_f32(bool mag, bool sort, bool yp, bool subtest, bool gridv, int nt)
{
    switch (nt) {
        case 128: return occupancy<128>(mag, sort, yp, subtest, gridv);
        case 512: return occupancy<512>(mag, sort, yp, subtest, gridv);
        default: return occupancy<256>(mag, sort, yp, subtest, gridv);
    }
}

}  // namespace bitpic
