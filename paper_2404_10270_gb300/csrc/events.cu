// events.cu -- instantiations of the rare-event kernel for both precisions.
#include "events.cuh"
#include "kernels.h"

namespace bitpic {

cudaError_t launch_events(const MoveArgs& a, int precision, int grid, cudaStream_t st)
{
    if (precision == PIC_FP64)
        k_events<double><<<grid, 128, 0, st>>>(a);
    else
        k_events<float><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_victims(const MoveArgs& a, int precision, int grid, cudaStream_t st)
{
    if (precision == PIC_FP64)
        k_victims<double><<<grid, 128, 0, st>>>(a);
    else
        k_victims<float><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_drift_y(const MoveArgs& a, int precision, int grid, cudaStream_t st)
{
    if (precision == PIC_FP64)
        k_drift_y<double><<<grid, 256, 0, st>>>(a);
    else
        k_drift_y<float><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bitpic
