// Persistent PCG kernels for 2D grids (both storage types, both tile
// shapes) and their host entry points (pcg_launch.h).
#include "pf_cg.cuh"
#include "pcg_launch.h"

using namespace pfdev;

cudaError_t pcg2_occupancy(bool fp64, int shape, bool mg, int block, int *per_sm)
{
    return fp64 ? pcg_occupancy_t<double, 2>(shape, mg, block, per_sm) : pcg_occupancy_t<float, 2>(shape, mg, block, per_sm);
}

cudaError_t pcg2_launch(bool fp64, int shape, bool mg, const void *jobs, int njobs, int grid, int block, cudaStream_t s)
{
    return fp64 ? pcg_launch_t<double, 2>(shape, mg, jobs, njobs, grid, block, s)
                : pcg_launch_t<float, 2>(shape, mg, jobs, njobs, grid, block, s);
}

cudaError_t pcg2_tables(const void *tabF, const void *tabD)
{
    cudaError_t e = cudaMemcpyToSymbol(cTabF, tabF, sizeof(Tab<float>));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cTabD, tabD, sizeof(Tab<double>));
    return e;
}
