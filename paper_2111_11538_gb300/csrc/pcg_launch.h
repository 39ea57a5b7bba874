// The persistent PCG kernels are compiled in their own translation units
// (pcg_2d.cu, pcg_3d.cu: one per dimension, built in parallel); the field
// library reaches them through these host functions.
#pragma once
#include <cuda_runtime.h>

// shape: 0 or 1 (the node tiles of pf_cg.cuh); mg: the multigrid-
// preconditioned variant (2D only; ignored in 3D); jobs: device table of
// PCGArgs<T, D>; tabF / tabD: host copies of the element tables.
cudaError_t pcg2_occupancy(bool fp64, int shape, bool mg, int block, int *per_sm);
cudaError_t pcg2_launch(bool fp64, int shape, bool mg, const void *jobs, int njobs, int grid, int block, cudaStream_t s);
cudaError_t pcg2_tables(const void *tabF, const void *tabD);
cudaError_t pcg3_occupancy(bool fp64, int shape, bool mg, int block, int *per_sm);
cudaError_t pcg3_launch(bool fp64, int shape, bool mg, const void *jobs, int njobs, int grid, int block, cudaStream_t s);
cudaError_t pcg3_tables(const void *tabF, const void *tabD);
