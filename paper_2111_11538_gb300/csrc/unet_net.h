// Internal interface between the field library and the warm-start network
// (both compiled into libpf.so; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

struct pf_unet;
struct UWork;

// Inference workspace for nb samples of nx * ny * nz cells (nullptr if the
// grid does not suit the network or memory is short).  Its buffers never
// move, so launches that read them may be captured into a CUDA graph.
UWork *unet_work_create(pf_unet *n, int nb, int nx, int ny, int nz);
void unet_work_destroy(UWork *w);
// y = net(x) on stream s; x: nb * cells * cin FP32 (device); *out points at
// the workspace's nb * cells * ndim FP32 result.  Returns a pf.h status.
int unet_forward_work(pf_unet *n, UWork *w, const float *in, const float **out, cudaStream_t s);
int unet_ndim(const pf_unet *n);
int unet_cin(const pf_unet *n);
int unet_check_grid(pf_unet *n, int nx, int ny, int nz);
const char *unet_error(const pf_unet *n);
