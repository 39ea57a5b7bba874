// Internal interface between the field library and the warm-start network
// (both compiled into libpf.so; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

struct pf_unet;

// y = net(x) on stream s; x: nb * cells * cin FP32, y: nb * cells * ndim FP32
// (device).  Returns a pf.h status; unet_error() gives the text.
int unet_forward_internal(pf_unet *n, const float *in, float *out, int nb, int nx, int ny, int nz, cudaStream_t s);
int unet_ndim(const pf_unet *n);
int unet_cin(const pf_unet *n);
int unet_check_grid(pf_unet *n, int nx, int ny, int nz);
const char *unet_error(const pf_unet *n);
