// Warm-start network: host orchestration of the U-Net kernels (forward,
// backward, Adam) behind the C ABI of include/pf_unet.h.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_unet.h"
#include "unet_kernels.cuh"
#include "unet_net.h"

using namespace unet;

namespace {

thread_local std::string g_unet_create_error;

// ---------------------------------------------------------------------------
// Small kernels (CUDA cores): input packing, pooling, the 1x1 output layer,
// loss, gradient plumbing, weight layouts, Adam.
// ---------------------------------------------------------------------------
__global__ void k_pack_input(long long n, int cin, const float *in, __nv_bfloat16 *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * 16; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i >> 4;
        const int c = (int)(i & 15);
        out[i] = __float2bfloat16(c < cin ? in[p * cin + c] : 0.f);
    }
}

// average of the 2^D children; dims are the child level's
template <int D>
__global__ void k_pool(Dims d, int C, const __nv_bfloat16 *a, __nv_bfloat16 *p)
{
    const int hx = d.nx >> 1, hy = d.ny >> 1, hz = D == 3 ? d.nz >> 1 : 1;
    const long long hc = (long long)hx * hy * hz, fc = (long long)d.nx * d.ny * (D == 3 ? d.nz : 1);
    const long long n = hc * d.nb * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int b = (int)(q / hc);
        q -= (long long)b * hc;
        const int x = (int)(q % hx), r = (int)(q / hx), y = r % hy, z = r / hy;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < (D == 3 ? 8 : 4); k++) {
            const int cx = 2 * x + (k & 1), cy = 2 * y + ((k >> 1) & 1), cz = D == 3 ? 2 * z + (k >> 2) : 0;
            const long long cp = (long long)b * fc + cx + (long long)d.nx * (cy + (long long)d.ny * cz);
            s += __bfloat162float(a[cp * C + c]);
        }
        p[i] = __float2bfloat16(s * (D == 3 ? 0.125f : 0.25f));
    }
}

// g_a[child] += g_p[parent] / 2^D  (average-pooling backward); dims are the child level's
template <int D>
__global__ void k_pool_bwd(Dims d, int C, const float *gp, float *ga)
{
    const int hx = d.nx >> 1, hy = d.ny >> 1, hz = D == 3 ? d.nz >> 1 : 1;
    const long long hc = (long long)hx * hy * hz, fc = (long long)d.nx * d.ny * (D == 3 ? d.nz : 1);
    const long long n = fc * d.nb * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int b = (int)(q / fc);
        q -= (long long)b * fc;
        const int x = (int)(q % d.nx), r = (int)(q / d.nx), y = r % d.ny, z = r / d.ny;
        const long long pp = (long long)b * hc + (x >> 1) + (long long)hx * ((y >> 1) + (long long)hy * (z >> 1));
        ga[i] += gp[pp * C + c] * (D == 3 ? 0.125f : 0.25f);
    }
}

// 1x1 output layer: y[p, o] = b[o] + sum_c W[o, c] d[p, c]  (FP32)
__global__ void k_out_fwd(long long n, int C, int CO, const __nv_bfloat16 *d, const float *W, const float *b, float *y)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        for (int o = 0; o < CO; o++) {
            float s = b[o];
            for (int c = 0; c < C; c++) s = fmaf(W[o * C + c], __bfloat162float(d[p * C + c]), s);
            y[p * CO + o] = s;
        }
    }
}

// gy = 2 (y - t) / n_elems; per-block partial sums of (y - t)^2 (FP64)
__global__ void k_loss(long long n, const float *y, const float *t, float *gy, double inv_n, double *part)
{
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        gy[i] = (float)(2.0 * inv_n) * e;
        s += (double)e * (double)e;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Stiffness-weighted gradient loss: per cell q the forward differences
// de_d(q) = e(q + e_d) - e(q) (e = y - t, periodic within the sample),
// loss += w_q sum_d |de_d(q)|^2, w_q = floor + (1 - floor)(1 - in[q, wch]);
// gy(q) = 2 inv_n sum_d [w_{q-e_d} de_d(q - e_d) - w_q de_d(q)].
template <int D>
__global__ void k_loss_grad(Dims dm, int C, const float *y, const float *t, const float *in, int cin, int wch,
                            float floor_w, float *gy, double inv_n, double *part)
{
    const int nx = dm.nx, ny = dm.ny, nz = D == 3 ? dm.nz : 1;
    const long long cells = (long long)nx * ny * nz;
    const long long n = cells * dm.nb;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long b = q / cells;
        const long long r = q - b * cells;
        const int x = (int)(r % nx), yy = (int)((r / nx) % ny), z = (int)(r / ((long long)nx * ny));
        auto at = [&](int xi, int yi, int zi) -> long long {
            xi = wrapc(xi, nx); yi = wrapc(yi, ny); zi = D == 3 ? wrapc(zi, nz) : 0;
            return b * cells + xi + (long long)nx * (yi + (long long)ny * zi);
        };
        auto wt = [&](long long p) { return floor_w + (1.f - floor_w) * (1.f - in[p * cin + wch]); };
        const float wq = wt(q);
        for (int c = 0; c < C; c++) {
            const float eq = y[q * C + c] - t[q * C + c];
            float g = 0.f;
            for (int d = 0; d < D; d++) {
                const long long pp = at(x + (d == 0), yy + (d == 1), z + (d == 2));
                const long long pm = at(x - (d == 0), yy - (d == 1), z - (d == 2));
                const float ep = y[pp * C + c] - t[pp * C + c];
                const float em = y[pm * C + c] - t[pm * C + c];
                const float dq = ep - eq, dm1 = eq - em;
                s += (double)wq * (double)dq * (double)dq;
                g += wt(pm) * dm1 - wq * dq;
            }
            gy[q * C + c] = (float)(2.0 * inv_n) * g;
        }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// output-layer backward: g_d[p, c] = sum_o W[o, c] gy[p, o]; gW[o, c] += sum_p gy[p, o] d[p, c]; gb[o] += sum_p gy
__global__ void k_out_bwd(long long n, int C, int CO, const __nv_bfloat16 *d, const float *W, const float *gy,
                          float *gd, float *gW, float *gb)
{
    extern __shared__ float sacc[];           // CO * C + CO
    for (int i = threadIdx.x; i < CO * C + CO; i += blockDim.x) sacc[i] = 0.f;
    __syncthreads();
    float loc[4 * 64 + 4];
    for (int i = 0; i < CO * C + CO; i++) loc[i] = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < C; c++) {
            float s = 0.f;
            const float dv = __bfloat162float(d[p * C + c]);
            for (int o = 0; o < CO; o++) {
                const float g = gy[p * CO + o];
                s = fmaf(W[o * C + c], g, s);
                loc[o * C + c] = fmaf(g, dv, loc[o * C + c]);
            }
            gd[p * C + c] = s;
        }
        for (int o = 0; o < CO; o++) loc[CO * C + o] += gy[p * CO + o];
    }
    for (int i = 0; i < CO * C + CO; i++) atomicAdd(&sacc[i], loc[i]);
    __syncthreads();
    for (int i = threadIdx.x; i < CO * C; i += blockDim.x) atomicAdd(&gW[i], sacc[i]);
    for (int i = threadIdx.x; i < CO; i += blockDim.x) atomicAdd(&gb[i], sacc[CO * C + i]);
}

// gz = bf16(g * [out > 0])  (ReLU backward at a convolution's output)
template <typename G>
__global__ void k_relu_mask(long long n, const G *g, const __nv_bfloat16 *out, __nv_bfloat16 *gz)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v;
        if constexpr (sizeof(G) == 4) v = (float)g[i];
        else v = __bfloat162float(g[i]);
        gz[i] = __float2bfloat16(__bfloat162float(out[i]) > 0.f ? v : 0.f);
    }
}

// g_skip[p, c] += gin[p, c] for c < C0  (the skip part of a concatenated input)
__global__ void k_acc_skip(long long n, int C0, int Cin, const __nv_bfloat16 *gin, float *gs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * C0; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C0;
        const int c = (int)(i % C0);
        gs[i] += __bfloat162float(gin[p * Cin + c]);
    }
}

// g_up[parent, c] = sum over the 2^D children of gin[child, C0 + c]  (nearest-upsample backward)
template <int D>
__global__ void k_up_bwd(Dims d, int C0, int C1, const __nv_bfloat16 *gin, float *gu)
{
    const int hx = d.nx >> 1, hy = d.ny >> 1, hz = D == 3 ? d.nz >> 1 : 1;
    const long long hc = (long long)hx * hy * hz, fc = (long long)d.nx * d.ny * (D == 3 ? d.nz : 1);
    const long long n = hc * d.nb * C1;
    const int Cin = C0 + C1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C1);
        long long q = i / C1;
        const int b = (int)(q / hc);
        q -= (long long)b * hc;
        const int x = (int)(q % hx), r = (int)(q / hx), y = r % hy, z = r / hy;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < (D == 3 ? 8 : 4); k++) {
            const int cx = 2 * x + (k & 1), cy = 2 * y + ((k >> 1) & 1), cz = D == 3 ? 2 * z + (k >> 2) : 0;
            const long long cp = (long long)b * fc + cx + (long long)d.nx * (cy + (long long)d.ny * cz);
            s += __bfloat162float(gin[cp * Cin + C0 + c]);
        }
        gu[i] = s;
    }
}

// gb[c] += sum_p gz[p, c]
__global__ void k_bias_grad(long long n, int C, const __nv_bfloat16 *gz, float *gb)
{
    __shared__ float s[64];
    for (int i = threadIdx.x; i < C; i += blockDim.x) s[i] = 0.f;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * C; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&s[i % C], __bfloat162float(gz[i]));
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(&gb[i], s[i]);
}

// weights in the kernels' layouts from the FP32 master W[co][ci][taps]:
// fwd[tap][co][cip] and, for the input-gradient pass, bwd[tap][cip][co]
__global__ void k_weights(int co_n, int ci_n, int cip, int taps, const float *W, __nv_bfloat16 *fwd, __nv_bfloat16 *bwd)
{
    const int n = taps * co_n * cip;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cip, r = i / cip, co = r % co_n, tap = r / co_n;
        const float w = ci < ci_n ? W[((size_t)co * ci_n + ci) * taps + tap] : 0.f;
        const __nv_bfloat16 v = __float2bfloat16(w);
        fwd[i] = v;
        if (bwd) bwd[((size_t)tap * cip + ci) * co_n + co] = v;
    }
}

// gW master layout [co][ci][taps] += kernel layout [tap][co][cip]
__global__ void k_wgrad_to_master(int co_n, int ci_n, int cip, int taps, const float *gk, float *gW)
{
    const int n = co_n * ci_n * taps;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i % taps, r = i / taps, ci = r % ci_n, co = r / ci_n;
        gW[i] += gk[((size_t)tap * co_n + co) * cip + ci];
    }
}

__global__ void k_adam(long long n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int blocks_for(long long n, int per = 256)
{
    long long b = (n + per - 1) / per;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Network object
// ---------------------------------------------------------------------------
struct ConvLayer {
    int ci, cip, co, taps;          // input channels (padded cip), output channels, taps
    long long woff, boff;           // offsets in the flat parameter vector
    __nv_bfloat16 *wf = nullptr, *wb = nullptr;   // kernel layouts
    float *gk = nullptr;            // weight gradient in the kernel layout
};

// Activations (and, for training, gradients) of one (nb, nx, ny, nz).  The
// network's own calls use the network's workspace; a field handle that
// replays the inference inside a CUDA graph owns a separate one, so that no
// call on the network can move buffers the graph points at.
struct UWork {
    int wnb = -1, wnx = -1, wny = -1, wnz = -1;
    bool grads = false;
    std::vector<void *> work;
    __nv_bfloat16 *x0 = nullptr;
    std::vector<__nv_bfloat16 *> enc1, enc2, pool, dec1, dec2;     // per level
    std::vector<float *> g_a, g_d, g_p;                            // FP32 gradients per level
    __nv_bfloat16 *gz = nullptr, *gin = nullptr;                   // scratch (largest level)
    float *y = nullptr, *gy = nullptr, *gd0 = nullptr;
    void release()
    {
        for (void *p : work) cudaFree(p);
        work.clear();
        wnb = wnx = wny = wnz = -1;
    }
};

struct pf_unet {
    pf_unet_config cfg;
    std::string err;
    std::vector<ConvLayer> layers;
    long long nparam = 0;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    long long adam_t = 0;
    double *part = nullptr;         // loss partials
    std::vector<void *> allocs;
    UWork train;                    // workspace of pf_unet_forward / pf_unet_loss_grad
    int loss_kind = 0;              // PF_UNET_LOSS_MSE / PF_UNET_LOSS_GRAD
    int loss_wch = 1;
    float loss_floor = 0.01f;

    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda(cudaError_t e, const char *what)
    {
        if (e == cudaSuccess) return PF_OK;
        return fail(e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    template <typename X>
    int alloc(X **p, size_t bytes, std::vector<void *> &list)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
        if (e != cudaSuccess) return fail(PF_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        list.push_back(q);
        *p = (X *)q;
        return PF_OK;
    }
};

#define UN_TRY(x) do { int _rc = (x); if (_rc != PF_OK) return _rc; } while (0)

namespace {

template <int D, int C>
void set_smem_attrs()
{
    cudaFuncSetAttribute(k_conv3<D, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3_smem<D, C>());
}

template <int D, int C>
void set_wgrad_attrs()
{
    cudaFuncSetAttribute(k_conv3_wgrad<D, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem<D, C>());
}

template <int D>
bool prepare_kernels()
{
    set_smem_attrs<D, 16>(); set_smem_attrs<D, 32>(); set_smem_attrs<D, 48>(); set_smem_attrs<D, 64>();
    set_smem_attrs<D, 80>(); set_smem_attrs<D, 96>(); set_smem_attrs<D, 112>(); set_smem_attrs<D, 128>();
    set_wgrad_attrs<D, 16>(); set_wgrad_attrs<D, 32>(); set_wgrad_attrs<D, 48>(); set_wgrad_attrs<D, 64>();
    return cudaGetLastError() == cudaSuccess;
}

template <int D, int C>
void launch_conv_t(const ConvArgs &a, long long tiles, cudaStream_t s)
{
    k_conv3<D, C><<<(unsigned)tiles, 256, conv3_smem<D, C>(), s>>>(a);
}

template <int D>
int launch_conv(int cout, const ConvArgs &a, long long tiles, cudaStream_t s)
{
    switch (cout) {
    case 16: launch_conv_t<D, 16>(a, tiles, s); break;
    case 32: launch_conv_t<D, 32>(a, tiles, s); break;
    case 48: launch_conv_t<D, 48>(a, tiles, s); break;
    case 64: launch_conv_t<D, 64>(a, tiles, s); break;
    case 80: launch_conv_t<D, 80>(a, tiles, s); break;
    case 96: launch_conv_t<D, 96>(a, tiles, s); break;
    case 112: launch_conv_t<D, 112>(a, tiles, s); break;
    case 128: launch_conv_t<D, 128>(a, tiles, s); break;
    default: return PF_EINVAL;
    }
    return PF_OK;
}

template <int D, int C>
void launch_wgrad_t(const WGradArgs &a, int cin, cudaStream_t s)
{
    long long gx = a.ntiles < 152 * 2 ? a.ntiles : 152 * 2;
    dim3 grid((unsigned)gx, (unsigned)(cin / 16), (unsigned)wgrad_zsplit<D, C>());
    k_conv3_wgrad<D, C><<<grid, 256, wgrad_smem<D, C>(), s>>>(a);
}

template <int D>
int launch_wgrad(int cout, const WGradArgs &a, int cin, cudaStream_t s)
{
    switch (cout) {
    case 16: launch_wgrad_t<D, 16>(a, cin, s); break;
    case 32: launch_wgrad_t<D, 32>(a, cin, s); break;
    case 48: launch_wgrad_t<D, 48>(a, cin, s); break;
    case 64: launch_wgrad_t<D, 64>(a, cin, s); break;
    default: return PF_EINVAL;
    }
    return PF_OK;
}

long long level_cells(const pf_unet *n, const UWork *w, int l)
{
    long long c = (long long)(w->wnx >> l) * (w->wny >> l);
    if (n->cfg.ndim == 3) c *= (w->wnz >> l);
    return c;
}

Dims level_dims(const pf_unet *n, const UWork *w, int l)
{
    Dims d;
    d.nx = w->wnx >> l;
    d.ny = w->wny >> l;
    d.nz = n->cfg.ndim == 3 ? w->wnz >> l : 1;
    d.nb = w->wnb;
    return d;
}

long long level_tiles(const pf_unet *n, const UWork *w, int l)
{
    const Dims d = level_dims(n, w, l);
    if (n->cfg.ndim == 2) return (long long)(d.nx / 16) * (d.ny / 8) * d.nb;
    return (long long)(d.nx / 16) * (d.ny / 4) * (d.nz / 2) * d.nb;
}

int check_dims(pf_unet *n, int nb, int nx, int ny, int nz)
{
    const int L = n->cfg.levels, f = 1 << (L - 1);
    if (nb < 1) return n->fail(PF_EINVAL, "nb < 1");
    if (n->cfg.ndim == 2) {
        if (nx % (16 * f) || ny % (8 * f)) return n->fail(PF_EINVAL, "2D grid must satisfy nx %% %d == 0 and ny %% %d == 0", 16 * f, 8 * f);
    } else {
        if (nx % (16 * f) || ny % (4 * f) || nz % (2 * f))
            return n->fail(PF_EINVAL, "3D grid must satisfy nx %% %d, ny %% %d, nz %% %d == 0", 16 * f, 4 * f, 2 * f);
    }
    return PF_OK;
}

int ensure_work(pf_unet *n, UWork *w, int nb, int nx, int ny, int nz, bool grads)
{
    if (n->cfg.ndim == 2) nz = 1;
    if (w->wnb == nb && w->wnx == nx && w->wny == ny && w->wnz == nz && (w->grads || !grads)) return PF_OK;
    w->release();
    w->grads = grads;
    w->wnb = nb; w->wnx = nx; w->wny = ny; w->wnz = nz;
    const int L = n->cfg.levels;
    const int D = n->cfg.ndim;
    w->enc1.assign(L, nullptr); w->enc2.assign(L, nullptr); w->pool.assign(L, nullptr);
    w->dec1.assign(L, nullptr); w->dec2.assign(L, nullptr);
    w->g_a.assign(L, nullptr); w->g_d.assign(L, nullptr); w->g_p.assign(L, nullptr);
    const long long c0 = level_cells(n, w, 0) * nb;
    UN_TRY(n->alloc(&w->x0, sizeof(__nv_bfloat16) * c0 * 16, w->work));
    size_t big = 0;
    for (int l = 0; l < L; l++) {
        const long long c = level_cells(n, w, l) * nb;
        const int C = n->cfg.channels[l];
        UN_TRY(n->alloc(&w->enc1[l], sizeof(__nv_bfloat16) * c * C, w->work));
        UN_TRY(n->alloc(&w->enc2[l], sizeof(__nv_bfloat16) * c * C, w->work));
        if (l > 0) UN_TRY(n->alloc(&w->pool[l], sizeof(__nv_bfloat16) * c * n->cfg.channels[l - 1], w->work));
        if (l < L - 1) {
            UN_TRY(n->alloc(&w->dec1[l], sizeof(__nv_bfloat16) * c * C, w->work));
            UN_TRY(n->alloc(&w->dec2[l], sizeof(__nv_bfloat16) * c * C, w->work));
        }
        if (grads) {
            UN_TRY(n->alloc(&w->g_a[l], sizeof(float) * c * C, w->work));
            UN_TRY(n->alloc(&w->g_d[l], sizeof(float) * c * C, w->work));
            if (l > 0) UN_TRY(n->alloc(&w->g_p[l], sizeof(float) * c * n->cfg.channels[l - 1], w->work));
        }
        // widest per-cell tensor of this level: a decoder input, a pooled
        // input or the padded network input
        int cin_max = n->cfg.channels[l] + (l + 1 < L ? n->cfg.channels[l + 1] : 0);
        if (l > 0 && n->cfg.channels[l - 1] > cin_max) cin_max = n->cfg.channels[l - 1];
        if (cin_max < 16) cin_max = 16;
        const size_t need = (size_t)c * cin_max;
        if (need > big) big = need;
    }
    UN_TRY(n->alloc(&w->y, sizeof(float) * c0 * D, w->work));
    if (grads) {
        UN_TRY(n->alloc(&w->gz, sizeof(__nv_bfloat16) * big, w->work));
        UN_TRY(n->alloc(&w->gin, sizeof(__nv_bfloat16) * big, w->work));
        UN_TRY(n->alloc(&w->gy, sizeof(float) * c0 * D, w->work));
        UN_TRY(n->alloc(&w->gd0, sizeof(float) * c0 * n->cfg.channels[0], w->work));
    }
    return PF_OK;
}

int upload_weights(pf_unet *n, cudaStream_t s)
{
    for (ConvLayer &c : n->layers) {
        if (c.taps == 1) continue;
        k_weights<<<blocks_for((long long)c.taps * c.co * c.cip), 256, 0, s>>>(c.co, c.ci, c.cip, c.taps, n->params + c.woff, c.wf, c.wb);
    }
    return n->cuda(cudaGetLastError(), "weight layout");
}

ConvArgs conv_args(const __nv_bfloat16 *in0, int C0, const __nv_bfloat16 *in1, int C1, const __nv_bfloat16 *w,
                   const float *bias, __nv_bfloat16 *out, int relu, int mirror, Dims d)
{
    ConvArgs a;
    a.in0 = in0; a.in1 = in1; a.C0 = C0; a.C1 = C1; a.wt = w; a.bias = bias; a.out = out;
    a.relu = relu; a.mirror = mirror; a.dim = d;
    return a;
}

template <int D>
int forward_t(pf_unet *n, UWork *w, const float *in, cudaStream_t s)
{
    const int L = n->cfg.levels;
    const long long c0 = level_cells(n, w, 0) * w->wnb;
    k_pack_input<<<blocks_for(c0 * 16), 256, 0, s>>>(c0, n->cfg.cin, in, w->x0);
    int k = 0;
    for (int l = 0; l < L; l++) {
        const Dims d = level_dims(n, w, l);
        const long long tiles = level_tiles(n, w, l);
        const __nv_bfloat16 *src = l == 0 ? w->x0 : w->pool[l];
        if (l > 0) {
            const Dims dp = level_dims(n, w, l - 1);
            const long long m = level_cells(n, w, l) * w->wnb * n->cfg.channels[l - 1];
            k_pool<D><<<blocks_for(m), 256, 0, s>>>(dp, n->cfg.channels[l - 1], w->enc2[l - 1], w->pool[l]);
        }
        ConvLayer &A = n->layers[k], &B = n->layers[k + 1];
        UN_TRY(launch_conv<D>(A.co, conv_args(src, A.cip, nullptr, 0, A.wf, n->params + A.boff, w->enc1[l], 1, 0, d), tiles, s));
        UN_TRY(launch_conv<D>(B.co, conv_args(w->enc1[l], B.cip, nullptr, 0, B.wf, n->params + B.boff, w->enc2[l], 1, 0, d), tiles, s));
        k += 2;
    }
    for (int l = L - 2; l >= 0; l--) {
        const Dims d = level_dims(n, w, l);
        const long long tiles = level_tiles(n, w, l);
        const __nv_bfloat16 *coarse = l == L - 2 ? w->enc2[L - 1] : w->dec2[l + 1];
        ConvLayer &A = n->layers[k], &B = n->layers[k + 1];
        const int C0 = n->cfg.channels[l], C1 = n->cfg.channels[l + 1];
        UN_TRY(launch_conv<D>(A.co, conv_args(w->enc2[l], C0, coarse, C1, A.wf, n->params + A.boff, w->dec1[l], 1, 0, d), tiles, s));
        UN_TRY(launch_conv<D>(B.co, conv_args(w->dec1[l], B.cip, nullptr, 0, B.wf, n->params + B.boff, w->dec2[l], 1, 0, d), tiles, s));
        k += 2;
    }
    const ConvLayer &O = n->layers[k];
    const __nv_bfloat16 *d0 = L > 1 ? w->dec2[0] : w->enc2[0];
    k_out_fwd<<<blocks_for(c0), 256, 0, s>>>(c0, O.ci, O.co, d0, n->params + O.woff, n->params + O.boff, w->y);
    return n->cuda(cudaGetLastError(), "forward");
}

// backward of one 3^D convolution with ReLU at its output: g (at the output,
// FP32 or BF16) -> gz; weight and bias gradients; input gradient in w->gin
// (BF16, Cin channels) unless skip_input.
template <int D, typename G>
int conv_backward(pf_unet *n, UWork *w, const ConvLayer &c, const G *g, const __nv_bfloat16 *out,
                  const __nv_bfloat16 *in0, int C0, const __nv_bfloat16 *in1, int C1, int l, bool skip_input,
                  cudaStream_t s)
{
    const Dims d = level_dims(n, w, l);
    const long long cells = level_cells(n, w, l) * w->wnb;
    const long long tiles = level_tiles(n, w, l);
    k_relu_mask<G><<<blocks_for(cells * c.co), 256, 0, s>>>(cells * c.co, g, out, w->gz);
    WGradArgs wa;
    wa.in0 = in0; wa.in1 = in1; wa.C0 = C0; wa.C1 = C1; wa.gz = w->gz; wa.gw = c.gk; wa.dim = d; wa.ntiles = tiles;
    UN_TRY(launch_wgrad<D>(c.co, wa, c.cip, s));
    k_bias_grad<<<blocks_for(cells * c.co, 1024), 256, 0, s>>>(cells, c.co, w->gz, n->grad + c.boff);
    if (!skip_input)
        UN_TRY(launch_conv<D>(c.cip, conv_args(w->gz, c.co, nullptr, 0, c.wb, nullptr, w->gin, 0, 1, d), tiles, s));
    return PF_OK;
}

template <int D>
int backward_t(pf_unet *n, UWork *w, const float *in, const float *target, double *loss, cudaStream_t s)
{
    const int L = n->cfg.levels;
    const long long c0 = level_cells(n, w, 0) * w->wnb;
    const int nblk = blocks_for(c0 * D);
    if (n->loss_kind == PF_UNET_LOSS_GRAD)
        k_loss_grad<D><<<blocks_for(c0), 256, 0, s>>>(level_dims(n, w, 0), D, w->y, target, in, n->cfg.cin, n->loss_wch,
                                                       n->loss_floor, w->gy, 1.0 / (double)(c0 * D), n->part);
    else
        k_loss<<<nblk, 256, 0, s>>>(c0 * D, w->y, target, w->gy, 1.0 / (double)(c0 * D), n->part);
    const int nparts = n->loss_kind == PF_UNET_LOSS_GRAD ? blocks_for(c0) : nblk;
    // zero gradients
    UN_TRY(n->cuda(cudaMemsetAsync(n->grad, 0, sizeof(float) * n->nparam, s), "zero"));
    for (ConvLayer &c : n->layers)
        if (c.gk) UN_TRY(n->cuda(cudaMemsetAsync(c.gk, 0, sizeof(float) * c.taps * c.co * c.cip, s), "zero"));
    for (int l = 0; l < L; l++) {
        UN_TRY(n->cuda(cudaMemsetAsync(w->g_a[l], 0, sizeof(float) * level_cells(n, w, l) * w->wnb * n->cfg.channels[l], s), "zero"));
        if (l > 0)
            UN_TRY(n->cuda(cudaMemsetAsync(w->g_p[l], 0, sizeof(float) * level_cells(n, w, l) * w->wnb * n->cfg.channels[l - 1], s), "zero"));
    }
    // output layer
    int k = (int)n->layers.size() - 1;
    const ConvLayer &O = n->layers[k];
    const __nv_bfloat16 *d0 = L > 1 ? w->dec2[0] : w->enc2[0];
    k_out_bwd<<<blocks_for(c0, 256) < 304 ? blocks_for(c0, 256) : 304, 256, sizeof(float) * (O.co * O.ci + O.co), s>>>(
        c0, O.ci, O.co, d0, n->params + O.woff, w->gy, L > 1 ? w->g_d[0] : w->g_a[0], n->grad + O.woff, n->grad + O.boff);
    k--;
    // decoder, level 0 first
    for (int l = 0; l <= L - 2; l++) {
        const ConvLayer &B = n->layers[k], &A = n->layers[k - 1];
        k -= 2;
        const int C0 = n->cfg.channels[l], C1 = n->cfg.channels[l + 1];
        const __nv_bfloat16 *coarse = l == L - 2 ? w->enc2[L - 1] : w->dec2[l + 1];
        // second conv: output dec2[l], input dec1[l]
        UN_TRY((conv_backward<D, float>(n, w, B, w->g_d[l], w->dec2[l], w->dec1[l], B.cip, nullptr, 0, l, false, s)));
        // first conv: output dec1[l] (gradient = gin of the second, BF16), input concat(enc2[l], up2(coarse))
        // gin is overwritten by this call's own input gradient, so mask it into gz first
        UN_TRY((conv_backward<D, __nv_bfloat16>(n, w, A, w->gin, w->dec1[l], w->enc2[l], C0, coarse, C1, l, false, s)));
        const long long cells = level_cells(n, w, l) * w->wnb;
        k_acc_skip<<<blocks_for(cells * C0), 256, 0, s>>>(cells, C0, C0 + C1, w->gin, w->g_a[l]);
        // up2 backward into the coarser level's gradient (written, not added:
        // g_d[l+1], or g_a[L-1] for the bottom, has no other contribution)
        float *gcoarse = l == L - 2 ? w->g_a[L - 1] : w->g_d[l + 1];
        const Dims d = level_dims(n, w, l);
        const long long hc = level_cells(n, w, l + 1) * w->wnb;
        k_up_bwd<D><<<blocks_for(hc * C1), 256, 0, s>>>(d, C0, C1, w->gin, gcoarse);
    }
    // encoder, deepest level first
    for (int l = L - 1; l >= 0; l--) {
        const ConvLayer &B = n->layers[k], &A = n->layers[k - 1];
        k -= 2;
        const __nv_bfloat16 *src = l == 0 ? w->x0 : w->pool[l];
        const int Cs = l == 0 ? 16 : n->cfg.channels[l - 1];
        UN_TRY((conv_backward<D, float>(n, w, B, w->g_a[l], w->enc2[l], w->enc1[l], B.cip, nullptr, 0, l, false, s)));
        UN_TRY((conv_backward<D, __nv_bfloat16>(n, w, A, w->gin, w->enc1[l], src, Cs, nullptr, 0, l, l == 0, s)));
        if (l > 0) {
            // gin = gradient at pool[l]; average-pooling backward into g_a[l-1]
            const long long hc = level_cells(n, w, l) * w->wnb;
            const int Cp = n->cfg.channels[l - 1];
            // convert gin (BF16, Cp channels) to FP32 g_p[l], then distribute
            k_acc_skip<<<blocks_for(hc * Cp), 256, 0, s>>>(hc, Cp, Cp, w->gin, w->g_p[l]);
            const Dims dc = level_dims(n, w, l - 1);
            k_pool_bwd<D><<<blocks_for(level_cells(n, w, l - 1) * w->wnb * Cp), 256, 0, s>>>(dc, Cp, w->g_p[l], w->g_a[l - 1]);
        }
    }
    // kernel-layout weight gradients into the master layout
    for (ConvLayer &c : n->layers) {
        if (c.taps == 1) continue;
        k_wgrad_to_master<<<blocks_for((long long)c.co * c.ci * c.taps), 256, 0, s>>>(c.co, c.ci, c.cip, c.taps, c.gk, n->grad + c.woff);
    }
    std::vector<double> part(nparts);
    UN_TRY(n->cuda(cudaMemcpyAsync(part.data(), n->part, sizeof(double) * nparts, cudaMemcpyDeviceToHost, s), "loss"));
    UN_TRY(n->cuda(cudaStreamSynchronize(s), "backward"));
    double sum = 0.0;
    for (double v : part) sum += v;
    *loss = sum / (double)(c0 * D);
    return PF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Internal entry points used by the field library (learned warm start)
// ---------------------------------------------------------------------------
UWork *unet_work_create(pf_unet *n, int nb, int nx, int ny, int nz)
{
    if (check_dims(n, nb, nx, ny, nz) != PF_OK) return nullptr;
    UWork *w = new (std::nothrow) UWork();
    if (!w) return nullptr;
    if (ensure_work(n, w, nb, nx, ny, nz, false) != PF_OK) {
        w->release();
        delete w;
        return nullptr;
    }
    return w;
}

void unet_work_destroy(UWork *w)
{
    if (!w) return;
    w->release();
    delete w;
}

int unet_forward_work(pf_unet *n, UWork *w, const float *in, const float **out, cudaStream_t s)
{
    UN_TRY(n->cfg.ndim == 2 ? forward_t<2>(n, w, in, s) : forward_t<3>(n, w, in, s));
    *out = w->y;
    return PF_OK;
}

int unet_ndim(const pf_unet *n) { return n->cfg.ndim; }
int unet_cin(const pf_unet *n) { return n->cfg.cin; }
int unet_check_grid(pf_unet *n, int nx, int ny, int nz) { return check_dims(n, 1, nx, ny, nz); }
const char *unet_error(const pf_unet *n) { return n->err.c_str(); }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int pf_unet_create(const pf_unet_config *cfg, pf_unet **out)
{
    if (!out) return PF_EINVAL;
    *out = nullptr;
    g_unet_create_error.clear();
    if (!cfg) { g_unet_create_error = "cfg is NULL"; return PF_EINVAL; }
    const pf_unet_config c = *cfg;
    if (c.ndim != 2 && c.ndim != 3) { g_unet_create_error = "ndim must be 2 or 3"; return PF_EINVAL; }
    if (c.cin < 1 || c.cin > 16) { g_unet_create_error = "cin must be 1..16"; return PF_EINVAL; }
    if (c.levels < 1 || c.levels > 5) { g_unet_create_error = "levels must be 1..5"; return PF_EINVAL; }
    for (int l = 0; l < c.levels; l++)
        if (c.channels[l] < 16 || c.channels[l] > 64 || c.channels[l] % 16) {
            g_unet_create_error = "channels must be 16, 32, 48 or 64";
            return PF_EINVAL;
        }
    pf_unet *n = new (std::nothrow) pf_unet();
    if (!n) { g_unet_create_error = "host allocation failed"; return PF_ENOMEM; }
    n->cfg = c;
    const int taps = c.ndim == 3 ? 27 : 9;
    const int L = c.levels;
    auto add = [&](int ci, int co, int t) {
        ConvLayer lay;
        lay.ci = ci;
        lay.cip = t == 1 ? ci : (ci < 16 ? 16 : ci);
        lay.co = co;
        lay.taps = t;
        lay.woff = n->nparam;
        n->nparam += (long long)ci * co * t;
        lay.boff = n->nparam;
        n->nparam += co;
        n->layers.push_back(lay);
    };
    int prev = c.cin;
    for (int l = 0; l < L; l++) {
        add(prev, c.channels[l], taps);
        add(c.channels[l], c.channels[l], taps);
        prev = c.channels[l];
    }
    for (int l = L - 2; l >= 0; l--) {
        add(c.channels[l] + c.channels[l + 1], c.channels[l], taps);
        add(c.channels[l], c.channels[l], taps);
    }
    add(c.channels[0], c.ndim, 1);
    int rc = PF_OK;
    auto A = [&](auto **p, size_t b) { if (rc == PF_OK) rc = n->alloc(p, b, n->allocs); };
    A(&n->params, sizeof(float) * n->nparam);
    A(&n->grad, sizeof(float) * n->nparam);
    A(&n->m, sizeof(float) * n->nparam);
    A(&n->v, sizeof(float) * n->nparam);
    A(&n->part, sizeof(double) * 152 * 32);
    for (ConvLayer &lay : n->layers) {
        if (lay.taps == 1) continue;
        A(&lay.wf, sizeof(__nv_bfloat16) * lay.taps * lay.co * lay.cip);
        A(&lay.wb, sizeof(__nv_bfloat16) * lay.taps * lay.co * lay.cip);
        A(&lay.gk, sizeof(float) * lay.taps * lay.co * lay.cip);
    }
    if (rc == PF_OK && !(c.ndim == 2 ? prepare_kernels<2>() : prepare_kernels<3>())) rc = n->fail(PF_ECUDA, "kernel attributes");
    if (rc == PF_OK) rc = n->cuda(cudaMemset(n->params, 0, sizeof(float) * n->nparam), "init");
    if (rc == PF_OK) rc = n->cuda(cudaMemset(n->m, 0, sizeof(float) * n->nparam), "init");
    if (rc == PF_OK) rc = n->cuda(cudaMemset(n->v, 0, sizeof(float) * n->nparam), "init");
    if (rc == PF_OK) rc = upload_weights(n, 0);
    if (rc == PF_OK) rc = n->cuda(cudaDeviceSynchronize(), "init");
    if (rc != PF_OK) {
        g_unet_create_error = n->err;
        pf_unet_destroy(n);
        return rc;
    }
    *out = n;
    return PF_OK;
}

long long pf_unet_param_count(const pf_unet *n) { return n ? n->nparam : 0; }

int pf_unet_set_loss(pf_unet *n, int kind, int weight_channel, double floor)
{
    if (!n) return PF_EINVAL;
    if (kind != PF_UNET_LOSS_MSE && kind != PF_UNET_LOSS_GRAD) return n->fail(PF_EINVAL, "unknown loss kind %d", kind);
    if (weight_channel < 0 || weight_channel >= n->cfg.cin) return n->fail(PF_EINVAL, "weight channel out of range");
    if (!(floor >= 0.0 && floor <= 1.0)) return n->fail(PF_EINVAL, "floor must be in [0, 1]");
    n->loss_kind = kind;
    n->loss_wch = weight_channel;
    n->loss_floor = (float)floor;
    return PF_OK;
}

int pf_unet_set_params(pf_unet *n, const float *host)
{
    if (!n || !host) return PF_EINVAL;
    UN_TRY(n->cuda(cudaMemcpy(n->params, host, sizeof(float) * n->nparam, cudaMemcpyHostToDevice), "params"));
    UN_TRY(n->cuda(cudaMemset(n->m, 0, sizeof(float) * n->nparam), "adam"));
    UN_TRY(n->cuda(cudaMemset(n->v, 0, sizeof(float) * n->nparam), "adam"));
    n->adam_t = 0;
    UN_TRY(upload_weights(n, 0));
    return n->cuda(cudaDeviceSynchronize(), "params");
}

int pf_unet_get_params(pf_unet *n, float *host)
{
    if (!n || !host) return PF_EINVAL;
    return n->cuda(cudaMemcpy(host, n->params, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost), "params");
}

int pf_unet_forward(pf_unet *n, const float *in, float *out, int nb, int nx, int ny, int nz, void *stream)
{
    if (!n || !in || !out) return PF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    UWork *w = &n->train;
    UN_TRY(check_dims(n, nb, nx, ny, nz));
    UN_TRY(ensure_work(n, w, nb, nx, ny, nz, false));
    UN_TRY(n->cfg.ndim == 2 ? forward_t<2>(n, w, in, s) : forward_t<3>(n, w, in, s));
    const long long c0 = level_cells(n, w, 0) * nb;
    UN_TRY(n->cuda(cudaMemcpyAsync(out, w->y, sizeof(float) * c0 * n->cfg.ndim, cudaMemcpyDeviceToDevice, s), "output"));
    return n->cuda(cudaStreamSynchronize(s), "forward");
}

int pf_unet_loss_grad(pf_unet *n, const float *in, const float *target, int nb, int nx, int ny, int nz,
                      double *loss, float *grad_host, void *stream)
{
    if (!n || !in || !target || !loss) return PF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    UN_TRY(check_dims(n, nb, nx, ny, nz));
    UWork *w = &n->train;
    UN_TRY(ensure_work(n, w, nb, nx, ny, nz, true));
    UN_TRY(n->cfg.ndim == 2 ? forward_t<2>(n, w, in, s) : forward_t<3>(n, w, in, s));
    UN_TRY(n->cfg.ndim == 2 ? backward_t<2>(n, w, in, target, loss, s) : backward_t<3>(n, w, in, target, loss, s));
    if (grad_host)
        UN_TRY(n->cuda(cudaMemcpy(grad_host, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost), "grad"));
    return PF_OK;
}

int pf_unet_adam_step(pf_unet *n, double lr, void *stream)
{
    if (!n) return PF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    n->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->adam_t)), c2 = (float)(1.0 - std::pow(0.999, (double)n->adam_t));
    k_adam<<<blocks_for(n->nparam), 256, 0, s>>>(n->nparam, n->params, n->grad, n->m, n->v, (float)lr, b1, b2, 1e-8f, c1, c2);
    UN_TRY(upload_weights(n, s));
    return n->cuda(cudaGetLastError(), "adam");
}

const char *pf_unet_last_error(const pf_unet *n)
{
    if (!n) return g_unet_create_error.c_str();
    return n->err.c_str();
}

void pf_unet_destroy(pf_unet *n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    n->train.release();
    for (void *p : n->allocs) cudaFree(p);
    delete n;
}

}  // extern "C"
