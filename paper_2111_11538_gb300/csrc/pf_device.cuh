// Device code of the coupled phase-field step (sm_103a).
//
// Storage: structure of arrays, row-major with x fastest (cell / node index
// i + nx*(j + ny*k)); node n is the lower corner of cell n.  T is the storage
// and arithmetic type of the fields (double for the plain FP64 method, float
// for the mixed method); reductions are carried in FP64 (per thread with
// compensated FP32 sums in the mixed method, then FP64 across threads).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pfdev {

constexpr int PSTRIDE = 24;       // doubles per block in a partials array
// Sync words, each on its own 128-byte line so that blocks polling the
// barrier generation do not contend with the arrival counter.
constexpr int SYNC_GEN = 32, SYNC_LAST = 64, SYNC_WORDS = 96;

// ---------------------------------------------------------------------------
// Parameters (by value to every kernel)
// ---------------------------------------------------------------------------
struct Params {
    int ndim, nx, ny, nz;
    long long N;
    double dt, c, w, eps, kappa, L;
    double DOs, DOg, DHs, DHg, DWs, DWg;
    double kfor, xHbc;
    double Ks, Gs, Kg, Gg;          // solid / gas bulk and shear moduli
    double eig0, sY, Hh, prestress;
    int plasticity;
};

// Element tables (Q1 unit square / cube, exact 2^d-point Gauss integration),
// written once per device by the host.
//   K?2: 8x8 (2D), K?3: 24x24 (3D), dof index = node*d + comp
//   Bb?: average shape-function gradient over the element, [node][axis]
//   Kdiag: the (equal) diagonal entries of K_lambda and K_mu
// Each table exists in double and float so that no FP64 -> FP32 conversion
// sits in the FP32 inner loops.
template <typename T> struct Tab {
    T Kl2[64], Km2[64], Kl3[576], Km3[576];
    T Bb2[8], Bb3[24];
    T Kdiag[4];   // [0],[1]: 2D lambda, mu; [2],[3]: 3D lambda, mu
};
// one copy per translation unit (no relocatable device code): every unit
// that launches kernels reading the tables uploads its own
static __constant__ Tab<double> cTabD;
static __constant__ Tab<float> cTabF;

template <typename T> __device__ __forceinline__ const Tab<T> &tab();
template <> __device__ __forceinline__ const Tab<double> &tab<double>() { return cTabD; }
template <> __device__ __forceinline__ const Tab<float> &tab<float>() { return cTabF; }

template <typename T, int D> __device__ __forceinline__ T Kl(int r, int c) { return D == 2 ? tab<T>().Kl2[r * 8 + c] : tab<T>().Kl3[r * 24 + c]; }
template <typename T, int D> __device__ __forceinline__ T Km(int r, int c) { return D == 2 ? tab<T>().Km2[r * 8 + c] : tab<T>().Km3[r * 24 + c]; }
template <typename T, int D> __device__ __forceinline__ T Bb(int a, int k) { return D == 2 ? tab<T>().Bb2[a * 2 + k] : tab<T>().Bb3[a * 3 + k]; }
template <typename T, int D> __device__ __forceinline__ T KdL() { return D == 2 ? tab<T>().Kdiag[0] : tab<T>().Kdiag[2]; }
template <typename T, int D> __device__ __forceinline__ T KdM() { return D == 2 ? tab<T>().Kdiag[1] : tab<T>().Kdiag[3]; }

template <int D> struct Dims { static constexpr int NV = D == 2 ? 3 : 6; static constexpr int NP = D == 2 ? 4 : 6; static constexpr int NN = 1 << D; };

// ---------------------------------------------------------------------------
// Scalars of one mechanics solve, in device memory
// ---------------------------------------------------------------------------
struct Scalars {
    double E[6];          // mean strain (Voigt, engineering shears) = Ebar
    double relres;        // final ||r|| / ||b||
    double bnorm;
    int iters;
    int status;           // PF_* code set by device code (0 = ok)
    int pad[2];
};

struct Diag {
    double sumO, sumH, sumW;
    double removedW, suppliedH;
    long long cg_total;
    int cg_last, cg_max;
    int status;
    int pad;
    double sumO_prev;       // sum of x_O before the last update (reduction rate)
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T ldg_(const T *p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ T ldcg_(const T *p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread accumulator: plain FP64 for double, compensated FP32 (sum and
// error term kept separately, product errors from fma) for float.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void addprod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add_plain(double x) { s += x; }
    __device__ __forceinline__ void fma_plain(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float t = s + x;
        float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ void addprod(float a, float b)
    {
        float p = a * b;
        float e = fmaf(a, b, -p);
        add(p);
        c += e;
    }
    // uncompensated: for the few terms one thread sums before the
    // compensated block and grid reductions take over
    __device__ __forceinline__ void add_plain(float x) { s += x; }
    __device__ __forceinline__ void fma_plain(float a, float b) { s = fmaf(a, b, s); }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Block-wide sum of K values; thread 0 writes them to dst[0..K).
template <int K>
__device__ void block_sum_store(double (&v)[K], double *dst)
{
    __shared__ double sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) sh[k][wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = lane < nw ? sh[k][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) dst[k] = s;
        }
    }
    __syncthreads();
}

// Sum of partials[b*PSTRIDE + k] over b < nb in a fixed order; every block
// that calls it gets bit-identical results.
template <int K>
__device__ void grid_sum(const double *partials, int nb, int off, double (&out)[K])
{
    __shared__ double res[K];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int b = lane; b < nb; b += 32) s += __ldcg(partials + (size_t)b * PSTRIDE + off + k);
            s = warp_sum(s);
            if (lane == 0) res[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) out[k] = res[k];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Block reduction of per-thread accumulators to one FP64 value per entry,
// written by thread 0 to dst.  FP32 accumulators are reduced as (sum, error)
// pairs with error-free additions, so no FP64 arithmetic runs per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_add(float &h, float &l, float h2, float l2)
{
    const float s = h + h2;
    const float bp = s - h;
    const float e = (h - (s - bp)) + (h2 - bp);
    l = l + l2 + e;
    h = s + l;
    l = l - (h - s);
}

template <int K>
__device__ void block_reduce_store(Acc<float> (&a)[K], double *dst)
{
    __shared__ float sh[K][32], sl[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        float h = a[k].s, l = a[k].c;
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
            pair_add(h, l, h2, l2);
        }
        if (lane == 0) { sh[k][wid] = h; sl[k][wid] = l; }
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            float h = lane < nw ? sh[k][lane] : 0.f, l = lane < nw ? sl[k][lane] : 0.f;
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
                pair_add(h, l, h2, l2);
            }
            if (lane == 0) dst[k] = (double)h + (double)l;
        }
    }
    __syncthreads();
}

template <int K>
__device__ void block_reduce_store(Acc<double> (&a)[K], double *dst)
{
    double v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[k].value();
    block_sum_store<K>(v, dst);
}

// FP32 path: the block's K sums as (hi, lo) float pairs, written by thread 0
// into the block's partials slot.
template <int K>
__device__ void block_reduce_pairs(Acc<float> (&a)[K], float2 *dst)
{
    __shared__ float sh[K][32], sl[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        float h = a[k].s, l = a[k].c;
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
            pair_add(h, l, h2, l2);
        }
        if (lane == 0) { sh[k][wid] = h; sl[k][wid] = l; }
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            float h = lane < nw ? sh[k][lane] : 0.f, l = lane < nw ? sl[k][lane] : 0.f;
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
                pair_add(h, l, h2, l2);
            }
            if (lane == 0) dst[k] = make_float2(h, l);
        }
    }
    __syncthreads();
}

// Last block: every thread loads the pairs of a fixed set of blocks (all
// loads independent), then a pair-arithmetic block tree; thread 0 publishes
// hi + lo in FP64.  The order depends only on indices.
template <int K>
__device__ void last_block_pairs(const double *partials, int nb, double *result)
{
    Acc<float> acc[K];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const float2 *src = reinterpret_cast<const float2 *>(partials + (size_t)b * PSTRIDE);
        float2 v[K];
#pragma unroll
        for (int k = 0; k < K; k++) v[k] = __ldcg(src + k);
#pragma unroll
        for (int k = 0; k < K; k++) pair_add(acc[k].s, acc[k].c, v[k].x, v[k].y);
    }
    __shared__ float2 tmp[K];
    block_reduce_pairs<K>(acc, tmp);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) result[k] = (double)tmp[k].x + (double)tmp[k].y;
    }
}

// FP64 path of the same: every thread sums a fixed set of blocks, then the
// block tree; thread 0 writes the totals to result.
template <int K>
__device__ void last_block_sums(const double *partials, int nb, double *result)
{
    double v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; k++) v[k] += __ldcg(partials + (size_t)b * PSTRIDE + k);
    }
    block_sum_store<K>(v, result);
}

// Asynchronous global -> shared copies of one element (cp.async): the
// thread goes on while the copy is in flight; commit groups the copies
// issued since the last commit, wait<n> blocks until at most n of the
// thread's groups are still pending (its own copies are then visible to
// it; other threads see them after a block barrier).
template <typename T>
__device__ __forceinline__ void cp_async(T *smem, const T *gmem)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// 16-byte copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// Bring the line holding p into the L1 cache (no register result): the
// operands of a later load whose latency would otherwise be exposed.  Data
// written by other blocks before a grid barrier may be cached this way: the
// barrier's acquire makes the writes visible to loads after it.
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }


// GPU-scope synchronisation primitives of the grid barrier: the arriving
// thread's acq_rel add publishes its block's partial sums and, for the last
// arrival, acquires every other block's; the last block's release add of the
// generation word publishes the totals; waiters acquire it.  (Each is one
// instruction; the fence-based protocol it replaces needed a full
// __threadfence around every atomic.)
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Bounded wait of one thread for a generation word to move past g: at most
// `limit` polls ~32 ns apart (plus the load latency); on expiry PF_ETIMEOUT
// (6) goes to *err and false is returned, so the kernel can leave with the
// context intact.  The grid barrier of the PCG and its self-test
// (pf_selftest_wait) use it.
constexpr long long SPIN_LIMIT = 1LL << 24;

__device__ __forceinline__ bool wait_generation(const unsigned int *gen, unsigned int g, int *err, long long limit)
{
    long long spins = 0;
    while (ld_acquire_gpu(gen) == g) {
        if (++spins > limit) {
            atomicExch(err, 6);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Model functions (Sec. 3.1 energies, R1 double well)
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T hfun(T x) { return x * x * x * (x * (T(6) * x - T(15)) + T(10)); }
template <typename T> __device__ __forceinline__ T hder(T x) { T y = x * (T(1) - x); return T(30) * y * y; }
template <typename T> __device__ __forceinline__ T mfun(T x) { T y = x * (T(1) - x); return y * y; }
template <typename T> __device__ __forceinline__ T mder(T x) { return T(2) * x * (T(1) - x) * (T(1) - T(2) * x); }

// CALPHAD polynomials and derivatives (scaled by V_mol / R theta).
template <typename T> __device__ __forceinline__ T f_fe(T x) { return (((T(163.708) * x - T(182.510)) * x + T(90.573)) * x - T(36.031)) * x - T(4.372); }
template <typename T> __device__ __forceinline__ T f_fe1(T x) { return ((T(654.832) * x - T(547.530)) * x + T(181.146)) * x - T(36.031); }
template <typename T> __device__ __forceinline__ T f_fe2(T x) { return (T(1964.496) * x - T(1095.060)) * x + T(181.146); }
template <typename T> __device__ __forceinline__ T f_wu(T x) { return (T(173.263) * x - T(213.460)) * x + T(41.953); }
template <typename T> __device__ __forceinline__ T f_wu1(T x) { return T(346.526) * x - T(213.460); }
template <typename T> __device__ __forceinline__ T f_wu2(T) { return T(346.526); }
template <typename T> __device__ __forceinline__ T f_ga(T x) { return T(1000) * x * x; }
template <typename T> __device__ __forceinline__ T f_ga1(T x) { return T(2000) * x; }
template <typename T> __device__ __forceinline__ T f_ga2(T) { return T(2000); }

// Phase weights W_f, W_w, W_g from theta and the fixed gas fraction.
template <typename T>
__device__ __forceinline__ void phase_weights(T th, T pg, T &Wf, T &Ww, T &Wg)
{
    T hg = hfun(pg), ht = hfun(th);
    T sol = T(1) - hg;
    Wf = sol * ht;
    Ww = sol - Wf;
    Wg = hg;
}

template <int D> __device__ __forceinline__ void cell_coords(const Params &P, long long n, int &i, int &j, int &k)
{
    i = (int)(n % P.nx);
    long long r = n / P.nx;
    j = (int)(r % P.ny);
    k = D == 3 ? (int)(r / P.ny) : 0;
}
__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
// periodic index for any a (tile halos of grids smaller than a tile)
__device__ __forceinline__ int wrapm(int a, int n) { int m = a % n; return m < 0 ? m + n : m; }
template <int D> __device__ __forceinline__ long long linm(const Params &P, int i, int j, int k)
{
    return (long long)wrapm(i, P.nx) + (long long)P.nx * ((long long)wrapm(j, P.ny) + (D == 3 ? (long long)P.ny * wrapm(k, P.nz) : 0LL));
}
template <int D> __device__ __forceinline__ long long lin(const Params &P, int i, int j, int k)
{
    return (long long)wrap(i, P.nx) + (long long)P.nx * ((long long)wrap(j, P.ny) + (D == 3 ? (long long)P.ny * wrap(k, P.nz) : 0LL));
}

// Isotropic stiffness in Voigt form (plane strain in-plane block in 2D).
template <typename T, int D>
__device__ __forceinline__ void voigt_stress(T lam, T mu, const T *e, T *s)
{
    if constexpr (D == 2) {
        T tr = e[0] + e[1];
        s[0] = lam * tr + T(2) * mu * e[0];
        s[1] = lam * tr + T(2) * mu * e[1];
        s[2] = mu * e[2];
    } else {
        T tr = e[0] + e[1] + e[2];
        s[0] = lam * tr + T(2) * mu * e[0];
        s[1] = lam * tr + T(2) * mu * e[1];
        s[2] = lam * tr + T(2) * mu * e[2];
        s[3] = mu * e[3]; s[4] = mu * e[4]; s[5] = mu * e[5];
    }
}

// Average (= centre) strain of an element from nodal values u[b][comp].
template <typename T, int D>
__device__ __forceinline__ void avg_strain(const T (*u)[D], T *e)
{
    T g[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int k = 0; k < D; k++) g[i][k] = T(0);
#pragma unroll
    for (int b = 0; b < (1 << D); b++)
#pragma unroll
        for (int k = 0; k < D; k++) {
            T bb = Bb<T, D>(b, k);
#pragma unroll
            for (int i = 0; i < D; i++) g[i][k] += bb * u[b][i];
        }
    if constexpr (D == 2) {
        e[0] = g[0][0]; e[1] = g[1][1]; e[2] = g[0][1] + g[1][0];
    } else {
        e[0] = g[0][0]; e[1] = g[1][1]; e[2] = g[2][2];
        e[3] = g[1][2] + g[2][1]; e[4] = g[0][2] + g[2][0]; e[5] = g[0][1] + g[1][0];
    }
}

// (Bbar_a^T s) for node a of an element with Voigt stress s.
template <typename T, int D>
__device__ __forceinline__ void bbar_t(int a, const T *s, T *out)
{
    T bx = Bb<T, D>(a, 0), by = Bb<T, D>(a, 1);
    if constexpr (D == 2) {
        out[0] = bx * s[0] + by * s[2];
        out[1] = by * s[1] + bx * s[2];
    } else {
        T bz = Bb<T, D>(a, 2);
        out[0] = bx * s[0] + by * s[5] + bz * s[4];
        out[1] = by * s[1] + bx * s[5] + bz * s[3];
        out[2] = bz * s[2] + by * s[3] + bx * s[4];
    }
}

} // namespace pfdev
