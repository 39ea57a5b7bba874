// Kernels of the warm-start network: a periodic 2D/3D U-Net whose 3^D
// convolutions run as implicit GEMMs on the BF16 tensor cores (FP32
// accumulation), with FP32 master weights and Adam.
//
// Activations are channels-last BF16: act[(b * cells + p) * C + c], p the
// x-fastest cell index of sample b.  Every channel count is a multiple of 16.
// A convolution's weights are staged as wt[tap][co][ci] (ci contiguous): the
// forward pass contracts over (tap, ci); the input-gradient pass uses the
// same kernel with the taps mirrored and ci/co exchanged.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace unet {

// Convolution tile: 8 rows of 16 cells.  2D: 8 y-rows; 3D: 2 z x 4 y rows.
template <int D> struct CTile;
template <> struct CTile<2> { static constexpr int X = 16, Y = 8, Z = 1; };
template <> struct CTile<3> { static constexpr int X = 16, Y = 4, Z = 2; };

struct Dims {
    int nx, ny, nz;      // grid of this level
    int nb;              // samples
};

__device__ __forceinline__ int wrapc(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1) : "r"(addr));
}

// D = A(16x16, row) * B(16x8, col) + D, BF16 operands, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
    const __nv_bfloat16 *in0;   // C0 channels at this level's resolution
    const __nv_bfloat16 *in1;   // C1 channels at half resolution (nearest up2), or null
    int C0, C1;
    const __nv_bfloat16 *wt;    // [taps][COUT][C0 + C1]
    const float *bias;          // [COUT] or null
    __nv_bfloat16 *out;         // [cells][COUT]
    int relu;
    int mirror;                 // 1: tap t reads the cell at -offset(t) (input-gradient pass)
    Dims dim;
};

// ---------------------------------------------------------------------------
// Periodic 3^D convolution as an implicit GEMM: out[p, co] = bias[co] +
// sum_{tap, ci} in[p + off(tap), ci] * W[tap, co, ci].  One block computes a
// tile of 128 cells x COUT channels; 8 warps, warp w owns the tile's row w
// (16 cells = one m16 fragment).  The K loop runs over 16-channel chunks of
// the input (staged with a one-cell halo) and over the taps.
// ---------------------------------------------------------------------------
template <int D, int COUT>
__host__ __device__ constexpr size_t conv3_smem()
{
    constexpr int HP = (CTile<D>::X + 2) * (CTile<D>::Y + 2) * (D == 3 ? CTile<D>::Z + 2 : 1);
    return sizeof(__nv_bfloat16) * 24 * (HP + (D == 3 ? 27 : 9) * COUT);
}

template <int D, int COUT>
__global__ void __launch_bounds__(256) k_conv3(const ConvArgs a)
{
    constexpr int TX = CTile<D>::X, TY = CTile<D>::Y, TZ = CTile<D>::Z;
    constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? TZ + 2 : 1;
    constexpr int HP = HX * HY * HZ;            // halo-tile cells
    constexpr int TAPS = D == 3 ? 27 : 9;
    constexpr int PS = 24;                      // bf16 per staged cell / weight row (16 + 8 pad)
    constexpr int NT = COUT / 8;                // n8 tiles
    static_assert(COUT % 16 == 0, "output channels come in pairs of n8 tiles");
    extern __shared__ __align__(16) unsigned char u_smem[];
    __nv_bfloat16 *s_in = (__nv_bfloat16 *)u_smem;          // [HP][PS]
    __nv_bfloat16 *s_w = s_in + HP * PS;                     // [TAPS * COUT][PS]

    const int nx = a.dim.nx, ny = a.dim.ny, nz = D == 3 ? a.dim.nz : 1;
    const int tx_n = nx / TX, ty_n = ny / TY, tz_n = nz / TZ;
    const long long cells = (long long)nx * ny * nz;
    const int Cin = a.C0 + a.C1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile
    long long t = blockIdx.x;
    const int tx = (int)(t % tx_n); t /= tx_n;
    const int ty = (int)(t % ty_n); t /= ty_n;
    const int tz = (int)(t % tz_n); t /= tz_n;
    const int b = (int)t;
    const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    const __nv_bfloat16 *in0 = a.in0 + (size_t)b * cells * a.C0;
    const long long cells1 = cells >> D;
    const __nv_bfloat16 *in1 = a.in1 ? a.in1 + (size_t)b * cells1 * a.C1 : nullptr;
    const int hx = nx >> 1, hy = ny >> 1;

    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    // this warp's row in the tile
    const int wy = warp % TY, wz = warp / TY;

    for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
        __syncthreads();
        // stage the input chunk: HP cells x 16 channels = 2 x 16 B per cell
        for (int q = threadIdx.x; q < HP * 2; q += blockDim.x) {
            const int cell = q >> 1, half = q & 1;
            const int hxi = cell % HX, r = cell / HX, hyi = r % HY, hzi = r / HY;
            const int gx = wrapc(x0 + hxi - 1, nx), gy = wrapc(y0 + hyi - 1, ny);
            const int gz = D == 3 ? wrapc(z0 + hzi - 1, nz) : 0;
            uint4 v;
            if (ci0 < a.C0) {
                const long long p = gx + (long long)nx * (gy + (long long)ny * gz);
                v = *(const uint4 *)(in0 + p * a.C0 + ci0 + half * 8);
            } else {
                const long long p = (gx >> 1) + (long long)hx * ((gy >> 1) + (long long)hy * (gz >> 1));
                v = *(const uint4 *)(in1 + p * a.C1 + (ci0 - a.C0) + half * 8);
            }
            *(uint4 *)(s_in + cell * PS + half * 8) = v;
        }
        // stage the weights of this chunk: [tap][co][16]
        for (int q = threadIdx.x; q < TAPS * COUT * 2; q += blockDim.x) {
            const int row = q >> 1, half = q & 1;
            const uint4 v = *(const uint4 *)(a.wt + (size_t)row * Cin + ci0 + half * 8);
            *(uint4 *)(s_w + row * PS + half * 8) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < TAPS; tap++) {
            int ox = tap % 3 - 1, oy = (tap / 3) % 3 - 1, oz = D == 3 ? tap / 9 - 1 : 0;
            if (a.mirror) { ox = -ox; oy = -oy; oz = -oz; }
            // A: 16 cells of this warp's row shifted by the tap, 16 channels
            const int m = lane & 15;                   // row of the A fragment (cell in the row)
            const int kh = lane >> 4;                  // which 8-channel half
            const int cell = (m + 1 + ox) + HX * ((wy + 1 + oy) + HY * (D == 3 ? wz + 1 + oz : 0));
            uint32_t a0, a1, a2, a3;
            ldsm_x4(smem_u32(s_in + cell * PS + kh * 8), a0, a1, a2, a3);
            // ldmatrix x4 order: lanes 0-7 rows 0-7 k0-7 (a0), 8-15 rows 8-15 k0-7 (a1),
            // 16-23 rows 0-7 k8-15 (a2), 24-31 rows 8-15 k8-15 (a3)
#pragma unroll
            for (int j = 0; j < NT; j += 2) {
                // B^T rows = output channels; lanes 0-7: n-tile j k0-7, 8-15: j k8-15,
                // 16-23: j+1 k0-7, 24-31: j+1 k8-15
                const int nn = (j + (lane >> 4)) * 8 + (lane & 7);
                const int kk = ((lane >> 3) & 1) * 8;
                uint32_t b0, b1, b2, b3;
                ldsm_x4(smem_u32(s_w + (tap * COUT + nn) * PS + kk), b0, b1, b2, b3);
                mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    // epilogue: bias, ReLU, BF16 store.  c0,c1: cell g, channels 2q,2q+1;
    // c2,c3: cell g+8.
    const int g = lane >> 2, qd = lane & 3;
    const int yy = y0 + wy, zz = z0 + wz;
    const long long rowbase = (long long)b * cells + (long long)nx * (yy + (long long)ny * zz) + x0;
#pragma unroll
    for (int j = 0; j < NT; j++) {
        const int co = j * 8 + qd * 2;
        float bb0 = a.bias ? a.bias[co] : 0.f, bb1 = a.bias ? a.bias[co + 1] : 0.f;
        float v0 = acc[j][0] + bb0, v1 = acc[j][1] + bb1, v2 = acc[j][2] + bb0, v3 = acc[j][3] + bb1;
        if (a.relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f); }
        __nv_bfloat162 lo = __floats2bfloat162_rn(v0, v1), hi = __floats2bfloat162_rn(v2, v3);
        *(__nv_bfloat162 *)(a.out + (rowbase + g) * COUT + co) = lo;
        *(__nv_bfloat162 *)(a.out + (rowbase + g + 8) * COUT + co) = hi;
    }
}

struct WGradArgs {
    const __nv_bfloat16 *in0, *in1;   // the forward input (as in ConvArgs)
    int C0, C1;
    const __nv_bfloat16 *gz;          // [cells][COUT] gradient at the pre-activation
    float *gw;                        // [taps][COUT][C0 + C1], accumulated (atomicAdd)
    Dims dim;
    long long ntiles;                 // tiles over all samples
};

// ---------------------------------------------------------------------------
// Weight gradient gW[tap, co, ci] = sum_p gz[p, co] * in[p + off(tap), ci]:
// a GEMM with M = co, N = ci (one 16-channel chunk per blockIdx.y), K = cells.
// A block walks tiles of 128 cells (K = 8 steps of 16 per tile), keeps its
// 9 (27) x COUT x 16 partial sums in registers and adds them to gW once.
// Work items (tap, m16 tile of co, n8 tile of ci) are dealt round-robin to
// the 8 warps.
// ---------------------------------------------------------------------------
// Items (tap, m16 tile of co, n8 tile of ci) per warp in one block; blocks
// along z take successive groups of 8 * PER items.
template <int D, int COUT>
__host__ __device__ constexpr int wgrad_per()
{
    constexpr int items = (D == 3 ? 27 : 9) * (COUT / 16) * 2;
    constexpr int per = (items + 7) / 8;
    return per < 12 ? per : 12;
}

template <int D, int COUT>
__host__ __device__ constexpr int wgrad_zsplit()
{
    constexpr int items = (D == 3 ? 27 : 9) * (COUT / 16) * 2;
    return (items + 8 * wgrad_per<D, COUT>() - 1) / (8 * wgrad_per<D, COUT>());
}

template <int D, int COUT>
__host__ __device__ constexpr size_t wgrad_smem()
{
    constexpr int HP = (CTile<D>::X + 2) * (CTile<D>::Y + 2) * (D == 3 ? CTile<D>::Z + 2 : 1);
    return sizeof(__nv_bfloat16) * (24 * HP + 128 * (COUT + 8));
}

template <int D, int COUT>
__global__ void __launch_bounds__(256) k_conv3_wgrad(const WGradArgs a)
{
    constexpr int TX = CTile<D>::X, TY = CTile<D>::Y, TZ = CTile<D>::Z;
    constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? TZ + 2 : 1;
    constexpr int HP = HX * HY * HZ;
    constexpr int TAPS = D == 3 ? 27 : 9;
    constexpr int PS = 24;
    constexpr int GS = COUT + 8;                         // bf16 per staged gz cell
    constexpr int ITEMS = TAPS * (COUT / 16) * 2;        // (tap, m-tile, n-tile)
    constexpr int PER = wgrad_per<D, COUT>();            // items per warp and block
    extern __shared__ __align__(16) unsigned char u_smem[];
    __nv_bfloat16 *s_in = (__nv_bfloat16 *)u_smem;                 // [HP][PS]
    __nv_bfloat16 *s_g = s_in + HP * PS;                            // [128][GS]
    const int item0 = blockIdx.z * 8 * PER;

    const int nx = a.dim.nx, ny = a.dim.ny, nz = D == 3 ? a.dim.nz : 1;
    const int tx_n = nx / TX, ty_n = ny / TY, tz_n = nz / TZ;
    const long long cells = (long long)nx * ny * nz;
    const long long cells1 = cells >> D;
    const int hx = nx >> 1, hy = ny >> 1;
    const int ci0 = blockIdx.y * 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float acc[PER][4];
#pragma unroll
    for (int i = 0; i < PER; i++) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;

    for (long long t0 = blockIdx.x; t0 < a.ntiles; t0 += gridDim.x) {
        long long t = t0;
        const int tx = (int)(t % tx_n); t /= tx_n;
        const int ty = (int)(t % ty_n); t /= ty_n;
        const int tz = (int)(t % tz_n); t /= tz_n;
        const int b = (int)t;
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        const __nv_bfloat16 *in0 = a.in0 + (size_t)b * cells * a.C0;
        const __nv_bfloat16 *in1 = a.in1 ? a.in1 + (size_t)b * cells1 * a.C1 : nullptr;
        __syncthreads();
        for (int q = threadIdx.x; q < HP * 2; q += blockDim.x) {
            const int cell = q >> 1, half = q & 1;
            const int hxi = cell % HX, r = cell / HX, hyi = r % HY, hzi = r / HY;
            const int gx = wrapc(x0 + hxi - 1, nx), gy = wrapc(y0 + hyi - 1, ny);
            const int gz = D == 3 ? wrapc(z0 + hzi - 1, nz) : 0;
            uint4 v;
            if (ci0 < a.C0) {
                const long long p = gx + (long long)nx * (gy + (long long)ny * gz);
                v = *(const uint4 *)(in0 + p * a.C0 + ci0 + half * 8);
            } else {
                const long long p = (gx >> 1) + (long long)hx * ((gy >> 1) + (long long)hy * (gz >> 1));
                v = *(const uint4 *)(in1 + p * a.C1 + (ci0 - a.C0) + half * 8);
            }
            *(uint4 *)(s_in + cell * PS + half * 8) = v;
        }
        // gz of the tile's 128 cells, in tile order (row-major: x, then y, z)
        for (int q = threadIdx.x; q < TX * TY * TZ * (COUT / 8); q += blockDim.x) {
            const int cell = q / (COUT / 8), part = q % (COUT / 8);
            const int cx = cell % TX, r = cell / TX, cy = r % TY, cz = r / TY;
            const long long p = (long long)b * cells + (x0 + cx) + (long long)nx * ((y0 + cy) + (long long)ny * (z0 + cz));
            *(uint4 *)(s_g + cell * GS + part * 8) = *(const uint4 *)(a.gz + p * COUT + part * 8);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int item = item0 + warp + i * 8;
            if (item >= ITEMS) break;
            const int nt = item & 1, mt = (item >> 1) % (COUT / 16), tap = (item >> 1) / (COUT / 16);
            const int ox = tap % 3 - 1, oy = (tap / 3) % 3 - 1, oz = D == 3 ? tap / 9 - 1 : 0;
#pragma unroll
            for (int ks = 0; ks < 8; ks++) {
                // K = 16 cells of tile row ks (cells ks*16 .. ks*16+15)
                // A[m = co][k = cell] = gz[cell][co]: transposed 8x8 loads from s_g
                // lanes 0-7: cells 0-7, co 0-7 (a0); 8-15: cells 0-7, co 8-15 (a1);
                // 16-23: cells 8-15, co 0-7 (a2); 24-31: cells 8-15, co 8-15 (a3)
                const int kc = ks * 16 + (lane & 7) + ((lane >> 4) & 1) * 8;
                const int cc = mt * 16 + ((lane >> 3) & 1) * 8;
                uint32_t a0, a1, a2, a3;
                ldsm_x4_t(smem_u32(s_g + kc * GS + cc), a0, a1, a2, a3);
                // B[k = cell][n = ci] = in[cell + off][ci]: transposed 8x8 loads from s_in
                // lanes 0-7: cells 0-7 (b0); 8-15: cells 8-15 (b1)
                const int kb = (lane & 7) + ((lane >> 3) & 1) * 8;     // cell within the 16
                const int wy = ks % TY, wz = ks / TY;
                const int hc = (kb + 1 + ox) + HX * ((wy + 1 + oy) + HY * (D == 3 ? wz + 1 + oz : 0));
                uint32_t b0, b1;
                ldsm_x2_t(smem_u32(s_in + hc * PS + nt * 8), b0, b1);
                mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // accumulate into gW: acc[i] c0,c1: co = mt*16 + g, ci = nt*8 + 2qd (+1); c2,c3: co + 8
    const int Cin = a.C0 + a.C1;
    const int g = lane >> 2, qd = lane & 3;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int item = item0 + warp + i * 8;
        if (item >= ITEMS) break;
        const int nt = item & 1, mt = (item >> 1) % (COUT / 16), tap = (item >> 1) / (COUT / 16);
        const int co = mt * 16 + g, ci = ci0 + nt * 8 + qd * 2;
        float *w = a.gw + ((size_t)tap * COUT + co) * Cin + ci;
        atomicAdd(w, acc[i][0]);
        atomicAdd(w + 1, acc[i][1]);
        atomicAdd(w + (size_t)8 * Cin, acc[i][2]);
        atomicAdd(w + (size_t)8 * Cin + 1, acc[i][3]);
    }
}

}  // namespace unet
