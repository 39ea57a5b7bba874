// Persistent Jacobi-PCG for the mechanics (K3/K4), one grid barrier per
// iteration.
//
// The iteration is the Chronopoulos-Gear form of preconditioned CG: with
// u = M^-1 r, w = A u, gamma = r.u, delta = w.u,
//     beta_i  = gamma_i / gamma_{i-1}
//     alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_{i-1})
//     p_i = u_i + beta_i p_{i-1},  s_i = w_i + beta_i s_{i-1}
//     x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i
// which produces the iterates of standard PCG but needs all its inner
// products at one point per iteration.  One sweep over node tiles does the
// vector updates, rebuilds u_{i+1} on the tile and its halo in shared memory
// from r_i, w_i, s_{i-1} (double-buffered in global memory), applies the Q1
// operator to it and accumulates gamma, delta and ||r||^2; the grid barrier
// then reduces those in a fixed order (the last block to arrive reduces).
//
// The few FP64 scalars of the iteration (alpha, beta, the mean-strain dofs)
// are computed by thread 0 of every block (identically, from the same
// reduced values) and broadcast through shared memory: FP64 runs at a small
// fraction of the FP32 rate on this GPU, so no other thread touches them.
#pragma once
#include <type_traits>

#include "pf_kernels.cuh"

namespace pfdev {

// Node tiles of the PCG sweep (one node per thread: the block has X*Y*Z
// threads); the shape is a launch option (pf_config.pcg_tile), picked per
// size class from measurements when left to the library.  The 32x16 tile
// runs one 512-thread block per SM: fewer blocks in each grid reduction and
// a smaller idle tail in the halo passes than two 256-thread blocks.
template <int D, int S> struct Tile;
template <> struct Tile<2, 0> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<2, 1> { static constexpr int X = 32, Y = 16, Z = 1; };
template <> struct Tile<3, 0> { static constexpr int X = 16, Y = 4, Z = 4; };
template <> struct Tile<3, 1> { static constexpr int X = 32, Y = 4, Z = 2; };
constexpr int PCG_SHAPES = 2;

template <typename T> struct MGHier;

template <typename T, int D>
struct PCGArgs {
    Params P;
    const T *lam, *mu;
    const T *sig[6];
    T *x[3], *p[3];
    T *r[2][3], *w[2][3], *s[2][3];
    T *dinv;                       // inverse of the Jacobi diagonal, written by the set-up
    T *u[3];                       // refinement mode: FP32 displacement written at the end
    double *x64[3];                // refinement mode: FP64 solution
    int refine;                    // 1: FP64 outer residual around the FP32 iteration
    double eta;                    // refinement mode: relative target of one FP32 pass
    double *partials;
    double *result;                // 32 doubles: [0,16) reductions, [24,30) FP64 mean strain
    unsigned int *bar_count, *bar_gen;
    Scalars *sc;
    Diag *dg;
    double rtol;
    int maxit;
    int warm;
    int block0, nblocks;           // this job's blocks in the launch
    const MGHier<T> *mg;           // multigrid hierarchy (2D, k_pcg<..., MG = true> only)
    double *b64[3];                // MG refinement mode: the FP64 right-hand side, kept from the
                                   // first pass for the later ones
};

// Grid barrier that also reduces K per-block values in a fixed order: the
// last block to arrive sums the partials (warp 0, lane-strided over blocks,
// then a butterfly) and publishes them before releasing the others.  After
// the call thread 0 holds the totals in out[].  Waits are bounded
// (SPIN_LIMIT polls, then PF_ETIMEOUT in *err and false is returned).
template <typename AccT, int K>
__device__ bool reduce_barrier(AccT (&acc)[K], double *partials, double *result, unsigned int *count,
                               unsigned int *gen, int *err, double (&out)[K], int bid, int nbk)
{
    constexpr bool pairs = std::is_same<AccT, Acc<float>>::value;
    __shared__ int s_last, s_ok;
    __shared__ unsigned int s_gen;
    if constexpr (pairs) block_reduce_pairs<K>(acc, reinterpret_cast<float2 *>(partials + (size_t)bid * PSTRIDE));
    else block_reduce_store<K>(acc, partials + (size_t)bid * PSTRIDE);
    if (threadIdx.x == 0) {
        s_ok = 1;
        s_gen = ld_relaxed_gpu(gen);
        const unsigned int arrived = atom_add_acq_rel_gpu(count, 1u);
        s_last = (arrived == (unsigned int)nbk - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last && pairs) {
        last_block_pairs<K>(partials, nbk, result);
        if (threadIdx.x == 0) {
            *count = 0u;
            red_add_release_gpu(gen, 1u);
        }
    } else if (s_last) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
#pragma unroll
            for (int k = 0; k < K; k++) {
                double sacc = 0.0;
                for (int b = lane; b < nbk; b += 32) sacc += __ldcg(partials + (size_t)b * PSTRIDE + k);
                sacc = warp_sum(sacc);
                if (lane == 0) result[k] = sacc;
            }
            if (lane == 0) {
                *count = 0u;
                red_add_release_gpu(gen, 1u);
            }
        }
    } else if (threadIdx.x == 0) {
        if (!wait_generation(gen, s_gen, err, SPIN_LIMIT)) s_ok = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) out[k] = __ldcg(result + k);
    }
    return s_ok != 0;
}

// q = sum over the 2^d cells around a node of (lam K_lam + mu K_mu) u_e, plus
// the mean-strain coupling B_a^T D_c UE, from shared-memory tiles.
// su: [D][HN] halo nodes, sl/sm: [HC] halo cells.  (lx, ly, lz): the node's
// halo-local coordinates.
template <typename T, int D, int HX, int HY, int CX, int CY>
__device__ __forceinline__ void apply_tile(const T *su, const T *sl, const T *sm, int HN, int lx, int ly, int lz,
                                           const T *ue, T (&q)[D], T (&eown)[Dims<D>::NV], T &lown, T &mown)
{
    constexpr int NN = Dims<D>::NN, NV = Dims<D>::NV;
#pragma unroll
    for (int d = 0; d < D; d++) q[d] = T(0);
#pragma unroll
    for (int a = 0; a < NN; a++) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = D == 3 ? (a >> 2) & 1 : 0;
        // Halo nodes and halo cells both start one before the tile, so the
        // cell whose lower corner is halo node (cx, cy, cz) has cell-local
        // coordinates (cx, cy, cz); cell a of this node has its lower corner
        // at the node minus bits(a).
        const int cx = lx - ax, cy = ly - ay, cz = lz - az;
        const int cl = cx + CX * (cy + CY * (D == 3 ? cz : 0));
        const T l = sl[cl], m = sm[cl];
        T ul[NN][D];
#pragma unroll
        for (int b = 0; b < NN; b++) {
            const int bx = b & 1, by = (b >> 1) & 1, bz = D == 3 ? (b >> 2) & 1 : 0;
            const int hn = (cx + bx) + HX * ((cy + by) + HY * (D == 3 ? cz + bz : 0));
#pragma unroll
            for (int d = 0; d < D; d++) ul[b][d] = su[d * HN + hn];
        }
#pragma unroll
        for (int co = 0; co < D; co++) {
            T acc = T(0);
#pragma unroll
            for (int b = 0; b < NN; b++)
#pragma unroll
                for (int cc = 0; cc < D; cc++)
                    acc += (l * Kl<T, D>(a * D + co, b * D + cc) + m * Km<T, D>(a * D + co, b * D + cc)) * ul[b][cc];
            q[co] += acc;
        }
        T se[NV], bt[D];
        voigt_stress<T, D>(l, m, ue, se);
        bbar_t<T, D>(a, se, bt);
#pragma unroll
        for (int d = 0; d < D; d++) q[d] += bt[d];
        if (a == 0) {
            avg_strain<T, D>(ul, eown);
            lown = l;
            mown = m;
        }
    }
}

// 2D Q1 element with constant moduli, exact form of its stiffness: writing
// the bilinear displacement of a unit cell as its average gradient G plus
// the hourglass mode h = u00 - u10 - u01 + u11 (per component), the strain is
// G + h * (eta - 1/2, xi - 1/2) terms whose cross products with G integrate
// to zero, so  K_e u = Bbar^T D eps(G) + (lam + 3 mu)/12 * gamma h  with
// gamma = (+1, -1, -1, +1) over the cell's nodes.  cell_force2 returns the
// average stress (without any mean strain) and the two hourglass forces.
template <typename TC>
__device__ __forceinline__ void cell_force2(TC l, TC m, const TC (&ue)[4][2], TC (&s)[3], TC (&fh)[2])
{
    const TC Gxu = TC(0.5) * ((ue[1][0] - ue[0][0]) + (ue[3][0] - ue[2][0]));
    const TC Gyu = TC(0.5) * ((ue[2][0] - ue[0][0]) + (ue[3][0] - ue[1][0]));
    const TC Gxv = TC(0.5) * ((ue[1][1] - ue[0][1]) + (ue[3][1] - ue[2][1]));
    const TC Gyv = TC(0.5) * ((ue[2][1] - ue[0][1]) + (ue[3][1] - ue[1][1]));
    const TC hu = (ue[0][0] - ue[1][0]) - (ue[2][0] - ue[3][0]);
    const TC hv = (ue[0][1] - ue[1][1]) - (ue[2][1] - ue[3][1]);
    const TC tr = Gxu + Gyv;
    s[0] = l * tr + TC(2) * m * Gxu;
    s[1] = l * tr + TC(2) * m * Gyv;
    s[2] = m * (Gyu + Gxv);
    const TC c = (l + TC(3) * m) * TC(1.0 / 12.0);
    fh[0] = c * hu;
    fh[1] = c * hv;
}

// force on the node with local index a of a 2D cell from its average stress
// s (mean strain included) and hourglass forces fh
template <typename TC>
__device__ __forceinline__ void node_force2(int a, const TC *s, const TC *fh, TC (&f)[2])
{
    const TC bx = (a & 1) ? TC(0.5) : TC(-0.5), by = (a >> 1) ? TC(0.5) : TC(-0.5);
    const TC g = (a == 0 || a == 3) ? TC(1) : TC(-1);
    f[0] = bx * s[0] + by * s[2] + g * fh[0];
    f[1] = by * s[1] + bx * s[2] + g * fh[1];
}

// 3D Q1 hex with constant moduli, exact form of its stiffness (the
// counterpart of the 2D decomposition): per displacement component the
// trilinear field of a unit cell is its mean, its average gradient G and the
// modes h1 = xi eta, h2 = eta zeta, h3 = zeta xi, h4 = xi eta zeta (centred
// coordinates).  2x2x2 Gauss integration of the strain energy splits into
// Bbar^T D eps(G) and a quadratic form in the twelve h coefficients whose
// gradient (with respect to h) gives the hourglass forces; the cross terms
// integrate to zero.  cell_force3 returns, in c[20]: the average stress
// (Voigt xx yy zz yz xz xy, without the mean strain) in c[0..5] and the
// forces g[k][comp] = dE/dh_k,comp in c[6 + 3k + comp]; c[18..19] pad.
template <typename TC>
__device__ __forceinline__ void cell_force3(TC l, TC m, const TC (&ue)[8][3], TC (&c)[20])
{
    TC G[3][3], h[4][3];     // G[comp][dir], h[mode][comp]
#pragma unroll
    for (int k = 0; k < 3; k++) {
        // node b = bx + 2 by + 4 bz; pairs along x
        const TC e00 = ue[0][k] + ue[1][k], d00 = ue[1][k] - ue[0][k];
        const TC e01 = ue[2][k] + ue[3][k], d01 = ue[3][k] - ue[2][k];
        const TC e10 = ue[4][k] + ue[5][k], d10 = ue[5][k] - ue[4][k];
        const TC e11 = ue[6][k] + ue[7][k], d11 = ue[7][k] - ue[6][k];
        G[k][0] = TC(0.25) * ((d00 + d01) + (d10 + d11));
        G[k][1] = TC(0.25) * ((e01 + e11) - (e00 + e10));
        G[k][2] = TC(0.25) * ((e10 + e11) - (e00 + e01));
        h[0][k] = TC(0.5) * ((d01 + d11) - (d00 + d10));     // sx sy
        h[1][k] = TC(0.5) * ((e11 - e10) - (e01 - e00));     // sy sz
        h[2][k] = TC(0.5) * ((d10 + d11) - (d00 + d01));     // sz sx
        h[3][k] = (d11 - d10) - (d01 - d00);                 // sx sy sz
    }
    const TC tr = G[0][0] + G[1][1] + G[2][2];
    c[0] = l * tr + TC(2) * m * G[0][0];
    c[1] = l * tr + TC(2) * m * G[1][1];
    c[2] = l * tr + TC(2) * m * G[2][2];
    c[3] = m * (G[1][2] + G[2][1]);
    c[4] = m * (G[0][2] + G[2][0]);
    c[5] = m * (G[0][1] + G[1][0]);
    const TC A = h[0][1] + h[2][2], B = h[0][0] + h[1][2], C = h[2][0] + h[1][1];
    const TC Pq = h[1][0] + h[2][1], Q = h[2][1] + h[0][2], R = h[0][2] + h[1][0];
    const TC c12 = TC(1.0 / 12.0), m3 = TC(3) * m, c144 = (l + TC(4) * m) * TC(1.0 / 144.0);
    c[6] = (l * B + m3 * h[0][0]) * c12;       // mode 1, x
    c[7] = (l * A + m3 * h[0][1]) * c12;       // mode 1, y
    c[8] = m * (Q + R) * c12;                  // mode 1, z
    c[9] = m * (Pq + R) * c12;                 // mode 2, x
    c[10] = (l * C + m3 * h[1][1]) * c12;      // mode 2, y
    c[11] = (l * B + m3 * h[1][2]) * c12;      // mode 2, z
    c[12] = (l * C + m3 * h[2][0]) * c12;      // mode 3, x
    c[13] = m * (Pq + Q) * c12;                // mode 3, y
    c[14] = (l * A + m3 * h[2][2]) * c12;      // mode 3, z
    c[15] = c144 * h[3][0];
    c[16] = c144 * h[3][1];
    c[17] = c144 * h[3][2];
    c[18] = TC(0);
    c[19] = TC(0);
}

// force on the node at corner (ax, ay, az) of a 3D cell from its average
// stress s (mean strain included) and hourglass forces g = c + 6
template <typename TC>
__device__ __forceinline__ void node_force3(int ax, int ay, int az, const TC *s, const TC *g, TC (&f)[3])
{
    const TC sx = ax ? TC(1) : TC(-1), sy = ay ? TC(1) : TC(-1), sz = az ? TC(1) : TC(-1);
    const TC w1 = TC(0.5) * sx * sy, w2 = TC(0.5) * sy * sz, w3 = TC(0.5) * sz * sx, w4 = sx * sy * sz;
    f[0] = TC(0.25) * (sx * s[0] + sy * s[5] + sz * s[4]) + w1 * g[0] + w2 * g[3] + w3 * g[6] + w4 * g[9];
    f[1] = TC(0.25) * (sy * s[1] + sx * s[5] + sz * s[3]) + w1 * g[1] + w2 * g[4] + w3 * g[7] + w4 * g[10];
    f[2] = TC(0.25) * (sz * s[2] + sy * s[3] + sx * s[4]) + w1 * g[2] + w2 * g[5] + w3 * g[8] + w4 * g[11];
}

// Per-node part of the solve's set-up: right-hand side b = sum_e Bbar^T sig*,
// Jacobi diagonal, A x (element tables + mean-strain coupling XE) and the own
// cell's quantities.  TC is the arithmetic type, TV the type of x.
template <typename T, typename TC, typename TV, int D>
__device__ __forceinline__ void node_setup(const Params &P, long long n, const T *lam, const T *mu, const T *const *sig,
                                           TV *const *x, const TC *XE, bool use_x, TC (&b)[D], TC (&ax)[D], TC &dgn,
                                           TC (&sig_own)[Dims<D>::NV], TC (&de_own)[Dims<D>::NV], TC &l_own, TC &m_own)
{
    constexpr int NN = Dims<D>::NN, NV = Dims<D>::NV;
    int i, j, k;
    cell_coords<D>(P, n, i, j, k);
#pragma unroll
    for (int d = 0; d < D; d++) { b[d] = TC(0); ax[d] = TC(0); }
#pragma unroll
    for (int v = 0; v < NV; v++) de_own[v] = TC(0);
    dgn = TC(0);
#pragma unroll
    for (int a = 0; a < NN; a++) {
        const int ox = a & 1, oy = (a >> 1) & 1, oz = D == 3 ? (a >> 2) & 1 : 0;
        const int ci = i - ox, cj = j - oy, ck = k - oz;
        const long long c = lin<D>(P, ci, cj, ck);
        const TC l = (TC)lam[c], m = (TC)mu[c];
        dgn += l * KdL<TC, D>() + m * KdM<TC, D>();
        TC s[NV], bt[D];
#pragma unroll
        for (int v = 0; v < NV; v++) s[v] = (TC)sig[v][c];
        bbar_t<TC, D>(a, s, bt);
#pragma unroll
        for (int d = 0; d < D; d++) b[d] += bt[d];
        if (a == 0) {
#pragma unroll
            for (int v = 0; v < NV; v++) sig_own[v] = s[v];
            l_own = l;
            m_own = m;
        }
        if (use_x) {
            TC ue[NN][D];
#pragma unroll
            for (int bn = 0; bn < NN; bn++) {
                const int px = bn & 1, py = (bn >> 1) & 1, pz = D == 3 ? (bn >> 2) & 1 : 0;
                const long long mm = lin<D>(P, ci + px, cj + py, ck + pz);
#pragma unroll
                for (int d = 0; d < D; d++) ue[bn][d] = (TC)__ldcg(x[d] + mm);
            }
            if constexpr (D == 2) {
                TC s3[3], fh[2], sx[3], f[2];
                cell_force2<TC>(l, m, ue, s3, fh);
                if (a == 0)
#pragma unroll
                    for (int v = 0; v < 3; v++) de_own[v] = s3[v];
                voigt_stress<TC, 2>(l, m, XE, sx);
#pragma unroll
                for (int v = 0; v < 3; v++) s3[v] += sx[v];
                node_force2<TC>(a, s3, fh, f);
                ax[0] += f[0];
                ax[1] += f[1];
            } else {
                // the exact hex decomposition: average stress (plus the mean
                // strain) and hourglass forces of the cell, force on this node
                TC c[20], sx[6], f[3];
                cell_force3<TC>(l, m, ue, c);
                if (a == 0)
#pragma unroll
                    for (int v = 0; v < 6; v++) de_own[v] = c[v];
                voigt_stress<TC, 3>(l, m, XE, sx);
#pragma unroll
                for (int v = 0; v < 6; v++) c[v] += sx[v];
                node_force3<TC>(ox, oy, oz, c, c + 6, f);
#pragma unroll
                for (int d = 0; d < 3; d++) ax[d] += f[d];
            }
        }
    }
}

// Periodic 32-bit index of a tile-halo position.  Halo coordinates lie in
// [-1, n - 1 + tile], so one conditional wrap per axis suffices unless the
// grid is not larger than a tile (small), where a modulo is used.
template <int D>
__device__ __forceinline__ int hidx(const Params &P, int x, int y, int z, bool small)
{
    if (small) return (int)linm<D>(P, x, y, z);
    x += (x < 0) ? P.nx : 0;
    x -= (x >= P.nx) ? P.nx : 0;
    y += (y < 0) ? P.ny : 0;
    y -= (y >= P.ny) ? P.ny : 0;
    if constexpr (D == 3) {
        z += (z < 0) ? P.nz : 0;
        z -= (z >= P.nz) ? P.nz : 0;
        return x + P.nx * (y + P.ny * z);
    }
    return x + P.nx * y;
}

// FP64 state of the iteration, in shared memory and touched only by thread 0
// (so it costs the other threads no registers).
struct PCGState {
    double XE[6];      // mean strain of x (plain) / of the correction (refine)
    double E64[6];     // FP64 mean strain of the solution (refine)
    double DiagE[6], invDiagE[6], RE[6], UE[6], PE[6], SE[6], WE[6];
    double Sl, Sm, bnorm, rho_final, target, prev_res;
    double gamma, delta, gamma_prev, alpha_prev, alpha, beta;
    double inv_gamma, inv_gamma_prev, inv_alpha, inv_alpha_prev;   // FP64 divisions are slow here
    double tot0[10];   // first pass's set-up sums [0, 10) (fixed during a solve; MG refinement reuses them)
    int it, it_total, conv;
};

// Scalar part of one CG update, thread 0 only: beta and alpha from gamma and
// delta (one division here, 1/alpha = den / gamma reusing 1/gamma, and one
// for 1/gamma after the reduction), then the mean-strain dofs' p, s, x, r
// and their Jacobi-preconditioned u.
template <int NV>
__device__ __forceinline__ void cg_scalar_update(PCGState &S)
{
    S.beta = (S.it == 0) ? 0.0 : S.gamma * S.inv_gamma_prev;
    const double den = (S.it == 0) ? S.delta : S.delta - S.beta * S.gamma * S.inv_alpha_prev;
    S.alpha = S.gamma / den;
    S.inv_alpha = den * S.inv_gamma;
    for (int vv = 0; vv < NV; vv++) {
        S.PE[vv] = S.UE[vv] + S.beta * S.PE[vv];
        S.SE[vv] = S.WE[vv] + S.beta * S.SE[vv];
        S.XE[vv] += S.alpha * S.PE[vv];
        S.RE[vv] -= S.alpha * S.SE[vv];
        S.UE[vv] = S.RE[vv] * S.invDiagE[vv];
    }
}

// Thread 0 after the reduction of gamma and delta: shift the previous
// iteration's values (not on the first sweep of a pass).
__device__ __forceinline__ void cg_take_gamma_delta(PCGState &S, double gnew, double dnew, bool first)
{
    if (!first) {
        S.gamma_prev = S.gamma;
        S.alpha_prev = S.alpha;
        S.inv_gamma_prev = S.inv_gamma;
        S.inv_alpha_prev = S.inv_alpha;
    }
    S.gamma = gnew;
    S.delta = dnew;
    S.inv_gamma = 1.0 / gnew;
}

// Control words broadcast by thread 0.
enum { CTL_RUN = 0, CTL_DONE = 1, CTL_ZERO = 2, CTL_STOP = 3 };

}  // namespace pfdev

#include "pf_mg.cuh"
#include "pf_mg3.cuh"

namespace pfdev {

// The solve.  Plain mode (refine = 0): x = A.x (the displacement itself).
// Refinement mode (FP32 storage): the solution is kept in FP64 (A.x64 and the
// FP64 mean strain); every outer pass forms the true residual b - A x64 in
// FP64, solves for a correction with the FP32 iteration (A.x holds the
// correction), adds it in FP64, and stops when the FP64 residual meets rtol;
// the FP32 displacement A.u is written from x64 at the end.
template <int D, int S>
constexpr int tile_threads() { return Tile<D, S>::X * Tile<D, S>::Y * Tile<D, S>::Z; }

template <typename T, int D, int SH, bool MG>
__global__ void __launch_bounds__(tile_threads<D, SH>(), 512 / tile_threads<D, SH>()) k_pcg(const PCGArgs<T, D> *jobs, int njobs)
{
    // this block's job, copied to shared memory
    __shared__ PCGArgs<T, D> sA;
    {
        const PCGArgs<T, D> *J = my_job(jobs, njobs);
        const int *src = reinterpret_cast<const int *>(J);
        int *dst = reinterpret_cast<int *>(&sA);
        for (int i = threadIdx.x; i < (int)(sizeof(PCGArgs<T, D>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    const PCGArgs<T, D> &A = sA;
    const int bid = (int)blockIdx.x - A.block0, nbk = A.nblocks;
    constexpr int NV = Dims<D>::NV;
    constexpr int TX = Tile<D, SH>::X, TY = Tile<D, SH>::Y, TZ = Tile<D, SH>::Z;
    constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? TZ + 2 : 1;
    constexpr int CX = TX + 1, CY = TY + 1, CZ = D == 3 ? TZ + 1 : 1;
    constexpr int HN = HX * HY * HZ, HC = CX * CY * CZ;
    constexpr int MAX_OUTER = 24;
    // the node and cell tiles of the plain sweep (the 3D multigrid variant
    // keeps its tiles in the dynamic shared memory)
    constexpr bool Z3 = MG && D == 3;
    __shared__ T su[Z3 ? 1 : D * HN];
    __shared__ T sl[Z3 ? 1 : HC], sm[Z3 ? 1 : HC];
    // per-cell stress and hourglass forces: 2D 5 values per cell; 3D FP32 on
    // the 16x4x4 tile 20 (five float4); other 3D variants use the
    // element-matrix path and need none
    constexpr bool CELL3 = D == 3 && sizeof(T) == 4 && SH == 0;
    __shared__ __align__(16) T scell2[D == 2 ? 5 * HC : 1];
    extern __shared__ __align__(16) unsigned char pcg_dyn[];   // CELL3: 20 * HC floats; MG: block-run levels
    T *scell = CELL3 ? reinterpret_cast<T *>(pcg_dyn) : scell2;
    __shared__ T s_ta, s_tb, s_ue[6], s_xe[6];
    __shared__ int s_ctl;

    const Params &P = A.P;
    const long long N = P.N;
    int *err = &A.sc->status;
    const int ntx = (P.nx + TX - 1) / TX, nty = (P.ny + TY - 1) / TY, ntz = D == 3 ? (P.nz + TZ - 1) / TZ : 1;
    const int ntiles = ntx * nty * ntz;
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = D == 3 ? threadIdx.x / (TX * TY) : 0;
    const long long t0 = bid * (long long)blockDim.x + threadIdx.x;
    const long long st = (long long)nbk * blockDim.x;
    const bool refine = A.refine != 0;
    const bool lead = threadIdx.x == 0;
    const bool small = P.nx < TX + 2 || P.ny < TY + 2 || (D == 3 && P.nz < TZ + 2);

    __shared__ PCGState S;
    double *XE = S.XE, *E64 = S.E64, *DiagE = S.DiagE, *RE = S.RE, *UE = S.UE, *PE = S.PE, *SE = S.SE, *WE = S.WE;
    double &Sl = S.Sl, &Sm = S.Sm, &bnorm = S.bnorm, &rho_final = S.rho_final, &target = S.target;
    double &gamma = S.gamma, &delta = S.delta, &gamma_prev = S.gamma_prev, &alpha_prev = S.alpha_prev;
    double &alpha = S.alpha, &beta = S.beta;
    int &it = S.it, &it_total = S.it_total;
    bool conv = false;
    if (lead) {
        for (int v = 0; v < 6; v++) { XE[v] = 0.0; E64[v] = 0.0; }
        Sl = Sm = bnorm = rho_final = target = 0.0;
        gamma = delta = alpha = beta = 0.0;
        gamma_prev = alpha_prev = 1.0;
        S.inv_gamma = S.inv_gamma_prev = S.inv_alpha = S.inv_alpha_prev = 1.0;
        it = 0;
        it_total = 0;
        if (A.warm)
            for (int v = 0; v < NV; v++) (refine ? E64 : XE)[v] = A.sc->E[v];
    }

    // MG: the hierarchy descriptor (read only during the launch) stays in
    // global memory; the coarse levels' moduli are rebuilt for this solve
    // the block-run levels' arrays: dynamic shared memory (pcg_dyn_smem)
    T *sblk = reinterpret_cast<T *>(pcg_dyn);
    if constexpr (MG && D == 2) {
        if (!mg_setup<T>(*A.mg, A.bar_count, A.bar_gen, err, bid, nbk)) return;
    } else if constexpr (MG) {
        if (!mg_setup3<T>(*A.mg, A.bar_count, A.bar_gen, err, bid, nbk)) return;
    }

    for (int outer = 0; outer < (refine ? MAX_OUTER : 1); outer++) {
        // ---------------- set-up: r0 = b - A x0, diagonal, cell sums --------
        const bool use_x = refine ? (A.warm || outer > 0) : (A.warm != 0);
        if (lead)
            for (int v = 0; v < NV; v++) s_xe[v] = (T)(refine ? 0.0 : XE[v]);
        __syncthreads();
        {
            // every thread needs the mean strain of x for A x: FP64 from the
            // previous pass (refine) or the FP32 copy broadcast above
            double xe64[6];
            T xeT[6];
            for (int v = 0; v < NV; v++) {
                xe64[v] = outer == 0 ? (A.warm ? A.sc->E[v] : 0.0) : __ldcg(A.result + 24 + v);
                xeT[v] = s_xe[v];
            }
            Acc<double> acc[16];
            if constexpr (MG && D == 2) {
                // 2D multigrid variant: the tiled FP64 set-up (cells once per
                // tile) in the dynamic shared memory; later refinement passes
                // only form the residual
                setup_tiled<T, TX, TY>(A, use_x, refine, refine && outer > 0, xe64,
                                       reinterpret_cast<double *>(pcg_dyn), acc, bid, nbk);
            } else if constexpr (MG) {
                // 3D multigrid variant: the z-marching sweep in FP64
                setup_march3<T>(A, use_x, refine, refine && outer > 0, xe64, reinterpret_cast<double *>(pcg_dyn), acc,
                                bid, nbk);
            } else
            for (long long n = t0; n < N; n += st) {
                double bv[D], rv[D];
                if (refine) {
                    double b[D], ax[D], dgn, so[NV], deo[NV], lo, mo;
                    node_setup<T, double, double, D>(P, n, A.lam, A.mu, A.sig, A.x64, xe64, use_x, b, ax, dgn, so, deo, lo, mo);
                    A.dinv[n] = (T)(1.0 / dgn);
#pragma unroll
                    for (int d = 0; d < D; d++) { bv[d] = b[d]; rv[d] = b[d] - ax[d]; }
                    acc[2].add(lo); acc[3].add(mo);
#pragma unroll
                    for (int v = 0; v < NV; v++) { acc[4 + v].add(so[v]); acc[10 + v].add(deo[v]); }
                    if (!use_x)
#pragma unroll
                        for (int d = 0; d < D; d++) A.x64[d][n] = 0.0;
                } else {
                    T b[D], ax[D], dgn, so[NV], deo[NV], lo, mo;
                    node_setup<T, T, T, D>(P, n, A.lam, A.mu, A.sig, A.x, xeT, use_x, b, ax, dgn, so, deo, lo, mo);
                    A.dinv[n] = T(1) / dgn;
#pragma unroll
                    for (int d = 0; d < D; d++) { bv[d] = (double)b[d]; rv[d] = (double)(b[d] - ax[d]); }
                    acc[2].add((double)lo); acc[3].add((double)mo);
#pragma unroll
                    for (int v = 0; v < NV; v++) { acc[4 + v].add((double)so[v]); acc[10 + v].add((double)deo[v]); }
                }
#pragma unroll
                for (int d = 0; d < D; d++) {
                    if (refine || !use_x) A.x[d][n] = T(0);
                    A.p[d][n] = T(0);
                    A.s[0][d][n] = T(0);
                    A.r[0][d][n] = (T)rv[d];
                    acc[0].addprod(bv[d], bv[d]);
                    acc[1].addprod(rv[d], rv[d]);
                }
            }
            double tot[16];
            if (!reduce_barrier<Acc<double>, 16>(acc, A.partials, A.result, A.bar_count, A.bar_gen, err, tot, bid, nbk)) return;
            if (lead) {
                // a residual-only pass reuses the first pass's sums of b, the
                // moduli and the eigenstress
                if (MG && refine) {
                    if (outer == 0)
                        for (int k = 0; k < 10; k++) S.tot0[k] = tot[k];
                    else
                        for (int k = 0; k < 10; k++)
                            if (k != 1) tot[k] = S.tot0[k];
                }
                // scalars of the mean-strain dofs
                Sl = tot[2];
                Sm = tot[3];
                double AXE[6], unit[6], s6[6];
                for (int vv = 0; vv < NV; vv++) {
                    for (int w = 0; w < NV; w++) unit[w] = (w == vv) ? 1.0 : 0.0;
                    dmat_mul<D>(Sl, Sm, unit, s6);
                    DiagE[vv] = s6[vv];
                    S.invDiagE[vv] = 1.0 / s6[vv];
                }
                dmat_mul<D>(Sl, Sm, refine ? E64 : XE, AXE);
                double bbt = tot[0], rho = tot[1];
                for (int vv = 0; vv < NV; vv++) {
                    const double BE = tot[4 + vv] + (vv < D ? (double)N * (-P.prestress) : 0.0);
                    RE[vv] = BE - (use_x ? tot[10 + vv] + AXE[vv] : 0.0);
                    UE[vv] = RE[vv] * S.invDiagE[vv];
                    bbt += BE * BE;
                    rho += RE[vv] * RE[vv];
                    PE[vv] = 0.0;
                    SE[vv] = 0.0;
                    if (refine) XE[vv] = 0.0;
                }
                bnorm = sqrt(bbt);
                rho_final = rho;
                int ctl = CTL_RUN;
                if (bnorm == 0.0) ctl = CTL_ZERO;
                else if (sqrt(rho) <= A.rtol * bnorm) ctl = CTL_DONE;
                // refinement that no longer halves the FP64 residual has
                // reached what the FP32 passes can resolve: stop (not converged)
                else if (refine && outer > 0 && sqrt(rho) > 0.5 * S.prev_res) ctl = CTL_STOP;
                S.prev_res = sqrt(rho);
                // target of this pass: the requested tolerance, or in refinement
                // mode what an FP32 iteration can deliver on this correction
                // (eta); when the final tolerance is within a factor 100 of that,
                // the pass aims for it directly, which saves a pass that would
                // otherwise start just above the tolerance
                if (refine) {
                    const double fin = 0.5 * A.rtol * bnorm, pass = A.eta * sqrt(rho);
                    target = fin >= 0.01 * pass ? fin : pass;
                } else {
                    target = A.rtol * bnorm;
                }
                gamma = 0.0; delta = 0.0; gamma_prev = 1.0; alpha_prev = 1.0; alpha = 0.0; beta = 0.0;
                S.inv_gamma = S.inv_gamma_prev = S.inv_alpha = S.inv_alpha_prev = 1.0;
                it = 0;
                s_ctl = ctl;
            }
            __syncthreads();
        }
        const int ctl0 = s_ctl;
        if (ctl0 == CTL_ZERO) {
            for (long long n = t0; n < N; n += st)
                for (int d = 0; d < D; d++) {
                    A.x[d][n] = T(0);
                    if (refine) A.x64[d][n] = 0.0;
                }
            if (lead) {
                for (int vv = 0; vv < NV; vv++) { XE[vv] = 0.0; E64[vv] = 0.0; }
                rho_final = 0.0;
            }
            conv = true;
            break;
        }
        if (ctl0 == CTL_DONE) { conv = true; break; }
        if (ctl0 == CTL_STOP) { conv = false; break; }

        // ---------------- sweeps: the first builds w_0, then iterations -----
        if constexpr (MG) {
            int rc;
            if constexpr (D == 2)
                rc = mg_pass<T, TX, TY>(A, *A.mg, S, su, sl, sm, scell, sblk, s_ta, s_tb, s_ue, s_ctl, bid, nbk, err);
            else
                rc = mg_pass3<T>(A, *A.mg, S, reinterpret_cast<T *>(pcg_dyn), s_ta, s_tb, s_ue, s_ctl, bid, nbk, err);
            if (rc < 0) return;
            if (lead) conv = rc == CTL_DONE;
        } else {
            bool first = true;
            int cur = 0;
            while (true) {
                if (lead) {
                    if (!first) cg_scalar_update<NV>(S);
                    s_ta = (T)alpha;
                    s_tb = (T)beta;
                    for (int vv = 0; vv < NV; vv++) s_ue[vv] = (T)UE[vv];
                }
                __syncthreads();
                const T ta = s_ta, tb = s_tb;
                T ue[NV];
    #pragma unroll
                for (int vv = 0; vv < NV; vv++) ue[vv] = s_ue[vv];
                const int nxt = first ? cur : 1 - cur;
                Acc<T> acc[3 + NV];      // gamma, delta, ||r||^2, mean-strain row
                // Register double buffering across tiles: the loads of the next
                // tile's halo (r, w, s, diag), cells (lam, mu) and own node are
                // issued before the current tile is staged and computed, so their
                // latency overlaps that work.
                constexpr int NT = TX * TY * TZ;       // threads = tile nodes
                constexpr int HS = (HN + NT - 1) / NT, CS = (HC + NT - 1) / NT;
                struct Raw {
                    T r[HS][D], w[HS][D], s[HS][D], dg[HS];
                    T l[CS], m[CS];
                    T ro[D], wo[D], so[D], xo[D], po[D], dgo;
                };
                auto load_raw = [&](int tile, Raw &R) {
                    const int bx = tile % ntx, by = (tile / ntx) % nty, bz = D == 3 ? tile / (ntx * nty) : 0;
                    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    #pragma unroll
                    for (int k = 0; k < HS; k++) {
                        const int h = threadIdx.x + NT * k;
                        if (h < HN) {
                            const int lx = h % HX, ly = (h / HX) % HY, lz = D == 3 ? h / (HX * HY) : 0;
                            const int g = hidx<D>(P, x0 - 1 + lx, y0 - 1 + ly, z0 - 1 + lz, small);
                            R.dg[k] = __ldcg(A.dinv + g);
    #pragma unroll
                            for (int d = 0; d < D; d++) {
                                R.r[k][d] = __ldcg(A.r[cur][d] + g);
                                if (!first) {
                                    R.w[k][d] = __ldcg(A.w[cur][d] + g);
                                    R.s[k][d] = __ldcg(A.s[cur][d] + g);
                                }
                            }
                        }
                    }
    #pragma unroll
                    for (int k = 0; k < CS; k++) {
                        const int h = threadIdx.x + NT * k;
                        if (h < HC) {
                            const int lx = h % CX, ly = (h / CX) % CY, lz = D == 3 ? h / (CX * CY) : 0;
                            const int g = hidx<D>(P, x0 - 1 + lx, y0 - 1 + ly, z0 - 1 + lz, small);
                            R.l[k] = __ldg(A.lam + g);
                            R.m[k] = __ldg(A.mu + g);
                        }
                    }
                    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
                    if (gx < P.nx && gy < P.ny && (D == 2 || gz < P.nz)) {
                        const int n = gx + P.nx * (gy + (D == 3 ? P.ny * gz : 0));
                        R.dgo = __ldcg(A.dinv + n);
    #pragma unroll
                        for (int d = 0; d < D; d++) {
                            R.ro[d] = __ldcg(A.r[cur][d] + n);
                            if (!first) {
                                R.wo[d] = __ldcg(A.w[cur][d] + n);
                                R.so[d] = __ldcg(A.s[cur][d] + n);
                                R.xo[d] = A.x[d][n];
                                R.po[d] = A.p[d][n];
                            }
                        }
                    }
                };
                Raw R;
                if (bid < ntiles) load_raw(bid, R);
                for (int tile = bid; tile < ntiles; tile += nbk) {
                    const int bx = tile % ntx, by = (tile / ntx) % nty, bz = D == 3 ? tile / (ntx * nty) : 0;
                    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
                    // stage this tile: u_{i+1} = (r_i - alpha (w_i + beta s_{i-1})) / diag
                    // on the halo nodes, lam / mu on the halo cells
    #pragma unroll
                    for (int k = 0; k < HS; k++) {
                        const int h = threadIdx.x + NT * k;
                        if (h < HN) {
                            const T inv = R.dg[k];
    #pragma unroll
                            for (int d = 0; d < D; d++) {
                                T rv = R.r[k][d];
                                if (!first) rv -= ta * (R.w[k][d] + tb * R.s[k][d]);
                                su[d * HN + h] = rv * inv;
                            }
                        }
                    }
    #pragma unroll
                    for (int k = 0; k < CS; k++) {
                        const int h = threadIdx.x + NT * k;
                        if (h < HC) {
                            sl[h] = R.l[k];
                            sm[h] = R.m[k];
                        }
                    }
                    T ro[D], wo[D], so[D], xo[D], po[D];
                    const T dgo = R.dgo;
    #pragma unroll
                    for (int d = 0; d < D; d++) { ro[d] = R.ro[d]; wo[d] = R.wo[d]; so[d] = R.so[d]; xo[d] = R.xo[d]; po[d] = R.po[d]; }
                    // issue the next tile's loads; they complete while this one computes
                    if (tile + nbk < ntiles) load_raw(tile + nbk, R);
                    __syncthreads();
                    if constexpr (CELL3) {
                        // per halo cell: average stress (mean strain UE included)
                        // and the twelve hourglass forces, shared by its 8 nodes
                        for (int h = threadIdx.x; h < HC; h += blockDim.x) {
                            const int cx = h % CX, cy = (h / CX) % CY, cz = h / (CX * CY);
                            T uc[8][3];
    #pragma unroll
                            for (int b = 0; b < 8; b++) {
                                const int hn = (cx + (b & 1)) + HX * ((cy + ((b >> 1) & 1)) + HY * (cz + (b >> 2)));
                                uc[b][0] = su[hn];
                                uc[b][1] = su[HN + hn];
                                uc[b][2] = su[2 * HN + hn];
                            }
                            const T l = sl[h], m = sm[h];
                            T c[20], sx[6];
                            cell_force3<T>(l, m, uc, c);
                            voigt_stress<T, 3>(l, m, ue, sx);
    #pragma unroll
                            for (int v = 0; v < 6; v++) c[v] += sx[v];
                            float4 *dst = reinterpret_cast<float4 *>(scell + 20 * h);
    #pragma unroll
                            for (int q4 = 0; q4 < 5; q4++) dst[q4] = make_float4(c[4 * q4], c[4 * q4 + 1], c[4 * q4 + 2], c[4 * q4 + 3]);
                        }
                        __syncthreads();
                    }
                    if constexpr (D == 2) {
                        // per halo cell: average stress (mean strain UE included)
                        // and hourglass forces, shared by the cell's four nodes
                        for (int h = threadIdx.x; h < HC; h += blockDim.x) {
                            const int cx = h % CX, cy = h / CX;
                            T uc[4][2];
    #pragma unroll
                            for (int b = 0; b < 4; b++) {
                                const int hn = (cx + (b & 1)) + HX * (cy + (b >> 1));
                                uc[b][0] = su[hn];
                                uc[b][1] = su[HN + hn];
                            }
                            const T l = sl[h], m = sm[h];
                            T s3[3], fh[2], sx[3];
                            cell_force2<T>(l, m, uc, s3, fh);
                            voigt_stress<T, 2>(l, m, ue, sx);
                            scell[h] = s3[0] + sx[0];
                            scell[HC + h] = s3[1] + sx[1];
                            scell[2 * HC + h] = s3[2] + sx[2];
                            scell[3 * HC + h] = fh[0];
                            scell[4 * HC + h] = fh[1];
                        }
                        __syncthreads();
                    }
                    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
                    const bool active = gx < P.nx && gy < P.ny && (D == 2 || gz < P.nz);
                    if (active) {
                        const int n = gx + P.nx * (gy + (D == 3 ? P.ny * gz : 0));
                        const int lx = tx + 1, ly = ty + 1, lz = D == 3 ? tz + 1 : 0;
                        const int hn = lx + HX * (ly + HY * lz);
                        T un[D];
    #pragma unroll
                        for (int d = 0; d < D; d++) un[d] = su[d * HN + hn];
                        T rn[D];
                        if (!first) {
                            const T inv = dgo;
    #pragma unroll
                            for (int d = 0; d < D; d++) {
                                const T ri = ro[d];
                                const T si = wo[d] + tb * so[d];
                                const T pi = ri * inv + tb * po[d];
                                A.p[d][n] = pi;
                                A.x[d][n] = xo[d] + ta * pi;
                                A.s[nxt][d][n] = si;
                                rn[d] = ri - ta * si;
                                A.r[nxt][d][n] = rn[d];
                            }
                        } else {
    #pragma unroll
                            for (int d = 0; d < D; d++) rn[d] = ro[d];
                        }
                        T q[D], se[NV];
                        if constexpr (D == 2) {
                            q[0] = T(0);
                            q[1] = T(0);
    #pragma unroll
                            for (int a = 0; a < 4; a++) {
                                const int cl = (lx - (a & 1)) + CX * (ly - (a >> 1));
                                const T s3[3] = {scell[cl], scell[HC + cl], scell[2 * HC + cl]};
                                const T fh[2] = {scell[3 * HC + cl], scell[4 * HC + cl]};
                                T f[2];
                                node_force2<T>(a, s3, fh, f);
                                q[0] += f[0];
                                q[1] += f[1];
                            }
                            // own cell's average stress without the mean strain
                            const int c0 = lx + CX * ly;
                            T sx[3];
                            voigt_stress<T, 2>(sl[c0], sm[c0], ue, sx);
                            se[0] = scell[c0] - sx[0];
                            se[1] = scell[HC + c0] - sx[1];
                            se[2] = scell[2 * HC + c0] - sx[2];
                        } else if constexpr (CELL3) {
                            q[0] = q[1] = q[2] = T(0);
    #pragma unroll
                            for (int a = 0; a < 8; a++) {
                                const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
                                const int cl = (lx - ax) + CX * ((ly - ay) + CY * (lz - az));
                                const float4 *src = reinterpret_cast<const float4 *>(scell + 20 * cl);
                                T c[20];
    #pragma unroll
                                for (int q4 = 0; q4 < 5; q4++) {
                                    const float4 v = src[q4];
                                    c[4 * q4] = v.x; c[4 * q4 + 1] = v.y; c[4 * q4 + 2] = v.z; c[4 * q4 + 3] = v.w;
                                }
                                T f[3];
                                node_force3<T>(ax, ay, az, c, c + 6, f);
                                q[0] += f[0];
                                q[1] += f[1];
                                q[2] += f[2];
                                if (a == 0) {
                                    // own cell's average stress without the mean strain
                                    T sx[6];
                                    voigt_stress<T, 3>(sl[cl], sm[cl], ue, sx);
    #pragma unroll
                                    for (int v = 0; v < 6; v++) se[v] = c[v] - sx[v];
                                }
                            }
                        } else {
                            T eo[NV], lo, mo;
                            apply_tile<T, D, HX, HY, CX, CY>(su, sl, sm, HN, lx, ly, lz, ue, q, eo, lo, mo);
                            voigt_stress<T, D>(lo, mo, eo, se);
                        }
    #pragma unroll
                        for (int d = 0; d < D; d++) {
                            A.w[nxt][d][n] = q[d];
                            acc[0].fma_plain(rn[d], un[d]);
                            acc[1].fma_plain(q[d], un[d]);
                            acc[2].fma_plain(rn[d], rn[d]);
                        }
    #pragma unroll
                        for (int vv = 0; vv < NV; vv++) acc[3 + vv].add_plain(se[vv]);
                    }
                    __syncthreads();
                }
                double tt[3 + NV];
                if (!reduce_barrier<Acc<T>, 3 + NV>(acc, A.partials, A.result, A.bar_count, A.bar_gen, err, tt, bid, nbk)) return;
                const bool was_first = first;
                if (lead) {
                    double s6[6];
                    dmat_mul<D>(Sl, Sm, UE, s6);
                    for (int vv = 0; vv < NV; vv++) WE[vv] = tt[3 + vv] + s6[vv];
                    double gnew = tt[0], dnew = tt[1], rnew = tt[2];
                    for (int vv = 0; vv < NV; vv++) {
                        gnew += RE[vv] * UE[vv];
                        dnew += WE[vv] * UE[vv];
                        rnew += RE[vv] * RE[vv];
                    }
                    int ctl = CTL_RUN;
                    if (!was_first) {
                        it++;
                        rho_final = rnew;
                        if (rnew <= target * target) ctl = CTL_DONE;      // ||r|| <= target without a square root
                        else if (it_total + it >= A.maxit) ctl = CTL_STOP;
                    }
                    cg_take_gamma_delta(S, gnew, dnew, was_first);
                    s_ctl = ctl;
                }
                __syncthreads();
                const int ctl = s_ctl;
                first = false;
                if (!was_first) cur = nxt;
                if (ctl == CTL_DONE || ctl == CTL_STOP) {
                    if (lead) conv = (ctl == CTL_DONE);
                    break;
                }
            }
        }
        if (lead) it_total += it;
        if (!refine) break;
        // refinement: x64 += correction, then a grid-wide sync before the
        // next pass reads x64 around every node
        for (long long n = t0; n < N; n += st)
#pragma unroll
            for (int d = 0; d < D; d++) A.x64[d][n] += (double)A.x[d][n];
        if (lead) {
            for (int vv = 0; vv < NV; vv++) E64[vv] += XE[vv];
            s_ctl = (it_total >= A.maxit) ? CTL_STOP : CTL_RUN;
            if (bid == 0)
                for (int vv = 0; vv < NV; vv++) A.result[24 + vv] = E64[vv];
        }
        __syncthreads();
        const int stop = s_ctl;
        Acc<T> dummy[1];
        double dres[1];
        if (!reduce_barrier<Acc<T>, 1>(dummy, A.partials, A.result, A.bar_count, A.bar_gen, err, dres, bid, nbk)) return;
        if (stop == CTL_STOP) { if (lead) conv = false; break; }
    }
    if (refine) {
        for (long long n = t0; n < N; n += st)
#pragma unroll
            for (int d = 0; d < D; d++) A.u[d][n] = (T)A.x64[d][n];
    }
    if (bid == 0 && lead) {
        for (int vv = 0; vv < NV; vv++) A.sc->E[vv] = refine ? E64[vv] : XE[vv];
        A.sc->iters = it_total;
        A.sc->bnorm = bnorm;
        A.sc->relres = bnorm > 0.0 ? sqrt(rho_final) / bnorm : 0.0;
        if (!conv) atomicMax(err, 4);
        A.dg->cg_last = it_total;
        if (it_total > A.dg->cg_max) A.dg->cg_max = it_total;
        A.dg->cg_total += it_total;
    }
}


// Host side of one translation unit's PCG instantiations: occupancy query,
// cooperative launch and the upload of that unit's copy of the element
// tables (constant memory is per unit).  Dynamic shared memory: the 3D FP32
// cell buffer of the 16x4x4 tile; with MG, the arrays of the block-run
// levels (the bound for any hierarchy, so one attribute serves all), which
// the FP64 set-up sweep uses as scratch before them, and the fused
// two-step smoothing sweep's scratch.
template <typename T, int D>
size_t pcg_dyn_smem(int shape, bool mg)
{
    if (D == 2 && mg) {
        // the block-run levels' arrays (or, before them in each pass, the
        // set-up sweep's FP64 scratch), then the fused two-step sweep's scratch
        if (shape == 1)
            return mg_pair_offset<T, Tile<2, 1>::X, Tile<2, 1>::Y>() +
                   sizeof(T) * (size_t)sweep2_words<Tile<2, 1>::X, Tile<2, 1>::Y>();
        return mg_pair_offset<T, Tile<2, 0>::X, Tile<2, 0>::Y>() +
               sizeof(T) * (size_t)sweep2_words<Tile<2, 0>::X, Tile<2, 0>::Y>();
    }
    if (D == 3 && mg) {
        // the 3D V-cycle's sweeps (mg_sweep3z in T), or the set-up sweep's
        // (FP64, three raw streams)
        const size_t cells = sizeof(T) * (size_t)mg_sweep3z_words<T>();
        const size_t stp = sizeof(double) * (size_t)mg_sweep3z_words<double, true>(3);
        static_assert(sizeof(DS) == sizeof(double) && V3S<DS>::WORDS == V3S<double>::WORDS,
                      "the double-single set-up sweep fits the FP64 one's shared memory");
        return cells > stp ? cells : stp;
    }
    if (D != 3 || sizeof(T) != 4 || shape != 0) return 0;
    constexpr int HC = (Tile<3, 0>::X + 1) * (Tile<3, 0>::Y + 1) * (Tile<3, 0>::Z + 1);
    return sizeof(float) * 20 * HC;
}

// the kernel variant of a tile shape, with or without the multigrid
// preconditioner (2D only)
template <typename T, int D>
const void *pcg_kernel(int shape, bool mg)
{
    if (mg) return shape == 1 ? (const void *)k_pcg<T, D, 1, true> : (const void *)k_pcg<T, D, 0, true>;
    return shape == 1 ? (const void *)k_pcg<T, D, 1, false> : (const void *)k_pcg<T, D, 0, false>;
}

template <typename T, int D>
cudaError_t pcg_occupancy_t(int shape, bool mg, int block, int *per_sm)
{
    const void *fn = pcg_kernel<T, D>(shape, mg);
    const size_t dyn = pcg_dyn_smem<T, D>(shape, mg);
    if (dyn) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, block, dyn);
}

template <typename T, int D>
cudaError_t pcg_launch_t(int shape, bool mg, const void *jobs, int njobs, int grid, int block, cudaStream_t s)
{
    const PCGArgs<T, D> *pj = (const PCGArgs<T, D> *)jobs;
    void *args[] = {(void *)&pj, (void *)&njobs};
    return cudaLaunchCooperativeKernel(pcg_kernel<T, D>(shape, mg), dim3(grid), dim3(block), args,
                                       pcg_dyn_smem<T, D>(shape, mg), s);
}

} // namespace pfdev
