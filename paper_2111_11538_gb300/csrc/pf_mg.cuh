// Geometric multigrid preconditioner of the 2D solve (K3/K4): u = M r is one
// V-cycle over a hierarchy of periodic Q1 grids, each coarse level with half
// the nodes per axis and the 2x2 average of its fine cells' moduli (the
// operator rediscretised, not the Galerkin product).  Smoothing is a
// Chebyshev iteration on D^-1 A over [b/30, b], where b is a bound on the
// largest eigenvalue of D^-1 A that holds for any cell moduli (the largest
// eigenvalue of diag(K_e)^-1 K_e of one element, set by the Poisson ratio);
// restriction is the transpose of bilinear prolongation.  With the same
// polynomial before and after the coarse correction and a polynomial coarse
// solve, the V-cycle is a fixed symmetric positive-definite operator, so it
// serves as a CG preconditioner.  The mean-strain dofs keep their Jacobi
// scaling (block-diagonal preconditioner).
//
// Levels with more than a few tiles: every Chebyshev step is one sweep of
// the tiled Q1 operator (the cell decomposition of cell_force2) and one grid
// barrier.  Operands that are pointwise in stored vectors are formed while
// the tile halo is staged (the Chebyshev direction from r and the previous
// direction, the restricted residual, the prolonged correction, the CG
// update), and the last step of a smoothing, which needs no operator
// product, is applied in the epilogue of the step before it, so no sweep is
// spent on either.  The coarse levels are run by the job's first block in
// its shared memory (whole levels, one pass per phase, block barriers).
#pragma once

namespace pfdev {

constexpr int MG_MAX_LEVELS = 12;
constexpr int MG_MAX_STEPS = 16;

template <typename T>
struct MGLevel {
    int nx, ny, nz;                // nodes (= cells) per axis, periodic (nz = 1 in 2D)
    T *lam, *mu;                   // cell moduli (level 0: the solve's own, read only)
    T *dinv;                       // inverse Jacobi diagonal (level 0: the solve's own)
    T *f[3];                       // right-hand side (levels >= 1; level 0 uses the CG residual)
    T *xpre[3];                    // iterate of the pre-smoothing (coarsest: of its solve)
    T *xpost[3];                   // iterate of the post-smoothing; the level's final correction
                                   // when it is done (finest level: u = M r)
    T *r[2][3], *d[2][3];          // [buffer][component]: residual, Chebyshev direction
};

template <typename T>
struct MGHier {
    int L;                         // levels
    int Lg;                        // levels [0, Lg) run on the whole grid, [Lg, L) by the job's first
                                   // block in shared memory (mg_block_words)
    int deg[MG_MAX_LEVELS];        // Chebyshev steps of each pre- and post-smoothing, per level
    int csteps;                    // Chebyshev steps of the coarsest solve (>= 2)
    T c1[MG_MAX_STEPS], c2[MG_MAX_STEPS];   // d_j = c1[j] d_{j-1} + c2[j] D^-1 r_j  (c1[0] = 0)
    MGLevel<T> lv[MG_MAX_LEVELS];
};

// Plain grid barrier (no reduction).  Waits are bounded like reduce_barrier.
__device__ __forceinline__ bool grid_sync(unsigned int *count, unsigned int *gen, int *err, int nbk)
{
    __shared__ int s_gok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_gok = 1;
        const unsigned int g = ld_relaxed_gpu(gen);
        const unsigned int arrived = atom_add_acq_rel_gpu(count, 1u);
        if (arrived == (unsigned int)nbk - 1) {
            *count = 0u;
            red_add_release_gpu(gen, 1u);
        } else if (!wait_generation(gen, g, err, SPIN_LIMIT)) {
            s_gok = 0;
        }
    }
    __syncthreads();
    return s_gok != 0;
}

__device__ __forceinline__ int mg_wrap(int a, int n, bool small) { return small ? wrapm(a, n) : wrap(a, n); }

// One sweep of the level's Q1 operator over node tiles TX x TY: val(gx, gy, v)
// gives the operand at any node (called for the tile and its halo), and
// epi(n, v, q, se) receives, at each own node n, the operand v, q = A v and
// (WITH_E) the own cell's average stress without the mean strain, the mean
// strain ue being added to every cell's stress for q.
template <typename T, int TX, int TY, bool WITH_E, class Val, class Epi>
__device__ __forceinline__ void mg_sweep(int nx, int ny, const T *lam, const T *mu, int bid, int nbk, T *su, T *sl,
                                         T *sm, T *scell, const T *ue, Val &&val, Epi &&epi)
{
    constexpr int HX = TX + 2, HY = TY + 2, CX = TX + 1, CY = TY + 1, HN = HX * HY, HC = CX * CY, NT = TX * TY;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntiles = ntx * nty;
    const bool small = nx < HX || ny < HY;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    for (int tile = bid; tile < ntiles; tile += nbk) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        for (int h = threadIdx.x; h < HN; h += NT) {
            T v[2];
            val(mg_wrap(x0 - 1 + h % HX, nx, small), mg_wrap(y0 - 1 + h / HX, ny, small), v);
            su[h] = v[0];
            su[HN + h] = v[1];
        }
        for (int h = threadIdx.x; h < HC; h += NT) {
            const int g = mg_wrap(x0 - 1 + h % CX, nx, small) + nx * mg_wrap(y0 - 1 + h / CX, ny, small);
            sl[h] = __ldcg(lam + g);
            sm[h] = __ldcg(mu + g);
        }
        __syncthreads();
        for (int h = threadIdx.x; h < HC; h += NT) {
            const int cx = h % CX, cy = h / CX;
            T uc[4][2];
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int hn = (cx + (b & 1)) + HX * (cy + (b >> 1));
                uc[b][0] = su[hn];
                uc[b][1] = su[HN + hn];
            }
            const T l = sl[h], m = sm[h];
            T s3[3], fh[2];
            cell_force2<T>(l, m, uc, s3, fh);
            if constexpr (WITH_E) {
                T sx[3];
                voigt_stress<T, 2>(l, m, ue, sx);
#pragma unroll
                for (int v = 0; v < 3; v++) s3[v] += sx[v];
            }
            scell[h] = s3[0];
            scell[HC + h] = s3[1];
            scell[2 * HC + h] = s3[2];
            scell[3 * HC + h] = fh[0];
            scell[4 * HC + h] = fh[1];
        }
        __syncthreads();
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < nx && gy < ny) {
            const int lx = tx + 1, ly = ty + 1, hn = lx + HX * ly;
            const T un[2] = {su[hn], su[HN + hn]};
            T q[2] = {T(0), T(0)}, se[3] = {T(0), T(0), T(0)};
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
            if constexpr (WITH_E) {
                const int c0 = lx + CX * ly;
                T sx[3];
                voigt_stress<T, 2>(sl[c0], sm[c0], ue, sx);
                se[0] = scell[c0] - sx[0];
                se[1] = scell[HC + c0] - sx[1];
                se[2] = scell[2 * HC + c0] - sx[2];
            }
            epi(gx + nx * gy, un, q, se);
        }
        __syncthreads();
    }
}

// Shared memory of the block-run levels [Lg, L), in words of T: per level 11
// arrays of its node count (x, r, d, f by component, then the inverse
// diagonal and the cell moduli), then the scratch of the largest level: the
// operand (2 per node) and the cell forces (5 per cell).  The first
// block-run level has at most NB nodes and each next a quarter of the one
// before, so mg_block_words_cap(NB) bounds the total.
constexpr int MG_BLK_ARRAYS = 11, MG_BLK_SCRATCH = 7;

// node count up to which a level is run by one block: the shared arrays of
// such levels fit next to two resident 256-thread PCG blocks per SM
template <typename T>
__host__ __device__ constexpr long long mg_block_nodes() { return sizeof(T) == 4 ? 1024 : 256; }

template <typename T>
__host__ __device__ inline long long mg_block_words(const MGHier<T> &H)
{
    long long w = 0, nmax = 0;
    for (int k = H.Lg; k < H.L; k++) {
        const long long n = (long long)H.lv[k].nx * H.lv[k].ny;
        w += MG_BLK_ARRAYS * n;
        nmax = n > nmax ? n : nmax;
    }
    return nmax ? w + MG_BLK_SCRATCH * nmax : 0;
}

__host__ __device__ inline long long mg_block_words_cap(long long nb)
{
    return MG_BLK_ARRAYS * (nb * 4 / 3 + 1) + MG_BLK_SCRATCH * nb;
}

// A block-run level's arrays in shared memory.
template <typename T>
struct BLevel {
    int nx, ny, n;
    T *x[2], *r[2], *d[2], *f[2], *dinv, *lam, *mu;
};

template <typename T>
__device__ __forceinline__ BLevel<T> blevel(T *base, const MGHier<T> &H, int k)
{
    long long off = 0;
    for (int m = H.Lg; m < k; m++) off += MG_BLK_ARRAYS * (long long)H.lv[m].nx * H.lv[m].ny;
    BLevel<T> B;
    B.nx = H.lv[k].nx;
    B.ny = H.lv[k].ny;
    B.n = B.nx * B.ny;
    T *p = base + off;
    const int n = B.n;
    B.x[0] = p; B.x[1] = p + n; B.r[0] = p + 2 * n; B.r[1] = p + 3 * n; B.d[0] = p + 4 * n; B.d[1] = p + 5 * n;
    B.f[0] = p + 6 * n; B.f[1] = p + 7 * n; B.dinv = p + 8 * n; B.lam = p + 9 * n; B.mu = p + 10 * n;
    return B;
}

// the scratch after the block-run levels
template <typename T>
__device__ __forceinline__ T *bscratch(T *base, const MGHier<T> &H)
{
    long long off = 0;
    for (int m = H.Lg; m < H.L; m++) off += MG_BLK_ARRAYS * (long long)H.lv[m].nx * H.lv[m].ny;
    return base + off;
}

// One sweep of a block-run level, whole level at once: val(i, v) for every
// node (called once per node, so it may store), then the cell forces, then
// epi(i, v, q) with q = A v at every node; block barriers between phases.
template <typename T, class Val, class Epi>
__device__ __forceinline__ void blk_sweep(const BLevel<T> &B, T *scr, int nmax, Val &&val, Epi &&epi)
{
    const int n = B.n, nx = B.nx, ny = B.ny;
    T *v0 = scr, *v1 = scr + nmax, *cf = scr + 2 * nmax;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T v[2];
        val(i, v);
        v0[i] = v[0];
        v1[i] = v[1];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int cx = c % nx, cy = c / nx;
        const int cx1 = cx + 1 == nx ? 0 : cx + 1, cy1 = cy + 1 == ny ? 0 : cy + 1;
        const int nd[4] = {c, cx1 + nx * cy, cx + nx * cy1, cx1 + nx * cy1};
        T uc[4][2];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            uc[b][0] = v0[nd[b]];
            uc[b][1] = v1[nd[b]];
        }
        T s3[3], fh[2];
        cell_force2<T>(B.lam[c], B.mu[c], uc, s3, fh);
        cf[c] = s3[0];
        cf[nmax + c] = s3[1];
        cf[2 * nmax + c] = s3[2];
        cf[3 * nmax + c] = fh[0];
        cf[4 * nmax + c] = fh[1];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ix = i % nx, iy = i / nx;
        T q[2] = {T(0), T(0)};
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int ex = (a & 1) ? (ix == 0 ? nx - 1 : ix - 1) : ix;
            const int ey = (a >> 1) ? (iy == 0 ? ny - 1 : iy - 1) : iy;
            const int c = ex + nx * ey;
            const T s3[3] = {cf[c], cf[nmax + c], cf[2 * nmax + c]};
            const T fh[2] = {cf[3 * nmax + c], cf[4 * nmax + c]};
            T f[2];
            node_force2<T>(a, s3, fh, f);
            q[0] += f[0];
            q[1] += f[1];
        }
        const T v[2] = {v0[i], v1[i]};
        epi(i, v, q);
    }
    __syncthreads();
}

// Shared memory (words of T) of mg_sweep2 for a TX x TY tile: two operands
// on the width-2 halo, the intermediate residual and second operand on the
// width-1 halo, and five values per cell of the width-2 halo.
template <int TX, int TY>
__host__ __device__ constexpr int sweep2_words()
{
    return 4 * (TX + 4) * (TY + 4) + 4 * (TX + 2) * (TY + 2) + 5 * (TX + 3) * (TY + 3);
}

// Two consecutive operator products on each tile with no grid barrier
// between them (the ring of halo nodes both need is recomputed by the
// neighbouring tiles): val(gx, gy, v0, a0) gives the first operand v0 and an
// auxiliary a0 on the width-2 halo; mid(g, v0, a0, q0, r1, v1) forms, on the
// width-1 halo, from v0, a0 and q0 = A v0, an intermediate r1 and the second
// operand v1; epi(n, v0, a0, r1, v1, q1, se) gets q1 = A v1 at every own
// node.  E2: the second product adds the mean strain ue to every cell's
// stress and se is the own cell's stress of v1 without it (else zero).
// Scratch: sweep2_words<TX, TY>() words of shared memory at scr.
template <typename T, int TX, int TY, bool E2, class Val, class Mid, class Epi>
__device__ __forceinline__ void mg_sweep2(int nx, int ny, const T *lam, const T *mu, int bid, int nbk, T *scr,
                                          const T *ue, Val &&val, Mid &&mid, Epi &&epi)
{
    constexpr int AX = TX + 4, AY = TY + 4, AN = AX * AY;     // width-2 halo nodes
    constexpr int BX = TX + 2, BY = TY + 2, BN = BX * BY;     // width-1 halo nodes
    constexpr int CX = TX + 3, CY = TY + 3, CN = CX * CY;     // cells of the width-2 halo
    constexpr int DX = TX + 1, DN = (TX + 1) * (TY + 1);      // cells of the width-1 halo
    constexpr int NT = TX * TY;
    T *v0 = scr, *a0 = scr + 2 * AN, *r1 = scr + 4 * AN, *v1 = r1 + 2 * BN, *cf = v1 + 2 * BN;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntiles = ntx * nty;
    const bool small = nx < AX || ny < AY;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    auto cells = [&](const T *u, int ux, int un, int ncx, int ncell, int ox, int oy, bool withE) {
        // cells with lower-left node (cx, cy) of the operand grid u (row
        // length ux, un nodes per component), global origin (ox, oy)
        for (int h = threadIdx.x; h < ncell; h += NT) {
            const int cx = h % ncx, cy = h / ncx;
            const int g = mg_wrap(ox + cx, nx, small) + nx * mg_wrap(oy + cy, ny, small);
            T uc[4][2];
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int hn = (cx + (b & 1)) + ux * (cy + (b >> 1));
                uc[b][0] = u[hn];
                uc[b][1] = u[un + hn];
            }
            T s3[3], fh[2];
            const T l = __ldcg(lam + g), m = __ldcg(mu + g);
            cell_force2<T>(l, m, uc, s3, fh);
            if (E2 && withE) {
                T sx[3];
                voigt_stress<T, 2>(l, m, ue, sx);
#pragma unroll
                for (int v = 0; v < 3; v++) s3[v] += sx[v];
            }
            cf[h] = s3[0];
            cf[CN + h] = s3[1];
            cf[2 * CN + h] = s3[2];
            cf[3 * CN + h] = fh[0];
            cf[4 * CN + h] = fh[1];
        }
    };
    auto force = [&](int lx, int ly, int ncx, T (&q)[2]) {
        // q at the node whose lower-left cell is (lx, ly) in cell coordinates
        q[0] = T(0);
        q[1] = T(0);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int cl = (lx - (a & 1)) + ncx * (ly - (a >> 1));
            const T s3[3] = {cf[cl], cf[CN + cl], cf[2 * CN + cl]};
            const T fh[2] = {cf[3 * CN + cl], cf[4 * CN + cl]};
            T f[2];
            node_force2<T>(a, s3, fh, f);
            q[0] += f[0];
            q[1] += f[1];
        }
    };
    for (int tile = bid; tile < ntiles; tile += nbk) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        for (int h = threadIdx.x; h < AN; h += NT) {
            T v[2], a[2];
            val(mg_wrap(x0 - 2 + h % AX, nx, small), mg_wrap(y0 - 2 + h / AX, ny, small), v, a);
            v0[h] = v[0];
            v0[AN + h] = v[1];
            a0[h] = a[0];
            a0[AN + h] = a[1];
        }
        __syncthreads();
        cells(v0, AX, AN, CX, CN, x0 - 2, y0 - 2, false);
        __syncthreads();
        for (int h = threadIdx.x; h < BN; h += NT) {
            const int mx = h % BX, my = h / BX, ah = (mx + 1) + AX * (my + 1);
            T q[2];
            force(mx + 1, my + 1, CX, q);
            const T vv[2] = {v0[ah], v0[AN + ah]}, aa[2] = {a0[ah], a0[AN + ah]};
            T rr[2], ww[2];
            mid(mg_wrap(x0 - 1 + mx, nx, small) + nx * mg_wrap(y0 - 1 + my, ny, small), vv, aa, q, rr, ww);
            r1[h] = rr[0];
            r1[BN + h] = rr[1];
            v1[h] = ww[0];
            v1[BN + h] = ww[1];
        }
        __syncthreads();
        cells(v1, BX, BN, DX, DN, x0 - 1, y0 - 1, true);
        __syncthreads();
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < nx && gy < ny) {
            const int ah = (tx + 2) + AX * (ty + 2), bh = (tx + 1) + BX * (ty + 1);
            T q[2];
            force(tx + 1, ty + 1, DX, q);
            const T vv[2] = {v0[ah], v0[AN + ah]}, aa[2] = {a0[ah], a0[AN + ah]};
            const T rr[2] = {r1[bh], r1[BN + bh]}, ww[2] = {v1[bh], v1[BN + bh]};
            const int n = gx + nx * gy;
            T se[3] = {T(0), T(0), T(0)};
            if constexpr (E2) {
                const int c0 = (tx + 1) + DX * (ty + 1);
                T sx[3];
                voigt_stress<T, 2>(__ldcg(lam + n), __ldcg(mu + n), ue, sx);
                se[0] = cf[c0] - sx[0];
                se[1] = cf[CN + c0] - sx[1];
                se[2] = cf[2 * CN + c0] - sx[2];
            }
            epi(n, vv, aa, rr, ww, q, se);
        }
        __syncthreads();
    }
}

// Coarse level C from fine level F (both in global memory): cell moduli =
// mean of the 2x2 fine cells, Jacobi diagonal from the four coarse cells
// around each node.  Threads t0, t0 + st, ... take the coarse nodes.
template <typename T>
__device__ void mg_coarsen(const MGLevel<T> &F, const MGLevel<T> &C, long long t0, long long st)
{
    const int n = C.nx * C.ny;
    auto avg = [&](const T *a, int cx, int cy) {
        const int i = 2 * cx + F.nx * (2 * cy);
        return T(0.25) * ((__ldcg(a + i) + __ldcg(a + i + 1)) + (__ldcg(a + i + F.nx) + __ldcg(a + i + F.nx + 1)));
    };
    for (long long i = t0; i < n; i += st) {
        const int cx = (int)(i % C.nx), cy = (int)(i / C.nx);
        C.lam[i] = avg(F.lam, cx, cy);
        C.mu[i] = avg(F.mu, cx, cy);
        T dg = T(0);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int ex = wrap(cx - (a & 1), C.nx), ey = wrap(cy - (a >> 1), C.ny);
            dg += avg(F.lam, ex, ey) * KdL<T, 2>() + avg(F.mu, ex, ey) * KdM<T, 2>();
        }
        C.dinv[i] = T(1) / dg;
    }
}

// The same into a block-run level's shared arrays, from a grid level
// (global, fl / fm / fnx) or the block-run level above (shared).
template <typename T>
__device__ void mg_coarsen_blk(const T *fl, const T *fm, int fnx, bool global, const BLevel<T> &C)
{
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
        const int cx = i % C.nx, cy = i / C.nx, f = 2 * cx + fnx * (2 * cy);
        auto ld = [&](const T *a, int o) { return global ? __ldcg(a + o) : a[o]; };
        C.lam[i] = T(0.25) * ((ld(fl, f) + ld(fl, f + 1)) + (ld(fl, f + fnx) + ld(fl, f + fnx + 1)));
        C.mu[i] = T(0.25) * ((ld(fm, f) + ld(fm, f + 1)) + (ld(fm, f + fnx) + ld(fm, f + fnx + 1)));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
        const int cx = i % C.nx, cy = i / C.nx;
        T dg = T(0);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int c = wrap(cx - (a & 1), C.nx) + C.nx * wrap(cy - (a >> 1), C.ny);
            dg += C.lam[c] * KdL<T, 2>() + C.mu[c] * KdM<T, 2>();
        }
        C.dinv[i] = T(1) / dg;
    }
    __syncthreads();
}

// Hierarchy set-up at the start of a solve (the cell moduli change every
// step): the grid levels below Lg, with a barrier after each.  Returns false
// if a barrier timed out.
template <typename T>
__device__ bool mg_setup(const MGHier<T> &H, unsigned int *bc, unsigned int *bg, int *err, int bid, int nbk)
{
    const int Lgw = H.Lg < H.L ? H.Lg : H.L;
    const long long t0 = bid * (long long)blockDim.x + threadIdx.x, st = (long long)nbk * blockDim.x;
    for (int k = 1; k < Lgw; k++) {
        mg_coarsen<T>(H.lv[k - 1], H.lv[k], t0, st);
        if (!grid_sync(bc, bg, err, nbk)) return false;
    }
    return true;
}

// The shared arrays of the block-run levels, filled by the job's first
// block at the start of every CG pass (the residual sweep before it uses
// the same shared memory as scratch).
template <typename T>
__device__ void mg_setup_block(const MGHier<T> &H, T *sblk)
{
    const int Lgw = H.Lg < H.L ? H.Lg : H.L;
    for (int k = Lgw; k < H.L; k++) {
            const BLevel<T> C = blevel<T>(sblk, H, k);
            if (k == Lgw) {
                mg_coarsen_blk<T>(H.lv[k - 1].lam, H.lv[k - 1].mu, H.lv[k - 1].nx, true, C);
            } else {
                const BLevel<T> F = blevel<T>(sblk, H, k - 1);
                mg_coarsen_blk<T>(F.lam, F.mu, F.nx, false, C);
            }
    }
}

// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (~48 significant bits).  Sums use Knuth's TwoSum, products
// the FMA form of TwoProduct; results are renormalised with the fast
// two-sum (|a| >= |b|).  The mixed method's refinement residual b - A x is
// formed this way: FP64 runs at a small fraction of the FP32 rate here.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_quick(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_from(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const DF u = df_quick(s.hi, s.lo + t.hi);
    return df_quick(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
// exact scaling by a power of two
__device__ __forceinline__ DF df_scale(DF a, float p2) { return {a.hi * p2, a.lo * p2}; }
__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p);
    return df_quick(p, fmaf(a.lo, b, e));
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return df_quick(p, e + fmaf(a.hi, b.lo, a.lo * b.hi));
}

// plane-strain stress of a Voigt strain e (engineering shear) in
// double-float: l tr e + 2 m e on the normals, m e on the shear
__device__ __forceinline__ void voigt2_df(float l, float m, const DF (&e)[3], DF (&s)[3])
{
    const float m2 = 2.0f * m;                 // exact
    const DF tr = df_add(e[0], e[1]);
    s[0] = df_add(df_mul_f(tr, l), df_mul_f(e[0], m2));
    s[1] = df_add(df_mul_f(tr, l), df_mul_f(e[1], m2));
    s[2] = df_mul_f(e[2], m);
}

// cell_force2 in double-float: average stress of the cell's displacement
// plus the mean-strain stress, hourglass forces (l, m: the FP32 moduli)
__device__ __forceinline__ void cell_force2_df(float l, float m, const DF (&ue)[4][2], const DF (&xe)[3], DF (&s)[3],
                                               DF (&fh)[2], DF (&s_own)[3])
{
    const DF Gxu = df_scale(df_add(df_sub(ue[1][0], ue[0][0]), df_sub(ue[3][0], ue[2][0])), 0.5f);
    const DF Gyu = df_scale(df_add(df_sub(ue[2][0], ue[0][0]), df_sub(ue[3][0], ue[1][0])), 0.5f);
    const DF Gxv = df_scale(df_add(df_sub(ue[1][1], ue[0][1]), df_sub(ue[3][1], ue[2][1])), 0.5f);
    const DF Gyv = df_scale(df_add(df_sub(ue[2][1], ue[0][1]), df_sub(ue[3][1], ue[1][1])), 0.5f);
    const DF hu = df_sub(df_sub(ue[0][0], ue[1][0]), df_sub(ue[2][0], ue[3][0]));
    const DF hv = df_sub(df_sub(ue[0][1], ue[1][1]), df_sub(ue[2][1], ue[3][1]));
    const DF G[3] = {Gxu, Gyv, df_add(Gyu, Gxv)};   // Voigt strain, engineering shear
    voigt2_df(l, m, G, s_own);
    DF sx[3];
    voigt2_df(l, m, xe, sx);
#pragma unroll
    for (int v = 0; v < 3; v++) s[v] = df_add(s_own[v], sx[v]);
    // (l + 3 m) / 12, with l + 3 m exact as a double-float
    const float p3 = 3.0f * m;
    const DF l3m = df_add(DF{l, 0.0f}, DF{p3, fmaf(3.0f, m, -p3)});
    const DF c = df_mul(l3m, df_from(1.0 / 12.0));
    fh[0] = df_mul(c, hu);
    fh[1] = df_mul(c, hv);
}

// node_force2 in double-float
__device__ __forceinline__ void node_force2_df(int a, const DF (&s)[3], const DF (&fh)[2], DF (&f)[2])
{
    const float bx = (a & 1) ? 0.5f : -0.5f, by = (a >> 1) ? 0.5f : -0.5f;
    const bool gp = (a == 0 || a == 3);
    const DF g0 = gp ? fh[0] : df_neg(fh[0]), g1 = gp ? fh[1] : df_neg(fh[1]);
    f[0] = df_add(df_add(df_scale(s[0], bx), df_scale(s[2], by)), g0);
    f[1] = df_add(df_add(df_scale(s[1], by), df_scale(s[2], bx)), g1);
}

// Shared memory (in doubles) of setup_tiled for a TX x TY tile: the FP64
// operand on the tile halo and five values per halo cell.
template <int TX, int TY>
__host__ __device__ constexpr int setup_tiled_doubles() { return 2 * (TX + 2) * (TY + 2) + 5 * (TX + 1) * (TY + 1); }

// Byte offset of mg_sweep2's scratch in the dynamic shared memory: after
// the block-run levels' arrays and the set-up sweep's scratch (which share
// the start), rounded to 16 bytes.  The total is pcg_dyn_smem.
template <typename T, int TX, int TY>
__host__ __device__ constexpr size_t mg_pair_offset()
{
    const size_t blk = sizeof(T) * (size_t)mg_block_words_cap(mg_block_nodes<T>());
    const size_t stp = sizeof(double) * (size_t)setup_tiled_doubles<TX, TY>();
    return ((blk > stp ? blk : stp) + 15) / 16 * 16;
}

// The set-up sweep of one CG pass, 2D, over node tiles: right-hand side
// b = sum_e Bbar^T sig*, Jacobi diagonal, r = b - A x (x: the FP64 solution
// in refinement mode, else the displacement; mean strain xe) with the
// operator applied in FP64 from per-cell average stress and hourglass forces
// computed once per tile (dscr: setup_tiled_doubles<TX, TY>() doubles of
// shared memory), and the per-node sums of the mean-strain rows: acc[0]
// ||b||^2, [1] ||r||^2, [2] sum lam, [3] sum mu, [4..6] sum sig*, [10..12]
// sum of the own cells' stress of x without the mean strain; in the mixed
// method the operator part is evaluated in double-float.  Also clears
// p, s and (when x is not used or in refinement mode) the iterate.  In
// refinement mode the first pass keeps b in A.b64; a residual-only pass
// (resid) reads it there and skips everything that does not change during
// a solve (b, the diagonal, sums [0] and [2, 10)).
template <typename T, int TX, int TY>
__device__ void setup_tiled(const PCGArgs<T, 2> &A, bool use_x, bool refine, bool resid, const double *xe,
                            double *dscr, Acc<double> (&acc)[16], int bid, int nbk)
{
    const Params &P = A.P;
    constexpr int HX = TX + 2, HY = TY + 2, CX = TX + 1, CY = TY + 1, HN = HX * HY, HC = CX * CY, NT = TX * TY;
    double *hu = dscr, *hc = dscr + 2 * HN;
    const int nx = P.nx, ny = P.ny;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntiles = ntx * nty;
    const bool small = nx < HX || ny < HY;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    // the mixed method's refinement residual: double-float instead of FP64
    const bool dfp = refine && sizeof(T) == 4;
    DF *du = reinterpret_cast<DF *>(dscr), *dc = du + 2 * HN;      // same bytes as hu, hc
    const DF xed[3] = {df_from(xe[0]), df_from(xe[1]), df_from(xe[2])};
    for (int tile = bid; tile < ntiles; tile += nbk) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        if (use_x && dfp) {
            for (int h = threadIdx.x; h < HN; h += NT) {
                const int g = mg_wrap(x0 - 1 + h % HX, nx, small) + nx * mg_wrap(y0 - 1 + h / HX, ny, small);
                du[h] = df_from(__ldcg(A.x64[0] + g));
                du[HN + h] = df_from(__ldcg(A.x64[1] + g));
            }
            __syncthreads();
            for (int h = threadIdx.x; h < HC; h += NT) {
                const int cx = h % CX, cy = h / CX;
                const int g = mg_wrap(x0 - 1 + cx, nx, small) + nx * mg_wrap(y0 - 1 + cy, ny, small);
                DF uc[4][2];
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int hn = (cx + (b & 1)) + HX * (cy + (b >> 1));
                    uc[b][0] = du[hn];
                    uc[b][1] = du[HN + hn];
                }
                DF s3[3], fh[2], own[3];
                cell_force2_df((float)A.lam[g], (float)A.mu[g], uc, xed, s3, fh, own);
                dc[h] = s3[0];
                dc[HC + h] = s3[1];
                dc[2 * HC + h] = s3[2];
                dc[3 * HC + h] = fh[0];
                dc[4 * HC + h] = fh[1];
            }
            __syncthreads();
        } else if (use_x) {
            for (int h = threadIdx.x; h < HN; h += NT) {
                const int g = mg_wrap(x0 - 1 + h % HX, nx, small) + nx * mg_wrap(y0 - 1 + h / HX, ny, small);
                hu[h] = refine ? __ldcg(A.x64[0] + g) : (double)A.x[0][g];
                hu[HN + h] = refine ? __ldcg(A.x64[1] + g) : (double)A.x[1][g];
            }
            __syncthreads();
            for (int h = threadIdx.x; h < HC; h += NT) {
                const int cx = h % CX, cy = h / CX;
                const int g = mg_wrap(x0 - 1 + cx, nx, small) + nx * mg_wrap(y0 - 1 + cy, ny, small);
                double uc[4][2];
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int hn = (cx + (b & 1)) + HX * (cy + (b >> 1));
                    uc[b][0] = hu[hn];
                    uc[b][1] = hu[HN + hn];
                }
                const double l = (double)A.lam[g], m = (double)A.mu[g];
                double s3[3], fh[2], sx[3];
                cell_force2<double>(l, m, uc, s3, fh);
                voigt_stress<double, 2>(l, m, xe, sx);
                hc[h] = s3[0] + sx[0];
                hc[HC + h] = s3[1] + sx[1];
                hc[2 * HC + h] = s3[2] + sx[2];
                hc[3 * HC + h] = fh[0];
                hc[4 * HC + h] = fh[1];
            }
            __syncthreads();
        }
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < nx && gy < ny) {
            const int n = gx + nx * gy, lx = tx + 1, ly = ty + 1;
            double b[2], ax[2] = {0.0, 0.0}, dgn = 1.0, so[3], deo[3] = {0.0, 0.0, 0.0}, lo, mo, unused[2], unused3[3];
            if (resid) {
                b[0] = __ldcg(A.b64[0] + n);
                b[1] = __ldcg(A.b64[1] + n);
                lo = (double)A.lam[n];
                mo = (double)A.mu[n];
            } else {
                node_setup<T, double, double, 2>(P, n, A.lam, A.mu, A.sig, A.x64, xe, false, b, unused, dgn, so, unused3,
                                                 lo, mo);
                if (refine) {
                    A.b64[0][n] = b[0];
                    A.b64[1][n] = b[1];
                }
            }
            double rv2[2] = {b[0], b[1]};
            if (use_x && dfp) {
                DF axd[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int cl = (lx - (a & 1)) + CX * (ly - (a >> 1));
                    const DF s3[3] = {dc[cl], dc[HC + cl], dc[2 * HC + cl]};
                    const DF fh[2] = {dc[3 * HC + cl], dc[4 * HC + cl]};
                    DF f[2];
                    node_force2_df(a, s3, fh, f);
                    axd[0] = df_add(axd[0], f[0]);
                    axd[1] = df_add(axd[1], f[1]);
                }
#pragma unroll
                for (int d = 0; d < 2; d++) rv2[d] = df_val(df_sub(df_from(b[d]), axd[d]));
                // the own cell's stress of x without the mean strain
                const int c0 = lx + CX * ly;
                DF sx[3];
                voigt2_df((float)lo, (float)mo, xed, sx);
#pragma unroll
                for (int v = 0; v < 3; v++) deo[v] = df_val(df_sub(dc[v * HC + c0], sx[v]));
            } else if (use_x) {
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int cl = (lx - (a & 1)) + CX * (ly - (a >> 1));
                    const double s3[3] = {hc[cl], hc[HC + cl], hc[2 * HC + cl]};
                    const double fh[2] = {hc[3 * HC + cl], hc[4 * HC + cl]};
                    double f[2];
                    node_force2<double>(a, s3, fh, f);
                    ax[0] += f[0];
                    ax[1] += f[1];
                }
                // the own cell's stress of x without the mean strain
                const int c0 = lx + CX * ly;
                double sx[3];
                voigt_stress<double, 2>(lo, mo, xe, sx);
                deo[0] = hc[c0] - sx[0];
                deo[1] = hc[HC + c0] - sx[1];
                deo[2] = hc[2 * HC + c0] - sx[2];
                rv2[0] = b[0] - ax[0];
                rv2[1] = b[1] - ax[1];
            }
            if (!resid) {
                A.dinv[n] = (T)(1.0 / dgn);
                acc[2].add(lo);
                acc[3].add(mo);
#pragma unroll
                for (int v = 0; v < 3; v++) acc[4 + v].add(so[v]);
            }
#pragma unroll
            for (int v = 0; v < 3; v++) acc[10 + v].add(deo[v]);
#pragma unroll
            for (int d = 0; d < 2; d++) {
                const double rv = rv2[d];
                if (refine && !use_x) A.x64[d][n] = 0.0;
                if (refine || !use_x) A.x[d][n] = T(0);
                A.p[d][n] = T(0);
                A.s[0][d][n] = T(0);
                A.r[0][d][n] = (T)rv;
                if (!resid) acc[0].addprod(b[d], b[d]);
                acc[1].addprod(rv, rv);
            }
        }
        __syncthreads();
    }
}

// One pass of MG-preconditioned CG (the Chronopoulos-Gear form of the
// Jacobi solve, with u = M r a V-cycle).  Per iteration i:
//   V-cycle on r_i, its first sweep also doing the update of iteration i-1
//   (p, s, x, r) and reducing ||r_i||^2 for the stopping test;
//   u_i = the V-cycle's result, w_i = A u_i, gamma_i = r_i.u_i, delta_i =
//   w_i.u_i and the mean-strain row in one sweep and one reduction.
// Returns CTL_DONE or CTL_STOP, or -1 when a barrier timed out.
template <typename T, int TX, int TY>
__device__ int mg_pass(const PCGArgs<T, 2> &A, const MGHier<T> &H, PCGState &S, T *su, T *sl, T *sm, T *scell,
                       T *sblk, T &s_ta, T &s_tb, T *s_ue, int &s_ctl, int bid, int nbk, int *err)
{
    constexpr int NV = 3;
    const bool lead = threadIdx.x == 0;
    const int L = H.L, Lgw = H.Lg < H.L ? H.Lg : H.L, cs = H.csteps;
    const MGLevel<T> &L0 = H.lv[0];
    unsigned int *bc = A.bar_count, *bg = A.bar_gen;

    // ---- grid levels --------------------------------------------------
    // Chebyshev step j on level k: d_j on the halo from buffer par, then
    // X += d_j, r_{j+1} = r_j - A d_j into buffer 1 - par.  last: apply
    // step j + 1 too (pointwise) and leave the final correction in xpost.
    auto cheb = [&](int k, int j, int par, bool post, bool last) {
        const MGLevel<T> &V = H.lv[k];
        T *const *X = post ? V.xpost : V.xpre;
        const T c1 = H.c1[j], c2 = H.c2[j], n1 = H.c1[j + 1], n2 = H.c2[j + 1];
        mg_sweep<T, TX, TY, false>(
            V.nx, V.ny, V.lam, V.mu, bid, nbk, su, sl, sm, scell, nullptr,
            [&](int gx, int gy, T (&v)[2]) {
                const int g = gx + V.nx * gy;
                const T di = c2 * __ldcg(V.dinv + g);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    T a = di * __ldcg(V.r[par][c] + g);
                    if (j > 0) a += c1 * __ldcg(V.d[par][c] + g);
                    v[c] = a;
                }
            },
            [&](int n, const T (&v)[2], const T (&q)[2], const T (&)[3]) {
                const T di = last ? n2 * __ldcg(V.dinv + n) : T(0);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const T x = __ldcg(X[c] + n) + v[c];
                    const T rn = __ldcg(V.r[par][c] + n) - q[c];
                    if (last) {
                        V.xpost[c][n] = x + (n1 * v[c] + di * rn);
                    } else {
                        X[c][n] = x;
                        V.r[1 - par][c][n] = rn;
                        V.d[1 - par][c][n] = v[c];
                    }
                }
            });
    };
    // restriction (transpose of bilinear prolongation) of grid level k-1's
    // residual after its pre-smoothing, at node (gx, gy) of level k
    auto restrict_g = [&](int k, int gx, int gy, T (&f)[2]) {
        const MGLevel<T> &F = H.lv[k - 1];
        const int pf = H.deg[k - 1] & 1;
        f[0] = T(0);
        f[1] = T(0);
#pragma unroll
        for (int b = -1; b <= 1; b++) {
            const int fy = wrap(2 * gy + b, F.ny);
            const T wy = b == 0 ? T(1) : T(0.5);
#pragma unroll
            for (int a = -1; a <= 1; a++) {
                const int i = wrap(2 * gx + a, F.nx) + F.nx * fy;
                const T w = wy * (a == 0 ? T(1) : T(0.5));
                f[0] += w * __ldcg(F.r[pf][0] + i);
                f[1] += w * __ldcg(F.r[pf][1] + i);
            }
        }
    };
    // first pre-smoothing sweep of a grid level k >= 1: f = R r_{k-1}, x = d_0
    auto pre_first = [&](int k) {
        const MGLevel<T> &V = H.lv[k];
        const T c2 = H.c2[0];
        mg_sweep<T, TX, TY, false>(
            V.nx, V.ny, V.lam, V.mu, bid, nbk, su, sl, sm, scell, nullptr,
            [&](int gx, int gy, T (&v)[2]) {
                T f[2];
                restrict_g(k, gx, gy, f);
                const T di = c2 * __ldcg(V.dinv + gx + V.nx * gy);
                v[0] = di * f[0];
                v[1] = di * f[1];
            },
            [&](int n, const T (&v)[2], const T (&q)[2], const T (&)[3]) {
                T f[2];
                restrict_g(k, n % V.nx, n / V.nx, f);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    V.f[c][n] = f[c];
                    V.xpre[c][n] = v[c];
                    V.r[1][c][n] = f[c] - q[c];
                    V.d[1][c][n] = v[c];
                }
            });
    };
    // first post-smoothing sweep of grid level k: x = x_pre + P e_{k+1}
    // (e: level k+1's final correction), r = f - A x; last (one-step
    // smoothing): apply that step, x + c2[0] D^-1 r, as the final correction
    auto post_first = [&](int k, int par, int cur, bool last) {
        const MGLevel<T> &V = H.lv[k];
        const MGLevel<T> &C = H.lv[k + 1];
        mg_sweep<T, TX, TY, false>(
            V.nx, V.ny, V.lam, V.mu, bid, nbk, su, sl, sm, scell, nullptr,
            [&](int gx, int gy, T (&v)[2]) {
                const int g = gx + V.nx * gy;
                const int ox = gx & 1, oy = gy & 1, ix = gx >> 1, iy = gy >> 1;
                const T w = (ox && oy) ? T(0.25) : ((ox || oy) ? T(0.5) : T(1));
                const int ix1 = ox ? (ix + 1 == C.nx ? 0 : ix + 1) : ix, iy1 = oy ? (iy + 1 == C.ny ? 0 : iy + 1) : iy;
                const int c00 = ix + C.nx * iy, c10 = ix1 + C.nx * iy, c01 = ix + C.nx * iy1, c11 = ix1 + C.nx * iy1;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    T e = __ldcg(C.xpost[c] + c00);
                    if (ox) e += __ldcg(C.xpost[c] + c10);
                    if (oy) e += __ldcg(C.xpost[c] + c01);
                    if (ox && oy) e += __ldcg(C.xpost[c] + c11);
                    v[c] = __ldcg(V.xpre[c] + g) + w * e;
                }
            },
            [&](int n, const T (&v)[2], const T (&q)[2], const T (&)[3]) {
                const T di = last ? H.c2[0] * __ldcg(V.dinv + n) : T(0);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const T f = k == 0 ? __ldcg(A.r[cur][c] + n) : __ldcg(V.f[c] + n);
                    if (last) {
                        V.xpost[c][n] = v[c] + di * (f - q[c]);
                    } else {
                        V.xpost[c][n] = v[c];
                        V.r[1 - par][c][n] = f - q[c];
                    }
                }
            });
    };
    // Two-step smoothing of a grid level k >= 1 in one fused sweep (degree 2,
    // not the coarsest): pre-smoothing from f = R r_{k-1} (x = d_0 + d_1,
    // r_2 and d_1 into buffer 0, which the restriction to level k+1 reads),
    // and post-smoothing from x_pre + P e_{k+1} with the final correction
    // into xpost.
    T *s2 = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(sblk) + mg_pair_offset<T, TX, TY>());
    auto pre2 = [&](int k) {
        const MGLevel<T> &V = H.lv[k];
        const T c20 = H.c2[0], c11 = H.c1[1], c21 = H.c2[1];
        mg_sweep2<T, TX, TY, false>(
            V.nx, V.ny, V.lam, V.mu, bid, nbk, s2, nullptr,
            [&](int gx, int gy, T (&v)[2], T (&a)[2]) {
                restrict_g(k, gx, gy, a);
                const T di = c20 * __ldcg(V.dinv + gx + V.nx * gy);
                v[0] = di * a[0];
                v[1] = di * a[1];
            },
            [&](int g, const T (&v)[2], const T (&a)[2], const T (&q)[2], T (&r)[2], T (&w)[2]) {
                const T di = c21 * __ldcg(V.dinv + g);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    r[c] = a[c] - q[c];
                    w[c] = c11 * v[c] + di * r[c];
                }
            },
            [&](int n, const T (&v)[2], const T (&a)[2], const T (&r)[2], const T (&w)[2], const T (&q)[2],
                const T (&)[3]) {
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    V.f[c][n] = a[c];
                    V.xpre[c][n] = v[c] + w[c];
                    V.r[0][c][n] = r[c] - q[c];
                    V.d[0][c][n] = w[c];
                }
            });
    };
    auto post2 = [&](int k) {
        const MGLevel<T> &V = H.lv[k];
        const MGLevel<T> &C = H.lv[k + 1];
        const T c20 = H.c2[0], c11 = H.c1[1], c21 = H.c2[1];
        mg_sweep2<T, TX, TY, false>(
            V.nx, V.ny, V.lam, V.mu, bid, nbk, s2, nullptr,
            [&](int gx, int gy, T (&v)[2], T (&a)[2]) {
                const int g = gx + V.nx * gy;
                const int ox = gx & 1, oy = gy & 1, ix = gx >> 1, iy = gy >> 1;
                const T wgt = (ox && oy) ? T(0.25) : ((ox || oy) ? T(0.5) : T(1));
                const int ix1 = ox ? (ix + 1 == C.nx ? 0 : ix + 1) : ix, iy1 = oy ? (iy + 1 == C.ny ? 0 : iy + 1) : iy;
                const int c00 = ix + C.nx * iy, c10 = ix1 + C.nx * iy, c01 = ix + C.nx * iy1, c11i = ix1 + C.nx * iy1;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    T e = __ldcg(C.xpost[c] + c00);
                    if (ox) e += __ldcg(C.xpost[c] + c10);
                    if (oy) e += __ldcg(C.xpost[c] + c01);
                    if (ox && oy) e += __ldcg(C.xpost[c] + c11i);
                    v[c] = __ldcg(V.xpre[c] + g) + wgt * e;
                    a[c] = __ldcg(V.f[c] + g);
                }
            },
            [&](int g, const T (&v)[2], const T (&a)[2], const T (&q)[2], T (&r)[2], T (&w)[2]) {
                const T di = c20 * __ldcg(V.dinv + g);
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    r[c] = a[c] - q[c];
                    w[c] = di * r[c];
                }
            },
            [&](int n, const T (&v)[2], const T (&)[2], const T (&r)[2], const T (&w)[2], const T (&q)[2],
                const T (&)[3]) {
                const T di = c21 * __ldcg(V.dinv + n);
#pragma unroll
                for (int c = 0; c < 2; c++) V.xpost[c][n] = v[c] + w[c] + (c11 * w[c] + di * (r[c] - q[c]));
            });
    };
    // the fused form serves grid levels with two-step smoothing
    auto fused = [&](int k) { return k >= 1 && k < L - 1 && H.deg[k] == 2; };

    // post-smoothing of grid level k
    auto post = [&](int k, int cur) {
        if (fused(k)) {
            post2(k);
            return grid_sync(bc, bg, err, nbk);
        }
        const int dk = H.deg[k];
        int par = dk & 1;
        post_first(k, par, cur, dk == 1);
        if (!grid_sync(bc, bg, err, nbk)) return false;
        par ^= 1;
        for (int j = 0; j + 1 < dk; j++) {
            cheb(k, j, par, true, j + 2 == dk);
            if (!grid_sync(bc, bg, err, nbk)) return false;
            par ^= 1;
        }
        return true;
    };
    // pre-smoothing (or the coarsest solve, csteps >= 3) of grid level k >= 1
    auto pre = [&](int k) {
        if (fused(k)) {
            pre2(k);
            return grid_sync(bc, bg, err, nbk);
        }
        pre_first(k);
        if (!grid_sync(bc, bg, err, nbk)) return false;
        int par = 1;
        const bool co = k == L - 1;
        const int nk = co ? cs - 1 : H.deg[k];
        for (int j = 1; j < nk; j++) {
            cheb(k, j, par, false, co && j + 1 == nk);
            if (!grid_sync(bc, bg, err, nbk)) return false;
            par ^= 1;
        }
        return true;
    };

    // ---- block-run levels (first block, shared memory, in place) ----------
    const int nmax = Lgw < L ? H.lv[Lgw].nx * H.lv[Lgw].ny : 0;
    T *scr = bscratch<T>(sblk, H);
    auto bcheb = [&](int k, int j, bool last) {
        const BLevel<T> B = blevel<T>(sblk, H, k);
        const T c1 = H.c1[j], c2 = H.c2[j], n1 = H.c1[j + 1], n2 = H.c2[j + 1];
        blk_sweep<T>(
            B, scr, nmax,
            [&](int i, T (&v)[2]) {
                const T di = c2 * B.dinv[i];
#pragma unroll
                for (int c = 0; c < 2; c++) v[c] = di * B.r[c][i] + (j > 0 ? c1 * B.d[c][i] : T(0));
            },
            [&](int i, const T (&v)[2], const T (&q)[2]) {
                const T di = n2 * B.dinv[i];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const T x = B.x[c][i] + v[c];
                    const T rn = B.r[c][i] - q[c];
                    if (last) {
                        B.x[c][i] = x + (n1 * v[c] + di * rn);
                    } else {
                        B.x[c][i] = x;
                        B.r[c][i] = rn;
                        B.d[c][i] = v[c];
                    }
                }
            });
    };
    auto bpre = [&](int k) {
        const BLevel<T> B = blevel<T>(sblk, H, k);
        const T c2 = H.c2[0];
        const bool top = k == Lgw;
        blk_sweep<T>(
            B, scr, nmax,
            [&](int i, T (&v)[2]) {
                const int ix = i % B.nx, iy = i / B.nx;
                T f[2];
                if (top) {
                    restrict_g(k, ix, iy, f);
                } else {
                    const BLevel<T> F = blevel<T>(sblk, H, k - 1);
                    f[0] = T(0);
                    f[1] = T(0);
#pragma unroll
                    for (int b = -1; b <= 1; b++) {
                        const int fy = wrap(2 * iy + b, F.ny);
                        const T wy = b == 0 ? T(1) : T(0.5);
#pragma unroll
                        for (int a = -1; a <= 1; a++) {
                            const int fi = wrap(2 * ix + a, F.nx) + F.nx * fy;
                            const T w = wy * (a == 0 ? T(1) : T(0.5));
                            f[0] += w * F.r[0][fi];
                            f[1] += w * F.r[1][fi];
                        }
                    }
                }
                B.f[0][i] = f[0];
                B.f[1][i] = f[1];
                const T di = c2 * B.dinv[i];
                v[0] = di * f[0];
                v[1] = di * f[1];
            },
            [&](int i, const T (&v)[2], const T (&q)[2]) {
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    B.x[c][i] = v[c];
                    B.r[c][i] = B.f[c][i] - q[c];
                    B.d[c][i] = v[c];
                }
            });
        const bool co = k == L - 1;
        const int nk = co ? cs - 1 : H.deg[k];
        for (int j = 1; j < nk; j++) bcheb(k, j, co && j + 1 == nk);
    };
    auto bpost = [&](int k) {
        const int dk = H.deg[k];
        const BLevel<T> B = blevel<T>(sblk, H, k);
        const BLevel<T> C = blevel<T>(sblk, H, k + 1);
        blk_sweep<T>(
            B, scr, nmax,
            [&](int i, T (&v)[2]) {
                const int gx = i % B.nx, gy = i / B.nx;
                const int ox = gx & 1, oy = gy & 1, ix = gx >> 1, iy = gy >> 1;
                const T w = (ox && oy) ? T(0.25) : ((ox || oy) ? T(0.5) : T(1));
                const int ix1 = ox ? (ix + 1 == C.nx ? 0 : ix + 1) : ix, iy1 = oy ? (iy + 1 == C.ny ? 0 : iy + 1) : iy;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    T e = C.x[c][ix + C.nx * iy];
                    if (ox) e += C.x[c][ix1 + C.nx * iy];
                    if (oy) e += C.x[c][ix + C.nx * iy1];
                    if (ox && oy) e += C.x[c][ix1 + C.nx * iy1];
                    v[c] = B.x[c][i] + w * e;
                }
            },
            [&](int i, const T (&v)[2], const T (&q)[2]) {
                const T di = H.c2[0] * B.dinv[i];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const T rn = B.f[c][i] - q[c];
                    B.x[c][i] = dk == 1 ? v[c] + di * rn : v[c];
                    B.r[c][i] = rn;
                }
            });
        for (int j = 0; j + 1 < dk; j++) bcheb(k, j, j + 2 == dk);
    };

    if (bid == 0 && Lgw < L) mg_setup_block<T>(H, sblk);

    int cur = 0;
    bool first = true;
    while (true) {
        if (lead) {
            if (!first) cg_scalar_update<NV>(S);
            s_ta = (T)S.alpha;
            s_tb = (T)S.beta;
            for (int vv = 0; vv < NV; vv++) s_ue[vv] = (T)S.UE[vv];
        }
        __syncthreads();
        const T ta = s_ta, tb = s_tb;
        const int nxt = first ? cur : 1 - cur;

        // ---- finest level, first pre-smoothing sweep; from the second
        // iteration on its own nodes also take the CG update
        //   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s
        // (u: the previous V-cycle's result, in L0.xpost) and the halo uses
        // the updated r formed on the fly
        Acc<T> racc[1];
        {
            const T c2 = H.c2[0];
            mg_sweep<T, TX, TY, false>(
                L0.nx, L0.ny, L0.lam, L0.mu, bid, nbk, su, sl, sm, scell, nullptr,
                [&](int gx, int gy, T (&v)[2]) {
                    const int g = gx + L0.nx * gy;
                    const T di = c2 * __ldcg(L0.dinv + g);
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        T rv = __ldcg(A.r[cur][c] + g);
                        if (!first) rv -= ta * (__ldcg(A.w[cur][c] + g) + tb * __ldcg(A.s[cur][c] + g));
                        v[c] = di * rv;
                    }
                },
                [&](int n, const T (&v)[2], const T (&q)[2], const T (&)[3]) {
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        T f = __ldcg(A.r[cur][c] + n);
                        if (!first) {
                            const T si = __ldcg(A.w[cur][c] + n) + tb * __ldcg(A.s[cur][c] + n);
                            const T pi = __ldcg(L0.xpost[c] + n) + tb * A.p[c][n];
                            A.p[c][n] = pi;
                            A.x[c][n] = A.x[c][n] + ta * pi;
                            A.s[nxt][c][n] = si;
                            f = f - ta * si;
                            A.r[nxt][c][n] = f;
                            racc[0].fma_plain(f, f);
                        }
                        L0.xpre[c][n] = v[c];
                        L0.r[1][c][n] = f - q[c];
                        L0.d[1][c][n] = v[c];
                    }
                });
        }
        if (!first) {
            double tr[1];
            if (!reduce_barrier<Acc<T>, 1>(racc, A.partials, A.result, A.bar_count, A.bar_gen, err, tr, bid, nbk)) return -1;
            if (lead) {
                double rnew = tr[0];
                for (int vv = 0; vv < NV; vv++) rnew += S.RE[vv] * S.RE[vv];
                S.it++;
                S.rho_final = rnew;
                int ctl = CTL_RUN;
                if (rnew <= S.target * S.target) ctl = CTL_DONE;
                else if (S.it_total + S.it >= A.maxit) ctl = CTL_STOP;
                s_ctl = ctl;
            }
            __syncthreads();
            cur = nxt;
            const int ctl = s_ctl;
            if (ctl != CTL_RUN) return ctl;
        } else if (!grid_sync(bc, bg, err, nbk)) {
            return -1;
        }

        // ---- rest of the V-cycle
        {
            int par = 1;
            const int n0 = L == 1 ? cs - 1 : H.deg[0];
            for (int j = 1; j < n0; j++) {
                cheb(0, j, par, false, L == 1 && j + 1 == n0);
                if (!grid_sync(bc, bg, err, nbk)) return -1;
                par ^= 1;
            }
        }
        for (int k = 1; k < Lgw; k++)
            if (!pre(k)) return -1;
        if (Lgw < L) {
            if (bid == 0) {
                for (int k = Lgw; k < L; k++) bpre(k);
                for (int k = L - 2; k >= Lgw; k--) bpost(k);
                // the top block-run level's correction, for the grid level above
                const BLevel<T> B = blevel<T>(sblk, H, Lgw);
                for (int i = threadIdx.x; i < B.n; i += blockDim.x) {
                    H.lv[Lgw].xpost[0][i] = B.x[0][i];
                    H.lv[Lgw].xpost[1][i] = B.x[1][i];
                }
            }
            if (!grid_sync(bc, bg, err, nbk)) return -1;
        }
        // the finest level's one-step post-smoothing fuses with the next sweep
        const bool fuse0 = L > 1 && H.deg[0] == 1;
        for (int k = (Lgw < L - 1 ? Lgw : L - 1) - 1; k >= (fuse0 ? 1 : 0); k--)
            if (!post(k, cur)) return -1;

        // ---- u = V-cycle result, w = A u (+ mean strain), gamma, delta, mean-strain row
        Acc<T> acc[2 + NV];
        if (fuse0) {
            // x = x_pre + P e_1, r = f - A x (f: the CG residual), u = x + c2[0] D^-1 r
            // on the width-1 ring, then w = A u on the tile
            const MGLevel<T> &C = H.lv[1];
            const T c20 = H.c2[0];
            mg_sweep2<T, TX, TY, true>(
                L0.nx, L0.ny, L0.lam, L0.mu, bid, nbk,
                reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(sblk) + mg_pair_offset<T, TX, TY>()), s_ue,
                [&](int gx, int gy, T (&v)[2], T (&a)[2]) {
                    const int g = gx + L0.nx * gy;
                    const int ox = gx & 1, oy = gy & 1, ix = gx >> 1, iy = gy >> 1;
                    const T wgt = (ox && oy) ? T(0.25) : ((ox || oy) ? T(0.5) : T(1));
                    const int ix1 = ox ? (ix + 1 == C.nx ? 0 : ix + 1) : ix, iy1 = oy ? (iy + 1 == C.ny ? 0 : iy + 1) : iy;
                    const int c00 = ix + C.nx * iy, c10 = ix1 + C.nx * iy, c01 = ix + C.nx * iy1, c11 = ix1 + C.nx * iy1;
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        T e = __ldcg(C.xpost[c] + c00);
                        if (ox) e += __ldcg(C.xpost[c] + c10);
                        if (oy) e += __ldcg(C.xpost[c] + c01);
                        if (ox && oy) e += __ldcg(C.xpost[c] + c11);
                        v[c] = __ldcg(L0.xpre[c] + g) + wgt * e;
                        a[c] = __ldcg(A.r[cur][c] + g);
                    }
                },
                [&](int g, const T (&v)[2], const T (&a)[2], const T (&q)[2], T (&r)[2], T (&w)[2]) {
                    const T di = c20 * __ldcg(L0.dinv + g);
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        r[c] = a[c] - q[c];
                        w[c] = v[c] + di * r[c];
                    }
                },
                [&](int n, const T (&)[2], const T (&a)[2], const T (&)[2], const T (&u)[2], const T (&q)[2],
                    const T (&se)[3]) {
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        L0.xpost[c][n] = u[c];
                        A.w[cur][c][n] = q[c];
                        acc[0].fma_plain(a[c], u[c]);
                        acc[1].fma_plain(q[c], u[c]);
                    }
#pragma unroll
                    for (int vv = 0; vv < NV; vv++) acc[2 + vv].add_plain(se[vv]);
                });
        } else {
            mg_sweep<T, TX, TY, true>(
                L0.nx, L0.ny, L0.lam, L0.mu, bid, nbk, su, sl, sm, scell, s_ue,
                [&](int gx, int gy, T (&v)[2]) {
                    const int g = gx + L0.nx * gy;
                    v[0] = __ldcg(L0.xpost[0] + g);
                    v[1] = __ldcg(L0.xpost[1] + g);
                },
                [&](int n, const T (&v)[2], const T (&q)[2], const T (&se)[3]) {
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        A.w[cur][c][n] = q[c];
                        acc[0].fma_plain(__ldcg(A.r[cur][c] + n), v[c]);
                        acc[1].fma_plain(q[c], v[c]);
                    }
#pragma unroll
                    for (int vv = 0; vv < NV; vv++) acc[2 + vv].add_plain(se[vv]);
                });
        }
        double tt[2 + NV];
        if (!reduce_barrier<Acc<T>, 2 + NV>(acc, A.partials, A.result, A.bar_count, A.bar_gen, err, tt, bid, nbk)) return -1;
        if (lead) {
            double s6[6];
            dmat_mul<2>(S.Sl, S.Sm, S.UE, s6);
            for (int vv = 0; vv < NV; vv++) S.WE[vv] = tt[2 + vv] + s6[vv];
            double gnew = tt[0], dnew = tt[1];
            for (int vv = 0; vv < NV; vv++) {
                gnew += S.RE[vv] * S.UE[vv];
                dnew += S.WE[vv] * S.UE[vv];
            }
            cg_take_gamma_delta(S, gnew, dnew, first);
        }
        first = false;
    }
}

}  // namespace pfdev
