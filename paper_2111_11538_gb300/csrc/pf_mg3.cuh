// Geometric multigrid preconditioner of the 3D solve: the V-cycle of
// pf_mg.cuh on periodic Q1 hex grids.  Each coarse level halves all three
// sizes; a coarse cell's moduli are the mean of its 2x2x2 fine cells times 2
// (the unit-cell element tables are used on every level, and a hex element's
// stiffness grows linearly with its edge, so that the rediscretised coarse
// operator matches the fine one under trilinear prolongation); restriction
// is the transpose of trilinear prolongation (27 fine nodes per coarse
// node).  The Chebyshev bound is the largest eigenvalue of diag(K_e)^-1 K_e
// of the 3D element.  All levels run on the whole grid, one tiled sweep of
// the operator (the exact cell decomposition of cell_force3 / node_force3)
// and one grid barrier per Chebyshev step; the CG update and the last step
// of each smoothing are folded into neighbouring sweeps as in 2D.  Data
// written by other blocks is read only after the grid barrier that follows
// the write (an acquire at GPU scope), so such loads may be cached in L1:
// the epilogues' operands are prefetched into L1 when a plane's work begins,
// and the restriction and prolongation gathers, which read each value from
// several neighbouring nodes, go through L1.
#pragma once

namespace pfdev {

// Double-single number (hi + lo, two floats, ~48 significant bits): the
// arithmetic of the mixed method's residual sweep, which needs about FP64
// accuracy and gets it from the FP32 pipes (GB300 runs FP64 at 1/64 of the
// FP32 rate).  Sums are error-free transformations (Knuth's two-sum,
// Dekker's fast two-sum), products take their rounding error from an FMA;
// the relative error of a sum or product is ~2^-44 of its operands, against
// FP64's 2^-53.
struct DS {
    float hi, lo;
    __host__ __device__ __forceinline__ DS() {}
    __host__ __device__ __forceinline__ DS(int x) : hi((float)x), lo(0.f) {}
    __host__ __device__ __forceinline__ DS(float x) : hi(x), lo(0.f) {}
    __host__ __device__ __forceinline__ DS(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ __forceinline__ DS(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ DS ds_fast(float a, float b)
{
    const float s = a + b;
    return DS(s, b - (s - a));
}
__device__ __forceinline__ DS operator+(DS x, DS y)
{
    const float s = x.hi + y.hi, v = s - x.hi;
    const float e = (x.hi - (s - v)) + (y.hi - v) + (x.lo + y.lo);
    return ds_fast(s, e);
}
__device__ __forceinline__ DS operator-(DS x) { return DS(-x.hi, -x.lo); }
__device__ __forceinline__ DS operator-(DS x, DS y) { return x + (-y); }
__device__ __forceinline__ DS operator*(DS x, DS y)
{
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p) + (x.hi * y.lo + x.lo * y.hi);
    return ds_fast(p, e);
}
__device__ __forceinline__ DS &operator+=(DS &x, DS y) { x = x + y; return x; }

// Shared-memory storage of 3-vectors: FP32 as one float4 per entry (one
// 128-bit access), FP64 and double-single as three planes of n values.
// WORDS values of T per entry.
template <typename T> struct V3S;
template <> struct V3S<float> {
    static constexpr int WORDS = 4;
    __device__ static __forceinline__ void st(float *b, int, int i, const float (&v)[3])
    {
        reinterpret_cast<float4 *>(b)[i] = make_float4(v[0], v[1], v[2], 0.f);
    }
    __device__ static __forceinline__ void ld(const float *b, int, int i, float (&v)[3])
    {
        const float4 a = reinterpret_cast<const float4 *>(b)[i];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
    }
};
template <typename T> struct V3Planes {
    static constexpr int WORDS = 3;
    __device__ static __forceinline__ void st(T *b, int n, int i, const T (&v)[3])
    {
        b[i] = v[0];
        b[n + i] = v[1];
        b[2 * n + i] = v[2];
    }
    __device__ static __forceinline__ void ld(const T *b, int n, int i, T (&v)[3])
    {
        v[0] = b[i];
        v[1] = b[n + i];
        v[2] = b[2 * n + i];
    }
};
template <> struct V3S<double> : V3Planes<double> {};
template <> struct V3S<DS> : V3Planes<DS> {};

// Forces of a 3D cell on its eight corner nodes, f[a][comp] with
// a = ax + 2 ay + 4 az, from its average stress s (mean strain included) and
// hourglass forces g (cell_force3).  This is node_force3 at every corner,
// factored: per component the corner value is a sum of the terms sx, sy, sz,
// sx sy, sy sz, sz sx and sx sy sz (s_i = +1 at the upper corner along axis
// i, -1 at the lower) with the coefficients below, and the eight sign
// patterns are formed by sums and differences.
template <typename TC>
__device__ __forceinline__ void corner_forces3(const TC *s, const TC *g, TC (&f)[8][3])
{
    constexpr int SXI[3] = {0, 5, 4}, SYI[3] = {5, 1, 3}, SZI[3] = {4, 3, 2};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const TC ax = TC(0.25) * s[SXI[k]], ay = TC(0.25) * s[SYI[k]], az = TC(0.25) * s[SZI[k]];
        const TC axy = TC(0.5) * g[k], ayz = TC(0.5) * g[3 + k], azx = TC(0.5) * g[6 + k], axyz = g[9 + k];
        const TC p1 = ay + ayz, p2 = ay - ayz, o1 = ax + azx, o2 = ax - azx, q1 = axy + axyz, q2 = axy - axyz;
        // (sy, sz) = (+, +), (-, +), (+, -), (-, -): even part E, odd part O in sx
        const TC Epp = p1 + az, Emp = az - p1, Epm = p2 - az, Emm = -(p2 + az);
        const TC Opp = o1 + q1, Omp = o1 - q1, Opm = o2 + q2, Omm = o2 - q2;
        f[7][k] = Epp + Opp;  f[6][k] = Epp - Opp;     // ay = 1, az = 1
        f[5][k] = Emp + Omp;  f[4][k] = Emp - Omp;     // ay = 0, az = 1
        f[3][k] = Epm + Opm;  f[2][k] = Epm - Opm;     // ay = 1, az = 0
        f[1][k] = Emm + Omm;  f[0][k] = Emm - Omm;     // ay = 0, az = 0
    }
}

// Tile of the z-marching 3D sweep: TX x TY nodes per plane, one thread each.
constexpr int MGZ_TX = 32, MGZ_TY = 8, MGZ_NP = (MGZ_TX + 2) * (MGZ_TY + 2);
// Streams (arrays read at a staged node) a sweep's operand is formed from,
// at most; and whether they are copied into shared memory one plane ahead
// (asynchronous copies, FP32) or read when the plane is staged (FP64, whose
// sweeps are bound by the FP64 pipe rather than by memory latency).
constexpr int MGZ_NS = 10;
template <typename T> struct MGZPipe { static constexpr bool on = sizeof(T) == 4; static constexpr int RB = on ? 2 : 1; };

// Shared memory (values of T) of mg_sweep3z with at most ns raw streams: two
// node planes, the eight corner forces of one cell plane with their halos,
// the staged nodes' raw streams (two planes when they are copied ahead,
// PIPE) and, in FP32, the cell moduli of three planes.
template <typename T, bool PIPE = MGZPipe<T>::on>
__host__ __device__ constexpr int mg_sweep3z_words(int ns = MGZ_NS)
{
    return V3S<T>::WORDS * (2 * (MGZ_TX + 2) * (MGZ_TY + 2) + 8 * (MGZ_TX + 1) * (MGZ_TY + 1)) +
           (PIPE ? 2 : 1) * ns * (MGZ_TX + 2) * (MGZ_TY + 2) +
           (PIPE && sizeof(T) == 4 ? 6 * (MGZ_TX + 1) * (MGZ_TY + 1) : 0);
}

// z-chunk of the 3D sweep on an nx x ny x nz level with nbk blocks: the
// candidate that minimises (work items per block, rounded up) x (planes per
// item + 1), ties to the longer chunk.
__device__ __forceinline__ int mg_zchunk(int nx, int ny, int nz, int nbk)
{
    const int ixy = ((nx + MGZ_TX - 1) / MGZ_TX) * ((ny + MGZ_TY - 1) / MGZ_TY);
    constexpr int cand[12] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    int best = nz;
    long long bcost = (long long)((ixy + nbk - 1) / nbk) * (nz + 1);
    for (int i = 0; i < 12; i++) {
        const int zc = cand[i];
        if (zc >= nz) break;
        const long long items = (long long)ixy * ((nz + zc - 1) / zc);
        const long long cost = ((items + nbk - 1) / nbk) * (zc + 1);
        if (cost <= bcost) {
            bcost = cost;
            best = zc;
        }
    }
    return best;
}

// One 3D sweep of the level's Q1 operator, marching along z.  A work item is
// a TX x TY column of node tiles over zc planes.  Per cell plane zp: the node
// plane zp + 1 (with its one-node halo in x and y) is formed by
// make(raw, h, gx, gy, gz, v) from its ns raw streams src[0 .. ns) (FP32:
// copied into shared memory one plane ahead, so that their latency overlaps
// the previous plane's work; raw[s * NP + h] is stream s at staged node h),
// every cell of the plane (with the halo cells at x0 - 1, y0 - 1) computes
// its average stress and hourglass forces once (cell_force3; its moduli, of
// type TM, are copied with the raw streams two planes ahead in FP32 and read
// one plane ahead in FP64; PIPE: the raw streams are copied into shared
// memory one plane ahead, the default in FP32) and its forces on its eight
// corners
// (corner_forces3), and each own node of plane zp adds its bottom-corner
// forces to the top-corner forces left by plane zp - 1: q = A v is complete
// and epi(n, v, q) receives it.  pref(n) runs for each own node of plane zp
// when the plane's work begins (before the node plane ahead is formed), so
// that the epilogue's operands can be fetched early.  WITH_E: the mean strain
// ue enters every cell's stress, and cell_e(c) receives the stress of every
// own cell without it (c[0..5]).  smem: mg_sweep3z_words<T>(ns) values; src:
// ns pointers (shared memory, set by the caller); two block barriers per
// plane.
template <typename T, bool WITH_E, bool PIPE_ = MGZPipe<T>::on, class TM, class Make, class Epi, class CellE,
          class Pref>
__device__ __forceinline__ void mg_sweep3z(int nx, int ny, int nz, int zc, const TM *lam, const TM *mu, int bid,
                                           int nbk, T *smem, const T *ue, int ns, const T *const *src, Make &&make,
                                           Epi &&epi, CellE &&cell_e, Pref &&pref)
{
    constexpr int TX = MGZ_TX, TY = MGZ_TY;
    constexpr int NX = TX + 2, NY = TY + 2, NP = NX * NY;
    constexpr int CX = TX + 1, CY = TY + 1, NC = CX * CY, NT = TX * TY;
    constexpr int W = V3S<T>::WORDS;
    constexpr bool PIPE = PIPE_, MODC = PIPE && sizeof(T) == 4;   // copied raw streams / moduli
    constexpr int CPT = (NC + NT - 1) / NT;                 // cells per thread
    T *const np0 = smem, *const np1 = smem + W * NP, *const cf = smem + 2 * W * NP;
    T *const rawb = cf + 8 * W * NC;                        // [PIPE ? 2 : 1][ns][NP]
    T *const modb = rawb + 2 * MGZ_NS * NP;                  // MODC: [3][lam, mu][NC]
    static_assert(!MODC || std::is_same<TM, T>::value, "copied moduli have the sweep's type");
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, nzc = (nz + zc - 1) / zc;
    const int items = ntx * nty * nzc;
    const bool small = nx < NX || ny < NY;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    auto zwrap = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
    for (int item = bid; item < items; item += nbk) {
        const int x0 = (item % ntx) * TX, y0 = ((item / ntx) % nty) * TY, z0 = (item / (ntx * nty)) * zc;
        const int z1 = min(z0 + zc, nz);
        const int gx = x0 + tx, gy = y0 + ty;
        const bool own = gx < nx && gy < ny;
        auto raw_of = [&](int z) { return rawb + (PIPE ? (z & 1) : 0) * (ns * NP); };
        // raw streams of node plane z: asynchronous copies (FP32) or loads
        auto issue = [&](int z) {
            const int zw = zwrap(z);
            T *raw = raw_of(z);
            for (int h = threadIdx.x; h < NP; h += NT) {
                const int lx = h % NX, ly = h / NX;
                const int g = mg_wrap(x0 - 1 + lx, nx, small) + nx * (mg_wrap(y0 - 1 + ly, ny, small) + ny * zw);
                for (int q = 0; q < ns; q++) {
                    if constexpr (PIPE) cp_async(raw + q * NP + h, src[q] + g);
                    else raw[q * NP + h] = __ldcg(src[q] + g);
                }
            }
            if constexpr (MODC) {
                // the moduli of this thread's cells of plane z (read by this
                // thread only)
                T *md = modb + ((z + 3) % 3) * 2 * NC;
#pragma unroll
                for (int u = 0; u < CPT; u++) {
                    const int h = threadIdx.x + u * NT;
                    if (h < NC) {
                        const int cx = h % CX, cy = h / CX;
                        const int g = mg_wrap(x0 - 1 + cx, nx, small) + nx * (mg_wrap(y0 - 1 + cy, ny, small) + ny * zw);
                        cp_async(md + h, reinterpret_cast<const T *>(lam) + g);
                        cp_async(md + NC + h, reinterpret_cast<const T *>(mu) + g);
                    }
                }
            }
        };
        // node plane z formed from its raw streams (each thread forms the
        // nodes whose streams it copied)
        auto form = [&](int z, T *buf) {
            const int zw = zwrap(z);
            const T *raw = raw_of(z);
            for (int h = threadIdx.x; h < NP; h += NT) {
                const int lx = h % NX, ly = h / NX;
                T v[3];
                make(raw, h, mg_wrap(x0 - 1 + lx, nx, small), mg_wrap(y0 - 1 + ly, ny, small), zw, v);
                V3S<T>::st(buf, NP, h, v);
            }
        };
        // moduli of this thread's cells of plane z (FP64: into registers)
        auto moduli = [&](int z, T (&l)[CPT], T (&m)[CPT]) {
            const int zw = zwrap(z);
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                const int h = threadIdx.x + u * NT;
                if (h < NC) {
                    const int cx = h % CX, cy = h / CX;
                    const int g = mg_wrap(x0 - 1 + cx, nx, small) + nx * (mg_wrap(y0 - 1 + cy, ny, small) + ny * zw);
                    l[u] = (T)__ldcg(lam + g);
                    m[u] = (T)__ldcg(mu + g);
                }
            }
        };
        issue(z0 - 1);
        if constexpr (PIPE) {
            cp_async_commit();
            issue(z0);
            cp_async_commit();
            cp_async_wait<1>();
        }
        form(z0 - 1, ((z0 - 1) & 1) ? np1 : np0);
        T lc[CPT], mc[CPT];
        if constexpr (!MODC) moduli(z0 - 1, lc, mc);
        T qt[3] = {T(0), T(0), T(0)};     // top-corner forces of the previous cell plane on the own node
        for (int zp = z0 - 1; zp < z1; zp++) {
            T *const nlo = (zp & 1) ? np1 : np0;
            T *const nhi = (zp & 1) ? np0 : np1;
            if (own && zp >= z0) pref(gx + nx * (gy + ny * zp));
            if constexpr (PIPE) {
                // copies of plane zp + 2 go out; plane zp + 1's have landed
                if (zp + 2 <= z1) issue(zp + 2);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                issue(zp + 1);
            }
            form(zp + 1, nhi);
            T ln[CPT], mn[CPT];
            if constexpr (!MODC)
                if (zp + 1 < z1) moduli(zp + 1, ln, mn);
            __syncthreads();
            const bool inner = zp >= z0;
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                const int h = threadIdx.x + u * NT;
                if (h >= NC) continue;
                const int cx = h % CX, cy = h / CX;
                const T *md = modb + ((zp + 3) % 3) * 2 * NC;
                const T l = MODC ? md[h] : lc[u], m = MODC ? md[NC + h] : mc[u];
                T uc[8][3];
#pragma unroll
                for (int b = 0; b < 8; b++) V3S<T>::ld((b >> 2) ? nhi : nlo, NP, (cx + (b & 1)) + NX * (cy + ((b >> 1) & 1)), uc[b]);
                T c[20];
                cell_force3<T>(l, m, uc, c);
                if constexpr (WITH_E) {
                    if (inner && cx >= 1 && cy >= 1 && x0 + cx - 1 < nx && y0 + cy - 1 < ny) cell_e(c);
                    T sx[6];
                    voigt_stress<T, 3>(l, m, ue, sx);
#pragma unroll
                    for (int v = 0; v < 6; v++) c[v] += sx[v];
                }
                T f[8][3];
                corner_forces3<T>(c, c + 6, f);
#pragma unroll
                for (int a = 0; a < 8; a++) V3S<T>::st(cf + a * W * NC, NC, h, f[a]);
            }
            T un[3];
            if (own && inner) V3S<T>::ld(nlo, NP, (tx + 1) + NX * (ty + 1), un);
            if constexpr (!MODC) {
                if (zp + 1 < z1) {
#pragma unroll
                    for (int u = 0; u < CPT; u++) { lc[u] = ln[u]; mc[u] = mn[u]; }
                }
            }
            __syncthreads();
            if (own) {
                // cells around the node in this plane: (tx, ty) is its lower-left
                // neighbour (the node is that cell's corner ax = ay = 1)
                const int c11 = tx + CX * ty, c01 = c11 + 1, c10 = c11 + CX, c00 = c10 + 1;
                T fb[3], ft[3], v[3];
                V3S<T>::ld(cf + 3 * W * NC, NC, c11, fb);
                V3S<T>::ld(cf + 7 * W * NC, NC, c11, ft);
#pragma unroll
                for (int k = 0; k < 3; k++) { fb[k] += qt[k]; }
                V3S<T>::ld(cf + 2 * W * NC, NC, c01, v);
#pragma unroll
                for (int k = 0; k < 3; k++) fb[k] += v[k];
                V3S<T>::ld(cf + 6 * W * NC, NC, c01, v);
#pragma unroll
                for (int k = 0; k < 3; k++) ft[k] += v[k];
                V3S<T>::ld(cf + 1 * W * NC, NC, c10, v);
#pragma unroll
                for (int k = 0; k < 3; k++) fb[k] += v[k];
                V3S<T>::ld(cf + 5 * W * NC, NC, c10, v);
#pragma unroll
                for (int k = 0; k < 3; k++) ft[k] += v[k];
                V3S<T>::ld(cf + 0 * W * NC, NC, c00, v);
#pragma unroll
                for (int k = 0; k < 3; k++) fb[k] += v[k];
                V3S<T>::ld(cf + 4 * W * NC, NC, c00, v);
#pragma unroll
                for (int k = 0; k < 3; k++) { ft[k] += v[k]; qt[k] = ft[k]; }
                if (inner) epi(gx + nx * (gy + ny * zp), un, fb);
            }
        }
        if constexpr (PIPE) cp_async_wait<0>();
    }
}

// Coarse 3D level C from F (global memory): cell moduli = 2 x the mean of
// the 2x2x2 fine cells, Jacobi diagonal from the eight coarse cells around
// each node.  Threads t0, t0 + st, ... take the coarse nodes.
template <typename T>
__device__ void mg_coarsen3(const MGLevel<T> &F, const MGLevel<T> &C, long long t0, long long st)
{
    const long long n = (long long)C.nx * C.ny * C.nz;
    auto avg = [&](const T *a, int cx, int cy, int cz) {
        const long long i = 2 * cx + (long long)F.nx * (2 * cy + (long long)F.ny * (2 * cz));
        const long long sy = F.nx, sz = (long long)F.nx * F.ny;
        const T lo = (__ldcg(a + i) + __ldcg(a + i + 1)) + (__ldcg(a + i + sy) + __ldcg(a + i + sy + 1));
        const T hi = (__ldcg(a + i + sz) + __ldcg(a + i + sz + 1)) + (__ldcg(a + i + sz + sy) + __ldcg(a + i + sz + sy + 1));
        return T(0.25) * (lo + hi);      // 2 x the mean of eight
    };
    for (long long i = t0; i < n; i += st) {
        const int cx = (int)(i % C.nx), cy = (int)((i / C.nx) % C.ny), cz = (int)(i / ((long long)C.nx * C.ny));
        C.lam[i] = avg(F.lam, cx, cy, cz);
        C.mu[i] = avg(F.mu, cx, cy, cz);
        T dg = T(0);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const int ex = wrap(cx - (a & 1), C.nx), ey = wrap(cy - ((a >> 1) & 1), C.ny), ez = wrap(cz - (a >> 2), C.nz);
            dg += avg(F.lam, ex, ey, ez) * KdL<T, 3>() + avg(F.mu, ex, ey, ez) * KdM<T, 3>();
        }
        C.dinv[i] = T(1) / dg;
    }
}

// b = sum over the 8 cells around node n of Bbar^T sig* in double-single
// arithmetic (the unit cell's Bbar entries are +-1/4, so each product with an
// FP32 sig* is exact in FP32), the Jacobi diagonal (FP32: it only scales the
// preconditioner), and the own cell's sig*, lam, mu; FP32 storage.
__device__ __forceinline__ void node_rhs_ds3(const Params &P, long long n, const float *lam, const float *mu,
                                             const float *const *sig, double (&b)[3], double &dgn, double (&so)[6],
                                             double &lo, double &mo)
{
    int i, j, k;
    cell_coords<3>(P, n, i, j, k);
    DS bs[3] = {DS(0), DS(0), DS(0)};
    float dg = 0.f;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const long long c = lin<3>(P, i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1));
        const float l = lam[c], m = mu[c];
        dg += l * KdL<float, 3>() + m * KdM<float, 3>();
        float sv[6];
#pragma unroll
        for (int v = 0; v < 6; v++) sv[v] = sig[v][c];
        const float bx = Bb<float, 3>(a, 0), by = Bb<float, 3>(a, 1), bz = Bb<float, 3>(a, 2);
        bs[0] += (DS(bx * sv[0]) + DS(by * sv[5])) + DS(bz * sv[4]);
        bs[1] += (DS(by * sv[1]) + DS(bx * sv[5])) + DS(bz * sv[3]);
        bs[2] += (DS(bz * sv[2]) + DS(by * sv[3])) + DS(bx * sv[4]);
        if (a == 0) {
#pragma unroll
            for (int v = 0; v < 6; v++) so[v] = sv[v];
            lo = l;
            mo = m;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; d++) b[d] = bs[d].value();
    dgn = dg;
}

// The set-up sweep of one CG pass in 3D, on the z-marching sweep in FP64
// (cell stress and hourglass forces once per cell, corner forces gathered per
// node): b, the Jacobi diagonal, r = b - A x and the sums of the mean-strain
// rows (acc[0] ||b||^2, [1] ||r||^2, [2] sum lam, [3] sum mu, [4..9] sum
// sig*, [10..15] the cells' stress of x without the mean strain).  resid: a
// later refinement pass, which reads b from A.b64 and skips what does not
// change during a solve.  Its three raw streams (x) are copied one plane ahead
// like the FP32 sweeps' (8-byte asynchronous copies).  The mixed method runs
// the operator in double-single arithmetic (DS) on the FP32 pipes, the FP64
// method in FP64.  smem: mg_sweep3z_words<double, true>(3) doubles.
template <typename T>
__device__ void setup_march3(const PCGArgs<T, 3> &A, bool use_x, bool refine, bool resid, const double *xe,
                             double *smem, Acc<double> (&acc)[16], int bid, int nbk)
{
    const Params &P = A.P;
    auto node = [&](int n, const double (&ax)[3]) {
        double b[3];
        if (resid) {
#pragma unroll
            for (int c = 0; c < 3; c++) b[c] = __ldcg(A.b64[c] + n);
        } else {
            double so[6], dgn, lo, mo;
            if constexpr (sizeof(T) == 4) {
                node_rhs_ds3(P, n, A.lam, A.mu, A.sig, b, dgn, so, lo, mo);
            } else {
                double unused[3], unused6[6];
                node_setup<T, double, double, 3>(P, n, A.lam, A.mu, A.sig, A.x64, xe, false, b, unused, dgn, so,
                                                 unused6, lo, mo);
            }
            if (refine)
#pragma unroll
                for (int c = 0; c < 3; c++) A.b64[c][n] = b[c];
            A.dinv[n] = (T)(1.0 / dgn);
            acc[2].add(lo);
            acc[3].add(mo);
#pragma unroll
            for (int v = 0; v < 6; v++) acc[4 + v].add(so[v]);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double rv = b[d] - ax[d];
            if (refine && !use_x) A.x64[d][n] = 0.0;
            if (refine || !use_x) A.x[d][n] = T(0);
            A.p[d][n] = T(0);
            A.s[0][d][n] = T(0);
            A.r[0][d][n] = (T)rv;
            if (!resid) acc[0].addprod(b[d], b[d]);
            acc[1].addprod(rv, rv);
        }
    };
    if (!use_x) {
        const long long t0 = bid * (long long)blockDim.x + threadIdx.x, st = (long long)nbk * blockDim.x;
        const double zero[3] = {0.0, 0.0, 0.0};
        for (long long n = t0; n < P.N; n += st) node((int)n, zero);
        return;
    }
    if constexpr (sizeof(T) == 4) {
        // mixed method: the sweep in double-single arithmetic; x64 is copied
        // as 8-byte words and split into hi + lo when its node plane is formed
        __shared__ DS s_xd[6];
        __shared__ const DS *s_xsd[3];
        if (threadIdx.x == 0) {
            for (int v = 0; v < 6; v++) s_xd[v] = DS(xe[v]);
            for (int c = 0; c < 3; c++) s_xsd[c] = reinterpret_cast<const DS *>(A.x64[c]);
        }
        __syncthreads();
        mg_sweep3z<DS, true, true>(
            P.nx, P.ny, P.nz, mg_zchunk(P.nx, P.ny, P.nz, nbk), A.lam, A.mu, bid, nbk, reinterpret_cast<DS *>(smem),
            s_xd, 3, s_xsd,
            [&](const DS *raw, int h, int, int, int, DS (&v)[3]) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    double x;
                    memcpy(&x, raw + c * MGZ_NP + h, sizeof(double));
                    v[c] = DS(x);
                }
            },
            [&](int n, const DS (&)[3], const DS (&q)[3]) {
                const double qd[3] = {q[0].value(), q[1].value(), q[2].value()};
                node(n, qd);
            },
            [&](const DS *c) {
#pragma unroll
                for (int v = 0; v < 6; v++) acc[10 + v].add(c[v].value());
            },
            [](int) {});
    } else {
        // x: the solution itself (FP64 method)
        __shared__ const double *s_xs[3];
        if (threadIdx.x == 0)
            for (int c = 0; c < 3; c++) s_xs[c] = refine ? A.x64[c] : reinterpret_cast<const double *>(A.x[c]);
        __syncthreads();
        mg_sweep3z<double, true, true>(
            P.nx, P.ny, P.nz, mg_zchunk(P.nx, P.ny, P.nz, nbk), A.lam, A.mu, bid, nbk, smem, xe, 3, s_xs,
            [&](const double *raw, int h, int, int, int, double (&v)[3]) {
#pragma unroll
                for (int c = 0; c < 3; c++) v[c] = raw[c * MGZ_NP + h];
            },
            [&](int n, const double (&)[3], const double (&q)[3]) { node(n, q); },
            [&](const double *c) {
#pragma unroll
                for (int v = 0; v < 6; v++) acc[10 + v].add(c[v]);
            },
            [](int) {});
    }
}

// Set-up of the 3D hierarchy at the start of a solve (grid levels, a barrier
// after each).  Returns false if a barrier timed out.
template <typename T>
__device__ bool mg_setup3(const MGHier<T> &H, unsigned int *bc, unsigned int *bg, int *err, int bid, int nbk)
{
    const long long t0 = bid * (long long)blockDim.x + threadIdx.x, st = (long long)nbk * blockDim.x;
    for (int k = 1; k < H.L; k++) {
        mg_coarsen3<T>(H.lv[k - 1], H.lv[k], t0, st);
        if (!grid_sync(bc, bg, err, nbk)) return false;
    }
    return true;
}

// One pass of MG-preconditioned CG in 3D: as mg_pass (pf_mg.cuh), every
// level on the whole grid.  scell: 20 * HC values of dynamic shared memory.
// Returns CTL_DONE or CTL_STOP, or -1 when a barrier timed out.
template <typename T>
__device__ int mg_pass3(const PCGArgs<T, 3> &A, const MGHier<T> &H, PCGState &S, T *smem, T &s_ta, T &s_tb,
                        T *s_ue, int &s_ctl, int bid, int nbk, int *err)
{
    constexpr int NV = 6;
    const bool lead = threadIdx.x == 0;
    const int L = H.L, cs = H.csteps;
    const MGLevel<T> &L0 = H.lv[0];
    unsigned int *bc = A.bar_count, *bg = A.bar_gen;
    auto sync = [&]() { return grid_sync(bc, bg, err, nbk); };
    auto lin3 = [](const MGLevel<T> &V, int x, int y, int z) { return x + V.nx * (y + V.ny * z); };
    // z-chunk of every level's sweeps for this job's blocks
    __shared__ int s_zc[MG_MAX_LEVELS];
    if (lead)
        for (int k = 0; k < L; k++) s_zc[k] = mg_zchunk(H.lv[k].nx, H.lv[k].ny, H.lv[k].nz, nbk);
    __syncthreads();
    auto none = [](const T *) {};
    // the streams of the next sweep (shared memory; every sweep is preceded
    // by a grid or block barrier after its streams are set)
    __shared__ const T *s_src[MGZ_NS];
    auto sweep = [&](int k, int ns, auto &&setsrc, auto &&make, auto &&epi, auto &&pref) {
        const MGLevel<T> &V = H.lv[k];
        if (lead) setsrc(s_src);
        __syncthreads();
        mg_sweep3z<T, false>(V.nx, V.ny, V.nz, s_zc[k], V.lam, V.mu, bid, nbk, smem, nullptr, ns, s_src, make, epi, none,
                             pref);
    };
    auto nopref = [](int) {};
    constexpr int NP = MGZ_NP;

    // Chebyshev step j on level k (buffer par -> 1 - par); last: also apply
    // step j + 1 and leave the final correction in xpost
    auto cheb = [&](int k, int j, int par, bool post, bool last) {
        const MGLevel<T> &V = H.lv[k];
        T *const *X = post ? V.xpost : V.xpre;
        const T c1 = H.c1[j], c2 = H.c2[j], n1 = H.c1[j + 1], n2 = H.c2[j + 1];
        sweep(k, j > 0 ? 7 : 4,
            [&](const T **src) {
                src[0] = V.dinv;
                for (int c = 0; c < 3; c++) { src[1 + c] = V.r[par][c]; src[4 + c] = V.d[par][c]; }
            },
            [&](const T *raw, int h, int, int, int, T (&v)[3]) {
                const T di = c2 * raw[h];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    T a = di * raw[(1 + c) * NP + h];
                    if (j > 0) a += c1 * raw[(4 + c) * NP + h];
                    v[c] = a;
                }
            },
            [&](int n, const T (&v)[3], const T (&q)[3]) {
                const T di = last ? n2 * __ldca(V.dinv + n) : T(0);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const T x = __ldca(X[c] + n) + v[c];
                    const T rn = __ldca(V.r[par][c] + n) - q[c];
                    if (last) {
                        V.xpost[c][n] = x + (n1 * v[c] + di * rn);
                    } else {
                        X[c][n] = x;
                        V.r[1 - par][c][n] = rn;
                        V.d[1 - par][c][n] = v[c];
                    }
                }
            },
            [&](int n) {
#pragma unroll
                for (int c = 0; c < 3; c++) { prefetch_l1(X[c] + n); prefetch_l1(V.r[par][c] + n); }
                if (last) prefetch_l1(V.dinv + n);
            });
    };
    // restriction (transpose of trilinear prolongation) of level k-1's
    // residual after its pre-smoothing, at node (gx, gy, gz) of level k
    auto restrict3 = [&](int k, int gx, int gy, int gz, T (&f)[3]) {
        const MGLevel<T> &F = H.lv[k - 1];
        const int pf = H.deg[k - 1] & 1;
        f[0] = f[1] = f[2] = T(0);
        for (int cz = -1; cz <= 1; cz++) {
            const int fz = wrap(2 * gz + cz, F.nz);
            const T wz = cz == 0 ? T(1) : T(0.5);
            for (int cy = -1; cy <= 1; cy++) {
                const int fy = wrap(2 * gy + cy, F.ny);
                const T wy = wz * (cy == 0 ? T(1) : T(0.5));
#pragma unroll
                for (int cx = -1; cx <= 1; cx++) {
                    const int i = lin3(F, wrap(2 * gx + cx, F.nx), fy, fz);
                    const T w = wy * (cx == 0 ? T(1) : T(0.5));
#pragma unroll
                    for (int c = 0; c < 3; c++) f[c] += w * __ldca(F.r[pf][c] + i);
                }
            }
        }
    };
    // first pre-smoothing sweep of level k >= 1: f = R r_{k-1}, x = d_0
    auto pre_first = [&](int k) {
        const MGLevel<T> &V = H.lv[k];
        const T c2 = H.c2[0];
        sweep(k, 1, [&](const T **src) { src[0] = V.dinv; },
            [&](const T *raw, int h, int gx, int gy, int gz, T (&v)[3]) {
                T f[3];
                restrict3(k, gx, gy, gz, f);
                const T di = c2 * raw[h];
                // the tile's own nodes keep f for their epilogue (a halo
                // plane's interior belongs to a neighbouring item, which
                // stores the same values)
                const int lx = h % (MGZ_TX + 2), ly = h / (MGZ_TX + 2);
                const bool inner = lx >= 1 && lx <= MGZ_TX && ly >= 1 && ly <= MGZ_TY;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    v[c] = di * f[c];
                    if (inner) V.f[c][lin3(V, gx, gy, gz)] = f[c];
                }
            },
            [&](int n, const T (&v)[3], const T (&q)[3]) {
                // f, stored by the forming of this plane (same block, before
                // the plane's barriers)
                T f[3];
#pragma unroll
                for (int c = 0; c < 3; c++) f[c] = __ldcg(V.f[c] + n);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    V.xpre[c][n] = v[c];
                    V.r[1][c][n] = f[c] - q[c];
                    V.d[1][c][n] = v[c];
                }
            },
            nopref);
    };
    // first post-smoothing sweep of level k: x = x_pre + P e_{k+1}, r = f - A x;
    // last (one-step smoothing): x + c2[0] D^-1 r is the final correction
    auto post_first = [&](int k, int par, int cur, bool last) {
        const MGLevel<T> &V = H.lv[k];
        const MGLevel<T> &C = H.lv[k + 1];
        sweep(k, 3, [&](const T **src) { for (int c = 0; c < 3; c++) src[c] = V.xpre[c]; },
            [&](const T *raw, int h, int gx, int gy, int gz, T (&v)[3]) {
                const int o[3] = {gx & 1, gy & 1, gz & 1}, ic[3] = {gx >> 1, gy >> 1, gz >> 1};
                const int nc[3] = {C.nx, C.ny, C.nz};
                int i1[3];
#pragma unroll
                for (int a = 0; a < 3; a++) i1[a] = o[a] ? (ic[a] + 1 == nc[a] ? 0 : ic[a] + 1) : ic[a];
                const T w = T(1) / T((1 + o[0]) * (1 + o[1]) * (1 + o[2]));
                T e[3] = {T(0), T(0), T(0)};
                for (int bz = 0; bz <= o[2]; bz++)
                    for (int by = 0; by <= o[1]; by++)
                        for (int bx = 0; bx <= o[0]; bx++) {
                            const int ci = lin3(C, bx ? i1[0] : ic[0], by ? i1[1] : ic[1], bz ? i1[2] : ic[2]);
#pragma unroll
                            for (int c = 0; c < 3; c++) e[c] += __ldca(C.xpost[c] + ci);
                        }
#pragma unroll
                for (int c = 0; c < 3; c++) v[c] = raw[c * NP + h] + w * e[c];
            },
            [&](int n, const T (&v)[3], const T (&q)[3]) {
                const T di = last ? H.c2[0] * __ldca(V.dinv + n) : T(0);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const T f = k == 0 ? __ldca(A.r[cur][c] + n) : __ldca(V.f[c] + n);
                    if (last) {
                        V.xpost[c][n] = v[c] + di * (f - q[c]);
                    } else {
                        V.xpost[c][n] = v[c];
                        V.r[1 - par][c][n] = f - q[c];
                    }
                }
            },
            [&](int n) {
#pragma unroll
                for (int c = 0; c < 3; c++) prefetch_l1((k == 0 ? A.r[cur][c] : V.f[c]) + n);
                if (last) prefetch_l1(V.dinv + n);
            });
    };
    auto post = [&](int k, int cur) {
        const int dk = H.deg[k];
        int par = dk & 1;
        post_first(k, par, cur, dk == 1);
        if (!sync()) return false;
        par ^= 1;
        for (int j = 0; j + 1 < dk; j++) {
            cheb(k, j, par, true, j + 2 == dk);
            if (!sync()) return false;
            par ^= 1;
        }
        return true;
    };
    auto pre = [&](int k) {
        pre_first(k);
        if (!sync()) return false;
        int par = 1;
        const bool co = k == L - 1;
        const int nk = co ? cs - 1 : H.deg[k];
        for (int j = 1; j < nk; j++) {
            cheb(k, j, par, false, co && j + 1 == nk);
            if (!sync()) return false;
            par ^= 1;
        }
        return true;
    };

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

        // ---- finest level, first pre-smoothing sweep (+ the CG update); its
        // Chebyshev direction is read only by further smoothing steps there
        Acc<T> racc[1];
        const bool d0 = (L == 1 ? cs - 1 : H.deg[0]) > 1;
        {
            const T c2 = H.c2[0];
            sweep(0, first ? 4 : 10,
                [&](const T **src) {
                    src[0] = L0.dinv;
                    for (int c = 0; c < 3; c++) { src[1 + c] = A.r[cur][c]; src[4 + c] = A.w[cur][c]; src[7 + c] = A.s[cur][c]; }
                },
                [&](const T *raw, int h, int, int, int, T (&v)[3]) {
                    const T di = c2 * raw[h];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        T rv = raw[(1 + c) * NP + h];
                        if (!first) rv -= ta * (raw[(4 + c) * NP + h] + tb * raw[(7 + c) * NP + h]);
                        v[c] = di * rv;
                    }
                },
                [&](int n, const T (&v)[3], const T (&q)[3]) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        T f = __ldca(A.r[cur][c] + n);
                        if (!first) {
                            const T si = __ldca(A.w[cur][c] + n) + tb * __ldca(A.s[cur][c] + n);
                            const T pi = __ldca(L0.xpost[c] + n) + tb * A.p[c][n];
                            A.p[c][n] = pi;
                            A.x[c][n] = A.x[c][n] + ta * pi;
                            A.s[nxt][c][n] = si;
                            f = f - ta * si;
                            A.r[nxt][c][n] = f;
                            racc[0].fma_plain(f, f);
                        }
                        L0.xpre[c][n] = v[c];
                        L0.r[1][c][n] = f - q[c];
                        if (d0) L0.d[1][c][n] = v[c];
                    }
                },
                [&](int n) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        prefetch_l1(A.r[cur][c] + n);
                        if (!first) {
                            prefetch_l1(A.w[cur][c] + n);
                            prefetch_l1(A.s[cur][c] + n);
                            prefetch_l1(L0.xpost[c] + n);
                            prefetch_l1(A.p[c] + n);
                            prefetch_l1(A.x[c] + n);
                        }
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
        } else if (!sync()) {
            return -1;
        }

        // ---- rest of the V-cycle
        {
            int par = 1;
            const int n0 = L == 1 ? cs - 1 : H.deg[0];
            for (int j = 1; j < n0; j++) {
                cheb(0, j, par, false, L == 1 && j + 1 == n0);
                if (!sync()) return -1;
                par ^= 1;
            }
        }
        for (int k = 1; k < L; k++)
            if (!pre(k)) return -1;
        for (int k = L - 2; k >= 0; k--)
            if (!post(k, cur)) return -1;

        // ---- u = V-cycle result, w = A u (+ mean strain), gamma, delta, mean-strain row
        Acc<T> acc[2 + NV];
        if (lead)
            for (int c = 0; c < 3; c++) s_src[c] = L0.xpost[c];
        __syncthreads();
        mg_sweep3z<T, true>(
            L0.nx, L0.ny, L0.nz, s_zc[0], L0.lam, L0.mu, bid, nbk, smem, s_ue, 3, s_src,
            [&](const T *raw, int h, int, int, int, T (&v)[3]) {
#pragma unroll
                for (int c = 0; c < 3; c++) v[c] = raw[c * NP + h];
            },
            [&](int n, const T (&v)[3], const T (&q)[3]) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    A.w[cur][c][n] = q[c];
                    acc[0].fma_plain(__ldca(A.r[cur][c] + n), v[c]);
                    acc[1].fma_plain(q[c], v[c]);
                }
            },
            [&](const T *se) {
#pragma unroll
                for (int vv = 0; vv < NV; vv++) acc[2 + vv].add_plain(se[vv]);
            },
            [&](int n) {
#pragma unroll
                for (int c = 0; c < 3; c++) prefetch_l1(A.r[cur][c] + n);
            });
        double tt[2 + NV];
        if (!reduce_barrier<Acc<T>, 2 + NV>(acc, A.partials, A.result, A.bar_count, A.bar_gen, err, tt, bid, nbk)) return -1;
        if (lead) {
            double s6[6];
            dmat_mul<3>(S.Sl, S.Sm, S.UE, s6);
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
