// Backward-Euler step of the field relations (Sec. 2.4, closing paragraph:
// the relations are integrated in time by backward Euler and each step is
// solved by Newton's method): device kernels of the Jacobian-free
// Newton-Krylov solve that pf_lib.cu drives.
//
// The unknown of one step is y = (theta, x_O, x_H, x_H2O) at the new time
// level, stored as four blocks of N cells.  Its equations are
//   F(y) = y - y_n - dt R(y)                       (free rows),
//   F(y) = x_H - x_H,bc and x_H2O - 0              (supply cells: held values),
// with R the right-hand sides of the explicit update (the same fluxes, the
// same driving force, the same reaction; the coupling scalars tr eps_e and
// |dev eps_e|^2 of the mechanics solved at y_n, held over the step).
// Jacobian-vector products are directional derivatives of F evaluated in
// forward mode (matrix-free); the linear solves are restarted GMRES
// preconditioned by a fixed Chebyshev polynomial of each field's own
// diffusion block (see k_be_pc_*), in FP64 or FP32 (k_be_pc32_*); FP64
// everywhere else.
#pragma once

namespace pfdev {

struct BEArgs {
    int nx, ny, nz;
    long long N;
    double dt;
    CellConst<double> K;                 // model constants (dt unused: see dt above)
    const double *phig, *mob, *trE, *devE2;
    const unsigned char *mask;
};

template <int D>
__device__ __forceinline__ void be_neighbours(const BEArgs &a, long long c, long long (&nb)[2 * D])
{
    const int i = (int)(c % a.nx);
    const long long r = c / a.nx;
    const int j = (int)(r % a.ny);
    const int k = D == 3 ? (int)(r / a.ny) : 0;
    const long long base = c - i, pl = (long long)a.nx * a.ny;
    nb[0] = base + (i == 0 ? a.nx - 1 : i - 1);
    nb[1] = base + (i == a.nx - 1 ? 0 : i + 1);
    nb[2] = c + (long long)a.nx * ((j == 0 ? a.ny - 1 : j - 1) - j);
    nb[3] = c + (long long)a.nx * ((j == a.ny - 1 ? 0 : j + 1) - j);
    if constexpr (D == 3) {
        nb[4] = c + pl * ((k == 0 ? a.nz - 1 : k - 1) - k);
        nb[5] = c + pl * ((k == a.nz - 1 ? 0 : k + 1) - k);
    }
}

// Forward-mode derivative (value, directional derivative): the kernels
// below evaluate R in it to get J z exactly (up to rounding) rather than by a
// difference quotient, whose rounding error grows with the stiffness of
// dt R.
struct Dual {
    double v, d;
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(double a) : v(a), d(0.0) {}
    __device__ __forceinline__ Dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ bool be_nonzero(double a) { return a != 0.0; }
__device__ __forceinline__ bool be_nonzero(Dual a) { return a.v != 0.0; }
__device__ __forceinline__ double be_val(double a) { return a; }
__device__ __forceinline__ double be_val(Dual a) { return a.v; }

// mu_O = c sum_a W_a f_a'(x_O) - kappa_O Lap x_O, M_O = D_O / (c sum_a W_a
// f_a''), D_H, D_H2O (Sec. 2.2, 3.2, Table 1; phase interpolation of the
// diffusivities) of cell c; ld(b, i) gives field b (theta, x_O, x_H, x_H2O)
// at cell i.
template <int D, typename S, class LD>
__device__ __forceinline__ void be_derive_cell(const BEArgs &a, long long c, LD &&ld, S (&out)[4])
{
    const CellConst<double> &K = a.K;
    long long nb[2 * D];
    be_neighbours<D>(a, c, nb);
    const S x = ld(1, c);
    S lap = S(-2.0 * D) * x;
#pragma unroll
    for (int q = 0; q < 2 * D; q++) lap += ld(1, nb[q]);
    S Wf, Ww, Wg;
    phase_weights<S>(ld(0, c), S(a.phig[c]), Wf, Ww, Wg);
    const S m1 = Wf * f_fe1(x) + Ww * f_wu1(x) + Wg * f_ga1(x);
    const S m2 = Wf * f_fe2(x) + Ww * f_wu2(x) + Wg * f_ga2(x);
    out[0] = S(K.c) * m1 - S(K.kappa) * lap;
    const S DO = (S(1.0) - Wg) * S(K.DOs) + Wg * S(K.DOg);
    const S den = S(K.c) * m2;
    out[1] = be_nonzero(den) ? DO / den : S(0.0);
    out[2] = (S(1.0) - Wg) * S(K.DHs) + Wg * S(K.DHg);
    out[3] = (S(1.0) - Wg) * S(K.DWs) + Wg * S(K.DWg);
}

// R(y) of cell c (Sec. 2.4): ld as above, ldd(b, i) the derived field b
// (mu, M, D_H, D_H2O) at cell i.
template <int D, typename S, class LD, class LDD>
__device__ __forceinline__ void be_rates_cell(const BEArgs &a, long long c, LD &&ld, LDD &&ldd, S (&R)[4])
{
    const CellConst<double> &K = a.K;
    long long nb[2 * D];
    be_neighbours<D>(a, c, nb);
    const S th = ld(0, c), xo = ld(1, c), xh = ld(2, c), xw = ld(3, c);
    const S mu0 = ldd(0, c), M0 = ldd(1, c), DH0 = ldd(2, c), DW0 = ldd(3, c);
    S lapt(0.0), dO(0.0), dH(0.0), dW(0.0);
#pragma unroll
    for (int q = 0; q < 2 * D; q++) {
        const long long n = nb[q];
        lapt += ld(0, n) - th;
        dO += S(0.5) * (M0 + ldd(1, n)) * (ldd(0, n) - mu0);
        dH += S(0.5) * (DH0 + ldd(2, n)) * (ld(2, n) - xh);
        dW += S(0.5) * (DW0 + ldd(3, n)) * (ld(3, n) - xw);
    }
    const double pg = a.phig[c], tE = a.trE[c], s2 = a.devE2[c];
    const double hg0 = hfun(pg), sol = 1.0 - hg0;
    const S hpt = hder(th);
    const S Af = S(K.c) * f_fe(xo) + S(0.5 * K.Ks * tE * tE + K.Gs * s2);
    const S Aw = S(K.c) * f_wu(xo) + S(0.5 * K.Ks * tE * tE + K.Gs * s2);
    const double Kmix = sol * K.Ks + hg0 * K.Kg;
    const S force = S(sol) * hpt * (Af - Aw) + S(K.w2) * mder(th) - S(K.eig3 * sol * Kmix * tE) * hpt;
    R[0] = S(K.Lh * a.mob[c]) * (force - S(K.eps2) * lapt);
    S rr = S(mfun(pg) * K.kf) * xo * xh;
    if (be_val(xw) >= 1.0) rr = S(0.0);
    R[1] = dO - rr;
    R[2] = dH - S(2.0) * rr;
    R[3] = dW + rr;
}

// derived fields of the state y: der = (mu, M, D_H, D_H2O)
template <int D>
__global__ void k_be_derive(const BEArgs a, const double *__restrict__ y, double *__restrict__ der)
{
    const long long N = a.N;
    auto ld = [&](int b, long long i) { return y[b * N + i]; };
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double o[4];
        be_derive_cell<D, double>(a, c, ld, o);
#pragma unroll
        for (int b = 0; b < 4; b++) der[b * N + c] = o[b];
    }
}

// Non-negative double as an ordered integer (atomicMax of a maximum norm).
__device__ __forceinline__ void be_atomic_max(unsigned long long *m, double v)
{
    atomicMax(m, (unsigned long long)__double_as_longlong(v));
}

// R(y) from the state y and its derived fields der.  mode 0: out = F(y)
// (y0 = y_n) and *maxabs = max |F|; mode 1: out = R(y) on every row.
template <int D>
__global__ void k_be_rates(const BEArgs a, const double *__restrict__ y, const double *__restrict__ y0,
                           const double *__restrict__ der, double *__restrict__ out, int mode,
                           unsigned long long *maxabs)
{
    const long long N = a.N;
    auto ld = [&](int b, long long i) { return y[b * N + i]; };
    auto ldd = [&](int b, long long i) { return der[b * N + i]; };
    double mx = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double R[4];
        be_rates_cell<D, double>(a, c, ld, ldd, R);
        if (mode == 1) {
#pragma unroll
            for (int b = 0; b < 4; b++) out[b * N + c] = R[b];
        } else {
            const bool held = a.mask[c] != 0;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                double f;
                if (held && b == 2) f = y[2 * N + c] - a.K.xHbc;
                else if (held && b == 3) f = y[3 * N + c];
                else f = y[b * N + c] - y0[b * N + c] - a.dt * R[b];
                out[b * N + c] = f;
                mx = fmax(mx, fabs(f));
            }
        }
    }
    if (mode == 0) {
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) be_atomic_max(maxabs, mx);
    }
}

// Jacobian-vector product J z = z - dt R'(y) z (free rows), z (held rows):
// the derived fields and R in forward mode along z.
template <int D>
__global__ void k_be_jderive(const BEArgs a, const double *__restrict__ y, const double *__restrict__ z,
                             double *__restrict__ dv, double *__restrict__ dd)
{
    const long long N = a.N;
    auto ld = [&](int b, long long i) { return Dual(y[b * N + i], z[b * N + i]); };
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Dual o[4];
        be_derive_cell<D, Dual>(a, c, ld, o);
#pragma unroll
        for (int b = 0; b < 4; b++) {
            dv[b * N + c] = o[b].v;
            dd[b * N + c] = o[b].d;
        }
    }
}

template <int D>
__global__ void k_be_jvp(const BEArgs a, const double *__restrict__ y, const double *__restrict__ z,
                         const double *__restrict__ dv, const double *__restrict__ dd, double *__restrict__ out)
{
    const long long N = a.N;
    auto ld = [&](int b, long long i) { return Dual(y[b * N + i], z[b * N + i]); };
    auto ldd = [&](int b, long long i) { return Dual(dv[b * N + i], dd[b * N + i]); };
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Dual R[4];
        be_rates_cell<D, Dual>(a, c, ld, ldd, R);
        const bool held = a.mask[c] != 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const double zz = z[b * N + c];
            out[b * N + c] = (held && b >= 2) ? zz : zz - a.dt * R[b].d;
        }
    }
}

// y = y_n with the held values on supply cells (the Newton start).
__global__ void k_be_init(const BEArgs a, const double *__restrict__ y0, double *__restrict__ y)
{
    const long long N = a.N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const bool held = a.mask[c] != 0;
        y[c] = y0[c];
        y[N + c] = y0[N + c];
        y[2 * N + c] = held ? a.K.xHbc : y0[2 * N + c];
        y[3 * N + c] = held ? 0.0 : y0[3 * N + c];
    }
}

// ---------------------------------------------------------------------------
// Preconditioner: per field the diffusion block of I - dt dR/dy,
//   theta: d + dt L eps mob_c sum_n (d_c - d_n)      (the gradient term),
//   x_i:   d + dt sum_n (D_c + D_n) / 2 (d_c - d_n)   (O with D_O, H, H2O),
// identity on held rows, and K Chebyshev steps on it with Jacobi scaling
// from z = 0, on the interval [1 - s, 1 + s], s = max over rows of
// (offdiagonal sum) / diagonal, which contains the spectrum of the scaled
// block (Gershgorin; the theta block is similar to a symmetric matrix).
// ---------------------------------------------------------------------------
// per-row diagonal of the four blocks, and max over rows of s per block
template <int D>
__global__ void k_be_pc_diag(const BEArgs a, const double *__restrict__ der, double *__restrict__ dg,
                             unsigned long long *smax)
{
    const long long N = a.N;
    const double cth = -a.dt * a.K.Lh * a.K.eps2;       // dt L eps
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        long long nb[2 * D];
        be_neighbours<D>(a, c, nb);
        const bool held = a.mask[c] != 0;
        double s[4];
        s[0] = 2.0 * D * cth * a.mob[c];
        const double DOc = (1.0 - hfun(a.phig[c])) * a.K.DOs + hfun(a.phig[c]) * a.K.DOg;
        double so = 0.0, sh = 0.0, sw = 0.0;
#pragma unroll
        for (int q = 0; q < 2 * D; q++) {
            const long long n = nb[q];
            const double hn = hfun(a.phig[n]);
            so += 0.5 * (DOc + (1.0 - hn) * a.K.DOs + hn * a.K.DOg);
            sh += 0.5 * (der[2 * N + c] + der[2 * N + n]);
            sw += 0.5 * (der[3 * N + c] + der[3 * N + n]);
        }
        s[1] = a.dt * so;
        s[2] = held ? 0.0 : a.dt * sh;
        s[3] = held ? 0.0 : a.dt * sw;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            dg[b * N + c] = 1.0 + s[b];
            m[b] = fmax(m[b], s[b] / (1.0 + s[b]));
        }
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        for (int o = 16; o > 0; o >>= 1) m[b] = fmax(m[b], __shfl_xor_sync(0xffffffffu, m[b], o));
        if ((threadIdx.x & 31) == 0) be_atomic_max(smax + b, m[b]);
    }
}

// q = A d for the four blocks (A as above)
template <int D>
__global__ void k_be_pc_apply(const BEArgs a, const double *__restrict__ der, const double *__restrict__ d,
                              double *__restrict__ q)
{
    const long long N = a.N;
    const double cth = -a.dt * a.K.Lh * a.K.eps2;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        long long nb[2 * D];
        be_neighbours<D>(a, c, nb);
        const bool held = a.mask[c] != 0;
        const double hc = hfun(a.phig[c]);
        const double DOc = (1.0 - hc) * a.K.DOs + hc * a.K.DOg;
        double lt = 0.0, fo = 0.0, fh = 0.0, fw = 0.0;
#pragma unroll
        for (int k = 0; k < 2 * D; k++) {
            const long long n = nb[k];
            const double hn = hfun(a.phig[n]);
            lt += d[c] - d[n];
            fo += 0.5 * (DOc + (1.0 - hn) * a.K.DOs + hn * a.K.DOg) * (d[N + c] - d[N + n]);
            fh += 0.5 * (der[2 * N + c] + der[2 * N + n]) * (d[2 * N + c] - d[2 * N + n]);
            fw += 0.5 * (der[3 * N + c] + der[3 * N + n]) * (d[3 * N + c] - d[3 * N + n]);
        }
        q[c] = d[c] + cth * a.mob[c] * lt;
        q[N + c] = d[N + c] + a.dt * fo;
        q[2 * N + c] = held ? d[2 * N + c] : d[2 * N + c] + a.dt * fh;
        q[3 * N + c] = held ? d[3 * N + c] : d[3 * N + c] + a.dt * fw;
    }
}

struct BECheb {
    double c1[4], c2[4];   // d = c1 d + c2 D^-1 r, per block
};

// z = 0, r = v, d = D^-1 r / theta_b  (c2 carries 1 / theta_b)
__global__ void k_be_pc_init(long long N, const double *__restrict__ v, const double *__restrict__ dg,
                             double *__restrict__ z, double *__restrict__ r, double *__restrict__ d, BECheb cf)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / N);
        z[i] = 0.0;
        r[i] = v[i];
        d[i] = cf.c2[b] * v[i] / dg[i];
    }
}

// one Chebyshev step after q = A d: z += d, r -= q, d = c1 d + c2 D^-1 r;
// last: z += d only
__global__ void k_be_pc_step(long long N, const double *__restrict__ q, const double *__restrict__ dg,
                             double *__restrict__ z, double *__restrict__ r, double *__restrict__ d, BECheb cf,
                             int last)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / N);
        const double dd = d[i];
        z[i] += dd;
        if (!last) {
            const double rr = r[i] - q[i];
            r[i] = rr;
            d[i] = cf.c1[b] * dd + cf.c2[b] * rr / dg[i];
        }
    }
}

// ---------------------------------------------------------------------------
// The same preconditioner in FP32 (pf_implicit_opts.pc_precision =
// PF_MIXED; GB300 runs FP32 at 64 times its FP64 rate): the blocks'
// coefficients packed once per Newton step, one fused kernel per Chebyshev
// step (the stencil reads the previous direction and writes the next, so no
// q pass), the result handed back in FP64.  The Krylov vectors, the
// Jacobian-vector products and the Newton residual stay FP64; only the
// preconditioner, an approximate inverse by construction, rounds to FP32.
// ---------------------------------------------------------------------------
struct BEPc32 {
    float *cth;        // N: the theta block's dt L eps mob_c (with its sign)
    float *DO, *DH, *DW;   // N: the diffusivities of the three species blocks
    float *dginv;      // 4N: inverse diagonals
    float *z, *r, *d0, *d1;   // 4N each: iterate, residual, directions (ping-pong)
};
struct BECheb32 {
    float c1[4], c2[4];
};

template <int D>
__device__ __forceinline__ void be_neighbours32(int nx, int ny, int nz, int c, int (&nb)[2 * D])
{
    const int i = c % nx, r = c / nx;
    const int j = r % ny, k = D == 3 ? r / ny : 0;
    const int base = c - i, pl = nx * ny;
    nb[0] = base + (i == 0 ? nx - 1 : i - 1);
    nb[1] = base + (i == nx - 1 ? 0 : i + 1);
    nb[2] = c + nx * ((j == 0 ? ny - 1 : j - 1) - j);
    nb[3] = c + nx * ((j == ny - 1 ? 0 : j + 1) - j);
    if constexpr (D == 3) {
        nb[4] = c + pl * ((k == 0 ? nz - 1 : k - 1) - k);
        nb[5] = c + pl * ((k == nz - 1 ? 0 : k + 1) - k);
    }
}

// the FP32 coefficients of the four blocks (after k_be_pc_diag)
__global__ void k_be_pc32_pack(const BEArgs a, const double *__restrict__ der, const double *__restrict__ dg,
                               BEPc32 P)
{
    const int N = (int)a.N;
    const double cth = -a.dt * a.K.Lh * a.K.eps2;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const double hc = hfun(a.phig[c]);
        P.cth[c] = (float)(cth * a.mob[c]);
        P.DO[c] = (float)((1.0 - hc) * a.K.DOs + hc * a.K.DOg);
        P.DH[c] = (float)der[2 * (size_t)N + c];
        P.DW[c] = (float)der[3 * (size_t)N + c];
#pragma unroll
        for (int b = 0; b < 4; b++) P.dginv[(size_t)b * N + c] = (float)(1.0 / dg[(size_t)b * N + c]);
    }
}

// z = 0, r = v, d0 = c2 D^-1 r
__global__ void k_be_pc32_init(int N, const double *__restrict__ v, BEPc32 P, BECheb32 cf)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const size_t i = (size_t)b * N + c;
            const float rv = (float)v[i];
            P.z[i] = 0.0f;
            P.r[i] = rv;
            P.d0[i] = cf.c2[b] * rv * P.dginv[i];
        }
}

// one Chebyshev step: q = A din at cell c, then z += din, r -= q,
// dout = c1 din + c2 D^-1 r
template <int D>
__global__ void k_be_pc32_step(int nx, int ny, int nz, int N, float dt, const unsigned char *__restrict__ mask,
                               BEPc32 P, const float *__restrict__ din, float *__restrict__ dout, BECheb32 cf)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int nb[2 * D];
        be_neighbours32<D>(nx, ny, nz, c, nb);
        const float d0c = din[c], d1c = din[N + c], d2c = din[2 * N + c], d3c = din[3 * N + c];
        const float DOc = P.DO[c], DHc = P.DH[c], DWc = P.DW[c];
        float lt = 0.0f, fo = 0.0f, fh = 0.0f, fw = 0.0f;
#pragma unroll
        for (int k = 0; k < 2 * D; k++) {
            const int n = nb[k];
            lt += d0c - din[n];
            fo += 0.5f * (DOc + P.DO[n]) * (d1c - din[N + n]);
            fh += 0.5f * (DHc + P.DH[n]) * (d2c - din[2 * N + n]);
            fw += 0.5f * (DWc + P.DW[n]) * (d3c - din[3 * N + n]);
        }
        const bool held = mask[c] != 0;
        float q[4], dc[4] = {d0c, d1c, d2c, d3c};
        q[0] = d0c + P.cth[c] * lt;
        q[1] = d1c + dt * fo;
        q[2] = held ? d2c : d2c + dt * fh;
        q[3] = held ? d3c : d3c + dt * fw;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const size_t i = (size_t)b * N + c;
            P.z[i] += dc[b];
            const float rr = P.r[i] - q[b];
            P.r[i] = rr;
            dout[i] = cf.c1[b] * dc[b] + cf.c2[b] * rr * P.dginv[i];
        }
    }
}

// the last step (z += din) into the FP64 result
__global__ void k_be_pc32_final(int N, BEPc32 P, const float *__restrict__ din, double *__restrict__ zo)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const size_t i = (size_t)b * N + c;
            zo[i] = (double)(P.z[i] + din[i]);
        }
}

// ---------------------------------------------------------------------------
// Vector kernels of the Krylov solve (length L = 4N).
// ---------------------------------------------------------------------------
// partial dot products of w with nv vectors V + k * L: blockIdx.y = k;
// part[k * gridDim.x + blockIdx.x]
__global__ void k_be_dots(long long L, const double *__restrict__ V, int nv, const double *__restrict__ w,
                          double *__restrict__ part)
{
    __shared__ double sh[32];
    const int k = blockIdx.y;
    if (k >= nv) return;
    const double *v = V + (size_t)k * L;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        s = fma(v[i], w[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (wid == 0) {
        s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
}

// w += sum_k c[k] V_k (c in device memory, nv <= 64)
__global__ void k_be_comb(long long L, const double *__restrict__ V, int nv, const double *__restrict__ c,
                          double *__restrict__ w)
{
    __shared__ double sc[64];
    if (threadIdx.x < nv) sc[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < nv; k++) s = fma(sc[k], V[(size_t)k * L + i], s);
        w[i] = s;
    }
}

// dst = a x + b y
__global__ void k_be_axpby(long long L, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                           double *__restrict__ dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        dst[i] = a * x[i] + b * y[i];
}

// Newton update y -= delta; max |delta| and max |y| (after the update)
__global__ void k_be_newton(long long L, const double *__restrict__ delta, double *__restrict__ y,
                            unsigned long long *mx)
{
    double md = 0.0, my = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
        const double v = y[i] - delta[i];
        y[i] = v;
        md = fmax(md, fabs(delta[i]));
        my = fmax(my, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
        my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        be_atomic_max(mx, md);
        be_atomic_max(mx + 1, my);
    }
}

// ---------------------------------------------------------------------------
// Gather / scatter between the field buffers and the state vector, and the
// balances of the finished step.
// ---------------------------------------------------------------------------
__global__ void k_be_gather(long long N, const double *__restrict__ th, const double *__restrict__ xo,
                            const double *__restrict__ xh, const double *__restrict__ xw, double *__restrict__ y)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        y[c] = th[c];
        y[N + c] = xo[c];
        y[2 * N + c] = xh[c];
        y[3 * N + c] = xw[c];
    }
}

// new fields from y; per-block partial sums of x_O, x_H, x_H2O, of the water
// the held cells' own relations would hold (removed) and of the hydrogen
// added to reach x_H,bc (supplied): the free relation's value is
// y_n + dt R(y) (R in rates)
__global__ void k_be_finish(const BEArgs a, const double *__restrict__ y, const double *__restrict__ y0,
                            const double *__restrict__ rates, double *__restrict__ th, double *__restrict__ xo,
                            double *__restrict__ xh, double *__restrict__ xw, double *__restrict__ part)
{
    const long long N = a.N;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        th[c] = y[c];
        xo[c] = y[N + c];
        xh[c] = y[2 * N + c];
        xw[c] = y[3 * N + c];
        s[0] += y[N + c];
        s[1] += y[2 * N + c];
        s[2] += y[3 * N + c];
        if (a.mask[c]) {
            s[3] += y0[3 * N + c] + a.dt * rates[3 * N + c];
            s[4] += a.K.xHbc - (y0[2 * N + c] + a.dt * rates[2 * N + c]);
        }
    }
    __shared__ double sh[5][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; k++) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 5; k++) {
            double v = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[(size_t)blockIdx.x * 5 + k] = v;
        }
    }
}

// the block partials of k_be_finish into the diagnostics (one warp, fixed order)
__global__ void k_be_diag(const double *__restrict__ part, int nb, Diag *dg)
{
    const int lane = threadIdx.x;
    double t[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        double v = 0.0;
        for (int b = lane; b < nb; b += 32) v += part[(size_t)b * 5 + k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        t[k] = v;
    }
    if (lane == 0) {
        dg->sumO_prev = dg->sumO;
        dg->sumO = t[0];
        dg->sumH = t[1];
        dg->sumW = t[2];
        dg->removedW += t[3];
        dg->suppliedH += t[4];
        if (!isfinite(t[0] + t[1] + t[2]) && dg->status == 0) dg->status = 5;
    }
}

}  // namespace pfdev
