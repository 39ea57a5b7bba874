// Finite-strain elastic equilibrium with the transformation stretch on the
// GPU (the C ABI's pf_finite_strain_solve, include/pf.h).
//
// Sec. 2.2 of the paper: the residual deformation F_R = F_T F_P with
// F_T = d_T^(1/3) I, d_T = 1 - W_f Omega (RulFloDefLocAlt, with the phase
// weights of the small-strain model); the elastic energy per reference
// volume psi = d_T phi(F_E), F_E = F F_R^-1 = d_T^(-1/3) F (F_P = I here),
// with the neo-Hooke energy of the phase mixture
//     phi(F_E) = K/4 (J_E^2 - 1 - 2 ln J_E) + G/2 (J_E^(-2/3) |F_E|^2 - 3)
// (DenEneFreIntElaPha; K, G the weighted bulk and shear moduli).  The
// equilibrium Div P = 0 (Sec. 2.4) is the stationarity of the total energy
// sum_cells w sum_gauss psi(F) - N pbar : Fbar over the periodic box, with
// F = Fbar + grad u at the 2^d Gauss points of Q1 voxel elements, Fbar
// symmetric, u = 0 at node 0; P = d psi / d F.  2D is plane strain
// (F_33 = 1).
//
// With a plastic deformation F_P per cell, F_E = d_T^(-1/3) F F_P^-1 and
// P = d_T^(2/3) (d phi / d F_E) F_P^-T; pf_finite_strain_step then takes one
// multiplicative J2 update per cell at the cell-centre deformation (Sec. 2.3
// PlaTwoJ, Sec. 2.4 RulFloPla; fs_return_map).
//
// Newton's method in load steps of Omega; each Newton system H delta = -r is
// solved by conjugate gradients (H, the Hessian of the energy, is symmetric)
// preconditioned by the diagonal of the small-strain operator; every
// product H v is the directional derivative of the residual along v,
// evaluated in forward mode (value, derivative) through the same cell
// function as the residual.  FP64 throughout.  Not on the explicit step's
// hot path: the call allocates and frees its device memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pf.h"

namespace {

thread_local std::string g_fs_error;

struct FD {   // value and directional derivative
    double v, d;
    __host__ __device__ FD() {}
    __host__ __device__ FD(double a) : v(a), d(0.0) {}
    __host__ __device__ FD(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ FD operator+(FD a, FD b) { return FD(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ FD operator-(FD a, FD b) { return FD(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ FD operator*(FD a, FD b) { return FD(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ FD operator/(FD a, FD b)
{
    const double q = a.v / b.v;
    return FD(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ FD fd_pow(FD a, double p)
{
    const double q = pow(a.v, p);
    return FD(q, p * q / a.v * a.d);
}
__device__ __forceinline__ double fd_pow(double a, double p) { return pow(a, p); }
__device__ __forceinline__ FD fd_exp(FD a)
{
    const double q = exp(a.v);
    return FD(q, q * a.d);
}
__device__ __forceinline__ double fd_exp(double a) { return exp(a); }
__device__ __forceinline__ FD fd_log(FD a) { return FD(log(a.v), a.d / a.v); }
__device__ __forceinline__ FD fd_sqrt(FD a)
{
    const double q = sqrt(a.v);
    return FD(q, 0.5 * a.d / q);
}

// The same pair in FP32, for the Hessian-vector products of the mixed
// method (GB300 runs FP32 at many times its FP64 rate)
struct FDf {
    float v, d;
    __host__ __device__ FDf() {}
    __host__ __device__ FDf(double a) : v((float)a), d(0.0f) {}
    __host__ __device__ FDf(double a, double b) : v((float)a), d((float)b) {}
    __host__ __device__ FDf(float a) : v(a), d(0.0f) {}
    __host__ __device__ FDf(float a, float b) : v(a), d(b) {}
};
__device__ __forceinline__ FDf operator+(FDf a, FDf b) { return FDf(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ FDf operator-(FDf a, FDf b) { return FDf(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ FDf operator*(FDf a, FDf b) { return FDf(a.v * b.v, fmaf(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ FDf operator/(FDf a, FDf b)
{
    const float q = a.v / b.v;
    return FDf(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ FDf fd_pow(FDf a, double p)
{
    const float q = powf(a.v, (float)p);
    return FDf(q, (float)p * q / a.v * a.d);
}

// the plain real type of each scalar kind
template <typename S> struct RealOf { typedef double type; };
template <> struct RealOf<FDf> { typedef float type; };

struct FSArgs {
    int d, nx, ny, nz;
    long long N;
    const double *K, *G, *Wf;    // per cell
    const double *FPinv;         // per cell 3 x 3 row-major inverse plastic deformation, or null (identity)
    double omega;                // transformation of this load step
};

// Gauss abscissae 1/2 -+ 1/(2 sqrt 3) of the unit interval
constexpr double FS_GA = 0.5 - 0.5 / 1.7320508075688772935, FS_GB = 0.5 + 0.5 / 1.7320508075688772935;

// local shape-function derivative dN/dx_k of corner a at Gauss point g
// (bit l of a: corner offset along axis l; bit l of g: Gauss abscissa FS_GA
// or FS_GB along axis l), the dimension fixed at compile time: with g, a, k
// from unrolled loops every value is a constant
template <int D, typename R>
__device__ __forceinline__ R dshape_c(int g, int a, int k)
{
    R v = R(1.0);
#pragma unroll
    for (int l = 0; l < D; l++) {
        const int bit = (a >> l) & 1;
        const R xi = ((g >> l) & 1) ? R(FS_GB) : R(FS_GA);
        v *= l == k ? (bit ? R(1.0) : R(-1.0)) : (bit ? xi : R(1.0) - xi);
    }
    return v;
}

// the 2^D corner nodes of cell c (corner a: offsets bit l of a along axis
// l), with 32-bit index arithmetic (the solver admits N < 2^31 cells)
template <int D>
__device__ __forceinline__ void fs_corners(const FSArgs &A, int c, int (&nd)[1 << D])
{
    const int nx = A.nx, ny = A.ny;
    const int i = c % nx, r = c / nx;
    const int j = r % ny, k = r / ny;
    const int i1 = i + 1 == nx ? 0 : i + 1, j1 = j + 1 == ny ? 0 : j + 1;
    const int k1 = D == 3 ? (k + 1 == A.nz ? 0 : k + 1) : 0;
    const int row[4] = {nx * (j + ny * k), nx * (j1 + ny * k), nx * (j + ny * k1), nx * (j1 + ny * k1)};
#pragma unroll
    for (int a = 0; a < (1 << D); a++) nd[a] = ((a & 1) ? i1 : i) + row[(a >> 1) & 3];
}

__device__ __forceinline__ long long fs_node(const FSArgs &A, long long c, int a)
{
    const int i = (int)(c % A.nx);
    const long long r = c / A.nx;
    const int j = (int)(r % A.ny), k = (int)(r / A.ny);
    const int ii = (i + (a & 1)) % A.nx, jj = (j + ((a >> 1) & 1)) % A.ny;
    const int kk = A.d == 3 ? (k + ((a >> 2) & 1)) % A.nz : 0;
    return ii + (long long)A.nx * (jj + (long long)A.ny * kk);
}

// The per-cell constants of the stress in the arithmetic type R, computed
// once per load step (k_fs_pack): the mixture moduli, d_T = 1 - W_f omega,
// s = d_T^(-1/3), d_T s, and the inverse plastic deformation.
template <typename R>
struct FSPack {
    R K, G, dTs, s;
    R Fi[9];
};

// first Piola stress at deformation F (3 x 3, row-major) of a cell with
// constants pk (hasFi: F_P is not the identity)
template <typename S>
__device__ __forceinline__ void fs_piola(const FSPack<typename RealOf<S>::type> &pk, bool hasFi, const S (&F)[9],
                                         S (&P)[9])
{
    typedef typename RealOf<S>::type R;
    const R s = pk.s, K = pk.K, G = pk.G;
    S Fe[9];
    if (hasFi) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                Fe[3 * i + j] = S(s) * (F[3 * i] * S(pk.Fi[j]) + F[3 * i + 1] * S(pk.Fi[3 + j]) +
                                        F[3 * i + 2] * S(pk.Fi[6 + j]));
    } else {
#pragma unroll
        for (int q = 0; q < 9; q++) Fe[q] = S(s) * F[q];
    }
    // cofactor matrix: J F^-T
    S cof[9];
    cof[0] = Fe[4] * Fe[8] - Fe[5] * Fe[7];
    cof[1] = Fe[5] * Fe[6] - Fe[3] * Fe[8];
    cof[2] = Fe[3] * Fe[7] - Fe[4] * Fe[6];
    cof[3] = Fe[2] * Fe[7] - Fe[1] * Fe[8];
    cof[4] = Fe[0] * Fe[8] - Fe[2] * Fe[6];
    cof[5] = Fe[1] * Fe[6] - Fe[0] * Fe[7];
    cof[6] = Fe[1] * Fe[5] - Fe[2] * Fe[4];
    cof[7] = Fe[2] * Fe[3] - Fe[0] * Fe[5];
    cof[8] = Fe[0] * Fe[4] - Fe[1] * Fe[3];
    const S J = Fe[0] * cof[0] + Fe[1] * cof[1] + Fe[2] * cof[2];
    S I1(0.0);
#pragma unroll
    for (int q = 0; q < 9; q++) I1 = I1 + Fe[q] * Fe[q];
    // d phi / d F_E = K/2 (J^2 - 1) F_E^-T + G J^(-2/3) (F_E - I1/3 F_E^-T)
    const S a1 = S(R(0.5) * K) * (J * J - S(1.0)) / J;       // times cof = J F^-T
    const S jm = fd_pow(J, -2.0 / 3.0);
    const S a2 = S(G) * jm;
    const S a3 = a2 * I1 / (S(3.0) * J);
    if (hasFi) {
        S D[9];
#pragma unroll
        for (int q = 0; q < 9; q++) D[q] = a1 * cof[q] + a2 * Fe[q] - a3 * cof[q];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                P[3 * i + j] = S(pk.dTs) * (D[3 * i] * S(pk.Fi[3 * j]) + D[3 * i + 1] * S(pk.Fi[3 * j + 1]) +
                                            D[3 * i + 2] * S(pk.Fi[3 * j + 2]));
    } else {
#pragma unroll
        for (int q = 0; q < 9; q++) P[q] = S(pk.dTs) * (a1 * cof[q] + a2 * Fe[q] - a3 * cof[q]);
    }
}

// ---------------------------------------------------------------------------
// Multiplicative J2 update of one point (Sec. 2.3 PlaTwoJ, Sec. 2.4
// RulFloPla), backward Euler with the exponential map:
//     F_P,new = exp(dl N) F_P,  N = dev M / |dev M|,
//     |dev M| = sqrt(2/3) (sigma_Y + H (eps_P + dl)),  dl >= 0,
// M the Mandel stress d_T (K/2 (det C - 1) I + G dev(det C^(-1/3) C)) of the
// elastic right Cauchy-Green tensor C = F_E^T F_E (the derivative of the
// energy above).  Isotropic elasticity keeps the update coaxial with the
// trial C_E: in its principal frame the elastic log stretches e solve
// e - e_trial + dl dev m / |dev m| = 0 and the yield condition, four
// equations by Newton (Jacobian in forward mode).
// ---------------------------------------------------------------------------
// eigenvalues w and eigenvectors (columns of V, row-major) of a symmetric
// 3 x 3 matrix by cyclic Jacobi rotations
__device__ void fs_eig3(const double (&A0)[9], double (&w)[3], double (&V)[9])
{
    double a[9];
    for (int q = 0; q < 9; q++) { a[q] = A0[q]; V[q] = (q % 4 == 0) ? 1.0 : 0.0; }
    for (int sweep = 0; sweep < 30; sweep++) {
        const double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
        const double nrm = a[0] * a[0] + a[4] * a[4] + a[8] * a[8] + 2.0 * off;
        if (off <= 1e-34 * nrm) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                const double apq = a[3 * p + q];
                if (apq == 0.0) continue;
                const double th = (a[3 * q + q] - a[3 * p + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; k++) {          // a = J^T a J on columns p, q
                    const double akp = a[3 * k + p], akq = a[3 * k + q];
                    a[3 * k + p] = c * akp - sn * akq;
                    a[3 * k + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {          // rows p, q
                    const double apk = a[3 * p + k], aqk = a[3 * q + k];
                    a[3 * p + k] = c * apk - sn * aqk;
                    a[3 * q + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    const double vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = c * vkp - sn * vkq;
                    V[3 * k + q] = sn * vkp + c * vkq;
                }
            }
    }
    w[0] = a[0]; w[1] = a[4]; w[2] = a[8];
}

// principal Mandel stresses of the elastic log stretches e
template <typename S>
__device__ void fs_mand(const S (&e)[3], double K, double G, double dT, S (&m)[3])
{
    S cc[3];
    for (int i = 0; i < 3; i++) cc[i] = fd_exp(S(2.0) * e[i]);
    const S J2 = cc[0] * cc[1] * cc[2];
    const S f = fd_pow(J2, -1.0 / 3.0);
    S uu[3];
    for (int i = 0; i < 3; i++) uu[i] = cc[i] * f;
    const S tr = (uu[0] + uu[1] + uu[2]) / S(3.0);
    for (int i = 0; i < 3; i++) m[i] = S(dT) * (S(0.5 * K) * (J2 - S(1.0)) + S(G) * (uu[i] - tr));
}

// residual of the four equations at (e, dl)
template <typename S>
__device__ void fs_rm_eqs(const S (&e)[3], S dl, const double (&etr)[3], double epsP, double K, double G, double dT,
                          double sY, double H, S (&r)[4])
{
    S m[3];
    fs_mand(e, K, G, dT, m);
    const S mean = (m[0] + m[1] + m[2]) / S(3.0);
    S dm[3];
    for (int i = 0; i < 3; i++) dm[i] = m[i] - mean;
    const S nm = fd_sqrt(dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]);
    for (int i = 0; i < 3; i++) r[i] = e[i] - S(etr[i]) + dl * dm[i] / nm;
    r[3] = nm - S(sqrt(2.0 / 3.0)) * (S(sY) + S(H) * (S(epsP) + dl));
}

// one point: F (deformation), FP and epsP in/out; returns 0, or 1 if the
// Newton iteration did not converge (the point is then left elastic)
__device__ int fs_return_map(const double (&F)[9], double (&FP)[9], double &epsP, double K, double G, double dT,
                             double sY, double H)
{
    const double s = pow(dT, -1.0 / 3.0);
    // F_P^-1 through its cofactors
    double ci[9];
    ci[0] = FP[4] * FP[8] - FP[5] * FP[7]; ci[1] = FP[2] * FP[7] - FP[1] * FP[8]; ci[2] = FP[1] * FP[5] - FP[2] * FP[4];
    ci[3] = FP[5] * FP[6] - FP[3] * FP[8]; ci[4] = FP[0] * FP[8] - FP[2] * FP[6]; ci[5] = FP[2] * FP[3] - FP[0] * FP[5];
    ci[6] = FP[3] * FP[7] - FP[4] * FP[6]; ci[7] = FP[1] * FP[6] - FP[0] * FP[7]; ci[8] = FP[0] * FP[4] - FP[1] * FP[3];
    const double det = FP[0] * ci[0] + FP[1] * ci[3] + FP[2] * ci[6];
    double Fe[9], C[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            Fe[3 * i + j] = s * (F[3 * i] * ci[j] + F[3 * i + 1] * ci[3 + j] + F[3 * i + 2] * ci[6 + j]) / det;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) C[3 * i + j] = Fe[i] * Fe[j] + Fe[3 + i] * Fe[3 + j] + Fe[6 + i] * Fe[6 + j];
    // trial: the Mandel stress of C and the yield function
    {
        const double J2 = C[0] * (C[4] * C[8] - C[5] * C[7]) - C[1] * (C[3] * C[8] - C[5] * C[6]) +
                          C[2] * (C[3] * C[7] - C[4] * C[6]);
        const double f = pow(J2, -1.0 / 3.0), tr = (C[0] + C[4] + C[8]) * f / 3.0;
        double dev2 = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const double v = dT * G * (C[3 * i + j] * f - (i == j ? tr : 0.0));
                dev2 += v * v;
            }
        if (sqrt(dev2) - sqrt(2.0 / 3.0) * (sY + H * epsP) <= 0.0) return 0;
    }
    double c[3], V[9];
    fs_eig3(C, c, V);
    double etr[3], v[4];
    for (int i = 0; i < 3; i++) { etr[i] = 0.5 * log(c[i]); v[i] = etr[i]; }
    v[3] = 0.0;
    bool conv = false;
    for (int it = 0; it < 60; it++) {
        double r[4], Jm[16];
        for (int col = 0; col < 4; col++) {
            FD e[3], dl = FD(v[3], col == 3 ? 1.0 : 0.0), rr[4];
            for (int i = 0; i < 3; i++) e[i] = FD(v[i], col == i ? 1.0 : 0.0);
            fs_rm_eqs(e, dl, etr, epsP, K, G, dT, sY, H, rr);
            for (int i = 0; i < 4; i++) { Jm[4 * i + col] = rr[i].d; r[i] = rr[i].v; }
        }
        double mv[3], e0[3] = {v[0], v[1], v[2]};
        fs_mand(e0, K, G, dT, mv);
        const double scale = fmax(1.0, fmax(fabs(mv[0]), fmax(fabs(mv[1]), fabs(mv[2]))));
        double rmax = 0.0;
        for (int i = 0; i < 4; i++) rmax = fmax(rmax, fabs(r[i]));
        if (rmax <= 1e-14 * scale) { conv = true; break; }
        // Gaussian elimination with partial pivoting on the 4 x 4 system
        double b[4] = {r[0], r[1], r[2], r[3]};
        for (int k = 0; k < 4; k++) {
            int pv = k;
            for (int i = k + 1; i < 4; i++) if (fabs(Jm[4 * i + k]) > fabs(Jm[4 * pv + k])) pv = i;
            if (pv != k) {
                for (int j = 0; j < 4; j++) { const double t = Jm[4 * k + j]; Jm[4 * k + j] = Jm[4 * pv + j]; Jm[4 * pv + j] = t; }
                const double t = b[k]; b[k] = b[pv]; b[pv] = t;
            }
            for (int i = k + 1; i < 4; i++) {
                const double f = Jm[4 * i + k] / Jm[4 * k + k];
                for (int j = k; j < 4; j++) Jm[4 * i + j] -= f * Jm[4 * k + j];
                b[i] -= f * b[k];
            }
        }
        double x[4];
        for (int k = 3; k >= 0; k--) {
            double t = b[k];
            for (int j = k + 1; j < 4; j++) t -= Jm[4 * k + j] * x[j];
            x[k] = t / Jm[4 * k + k];
        }
        for (int i = 0; i < 4; i++) v[i] -= x[i];
    }
    if (!conv) return 1;
    double m[3], e[3] = {v[0], v[1], v[2]};
    fs_mand(e, K, G, dT, m);
    const double mean = (m[0] + m[1] + m[2]) / 3.0;
    const double nm = sqrt((m[0] - mean) * (m[0] - mean) + (m[1] - mean) * (m[1] - mean) + (m[2] - mean) * (m[2] - mean));
    double ex[3];
    for (int i = 0; i < 3; i++) ex[i] = exp(v[3] * (m[i] - mean) / nm);
    // exp(dl N) = V diag(ex) V^T; FP <- exp(dl N) FP
    double E[9], FPn[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) E[3 * i + j] = V[3 * i] * ex[0] * V[3 * j] + V[3 * i + 1] * ex[1] * V[3 * j + 1] +
                                                   V[3 * i + 2] * ex[2] * V[3 * j + 2];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) FPn[3 * i + j] = E[3 * i] * FP[j] + E[3 * i + 1] * FP[3 + j] + E[3 * i + 2] * FP[6 + j];
    for (int q = 0; q < 9; q++) FP[q] = FPn[q];
    epsP += v[3];
    return 0;
}

// forces of cell c (constants pk) on its 2^d corners (f[a * d + i]) and
// its weighted sum of the Gauss-point stresses (pm, d x d row-major), for
// the state (u, Fbar) given by ld_u(node, comp) and fb (3 x 3 symmetric)
template <int D, typename S, class LU>
__device__ __forceinline__ void fs_cell(const FSArgs &A, long long c, const FSPack<typename RealOf<S>::type> &pk,
                                        LU &&ld_u, const S (&fb)[9], S (&f)[24], S (&pm)[9])
{
    const bool hasFi = A.FPinv != nullptr;
    typedef typename RealOf<S>::type R;
    constexpr int na = 1 << D;
    constexpr double w = 1.0 / na;
    int nodes[na];
    fs_corners<D>(A, (int)c, nodes);
    S ua[na][D];
#pragma unroll
    for (int a = 0; a < na; a++) {
#pragma unroll
        for (int i = 0; i < D; i++) ua[a][i] = ld_u((long long)nodes[a], i);
    }
#pragma unroll
    for (int q = 0; q < 24; q++) f[q] = S(0.0);
#pragma unroll
    for (int q = 0; q < 9; q++) pm[q] = S(0.0);
#pragma unroll
    for (int g = 0; g < na; g++) {
        S F[9];
#pragma unroll
        for (int q = 0; q < 9; q++) F[q] = fb[q];
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int k = 0; k < D; k++) {
                S t = F[3 * i + k];
#pragma unroll
                for (int a = 0; a < na; a++) t = t + ua[a][i] * S(dshape_c<D, R>(g, a, k));
                F[3 * i + k] = t;
            }
        if (D == 2) {
            F[2] = F[5] = F[6] = F[7] = S(0.0);
            F[8] = S(1.0);
        }
        S P[9];
        fs_piola(pk, hasFi, F, P);
#pragma unroll
        for (int a = 0; a < na; a++)
#pragma unroll
            for (int i = 0; i < D; i++) {
                S t = f[a * D + i];
#pragma unroll
                for (int k = 0; k < D; k++) t = t + S(R(w) * dshape_c<D, R>(g, a, k)) * P[3 * i + k];
                f[a * D + i] = t;
            }
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int k = 0; k < D; k++) pm[3 * i + k] = pm[3 * i + k] + S(w) * P[3 * i + k];
    }
}

// Conjugate gradients keep every scalar on the device: the host launches
// FS_CHUNK iterations at a time and reads this state once per chunk; after
// convergence (done) or breakdown (stop) the remaining launches of the chunk
// return at once.
struct FSCG {
    double rz;      // (r, M r)
    double al;      // step along p
    double beta;    // direction update
    double tol;     // stop when |r| <= tol
    int stop;       // (p, H p) <= 0: no positive curvature along p
    int done;       // converged or at maxit
    int iters, maxit;
};
__device__ __forceinline__ bool fs_cg_over(const FSCG *cg) { return cg && (cg->stop || cg->done); }

// symmetric Fbar (3 x 3) from the m trailing entries of a vector
template <typename T, typename R>
__device__ __forceinline__ void fs_fbar(int d, const T *zf, R (&fb)[9])
{
#pragma unroll
    for (int q = 0; q < 9; q++) fb[q] = R(0.0);
    if (d == 3) {
        fb[0] = R(zf[0]); fb[4] = R(zf[1]); fb[8] = R(zf[2]);
        fb[5] = fb[7] = R(zf[3]); fb[2] = fb[6] = R(zf[4]); fb[1] = fb[3] = R(zf[5]);
    } else {
        fb[0] = R(zf[0]); fb[4] = R(zf[1]); fb[1] = fb[3] = R(zf[2]);
    }
}

// the per-cell constants of a load step (omega in A) in type R
template <typename R>
__global__ void k_fs_pack(FSArgs A, FSPack<R> *pk)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < A.N; c += (long long)gridDim.x * blockDim.x) {
        const double dT = 1.0 - A.Wf[c] * A.omega, s = pow(dT, -1.0 / 3.0);
        FSPack<R> p;
        p.K = R(A.K[c]);
        p.G = R(A.G[c]);
        p.s = R(s);
        p.dTs = R(dT * s);
        for (int q = 0; q < 9; q++) p.Fi[q] = R(A.FPinv ? A.FPinv[c * 9 + q] : (q % 4 == 0 ? 1.0 : 0.0));
        pk[c] = p;
    }
}

// x32 = (float) x on [0, L)
__global__ void k_fs_to32(long long L, const double *x, float *x32)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        x32[i] = (float)x[i];
}

// block sums of nv values per thread (warp shuffles in the values' type,
// then the warps in order in FP64), written by thread 0..nv-1 to
// out[q * gridDim.x + blockIdx.x]; blockDim.x a multiple of 32, at most 1024
template <int NV, typename T>
__device__ __forceinline__ void fs_block_partials(T (&v)[NV], double *out)
{
    __shared__ double sh[NV][32];
#pragma unroll
    for (int q = 0; q < NV; q++) {
        T t = v[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[threadIdx.x][k];
        out[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// per cell: corner forces of the state z into cf[c][a][i] (FP64, with the
// cell constants pk) and the block partial stress sums into part9
// (9 x gridDim.x): the residual
template <int D>
__global__ void k_fs_res(FSArgs A, const FSPack<double> *pk, const double *z, double *cf, double *part9)
{
    const long long N = A.N;
    const double *zf = z + (size_t)D * N;
    double fb[9], acc[9];
    fs_fbar(D, zf, fb);
#pragma unroll
    for (int q = 0; q < 9; q++) acc[q] = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double f[24], pm[9];
        const FSPack<double> p = pk[c];
        fs_cell<D, double>(A, c, p, [&](long long n, int i) { return z[n * D + i]; }, fb, f, pm);
#pragma unroll
        for (int q = 0; q < (1 << D) * D; q++) cf[c * 24 + q] = f[q];
#pragma unroll
        for (int q = 0; q < 9; q++) acc[q] += pm[q];
    }
    fs_block_partials<9>(acc, part9);
}

// the same, differentiated along v in forward mode: one Hessian-vector
// product of the energy.  S = FD: FP64 (z, v the solver's vectors); S = FDf:
// FP32 (z, v their FP32 copies, cf FP32)
template <int D, typename S>
__global__ void __launch_bounds__(128, 4)
k_fs_hvp(FSArgs A, const FSPack<typename RealOf<S>::type> *pk, const typename RealOf<S>::type *z,
         const typename RealOf<S>::type *v, typename RealOf<S>::type *cf, double *part9, const FSCG *cg)
{
    typedef typename RealOf<S>::type R;
    if (fs_cg_over(cg)) return;
    const long long N = A.N;
    R fb0[9], fb1[9];
    fs_fbar(D, z + (size_t)D * N, fb0);
    fs_fbar(D, v + (size_t)D * N, fb1);
    S fb[9];
#pragma unroll
    for (int q = 0; q < 9; q++) fb[q] = S(fb0[q], fb1[q]);
    R acc[9];
#pragma unroll
    for (int q = 0; q < 9; q++) acc[q] = R(0.0);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        S f[24], pm[9];
        const FSPack<R> p = pk[c];
        fs_cell<D, S>(A, c, p, [&](long long n, int i) { return S(z[n * D + i], v[n * D + i]); }, fb, f, pm);
#pragma unroll
        for (int q = 0; q < (1 << D) * D; q++) cf[c * 24 + q] = f[q].d;
#pragma unroll
        for (int q = 0; q < 9; q++) acc[q] += pm[q].d;
    }
    fs_block_partials<9>(acc, part9);
}

// nodal forces: each node sums the corner forces of its 2^d cells (in the
// corner forces' type); node 0 is held (zero).  With p given, also the block
// partials of (p, out) over the displacement dofs into partdot.
template <typename R>
__global__ void k_fs_gather(FSArgs A, const R *cf, double *out, const double *p, double *partdot, const FSCG *cg)
{
    if (fs_cg_over(cg)) return;
    const int d = A.d, na = 1 << d, nx = A.nx, ny = A.ny;
    double dot[1] = {0.0};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)A.N; n += gridDim.x * blockDim.x) {
        const int i = n % nx, r = n / nx;
        const int j = r % ny, k = r / ny;
        const int i0 = i == 0 ? nx - 1 : i - 1, j0 = j == 0 ? ny - 1 : j - 1;
        const int k0 = d == 3 ? (k == 0 ? A.nz - 1 : k - 1) : 0;
        R s[3] = {R(0.0), R(0.0), R(0.0)};
        for (int a = 0; a < na; a++) {
            const int ci = (a & 1) ? i0 : i, cj = (a & 2) ? j0 : j, ck = (a & 4) ? k0 : k;
            const size_t c = (size_t)ci + (size_t)nx * (cj + (size_t)ny * ck);
            for (int q = 0; q < d; q++) s[q] += cf[c * 24 + a * d + q];
        }
        for (int q = 0; q < d; q++) {
            const double o = n == 0 ? 0.0 : (double)s[q];
            out[n * d + q] = o;
            if (p) dot[0] = fma(p[n * d + q], o, dot[0]);
        }
    }
    if (p) fs_block_partials<1>(dot, partdot);
}

// Jacobi diagonal of the displacement dofs from the small-strain operator
// (lambda = K - 2G/3, mu = G) of the 2^d cells around each node
__global__ void k_fs_diag(FSArgs A, double dl, double dm, double *dg)
{
    const int d = A.d, na = 1 << d;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < A.N; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % A.nx);
        const long long r = n / A.nx;
        const int j = (int)(r % A.ny), k = (int)(r / A.ny);
        double s = 0.0;
        for (int a = 0; a < na; a++) {
            const int ci = (i - (a & 1) + A.nx) % A.nx, cj = (j - ((a >> 1) & 1) + A.ny) % A.ny;
            const int ck = d == 3 ? (k - ((a >> 2) & 1) + A.nz) % A.nz : 0;
            const long long c = ci + (long long)A.nx * (cj + (long long)A.ny * ck);
            s += (A.K[c] - 2.0 * A.G[c] / 3.0) * dl + A.G[c] * dm;
        }
        for (int q = 0; q < d; q++) dg[n * d + q] = s;
    }
}

__global__ void k_fs_moduli(long long N, const double *theta, const double *phig, double Ks, double Gs, double Kg,
                            double Gg, double *K, double *G, double *Wf)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        auto h = [](double x) { return x * x * x * (x * (6.0 * x - 15.0) + 10.0); };
        const double hg = h(phig[c]), ht = h(theta[c]);
        const double wf = (1.0 - hg) * ht, ww = (1.0 - hg) * (1.0 - ht);
        K[c] = (wf + ww) * Ks + hg * Kg;
        G[c] = (wf + ww) * Gs + hg * Gg;
        Wf[c] = wf;
    }
}

__global__ void k_fs_dot(long long L, const double *a, const double *b, double *part)
{
    __shared__ double sh[8];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
        part[blockIdx.x] = t;
    }
}

// y = a x + b y on [0, L); the inverse Jacobi diagonal: 1 / dg over
// [0, nd), 1 / dgf beyond
__global__ void k_fs_axpby(long long L, double a, const double *x, double b, double *y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
__global__ void k_fs_dginv(long long L, long long nd, const double *dg, double dgf, double *dginv)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        dginv[i] = 1.0 / (i < nd ? dg[i] : dgf);
}

// ---------------------------------------------------------------------------
// The CG scalar kernels (one block of 256 threads; sums in a fixed order)
// ---------------------------------------------------------------------------
struct Mat9 {
    double v[9];
};

// sums over the n partials of each of NV rows (row q at part + q * n) by
// the block: thread t takes t, t + 256, ...; then fs_block_partials' tree
template <int NV>
__device__ __forceinline__ void fs_sum_rows(const double *part, int n, double (&tot)[NV])
{
    __shared__ double res[NV];
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) v[q] = 0.0;
    // the rows inside the loop over k: NV independent loads per step
#pragma unroll 2
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) t[q] = part[(size_t)q * n + k];
#pragma unroll
        for (int q = 0; q < NV; q++) v[q] += t[q];
    }
    __shared__ double sh[NV][8];
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double t = v[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[threadIdx.x][k];
        res[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; q++) tot[q] = res[q];
}

// the m mean-deformation rows from the summed stresses ps: the diagonal
// entries, ps_ij + ps_ji off it
__device__ __forceinline__ void fs_rows_of(int d, const double (&ps)[9], double (&rf)[6])
{
    const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
    const int i2[3] = {0, 1, 0}, j2[3] = {0, 1, 1};
    const int m = d == 3 ? 6 : 3;
    for (int k = 0; k < m; k++) {
        const int i = d == 3 ? ii[k] : i2[k], j = d == 3 ? jj[k] : j2[k];
        rf[k] = i == j ? ps[3 * i + i] : ps[3 * i + j] + ps[3 * j + i];
    }
}

// the residual's mean-deformation rows: summed stresses minus N pbar
__global__ void k_fs_rows(int d, int nb, const double *part9, Mat9 pbar, double Nc, double *outf)
{
    double ps[9];
    fs_sum_rows<9>(part9, nb, ps);
    if (threadIdx.x != 0) return;
    for (int q = 0; q < 9; q++) ps[q] -= Nc * pbar.v[q];
    double rf[6];
    fs_rows_of(d, ps, rf);
    for (int k = 0; k < (d == 3 ? 6 : 3); k++) outf[k] = rf[k];
}

// the product's mean-deformation rows into qf, then
// al = rz / (p, H p) with (p, H p) = the gather's partials + the rows' part
__global__ void k_fs_cg_alpha(int d, int nb, const double *part9, int ng, const double *partdot, const double *pf,
                              double *qf, FSCG *cg)
{
    if (fs_cg_over(cg)) return;
    double ps[9], pd[1];
    fs_sum_rows<9>(part9, nb, ps);
    fs_sum_rows<1>(partdot, ng, pd);
    if (threadIdx.x != 0) return;
    double rf[6];
    fs_rows_of(d, ps, rf);
    double pq = pd[0];
    for (int k = 0; k < (d == 3 ? 6 : 3); k++) {
        qf[k] = rf[k];
        pq = fma(pf[k], rf[k], pq);
    }
    if (!(pq > 0.0)) {
        cg->stop = 1;                 // no positive curvature along p
        return;
    }
    cg->al = cg->rz / pq;
}

// dz += al p, r -= al q, s = M r (Jacobi: dginv the inverse diagonal);
// block partials of (r, r) and (r, s) into part2 (2 x gridDim.x)
__global__ void k_fs_cg_update(long long L, const double *dginv, const double *p, const double *q, double *dz,
                               double *r, double *s, const FSCG *cg, double *part2)
{
    if (fs_cg_over(cg)) return;
    const double al = cg->al;
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
        dz[i] = fma(al, p[i], dz[i]);
        const double ri = fma(-al, q[i], r[i]);
        r[i] = ri;
        const double si = ri * dginv[i];
        s[i] = si;
        acc[0] = fma(ri, ri, acc[0]);
        acc[1] = fma(ri, si, acc[1]);
    }
    fs_block_partials<2>(acc, part2);
}

// |r| against the tolerance, then beta = (r, s)_new / (r, s)_old
__global__ void k_fs_cg_beta(int nb, const double *part2, FSCG *cg)
{
    if (fs_cg_over(cg)) return;
    double t[2];
    fs_sum_rows<2>(part2, nb, t);
    if (threadIdx.x != 0) return;
    cg->iters++;
    if (sqrt(t[0]) <= cg->tol || cg->iters >= cg->maxit) {
        cg->done = 1;
        return;
    }
    cg->beta = t[1] / cg->rz;
    cg->rz = t[1];
}

// p = s + beta p (and its FP32 copy, if kept)
__global__ void k_fs_cg_dir(long long L, const double *s, double *p, float *p32, const FSCG *cg)
{
    if (fs_cg_over(cg)) return;
    const double b = cg->beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
        const double v = fma(b, p[i], s[i]);
        p[i] = v;
        if (p32) p32[i] = (float)v;
    }
}

// z = x * dginv elementwise
__global__ void k_fs_scale(long long L, const double *x, const double *dginv, double *z)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        z[i] = x[i] * dginv[i];
}

// per cell: the inverse of the plastic deformation (row-major 3 x 3)
__global__ void k_fs_inv(long long N, const double *FP, double *FPinv)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double *a = FP + c * 9;
        double ci[9];
        ci[0] = a[4] * a[8] - a[5] * a[7]; ci[1] = a[2] * a[7] - a[1] * a[8]; ci[2] = a[1] * a[5] - a[2] * a[4];
        ci[3] = a[5] * a[6] - a[3] * a[8]; ci[4] = a[0] * a[8] - a[2] * a[6]; ci[5] = a[2] * a[3] - a[0] * a[5];
        ci[6] = a[3] * a[7] - a[4] * a[6]; ci[7] = a[1] * a[6] - a[0] * a[7]; ci[8] = a[0] * a[4] - a[1] * a[3];
        const double det = a[0] * ci[0] + a[1] * ci[3] + a[2] * ci[6];
        for (int q = 0; q < 9; q++) FPinv[c * 9 + q] = ci[q] / det;
    }
}

// per cell: one multiplicative J2 update at the cell-centre deformation
// Fbar + sum_a u_a (x) grad N_a(centre); bad[0] counts points whose update
// did not converge
__global__ void k_fs_return_cells(FSArgs A, const double *z, double sY, double H, double *FP, double *epsP,
                                  unsigned int *bad)
{
    const int d = A.d, na = 1 << d;
    const long long N = A.N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double F[9];
        fs_fbar(d, z + (size_t)d * N, F);
        for (int i = 0; i < d; i++)
            for (int k = 0; k < d; k++) {
                double t = F[3 * i + k];
                for (int a = 0; a < na; a++) {
                    double g = 1.0;
                    for (int l = 0; l < d; l++) g *= l == k ? (((a >> l) & 1) ? 1.0 : -1.0) : 0.5;
                    t += z[fs_node(A, c, a) * d + i] * g;
                }
                F[3 * i + k] = t;
            }
        if (d == 2) {
            F[2] = F[5] = F[6] = F[7] = 0.0;
            F[8] = 1.0;
        }
        double fp[9];
        for (int q = 0; q < 9; q++) fp[q] = FP[c * 9 + q];
        double ep = epsP[c];
        const double dT = 1.0 - A.Wf[c] * A.omega;
        if (fs_return_map(F, fp, ep, A.K[c], A.G[c], dT, sY, H)) atomicAdd(bad, 1u);
        for (int q = 0; q < 9; q++) FP[c * 9 + q] = fp[q];
        epsP[c] = ep;
    }
}

// independent points: F, FP, epsP, K, G, dT per point
__global__ void k_fs_return_points(int n, const double *F, double *FP, double *epsP, const double *K, const double *G,
                                   const double *dT, double sY, double H, unsigned int *bad)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double f[9], fp[9];
        for (int q = 0; q < 9; q++) { f[q] = F[c * 9 + q]; fp[q] = FP[c * 9 + q]; }
        double ep = epsP[c];
        if (fs_return_map(f, fp, ep, K[c], G[c], dT[c], sY, H)) atomicAdd(bad, 1u);
        for (int q = 0; q < 9; q++) FP[c * 9 + q] = fp[q];
        epsP[c] = ep;
    }
}

// per cell: d psi / d theta at fixed deformation (the cell-centre
// deformation of the state z) and plastic deformation: the elastic part of
// the order parameter's driving force (the derivative through W_f in d_T and
// through the mixture moduli), in forward mode along theta
//
// mode 1: instead, the small-strain coupling scalar tr eps_e that gives the
// marching update the same force.  K and G do not depend on theta (the solid
// phases share K_s, G_s), so d psi / d theta = -Omega (1 - h(phi_g)) h'(theta)
// d psi / d d_T, and the update's elastic term -3 eig0 (1 - h(phi_g))
// h'(theta) K_mix tr eps_e equals it for tr eps_e = Omega (d psi / d d_T) /
// (3 eig0 K_mix), K_mix = (1 - h(phi_g)) K_s + h(phi_g) K_g: the derivative is
// taken along d_T.
__global__ void k_fs_force(FSArgs A, const double *z, const double *theta, const double *phig, double Ks, double Gs,
                           double Kg, double Gg, double *force, int mode, double eig0)
{
    const int d = A.d, na = 1 << d;
    const long long N = A.N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double F[9];
        fs_fbar(d, z + (size_t)d * N, F);
        for (int i = 0; i < d; i++)
            for (int k = 0; k < d; k++) {
                double t = F[3 * i + k];
                for (int a = 0; a < na; a++) {
                    double g = 1.0;
                    for (int l = 0; l < d; l++) g *= l == k ? (((a >> l) & 1) ? 1.0 : -1.0) : 0.5;
                    t += z[fs_node(A, c, a) * d + i] * g;
                }
                F[3 * i + k] = t;
            }
        if (d == 2) {
            F[2] = F[5] = F[6] = F[7] = 0.0;
            F[8] = 1.0;
        }
        const FD th(theta[c], mode == 0 ? 1.0 : 0.0);
        const double hg = phig[c] * phig[c] * phig[c] * (phig[c] * (6.0 * phig[c] - 15.0) + 10.0);
        const FD ht = th * th * th * (th * (FD(6.0) * th - FD(15.0)) + FD(10.0));
        const FD wf = FD(1.0 - hg) * ht, ww = FD(1.0 - hg) * (FD(1.0) - ht);
        const FD K = (wf + ww) * FD(Ks) + FD(hg * Kg), G = (wf + ww) * FD(Gs) + FD(hg * Gg);
        FD dT = FD(1.0) - wf * FD(A.omega);
        if (mode == 1) dT.d = 1.0;
        const FD s = fd_pow(dT, -1.0 / 3.0);
        const double *Fi = A.FPinv ? A.FPinv + c * 9 : nullptr;
        FD Fe[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const double v = Fi ? F[3 * i] * Fi[j] + F[3 * i + 1] * Fi[3 + j] + F[3 * i + 2] * Fi[6 + j] : F[3 * i + j];
                Fe[3 * i + j] = s * FD(v);
            }
        const FD J = Fe[0] * (Fe[4] * Fe[8] - Fe[5] * Fe[7]) - Fe[1] * (Fe[3] * Fe[8] - Fe[5] * Fe[6]) +
                     Fe[2] * (Fe[3] * Fe[7] - Fe[4] * Fe[6]);
        FD I1(0.0);
        for (int q = 0; q < 9; q++) I1 = I1 + Fe[q] * Fe[q];
        const FD psi = dT * (FD(0.25) * K * (J * J - FD(1.0) - FD(2.0) * fd_log(J)) +
                             FD(0.5) * G * (fd_pow(J, -2.0 / 3.0) * I1 - FD(3.0)));
        const double Kmix = (1.0 - hg) * Ks + hg * Kg;
        // Kmix == 0 only in a pure gas cell with a zero gas modulus, where the
        // solid factor (1 - h(phi_g)) of the force vanishes: no coupling.
        force[c] = mode == 0 ? psi.d : (Kmix != 0.0 ? A.omega * psi.d / (3.0 * eig0 * Kmix) : 0.0);
    }
}

constexpr int FS_NB = 128;     // blocks of the reductions
constexpr int FS_CHUNK = 16;   // CG iterations launched between two host reads of the CG state
// the mixed method's CG stops at a relative residual of at least this: its
// FP32 products carry ~1e-7 relative rounding, more along smooth directions
// (whose nodal sums cancel), and tighter solves only add iterations (inexact
// Newton: the residual itself is FP64, so Newton still reaches its
// tolerance; at 64^3, 1e-5 took 1,382 CG iterations in 8 Newton steps, 1e-6
// 2,756 in 9, 1e-4 2,333 in 12)
constexpr double FS_MIXED_RTOL = 1e-5;

struct FSSolver {
    FSArgs A;
    long long N, nd, L;
    int m;
    double pbar[9];
    double *z = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *s = nullptr, *dz = nullptr, *dg = nullptr;
    double *dginv = nullptr;             // inverse Jacobi diagonal over [0, L)
    double *cf = nullptr;                // corner forces, N x 24 (FP32 in the mixed product)
    double *part = nullptr;              // FS_NB partials of host-read dot products
    double *part9 = nullptr, *partdot = nullptr;   // grid x 9 stress and grid (p, Hp) partials
    double *part2 = nullptr;             // 2 x grid partials of (r, r), (r, s)
    double *K = nullptr, *G = nullptr, *Wf = nullptr, *th = nullptr, *pg = nullptr;
    FSPack<double> *pk64 = nullptr;      // cell constants of the load step
    FSPack<float> *pk32 = nullptr;       // their FP32 copy (mixed)
    float *z32 = nullptr, *p32 = nullptr;  // FP32 copies of z and p (mixed)
    FSCG *cg = nullptr;                  // device CG state
    std::vector<void *> mem;
    std::vector<double> hp;
    int grid = 0;
    int mixed = 0;                       // FP32 Hessian-vector products
    cudaEvent_t ev[2 * FS_CHUNK];        // around each product of a chunk
    bool have_ev = false;
    double hvp_ms = 0.0;
    long long hvp_launches = 0;

    template <typename T>
    cudaError_t alloc(T **x, size_t n)
    {
        cudaError_t e = cudaMalloc((void **)x, sizeof(T) * (n ? n : 1));
        if (e == cudaSuccess) mem.push_back(*x);
        return e;
    }
    ~FSSolver()
    {
        for (void *v : mem) cudaFree(v);
        if (have_ev)
            for (cudaEvent_t &e : ev) cudaEventDestroy(e);
    }
    double dot(const double *a, const double *b)
    {
        k_fs_dot<<<FS_NB, 256>>>(L, a, b, part);
        cudaMemcpy(hp.data(), part, sizeof(double) * FS_NB, cudaMemcpyDeviceToHost);
        double t = 0.0;
        for (int k = 0; k < FS_NB; k++) t += hp[k];
        return t;
    }
    // the cell constants of the current load step (A.omega)
    void pack()
    {
        k_fs_pack<double><<<grid, 128>>>(A, pk64);
        if (mixed) k_fs_pack<float><<<grid, 128>>>(A, pk32);
    }
    // the residual of the state z into r (FP64); no host synchronisation
    void residual()
    {
        if (A.d == 3) k_fs_res<3><<<grid, 128>>>(A, pk64, z, cf, part9);
        else k_fs_res<2><<<grid, 128>>>(A, pk64, z, cf, part9);
        k_fs_gather<double><<<grid, 128>>>(A, cf, r, nullptr, nullptr, nullptr);
        Mat9 pb;
        for (int k = 0; k < 9; k++) pb.v[k] = pbar[k];
        k_fs_rows<<<1, 256>>>(A.d, grid, part9, pb, (double)N, r + nd);
    }
    // q = H p (events ev0/ev1 around the product kernel), then al
    void product(cudaEvent_t ev0, cudaEvent_t ev1)
    {
        const int d = A.d;
        if (ev0) cudaEventRecord(ev0);
        if (mixed) {
            float *cf32 = reinterpret_cast<float *>(cf);
            if (d == 3) k_fs_hvp<3, FDf><<<grid, 128>>>(A, pk32, z32, p32, cf32, part9, cg);
            else k_fs_hvp<2, FDf><<<grid, 128>>>(A, pk32, z32, p32, cf32, part9, cg);
            if (ev1) cudaEventRecord(ev1);
            k_fs_gather<float><<<grid, 128>>>(A, cf32, q, p, partdot, cg);
        } else {
            if (d == 3) k_fs_hvp<3, FD><<<grid, 128>>>(A, pk64, z, p, cf, part9, cg);
            else k_fs_hvp<2, FD><<<grid, 128>>>(A, pk64, z, p, cf, part9, cg);
            if (ev1) cudaEventRecord(ev1);
            k_fs_gather<double><<<grid, 128>>>(A, cf, q, p, partdot, cg);
        }
        k_fs_cg_alpha<<<1, 256>>>(d, grid, part9, grid, partdot, p + nd, q + nd, cg);
    }
    // PCG on H dz = -r from dz = 0 (r, p, q, s: residual, direction, H p,
    // preconditioned residual), then z += dz; returns the iterations taken
    int cg_solve(double rtol, int maxit)
    {
        cudaMemset(dz, 0, sizeof(double) * L);
        k_fs_axpby<<<grid, 128>>>(L, -1.0, r, 0.0, r);
        const double r0 = std::sqrt(dot(r, r));
        k_fs_scale<<<grid, 128>>>(L, r, dginv, s);
        cudaMemcpy(p, s, sizeof(double) * L, cudaMemcpyDeviceToDevice);
        if (mixed) {
            k_fs_to32<<<grid, 128>>>(L, z, z32);
            k_fs_to32<<<grid, 128>>>(L, p, p32);
        }
        FSCG h;
        memset(&h, 0, sizeof(h));
        h.rz = dot(r, s);
        h.tol = rtol * r0;
        h.maxit = maxit;
        cudaMemcpy(cg, &h, sizeof(h), cudaMemcpyHostToDevice);
        for (;;) {
            const int before = h.iters;
            for (int k = 0; k < FS_CHUNK; k++) {
                product(have_ev ? ev[2 * k] : nullptr, have_ev ? ev[2 * k + 1] : nullptr);
                k_fs_cg_update<<<grid, 128>>>(L, dginv, p, q, dz, r, s, cg, part2);
                k_fs_cg_beta<<<1, 256>>>(grid, part2, cg);
                k_fs_cg_dir<<<grid, 128>>>(L, s, p, mixed ? p32 : nullptr, cg);
            }
            cudaMemcpy(&h, cg, sizeof(h), cudaMemcpyDeviceToHost);
            // products that did work: one per completed iteration, and the
            // one that found no positive curvature
            const int ran = h.iters - before + (h.stop ? 1 : 0);
            if (have_ev)
                for (int k = 0; k < ran && k < FS_CHUNK; k++) {
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
                    hvp_ms += ms;
                }
            hvp_launches += ran;
            if (h.stop || h.done) break;
        }
        k_fs_axpby<<<grid, 128>>>(L, 1.0, dz, 1.0, z);
        return h.iters;
    }
    double maxabs(const double *x)
    {
        std::vector<double> h((size_t)L);
        cudaMemcpy(h.data(), x, sizeof(double) * L, cudaMemcpyDeviceToHost);
        double mx = 0.0;
        for (double v : h) mx = std::max(mx, std::fabs(v));
        return mx;
    }
};

int fs_fail(int code, const char *msg)
{
    g_fs_error = msg;
    return code;
}

// the equilibrium with the plastic deformation FP (N x 9, or null: identity)
// and, with cfg->plasticity, FP and epsP (N) updated by one return map per
// cell after it
int fs_force(const pf_config *cfg, const double *theta, const double *phi_g, double omega, const double *u,
             const double *Fbar, const double *FP, double *force, int mode);

int fs_run(const pf_config *cfg, const double *theta, const double *phi_g, double omega, const double *pbar,
           const pf_fs_opts *opts, double *u, double *Fbar, double *FP, double *epsP, pf_fs_stats *stats)
{
    if (!cfg || !theta || !phi_g || !opts || !u || !Fbar) return fs_fail(PF_EINVAL, "null argument");
    const int d = cfg->ndim;
    if (d != 2 && d != 3) return fs_fail(PF_EINVAL, "ndim must be 2 or 3");
    if (cfg->nx < 2 || cfg->ny < 2 || (d == 3 && cfg->nz < 2)) return fs_fail(PF_EINVAL, "grid sizes must be >= 2");
    if ((long long)cfg->nx * cfg->ny * (d == 3 ? cfg->nz : 1) * d + 6 >= (1LL << 31))
        return fs_fail(PF_EINVAL, "finite-strain grids hold fewer than 2^31 / ndim cells");
    if (opts->nload < 1 || opts->newton_maxit < 1 || !(opts->newton_tol > 0.0) || opts->cg_maxit < 1 ||
        !(opts->cg_rtol > 0.0 && opts->cg_rtol < 1.0))
        return fs_fail(PF_EINVAL, "invalid pf_fs_opts");
    if (opts->precision != PF_FP64 && opts->precision != PF_MIXED)
        return fs_fail(PF_EINVAL, "pf_fs_opts precision must be PF_FP64 or PF_MIXED");
    const double nu = cfg->p.nu, Es = cfg->p.E_s, Eg = Es * cfg->p.E_g_ratio;
    if (!(Es > 0.0) || !(nu > -1.0 && nu < 0.5)) return fs_fail(PF_EINVAL, "E_s > 0 and -1 < nu < 0.5 required");
    FSSolver S;
    S.mixed = opts->precision == PF_MIXED;
    S.N = (long long)cfg->nx * cfg->ny * (d == 3 ? cfg->nz : 1);
    S.m = d == 3 ? 6 : 3;
    S.nd = (long long)d * S.N;
    S.L = S.nd + S.m;
    S.hp.assign((size_t)FS_NB * 9, 0.0);
    for (int q = 0; q < 9; q++) S.pbar[q] = 0.0;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) S.pbar[3 * i + j] = pbar ? pbar[i * d + j] : (i == j ? -cfg->p.prestress : 0.0);
    const long long N = S.N, L = S.L;
    // one resident wave of the product kernel (4 blocks of 128 per SM): its
    // block partials, summed in FP64 by one block, stay few
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fs_fail(PF_ECUDA, "no CUDA device");
    S.grid = (int)std::min<long long>((N + 127) / 128, 4LL * std::max(sms, 1));
    double **bufs[11] = {&S.z, &S.r, &S.p, &S.q, &S.s, &S.dz, &S.dg, &S.dginv, &S.part, &S.part2, &S.partdot};
    const size_t lens[11] = {(size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)S.nd,
                             (size_t)L, (size_t)FS_NB, (size_t)S.grid * 2, (size_t)S.grid};
    for (int k = 0; k < 11; k++)
        if (S.alloc(bufs[k], lens[k]) != cudaSuccess) return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    if (S.alloc(&S.part9, (size_t)S.grid * 9) != cudaSuccess || S.alloc(&S.cg, 1) != cudaSuccess ||
        S.alloc(&S.pk64, (size_t)N) != cudaSuccess)
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    if (S.mixed && (S.alloc(&S.pk32, (size_t)N) != cudaSuccess || S.alloc(&S.z32, (size_t)L) != cudaSuccess ||
                    S.alloc(&S.p32, (size_t)L) != cudaSuccess))
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    {
        int ok = 0;
        while (ok < 2 * FS_CHUNK && cudaEventCreate(&S.ev[ok]) == cudaSuccess) ok++;
        if (ok < 2 * FS_CHUNK) {
            for (int k = 0; k < ok; k++) cudaEventDestroy(S.ev[k]);
            return fs_fail(PF_ECUDA, "cudaEventCreate failed");
        }
        S.have_ev = true;
    }
    if (S.alloc(&S.cf, (size_t)N * 24) != cudaSuccess || S.alloc(&S.K, N) != cudaSuccess || S.alloc(&S.G, N) != cudaSuccess || S.alloc(&S.Wf, N) != cudaSuccess ||
        S.alloc(&S.th, N) != cudaSuccess || S.alloc(&S.pg, N) != cudaSuccess)
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    cudaMemcpy(S.th, theta, sizeof(double) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(S.pg, phi_g, sizeof(double) * N, cudaMemcpyHostToDevice);
    double *dFP = nullptr, *dFPinv = nullptr, *dEp = nullptr;
    unsigned int *dbad = nullptr;
    if (FP) {
        if (S.alloc(&dFP, (size_t)N * 9) != cudaSuccess || S.alloc(&dFPinv, (size_t)N * 9) != cudaSuccess ||
            S.alloc(&dEp, N) != cudaSuccess || S.alloc(&dbad, 1) != cudaSuccess)
            return fs_fail(PF_ENOMEM, "cudaMalloc failed");
        cudaMemcpy(dFP, FP, sizeof(double) * N * 9, cudaMemcpyHostToDevice);
        cudaMemcpy(dEp, epsP, sizeof(double) * N, cudaMemcpyHostToDevice);
        cudaMemset(dbad, 0, sizeof(unsigned int));
    }
    const double Ks = Es / (3 * (1 - 2 * nu)), Gs = Es / (2 * (1 + nu));
    const double Kg = Eg / (3 * (1 - 2 * nu)), Gg = Eg / (2 * (1 + nu));
    k_fs_moduli<<<S.grid, 128>>>(N, S.th, S.pg, Ks, Gs, Kg, Gg, S.K, S.G, S.Wf);
    S.A.d = d; S.A.nx = cfg->nx; S.A.ny = cfg->ny; S.A.nz = d == 3 ? cfg->nz : 1; S.A.N = N;
    S.A.K = S.K; S.A.G = S.G; S.A.Wf = S.Wf; S.A.omega = 0.0;
    S.A.FPinv = nullptr;
    if (FP) {
        k_fs_inv<<<S.grid, 128>>>(N, dFP, dFPinv);
        S.A.FPinv = dFPinv;
    }
    // small-strain diagonals of a displacement dof per unit lambda and mu:
    // sum over Gauss points of w (dN_i)^2 and w (|dN|^2 + dN_i^2); equal
    // for every corner and component
    {
        const double ga = 0.5 - 0.5 / std::sqrt(3.0), gb = 0.5 + 0.5 / std::sqrt(3.0);
        const int na = 1 << d;
        double dl = 0.0, dm = 0.0;
        for (int g = 0; g < na; g++) {
            double dn[3];
            for (int k = 0; k < d; k++) {
                double v = 1.0;
                for (int l = 0; l < d; l++) {
                    const double xi = ((g >> l) & 1) ? gb : ga;
                    v *= l == k ? -1.0 : 1.0 - xi;     // corner a = 0
                }
                dn[k] = v;
            }
            double n2 = 0.0;
            for (int k = 0; k < d; k++) n2 += dn[k] * dn[k];
            dl += dn[0] * dn[0] / na;
            dm += (n2 + dn[0] * dn[0]) / na;
        }
        k_fs_diag<<<S.grid, 128>>>(S.A, dl, dm, S.dg);
    }
    // the mean-deformation dofs: scale of the summed moduli
    std::vector<double> hK((size_t)N), hG((size_t)N);
    cudaMemcpy(hK.data(), S.K, sizeof(double) * N, cudaMemcpyDeviceToHost);
    cudaMemcpy(hG.data(), S.G, sizeof(double) * N, cudaMemcpyDeviceToHost);
    double sK = 0.0, sG = 0.0;
    for (long long c = 0; c < N; c++) { sK += hK[c]; sG += hG[c]; }
    const double dgf = sK + 4.0 * sG / 3.0;
    k_fs_dginv<<<S.grid, 128>>>(L, S.nd, S.dg, dgf, S.dginv);
    // start: u = 0, Fbar = I
    std::vector<double> z0((size_t)L, 0.0);
    for (int i = 0; i < d; i++) z0[S.nd + i] = 1.0;
    cudaMemcpy(S.z, z0.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
    pf_fs_stats st;
    memset(&st, 0, sizeof(st));
    double res = 0.0;
    for (int step = 1; step <= opts->nload; step++) {
        S.A.omega = omega * step / opts->nload;
        S.pack();
        for (int it = 0;; it++) {
            S.residual();
            res = S.maxabs(S.r);
            if (res <= opts->newton_tol) break;
            if (it == opts->newton_maxit) {
                st.residual = res;
                st.hvp_ms = S.hvp_ms;
                st.hvp_launches = S.hvp_launches;
                if (stats) *stats = st;
                return fs_fail(PF_ENOTCONV, "finite-strain Newton iteration did not converge");
            }
            st.newton_iters++;
            st.cg_iters += S.cg_solve(S.mixed ? std::max(opts->cg_rtol, FS_MIXED_RTOL) : opts->cg_rtol, opts->cg_maxit);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fs_fail(PF_ECUDA, cudaGetErrorString(e));
    std::vector<double> zh((size_t)L);
    cudaMemcpy(zh.data(), S.z, sizeof(double) * L, cudaMemcpyDeviceToHost);
    memcpy(u, zh.data(), sizeof(double) * S.nd);
    double fb[9];
    for (int q = 0; q < 9; q++) fb[q] = 0.0;
    const double *zf = zh.data() + S.nd;
    if (d == 3) {
        fb[0] = zf[0]; fb[4] = zf[1]; fb[8] = zf[2];
        fb[5] = fb[7] = zf[3]; fb[2] = fb[6] = zf[4]; fb[1] = fb[3] = zf[5];
    } else {
        fb[0] = zf[0]; fb[4] = zf[1]; fb[1] = fb[3] = zf[2];
    }
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) Fbar[i * d + j] = fb[3 * i + j];
    st.residual = res;
    st.hvp_ms = S.hvp_ms;
    st.hvp_launches = S.hvp_launches;
    if (FP && cfg->plasticity) {
        S.A.omega = omega;
        k_fs_return_cells<<<S.grid, 64>>>(S.A, S.z, cfg->p.sigma_Y, cfg->p.H_hard, dFP, dEp, dbad);
        unsigned int nbad = 0;
        cudaMemcpy(&nbad, dbad, sizeof(unsigned int), cudaMemcpyDeviceToHost);
        cudaMemcpy(FP, dFP, sizeof(double) * N * 9, cudaMemcpyDeviceToHost);
        cudaMemcpy(epsP, dEp, sizeof(double) * N, cudaMemcpyDeviceToHost);
        if (nbad) {
            if (stats) *stats = st;
            return fs_fail(PF_ENOTCONV, "return map did not converge");
        }
    }
    if (stats) *stats = st;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fs_fail(PF_ECUDA, cudaGetErrorString(e));
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_finite_strain_solve(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                           const double *pbar, const pf_fs_opts *opts, double *u, double *Fbar, pf_fs_stats *stats)
{
    return fs_run(cfg, theta, phi_g, omega, pbar, opts, u, Fbar, nullptr, nullptr, stats);
}

int pf_finite_strain_step(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                          const double *pbar, const pf_fs_opts *opts, double *u, double *Fbar, double *FP,
                          double *epsP, pf_fs_stats *stats)
{
    if (!FP || !epsP) return fs_fail(PF_EINVAL, "FP and epsP are required");
    return fs_run(cfg, theta, phi_g, omega, pbar, opts, u, Fbar, FP, epsP, stats);
}

int pf_fs_coupling(const pf_config *cfg, const double *theta, const double *phi_g, double omega, const double *u,
                   const double *Fbar, const double *FP, double *trE)
{
    if (cfg && cfg->p.eig0 == 0.0) return fs_fail(PF_EINVAL, "eig0 must be nonzero");
    return fs_force(cfg, theta, phi_g, omega, u, Fbar, FP, trE, 1);
}

int pf_fs_elastic_force(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                        const double *u, const double *Fbar, const double *FP, double *force)
{
    return fs_force(cfg, theta, phi_g, omega, u, Fbar, FP, force, 0);
}

}  // extern "C"

namespace {

int fs_force(const pf_config *cfg, const double *theta, const double *phi_g, double omega, const double *u,
             const double *Fbar, const double *FP, double *force, int mode)
{
    if (!cfg || !theta || !phi_g || !u || !Fbar || !force) return fs_fail(PF_EINVAL, "null argument");
    const int d = cfg->ndim;
    if (d != 2 && d != 3) return fs_fail(PF_EINVAL, "ndim must be 2 or 3");
    if (cfg->nx < 2 || cfg->ny < 2 || (d == 3 && cfg->nz < 2)) return fs_fail(PF_EINVAL, "grid sizes must be >= 2");
    if ((long long)cfg->nx * cfg->ny * (d == 3 ? cfg->nz : 1) * d + 6 >= (1LL << 31))
        return fs_fail(PF_EINVAL, "finite-strain grids hold fewer than 2^31 / ndim cells");
    const double nu = cfg->p.nu, Es = cfg->p.E_s, Eg = Es * cfg->p.E_g_ratio;
    const long long N = (long long)cfg->nx * cfg->ny * (d == 3 ? cfg->nz : 1);
    const int m = d == 3 ? 6 : 3;
    // the state vector: u, then the symmetric components of Fbar
    std::vector<double> z((size_t)d * N + m);
    memcpy(z.data(), u, sizeof(double) * d * N);
    if (d == 3) {
        const double zf[6] = {Fbar[0], Fbar[4], Fbar[8], Fbar[5], Fbar[2], Fbar[1]};
        memcpy(z.data() + d * N, zf, sizeof(zf));
    } else {
        const double zf[3] = {Fbar[0], Fbar[3], Fbar[1]};
        memcpy(z.data() + d * N, zf, sizeof(zf));
    }
    FSSolver S;          // device buffers freed with it
    double *dz, *dth, *dpg, *dF, *dFP = nullptr, *dFPinv = nullptr;
    if (S.alloc(&dz, z.size()) != cudaSuccess || S.alloc(&dth, N) != cudaSuccess || S.alloc(&dpg, N) != cudaSuccess ||
        S.alloc(&dF, N) != cudaSuccess)
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    if (FP && (S.alloc(&dFP, (size_t)N * 9) != cudaSuccess || S.alloc(&dFPinv, (size_t)N * 9) != cudaSuccess))
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    cudaMemcpy(dz, z.data(), sizeof(double) * z.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dth, theta, sizeof(double) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(dpg, phi_g, sizeof(double) * N, cudaMemcpyHostToDevice);
    const int grid = (int)std::min<long long>((N + 127) / 128, 4096);
    FSArgs A;
    memset(&A, 0, sizeof(A));
    A.d = d; A.nx = cfg->nx; A.ny = cfg->ny; A.nz = d == 3 ? cfg->nz : 1; A.N = N; A.omega = omega;
    if (FP) {
        cudaMemcpy(dFP, FP, sizeof(double) * N * 9, cudaMemcpyHostToDevice);
        k_fs_inv<<<grid, 128>>>(N, dFP, dFPinv);
        A.FPinv = dFPinv;
    }
    const double Ks = Es / (3 * (1 - 2 * nu)), Gs = Es / (2 * (1 + nu));
    const double Kg = Eg / (3 * (1 - 2 * nu)), Gg = Eg / (2 * (1 + nu));
    k_fs_force<<<grid, 128>>>(A, dz, dth, dpg, Ks, Gs, Kg, Gg, dF, mode, cfg->p.eig0);
    cudaMemcpy(force, dF, sizeof(double) * N, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fs_fail(PF_ECUDA, cudaGetErrorString(e));
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_fs_return_map(int n, const double *F, double *FP, double *epsP, const double *K, const double *G,
                     const double *dT, double sigma_Y, double H)
{
    if (n < 0 || (n > 0 && (!F || !FP || !epsP || !K || !G || !dT))) return fs_fail(PF_EINVAL, "null argument");
    if (n == 0) return PF_OK;
    double *b[7] = {};
    const size_t len[7] = {(size_t)n * 9, (size_t)n * 9, (size_t)n, (size_t)n, (size_t)n, (size_t)n, 1};
    for (int k = 0; k < 7; k++)
        if (cudaMalloc((void **)&b[k], sizeof(double) * len[k]) != cudaSuccess) {
            for (int j = 0; j < k; j++) cudaFree(b[j]);
            return fs_fail(PF_ENOMEM, "cudaMalloc failed");
        }
    cudaMemcpy(b[0], F, sizeof(double) * n * 9, cudaMemcpyHostToDevice);
    cudaMemcpy(b[1], FP, sizeof(double) * n * 9, cudaMemcpyHostToDevice);
    cudaMemcpy(b[2], epsP, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b[3], K, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b[4], G, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b[5], dT, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemset(b[6], 0, sizeof(double));
    unsigned int *bad = reinterpret_cast<unsigned int *>(b[6]);
    k_fs_return_points<<<(n + 63) / 64, 64>>>(n, b[0], b[1], b[2], b[3], b[4], b[5], sigma_Y, H, bad);
    unsigned int nbad = 0;
    cudaMemcpy(&nbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    cudaMemcpy(FP, b[1], sizeof(double) * n * 9, cudaMemcpyDeviceToHost);
    cudaMemcpy(epsP, b[2], sizeof(double) * n, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    for (int k = 0; k < 7; k++) cudaFree(b[k]);
    if (e != cudaSuccess) return fs_fail(PF_ECUDA, cudaGetErrorString(e));
    if (nbad) return fs_fail(PF_ENOTCONV, "return map did not converge");
    return PF_OK;
}

const char *pf_fs_last_error(void) { return g_fs_error.c_str(); }

}  // extern "C"
