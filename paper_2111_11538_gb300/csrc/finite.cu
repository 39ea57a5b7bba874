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

struct FSArgs {
    int d, nx, ny, nz;
    long long N;
    const double *K, *G, *Wf;    // per cell
    const double *FPinv;         // per cell 3 x 3 row-major inverse plastic deformation, or null (identity)
    double omega;                // transformation of this load step
};

// local shape-function derivative dN/dx_k of corner a at Gauss point g
// (bit l of a: corner offset along axis l; bit l of g: Gauss abscissa
// 1/2 +- 1/(2 sqrt 3) along axis l)
__device__ __forceinline__ double dshape(int d, int g, int a, int k)
{
    const double ga = 0.5 - 0.5 / sqrt(3.0), gb = 0.5 + 0.5 / sqrt(3.0);
    double v = 1.0;
    for (int l = 0; l < d; l++) {
        const int bit = (a >> l) & 1;
        const double xi = ((g >> l) & 1) ? gb : ga;
        v *= l == k ? (bit ? 1.0 : -1.0) : (bit ? xi : 1.0 - xi);
    }
    return v;
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

// first Piola stress of cell c at deformation F (3 x 3, row-major)
template <typename S>
__device__ void fs_piola(const FSArgs &A, long long c, const S (&F)[9], S (&P)[9])
{
    const double dT = 1.0 - A.Wf[c] * A.omega, s = pow(dT, -1.0 / 3.0);
    const double K = A.K[c], G = A.G[c];
    const double *Fi = A.FPinv ? A.FPinv + c * 9 : nullptr;
    S Fe[9];
    if (Fi) {
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                Fe[3 * i + j] = S(s) * (F[3 * i] * S(Fi[j]) + F[3 * i + 1] * S(Fi[3 + j]) + F[3 * i + 2] * S(Fi[6 + j]));
    } else {
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
    for (int q = 0; q < 9; q++) I1 = I1 + Fe[q] * Fe[q];
    // d phi / d F_E = K/2 (J^2 - 1) F_E^-T + G J^(-2/3) (F_E - I1/3 F_E^-T)
    const S a1 = S(0.5 * K) * (J * J - S(1.0)) / J;          // times cof = J F^-T
    const S jm = fd_pow(J, -2.0 / 3.0);
    const S a2 = S(G) * jm;
    const S a3 = a2 * I1 / (S(3.0) * J);
    if (Fi) {
        S D[9];
        for (int q = 0; q < 9; q++) D[q] = a1 * cof[q] + a2 * Fe[q] - a3 * cof[q];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                P[3 * i + j] = S(dT * s) * (D[3 * i] * S(Fi[3 * j]) + D[3 * i + 1] * S(Fi[3 * j + 1]) +
                                            D[3 * i + 2] * S(Fi[3 * j + 2]));
    } else {
        for (int q = 0; q < 9; q++) P[q] = S(dT * s) * (a1 * cof[q] + a2 * Fe[q] - a3 * cof[q]);
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

// forces of cell c on its 2^d corners (f[a * d + i]) and its weighted sum of
// the Gauss-point stresses (pm, d x d row-major), for the state (u, Fbar)
// given by ld_u(node, comp) and fb (3 x 3 symmetric)
template <typename S, class LU>
__device__ void fs_cell(const FSArgs &A, long long c, LU &&ld_u, const S (&fb)[9], S (&f)[24], S (&pm)[9])
{
    const int d = A.d, na = 1 << d;
    const double w = 1.0 / na;
    S ua[8][3];
    for (int a = 0; a < na; a++) {
        const long long n = fs_node(A, c, a);
        for (int i = 0; i < d; i++) ua[a][i] = ld_u(n, i);
    }
    for (int q = 0; q < 24; q++) f[q] = S(0.0);
    for (int q = 0; q < 9; q++) pm[q] = S(0.0);
    for (int g = 0; g < na; g++) {
        S F[9];
        for (int q = 0; q < 9; q++) F[q] = fb[q];
        for (int i = 0; i < d; i++)
            for (int k = 0; k < d; k++) {
                S t = F[3 * i + k];
                for (int a = 0; a < na; a++) t = t + ua[a][i] * S(dshape(d, g, a, k));
                F[3 * i + k] = t;
            }
        if (d == 2) {
            F[2] = F[5] = F[6] = F[7] = S(0.0);
            F[8] = S(1.0);
        }
        S P[9];
        fs_piola(A, c, F, P);
        for (int a = 0; a < na; a++)
            for (int i = 0; i < d; i++) {
                S t = f[a * d + i];
                for (int k = 0; k < d; k++) t = t + S(w) * P[3 * i + k] * S(dshape(d, g, a, k));
                f[a * d + i] = t;
            }
        for (int i = 0; i < d; i++)
            for (int k = 0; k < d; k++) pm[3 * i + k] = pm[3 * i + k] + S(w) * P[3 * i + k];
    }
}

// symmetric Fbar (3 x 3) from the m trailing entries of a vector
__device__ __forceinline__ void fs_fbar(int d, const double *zf, double (&fb)[9])
{
    for (int q = 0; q < 9; q++) fb[q] = 0.0;
    if (d == 3) {
        fb[0] = zf[0]; fb[4] = zf[1]; fb[8] = zf[2];
        fb[5] = fb[7] = zf[3]; fb[2] = fb[6] = zf[4]; fb[1] = fb[3] = zf[5];
    } else {
        fb[0] = zf[0]; fb[4] = zf[1]; fb[1] = fb[3] = zf[2];
    }
}

// per cell: corner forces (value, or with v != nullptr the directional
// derivative along v) into cf[c][a][i] and the stress sums into pc[c][9]
__global__ void k_fs_cells(FSArgs A, const double *z, const double *v, double *cf, double *pc)
{
    const int d = A.d, na = 1 << d;
    const long long N = A.N;
    const double *zf = z + (size_t)d * N, *vf = v ? v + (size_t)d * N : nullptr;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        if (!v) {
            double fb[9], f[24], pm[9];
            fs_fbar(d, zf, fb);
            fs_cell<double>(A, c, [&](long long n, int i) { return z[n * d + i]; }, fb, f, pm);
            for (int q = 0; q < na * d; q++) cf[c * 24 + q] = f[q];
            for (int q = 0; q < 9; q++) pc[c * 9 + q] = pm[q];
        } else {
            double fb0[9], fb1[9];
            fs_fbar(d, zf, fb0);
            fs_fbar(d, vf, fb1);
            FD fb[9], f[24], pm[9];
            for (int q = 0; q < 9; q++) fb[q] = FD(fb0[q], fb1[q]);
            fs_cell<FD>(A, c, [&](long long n, int i) { return FD(z[n * d + i], v[n * d + i]); }, fb, f, pm);
            for (int q = 0; q < na * d; q++) cf[c * 24 + q] = f[q].d;
            for (int q = 0; q < 9; q++) pc[c * 9 + q] = pm[q].d;
        }
    }
}

// nodal forces: each node sums the corner forces of its 2^d cells; node 0
// is held (zero)
__global__ void k_fs_gather(FSArgs A, const double *cf, double *out)
{
    const int d = A.d, na = 1 << d;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < A.N; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % A.nx);
        const long long r = n / A.nx;
        const int j = (int)(r % A.ny), k = (int)(r / A.ny);
        double s[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < na; a++) {
            const int ci = (i - (a & 1) + A.nx) % A.nx, cj = (j - ((a >> 1) & 1) + A.ny) % A.ny;
            const int ck = d == 3 ? (k - ((a >> 2) & 1) + A.nz) % A.nz : 0;
            const long long c = ci + (long long)A.nx * (cj + (long long)A.ny * ck);
            for (int q = 0; q < d; q++) s[q] += cf[c * 24 + a * d + q];
        }
        for (int q = 0; q < d; q++) out[n * d + q] = n == 0 ? 0.0 : s[q];
    }
}

// block partial sums of the cells' stress sums (fixed order)
__global__ void k_fs_psum(long long N, const double *pc, double *part)
{
    __shared__ double sh[9][8];
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        for (int q = 0; q < 9; q++) s[q] += pc[c * 9 + q];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 9; q++) {
        double t = s[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[threadIdx.x][k];
        part[blockIdx.x * 9 + threadIdx.x] = t;
    }
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

// y = a x + b y on [0, L); z = x / dg elementwise with dg over [0, nd) and
// 1 / dgf beyond (mode 1)
__global__ void k_fs_axpby(long long L, double a, const double *x, double b, double *y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
__global__ void k_fs_precond(long long L, long long nd, const double *x, const double *dg, double dgf, double *z)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        z[i] = i < nd ? x[i] / dg[i] : x[i] / dgf;
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

struct FSSolver {
    FSArgs A;
    long long N, nd, L;
    int m;
    double pbar[9];
    double *z = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *s = nullptr, *dz = nullptr, *dg = nullptr;
    double *cf = nullptr, *pc = nullptr, *part = nullptr, *K = nullptr, *G = nullptr, *Wf = nullptr;
    double *th = nullptr, *pg = nullptr;
    std::vector<void *> mem;
    std::vector<double> hp;
    int grid = 0;

    cudaError_t alloc(double **x, size_t n)
    {
        cudaError_t e = cudaMalloc((void **)x, sizeof(double) * (n ? n : 1));
        if (e == cudaSuccess) mem.push_back(*x);
        return e;
    }
    ~FSSolver()
    {
        for (void *v : mem) cudaFree(v);
    }
    double dot(const double *a, const double *b)
    {
        k_fs_dot<<<FS_NB, 256>>>(L, a, b, part);
        cudaMemcpy(hp.data(), part, sizeof(double) * FS_NB, cudaMemcpyDeviceToHost);
        double t = 0.0;
        for (int k = 0; k < FS_NB; k++) t += hp[k];
        return t;
    }
    // the residual (v == nullptr) or its directional derivative along v,
    // into out (length L)
    void apply(const double *v, double *out)
    {
        const int d = A.d;
        k_fs_cells<<<grid, 128>>>(A, z, v, cf, pc);
        k_fs_gather<<<grid, 128>>>(A, cf, out);
        k_fs_psum<<<FS_NB, 256>>>(N, pc, part);
        cudaMemcpy(hp.data(), part, sizeof(double) * FS_NB * 9, cudaMemcpyDeviceToHost);
        double ps[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < FS_NB; k++)
            for (int q = 0; q < 9; q++) ps[q] += hp[(size_t)k * 9 + q];
        if (!v)
            for (int q = 0; q < 9; q++) ps[q] -= (double)N * pbar[q];
        double rf[6];
        const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
        const int i2[3] = {0, 1, 0}, j2[3] = {0, 1, 1};
        for (int k = 0; k < m; k++) {
            const int i = d == 3 ? ii[k] : i2[k], j = d == 3 ? jj[k] : j2[k];
            rf[k] = i == j ? ps[3 * i + i] : ps[3 * i + j] + ps[3 * j + i];
        }
        cudaMemcpy(out + nd, rf, sizeof(double) * m, cudaMemcpyHostToDevice);
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
    if (opts->nload < 1 || opts->newton_maxit < 1 || !(opts->newton_tol > 0.0) || opts->cg_maxit < 1 ||
        !(opts->cg_rtol > 0.0 && opts->cg_rtol < 1.0))
        return fs_fail(PF_EINVAL, "invalid pf_fs_opts");
    const double nu = cfg->p.nu, Es = cfg->p.E_s, Eg = Es * cfg->p.E_g_ratio;
    if (!(Es > 0.0) || !(nu > -1.0 && nu < 0.5)) return fs_fail(PF_EINVAL, "E_s > 0 and -1 < nu < 0.5 required");
    FSSolver S;
    S.N = (long long)cfg->nx * cfg->ny * (d == 3 ? cfg->nz : 1);
    S.m = d == 3 ? 6 : 3;
    S.nd = (long long)d * S.N;
    S.L = S.nd + S.m;
    S.hp.assign((size_t)FS_NB * 9, 0.0);
    for (int q = 0; q < 9; q++) S.pbar[q] = 0.0;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) S.pbar[3 * i + j] = pbar ? pbar[i * d + j] : (i == j ? -cfg->p.prestress : 0.0);
    const long long N = S.N, L = S.L;
    double **bufs[8] = {&S.z, &S.r, &S.p, &S.q, &S.s, &S.dz, &S.dg, &S.part};
    const size_t lens[8] = {(size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)L, (size_t)S.nd,
                            (size_t)FS_NB * 9};
    for (int k = 0; k < 8; k++)
        if (S.alloc(bufs[k], lens[k]) != cudaSuccess) return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    if (S.alloc(&S.cf, (size_t)N * 24) != cudaSuccess || S.alloc(&S.pc, (size_t)N * 9) != cudaSuccess ||
        S.alloc(&S.K, N) != cudaSuccess || S.alloc(&S.G, N) != cudaSuccess || S.alloc(&S.Wf, N) != cudaSuccess ||
        S.alloc(&S.th, N) != cudaSuccess || S.alloc(&S.pg, N) != cudaSuccess)
        return fs_fail(PF_ENOMEM, "cudaMalloc failed");
    cudaMemcpy(S.th, theta, sizeof(double) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(S.pg, phi_g, sizeof(double) * N, cudaMemcpyHostToDevice);
    double *dFP = nullptr, *dFPinv = nullptr, *dEp = nullptr;
    unsigned int *dbad = nullptr;
    if (FP) {
        if (S.alloc(&dFP, (size_t)N * 9) != cudaSuccess || S.alloc(&dFPinv, (size_t)N * 9) != cudaSuccess ||
            S.alloc(&dEp, N) != cudaSuccess || S.alloc(reinterpret_cast<double **>(&dbad), 1) != cudaSuccess)
            return fs_fail(PF_ENOMEM, "cudaMalloc failed");
        cudaMemcpy(dFP, FP, sizeof(double) * N * 9, cudaMemcpyHostToDevice);
        cudaMemcpy(dEp, epsP, sizeof(double) * N, cudaMemcpyHostToDevice);
        cudaMemset(dbad, 0, sizeof(unsigned int));
    }
    S.grid = (int)std::min<long long>((N + 127) / 128, 4096);
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
    // start: u = 0, Fbar = I
    std::vector<double> z0((size_t)L, 0.0);
    for (int i = 0; i < d; i++) z0[S.nd + i] = 1.0;
    cudaMemcpy(S.z, z0.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
    pf_fs_stats st;
    memset(&st, 0, sizeof(st));
    double res = 0.0;
    for (int step = 1; step <= opts->nload; step++) {
        S.A.omega = omega * step / opts->nload;
        for (int it = 0;; it++) {
            S.apply(nullptr, S.r);
            res = S.maxabs(S.r);
            if (res <= opts->newton_tol) break;
            if (it == opts->newton_maxit) {
                st.residual = res;
                if (stats) *stats = st;
                return fs_fail(PF_ENOTCONV, "finite-strain Newton iteration did not converge");
            }
            st.newton_iters++;
            // PCG on H dz = -r from dz = 0 (r, p, q, s: residual, direction,
            // H p, preconditioned residual)
            cudaMemset(S.dz, 0, sizeof(double) * L);
            k_fs_axpby<<<S.grid, 128>>>(L, -1.0, S.r, 0.0, S.r);
            const double r0 = std::sqrt(S.dot(S.r, S.r));
            k_fs_precond<<<S.grid, 128>>>(L, S.nd, S.r, S.dg, dgf, S.s);
            cudaMemcpy(S.p, S.s, sizeof(double) * L, cudaMemcpyDeviceToDevice);
            double rz = S.dot(S.r, S.s);
            for (int k = 0; k < opts->cg_maxit; k++) {
                S.apply(S.p, S.q);
                const double pq = S.dot(S.p, S.q);
                if (!(pq > 0.0)) break;                  // not positive definite along p
                const double al = rz / pq;
                k_fs_axpby<<<S.grid, 128>>>(L, al, S.p, 1.0, S.dz);
                k_fs_axpby<<<S.grid, 128>>>(L, -al, S.q, 1.0, S.r);
                st.cg_iters++;
                if (std::sqrt(S.dot(S.r, S.r)) <= opts->cg_rtol * r0) break;
                k_fs_precond<<<S.grid, 128>>>(L, S.nd, S.r, S.dg, dgf, S.s);
                const double rz1 = S.dot(S.r, S.s);
                k_fs_axpby<<<S.grid, 128>>>(L, 1.0, S.s, rz1 / rz, S.p);
                rz = rz1;
            }
            k_fs_axpby<<<S.grid, 128>>>(L, 1.0, S.dz, 1.0, S.z);
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
