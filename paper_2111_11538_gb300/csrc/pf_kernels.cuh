// Kernels of the coupled step.  See pf_device.cuh for layout and helpers.
#pragma once
#include "pf_device.cuh"

namespace pfdev {

// ---------------------------------------------------------------------------
// K2: per-cell Lame parameters and eigenstress C : eps* (Voigt) for the
// mechanics right-hand side.  eps* = eig0 W_f I + eps_p (linearised
// transformation strain of Sec. 2.2, plus the plastic strain).
// ---------------------------------------------------------------------------
template <typename T, int D>
struct FieldPtrs {
    const T *theta, *phig, *xO, *xH, *xW, *mob;
    const unsigned char *mask;
    T *theta_o, *xO_o, *xH_o, *xW_o;
    T *muO, *MO;
    T *trE, *devE2;
    T *lam, *mu;
    T *sig[6];
    T *ep[6];
    T *alpha;
    T *sigma_out[6];
    T *u[3];
};

// One grid (instance) of a launch.  A launch serves one or many instances:
// its blocks are split into consecutive ranges, one per job, and every block
// works on its job's grid only (block bid of nbk within the job).
// Model constants in the storage type, converted once on the host: GB300's
// FP64 pipe is narrow, and per-tile double->float conversions alone can
// saturate it in a kernel that otherwise runs in FP32.
template <typename T>
struct CellConst {
    T c, kappa, DOs, DOg, DHs, DHg, DWs, DWg;      // mu_O, M_O, D_H, D_H2O
    T eps2, dt, Ks, Gs, Kg, w2, eig3, Lh, kf, xHbc; // update
};

template <typename T>
inline CellConst<T> cell_const(const Params &P)
{
    CellConst<T> k;
    k.c = T(P.c); k.kappa = T(P.kappa);
    k.DOs = T(P.DOs); k.DOg = T(P.DOg); k.DHs = T(P.DHs); k.DHg = T(P.DHg); k.DWs = T(P.DWs); k.DWg = T(P.DWg);
    k.eps2 = T(2 * P.eps); k.dt = T(P.dt); k.Ks = T(P.Ks); k.Gs = T(P.Gs); k.Kg = T(P.Kg);
    k.w2 = T(2 * P.w); k.eig3 = T(P.eig0) * T(3); k.Lh = T(-0.5 * P.L); k.kf = T(P.kfor); k.xHbc = T(P.xHbc);
    return k;
}

template <typename T, int D>
struct CellJob {
    Params P;
    CellConst<T> K;
    FieldPtrs<T, D> F;
    const Scalars *sc;       // mean strain for the return map
    double *partials;        // per-block sums of the update
    unsigned int *counter;   // last-block counter of the update
    Diag *dg;
    int block0, nblocks;
    int strip_rows;          // k_fusedz: planes per chunk along the marching axis
};

// Job of this block: the last job whose first block is <= blockIdx.x (jobs
// are sorted by block0).
template <typename Job>
__device__ __forceinline__ const Job *my_job(const Job *jobs, int njobs)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return jobs + lo;
}

// The jobs of a cell launch: a device table (sorted by block0), or, when the
// table is null, the single job carried in the launch parameters (used by
// callers that must not copy anything to the device before the launch).
template <typename Job>
struct JobSet {
    const Job *table;
    int njobs;
    Job one;
};

template <typename Job>
__device__ __forceinline__ const Job *my_job(const JobSet<Job> &js)
{
    return js.table ? my_job(js.table, js.njobs) : &js.one;
}

#define PF_CELL_JOB_PROLOGUE                                   \
    const CellJob<T, D> *J_ = my_job(js);                      \
    const Params P = J_->P;                                    \
    const FieldPtrs<T, D> F = J_->F;                           \
    const long long bid = (long long)blockIdx.x - J_->block0;  \
    const long long nbk = J_->nblocks;

template <typename T, int D>
__global__ void k_setup(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    constexpr int NV = Dims<D>::NV;
    PF_CELL_JOB_PROLOGUE
    for (long long c = bid * blockDim.x + threadIdx.x; c < P.N; c += nbk * blockDim.x) {
        T Wf, Ww, Wg;
        phase_weights(F.theta[c], F.phig[c], Wf, Ww, Wg);
        T K = (Wf + Ww) * T(P.Ks) + Wg * T(P.Kg);
        T G = (Wf + Ww) * T(P.Gs) + Wg * T(P.Gg);
        T lam = K - T(2.0 / 3.0) * G;
        F.lam[c] = lam;
        F.mu[c] = G;
        T e0 = T(P.eig0) * Wf;
        // eigenstrain tensor components xx, yy, zz, yz, xz, xy
        T es[6];
        if constexpr (D == 2) {
            es[0] = e0 + F.ep[0][c]; es[1] = e0 + F.ep[1][c]; es[2] = e0 + F.ep[2][c];
            es[3] = T(0); es[4] = T(0); es[5] = F.ep[3][c];
        } else {
#pragma unroll
            for (int v = 0; v < 6; v++) es[v] = (v < 3 ? e0 : T(0)) + F.ep[v][c];
        }
        T tr = es[0] + es[1] + es[2];
        if constexpr (D == 2) {
            F.sig[0][c] = lam * tr + T(2) * G * es[0];
            F.sig[1][c] = lam * tr + T(2) * G * es[1];
            F.sig[2][c] = T(2) * G * es[5];
        } else {
#pragma unroll
            for (int v = 0; v < 3; v++) F.sig[v][c] = lam * tr + T(2) * G * es[v];
#pragma unroll
            for (int v = 3; v < 6; v++) F.sig[v][c] = T(2) * G * es[v];
        }
        (void)NV;
    }
}

// Voigt stiffness D(lam, mu) times e (double, used for the few mean-strain dofs)
template <int D>
__device__ __forceinline__ void dmat_mul(double lam, double mu, const double *e, double *s)
{
    if constexpr (D == 2) {
        double tr = e[0] + e[1];
        s[0] = lam * tr + 2 * mu * e[0]; s[1] = lam * tr + 2 * mu * e[1]; s[2] = mu * e[2];
    } else {
        double tr = e[0] + e[1] + e[2];
        for (int v = 0; v < 3; v++) s[v] = lam * tr + 2 * mu * e[v];
        for (int v = 3; v < 6; v++) s[v] = mu * e[v];
    }
}

template <int D>
__device__ __forceinline__ void node_of(int a, int &ox, int &oy, int &oz)
{
    ox = a & 1; oy = (a >> 1) & 1; oz = D == 3 ? (a >> 2) & 1 : 0;
}

// ---------------------------------------------------------------------------
// K5: per-cell stress and J2 radial return (Sec. 2.3 PlaTwoJ, small-strain
// form): yield |dev sigma| - sqrt(2/3)(sigma_Y + H a) <= 0, flow along
// dev sigma / |dev sigma|, da = dlambda = f / (2G + sqrt(2/3) H).
// Outputs eps_p, alpha, the coupling scalars t = tr eps_e and s = |dev eps_e|^2
// and the stress.
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void k_return(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    constexpr int NN = Dims<D>::NN, NV = Dims<D>::NV;
    PF_CELL_JOB_PROLOGUE
    const Scalars *sc = J_->sc;
    const int want_sigma = 1;
    double Ed[6];
    for (int v = 0; v < NV; v++) Ed[v] = sc->E[v];
    for (long long c = bid * blockDim.x + threadIdx.x; c < P.N; c += nbk * blockDim.x) {
        int i, j, k;
        cell_coords<D>(P, c, i, j, k);
        T ue[NN][D];
#pragma unroll
        for (int b = 0; b < NN; b++) {
            int px, py, pz;
            node_of<D>(b, px, py, pz);
            const long long m = lin<D>(P, i + px, j + py, k + pz);
#pragma unroll
            for (int d = 0; d < D; d++) ue[b][d] = F.u[d][m];
        }
        T ev[NV];
        avg_strain<T, D>(ue, ev);
#pragma unroll
        for (int v = 0; v < NV; v++) ev[v] += (T)Ed[v];
        // total strain tensor xx, yy, zz, yz, xz, xy
        T et[6];
        if constexpr (D == 2) {
            et[0] = ev[0]; et[1] = ev[1]; et[2] = T(0); et[3] = T(0); et[4] = T(0); et[5] = T(0.5) * ev[2];
        } else {
            et[0] = ev[0]; et[1] = ev[1]; et[2] = ev[2];
            et[3] = T(0.5) * ev[3]; et[4] = T(0.5) * ev[4]; et[5] = T(0.5) * ev[5];
        }
        T Wf, Ww, Wg;
        phase_weights(F.theta[c], F.phig[c], Wf, Ww, Wg);
        const T K = (Wf + Ww) * T(P.Ks) + Wg * T(P.Kg);
        const T G = (Wf + Ww) * T(P.Gs) + Wg * T(P.Gg);
        const T e0 = T(P.eig0) * Wf;
        T ep[6];
        if constexpr (D == 2) {
            ep[0] = F.ep[0][c]; ep[1] = F.ep[1][c]; ep[2] = F.ep[2][c]; ep[3] = T(0); ep[4] = T(0); ep[5] = F.ep[3][c];
        } else {
#pragma unroll
            for (int v = 0; v < 6; v++) ep[v] = F.ep[v][c];
        }
        T ee[6];
#pragma unroll
        for (int v = 0; v < 6; v++) ee[v] = et[v] - ep[v] - (v < 3 ? e0 : T(0));
        T tr = ee[0] + ee[1] + ee[2];
        T dev[6];
#pragma unroll
        for (int v = 0; v < 6; v++) dev[v] = ee[v] - (v < 3 ? tr / T(3) : T(0));
        T n2 = dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2] + T(2) * (dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
        if (P.plasticity) {
            T a = F.alpha[c];
            const T nrm = sqrt(n2);
            const T f = T(2) * G * nrm - T(0.816496580927726) * (T(P.sY) + T(P.Hh) * a);
            if (f > T(0)) {
                const T dl = f / (T(2) * G + T(0.816496580927726) * T(P.Hh));
                const T sc_ = dl / nrm;
#pragma unroll
                for (int v = 0; v < 6; v++) { T dep = sc_ * dev[v]; ep[v] += dep; dev[v] -= dep; ee[v] -= dep; }
                a += dl;
                F.alpha[c] = a;
                if constexpr (D == 2) {
                    F.ep[0][c] = ep[0]; F.ep[1][c] = ep[1]; F.ep[2][c] = ep[2]; F.ep[3][c] = ep[5];
                } else {
#pragma unroll
                    for (int v = 0; v < 6; v++) F.ep[v][c] = ep[v];
                }
                tr = ee[0] + ee[1] + ee[2];
                n2 = dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2] + T(2) * (dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
            }
        }
        F.trE[c] = tr;
        F.devE2[c] = n2;
        if (want_sigma) {
            T sg[6];
#pragma unroll
            for (int v = 0; v < 6; v++) sg[v] = T(2) * G * dev[v] + (v < 3 ? K * tr : T(0));
            if constexpr (D == 2) {
                F.sigma_out[0][c] = sg[0]; F.sigma_out[1][c] = sg[1]; F.sigma_out[2][c] = sg[2]; F.sigma_out[3][c] = sg[5];
            } else {
#pragma unroll
                for (int v = 0; v < 6; v++) F.sigma_out[v][c] = sg[v];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K1a: oxygen chemical potential mu_O = sum_a W_a c f_a'(x_O) - kappa Lap x_O
// and mobility M_O = D_O(phi_g) / (c sum_a W_a f_a''(x_O))   (Sec. 2.2, 3.2)
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void k_mu(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    PF_CELL_JOB_PROLOGUE
    for (long long c = bid * blockDim.x + threadIdx.x; c < P.N; c += nbk * blockDim.x) {
        int i, j, k;
        cell_coords<D>(P, c, i, j, k);
        const T x = F.xO[c];
        T lap = F.xO[lin<D>(P, i - 1, j, k)] + F.xO[lin<D>(P, i + 1, j, k)]
              + F.xO[lin<D>(P, i, j - 1, k)] + F.xO[lin<D>(P, i, j + 1, k)] - T(2 * D) * x;
        if constexpr (D == 3) lap += F.xO[lin<D>(P, i, j, k - 1)] + F.xO[lin<D>(P, i, j, k + 1)];
        T Wf, Ww, Wg;
        phase_weights(F.theta[c], F.phig[c], Wf, Ww, Wg);
        const T cc = T(P.c);
        const T m1 = Wf * f_fe1(x) + Ww * f_wu1(x) + Wg * f_ga1(x);
        const T m2 = Wf * f_fe2(x) + Ww * f_wu2(x) + Wg * f_ga2(x);
        F.muO[c] = cc * m1 - T(P.kappa) * lap;
        const T DO = (T(1) - Wg) * T(P.DOs) + Wg * T(P.DOg);
        const T den = cc * m2;
        F.MO[c] = den != T(0) ? DO / den : T(0);
    }
}

// ---------------------------------------------------------------------------
// K1b: explicit Euler update (Sec. 2.4 field relations, R2 order parameter)
//   theta' = -(L g / 2) [force(theta) - 2 eps Lap theta]
//   x_O'   = div(M_O grad mu_O) - r
//   x_H'   = div(D_H grad x_H) - 2 r
//   x_W'   = div(D_W grad x_W) + r,     r = m(phi_g) k x_O x_H (0 if x_W >= 1)
// face values are arithmetic means; then the supply reset.  Per-block sums
// of the new fields and of the supply exchange are reduced by the last block.
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(256) k_update(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    PF_CELL_JOB_PROLOGUE
    double *partials = J_->partials;
    unsigned int *counter = J_->counter;
    Diag *dg = J_->dg;
    Acc<T> acc[6];           // sum x_O, x_H, x_H2O, removed water, supplied H, non-finite count
    Acc<T> &sO = acc[0], &sH = acc[1], &sW = acc[2], &rem = acc[3], &sup = acc[4];
    int bad = 0;
    const T cc = T(P.c), eps2 = T(2 * P.eps), dt = T(P.dt);
    for (long long c = bid * blockDim.x + threadIdx.x; c < P.N; c += nbk * blockDim.x) {
        int i, j, k;
        cell_coords<D>(P, c, i, j, k);
        long long nbr[2 * D];
        nbr[0] = lin<D>(P, i - 1, j, k); nbr[1] = lin<D>(P, i + 1, j, k);
        nbr[2] = lin<D>(P, i, j - 1, k); nbr[3] = lin<D>(P, i, j + 1, k);
        if constexpr (D == 3) { nbr[4] = lin<D>(P, i, j, k - 1); nbr[5] = lin<D>(P, i, j, k + 1); }
        const T th = F.theta[c], pg = F.phig[c];
        const T xo = F.xO[c], xh = F.xH[c], xw = F.xW[c];
        const T mu0 = F.muO[c], M0 = F.MO[c];
        const T hg0 = hfun(pg);
        const T DH0 = (T(1) - hg0) * T(P.DHs) + hg0 * T(P.DHg);
        const T DW0 = (T(1) - hg0) * T(P.DWs) + hg0 * T(P.DWg);
        T lapt = T(0), dO = T(0), dH = T(0), dW = T(0);
#pragma unroll
        for (int q = 0; q < 2 * D; q++) {
            const long long m = nbr[q];
            lapt += F.theta[m] - th;
            dO += T(0.5) * (M0 + F.MO[m]) * (F.muO[m] - mu0);
            const T hg = hfun(F.phig[m]);
            const T DHm = (T(1) - hg) * T(P.DHs) + hg * T(P.DHg);
            const T DWm = (T(1) - hg) * T(P.DWs) + hg * T(P.DWg);
            dH += T(0.5) * (DH0 + DHm) * (F.xH[m] - xh);
            dW += T(0.5) * (DW0 + DWm) * (F.xW[m] - xw);
        }
        // local force of the theta equation
        const T t = F.trE[c], s2 = F.devE2[c];
        const T ht = hfun(th), hpt = hder(th);
        const T sol = T(1) - hg0;
        const T Af = cc * f_fe(xo) + T(0.5) * T(P.Ks) * t * t + T(P.Gs) * s2;
        const T Aw = cc * f_wu(xo) + T(0.5) * T(P.Ks) * t * t + T(P.Gs) * s2;
        const T Kmix = sol * T(P.Ks) + hg0 * T(P.Kg);
        const T force = sol * hpt * (Af - Aw) + T(2 * P.w) * mder(th) - T(P.eig0) * sol * hpt * T(3) * Kmix * t;
        (void)ht;
        const T rate = T(-0.5 * P.L) * F.mob[c] * (force - eps2 * lapt);
        T r = mfun(pg) * T(P.kfor) * xo * xh;
        if (xw >= T(1)) r = T(0);
        const T nth = th + dt * rate;
        const T nxo = xo + dt * (dO - r);
        T nxh = xh + dt * (dH - T(2) * r);
        T nxw = xw + dt * (dW + r);
        if (F.mask[c]) {
            rem.add(nxw);
            sup.add(T(P.xHbc) - nxh);
            nxh = T(P.xHbc);
            nxw = T(0);
        }
        F.theta_o[c] = nth;
        F.xO_o[c] = nxo;
        F.xH_o[c] = nxh;
        F.xW_o[c] = nxw;
        sO.add(nxo); sH.add(nxh); sW.add(nxw);
        if (!(isfinite(nth) && isfinite(nxo) && isfinite(nxh) && isfinite(nxw))) bad = 1;
    }
    acc[5].add(T(bad));
    // per-block sums (FP32 pairs in the mixed method: no FP64 per thread)
    block_reduce_store<6>(acc, partials + (size_t)bid * PSTRIDE);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int tk = atomicAdd(counter, 1u);
        last = (tk == (unsigned int)nbk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        __shared__ double tot[6];
        last_block_sums<6>(partials, (int)nbk, tot);
        if (threadIdx.x == 0) {
            dg->sumO_prev = dg->sumO;
            dg->sumO = tot[0]; dg->sumH = tot[1]; dg->sumW = tot[2];
            dg->removedW += tot[3];
            dg->suppliedH += tot[4];
            if (tot[5] > 0.0 && dg->status == 0) dg->status = 5;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// K1: the fused explicit step -- oxygen chemical potential and mobility
// (K1a) and the explicit Euler update (K1b) in one pass over the grid.
//
// Each block walks tiles of TX x TY (x TZ) cells.  Per tile it stages in
// shared memory x_O with a halo of two cells and theta, phi_g, x_H, x_H2O
// with a halo of one, evaluates mu_O and M_O on the tile plus one halo
// cell, then updates the tile's cells from shared memory.  HBM sees each
// field once per step (the halo re-reads hit L2); mu_O and M_O never leave
// the SM.  Arithmetic and operand order per cell are those of k_mu and
// k_update.
// ---------------------------------------------------------------------------
template <int D, int TX, int TY, int TZ>
struct FusedTile {
    static constexpr int EX = TX + 2, EY = TY + 2, EZ = D == 3 ? TZ + 2 : 1;   // halo 1
    static constexpr int GX = TX + 4, GY = TY + 4, GZ = D == 3 ? TZ + 4 : 1;   // halo 2
    static constexpr int E = EX * EY * EZ, G = GX * GY * GZ, C = TX * TY * (D == 3 ? TZ : 1);
    // shared words: x_O (G); theta, phi_g, x_H, x_H2O, mu_O, M_O, D_H, D_H2O (E each)
    static constexpr int WORDS = G + 8 * E;
    static constexpr int NT = 256;                       // threads per block
    static constexpr int CPT = (C + NT - 1) / NT;        // tile cells per thread
};

// Quotient for the mobility M_O = D_O / psi'': the FP32 method takes the
// hardware approximate divide (2 ulp; its fields are held to 1e-4), FP64 the
// IEEE divide.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// periodic coordinate; any a (grids smaller than a tile wrap several times)
__device__ __forceinline__ int pwrap(int a, int n)
{
    if (a < 0) a += n;
    if (a >= n) a -= n;
    if ((unsigned)a >= (unsigned)n) a = wrapm(a, n);
    return a;
}

template <typename T, int D, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && D == 2) ? 3 : 2) k_fused(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    using FT = FusedTile<D, TX, TY, TZ>;
    static_assert(TX == 32, "the staging maps one warp lane to one tile column");
    constexpr int EX = FT::EX, EY = FT::EY, GX = FT::GX, GY = FT::GY, NT = FT::NT, CPT = FT::CPT;
    constexpr int TZe = D == 3 ? TZ : 1;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    T *sXO = (T *)fsm_raw;
    T *sTh = sXO + FT::G, *sPg = sTh + FT::E, *sXH = sPg + FT::E, *sXW = sXH + FT::E;
    T *sMu = sXW + FT::E, *sM = sMu + FT::E, *sDH = sM + FT::E, *sDW = sDH + FT::E;

    // the job lives in shared memory: its parameters are read where they
    // are used instead of occupying registers for the whole kernel
    __shared__ __align__(16) CellJob<T, D> sJ;
    {
        const CellJob<T, D> *J_ = my_job(js);
        const int *src = (const int *)J_;
        int *dst = (int *)&sJ;
        for (int w = threadIdx.x; w < (int)(sizeof(CellJob<T, D>) / sizeof(int)); w += NT) dst[w] = src[w];
    }
    __syncthreads();
    const Params &P = sJ.P;
    const FieldPtrs<T, D> &F = sJ.F;
    const long long bid = (long long)blockIdx.x - sJ.block0;
    const long long nbk = sJ.nblocks;
    const int nx = P.nx, ny = P.ny, nz = D == 3 ? P.nz : 1;
    const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY, tiles_z = (nz + TZe - 1) / TZe;
    const long long ntiles = (long long)tiles_x * tiles_y * tiles_z;
    const unsigned sxy = (unsigned)nx * (unsigned)ny;   // grids hold < 2^31 cells

    Acc<T> acc[5];           // sum x_O, x_H, x_H2O, removed water, supplied H
    bool bad = false;

    for (long long t = bid; t < ntiles; t += nbk) {
        const int tx = (int)(t % tiles_x);
        const long long tr = t / tiles_x;
        const int ty = (int)(tr % tiles_y), tz = (int)(tr / tiles_y);
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZe;

        // per-cell inputs of this thread's cells, requested first so that
        // they arrive while the tile is staged
        int gc[CPT];
        T pre_tE[CPT], pre_s2[CPT], pre_mob[CPT];
        unsigned char pre_mask[CPT];
#pragma unroll
        for (int u = 0; u < CPT; u++) {
            const int l = threadIdx.x + u * NT;
            const int a = l % TX, r = l / TX, b = r % TY, c = r / TY;
            const int i = x0 + a, j = y0 + b, k = z0 + c;
            const bool in = l < FT::C && i < nx && j < ny && (D == 2 || k < nz);
            gc[u] = in ? (int)((unsigned)i + (unsigned)nx * (unsigned)j + sxy * (unsigned)k) : -1;
            if (in) {
                pre_tE[u] = F.trE[gc[u]];
                pre_s2[u] = F.devE2[gc[u]];
                pre_mob[u] = F.mob[gc[u]];
                pre_mask[u] = F.mask[gc[u]];
            }
        }
        // Stage x_O (halo 2) and theta, phi_g, x_H, x_H2O (halo 1).  Warps take
        // whole rows: lane L loads column L, lanes 0..(extra-1) the columns
        // past 32; the periodic wrap is computed once per row and column, and
        // every load of a thread is issued before its shared-memory stores.
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            constexpr int NW = NT / 32;
            constexpr int RG = FT::GY * FT::GZ, RE = EY * FT::EZ;
            constexpr int NRG = (RG + NW - 1) / NW, NRE = (RE + NW - 1) / NW;
            const int ci2 = pwrap(x0 + lane - 2, nx), ci2x = pwrap(x0 + 32 + lane - 2, nx);
            const int ci1 = pwrap(x0 + lane - 1, nx), ci1x = pwrap(x0 + 32 + lane - 1, nx);
            const bool xg = lane < GX - 32, xe = lane < EX - 32;
            T v[NRG], vx[NRG];
#pragma unroll
            for (int u = 0; u < NRG; u++) {
                const int row = warp + u * NW;
                if (row < RG) {
                    const int b = row % GY, c = row / GY;
                    const int gj = pwrap(y0 + b - 2, ny), gk = D == 3 ? pwrap(z0 + c - 2, nz) : 0;
                    const T *src = F.xO + ((unsigned)nx * (unsigned)gj + sxy * (unsigned)gk);
                    v[u] = src[ci2];
                    if (xg) vx[u] = src[ci2x];
                }
            }
            T e0[NRE], e1[NRE], e2[NRE], e3[NRE], x0v[NRE], x1v[NRE], x2v[NRE], x3v[NRE];
#pragma unroll
            for (int u = 0; u < NRE; u++) {
                const int row = warp + u * NW;
                if (row < RE) {
                    const int b = row % EY, c = row / EY;
                    const int gj = pwrap(y0 + b - 1, ny), gk = D == 3 ? pwrap(z0 + c - 1, nz) : 0;
                    const unsigned rb = (unsigned)nx * (unsigned)gj + sxy * (unsigned)gk;
                    e0[u] = F.theta[rb + ci1]; e1[u] = F.phig[rb + ci1]; e2[u] = F.xH[rb + ci1]; e3[u] = F.xW[rb + ci1];
                    if (xe) {
                        x0v[u] = F.theta[rb + ci1x]; x1v[u] = F.phig[rb + ci1x];
                        x2v[u] = F.xH[rb + ci1x]; x3v[u] = F.xW[rb + ci1x];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < NRG; u++) {
                const int row = warp + u * NW;
                if (row < RG) {
                    sXO[row * GX + lane] = v[u];
                    if (xg) sXO[row * GX + 32 + lane] = vx[u];
                }
            }
#pragma unroll
            for (int u = 0; u < NRE; u++) {
                const int row = warp + u * NW;
                if (row < RE) {
                    const int q = row * EX + lane;
                    sTh[q] = e0[u]; sPg[q] = e1[u]; sXH[q] = e2[u]; sXW[q] = e3[u];
                    if (xe) { sTh[q + 32] = x0v[u]; sPg[q + 32] = x1v[u]; sXH[q + 32] = x2v[u]; sXW[q + 32] = x3v[u]; }
                }
            }
        }
        __syncthreads();
        // mu_O, M_O (Sec. 2.2, 3.2) and the species diffusivities (R4) on the
        // tile plus one halo cell
        {
            const CellConst<T> &K = sJ.K;
            const T cc = K.c, kap = K.kappa;
            const T DOs = K.DOs, DOg = K.DOg, DHs = K.DHs, DHg = K.DHg, DWs = K.DWs, DWg = K.DWg;
            constexpr int NI = (FT::E + NT - 1) / NT;
#pragma unroll
            for (int u = 0; u < NI; u++) {
                const int l = threadIdx.x + u * NT;
                if (l < FT::E) {
                    const int a = l % EX, r = l / EX, b = r % EY, c = r / EY;
                    const int q = (a + 1) + GX * ((b + 1) + GY * (D == 3 ? c + 1 : 0));
                    const T x = sXO[q];
                    T lap = sXO[q - 1] + sXO[q + 1] + sXO[q - GX] + sXO[q + GX] - T(2 * D) * x;
                    if constexpr (D == 3) lap += sXO[q - GX * GY] + sXO[q + GX * GY];
                    T Wf, Ww, Wg;
                    phase_weights(sTh[l], sPg[l], Wf, Ww, Wg);
                    const T m1 = Wf * f_fe1(x) + Ww * f_wu1(x) + Wg * f_ga1(x);
                    const T m2 = Wf * f_fe2(x) + Ww * f_wu2(x) + Wg * f_ga2(x);
                    sMu[l] = cc * m1 - kap * lap;
                    const T DO = (T(1) - Wg) * DOs + Wg * DOg;
                    const T den = cc * m2;
                    sM[l] = den != T(0) ? fast_div(DO, den) : T(0);
                    sDH[l] = (T(1) - Wg) * DHs + Wg * DHg;
                    sDW[l] = (T(1) - Wg) * DWs + Wg * DWg;
                }
            }
        }
        __syncthreads();
        // explicit Euler update of the tile's cells (Sec. 2.4, R2)
        {
            const CellConst<T> &K = sJ.K;
            const T cc = K.c, eps2 = K.eps2, dt = K.dt;
            const T Ks = K.Ks, Gs = K.Gs, Kg = K.Kg, w2 = K.w2, eig3 = K.eig3;
            const T Lh = K.Lh, kf = K.kf, xHbc = K.xHbc;
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                if (gc[u] < 0) continue;
                const int l = threadIdx.x + u * NT;
                const int a = l % TX, r = l / TX, b = r % TY, c = r / TY;
                const int e = (a + 1) + EX * ((b + 1) + EY * (D == 3 ? c + 1 : 0));
                int nb[2 * D];
                nb[0] = e - 1; nb[1] = e + 1; nb[2] = e - EX; nb[3] = e + EX;
                if constexpr (D == 3) { nb[4] = e - EX * EY; nb[5] = e + EX * EY; }
                const T th = sTh[e], pg = sPg[e];
                const T xo = sXO[(a + 2) + GX * ((b + 2) + GY * (D == 3 ? c + 2 : 0))];
                const T xh = sXH[e], xw = sXW[e];
                const T mu0 = sMu[e], M0 = sM[e], DH0 = sDH[e], DW0 = sDW[e];
                T lapt = T(0), dO = T(0), dH = T(0), dW = T(0);
#pragma unroll
                for (int q = 0; q < 2 * D; q++) {
                    const int m = nb[q];
                    lapt += sTh[m] - th;
                    dO += T(0.5) * (M0 + sM[m]) * (sMu[m] - mu0);
                    dH += T(0.5) * (DH0 + sDH[m]) * (sXH[m] - xh);
                    dW += T(0.5) * (DW0 + sDW[m]) * (sXW[m] - xw);
                }
                const T tE = pre_tE[u], s2 = pre_s2[u];
                const T hg0 = hfun(pg);
                const T hpt = hder(th);
                const T sol = T(1) - hg0;
                const T Af = cc * f_fe(xo) + T(0.5) * Ks * tE * tE + Gs * s2;
                const T Aw = cc * f_wu(xo) + T(0.5) * Ks * tE * tE + Gs * s2;
                const T Kmix = sol * Ks + hg0 * Kg;
                const T force = sol * hpt * (Af - Aw) + w2 * mder(th) - eig3 * sol * hpt * Kmix * tE;
                const T rate = Lh * pre_mob[u] * (force - eps2 * lapt);
                T rr = mfun(pg) * kf * xo * xh;
                if (xw >= T(1)) rr = T(0);
                const T nth = th + dt * rate;
                const T nxo = xo + dt * (dO - rr);
                T nxh = xh + dt * (dH - T(2) * rr);
                T nxw = xw + dt * (dW + rr);
                if (pre_mask[u]) {
                    acc[3].add(nxw);
                    acc[4].add(xHbc - nxh);
                    nxh = xHbc;
                    nxw = T(0);
                }
                const unsigned g = (unsigned)gc[u];
                F.theta_o[g] = nth;
                F.xO_o[g] = nxo;
                F.xH_o[g] = nxh;
                F.xW_o[g] = nxw;
                acc[0].add(nxo); acc[1].add(nxh); acc[2].add(nxw);
                // a non-finite value anywhere makes the sum non-finite
                bad |= !isfinite(nth + nxo + nxh + nxw);
            }
        }
        __syncthreads();
    }
    Acc<T> acc6[6];
#pragma unroll
    for (int q = 0; q < 5; q++) acc6[q] = acc[q];
    acc6[5].add(T(bad ? 1 : 0));
    double *partials = sJ.partials;
    unsigned int *counter = sJ.counter;
    block_reduce_store<6>(acc6, partials + (size_t)bid * PSTRIDE);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int tk = atomicAdd(counter, 1u);
        last = (tk == (unsigned int)nbk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        __shared__ double tot[6];
        last_block_sums<6>(partials, (int)nbk, tot);
        if (threadIdx.x == 0) {
            Diag *dg = sJ.dg;
            dg->sumO_prev = dg->sumO;
            dg->sumO = tot[0]; dg->sumH = tot[1]; dg->sumW = tot[2];
            dg->removedW += tot[3];
            dg->suppliedH += tot[4];
            if (tot[5] > 0.0 && dg->status == 0) dg->status = 5;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// K1 in 2D by column strips (k_fused_cm): the same arithmetic as k_fused,
// without shared memory.  Each warp walks one strip of 32 lanes over a
// block's range of rows; lane L holds column x0 - 1 + L (x0 = 30 * strip column),
// so lanes 1..30 are the strip's output columns and lanes 0 and 31 its halo.
// Every lane evaluates mu_O, M_O and the diffusivities of its own column in
// a three-row register window (x_O at the lane's left/right from shuffles,
// from an extra load at lanes 0 and 31); the update of row j takes its
// vertical neighbours from the window and its horizontal ones by shuffle.
// Raw fields are loaded two rows ahead of their use.
// ---------------------------------------------------------------------------
template <typename T>
struct CmRaw {
    T th, pg, xo, xh, xw;
};

template <typename T>
__device__ __forceinline__ void cm_load(const FieldPtrs<T, 2> &F, unsigned g, CmRaw<T> &R)
{
    R.th = F.theta[g];
    R.pg = F.phig[g];
    R.xo = F.xO[g];
    R.xh = F.xH[g];
    R.xw = F.xW[g];
}

template <typename T>
struct CmDer {
    T mu, M, DH, DW;
};

// mu_O, M_O, D_H, D_H2O of a cell from its theta, phi_g, x_O and the
// Laplacian of x_O (Sec. 2.2, 3.2; R4)
template <typename T>
__device__ __forceinline__ void cm_derive(const CellConst<T> &K, T th, T pg, T x, T lap, CmDer<T> &Dv)
{
    T Wf, Ww, Wg;
    phase_weights(th, pg, Wf, Ww, Wg);
    const T m1 = Wf * f_fe1(x) + Ww * f_wu1(x) + Wg * f_ga1(x);
    const T m2 = Wf * f_fe2(x) + Ww * f_wu2(x) + Wg * f_ga2(x);
    Dv.mu = K.c * m1 - K.kappa * lap;
    const T DO = (T(1) - Wg) * K.DOs + Wg * K.DOg;
    const T den = K.c * m2;
    Dv.M = den != T(0) ? fast_div(DO, den) : T(0);
    Dv.DH = (T(1) - Wg) * K.DHs + Wg * K.DHg;
    Dv.DW = (T(1) - Wg) * K.DWs + Wg * K.DWg;
}

template <typename T>
__device__ __forceinline__ T up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T dn1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_fused_cm(const __grid_constant__ JobSet<CellJob<T, 2>> js)
{
    __shared__ __align__(16) CellJob<T, 2> sJ;
    {
        const CellJob<T, 2> *J_ = my_job(js);
        const int *src = (const int *)J_;
        int *dst = (int *)&sJ;
        for (int w = threadIdx.x; w < (int)(sizeof(CellJob<T, 2>) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const FieldPtrs<T, 2> &F = sJ.F;       // pointers and constants are read from the
    const CellConst<T> &K = sJ.K;          // job's shared-memory copy where used
    const int nx = sJ.P.nx, ny = sJ.P.ny;
    const int bid = (int)blockIdx.x - sJ.block0, nbk = sJ.nblocks;
    const int lane = threadIdx.x & 31;
    const int WB = blockDim.x >> 5, wib = threadIdx.x >> 5;
    // strips are grouped WB at a time (one per warp of a block: adjacent
    // strips share the 128-byte lines of their boundary columns, and the
    // warps of one block read them together); the (group, row) space is
    // cut into equal contiguous chunks, one per block, and a chunk that
    // crosses a group is two segments
    const int nsx = (nx + 29) / 30;
    const int ngx = (nsx + WB - 1) / WB;
    const long long total = (long long)ngx * ny;
    const long long per = (total + nbk - 1) / nbk;
    long long u = (long long)bid * per;
    const long long uend = u + per < total ? u + per : total;
    Acc<T> acc[5];
    bool bad = false;
    while (u < uend) {
        const int gxi = (int)(u / ny), j0 = (int)(u % ny);
        const int j1 = (int)((ny - j0) < (uend - u) ? ny : j0 + (uend - u));
        u += j1 - j0;
        const int sxi = gxi * WB + wib;
        if (sxi >= nsx) continue;                                // warp-uniform
        const int x0 = sxi * 30;
        const int craw = x0 - 1 + lane;
        const int c = craw < 0 ? craw + nx : (craw >= nx ? craw - nx : craw);
        const int cw = c % nx;                                   // grids narrower than a strip wrap again
        const bool out = lane >= 1 && lane <= 30 && craw < nx;   // this lane writes its column
        int cext = lane == 0 ? cw - 1 : cw + 1;                  // x_O beyond the halo lanes
        cext = cext < 0 ? cext + nx : (cext >= nx ? cext - nx : cext);
        auto row = [&](int j) {
            int r = j < 0 ? j + ny : (j >= ny ? j - ny : j);
            if ((unsigned)r >= (unsigned)ny) r = ((j % ny) + ny) % ny;   // grids of a few rows
            return r;
        };
        auto at = [&](int col, int j) { return (unsigned)col + (unsigned)nx * (unsigned)row(j); };
        // window: raw rows j-1 .. j+2, derived rows j-1, j
        CmRaw<T> rm, r0, r1, r2;
        T xe0, xe1, xe2;          // x_O beyond the halo lane, rows j, j+1, j+2 (lanes 0 and 31)
        CmDer<T> dm, d0;
        {
            const T xo_m2 = F.xO[at(cw, j0 - 2)];
            T xe_m1 = T(0);
            cm_load(F, at(cw, j0 - 1), rm);
            cm_load(F, at(cw, j0), r0);
            cm_load(F, at(cw, j0 + 1), r1);
            cm_load(F, at(cw, j0 + 2), r2);
            if (lane == 0 || lane == 31) {
                xe_m1 = F.xO[at(cext, j0 - 1)];
                xe0 = F.xO[at(cext, j0)];
                xe1 = F.xO[at(cext, j0 + 1)];
                xe2 = F.xO[at(cext, j0 + 2)];
            } else {
                xe0 = xe1 = xe2 = T(0);
            }
            // derived of rows j0-1 and j0: Laplacians of x_O
            T l, r;
            l = up1(rm.xo); r = dn1(rm.xo);
            if (lane == 0) l = xe_m1;
            if (lane == 31) r = xe_m1;
            cm_derive(K, rm.th, rm.pg, rm.xo, l + r + xo_m2 + r0.xo - T(4) * rm.xo, dm);
            l = up1(r0.xo); r = dn1(r0.xo);
            if (lane == 0) l = xe0;
            if (lane == 31) r = xe0;
            cm_derive(K, r0.th, r0.pg, r0.xo, l + r + rm.xo + r1.xo - T(4) * r0.xo, d0);
        }
        for (int j = j0; j < j1; j++) {
            // raw values two rows ahead, and this row's per-cell inputs
            CmRaw<T> r3;
            T xe3 = T(0);
            cm_load(F, at(cw, j + 3), r3);
            if (lane == 0 || lane == 31) xe3 = F.xO[at(cext, j + 3)];
            const unsigned g = at(cw, j);
            T tE = T(0), s2 = T(0), mob = T(0);
            unsigned char msk = 0;
            if (out) { tE = F.trE[g]; s2 = F.devE2[g]; mob = F.mob[g]; msk = F.mask[g]; }
            // derived of row j+1
            CmDer<T> d1;
            {
                T l = up1(r1.xo), r = dn1(r1.xo);
                if (lane == 0) l = xe1;
                if (lane == 31) r = xe1;
                cm_derive(K, r1.th, r1.pg, r1.xo, l + r + r0.xo + r2.xo - T(4) * r1.xo, d1);
            }
            // horizontal neighbours of row j
            const T thl = up1(r0.th), thr = dn1(r0.th);
            const T mul = up1(d0.mu), mur = dn1(d0.mu), Ml = up1(d0.M), Mr = dn1(d0.M);
            const T DHl = up1(d0.DH), DHr = dn1(d0.DH), DWl = up1(d0.DW), DWr = dn1(d0.DW);
            const T xhl = up1(r0.xh), xhr = dn1(r0.xh), xwl = up1(r0.xw), xwr = dn1(r0.xw);
            if (out) {
                const T th = r0.th, pg = r0.pg, xo = r0.xo, xh = r0.xh, xw = r0.xw;
                const T mu0 = d0.mu, M0 = d0.M, DH0 = d0.DH, DW0 = d0.DW;
                const T half = T(0.5);
                const T lapt = (thl - th) + (thr - th) + (rm.th - th) + (r1.th - th);
                const T dO = half * (M0 + Ml) * (mul - mu0) + half * (M0 + Mr) * (mur - mu0)
                           + half * (M0 + dm.M) * (dm.mu - mu0) + half * (M0 + d1.M) * (d1.mu - mu0);
                const T dH = half * (DH0 + DHl) * (xhl - xh) + half * (DH0 + DHr) * (xhr - xh)
                           + half * (DH0 + dm.DH) * (rm.xh - xh) + half * (DH0 + d1.DH) * (r1.xh - xh);
                const T dW = half * (DW0 + DWl) * (xwl - xw) + half * (DW0 + DWr) * (xwr - xw)
                           + half * (DW0 + dm.DW) * (rm.xw - xw) + half * (DW0 + d1.DW) * (r1.xw - xw);
                const T hg0 = hfun(pg);
                const T hpt = hder(th);
                const T sol = T(1) - hg0;
                const T Af = K.c * f_fe(xo) + half * K.Ks * tE * tE + K.Gs * s2;
                const T Aw = K.c * f_wu(xo) + half * K.Ks * tE * tE + K.Gs * s2;
                const T Kmix = sol * K.Ks + hg0 * K.Kg;
                const T force = sol * hpt * (Af - Aw) + K.w2 * mder(th) - K.eig3 * sol * hpt * Kmix * tE;
                const T rate = K.Lh * mob * (force - K.eps2 * lapt);
                T rr = mfun(pg) * K.kf * xo * xh;
                if (xw >= T(1)) rr = T(0);
                const T nth = th + K.dt * rate;
                const T nxo = xo + K.dt * (dO - rr);
                T nxh = xh + K.dt * (dH - T(2) * rr);
                T nxw = xw + K.dt * (dW + rr);
                if (msk) {
                    acc[3].add(nxw);
                    acc[4].add(K.xHbc - nxh);
                    nxh = K.xHbc;
                    nxw = T(0);
                }
                F.theta_o[g] = nth;
                F.xO_o[g] = nxo;
                F.xH_o[g] = nxh;
                F.xW_o[g] = nxw;
                acc[0].add(nxo); acc[1].add(nxh); acc[2].add(nxw);
                bad |= !isfinite(nth + nxo + nxh + nxw);
            }
            // shift the window one row up
            rm = r0; r0 = r1; r1 = r2; r2 = r3;
            xe0 = xe1; xe1 = xe2; xe2 = xe3;
            dm = d0; d0 = d1;
        }
    }
    Acc<T> acc6[6];
#pragma unroll
    for (int q = 0; q < 5; q++) acc6[q] = acc[q];
    acc6[5].add(T(bad ? 1 : 0));
    double *partials = sJ.partials;
    unsigned int *counter = sJ.counter;
    block_reduce_store<6>(acc6, partials + (size_t)bid * PSTRIDE);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int tk = atomicAdd(counter, 1u);
        last = (tk == (unsigned int)nbk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        __shared__ double tot[6];
        last_block_sums<6>(partials, nbk, tot);
        if (threadIdx.x == 0) {
            Diag *dg = sJ.dg;
            dg->sumO_prev = dg->sumO;
            dg->sumO = tot[0]; dg->sumH = tot[1]; dg->sumW = tot[2];
            dg->removedW += tot[3];
            dg->suppliedH += tot[4];
            if (tot[5] > 0.0 && dg->status == 0) dg->status = 5;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// K1 marching along the slowest axis (k_fusedz): the same arithmetic as
// k_fused, with the grid cut into planes (3D: 32 x 8 cells of an x-y plane,
// marching along z; 2D: 256-cell row segments, marching along y).  A block
// walks a chunk of planes of one tile column: x_O with a halo of two cells
// in the plane and theta, phi_g, x_H, x_H2O with a halo of one are copied
// into ring buffers of planes by asynchronous copies (cp.async) issued one
// plane ahead, so that their latency overlaps the work on the current
// plane; mu_O, M_O, D_H, D_H2O are evaluated one plane ahead of the update
// (the cross-plane neighbours come from the rings), and the plane's own
// cells are updated.  Every field is read from HBM once per step plus the
// in-plane halo (L2 hits) and the chunk's first planes.
// ---------------------------------------------------------------------------
template <int D>
struct FusedZ {
    static constexpr int TX = D == 3 ? 32 : 256, TY = D == 3 ? 8 : 1;
    // shared-memory rows are RS values wide with the tile's first column at
    // CO (16-byte aligned), so that the row interior is copied in 16-byte
    // pieces; x_O keeps two halo columns each side, the other fields one
    static constexpr int RS = TX + 8, CO = 4;
    static constexpr int EY = D == 3 ? TY + 2 : 1, GY = D == 3 ? TY + 4 : 1;   // rows: halo 1 / halo 2
    static constexpr int E = EY * RS, G = GY * RS;                             // values per plane
    static constexpr int EX = TX + 2;                                          // halo-1 cells per row
    static constexpr int NE = EX * EY;                                         // halo-1 cells per plane
    // ring depths (planes): x_O and the raw fields hold the planes being
    // read (update m - 1 .. m + 1 and the derived plane m + 1) plus the one
    // in flight; mu, M, D_H, D_H2O three planes
    static constexpr int RO = 5, RE = 5, RM = 3;
    static constexpr int WORDS = RO * G + 4 * RE * E + 4 * RM * E;
    static constexpr int NT = 256;
    static_assert(TX * TY == NT, "one own cell per thread");
    // copy tasks per plane on the aligned path: x_O rows of TX / 4 16-byte
    // pieces plus four halo values, raw-field rows of TX / 4 pieces plus two
    static constexpr int VW = TX / 4;
    static constexpr int TO = GY * (VW + 4), TE = EY * (VW + 2);
    static_assert(TO + TE <= NT, "one copy task per thread and plane");
    static constexpr int DPT = (NE + NT - 1) / NT;                             // derived cells per thread
};

template <typename T, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_fusedz(const __grid_constant__ JobSet<CellJob<T, D>> js)
{
    using Z = FusedZ<D>;
    constexpr int TX = Z::TX, TY = Z::TY, RS = Z::RS, CO = Z::CO, E = Z::E, G = Z::G, NT = Z::NT;
    constexpr int EX = Z::EX, NE = Z::NE, VW = Z::VW, DPT = Z::DPT;
    constexpr int XR = D == 3 ? 1 : 0;          // x_O row of raw-field row r is r + XR
    extern __shared__ __align__(16) unsigned char fsz_raw[];
    T *const sXO = (T *)fsz_raw;                                   // [RO][G]
    T *const sTh = sXO + Z::RO * G, *const sPg = sTh + Z::RE * E;  // [RE][E] each
    T *const sXH = sPg + Z::RE * E, *const sXW = sXH + Z::RE * E;
    T *const sMu = sXW + Z::RE * E, *const sM = sMu + Z::RM * E;   // [RM][E] each
    T *const sDH = sM + Z::RM * E, *const sDW = sDH + Z::RM * E;

    __shared__ __align__(16) CellJob<T, D> sJ;
    {
        const CellJob<T, D> *J_ = my_job(js);
        const int *src = (const int *)J_;
        int *dst = (int *)&sJ;
        for (int w = threadIdx.x; w < (int)(sizeof(CellJob<T, D>) / sizeof(int)); w += NT) dst[w] = src[w];
    }
    __syncthreads();
    const Params &P = sJ.P;
    const FieldPtrs<T, D> &F = sJ.F;
    const int bid = (int)blockIdx.x - sJ.block0, nbk = sJ.nblocks;
    const int nx = P.nx, ny = P.ny, nm = D == 3 ? P.nz : P.ny;     // nm: planes along the marching axis
    const unsigned ps = D == 3 ? (unsigned)nx * (unsigned)ny : (unsigned)nx;   // cells per plane (grids < 2^31 cells)
    const int ntx = (nx + TX - 1) / TX, nty = D == 3 ? (ny + TY - 1) / TY : 1;
    const int zc = sJ.strip_rows, nch = (nm + zc - 1) / zc;
    const int items = ntx * nty * nch;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    auto slot5 = [](int m) { return (m + 10) % 5; };              // m >= -3
    auto slot3 = [](int m) { return (m + 3) % 3; };                // m >= -2
    // this thread's derived cells (halo-1 cells of a plane): shared-memory
    // index in a raw-field plane; the x_O plane's is RS * XR further
    int dix[DPT];
#pragma unroll
    for (int u = 0; u < DPT; u++) {
        const int l = threadIdx.x + u * NT;
        dix[u] = l < NE ? (l / EX) * RS + (l % EX) + CO - 1 : -1;
    }
    const int eown = (D == 3 ? (ty + 1) * RS : 0) + tx + CO;     // own cell in a raw-field plane
    Acc<T> acc[5];           // sum x_O, x_H, x_H2O, removed water, supplied H
    bool bad = false;

    for (int item = bid; item < items; item += nbk) {
        const int x0 = (item % ntx) * TX, y0 = D == 3 ? ((item / ntx) % nty) * TY : 0;
        const int m0 = (item / (ntx * nty)) * zc, m1 = min(m0 + zc, nm);
        // in-plane offset of a (possibly out-of-range) position
        auto off = [&](int x, int y) -> unsigned {
            return (unsigned)pwrap(x, nx) + (D == 3 ? (unsigned)nx * (unsigned)pwrap(y, ny) : 0u);
        };
        // aligned path: the tile's columns lie inside the grid and rows start
        // on 16-byte boundaries; this thread's copy task of every plane
        const bool vec = (nx % 4) == 0 && x0 + TX <= nx;
        int task = -1;               // 0: x_O piece / value, 1: raw-field piece / value
        bool piece = false;
        unsigned toff = 0;           // in-plane source offset
        int tdst = 0;                // shared-memory offset within a plane
        if (vec) {
            const int t = threadIdx.x;
            if (t >= Z::TE && t < Z::TE + Z::TO) {
                task = 0;
                const int r = (t - Z::TE) / (VW + 4), k = (t - Z::TE) % (VW + 4);
                const int col = k < VW ? CO + 4 * k : (k - VW < 2 ? CO - 2 + (k - VW) : CO + TX + (k - VW - 2));
                piece = k < VW;
                toff = off(x0 - CO + col, y0 - 2 + r);
                tdst = r * RS + col;
            } else if (t < Z::TE) {
                task = 1;
                const int t2 = t, r = t2 / (VW + 2), k = t2 % (VW + 2);
                const int col = k < VW ? CO + 4 * k : (k == VW ? CO - 1 : CO + TX);
                piece = k < VW;
                toff = off(x0 - CO + col, y0 - 1 + r);
                tdst = r * RS + col;
            }
        }
        auto issue_o = [&](int m) {
            const unsigned pb = ps * (unsigned)pwrap(m, nm);
            T *dst = sXO + slot5(m) * G;
            if (vec) {
                if (task == 0) {
                    if (piece) {
                        if constexpr (sizeof(T) == 4) cp_async16(dst + tdst, F.xO + (pb + toff));
                        else { cp_async16(dst + tdst, F.xO + (pb + toff)); cp_async16(dst + tdst + 2, F.xO + (pb + toff + 2)); }
                    } else {
                        cp_async(dst + tdst, F.xO + (pb + toff));
                    }
                }
                return;
            }
            for (int l = threadIdx.x; l < (TX + 4) * Z::GY; l += NT) {
                const int c = l % (TX + 4), r = l / (TX + 4);
                cp_async(dst + r * RS + c + CO - 2, F.xO + (pb + off(x0 - 2 + c, y0 - 2 + r)));
            }
        };
        auto issue_e = [&](int m) {
            const unsigned pb = ps * (unsigned)pwrap(m, nm);
            const int so = slot5(m) * E;
            if (vec) {
                if (task == 1) {
                    const unsigned g = pb + toff;
                    const int d = so + tdst;
                    if (piece) {
                        if constexpr (sizeof(T) == 4) {
                            cp_async16(sTh + d, F.theta + g); cp_async16(sPg + d, F.phig + g);
                            cp_async16(sXH + d, F.xH + g); cp_async16(sXW + d, F.xW + g);
                        } else {
                            cp_async16(sTh + d, F.theta + g); cp_async16(sPg + d, F.phig + g);
                            cp_async16(sXH + d, F.xH + g); cp_async16(sXW + d, F.xW + g);
                            cp_async16(sTh + d + 2, F.theta + g + 2); cp_async16(sPg + d + 2, F.phig + g + 2);
                            cp_async16(sXH + d + 2, F.xH + g + 2); cp_async16(sXW + d + 2, F.xW + g + 2);
                        }
                    } else {
                        cp_async(sTh + d, F.theta + g); cp_async(sPg + d, F.phig + g);
                        cp_async(sXH + d, F.xH + g); cp_async(sXW + d, F.xW + g);
                    }
                }
                return;
            }
            for (int l = threadIdx.x; l < NE; l += NT) {
                const int c = l % EX, r = l / EX;
                const unsigned g = pb + off(x0 - 1 + c, y0 - 1 + r);
                const int d = so + r * RS + c + CO - 1;
                cp_async(sTh + d, F.theta + g);
                cp_async(sPg + d, F.phig + g);
                cp_async(sXH + d, F.xH + g);
                cp_async(sXW + d, F.xW + g);
            }
        };
        // mu_O, M_O (Sec. 2.2, 3.2) and the species diffusivities (R4) of
        // plane m, own cells plus one halo cell in the plane
        auto derive = [&](int m) {
            const CellConst<T> &K = sJ.K;
            const T *xo = sXO + slot5(m) * G, *xlo = sXO + slot5(m - 1) * G, *xhi = sXO + slot5(m + 1) * G;
            const int se = slot5(m) * E, sm = slot3(m) * E;
#pragma unroll
            for (int u = 0; u < DPT; u++) {
                const int l = dix[u];
                if (l < 0) continue;
                const int q = l + RS * XR;
                const T x = xo[q];
                T lap;
                if constexpr (D == 3) {
                    lap = xo[q - 1] + xo[q + 1] + xo[q - RS] + xo[q + RS] - T(2 * D) * x;
                    lap += xlo[q] + xhi[q];
                } else {
                    lap = xo[q - 1] + xo[q + 1] + xlo[q] + xhi[q] - T(2 * D) * x;
                }
                T Wf, Ww, Wg;
                phase_weights(sTh[se + l], sPg[se + l], Wf, Ww, Wg);
                const T m1_ = Wf * f_fe1(x) + Ww * f_wu1(x) + Wg * f_ga1(x);
                const T m2_ = Wf * f_fe2(x) + Ww * f_wu2(x) + Wg * f_ga2(x);
                sMu[sm + l] = K.c * m1_ - K.kappa * lap;
                const T DO = (T(1) - Wg) * K.DOs + Wg * K.DOg;
                const T den = K.c * m2_;
                sM[sm + l] = den != T(0) ? fast_div(DO, den) : T(0);
                sDH[sm + l] = (T(1) - Wg) * K.DHs + Wg * K.DHg;
                sDW[sm + l] = (T(1) - Wg) * K.DWs + Wg * K.DWg;
            }
        };
        const int gxo = x0 + tx, gyo = y0 + ty;
        const bool own = gxo < nx && (D == 2 || gyo < ny);
        const unsigned goff = (unsigned)gxo + (D == 3 ? (unsigned)nx * (unsigned)gyo : 0u);
        // start-up: x_O planes m0 - 2 .. m0 + 1 and raw planes m0 - 1, m0 in
        // one group, x_O m0 + 2 and raw m0 + 1 in the next (the first
        // iteration's), then mu etc. of planes m0 - 1 and m0
        issue_o(m0 - 2);
        issue_o(m0 - 1);
        issue_o(m0);
        issue_o(m0 + 1);
        issue_e(m0 - 1);
        issue_e(m0);
        cp_async_commit();
        issue_o(m0 + 2);
        issue_e(m0 + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        derive(m0 - 1);
        derive(m0);
        // per-cell inputs of the first plane
        T tE = T(0), s2 = T(0), mob = T(0);
        unsigned char msk = 0;
        T cTh[3], cXH[3], cXW[3], cMu[3], cM[3], cDH[3], cDW[3];   // own cell, planes m - 1, m, m + 1
        if (own) {
            const unsigned g = goff + ps * (unsigned)m0;
            tE = F.trE[g]; s2 = F.devE2[g]; mob = F.mob[g]; msk = F.mask[g];
        }
        for (int m = m0; m < m1; m++) {
            // the next plane's copies go out first (group of plane m + 1 for
            // the raw fields, m + 2 for x_O is already in flight), then this
            // iteration waits for the group issued one iteration ago
            if (m + 1 < m1) {
                issue_o(m + 3);
                issue_e(m + 2);
            }
            cp_async_commit();
            cp_async_wait<1>();
            // the next plane's per-cell inputs (registers)
            T tEn = T(0), s2n = T(0), mobn = T(0);
            unsigned char mskn = 0;
            if (own && m + 1 < m1) {
                const unsigned gn = goff + ps * (unsigned)(m + 1);
                tEn = F.trE[gn]; s2n = F.devE2[gn]; mobn = F.mob[gn]; mskn = F.mask[gn];
            }
            __syncthreads();
            derive(m + 1);
            __syncthreads();
            if (own) {
                const CellConst<T> &K = sJ.K;
                const unsigned g = goff + ps * (unsigned)m;
                const int e = eown;
                const int sc = slot5(m) * E, sh = slot5(m + 1) * E;
                const int mc = slot3(m) * E, mh = slot3(m + 1) * E;
                // the own cell's values of the planes before and after (the
                // cross-plane neighbours) roll through registers
                if (m == m0) {
                    const int sl = slot5(m - 1) * E, ml = slot3(m - 1) * E;
                    cTh[0] = sTh[sl + e]; cXH[0] = sXH[sl + e]; cXW[0] = sXW[sl + e];
                    cMu[0] = sMu[ml + e]; cM[0] = sM[ml + e]; cDH[0] = sDH[ml + e]; cDW[0] = sDW[ml + e];
                    cTh[1] = sTh[sc + e]; cXH[1] = sXH[sc + e]; cXW[1] = sXW[sc + e];
                    cMu[1] = sMu[mc + e]; cM[1] = sM[mc + e]; cDH[1] = sDH[mc + e]; cDW[1] = sDW[mc + e];
                }
                cTh[2] = sTh[sh + e]; cXH[2] = sXH[sh + e]; cXW[2] = sXW[sh + e];
                cMu[2] = sMu[mh + e]; cM[2] = sM[mh + e]; cDH[2] = sDH[mh + e]; cDW[2] = sDW[mh + e];
                const T th = cTh[1], pg = sPg[sc + e];
                const T xo = sXO[slot5(m) * G + e + RS * XR];
                const T xh = cXH[1], xw = cXW[1];
                const T mu0 = cMu[1], M0 = cM[1], DH0 = cDH[1], DW0 = cDW[1];
                // neighbours in the order x-, x+, y-, y+ (, z-, z+): in-plane
                // ones from shared memory, then the planes before and after
                constexpr int NI = D == 3 ? 4 : 2;      // in-plane neighbours
                const int io[4] = {-1, 1, -RS, RS};
                T lapt = T(0), dO = T(0), dH = T(0), dW = T(0);
#pragma unroll
                for (int qn = 0; qn < NI; qn++) {
                    const int a = sc + e + io[qn], b = mc + e + io[qn];
                    lapt += sTh[a] - th;
                    dO += T(0.5) * (M0 + sM[b]) * (sMu[b] - mu0);
                    dH += T(0.5) * (DH0 + sDH[b]) * (sXH[a] - xh);
                    dW += T(0.5) * (DW0 + sDW[b]) * (sXW[a] - xw);
                }
#pragma unroll
                for (int k = 0; k < 3; k += 2) {
                    lapt += cTh[k] - th;
                    dO += T(0.5) * (M0 + cM[k]) * (cMu[k] - mu0);
                    dH += T(0.5) * (DH0 + cDH[k]) * (cXH[k] - xh);
                    dW += T(0.5) * (DW0 + cDW[k]) * (cXW[k] - xw);
                }
                cTh[0] = cTh[1]; cXH[0] = cXH[1]; cXW[0] = cXW[1];
                cMu[0] = cMu[1]; cM[0] = cM[1]; cDH[0] = cDH[1]; cDW[0] = cDW[1];
                cTh[1] = cTh[2]; cXH[1] = cXH[2]; cXW[1] = cXW[2];
                cMu[1] = cMu[2]; cM[1] = cM[2]; cDH[1] = cDH[2]; cDW[1] = cDW[2];
                const T hg0 = hfun(pg);
                const T hpt = hder(th);
                const T sol = T(1) - hg0;
                const T Af = K.c * f_fe(xo) + T(0.5) * K.Ks * tE * tE + K.Gs * s2;
                const T Aw = K.c * f_wu(xo) + T(0.5) * K.Ks * tE * tE + K.Gs * s2;
                const T Kmix = sol * K.Ks + hg0 * K.Kg;
                const T force = sol * hpt * (Af - Aw) + K.w2 * mder(th) - K.eig3 * sol * hpt * Kmix * tE;
                const T rate = K.Lh * mob * (force - K.eps2 * lapt);
                T rr = mfun(pg) * K.kf * xo * xh;
                if (xw >= T(1)) rr = T(0);
                const T nth = th + K.dt * rate;
                const T nxo = xo + K.dt * (dO - rr);
                T nxh = xh + K.dt * (dH - T(2) * rr);
                T nxw = xw + K.dt * (dW + rr);
                if (msk) {
                    acc[3].add(nxw);
                    acc[4].add(K.xHbc - nxh);
                    nxh = K.xHbc;
                    nxw = T(0);
                }
                F.theta_o[g] = nth;
                F.xO_o[g] = nxo;
                F.xH_o[g] = nxh;
                F.xW_o[g] = nxw;
                acc[0].add(nxo); acc[1].add(nxh); acc[2].add(nxw);
                bad |= !isfinite(nth + nxo + nxh + nxw);
            }
            tE = tEn; s2 = s2n; mob = mobn; msk = mskn;
        }
        cp_async_wait<0>();
        __syncthreads();       // the next item's copies reuse every ring slot
    }
    Acc<T> acc6[6];
#pragma unroll
    for (int q = 0; q < 5; q++) acc6[q] = acc[q];
    acc6[5].add(T(bad ? 1 : 0));
    double *partials = sJ.partials;
    unsigned int *counter = sJ.counter;
    block_reduce_store<6>(acc6, partials + (size_t)bid * PSTRIDE);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int tk = atomicAdd(counter, 1u);
        last = (tk == (unsigned int)nbk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        __shared__ double tot[6];
        last_block_sums<6>(partials, nbk, tot);
        if (threadIdx.x == 0) {
            Diag *dg = sJ.dg;
            dg->sumO_prev = dg->sumO;
            dg->sumO = tot[0]; dg->sumH = tot[1]; dg->sumW = tot[2];
            dg->removedW += tot[3];
            dg->suppliedH += tot[4];
            if (tot[5] > 0.0 && dg->status == 0) dg->status = 5;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Learned warm start: network inputs and the guess update.  The network
// predicts the rate of the displacement, du/dt / |eig0|, from the phase
// weights, the prestress and the rate of the ferrite weight, dW_f/dt.
// ---------------------------------------------------------------------------
// in[4c..4c+3] = W_f, W_g, p/|eig0|, (W_f - W_f,prev) / dt (0 on the first
// step after pf_set_fields, mode != 0); W_f,prev = W_f.
template <typename T>
__global__ void k_net_input(long long N, const T *theta, const T *phig, float pscaled, float inv_dt,
                            const int *mode, float *wf_prev, float *in)
{
    const int md = *mode;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        T Wf, Ww, Wg;
        phase_weights(theta[c], phig[c], Wf, Ww, Wg);
        const float wf = (float)Wf;
        in[4 * c] = wf;
        in[4 * c + 1] = (float)Wg;
        in[4 * c + 2] = pscaled;
        in[4 * c + 3] = md == 0 ? (wf - wf_prev[c]) * inv_dt : 0.f;
        wf_prev[c] = wf;
    }
}

// u += s y (s = |eig0| dt) unless this is the first step after
// pf_set_fields (mode != 0).  In the mixed method the FP64 copy x64 is the
// solve's initial guess and u follows it.
template <typename T, int D>
__global__ void k_net_guess(long long N, const float *y, const int *mode, double s,
                            T *u0, T *u1, T *u2, double *x0, double *x1, double *x2)
{
    if (*mode != 0) return;
    T *u[3] = {u0, u1, u2};
    double *x[3] = {x0, x1, x2};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < D; d++) {
            const double delta = s * (double)y[D * c + d];
            if (x[d]) {
                const double v = x[d][c] + delta;
                x[d][c] = v;
                u[d][c] = (T)v;
            } else {
                u[d][c] = (T)((double)u[d][c] + delta);
            }
        }
    }
}

static __global__ void k_net_mode_clear(int *mode) { *mode = 0; }

// Extrapolated initial guess of the solve (PF_WS_EXTRAP, order 1;
// PF_WS_EXTRAP2, order 2): with x_n the last solution and h0 = x_{n-1},
// h1 = x_{n-2} the ones before it, the guess is 2 x_n - x_{n-1} (linear in
// time) or 3 x_n - 3 x_{n-1} + x_{n-2} (quadratic); the history then shifts
// by one.  *count (reset by pf_set_fields) is the number of guesses formed
// since: the state set by the caller is not a solution of a previous step,
// so a guess of order k needs count >= k + 1, and lower orders are used
// while the history fills.  In the mixed method the FP64 copy x64 is the
// solve's initial guess and u follows it.  h1 may be null (order 1).
template <typename T, int D>
__global__ void k_extrap(long long N, const int *count, int order, T *u0, T *u1, T *u2, double *x0, double *x1,
                         double *x2, double *h00, double *h01, double *h02, double *h10, double *h11, double *h12)
{
    const int cnt = *count;
    const int ord = order >= 2 && cnt >= 3 ? 2 : (cnt >= 2 ? 1 : 0);
    T *u[3] = {u0, u1, u2};
    double *x[3] = {x0, x1, x2}, *h0[3] = {h00, h01, h02}, *h1[3] = {h10, h11, h12};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < D; d++) {
            const double xn = x[d] ? x[d][c] : (double)u[d][c];
            const double x1v = h0[d][c];
            if (ord > 0) {
                const double g = ord == 2 ? 3.0 * (xn - x1v) + h1[d][c] : 2.0 * xn - x1v;
                if (x[d]) x[d][c] = g;
                u[d][c] = (T)g;
            }
            if (h1[d]) h1[d][c] = x1v;
            h0[d][c] = xn;
        }
    }
}

// The mean strain's part of the extrapolated guess (Eh: [0, 6) the
// previous, [6, 12) the one before), and the count.
static __global__ void k_extrap_tail(int *count, int order, double *E, double *Eh, int nv)
{
    if (threadIdx.x != 0) return;
    const int cnt = *count;
    const int ord = order >= 2 && cnt >= 3 ? 2 : (cnt >= 2 ? 1 : 0);
    for (int v = 0; v < nv; v++) {
        const double en = E[v], e1 = Eh[v];
        if (ord == 2) E[v] = 3.0 * (en - e1) + Eh[6 + v];
        else if (ord == 1) E[v] = 2.0 * en - e1;
        Eh[6 + v] = e1;
        Eh[v] = en;
    }
    if (cnt < 3) *count = cnt + 1;
}

// Self-test of the bounded wait: one thread waits on a generation word that
// nothing advances.
static __global__ void k_wait_selftest(const unsigned int *gen, int *err, long long limit)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) wait_generation(gen, 0u, err, limit);
}

// ---------------------------------------------------------------------------
// Conversions between the caller's FP64 cell-major arrays and device storage
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_in_scalar(long long N, const double *src, T *dst, double dflt)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        dst[c] = (T)(src ? src[c] : dflt);
}

template <typename T>
__global__ void k_in_comp(long long N, int ncomp, const double *src, T *const *dst)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        for (int k = 0; k < ncomp; k++) dst[k][c] = (T)(src ? src[c * ncomp + k] : 0.0);
}

// *changed = 1 if any component differs from (double) of the stored one
template <typename T>
__global__ void k_comp_differs(long long N, int ncomp, const double *src, const T *const *cur, int *changed)
{
    bool diff = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        for (int k = 0; k < ncomp; k++)
            if ((src ? src[c * ncomp + k] : 0.0) != (double)cur[k][c]) diff = true;
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) *changed = 1;
}

// k_in_comp, unless *changed == 0 (changed == nullptr: always)
template <typename T>
__global__ void k_in_comp_if(long long N, int ncomp, const double *src, T *const *dst, const int *changed)
{
    if (changed && *changed == 0) return;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        for (int k = 0; k < ncomp; k++) dst[k][c] = (T)(src ? src[c * ncomp + k] : 0.0);
}

// the extrapolated guess starts over unless the displacement came back
// unchanged (changed == nullptr: always)
static __global__ void k_ext_restart(const int *changed, int *count)
{
    if (!changed || *changed) *count = 0;
}

// (phi_f, phi_w) -> theta = phi_f / (phi_f + phi_w) (0 where no solid), phi_g
template <typename T>
__global__ void k_in_phase(long long N, const double *pf, const double *pw, T *theta, T *phig)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double s = pf[c] + pw[c];
        theta[c] = (T)(s > 0.0 ? pf[c] / s : 0.0);
        phig[c] = (T)(1.0 - s);
    }
}

template <typename T>
__global__ void k_out_scalar(long long N, const T *src, double *dst)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        dst[c] = (double)src[c];
}

template <typename T>
__global__ void k_out_comp(long long N, int ncomp, T *const *src, double *dst)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        for (int k = 0; k < ncomp; k++) dst[c * ncomp + k] = (double)src[k][c];
}

template <typename T>
__global__ void k_out_phase(long long N, const T *theta, const T *phig, double *pf, double *pw)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double s = 1.0 - (double)phig[c];
        if (pf) pf[c] = s * (double)theta[c];
        if (pw) pw[c] = s * (1.0 - (double)theta[c]);
    }
}

// sum of x_O (for the initial reference of the reduction degree)
template <typename T>
__global__ void k_sum(long long N, const T *a, double *partials)
{
    Acc<T> s;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) s.add(a[c]);
    double v[1] = {s.value()};
    block_sum_store<1>(v, partials + (size_t)blockIdx.x * PSTRIDE);
}

// Discrete free energy (per-block partials): cell bulk + well + elastic
// energy and forward-face gradient energies.
template <typename T, int D>
__global__ void k_free_energy(Params P, FieldPtrs<T, D> F, double *partials)
{
    Acc<double> e;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < P.N; c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords<D>(P, c, i, j, k);
        const double th = F.theta[c], pg = F.phig[c], x = F.xO[c];
        const double t = F.trE[c], s2 = F.devE2[c];
        double Wf, Ww, Wg;
        phase_weights<double>(th, pg, Wf, Ww, Wg);
        double v = Wf * (P.c * f_fe(x) + 0.5 * P.Ks * t * t + P.Gs * s2)
                 + Ww * (P.c * f_wu(x) + 0.5 * P.Ks * t * t + P.Gs * s2)
                 + Wg * (P.c * f_ga(x) + 0.5 * P.Kg * t * t + P.Gg * s2)
                 + 2.0 * P.w * mfun(th);
        long long nb[3] = {lin<D>(P, i + 1, j, k), lin<D>(P, i, j + 1, k), D == 3 ? lin<D>(P, i, j, k + 1) : 0};
        for (int q = 0; q < D; q++) {
            const double gt = (double)F.theta[nb[q]] - th, gx = (double)F.xO[nb[q]] - x;
            v += P.eps * gt * gt + 0.5 * P.kappa * gx * gx;
        }
        e.add(v);
    }
    double vv[1] = {e.value()};
    block_sum_store<1>(vv, partials + (size_t)blockIdx.x * PSTRIDE);
}

} // namespace pfdev
