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
template <typename T, int D>
struct CellJob {
    Params P;
    FieldPtrs<T, D> F;
    const Scalars *sc;       // mean strain for the return map
    double *partials;        // per-block sums of the update
    unsigned int *counter;   // last-block counter of the update
    Diag *dg;
    int block0, nblocks;
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
            dg->sumO = tot[0]; dg->sumH = tot[1]; dg->sumW = tot[2];
            dg->removedW += tot[3];
            dg->suppliedH += tot[4];
            if (tot[5] > 0.0 && dg->status == 0) dg->status = 5;
            *counter = 0u;
        }
    }
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
