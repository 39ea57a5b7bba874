// Host side of the C ABI declared in include/pf.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>
#include <mutex>

#include "pf.h"
#include "pf_unet.h"
#include "unet_net.h"
#include "pf_cg.cuh"
#include "pcg_launch.h"
#include "pf_implicit.cuh"

// k_extrap_tail addresses the mean strain as the start of Scalars
static_assert(offsetof(pfdev::Scalars, E) == 0, "Scalars::E must be the first member");

// Launch shapes per size class, written by paper_2111_11538_gb300/autotune.py
// from its measurements on GB300 (PCG node tiles of the Jacobi and the 2D
// multigrid solves, start-up weight of the marching update's chunk choice).
#include "tuning.h"

using namespace pfdev;

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------------------
// Element tables: Q1 unit square / cube, stiffness split into the lambda and
// mu parts, integrated exactly with 2^d Gauss points.
// ---------------------------------------------------------------------------
void element_tables(int d, std::vector<double> &Kl, std::vector<double> &Km, std::vector<double> &Bb)
{
    const int nn = 1 << d, ne = nn * d, nv = d == 2 ? 3 : 6;
    Kl.assign(ne * ne, 0.0);
    Km.assign(ne * ne, 0.0);
    Bb.assign(nn * d, 0.0);
    const double g0 = 0.5 - 0.5 / std::sqrt(3.0), g1 = 0.5 + 0.5 / std::sqrt(3.0);
    const double wgt = 1.0 / nn;
    for (int g = 0; g < nn; g++) {
        double xi[3];
        for (int l = 0; l < d; l++) xi[l] = ((g >> l) & 1) ? g1 : g0;
        double dn[8][3];
        for (int a = 0; a < nn; a++)
            for (int k = 0; k < d; k++) {
                double v = 1.0;
                for (int l = 0; l < d; l++) {
                    const int bit = (a >> l) & 1;
                    if (l == k) v *= bit ? 1.0 : -1.0;
                    else v *= bit ? xi[l] : 1.0 - xi[l];
                }
                dn[a][k] = v;
                Bb[a * d + k] += wgt * v;
            }
        // strain-displacement matrix B (nv x ne), engineering shears
        std::vector<double> B(nv * ne, 0.0);
        for (int a = 0; a < nn; a++) {
            auto at = [&](int row, int comp, double v) { B[row * ne + a * d + comp] = v; };
            if (d == 2) {
                at(0, 0, dn[a][0]); at(1, 1, dn[a][1]);
                at(2, 0, dn[a][1]); at(2, 1, dn[a][0]);
            } else {
                at(0, 0, dn[a][0]); at(1, 1, dn[a][1]); at(2, 2, dn[a][2]);
                at(3, 1, dn[a][2]); at(3, 2, dn[a][1]);
                at(4, 0, dn[a][2]); at(4, 2, dn[a][0]);
                at(5, 0, dn[a][1]); at(5, 1, dn[a][0]);
            }
        }
        // D_lambda = m m^T (normal rows), D_mu = diag(2 on normals, 1 on shears)
        for (int r = 0; r < ne; r++)
            for (int c = 0; c < ne; c++) {
                double trr = 0.0, trc = 0.0, mu = 0.0;
                for (int v = 0; v < d; v++) { trr += B[v * ne + r]; trc += B[v * ne + c]; }
                for (int v = 0; v < nv; v++) mu += (v < d ? 2.0 : 1.0) * B[v * ne + r] * B[v * ne + c];
                Kl[r * ne + c] += wgt * trr * trc;
                Km[r * ne + c] += wgt * mu;
            }
    }
}

template <typename T>
void fill_tab(Tab<T> &t)
{
    std::vector<double> Kl, Km, Bb;
    element_tables(2, Kl, Km, Bb);
    for (int i = 0; i < 64; i++) { t.Kl2[i] = (T)Kl[i]; t.Km2[i] = (T)Km[i]; }
    for (int i = 0; i < 8; i++) t.Bb2[i] = (T)Bb[i];
    t.Kdiag[0] = (T)Kl[0]; t.Kdiag[1] = (T)Km[0];
    element_tables(3, Kl, Km, Bb);
    for (int i = 0; i < 576; i++) { t.Kl3[i] = (T)Kl[i]; t.Km3[i] = (T)Km[i]; }
    for (int i = 0; i < 24; i++) t.Bb3[i] = (T)Bb[i];
    t.Kdiag[2] = (T)Kl[0]; t.Kdiag[3] = (T)Km[0];
}

bool upload_tables(int dev)
{
    static bool done[64] = {false};
    if (dev >= 0 && dev < 64 && done[dev]) return true;
    Tab<double> td;
    Tab<float> tf;
    fill_tab(td);
    fill_tab(tf);
    if (cudaMemcpyToSymbol(cTabD, &td, sizeof(td)) != cudaSuccess) return false;
    if (cudaMemcpyToSymbol(cTabF, &tf, sizeof(tf)) != cudaSuccess) return false;
    if (pcg2_tables(&tf, &td) != cudaSuccess) return false;
    if (pcg3_tables(&tf, &td) != cudaSuccess) return false;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return true;
}

double dt_stable_impl(const pf_config *c)
{
    const int d = c->ndim;
    const pf_params &p = c->p;
    const double Ds[6] = {p.D_O_s, p.D_O_g, p.D_H_s, p.D_H_g, p.D_W_s, p.D_W_g};
    double Dmax = 0.0;
    for (double v : Ds) Dmax = std::fmax(Dmax, v);
    double dt = 1.0e300;
    if (Dmax > 0.0) dt = std::fmin(dt, 1.0 / (2.0 * d * Dmax));
    // smallest curvature of the phase energies: the ferrite quartic's minimum
    // second derivative (at x = 6 * 182.510 / (24 * 163.708)) or wuestite's
    const double xm = 6.0 * 182.510 / (24.0 * 163.708);
    double fmin = 12.0 * 163.708 * xm * xm - 6.0 * 182.510 * xm + 2.0 * 90.573;
    fmin = std::fmin(fmin, 2.0 * 173.263);
    if (p.kappa_O > 0.0 && p.c_chem > 0.0 && Dmax > 0.0) {
        const double Mmax = Dmax / (p.c_chem * fmin);
        dt = std::fmin(dt, 2.0 / (Mmax * p.kappa_O * (4.0 * d) * (4.0 * d)));
    }
    if (p.L > 0.0) dt = std::fmin(dt, 1.0 / (1.2 * p.L * (2.0 * d * p.eps_phi + 2.0 * p.w)));
    if (p.k_for > 0.0) dt = std::fmin(dt, 1.0 / (p.k_for * (1.0 / 16.0) * (0.571 + 2.0 * p.xH_bc)));
    return dt;
}

// Device parameter block of a (validated) configuration; 2D grids use nz = 1.
void fill_params(const pf_config &c, long long N, Params &P)
{
    memset(&P, 0, sizeof(P));
    P.ndim = c.ndim; P.nx = c.nx; P.ny = c.ny; P.nz = c.ndim == 3 ? c.nz : 1; P.N = N;
    P.dt = c.dt > 0.0 ? c.dt : 0.2 * dt_stable_impl(&c);
    P.c = c.p.c_chem; P.w = c.p.w; P.eps = c.p.eps_phi; P.kappa = c.p.kappa_O; P.L = c.p.L;
    P.DOs = c.p.D_O_s; P.DOg = c.p.D_O_g; P.DHs = c.p.D_H_s; P.DHg = c.p.D_H_g; P.DWs = c.p.D_W_s; P.DWg = c.p.D_W_g;
    P.kfor = c.p.k_for; P.xHbc = c.p.xH_bc;
    const double Es = c.p.E_s, Eg = c.p.E_s * c.p.E_g_ratio, nu = c.p.nu;
    P.Ks = Es / (3.0 * (1.0 - 2.0 * nu)); P.Gs = Es / (2.0 * (1.0 + nu));
    P.Kg = Eg / (3.0 * (1.0 - 2.0 * nu)); P.Gg = Eg / (2.0 * (1.0 + nu));
    P.eig0 = c.p.eig0; P.sY = c.p.sigma_Y; P.Hh = c.p.H_hard; P.prestress = c.p.prestress;
    P.plasticity = c.plasticity;
}

} // namespace

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct pf_handle {
    pf_config cfg;
    Params P;
    int dev = 0, sms = 0;
    bool fp64 = true;
    size_t tsz = 8;
    cudaStream_t own = nullptr;
    std::string err;
    bool have_fields = false;
    long long steps = 0;
    double sumO0 = 0.0;
    long long bytes = 0;
    std::vector<void *> allocs;

    // device arrays (void* so one handle type serves both precisions)
    void *theta[2] = {nullptr, nullptr}, *xO[2] = {}, *xH[2] = {}, *xW[2] = {};
    int cur = 0;
    void *phig = nullptr, *mob = nullptr, *muO = nullptr, *MO = nullptr, *trE = nullptr, *devE2 = nullptr;
    void *lam = nullptr, *mu = nullptr, *sig[6] = {}, *ep[6] = {}, *alpha = nullptr, *sigma[6] = {};
    void *u[3] = {}, *p[3] = {}, *r[2][3] = {}, *w[2][3] = {}, *s[2][3] = {}, *diag = nullptr;
    void *corr[3] = {};                // mixed mode: FP32 correction of one refinement pass
    double *x64[3] = {};               // mixed mode: FP64 displacement
    bool refine = false;
    double *result = nullptr;
    unsigned char *mask = nullptr;
    double *partials = nullptr;
    int npart = 0;
    unsigned int *sync = nullptr;      // barrier count, barrier generation, last-block counter (own 128-B lines)
    Scalars *sc = nullptr;
    Diag *dg = nullptr;
    double *stage = nullptr, *stage2 = nullptr;
    void **ptrtab = nullptr;           // device table of component pointers (6 entries)
    int cg_block = 256;
    bool sigma_valid = false;

    // Launch plan.  Every kernel of a step serves all instances of the handle
    // (one for pf_create, several for pf_batch_create) through job tables in
    // device memory; tables [k] describe the state k steps from now.
    bool is_batch = false;
    std::vector<pf_handle *> members;   // batch members (owned by the batch)
    void *d_cell_jobs[2] = {nullptr, nullptr};
    void *d_fused_jobs[2] = {nullptr, nullptr};
    void *d_pcg_jobs = nullptr;
    int cell_grid = 0, fused_grid = 0, pcg_grid = 0, njobs = 0;
    int cg_per_sm = 0;
    int fused_per_sm = 0;               // resident blocks per SM of the marching update
    int pcg_shape = 0;                  // node tile of the PCG sweep (pf_cg.cuh Tile<D, S>)
    bool mg = false;                    // multigrid-preconditioned CG (pf_mg.cuh)
    double *b64[3] = {};                // MG mixed method: FP64 right-hand side kept across passes
    void *d_mg = nullptr;               // device MGHier<T> of this instance
    bool plan_ready = false;
    int plan_par = 0;                   // which table describes the current state
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step from job tables [k]
    bool graph_failed = false;
    bool use_graph = true;

    // backward-Euler steps (pf_step_implicit): work arrays allocated at the
    // first call (be_len values) and the time step of the last step taken
    // that way (0 after explicit steps: the configured dt)
    double *be_ws = nullptr;
    size_t be_len = 0;
    double dt_last = 0.0;

    // learned warm start (pf_attach_unet)
    pf_unet *net = nullptr;
    UWork *net_work = nullptr;
    float *net_in = nullptr;            // N x 4 network inputs
    float *net_prev = nullptr;          // N previous ferrite weight
    int *net_mode = nullptr;            // 1: first step after pf_set_fields (no guess), 0: guess
    // extrapolated warm start (PF_WS_EXTRAP): the previous solution (FP64),
    // the previous mean strain, and the number of guesses since set_fields
    double *ext_hist[2][3] = {};       // [0]: x_{n-1}, [1]: x_{n-2} (order 2 only)
    double *ext_E = nullptr;
    int *ext_count = nullptr;
    int *u_changed = nullptr;          // set_fields: the displacement differs from the handle's own
    std::vector<void *> net_allocs;

    // profiling: event pairs around each launch while enabled
    bool prof_on = false;
    pf_profile prof;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_class;   // class of each recorded pair
    size_t ev_used = 0;          // events recorded since the last harvest
    long long cg_total_seen = 0; // CG iteration total at the end of the last pf_step

    cudaEvent_t next_event()
    {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }
    void mark_begin(int cls, cudaStream_t s)
    {
        prof.launches++;
        prof.count[cls]++;
        if (!prof_on) return;
        cudaEvent_t e = next_event();
        if (e) cudaEventRecord(e, s);
        ev_class.push_back(cls);
    }
    void mark_end(cudaStream_t s)
    {
        if (!prof_on) return;
        cudaEvent_t e = next_event();
        if (e) cudaEventRecord(e, s);
    }
    void harvest()
    {
        for (size_t k = 0; k + 1 < ev_used && k / 2 < ev_class.size(); k += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev_pool[k], ev_pool[k + 1]) == cudaSuccess) prof.ms[ev_class[k / 2]] += ms;
        }
        ev_used = 0;
        ev_class.clear();
    }

    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda(cudaError_t e, const char *what)
    {
        if (e == cudaSuccess) return PF_OK;
        return fail(e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    template <typename X>
    int alloc(X **ptr, size_t bytes_)
    {
        void *v = nullptr;
        cudaError_t e = cudaMalloc(&v, bytes_ ? bytes_ : 16);
        if (e != cudaSuccess) return fail(PF_ENOMEM, "cudaMalloc(%zu): %s", bytes_, cudaGetErrorString(e));
        allocs.push_back(v);
        bytes += (long long)bytes_;
        *ptr = (X *)v;
        return PF_OK;
    }
};

#define PF_TRY(x) do { int _rc = (x); if (_rc != PF_OK) return _rc; } while (0)

namespace {

int grid_for(const pf_handle *h, long long n, int block = 256)
{
    long long g = (n + block - 1) / block;
    long long cap = (long long)h->sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T, int D>
FieldPtrs<T, D> field_ptrs(pf_handle *h)
{
    FieldPtrs<T, D> F;
    const int c = h->cur, o = 1 - h->cur;
    F.theta = (const T *)h->theta[c]; F.xO = (const T *)h->xO[c]; F.xH = (const T *)h->xH[c]; F.xW = (const T *)h->xW[c];
    F.theta_o = (T *)h->theta[o]; F.xO_o = (T *)h->xO[o]; F.xH_o = (T *)h->xH[o]; F.xW_o = (T *)h->xW[o];
    F.phig = (const T *)h->phig; F.mob = (const T *)h->mob; F.mask = h->mask;
    F.muO = (T *)h->muO; F.MO = (T *)h->MO; F.trE = (T *)h->trE; F.devE2 = (T *)h->devE2;
    F.lam = (T *)h->lam; F.mu = (T *)h->mu;
    for (int v = 0; v < 6; v++) { F.sig[v] = (T *)h->sig[v]; F.ep[v] = (T *)h->ep[v]; F.sigma_out[v] = (T *)h->sigma[v]; }
    F.alpha = (T *)h->alpha;
    for (int d = 0; d < 3; d++) F.u[d] = (T *)h->u[d];
    return F;
}

std::vector<pf_handle *> instances(pf_handle *h)
{
    return h->is_batch ? h->members : std::vector<pf_handle *>{h};
}

// Node tile of the PCG sweep for a grid of N nodes: pf_config.pcg_tile if
// set (1 or 2 select shape 0 or 1), else the per-size-class choice measured
// on GB300 (paper_2111_11538_gb300/autotune.py prints the table).
int default_pcg_shape(int ndim, long long N, bool fp64)
{
    if (ndim == 2) {
        if (fp64) return N <= (1LL << 18) ? PCG_TABLE_2D_F64_SMALL : PCG_TABLE_2D_F64_LARGE;
        return N <= (1LL << 18) ? PCG_TABLE_2D_F32_SMALL : PCG_TABLE_2D_F32_LARGE;
    }
    return fp64 ? PCG_TABLE_3D_F64 : PCG_TABLE_3D_F32;
}

// Node tile of the 2D multigrid-preconditioned solve (its V-cycle sweeps use
// the same tile), per size class.
int mg2_pcg_shape(long long N, bool fp64)
{
    if (fp64) return N <= (1LL << 18) ? PCG_TABLE_MG2D_F64_SMALL : PCG_TABLE_MG2D_F64_LARGE;
    return N <= (1LL << 18) ? PCG_TABLE_MG2D_F32_SMALL : PCG_TABLE_MG2D_F32_LARGE;
}

// Largest eigenvalue of diag(K_e)^-1 K_e for the d-dimensional Q1 element
// with Poisson ratio nu (power iteration on the symmetric scaling
// D^-1/2 K_e D^-1/2).
// Summing x_e^T K_e x_e <= w x_e^T diag(K_e) x_e over the cells bounds the
// largest eigenvalue of D^-1 A by w for any cell moduli with this ratio.
double element_bound(double nu, int d)
{
    std::vector<double> Kl, Km, Bb;
    element_tables(d, Kl, Km, Bb);
    const int ne = d == 2 ? 8 : 24;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 0.5 / (1.0 + nu);
    std::vector<double> K(ne * ne), sc(ne), v(ne), w(ne);
    for (int i = 0; i < ne * ne; i++) K[i] = lam * Kl[i] + mu * Km[i];
    for (int i = 0; i < ne; i++) { sc[i] = 1.0 / std::sqrt(K[i * (ne + 1)]); v[i] = 1.0 + 0.1 * i; }
    double ray = 0.0;
    for (int it = 0; it < 2000; it++) {
        double nv = 0.0, vw = 0.0, vv = 0.0;
        for (int i = 0; i < ne; i++) {
            double acc = 0.0;
            for (int j = 0; j < ne; j++) acc += sc[i] * K[i * ne + j] * sc[j] * v[j];
            w[i] = acc;
        }
        for (int i = 0; i < ne; i++) { vw += v[i] * w[i]; nv += w[i] * w[i]; vv += v[i] * v[i]; }
        ray = vw / vv;
        nv = 1.0 / std::sqrt(nv);
        for (int i = 0; i < ne; i++) v[i] = w[i] * nv;
    }
    return ray;
}

// Multigrid hierarchy of one 2D instance (pf_mg.cuh): coarsen while both
// sizes stay even and the coarse grid keeps >= 8 nodes per axis; levels of
// at most mg_block_nodes<T>() nodes are run by one block in shared memory;
// Chebyshev coefficients over [b/30, b] with b 2% above the element bound.
// The device descriptor is written once (the arrays never move).
// Smoothing steps per level: one on the finest (its sweeps are the
// expensive ones, and a second step there does not lower the iteration
// count), two on the other levels (measured on GB300 at 512^2: three on the
// shared-memory levels made a step slower, 1.30 vs 1.14 ms); the coarsest
// solve takes MG_CSTEPS (>= 3: its last sweep is then a Chebyshev step,
// whose epilogue applies the final pointwise step; 6 was no faster).
constexpr int MG_DEG_FINE = 1, MG_DEG_GRID = 2, MG_DEG_BLOCK = 2, MG_CSTEPS = 8;
static_assert(MG_CSTEPS >= 3 && MG_CSTEPS < MG_MAX_STEPS && MG_DEG_BLOCK + 1 < MG_MAX_STEPS, "multigrid step counts");

// Levels of the multigrid hierarchy of an nx x ny grid.
int mg_levels(int nx, int ny)
{
    int L = 1;
    while (L < MG_MAX_LEVELS && nx % 2 == 0 && ny % 2 == 0 && nx >= 16 && ny >= 16) {
        nx /= 2;
        ny /= 2;
        L++;
    }
    return L;
}

// Levels of the 3D hierarchy: halve while all three sizes are even and the
// coarse grid keeps >= 8 nodes per axis.
int mg_levels3(int nx, int ny, int nz)
{
    int L = 1;
    while (L < MG_MAX_LEVELS && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && nx >= 16 && ny >= 16 && nz >= 16) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        L++;
    }
    return L;
}

// PF_PC_AUTO: multigrid for grids with at least three levels (sizes
// divisible by 4 and >= 32), where it needs a small fraction of Jacobi's
// iterations and, measured on GB300, less time (2D 512^2: 1.9x per step;
// 3D 96^3 and 128^3: 2.1x and 2.6x); Jacobi otherwise.
bool auto_mg(const pf_config &c)
{
    if (!c.mechanics) return false;
    return c.ndim == 2 ? mg_levels(c.nx, c.ny) >= 3 : mg_levels3(c.nx, c.ny, c.nz) >= 3;
}

template <typename T, int D>
int build_mg(pf_handle *h)
{
    MGHier<T> H;
    memset(&H, 0, sizeof(H));
    int nx = h->P.nx, ny = h->P.ny, nz = D == 3 ? h->P.nz : 1;
    const int L = D == 2 ? mg_levels(nx, ny) : mg_levels3(nx, ny, nz);
    H.L = L;
    H.Lg = L;                  // 3D: every level on the whole grid
    H.csteps = MG_CSTEPS;
    for (int k = 0; k < L; k++) {
        MGLevel<T> &V = H.lv[k];
        V.nx = nx;
        V.ny = ny;
        V.nz = nz;
        const size_t nodes = (size_t)nx * (size_t)ny * (size_t)nz, b = sizeof(T) * nodes;
        if (k == 0) {
            V.lam = (T *)h->lam;
            V.mu = (T *)h->mu;
            V.dinv = (T *)h->diag;
        } else if (D == 2 && H.Lg == L && (long long)nodes <= mg_block_nodes<T>()) {
            H.Lg = k;
        }
        // block-run levels keep their arrays in shared memory; the top one
        // still publishes its correction (xpost) for the grid level above
        const bool blk = k > 0 && H.Lg <= k;
        if (k > 0 && !blk) {
            PF_TRY(h->alloc(&V.lam, b));
            PF_TRY(h->alloc(&V.mu, b));
            PF_TRY(h->alloc(&V.dinv, b));
            for (int c = 0; c < D; c++) PF_TRY(h->alloc(&V.f[c], b));
        }
        for (int c = 0; c < D; c++) {
            PF_TRY(h->alloc(&V.xpost[c], b));
            if (blk) continue;
            PF_TRY(h->alloc(&V.xpre[c], b));
            for (int q = 0; q < 2; q++) {
                PF_TRY(h->alloc(&V.r[q][c], b));
                PF_TRY(h->alloc(&V.d[q][c], b));
            }
        }
        nx /= 2;
        ny /= 2;
        if (D == 3) nz /= 2;
    }
    for (int k = 0; k < L; k++) H.deg[k] = k == 0 ? MG_DEG_FINE : (k < H.Lg ? MG_DEG_GRID : MG_DEG_BLOCK);
    // Chebyshev iteration on [bmin, bmax]: d_0 = D^-1 r_0 / theta,
    // rho_j = 1 / (2 sigma - rho_{j-1}), d_j = rho_j rho_{j-1} d_{j-1} + 2 rho_j / delta D^-1 r_j
    const double bmax = 1.02 * element_bound(h->cfg.p.nu, D), bmin = bmax / 30.0;
    const double theta = 0.5 * (bmax + bmin), delta = 0.5 * (bmax - bmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    H.c1[0] = T(0);
    H.c2[0] = (T)(1.0 / theta);
    for (int j = 1; j < MG_MAX_STEPS; j++) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        H.c1[j] = (T)(rn * rho);
        H.c2[j] = (T)(2.0 * rn / delta);
        rho = rn;
    }
    // mixed method: the first refinement pass keeps b (FP64) for the later ones
    if (h->refine)
        for (int c = 0; c < D; c++) PF_TRY(h->alloc(&h->b64[c], sizeof(double) * (size_t)h->P.N));
    if (!h->d_mg) PF_TRY(h->alloc(&h->d_mg, sizeof(H)));
    return h->cuda(cudaMemcpy(h->d_mg, &H, sizeof(H), cudaMemcpyHostToDevice), "multigrid descriptor");
}

template <typename T, int D>
int setup_cg_launch(pf_handle *h)
{
    const bool fp64 = sizeof(T) == 8;
    h->mg = h->cfg.precond == PF_PC_MG || (h->cfg.precond == PF_PC_AUTO && auto_mg(h->cfg));
    // 2D: the V-cycle's coarse grid levels have few tiles, and the 32x16
    // tile (one 512-thread block per SM) halves the blocks in each of their
    // barriers; 3D: the 16x4x4 tile of the cell path
    h->pcg_shape = h->cfg.pcg_tile > 0 ? h->cfg.pcg_tile - 1
                                       : (h->mg ? (D == 2 ? mg2_pcg_shape(h->P.N, fp64) : 0)
                                                : default_pcg_shape(D, h->P.N, fp64));
    h->cg_block = h->pcg_shape ? tile_threads<D, 1>() : tile_threads<D, 0>();     // one thread per tile node
    if (h->mg) PF_TRY((build_mg<T, D>(h)));
    int per_sm = 0;
    cudaError_t e = D == 2 ? pcg2_occupancy(fp64, h->pcg_shape, h->mg, h->cg_block, &per_sm)
                           : pcg3_occupancy(fp64, h->pcg_shape, h->mg, h->cg_block, &per_sm);
    if (e != cudaSuccess) return h->cuda(e, "occupancy query");
    if (per_sm < 1) return h->fail(PF_ECUDA, "CG kernel cannot be resident");
    if (per_sm > 4) per_sm = 4;
    h->cg_per_sm = per_sm;
    return PF_OK;
}

template <typename T, int D>
PCGArgs<T, D> pcg_args(pf_handle *m)
{
    PCGArgs<T, D> A;
    memset(&A, 0, sizeof(A));
    A.P = m->P;
    A.lam = (const T *)m->lam; A.mu = (const T *)m->mu;
    for (int v = 0; v < 6; v++) A.sig[v] = (const T *)m->sig[v];
    for (int d = 0; d < 3; d++) {
        A.x[d] = (T *)(m->refine ? m->corr[d] : m->u[d]); A.p[d] = (T *)m->p[d];
        A.u[d] = (T *)m->u[d]; A.x64[d] = m->x64[d];
        for (int k = 0; k < 2; k++) { A.r[k][d] = (T *)m->r[k][d]; A.w[k][d] = (T *)m->w[k][d]; A.s[k][d] = (T *)m->s[k][d]; }
    }
    A.refine = m->refine ? 1 : 0;
    A.eta = 1e-3;
    A.dinv = (T *)m->diag;
    A.partials = m->partials;
    A.result = m->result;
    A.bar_count = m->sync; A.bar_gen = m->sync + SYNC_GEN;
    A.sc = m->sc; A.dg = m->dg;
    A.rtol = m->cfg.cg_rtol; A.maxit = m->cfg.cg_maxit;
    A.warm = m->cfg.warm_start != PF_WS_ZERO ? 1 : 0;
    A.mg = (const MGHier<T> *)m->d_mg;
    for (int d = 0; d < 3; d++) A.b64[d] = m->b64[d];
    return A;
}

template <typename T, int D>
size_t fused_smem()
{
    return sizeof(T) * FusedZ<D>::WORDS;
}

template <typename T, int D>
int prepare_fused(pf_handle *h)
{
    cudaError_t e = cudaFuncSetAttribute(k_fusedz<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_smem<T, D>());
    if (e == cudaSuccess && !h->fused_per_sm)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->fused_per_sm, k_fusedz<T, D>, 256, fused_smem<T, D>());
    return h->cuda(e, "fused kernel shared memory");
}

template <typename T, int D>
void launch_fused(int grid, const JobSet<CellJob<T, D>> &js, cudaStream_t s)
{
    k_fusedz<T, D><<<grid, 256, fused_smem<T, D>(), s>>>(js);
}

// Chunk length (planes along the marching axis) of the marching update for
// a grid with `cols` tile columns and nm planes, and its block count: the
// explicit length `fixed` if > 0, else the length that minimises (work items
// per block, rounded up) x (planes per item + w), w the start-up cost of a
// chunk in planes, with at most cap blocks.
int fused_chunk(long long cols, int nm, long long cap, int w, int fixed, int &nblocks)
{
    int best = fixed > 0 ? std::min(fixed, nm) : nm;
    if (fixed <= 0) {
        long long bcost = -1;
        for (int zc = 1; zc <= nm; zc++) {
            const long long items = cols * ((nm + zc - 1) / zc);
            const long long nb = std::min(items, cap);
            const long long cost = ((items + nb - 1) / nb) * (zc + w);
            if (bcost < 0 || cost < bcost) {
                bcost = cost;
                best = zc;
            }
        }
    }
    const long long items = cols * ((nm + best - 1) / best);
    nblocks = (int)std::max<long long>(1, std::min(items, cap));
    return best;
}

// Build the job tables of every instance: cell kernels get ~N/256 blocks per
// instance; the cooperative PCG launch splits the co-resident block capacity
// over the instances in proportion to their tile counts (at least one each).
template <typename T, int D>
int build_plan(pf_handle *h)
{
    PF_TRY((prepare_fused<T, D>(h)));
    std::vector<pf_handle *> I = instances(h);
    const int n = (int)I.size();
    std::vector<CellJob<T, D>> cj[2];
    cj[0].resize(n);
    cj[1].resize(n);
    int b0 = 0;
    for (int i = 0; i < n; i++) {
        pf_handle *m = I[i];
        const int nb = grid_for(m, m->P.N);
        for (int k = 0; k < 2; k++) {
            const int saved = m->cur;
            m->cur = saved ^ k;
            CellJob<T, D> &j = cj[k][i];
            memset(&j, 0, sizeof(j));
            j.P = m->P;
            j.K = cell_const<T>(m->P);
            j.F = field_ptrs<T, D>(m);
            m->cur = saved;
            j.sc = m->sc;
            j.partials = m->partials;
            j.counter = m->sync + SYNC_LAST;
            j.dg = m->dg;
            j.block0 = b0;
            j.nblocks = nb;
        }
        b0 += nb;
    }
    h->cell_grid = b0;
    h->njobs = n;
    // blocks of the marching update per instance: one wave of resident
    // blocks at most, each walking chunks of planes of its tile columns
    std::vector<CellJob<T, D>> fj[2] = {cj[0], cj[1]};
    int f0 = 0;
    for (int i = 0; i < n; i++) {
        const Params &P = I[i]->P;
        const long long cols = (long long)((P.nx + FusedZ<D>::TX - 1) / FusedZ<D>::TX) *
                               (D == 3 ? (P.ny + FusedZ<D>::TY - 1) / FusedZ<D>::TY : 1);
        const long long cap = (long long)h->sms * std::max(1, h->fused_per_sm);
        int nb = 1;
        const int zc = fused_chunk(cols, D == 3 ? P.nz : P.ny, cap, D == 3 ? FUSED_STARTUP_3D : FUSED_STARTUP_2D,
                                   I[i]->cfg.fused_chunk, nb);
        for (int k = 0; k < 2; k++) { fj[k][i].block0 = f0; fj[k][i].nblocks = nb; fj[k][i].strip_rows = zc; }
        f0 += nb;
    }
    h->fused_grid = f0;
    const size_t cbytes = sizeof(CellJob<T, D>) * (size_t)n;
    if (!h->d_cell_jobs[0]) {
        for (int k = 0; k < 2; k++) {
            PF_TRY(h->alloc(&h->d_cell_jobs[k], cbytes));
            PF_TRY(h->alloc(&h->d_fused_jobs[k], cbytes));
        }
    }
    for (int k = 0; k < 2; k++) {
        PF_TRY(h->cuda(cudaMemcpy(h->d_cell_jobs[k], cj[k].data(), cbytes, cudaMemcpyHostToDevice), "job table"));
        PF_TRY(h->cuda(cudaMemcpy(h->d_fused_jobs[k], fj[k].data(), cbytes, cudaMemcpyHostToDevice), "job table"));
    }
    if (h->cfg.mechanics) {
        const int TX = h->pcg_shape ? Tile<D, 1>::X : Tile<D, 0>::X;
        const int TY = h->pcg_shape ? Tile<D, 1>::Y : Tile<D, 0>::Y;
        const int TZ = h->pcg_shape ? Tile<D, 1>::Z : Tile<D, 0>::Z;
        // Jacobi-PCG iteration counts grow with the grid's linear size, so
        // an instance's work per solve is ~ tiles x linear size (MG: ~ tiles):
        // blocks are shared out in proportion to that, so that instances
        // finish together
        std::vector<long long> tiles(n);
        std::vector<double> work(n);
        double wtot = 0.0;
        for (int i = 0; i < n; i++) {
            const Params &P = I[i]->P;
            tiles[i] = (long long)((P.nx + TX - 1) / TX) * ((P.ny + TY - 1) / TY) * (D == 3 ? (P.nz + TZ - 1) / TZ : 1);
            const double lin = (double)std::max(P.nx, std::max(P.ny, D == 3 ? P.nz : 1));
            work[i] = (double)tiles[i] * (I[i]->mg ? 1.0 : lin);     // MG: iterations ~ independent of size
            wtot += work[i];
        }
        const long long cap = (long long)h->cg_per_sm * h->sms;
        if (cap < n) return h->fail(PF_EINVAL, "batch of %d instances exceeds the %lld co-resident CG blocks", n, cap);
        std::vector<PCGArgs<T, D>> pj(n);
        int g0 = 0;
        for (int i = 0; i < n; i++) {
            long long nb = 1 + (long long)((double)(cap - n) * work[i] / wtot);
            if (nb > tiles[i]) nb = tiles[i] > 0 ? tiles[i] : 1;
            pj[i] = pcg_args<T, D>(I[i]);
            pj[i].block0 = g0;
            pj[i].nblocks = (int)nb;
            g0 += (int)nb;
        }
        h->pcg_grid = g0;
        const size_t pbytes = sizeof(PCGArgs<T, D>) * (size_t)n;
        if (!h->d_pcg_jobs) PF_TRY(h->alloc(&h->d_pcg_jobs, pbytes));
        PF_TRY(h->cuda(cudaMemcpy(h->d_pcg_jobs, pj.data(), pbytes, cudaMemcpyHostToDevice), "job table"));
    }
    for (int k = 0; k < 2; k++) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        h->graph[k] = nullptr;
    }
    h->plan_par = 0;
    h->plan_ready = true;
    return PF_OK;
}

// Learned warm start of one instance: network inputs from the current state
// (W_f, W_g, prestress / |eig0|, dW_f/dt since the previous step), one
// inference y ~ du/dt / |eig0|, then the guess u += |eig0| dt y (not on the
// first step after pf_set_fields, which has no previous W_f).  The current
// state is theta[cur]: cur advances with the job-table parity, so a graph
// captured for one parity always replays with that parity's buffer.
template <typename T, int D>
int learned_guess(pf_handle *m, cudaStream_t s)
{
    const long long N = m->P.N;
    const int c = m->cur;
    const int g = grid_for(m, N);
    const double ae = std::fabs(m->P.eig0) > 0.0 ? std::fabs(m->P.eig0) : 1.0;
    k_net_input<T><<<g, 256, 0, s>>>(N, (const T *)m->theta[c], (const T *)m->phig, (float)(m->cfg.p.prestress / ae),
                                     (float)(1.0 / m->P.dt), m->net_mode, m->net_prev, m->net_in);
    const float *y = nullptr;
    const int rc = unet_forward_work(m->net, m->net_work, m->net_in, &y, s);
    if (rc != PF_OK) return m->fail(rc, "warm-start network: %s", unet_error(m->net));
    T *u[3] = {(T *)m->u[0], (T *)m->u[1], (T *)m->u[2]};
    k_net_guess<T, D><<<g, 256, 0, s>>>(N, y, m->net_mode, ae * m->P.dt, u[0], u[1], u[2],
                                        m->refine ? m->x64[0] : nullptr, m->refine ? m->x64[1] : nullptr,
                                        m->refine ? m->x64[2] : nullptr);
    k_net_mode_clear<<<1, 1, 0, s>>>(m->net_mode);
    return PF_OK;
}

// Queue the mechanics of one step of every instance (moduli and eigenstress,
// the initial guess, the solve, the return map); k selects the job tables
// (0: current state, 1: one step later).
template <typename T, int D>
int launch_mechanics(pf_handle *h, cudaStream_t s, int k)
{
    JobSet<CellJob<T, D>> cj;
    memset(&cj, 0, sizeof(cj));
    cj.table = (const CellJob<T, D> *)h->d_cell_jobs[k];
    cj.njobs = h->njobs;
    const int n = h->njobs;
    if (h->cfg.mechanics) {
        h->mark_begin(PF_K_SETUP, s);
        k_setup<T, D><<<h->cell_grid, 256, 0, s>>>(cj);
        h->mark_end(s);
        if (h->cfg.warm_start == PF_WS_EXTRAP || h->cfg.warm_start == PF_WS_EXTRAP2) {
            const int order = h->cfg.warm_start == PF_WS_EXTRAP2 ? 2 : 1;
            h->mark_begin(PF_K_WARM, s);
            for (pf_handle *m : instances(h)) {
                const long long N = m->P.N;
                T *u[3] = {(T *)m->u[0], (T *)m->u[1], (T *)m->u[2]};
                double *x[3] = {m->refine ? m->x64[0] : nullptr, m->refine ? m->x64[1] : nullptr,
                                m->refine ? m->x64[2] : nullptr};
                double *const *h0 = m->ext_hist[0], *const *h1 = m->ext_hist[1];
                k_extrap<T, D><<<grid_for(m, N), 256, 0, s>>>(N, m->ext_count, order, u[0], u[1], u[2], x[0], x[1],
                                                             x[2], h0[0], h0[1], h0[2], h1[0], h1[1], h1[2]);
                k_extrap_tail<<<1, 32, 0, s>>>(m->ext_count, order, reinterpret_cast<double *>(m->sc), m->ext_E,
                                               D == 2 ? 3 : 6);       // Scalars::E is the first member
            }
            h->mark_end(s);
        }
        if (h->cfg.warm_start == PF_WS_LEARNED) {
            h->mark_begin(PF_K_WARM, s);
            for (pf_handle *m : instances(h)) {
                if (!m->net) continue;
                PF_TRY((learned_guess<T, D>(m, s)));
            }
            h->mark_end(s);
        }
        h->mark_begin(PF_K_CG, s);
        const bool fp64 = sizeof(T) == 8;
        cudaError_t e = D == 2 ? pcg2_launch(fp64, h->pcg_shape, h->mg, h->d_pcg_jobs, n, h->pcg_grid, h->cg_block, s)
                               : pcg3_launch(fp64, h->pcg_shape, h->mg, h->d_pcg_jobs, n, h->pcg_grid, h->cg_block, s);
        h->mark_end(s);
        if (e != cudaSuccess) return h->cuda(e, "cooperative CG launch");
        h->mark_begin(PF_K_RETURN, s);
        k_return<T, D><<<h->cell_grid, 256, 0, s>>>(cj);
        h->mark_end(s);
    }
    return PF_OK;
}

// One explicit step from job tables [k]: the mechanics at the current state,
// then the fused field update.
template <typename T, int D>
int launch_step(pf_handle *h, cudaStream_t s, int k)
{
    PF_TRY((launch_mechanics<T, D>(h, s, k)));
    JobSet<CellJob<T, D>> fj;
    memset(&fj, 0, sizeof(fj));
    fj.njobs = h->njobs;
    fj.table = (const CellJob<T, D> *)h->d_fused_jobs[k];
    h->mark_begin(PF_K_UPDATE, s);
    launch_fused<T, D>(h->fused_grid, fj, s);
    h->mark_end(s);
    return h->cuda(cudaGetLastError(), "kernel launch");
}

void advance(pf_handle *h, int nsteps)
{
    for (pf_handle *m : instances(h)) {
        m->cur ^= (nsteps & 1);
        m->steps += nsteps;
        m->sigma_valid = true;
    }
    if (h->is_batch) h->steps += nsteps;
    h->plan_par ^= (nsteps & 1);
}

// Steps are replayed from CUDA graphs of one step, one per job-table parity
// (captured once per plan on the handle's stream), unless per-kernel timing
// is on; a graph that cannot be captured falls back to direct launches.
template <typename T, int D>
int run_steps(pf_handle *h, int nsteps, cudaStream_t s)
{
    if (!h->plan_ready) PF_TRY((build_plan<T, D>(h)));
    while (nsteps > 0) {
        const int k = h->plan_par;
        const bool graphable = h->use_graph && !h->prof_on && !h->graph_failed;
        if (graphable && !h->graph[k]) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal);
            int rc = PF_OK;
            pf_profile saved = h->prof;
            if (e == cudaSuccess) {
                rc = launch_step<T, D>(h, h->own, k);
                e = cudaStreamEndCapture(h->own, &g);
            }
            // launches recorded during capture are not executions
            h->prof = saved;
            if (e == cudaSuccess && rc == PF_OK && g) e = cudaGraphInstantiate(&h->graph[k], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess || rc != PF_OK || !h->graph[k]) {
                h->graph_failed = true;
                h->graph[k] = nullptr;
                cudaGetLastError();
                h->err.clear();
                continue;
            }
        }
        if (graphable && h->graph[k]) {
            PF_TRY(h->cuda(cudaGraphLaunch(h->graph[k], s), "graph launch"));
            // one launch per kernel class of the step, whatever the batch size
            const int cls[4] = {PF_K_UPDATE, PF_K_SETUP, PF_K_CG, PF_K_RETURN};
            const int per = h->cfg.mechanics ? 4 : 1;
            if (h->cfg.mechanics && h->cfg.warm_start == PF_WS_LEARNED) h->prof.count[PF_K_WARM] += 1;
            h->prof.launches += per;
            for (int c = 0; c < per; c++) h->prof.count[cls[c]] += 1;
            h->prof.graph_steps += 1;
        } else {
            PF_TRY((launch_step<T, D>(h, s, k)));
        }
        advance(h, 1);
        nsteps -= 1;
    }
    return PF_OK;
}

template <typename T>
int set_fields_t(pf_handle *h, const pf_fields *f, int where, cudaStream_t s)
{
    const long long N = h->P.N;
    // the state goes into the current parity's buffers: the step plan (job
    // tables and captured graphs, laid out relative to that parity) stays
    const int c0 = h->cur;
    const int D = h->cfg.ndim, NP = D == 2 ? 4 : 6, NV = D == 2 ? 3 : 6;
    const int g = grid_for(h, N);
    const size_t nb = sizeof(double) * (size_t)N;
    auto src = [&](const double *ptr, size_t bytes_, double *stage) -> const double * {
        if (!ptr) return nullptr;
        if (where == PF_DEVICE) return ptr;
        if (cudaMemcpyAsync(stage, ptr, bytes_, cudaMemcpyHostToDevice, s) != cudaSuccess) return (const double *)-1;
        return stage;
    };
#define PF_SRC(var, ptr, bytes_, stg) const double *var = src(ptr, bytes_, stg); if (var == (const double *)-1) return h->fail(PF_ECUDA, "host-to-device copy failed");
    {
        PF_SRC(pf, f->phi_f, nb, h->stage);
        PF_SRC(pw, f->phi_w, nb, h->stage2);
        k_in_phase<T><<<g, 256, 0, s>>>(N, pf, pw, (T *)h->theta[c0], (T *)h->phig);
    }
    if (f->theta) {
        // the order parameter itself (exact restore, also where phi_g = 1)
        PF_SRC(a, f->theta, nb, h->stage);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, a, (T *)h->theta[c0], 0.0);
    }
    if (f->phi_g) {
        PF_SRC(a, f->phi_g, nb, h->stage2);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, a, (T *)h->phig, 0.0);
    }
    {
        PF_SRC(a, f->x_O, nb, h->stage);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, a, (T *)h->xO[c0], 0.0);
        PF_SRC(b, f->x_H, nb, h->stage2);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, b, (T *)h->xH[c0], 0.0);
    }
    {
        PF_SRC(a, f->x_H2O, nb, h->stage);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, a, (T *)h->xW[c0], 0.0);
        PF_SRC(b, f->mobility, nb, h->stage2);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, b, (T *)h->mob, 1.0);
    }
    {
        PF_SRC(a, f->alpha, nb, h->stage);
        k_in_scalar<T><<<g, 256, 0, s>>>(N, a, (T *)h->alpha, 0.0);
    }
    // component arrays through the device pointer table
    void *tab[6];
    {
        for (int d = 0; d < 3; d++) tab[d] = h->u[d];
        PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
        PF_SRC(a, f->u, nb * D, h->stage);
        // a displacement equal to the handle's own, bit for bit as
        // pf_get_fields exports it (a state round trip), keeps the
        // extrapolation history and the FP64 copy of the solve
        // (the mixed form exports its FP64 copy)
        if (h->u_changed) {
            PF_TRY(h->cuda(cudaMemsetAsync(h->u_changed, 0, sizeof(int), s), "round-trip flag"));
            if (h->refine) {
                void *t64[6] = {};
                for (int d = 0; d < D; d++) t64[d] = h->x64[d];
                PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, t64, sizeof(t64), cudaMemcpyHostToDevice, s), "pointer table"));
                k_comp_differs<double><<<g, 256, 0, s>>>(N, D, a, (double *const *)h->ptrtab, h->u_changed);
                PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
            } else {
                k_comp_differs<T><<<g, 256, 0, s>>>(N, D, a, (T *const *)h->ptrtab, h->u_changed);
            }
        }
        k_in_comp_if<T><<<g, 256, 0, s>>>(N, D, a, (T *const *)h->ptrtab, h->u_changed);
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "set_fields sync"));
        if (h->refine) {
            for (int d = 0; d < 3; d++) tab[d] = h->x64[d];
            PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
            k_in_comp_if<double><<<g, 256, 0, s>>>(N, D, a, (double *const *)h->ptrtab, h->u_changed);
            PF_TRY(h->cuda(cudaStreamSynchronize(s), "set_fields sync"));
        }
    }
    {
        for (int v = 0; v < 6; v++) tab[v] = h->ep[v];
        PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
        PF_SRC(a, f->eps_p, nb * NP, h->stage);
        k_in_comp<T><<<g, 256, 0, s>>>(N, NP, a, (T *const *)h->ptrtab);
    }
    if (f->dirichlet) {
        PF_TRY(h->cuda(cudaMemcpyAsync(h->mask, f->dirichlet, (size_t)N, where == PF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s), "mask copy"));
    } else {
        PF_TRY(h->cuda(cudaMemsetAsync(h->mask, 0, (size_t)N, s), "mask clear"));
    }
    // scalars: mean strain, diagnostics
    Scalars sc;
    memset(&sc, 0, sizeof(sc));
    if (f->Ebar) {
        if (where == PF_DEVICE) {
            PF_TRY(h->cuda(cudaMemcpyAsync(sc.E, f->Ebar, sizeof(double) * NV, cudaMemcpyDeviceToHost, s), "Ebar copy"));
            PF_TRY(h->cuda(cudaStreamSynchronize(s), "Ebar sync"));
        } else {
            memcpy(sc.E, f->Ebar, sizeof(double) * NV);
        }
    }
    PF_TRY(h->cuda(cudaMemcpyAsync(h->sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, s), "scalars"));
    Diag dg;
    memset(&dg, 0, sizeof(dg));
    PF_TRY(h->cuda(cudaMemcpyAsync(h->dg, &dg, sizeof(dg), cudaMemcpyHostToDevice, s), "diag"));
    PF_TRY(h->cuda(cudaMemsetAsync(h->sync, 0, sizeof(unsigned int) * SYNC_WORDS, s), "sync words"));
    PF_TRY(h->cuda(cudaMemsetAsync(h->trE, 0, h->tsz * (size_t)N, s), "coupling"));
    PF_TRY(h->cuda(cudaMemsetAsync(h->devE2, 0, h->tsz * (size_t)N, s), "coupling"));
    // reference oxygen content
    const int gs = grid_for(h, N);
    k_sum<T><<<gs, 256, 0, s>>>(N, (const T *)h->xO[c0], h->partials);
    std::vector<double> part((size_t)gs * PSTRIDE);
    PF_TRY(h->cuda(cudaMemcpyAsync(part.data(), h->partials, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s), "partials"));
    PF_TRY(h->cuda(cudaStreamSynchronize(s), "set_fields sync"));
    double s0 = 0.0;
    for (int b = 0; b < gs; b++) s0 += part[(size_t)b * PSTRIDE];
    h->sumO0 = s0;
    h->steps = 0;
    h->cg_total_seen = 0;
    h->have_fields = true;
    h->sigma_valid = false;
    if (h->net_mode) {
        static const int first = 1;
        PF_TRY(h->cuda(cudaMemcpyAsync(h->net_mode, &first, sizeof(int), cudaMemcpyHostToDevice, s), "net mode"));
    }
    if (h->ext_count) k_ext_restart<<<1, 1, 0, s>>>(h->u_changed, h->ext_count);
    return h->cuda(cudaGetLastError(), "set_fields kernels");
#undef PF_SRC
}

template <typename T>
int get_fields_t(pf_handle *h, pf_fields *f, int where, cudaStream_t s)
{
    const long long N = h->P.N;
    const int D = h->cfg.ndim, NP = D == 2 ? 4 : 6, NV = D == 2 ? 3 : 6;
    const int g = grid_for(h, N);
    const size_t nb = sizeof(double) * (size_t)N;
    const int c = h->cur;
    auto finish = [&](double *dst, double *stage, size_t bytes_) -> int {
        if (where == PF_DEVICE) return PF_OK;
        return h->cuda(cudaMemcpyAsync(dst, stage, bytes_, cudaMemcpyDeviceToHost, s), "device-to-host copy");
    };
    auto out = [&](double *dst, double *stage) -> double * { return where == PF_DEVICE ? dst : stage; };
    if (f->phi_f || f->phi_w) {
        double *a = f->phi_f ? out(f->phi_f, h->stage) : nullptr;
        double *b = f->phi_w ? out(f->phi_w, h->stage2) : nullptr;
        k_out_phase<T><<<g, 256, 0, s>>>(N, (const T *)h->theta[c], (const T *)h->phig, a, b);
        if (f->phi_f) PF_TRY(finish(f->phi_f, h->stage, nb));
        if (f->phi_w) PF_TRY(finish(f->phi_w, h->stage2, nb));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "get sync"));
    }
    struct One { double *dst; const void *src; };
    One ones[6] = {{f->x_O, h->xO[c]}, {f->x_H, h->xH[c]}, {f->x_H2O, h->xW[c]}, {f->alpha, h->alpha},
                   {f->theta, h->theta[c]}, {f->phi_g, h->phig}};
    for (auto &o : ones) {
        if (!o.dst) continue;
        k_out_scalar<T><<<g, 256, 0, s>>>(N, (const T *)o.src, out(o.dst, h->stage));
        PF_TRY(finish(o.dst, h->stage, nb));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "get sync"));
    }
    struct Comp { double *dst; void *const *src; int n; };
    Comp comps[3] = {{f->u, h->u, D}, {f->eps_p, h->ep, NP}, {f->sigma, h->sigma, NP}};
    if (f->u && h->refine) {
        // mixed mode keeps the displacement in FP64
        void *tab[6] = {};
        for (int k = 0; k < D; k++) tab[k] = h->x64[k];
        PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
        k_out_comp<double><<<g, 256, 0, s>>>(N, D, (double *const *)h->ptrtab, out(f->u, h->stage));
        PF_TRY(finish(f->u, h->stage, nb * D));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "get sync"));
        comps[0].dst = nullptr;
    }
    for (auto &o : comps) {
        if (!o.dst) continue;
        void *tab[6] = {};
        for (int k = 0; k < o.n; k++) tab[k] = o.src[k];
        PF_TRY(h->cuda(cudaMemcpyAsync(h->ptrtab, tab, sizeof(tab), cudaMemcpyHostToDevice, s), "pointer table"));
        k_out_comp<T><<<g, 256, 0, s>>>(N, o.n, (T *const *)h->ptrtab, out(o.dst, h->stage));
        PF_TRY(finish(o.dst, h->stage, nb * o.n));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "get sync"));
    }
    if (f->Ebar) {
        Scalars sc;
        PF_TRY(h->cuda(cudaMemcpyAsync(&sc, h->sc, sizeof(sc), cudaMemcpyDeviceToHost, s), "scalars"));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "get sync"));
        if (where == PF_DEVICE) {
            PF_TRY(h->cuda(cudaMemcpy(f->Ebar, sc.E, sizeof(double) * NV, cudaMemcpyHostToDevice), "Ebar"));
        } else {
            memcpy(f->Ebar, sc.E, sizeof(double) * NV);
        }
    }
    return h->cuda(cudaGetLastError(), "get_fields kernels");
}

template <typename T>
int alloc_fields(pf_handle *h)
{
    const long long N = h->P.N;
    const int D = h->cfg.ndim, NP = D == 2 ? 4 : 6, NV = D == 2 ? 3 : 6;
    const size_t b = sizeof(T) * (size_t)N;
    for (int k = 0; k < 2; k++) {
        PF_TRY(h->alloc(&h->theta[k], b)); PF_TRY(h->alloc(&h->xO[k], b));
        PF_TRY(h->alloc(&h->xH[k], b)); PF_TRY(h->alloc(&h->xW[k], b));
    }
    PF_TRY(h->alloc(&h->phig, b)); PF_TRY(h->alloc(&h->mob, b));
    PF_TRY(h->alloc(&h->muO, b)); PF_TRY(h->alloc(&h->MO, b));
    PF_TRY(h->alloc(&h->trE, b)); PF_TRY(h->alloc(&h->devE2, b));
    PF_TRY(h->alloc(&h->mask, (size_t)N));
    if (h->cfg.mechanics) {
        PF_TRY(h->alloc(&h->lam, b)); PF_TRY(h->alloc(&h->mu, b));
        for (int v = 0; v < NV; v++) PF_TRY(h->alloc(&h->sig[v], b));
        for (int d = 0; d < D; d++) {
            PF_TRY(h->alloc(&h->p[d], b));
            for (int k = 0; k < 2; k++) {
                PF_TRY(h->alloc(&h->r[k][d], b)); PF_TRY(h->alloc(&h->w[k][d], b)); PF_TRY(h->alloc(&h->s[k][d], b));
            }
        }
        PF_TRY(h->alloc(&h->result, sizeof(double) * 32));
        PF_TRY(h->alloc(&h->diag, b));
        if (h->cfg.warm_start == PF_WS_EXTRAP || h->cfg.warm_start == PF_WS_EXTRAP2) {
            const int nh = h->cfg.warm_start == PF_WS_EXTRAP2 ? 2 : 1;
            for (int k = 0; k < nh; k++)
                for (int d = 0; d < D; d++) PF_TRY(h->alloc(&h->ext_hist[k][d], sizeof(double) * (size_t)N));
            PF_TRY(h->alloc(&h->ext_E, sizeof(double) * 12));
            PF_TRY(h->alloc(&h->ext_count, sizeof(int)));
            PF_TRY(h->cuda(cudaMemset(h->ext_count, 0, sizeof(int)), "extrapolation count"));
            PF_TRY(h->alloc(&h->u_changed, sizeof(int)));
        }
        if (!h->fp64) {
            h->refine = true;
            for (int d = 0; d < D; d++) {
                PF_TRY(h->alloc(&h->corr[d], b));
                PF_TRY(h->alloc(&h->x64[d], sizeof(double) * (size_t)N));
            }
        }
    }
    for (int d = 0; d < D; d++) PF_TRY(h->alloc(&h->u[d], b));
    for (int v = 0; v < NP; v++) { PF_TRY(h->alloc(&h->ep[v], b)); PF_TRY(h->alloc(&h->sigma[v], b)); }
    PF_TRY(h->alloc(&h->alpha, b));
    const size_t stage = sizeof(double) * (size_t)N * (size_t)(NP > D ? NP : D);
    PF_TRY(h->alloc(&h->stage, stage));
    PF_TRY(h->alloc(&h->stage2, sizeof(double) * (size_t)N));
    h->npart = h->sms * 16 > 4096 ? h->sms * 16 : 4096;
    PF_TRY(h->alloc(&h->partials, sizeof(double) * PSTRIDE * (size_t)h->npart));
    PF_TRY(h->alloc(&h->sync, sizeof(unsigned int) * SYNC_WORDS));
    PF_TRY(h->alloc(&h->sc, sizeof(Scalars)));
    PF_TRY(h->alloc(&h->dg, sizeof(Diag)));
    PF_TRY(h->alloc(&h->ptrtab, sizeof(void *) * 6));
    PF_TRY(h->cuda(cudaMemset(h->sync, 0, sizeof(unsigned int) * SYNC_WORDS), "sync init"));
    for (int v = 0; v < NP; v++) PF_TRY(h->cuda(cudaMemset(h->sigma[v], 0, b), "sigma init"));
    return PF_OK;
}

void free_all(pf_handle *h)
{
    for (int k = 0; k < 2; k++) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        h->graph[k] = nullptr;
    }
    for (pf_handle *m : h->members) {
        free_all(m);
        delete m;
    }
    h->members.clear();
    unet_work_destroy(h->net_work);
    h->net_work = nullptr;
    for (void *p : h->net_allocs) cudaFree(p);
    h->net_allocs.clear();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->own) cudaStreamDestroy(h->own);
    h->own = nullptr;
}

// Validate a configuration and create one instance (device arrays, stream,
// CG launch shape).  On failure *out stays null and err says why.
int create_one(const pf_config *cfg, pf_handle **out, std::string &err)
{
    if (!cfg) { err = "cfg is NULL"; return PF_EINVAL; }
    const pf_config &c = *cfg;
    if (c.ndim != 2 && c.ndim != 3) { err = "ndim must be 2 or 3"; return PF_EINVAL; }
    if (c.nx < 2 || c.ny < 2 || (c.ndim == 3 && c.nz < 2)) { err = "grid sizes must be >= 2"; return PF_EINVAL; }
    if (c.precision != PF_FP64 && c.precision != PF_MIXED) { err = "precision must be PF_FP64 or PF_MIXED"; return PF_EINVAL; }
    if (c.warm_start != PF_WS_ZERO && c.warm_start != PF_WS_PREV && c.warm_start != PF_WS_LEARNED &&
        c.warm_start != PF_WS_EXTRAP && c.warm_start != PF_WS_EXTRAP2) {
        err = "warm_start must be PF_WS_ZERO, PF_WS_PREV or PF_WS_LEARNED";
        return PF_EINVAL;
    }
    if (c.mechanics && (c.cg_maxit <= 0 || !(c.cg_rtol > 0.0))) { err = "cg_maxit must be > 0 and cg_rtol > 0"; return PF_EINVAL; }
    if (c.pcg_tile < 0 || c.pcg_tile > PCG_SHAPES) { err = "pcg_tile must be 0 (library choice), 1 or 2"; return PF_EINVAL; }
    if (c.fused_chunk < 0) { err = "fused_chunk must be >= 0 (0: library choice)"; return PF_EINVAL; }
    if (c.precond != PF_PC_AUTO && c.precond != PF_PC_JACOBI && c.precond != PF_PC_MG) {
        err = "precond must be PF_PC_AUTO, PF_PC_JACOBI or PF_PC_MG";
        return PF_EINVAL;
    }
    if (!(c.p.nu > -1.0 && c.p.nu < 0.5) || !(c.p.E_s > 0.0) || !(c.p.E_g_ratio > 0.0)) { err = "elastic constants out of range"; return PF_EINVAL; }
    const long long N = (long long)c.nx * c.ny * (c.ndim == 3 ? c.nz : 1);
    if (N > (1LL << 31)) { err = "grid too large (more than 2^31 cells)"; return PF_EINVAL; }

    pf_handle *h = new (std::nothrow) pf_handle();
    if (!h) { err = "host allocation failed"; return PF_ENOMEM; }
    h->cfg = c;
    memset(&h->prof, 0, sizeof(h->prof));
    if (c.ndim == 2) h->cfg.nz = 1;
    h->fp64 = c.precision == PF_FP64;
    h->tsz = h->fp64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaGetDevice(&h->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        err = std::string("CUDA unavailable: ") + cudaGetErrorString(e);
        delete h;
        return PF_ECUDA;
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev);
    if (!coop) { err = "device lacks cooperative launch"; free_all(h); delete h; return PF_ECUDA; }
    if (!upload_tables(h->dev)) { err = "constant table upload failed"; free_all(h); delete h; return PF_ECUDA; }

    fill_params(h->cfg, N, h->P);

    int rc = h->fp64 ? alloc_fields<double>(h) : alloc_fields<float>(h);
    if (rc == PF_OK && c.mechanics) {
        if (c.ndim == 2) rc = h->fp64 ? setup_cg_launch<double, 2>(h) : setup_cg_launch<float, 2>(h);
        else rc = h->fp64 ? setup_cg_launch<double, 3>(h) : setup_cg_launch<float, 3>(h);
    }
    if (rc != PF_OK) {
        err = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return PF_OK;
}


// ---------------------------------------------------------------------------
// Backward-Euler steps of the field relations (pf_step_implicit): the
// mechanics of the explicit step at y_n, then Newton's method on
// F(y) = y - y_n - dt R(y) with matrix-free GMRES (pf_implicit.cuh).
// ---------------------------------------------------------------------------
constexpr int BE_NDOT = 256;   // blocks of the dot-product kernel
constexpr int BE_MAX_RESTART = 60;
// partial sums: the dot products of up to BE_MAX_RESTART + 1 vectors, or the
// five balance sums of up to 16 blocks per SM on 152 SMs and more
constexpr size_t BE_NPART = (size_t)BE_NDOT * 65;

struct BEWork {
    long long N, L;
    int m;
    double *y, *y0, *F0, *Ft, *t, *der, *z, *r, *d, *q, *dg, *x, *u, *V;
    double *part, *hvec;
    unsigned long long *mx;    // [0] max |F|, [2..3] max |delta|, max |y|, [4..7] Gershgorin s per block
    BEPc32 pc32;               // the FP32 preconditioner's arrays (24 N floats)
};

int be_work(pf_handle *h, int m, BEWork &w)
{
    const long long N = h->P.N, L = 4 * N;
    const size_t nvec = 14 + (size_t)(m + 1) + 3;     // the last 3: 24 N floats of the FP32 preconditioner
    const size_t len = nvec * (size_t)L + BE_NPART + 64 + 8;
    if (h->be_len < len) {
        PF_TRY(h->alloc(&h->be_ws, sizeof(double) * len));
        h->be_len = len;
    }
    double *p = h->be_ws;
    w.N = N; w.L = L; w.m = m;
    double **vec[14] = {&w.y, &w.y0, &w.F0, &w.Ft, &w.t, &w.der, &w.z, &w.r, &w.d, &w.q, &w.dg, &w.x, &w.u, &w.V};
    for (int k = 0; k < 14; k++) { *vec[k] = p; p += L; }
    p += (size_t)m * L;                       // V holds m + 1 vectors
    float *f = reinterpret_cast<float *>(p);
    p += 3 * (size_t)L;
    float **fv[9] = {&w.pc32.cth, &w.pc32.DO, &w.pc32.DH, &w.pc32.DW, &w.pc32.dginv, &w.pc32.z, &w.pc32.r,
                     &w.pc32.d0, &w.pc32.d1};
    const long long flen[9] = {N, N, N, N, L, L, L, L, L};
    for (int k = 0; k < 9; k++) { *fv[k] = f; f += flen[k]; }
    w.part = p; p += BE_NPART;
    w.hvec = p; p += 64;
    w.mx = reinterpret_cast<unsigned long long *>(p);
    return PF_OK;
}

template <int D>
int be_steps(pf_handle *h, int nsteps, const pf_implicit_opts &o, pf_implicit_stats &st, cudaStream_t s)
{
    if (!h->plan_ready) PF_TRY((build_plan<double, D>(h)));
    const int m = o.gmres_restart, K = o.pc_degree;
    BEWork w;
    PF_TRY(be_work(h, m, w));
    const long long N = w.N, L = w.L;
    const int gN = grid_for(h, N), gL = grid_for(h, L);
    BEArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = h->P.nx; a.ny = h->P.ny; a.nz = D == 3 ? h->P.nz : 1; a.N = N; a.dt = o.dt;
    a.K = cell_const<double>(h->P);
    a.phig = (const double *)h->phig; a.mob = (const double *)h->mob;
    a.trE = (const double *)h->trE; a.devE2 = (const double *)h->devE2; a.mask = h->mask;
    std::vector<double> hp((size_t)BE_NDOT * (m + 1));
    auto check = [&](const char *what) { return h->cuda(cudaGetLastError(), what); };
    // dot products of w with nv vectors starting at V (fixed summation order)
    auto dots = [&](const double *Vb, int nv, const double *vw, double *res) -> int {
        k_be_dots<<<dim3(BE_NDOT, nv), 256, 0, s>>>(L, Vb, nv, vw, w.part);
        PF_TRY(h->cuda(cudaMemcpyAsync(hp.data(), w.part, sizeof(double) * BE_NDOT * nv, cudaMemcpyDeviceToHost, s),
                       "dot products"));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "dot products"));
        for (int k = 0; k < nv; k++) {
            double t = 0.0;
            for (int b = 0; b < BE_NDOT; b++) t += hp[(size_t)k * BE_NDOT + b];
            res[k] = t;
        }
        return PF_OK;
    };
    auto comb = [&](const double *Vb, int nv, const double *c, double *out) -> int {
        PF_TRY(h->cuda(cudaMemcpyAsync(w.hvec, c, sizeof(double) * nv, cudaMemcpyHostToDevice, s), "coefficients"));
        k_be_comb<<<gL, 256, 0, s>>>(L, Vb, nv, w.hvec, out);
        return check("combination");
    };
    auto read_max = [&](int k0, int n, double *out) -> int {
        unsigned long long v[8];
        PF_TRY(h->cuda(cudaMemcpyAsync(v, w.mx + k0, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s), "max"));
        PF_TRY(h->cuda(cudaStreamSynchronize(s), "max"));
        for (int k = 0; k < n; k++) {
            const long long b = (long long)v[k];
            memcpy(&out[k], &b, sizeof(double));
        }
        return PF_OK;
    };
    // F(yy) into out, max |F| into mx[0]
    auto Fval = [&](const double *yy, double *out) -> int {
        PF_TRY(h->cuda(cudaMemsetAsync(w.mx, 0, sizeof(unsigned long long), s), "max"));
        k_be_derive<D><<<gN, 256, 0, s>>>(a, yy, w.der);
        k_be_rates<D><<<gN, 256, 0, s>>>(a, yy, w.y0, w.der, out, 0, w.mx);
        return check("residual");
    };
    // Chebyshev coefficients of the block preconditioner
    std::vector<BECheb> cheb;
    BECheb cinit;
    std::vector<BECheb32> cheb32;
    BECheb32 cinit32;
    const bool pc32 = o.pc_precision == PF_MIXED;
    auto precond = [&](const double *v, double *zo) -> int {
        if (K == 0) return h->cuda(cudaMemcpyAsync(zo, v, sizeof(double) * L, cudaMemcpyDeviceToDevice, s), "copy");
        if (pc32) {
            const int n32 = (int)N;
            k_be_pc32_init<<<gN, 256, 0, s>>>(n32, v, w.pc32, cinit32);
            float *din = w.pc32.d0, *dout = w.pc32.d1;
            for (int k = 0; k + 1 < K; k++) {
                k_be_pc32_step<D><<<gN, 256, 0, s>>>(a.nx, a.ny, a.nz, n32, (float)a.dt, a.mask, w.pc32, din, dout,
                                                     cheb32[k]);
                std::swap(din, dout);
            }
            k_be_pc32_final<<<gN, 256, 0, s>>>(n32, w.pc32, din, zo);
            return check("preconditioner");
        }
        k_be_pc_init<<<gL, 256, 0, s>>>(N, v, w.dg, zo, w.r, w.d, cinit);
        for (int k = 0; k + 1 < K; k++) {
            k_be_pc_apply<D><<<gN, 256, 0, s>>>(a, w.der, w.d, w.q);
            k_be_pc_step<<<gL, 256, 0, s>>>(N, w.q, w.dg, zo, w.r, w.d, cheb[k], 0);
        }
        k_be_pc_step<<<gL, 256, 0, s>>>(N, w.q, w.dg, zo, w.r, w.d, cinit, 1);
        return check("preconditioner");
    };
    // J zz: the directional derivative of F at y, in forward mode
    auto jvp = [&](const double *zz, double *out) -> int {
        k_be_jderive<D><<<gN, 256, 0, s>>>(a, w.y, zz, w.t, w.Ft);
        k_be_jvp<D><<<gN, 256, 0, s>>>(a, w.y, zz, w.t, w.Ft, out);
        return check("jvp");
    };

    st.newton_iters = 0;
    for (int step = 0; step < nsteps; step++) {
        // mechanics at y_n (staggered, as in the explicit step)
        PF_TRY((launch_mechanics<double, D>(h, s, h->plan_par)));
        const int c = h->cur;
        k_be_gather<<<gN, 256, 0, s>>>(N, (const double *)h->theta[c], (const double *)h->xO[c],
                                        (const double *)h->xH[c], (const double *)h->xW[c], w.y0);
        k_be_init<<<gN, 256, 0, s>>>(a, w.y0, w.y);
        // the preconditioner's blocks depend on phi_g and the mobility only
        PF_TRY(h->cuda(cudaMemsetAsync(w.mx + 4, 0, 4 * sizeof(unsigned long long), s), "bounds"));
        k_be_derive<D><<<gN, 256, 0, s>>>(a, w.y, w.der);
        k_be_pc_diag<D><<<gN, 256, 0, s>>>(a, w.der, w.dg, w.mx + 4);
        PF_TRY(check("preconditioner set-up"));
        double sb[4];
        PF_TRY(read_max(4, 4, sb));
        cheb.assign(K > 0 ? K : 1, BECheb{});
        {
            double sig1[4], rho0[4];
            for (int b = 0; b < 4; b++) {
                const double del = std::max(sb[b], 1e-12);
                sig1[b] = 1.0 / del;               // theta = 1
                rho0[b] = 1.0 / sig1[b];
                cinit.c1[b] = 0.0;
                cinit.c2[b] = 1.0;                 // d_0 = D^-1 r_0 / theta
            }
            for (int k = 0; k + 1 < K; k++)
                for (int b = 0; b < 4; b++) {
                    const double del = std::max(sb[b], 1e-12);
                    const double rho1 = 1.0 / (2.0 * sig1[b] - rho0[b]);
                    cheb[k].c1[b] = rho1 * rho0[b];
                    cheb[k].c2[b] = 2.0 * rho1 / del;
                    rho0[b] = rho1;
                }
            cheb32.assign(cheb.size(), BECheb32{});
            for (size_t k = 0; k < cheb.size(); k++)
                for (int b = 0; b < 4; b++) {
                    cheb32[k].c1[b] = (float)cheb[k].c1[b];
                    cheb32[k].c2[b] = (float)cheb[k].c2[b];
                }
            for (int b = 0; b < 4; b++) {
                cinit32.c1[b] = (float)cinit.c1[b];
                cinit32.c2[b] = (float)cinit.c2[b];
            }
        }
        if (pc32 && K > 0) k_be_pc32_pack<<<gN, 256, 0, s>>>(a, w.der, w.dg, w.pc32);
        PF_TRY(Fval(w.y, w.F0));
        double fmax;
        PF_TRY(read_max(0, 1, &fmax));
        // the update rule counts only after a linear solve that met its
        // target (a stalled GMRES also gives small updates)
        double moved = INFINITY, ymax = 0.0;
        bool solved = false;
        int it = 0;
        bool conv = false;
        for (;; it++) {
            if (fmax <= o.newton_tol || (solved && moved <= o.newton_tol * std::max(1.0, ymax))) {
                conv = true;
                break;
            }
            if (it == o.newton_maxit) break;
            // GMRES(m) on J delta = F0, right preconditioned, from delta = 0
            PF_TRY(h->cuda(cudaMemsetAsync(w.x, 0, sizeof(double) * L, s), "gmres"));
            double beta;
            PF_TRY(dots(w.F0, 1, w.F0, &beta));
            beta = sqrt(beta);
            const double target = o.gmres_rtol * beta;
            int inner = 0;
            bool first = true;
            while (beta > target && inner < o.gmres_maxit) {
                if (first) {
                    k_be_axpby<<<gL, 256, 0, s>>>(L, 1.0 / beta, w.F0, 0.0, w.F0, w.V);
                } else {
                    // r = F0 - J x
                    PF_TRY(jvp(w.x, w.u));
                    k_be_axpby<<<gL, 256, 0, s>>>(L, 1.0, w.F0, -1.0, w.u, w.u);
                    double b2;
                    PF_TRY(dots(w.u, 1, w.u, &b2));
                    beta = sqrt(b2);
                    if (beta <= target) break;
                    k_be_axpby<<<gL, 256, 0, s>>>(L, 1.0 / beta, w.u, 0.0, w.u, w.V);
                }
                first = false;
                std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
                g[0] = beta;
                int j = 0;
                double res = beta;
                for (; j < m && inner < o.gmres_maxit;) {
                    double *vj = w.V + (size_t)j * L, *vn = w.V + (size_t)(j + 1) * L;
                    PF_TRY(precond(vj, w.z));
                    PF_TRY(jvp(w.z, vn));
                    // classical Gram-Schmidt, twice
                    double hc[64], h2[64], nh[64];
                    PF_TRY(dots(w.V, j + 1, vn, hc));
                    for (int k = 0; k <= j; k++) nh[k] = -hc[k];
                    PF_TRY(comb(w.V, j + 1, nh, vn));
                    PF_TRY(dots(w.V, j + 1, vn, h2));
                    for (int k = 0; k <= j; k++) { nh[k] = -h2[k]; hc[k] += h2[k]; }
                    PF_TRY(comb(w.V, j + 1, nh, vn));
                    double hn;
                    PF_TRY(dots(vn, 1, vn, &hn));
                    hn = sqrt(hn);
                    for (int k = 0; k <= j; k++) H[(size_t)k * m + j] = hc[k];
                    H[(size_t)(j + 1) * m + j] = hn;
                    if (hn > 0.0) k_be_axpby<<<gL, 256, 0, s>>>(L, 1.0 / hn, vn, 0.0, vn, vn);
                    // Givens rotations of column j
                    for (int k = 0; k < j; k++) {
                        const double a0 = H[(size_t)k * m + j], a1 = H[(size_t)(k + 1) * m + j];
                        H[(size_t)k * m + j] = cs[k] * a0 + sn[k] * a1;
                        H[(size_t)(k + 1) * m + j] = -sn[k] * a0 + cs[k] * a1;
                    }
                    const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
                    const double rr = hypot(a0, a1);
                    cs[j] = rr > 0.0 ? a0 / rr : 1.0;
                    sn[j] = rr > 0.0 ? a1 / rr : 0.0;
                    H[(size_t)j * m + j] = rr;
                    H[(size_t)(j + 1) * m + j] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    res = fabs(g[j + 1]);
                    j++;
                    inner++;
                    if (res <= target || hn == 0.0) break;
                }
                // x += M^-1 V y, H y = g (upper triangular, j x j)
                std::vector<double> yv(j, 0.0);
                for (int k = j - 1; k >= 0; k--) {
                    double t = g[k];
                    for (int l = k + 1; l < j; l++) t -= H[(size_t)k * m + l] * yv[l];
                    yv[k] = H[(size_t)k * m + k] != 0.0 ? t / H[(size_t)k * m + k] : 0.0;
                }
                PF_TRY(h->cuda(cudaMemsetAsync(w.u, 0, sizeof(double) * L, s), "gmres"));
                if (j > 0) PF_TRY(comb(w.V, j, yv.data(), w.u));
                PF_TRY(precond(w.u, w.z));
                k_be_axpby<<<gL, 256, 0, s>>>(L, 1.0, w.x, 1.0, w.z, w.x);
                beta = res;
            }
            st.gmres_iters += inner;
            solved = beta <= target;
            // Newton update
            PF_TRY(h->cuda(cudaMemsetAsync(w.mx + 2, 0, 2 * sizeof(unsigned long long), s), "max"));
            k_be_newton<<<gL, 256, 0, s>>>(L, w.x, w.y, w.mx + 2);
            PF_TRY(check("newton update"));
            double mm[2];
            PF_TRY(read_max(2, 2, mm));
            moved = mm[0];
            ymax = mm[1];
            PF_TRY(Fval(w.y, w.F0));
            PF_TRY(read_max(0, 1, &fmax));
        }
        st.newton_iters = it;
        st.newton_iters_total += it;
        st.residual = fmax;
        if (!conv) return h->fail(PF_ENOTCONV, "backward-Euler Newton iteration did not converge (max |F| %.3e)", fmax);
        // the new fields, the balances of the step
        k_be_rates<D><<<gN, 256, 0, s>>>(a, w.y, w.y0, w.der, w.Ft, 1, w.mx);
        const int o_ = 1 - c;
        const int nbf = std::min(gN, (int)(BE_NPART / 5));
        k_be_finish<<<nbf, 256, 0, s>>>(a, w.y, w.y0, w.Ft, (double *)h->theta[o_], (double *)h->xO[o_],
                                        (double *)h->xH[o_], (double *)h->xW[o_], w.part);
        k_be_diag<<<1, 32, 0, s>>>(w.part, nbf, h->dg);
        PF_TRY(check("backward-Euler step"));
        advance(h, 1);
        h->dt_last = o.dt;
    }
    return PF_OK;
}

} // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

double pf_dt_stable(const pf_config *cfg)
{
    if (!cfg || (cfg->ndim != 2 && cfg->ndim != 3)) return -1.0;
    return dt_stable_impl(cfg);
}

int pf_create(const pf_config *cfg, pf_handle **out)
{
    if (!out) return PF_EINVAL;
    *out = nullptr;
    g_create_error.clear();
    return create_one(cfg, out, g_create_error);
}

int pf_batch_create(const pf_config *cfgs, int n, pf_handle **out)
{
    if (!out) return PF_EINVAL;
    *out = nullptr;
    g_create_error.clear();
    if (!cfgs || n < 1) { g_create_error = "cfgs is NULL or n < 1"; return PF_EINVAL; }
    for (int i = 1; i < n; i++) {
        if (cfgs[i].ndim != cfgs[0].ndim || cfgs[i].precision != cfgs[0].precision
            || (cfgs[i].mechanics != 0) != (cfgs[0].mechanics != 0) || cfgs[i].precond != cfgs[0].precond) {
            g_create_error = "batch instances must share ndim, precision, mechanics and precond";
            return PF_EINVAL;
        }
    }
    // PF_PC_AUTO picks one preconditioner for the whole batch (one kernel
    // serves all instances): multigrid only if every instance qualifies
    bool all_mg = true;
    for (int i = 0; i < n; i++) all_mg = all_mg && auto_mg(cfgs[i]);
    pf_handle *b = new (std::nothrow) pf_handle();
    if (!b) { g_create_error = "host allocation failed"; return PF_ENOMEM; }
    b->is_batch = true;
    memset(&b->prof, 0, sizeof(b->prof));
    for (int i = 0; i < n; i++) {
        pf_handle *m = nullptr;
        std::string err;
        pf_config ci = cfgs[i];
        if (ci.precond == PF_PC_AUTO) ci.precond = all_mg ? PF_PC_MG : PF_PC_JACOBI;
        int rc = create_one(&ci, &m, err);
        if (rc != PF_OK) {
            char buf[64];
            snprintf(buf, sizeof(buf), "instance %d: ", i);
            g_create_error = buf + err;
            free_all(b);
            delete b;
            return rc;
        }
        b->members.push_back(m);
    }
    pf_handle *m0 = b->members[0];
    b->cfg = m0->cfg;
    b->P = m0->P;
    b->fp64 = m0->fp64;
    b->tsz = m0->tsz;
    b->dev = m0->dev;
    b->sms = m0->sms;
    b->cg_block = m0->cg_block;
    b->cg_per_sm = m0->cg_per_sm;
    b->pcg_shape = m0->pcg_shape;
    b->mg = m0->mg;
    for (pf_handle *m : b->members) b->bytes += m->bytes;
    cudaError_t e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        g_create_error = std::string("stream: ") + cudaGetErrorString(e);
        free_all(b);
        delete b;
        return PF_ECUDA;
    }
    *out = b;
    return PF_OK;
}

int pf_batch_size(const pf_handle *h)
{
    if (!h) return 0;
    return h->is_batch ? (int)h->members.size() : 1;
}

int pf_batch_set_fields(pf_handle *b, int i, const pf_fields *f, int where)
{
    if (!b) return PF_EINVAL;
    if (!b->is_batch) return b->fail(PF_EINVAL, "not a batch handle");
    if (i < 0 || i >= (int)b->members.size()) return b->fail(PF_EINVAL, "instance %d out of range", i);
    cudaStreamSynchronize(b->own);
    int rc = pf_set_fields(b->members[i], f, where);
    if (rc != PF_OK) return b->fail(rc, "instance %d: %s", i, b->members[i]->err.c_str());
    b->plan_ready = false;
    return PF_OK;
}

int pf_batch_get_fields(pf_handle *b, int i, pf_fields *out, int where)
{
    if (!b) return PF_EINVAL;
    if (!b->is_batch) return b->fail(PF_EINVAL, "not a batch handle");
    if (i < 0 || i >= (int)b->members.size()) return b->fail(PF_EINVAL, "instance %d out of range", i);
    int rc = pf_get_fields(b->members[i], out, where);
    if (rc != PF_OK) return b->fail(rc, "instance %d: %s", i, b->members[i]->err.c_str());
    return PF_OK;
}

int pf_batch_get_diagnostics(pf_handle *b, int i, pf_diag *out)
{
    if (!b) return PF_EINVAL;
    if (!b->is_batch) return b->fail(PF_EINVAL, "not a batch handle");
    if (i < 0 || i >= (int)b->members.size()) return b->fail(PF_EINVAL, "instance %d out of range", i);
    int rc = pf_get_diagnostics(b->members[i], out);
    if (rc != PF_OK) return b->fail(rc, "instance %d: %s", i, b->members[i]->err.c_str());
    return PF_OK;
}

int pf_set_fields(pf_handle *h, const pf_fields *f, int where)
{
    if (!h) return PF_EINVAL;
    if (h->is_batch) return h->fail(PF_EINVAL, "batch handle: use the pf_batch_ call for one instance");
    if (!f || !f->phi_f || !f->phi_w || !f->x_O || !f->x_H || !f->x_H2O)
        return h->fail(PF_EINVAL, "phi_f, phi_w, x_O, x_H and x_H2O are required");
    if (where != PF_HOST && where != PF_DEVICE) return h->fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    cudaStream_t s = h->own;
    const int rc = h->fp64 ? set_fields_t<double>(h, f, where, s) : set_fields_t<float>(h, f, where, s);
    if (rc == PF_OK) h->dt_last = 0.0;
    return rc;
}

int pf_step(pf_handle *h, int nsteps, void *stream)
{
    if (!h) return PF_EINVAL;
    if (nsteps < 0) return h->fail(PF_EINVAL, "nsteps < 0");
    for (pf_handle *m : instances(h))
        if (!m->have_fields) return h->fail(PF_ESTATE, "pf_step before the fields were set");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own;
    {
        // order the caller's stream after anything queued on the library
        // streams (the handle's and, in a batch, its members')
        cudaEvent_t ev;
        PF_TRY(h->cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event"));
        for (pf_handle *m : instances(h)) {
            if (m->own == s) continue;
            cudaEventRecord(ev, m->own);
            cudaStreamWaitEvent(s, ev, 0);
        }
        if (h->is_batch && h->own != s) {
            cudaEventRecord(ev, h->own);
            cudaStreamWaitEvent(s, ev, 0);
        }
        cudaEventDestroy(ev);
    }
    // clear the sticky device status words of this call
    for (pf_handle *m : instances(h)) {
        PF_TRY(h->cuda(cudaMemsetAsync(&m->sc->status, 0, sizeof(int), s), "status clear"));
        PF_TRY(h->cuda(cudaMemsetAsync(&m->dg->status, 0, sizeof(int), s), "status clear"));
        PF_TRY(h->cuda(cudaMemsetAsync(&m->dg->cg_max, 0, sizeof(int), s), "status clear"));
    }
    int rc;
    if (h->cfg.ndim == 2) rc = h->fp64 ? run_steps<double, 2>(h, nsteps, s) : run_steps<float, 2>(h, nsteps, s);
    else rc = h->fp64 ? run_steps<double, 3>(h, nsteps, s) : run_steps<float, 3>(h, nsteps, s);
    if (rc != PF_OK) return rc;
    if (nsteps > 0)
        for (pf_handle *m : instances(h)) m->dt_last = 0.0;
    std::vector<pf_handle *> I = instances(h);
    std::vector<Scalars> scs(I.size());
    std::vector<Diag> dgs(I.size());
    for (size_t i = 0; i < I.size(); i++) {
        PF_TRY(h->cuda(cudaMemcpyAsync(&scs[i], I[i]->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "status read"));
        PF_TRY(h->cuda(cudaMemcpyAsync(&dgs[i], I[i]->dg, sizeof(Diag), cudaMemcpyDeviceToHost, s), "status read"));
    }
    PF_TRY(h->cuda(cudaStreamSynchronize(s), "pf_step"));
    long long cg_new = 0;
    int st = PF_OK;
    for (size_t i = 0; i < I.size(); i++) {
        cg_new += dgs[i].cg_total - I[i]->cg_total_seen;
        I[i]->cg_total_seen = dgs[i].cg_total;
        int sti = PF_OK;
        if (scs[i].status == 6 || dgs[i].status == 6) sti = PF_ETIMEOUT;
        else if (dgs[i].status == 5) sti = PF_ENONFINITE;
        else if (scs[i].status == 4) sti = PF_ENOTCONV;
        if (sti == PF_ETIMEOUT || (sti == PF_ENONFINITE && st != PF_ETIMEOUT) || (sti == PF_ENOTCONV && st == PF_OK)) st = sti;
    }
    if (h->prof_on) {
        h->harvest();
        h->prof.cg_iters += cg_new;
    }
    if (st == PF_ETIMEOUT) return h->fail(st, "a bounded device-side wait gave up");
    if (st == PF_ENONFINITE) return h->fail(st, "non-finite value in the fields");
    if (st == PF_ENOTCONV) return h->fail(st, "CG reached cg_maxit without meeting cg_rtol");
    return PF_OK;
}

int pf_step_implicit(pf_handle *h, int nsteps, const pf_implicit_opts *opts, pf_implicit_stats *stats, void *stream)
{
    if (!h || !opts) return PF_EINVAL;
    if (nsteps < 0) return h->fail(PF_EINVAL, "nsteps < 0");
    if (h->is_batch) return h->fail(PF_EINVAL, "backward-Euler steps take a single-grid handle");
    if (!h->fp64) return h->fail(PF_EINVAL, "backward-Euler steps need precision PF_FP64");
    if (!h->have_fields) return h->fail(PF_ESTATE, "pf_step_implicit before the fields were set");
    const pf_implicit_opts &o = *opts;
    if (!(o.dt > 0.0) || !(o.newton_tol > 0.0) || o.newton_maxit < 1 || !(o.gmres_rtol > 0.0 && o.gmres_rtol < 1.0) ||
        o.gmres_restart < 1 || o.gmres_restart > BE_MAX_RESTART || o.gmres_maxit < 1 || o.pc_degree < 0 ||
        o.pc_degree > 64 || (o.pc_precision != PF_FP64 && o.pc_precision != PF_MIXED))
        return h->fail(PF_EINVAL, "invalid pf_implicit_opts");
    if (o.pc_precision == PF_MIXED && 4 * h->P.N >= (1LL << 31))
        return h->fail(PF_EINVAL, "the FP32 preconditioner takes grids of fewer than 2^29 cells");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own;
    if (h->own != s) {
        cudaEvent_t ev;
        PF_TRY(h->cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event"));
        cudaEventRecord(ev, h->own);
        cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
    }
    PF_TRY(h->cuda(cudaMemsetAsync(&h->sc->status, 0, sizeof(int), s), "status clear"));
    PF_TRY(h->cuda(cudaMemsetAsync(&h->dg->status, 0, sizeof(int), s), "status clear"));
    PF_TRY(h->cuda(cudaMemsetAsync(&h->dg->cg_max, 0, sizeof(int), s), "status clear"));
    pf_implicit_stats st;
    memset(&st, 0, sizeof(st));
    const int rc = h->cfg.ndim == 2 ? be_steps<2>(h, nsteps, o, st, s) : be_steps<3>(h, nsteps, o, st, s);
    if (stats) *stats = st;
    if (rc != PF_OK) return rc;
    Scalars sc;
    Diag dg;
    PF_TRY(h->cuda(cudaMemcpyAsync(&sc, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "status read"));
    PF_TRY(h->cuda(cudaMemcpyAsync(&dg, h->dg, sizeof(Diag), cudaMemcpyDeviceToHost, s), "status read"));
    PF_TRY(h->cuda(cudaStreamSynchronize(s), "pf_step_implicit"));
    if (sc.status == 6 || dg.status == 6) return h->fail(PF_ETIMEOUT, "a bounded device-side wait gave up");
    if (dg.status == 5) return h->fail(PF_ENONFINITE, "non-finite value in the fields");
    if (sc.status == 4) return h->fail(PF_ENOTCONV, "CG reached cg_maxit without meeting cg_rtol");
    return PF_OK;
}

int pf_set_coupling(pf_handle *h, const double *trE, const double *devE2, int where)
{
    if (!h) return PF_EINVAL;
    if (h->is_batch) return h->fail(PF_EINVAL, "pf_set_coupling takes a single-grid handle");
    if (where != PF_HOST && where != PF_DEVICE) return h->fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    if (h->cfg.mechanics)
        return h->fail(PF_ESTATE, "pf_set_coupling needs mechanics = 0 (the step's own solve sets the coupling)");
    if (!h->have_fields) return h->fail(PF_ESTATE, "pf_set_coupling before the fields were set");
    const long long N = h->P.N;
    const size_t nb = sizeof(double) * (size_t)N;
    const int g = grid_for(h, N);
    cudaStream_t s = h->own;
    const double *src[2] = {trE, devE2};
    void *dst[2] = {h->trE, h->devE2};
    double *stage[2] = {h->stage, h->stage2};
    for (int k = 0; k < 2; k++) {
        if (!src[k]) {
            PF_TRY(h->cuda(cudaMemsetAsync(dst[k], 0, h->tsz * (size_t)N, s), "coupling"));
            continue;
        }
        const double *a = src[k];
        if (where == PF_HOST) {
            PF_TRY(h->cuda(cudaMemcpyAsync(stage[k], src[k], nb, cudaMemcpyHostToDevice, s), "coupling"));
            a = stage[k];
        }
        if (h->fp64) k_in_scalar<double><<<g, 256, 0, s>>>(N, a, (double *)dst[k], 0.0);
        else k_in_scalar<float><<<g, 256, 0, s>>>(N, a, (float *)dst[k], 0.0);
    }
    PF_TRY(h->cuda(cudaGetLastError(), "coupling"));
    return h->cuda(cudaStreamSynchronize(s), "coupling");
}

int pf_get_fields(pf_handle *h, pf_fields *out, int where)
{
    if (!h || !out) return PF_EINVAL;
    if (h->is_batch) return h->fail(PF_EINVAL, "batch handle: use the pf_batch_ call for one instance");
    if (!h->have_fields) return h->fail(PF_ESTATE, "pf_get_fields before pf_set_fields");
    if (where != PF_HOST && where != PF_DEVICE) return h->fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    return h->fp64 ? get_fields_t<double>(h, out, where, h->own) : get_fields_t<float>(h, out, where, h->own);
}

int pf_get_diagnostics(pf_handle *h, pf_diag *out)
{
    if (!h || !out) return PF_EINVAL;
    if (h->is_batch) return h->fail(PF_EINVAL, "batch handle: use the pf_batch_ call for one instance");
    Scalars sc;
    Diag dg;
    PF_TRY(h->cuda(cudaMemcpy(&sc, h->sc, sizeof(sc), cudaMemcpyDeviceToHost), "scalars"));
    PF_TRY(h->cuda(cudaMemcpy(&dg, h->dg, sizeof(dg), cudaMemcpyDeviceToHost), "diag"));
    memset(out, 0, sizeof(*out));
    out->sum_O = dg.sumO; out->sum_H = dg.sumH; out->sum_H2O = dg.sumW;
    out->removed_H2O = dg.removedW; out->supplied_H = dg.suppliedH;
    out->sum_O_init = h->sumO0;
    out->reduction_degree = h->sumO0 != 0.0 && h->steps > 0 ? 1.0 - dg.sumO / h->sumO0 : 0.0;
    // reduction rate of the last step, -(sum x_O,n - sum x_O,n-1) / (sum x_O,init dt)
    // (Sec. 4.2.1); before the first update the previous sum is the initial one
    const double prevO = h->steps == 1 ? h->sumO0 : dg.sumO_prev;
    // the last step's time step: backward-Euler steps take their own
    const double dt = h->dt_last > 0.0 ? h->dt_last : h->P.dt;
    out->reduction_rate = h->sumO0 != 0.0 && h->steps > 0 ? (prevO - dg.sumO) / (h->sumO0 * dt) : 0.0;
    out->cg_rel_residual = sc.relres;
    out->cg_iters_last = dg.cg_last;
    out->cg_iters_max = dg.cg_max;
    out->cg_iters_total = dg.cg_total;
    out->steps = h->steps;
    out->dt = dt;
    out->status = dg.status ? dg.status : sc.status;
    out->precond = h->mg ? PF_PC_MG : PF_PC_JACOBI;
    out->mg_levels = !h->mg ? 0 : (h->cfg.ndim == 2 ? mg_levels(h->P.nx, h->P.ny) : mg_levels3(h->P.nx, h->P.ny, h->P.nz));
    return PF_OK;
}

int pf_free_energy(pf_handle *h, double *out)
{
    if (!h || !out) return PF_EINVAL;
    if (h->is_batch) return h->fail(PF_EINVAL, "batch handle: use the pf_batch_ call for one instance");
    if (!h->have_fields) return h->fail(PF_ESTATE, "no fields");
    const int g = grid_for(h, h->P.N);
    if (h->cfg.ndim == 2) {
        if (h->fp64) k_free_energy<double, 2><<<g, 256, 0, h->own>>>(h->P, field_ptrs<double, 2>(h), h->partials);
        else k_free_energy<float, 2><<<g, 256, 0, h->own>>>(h->P, field_ptrs<float, 2>(h), h->partials);
    } else {
        if (h->fp64) k_free_energy<double, 3><<<g, 256, 0, h->own>>>(h->P, field_ptrs<double, 3>(h), h->partials);
        else k_free_energy<float, 3><<<g, 256, 0, h->own>>>(h->P, field_ptrs<float, 3>(h), h->partials);
    }
    std::vector<double> part((size_t)g * PSTRIDE);
    PF_TRY(h->cuda(cudaMemcpyAsync(part.data(), h->partials, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->own), "partials"));
    PF_TRY(h->cuda(cudaStreamSynchronize(h->own), "free energy"));
    double s = 0.0;
    for (int b = 0; b < g; b++) s += part[(size_t)b * PSTRIDE];
    *out = s;
    return PF_OK;
}

int pf_profile_enable(pf_handle *h, int on)
{
    if (!h) return PF_EINVAL;
    cudaStreamSynchronize(h->own);
    h->ev_used = 0;
    h->ev_class.clear();
    memset(&h->prof, 0, sizeof(h->prof));
    h->prof_on = on != 0;
    h->prof.enabled = h->prof_on ? 1 : 0;
    return PF_OK;
}

int pf_profile_read(pf_handle *h, pf_profile *out)
{
    if (!h || !out) return PF_EINVAL;
    *out = h->prof;
    return PF_OK;
}

int pf_attach_unet(pf_handle *h, pf_unet *net)
{
    if (!h) return PF_EINVAL;
    for (pf_handle *m : instances(h)) {
        cudaStreamSynchronize(m->own);
        unet_work_destroy(m->net_work);
        m->net_work = nullptr;
        for (void *p : m->net_allocs) cudaFree(p);
        m->net_allocs.clear();
        m->net = nullptr;
        m->net_in = m->net_prev = nullptr;
        m->net_mode = nullptr;
    }
    h->plan_ready = false;
    if (!net) return PF_OK;
    if (unet_ndim(net) != h->cfg.ndim) return h->fail(PF_EINVAL, "network is %dD, grid is %dD", unet_ndim(net), h->cfg.ndim);
    if (unet_cin(net) != 4) return h->fail(PF_EINVAL, "warm-start network needs 4 input channels");
    for (pf_handle *m : instances(h)) {
        const int nz = m->cfg.ndim == 3 ? m->cfg.nz : 1;
        m->net_work = unet_work_create(net, 1, m->cfg.nx, m->cfg.ny, nz);
        if (!m->net_work) {
            std::string why = unet_error(net);
            pf_attach_unet(h, nullptr);
            return h->fail(PF_EINVAL, "grid %dx%dx%d does not suit the network: %s", m->cfg.nx, m->cfg.ny, nz, why.c_str());
        }
        const size_t N = (size_t)m->P.N;
        void *a = nullptr, *b = nullptr, *c = nullptr;
        if (cudaMalloc(&a, sizeof(float) * N * 4) != cudaSuccess || cudaMalloc(&b, sizeof(float) * N) != cudaSuccess
            || cudaMalloc(&c, sizeof(int)) != cudaSuccess) {
            if (a) cudaFree(a);
            if (b) cudaFree(b);
            pf_attach_unet(h, nullptr);
            return h->fail(PF_ENOMEM, "warm-start buffers");
        }
        m->net_allocs = {a, b, c};
        m->net_in = (float *)a;
        m->net_prev = (float *)b;
        m->net_mode = (int *)c;
        cudaMemset(m->net_prev, 0, sizeof(float) * N);
        const int first = 1;
        cudaMemcpy(m->net_mode, &first, sizeof(int), cudaMemcpyHostToDevice);
        m->net = net;
    }
    return h->cuda(cudaDeviceSynchronize(), "attach");
}

int pf_selftest_wait(long long spin_limit)
{
    if (spin_limit < 1 || spin_limit > SPIN_LIMIT) return PF_EINVAL;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return PF_ENOMEM;
    int rc = PF_OK;
    int err = 0;
    if (cudaMemset(buf, 0, 2 * sizeof(int)) != cudaSuccess) rc = PF_ECUDA;
    if (rc == PF_OK) {
        k_wait_selftest<<<1, 32>>>((const unsigned int *)buf, (int *)buf + 1, spin_limit);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = PF_ECUDA;
    }
    if (rc == PF_OK && cudaMemcpy(&err, (int *)buf + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = PF_ECUDA;
    cudaFree(buf);
    if (rc != PF_OK) return rc;
    return err == 6 ? PF_ETIMEOUT : PF_ECUDA;
}

long long pf_device_bytes(const pf_handle *h) { return h ? h->bytes : 0; }

const char *pf_last_error(const pf_handle *h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void pf_destroy(pf_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->own);
    free_all(h);
    delete h;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free field update.
//
// Some callers cannot allocate device memory where they run the step: host
// runtimes that hand out a fixed device-memory budget up front and forbid
// allocations afterwards, and callers that must not touch the allocator
// state of a process they share.  For them,
// pf_fields_update_static runs the explicit field update of one step with its
// working arrays in the fixed device array below instead of in memory it
// allocates.  The array exists once per device that loads the library, for
// the life of the process.  Every call shares it: calls whose work overlaps
// on the GPU (other streams, other host threads) race and must be
// serialised by the caller.
// ---------------------------------------------------------------------------
namespace {

constexpr long long STATIC_MAX_CELLS = PF_STATIC_MAX_CELLS;
constexpr int STATIC_BLOCKS = 512;
// theta, phi_g, mu_O, M_O, theta_out, zero, zero, one  (8 FP64 arrays), then
// the partial sums, the last-block counter, the diagnostics record and the
// zero mask.
constexpr size_t STATIC_ARRAYS = 8;
constexpr size_t STATIC_DOUBLES = STATIC_ARRAYS * STATIC_MAX_CELLS + (size_t)STATIC_BLOCKS * PSTRIDE + 64;
constexpr size_t STATIC_BYTES = STATIC_DOUBLES * sizeof(double) + STATIC_MAX_CELLS;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

std::mutex g_static_mu;
void *g_static_addr[64] = {};

// Device address of the scratch array for the current device (looked up once
// per device, by the first call made with that device current; the
// host-side name is only a stand-in for it).  The address is cached for the
// life of the process: after cudaDeviceReset the array has a new address in
// the new context, so the library must not be used across a device reset.
int static_scratch(void **out, std::string &err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return PF_ECUDA; }
    if (dev < 0 || dev >= 64) { err = "device index out of range"; return PF_ECUDA; }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PF_ECUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return PF_OK;
}

thread_local std::string g_static_error;

// Records the error of the failing CUDA call (cudaSuccess if none failed).
template <int D>
int fields_update_static_t(const Params &P, const pf_fields *in, const double *trE, const double *devE2,
                           pf_fields *out, cudaStream_t s, void *base, cudaError_t &cerr)
{
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && cerr == cudaSuccess) cerr = e; return e == cudaSuccess; };
    const long long N = P.N;
    double *a = (double *)base;
    double *theta = a, *phig = a + N, *muO = a + 2 * N, *MO = a + 3 * N, *theta_o = a + 4 * N;
    double *zero0 = a + 5 * N, *zero1 = a + 6 * N, *one = a + 7 * N;
    double *partials = a + STATIC_ARRAYS * STATIC_MAX_CELLS;
    double *tail = partials + (size_t)STATIC_BLOCKS * PSTRIDE;
    unsigned int *counter = (unsigned int *)tail;
    Diag *dg = (Diag *)(tail + 8);
    unsigned char *mask0 = (unsigned char *)(a + STATIC_DOUBLES);
    const int g = (int)std::min<long long>((N + 255) / 256, STATIC_BLOCKS);
    // state that must start at zero on every call
    if (!ck(cudaMemsetAsync(tail, 0, 64 * sizeof(double), s))) return PF_ECUDA;
    if (!trE || !devE2) {
        if (!ck(cudaMemsetAsync(zero0, 0, sizeof(double) * N, s))) return PF_ECUDA;
        if (!ck(cudaMemsetAsync(zero1, 0, sizeof(double) * N, s))) return PF_ECUDA;
    }
    if (!in->dirichlet && !ck(cudaMemsetAsync(mask0, 0, (size_t)N, s))) return PF_ECUDA;
    if (!in->mobility) k_in_scalar<double><<<g, 256, 0, s>>>(N, nullptr, one, 1.0);
    k_in_phase<double><<<g, 256, 0, s>>>(N, in->phi_f, in->phi_w, theta, phig);
    FieldPtrs<double, D> F;
    memset(&F, 0, sizeof(F));
    F.theta = theta; F.phig = phig; F.xO = in->x_O; F.xH = in->x_H; F.xW = in->x_H2O;
    F.mob = in->mobility ? in->mobility : one;
    F.mask = in->dirichlet ? in->dirichlet : mask0;
    F.theta_o = theta_o; F.xO_o = out->x_O; F.xH_o = out->x_H; F.xW_o = out->x_H2O;
    F.muO = muO; F.MO = MO;
    F.trE = const_cast<double *>(trE ? trE : zero0);
    F.devE2 = const_cast<double *>(devE2 ? devE2 : zero1);
    // the job travels in the launch parameters: nothing is copied to the
    // device before the launches
    JobSet<CellJob<double, D>> js;
    memset(&js, 0, sizeof(js));
    js.one.P = P;
    js.one.K = cell_const<double>(P);
    js.one.F = F;
    js.one.partials = partials;
    js.one.counter = counter;
    js.one.dg = dg;
    js.one.block0 = 0;
    js.one.nblocks = g;
    k_mu<double, D><<<g, 256, 0, s>>>(js);
    k_update<double, D><<<g, 256, 0, s>>>(js);
    k_out_phase<double><<<g, 256, 0, s>>>(N, theta_o, phig, out->phi_f, out->phi_w);
    if (!ck(cudaGetLastError())) return PF_ECUDA;
    int status = 0;
    if (!ck(cudaMemcpyAsync(&status, &dg->status, sizeof(int), cudaMemcpyDeviceToHost, s))) return PF_ECUDA;
    if (!ck(cudaStreamSynchronize(s))) return PF_ECUDA;
    return status == 5 ? PF_ENONFINITE : PF_OK;
}

} // namespace

extern "C" {

int pf_fields_update_static(const pf_config *cfg, const pf_fields *in, const double *trE, const double *devE2,
                            pf_fields *out, void *cudaStream)
{
    g_static_error.clear();
    if (!cfg || !in || !out) { g_static_error = "cfg, in and out are required"; return PF_EINVAL; }
    if (cfg->ndim != 2 && cfg->ndim != 3) { g_static_error = "ndim must be 2 or 3"; return PF_EINVAL; }
    if (cfg->nx < 2 || cfg->ny < 2 || (cfg->ndim == 3 && cfg->nz < 2)) { g_static_error = "grid sizes must be >= 2"; return PF_EINVAL; }
    const long long N = (long long)cfg->nx * cfg->ny * (cfg->ndim == 3 ? cfg->nz : 1);
    if (N > STATIC_MAX_CELLS) {
        char buf[160];
        snprintf(buf, sizeof(buf), "grid has %lld cells; pf_fields_update_static handles at most %lld (PF_STATIC_MAX_CELLS)",
                 N, STATIC_MAX_CELLS);
        g_static_error = buf;
        return PF_EINVAL;
    }
    if (!in->phi_f || !in->phi_w || !in->x_O || !in->x_H || !in->x_H2O ||
        !out->phi_f || !out->phi_w || !out->x_O || !out->x_H || !out->x_H2O) {
        g_static_error = "phi_f, phi_w, x_O, x_H and x_H2O are required in `in` and `out`";
        return PF_EINVAL;
    }
    void *base = nullptr;
    int rc = static_scratch(&base, g_static_error);
    if (rc != PF_OK) return rc;
    pf_config c = *cfg;
    if (c.ndim == 2) c.nz = 1;
    Params P;
    fill_params(c, N, P);
    cudaStream_t s = (cudaStream_t)cudaStream;
    cudaError_t cerr = cudaSuccess;
    rc = c.ndim == 2 ? fields_update_static_t<2>(P, in, trE, devE2, out, s, base, cerr)
                     : fields_update_static_t<3>(P, in, trE, devE2, out, s, base, cerr);
    if (rc == PF_ECUDA) g_static_error = std::string("CUDA error: ") + cudaGetErrorString(cerr);
    else if (rc == PF_ENONFINITE) g_static_error = "non-finite value in the fields";
    return rc;
}

const char *pf_static_last_error(void) { return g_static_error.c_str(); }

} // extern "C"
