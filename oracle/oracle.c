/*
 * Plain FP64 CPU oracle for one explicit time step of the chemo-mechanical
 * phase-field model of wuestite-to-iron reduction by hydrogen
 * (Bai, Mianroodi et al., arXiv 2111.11538).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA path; only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.
 *
 * Everything is written as plain loops over cells / elements in the order the
 * method states it, in double precision, single-threaded.
 *
 * Paper passages followed (section + equation label of the paper):
 *   phase interpolation h(x) ............... Sec. 3.1, below (DenEneFreChePha)
 *   chemical energies f_f, f_w, f_g ........ Sec. 3.1, (DenEneFreChePha), (free-energy-gas-phase)
 *   bulk / interface energy ................ Sec. 2.2, (DenEneFreBul), (DenEneFreInt)
 *   dependent gas phase .................... Sec. 2.2, (PhaParOrdDer)
 *   field relations ........................ Sec. 2.4, (FieRelDRI)
 *   driving forces ......................... Sec. 2.4, (FiePhaDenEneFreDerPar)
 *   chemical potential / fluxes ............ Sec. 2.2-2.3, (ConEneMixIOR), (ConKinMixIOR)
 *   oxygen mobility M_O = D_O / psi_che'' .. Sec. 3.2 (parameter notes)
 *   reaction rate r = m(phi_g) k x_O x_H ... Sec. 2.3.1, (EmpModRea), (forward-k)
 *   reaction halts when x_H2O = 1 .......... Sec. 4.3 (isolated pores)
 *   effective moduli ....................... Sec. 2.4, (ModElaEff)
 *   transformation eigenstrain ............. Sec. 2.2, (RulFloDefLocAlt), linearised
 *   J2 plasticity, linear hardening ........ Sec. 2.3, (PlaTwoJ); Sec. 2.4, (RulFloPla)
 *   reduction degree ....................... Sec. 4.2.1, (reduction-degree)
 *
 * Readings of the paper taken where it is silent or inconsistent (each is
 * listed in the design notes of the repository):
 *   R1  m(x) = x^2 (1-x)^2 (the paper uses m but never defines it).
 *   R2  The gas (pore) fraction phi_g = 1 - phi_f - phi_w is held fixed and
 *       the solid is split by the order parameter theta = phi_f / (phi_f +
 *       phi_w).  Phase weights W_f = (1 - h(phi_g)) h(theta),
 *       W_w = (1 - h(phi_g)) (1 - h(theta)), W_g = h(phi_g) replace h(phi_a);
 *       they equal h(phi_a) on every two-phase interface and sum to one.  The
 *       double well and gradient energy of the solid pair become 2 w m(theta)
 *       and eps |grad theta|^2 (their two-phase values), and theta follows
 *       dtheta/dt = -(L/2) delta psi / delta theta, which on a ferrite /
 *       wuestite interface is the paper's pair of Allen-Cahn relations with
 *       phi_g kept at zero.  Taken literally, with absolute CALPHAD energies
 *       and independent phi_f, phi_w, those relations create or destroy gas
 *       inside ferrite/wuestite interfaces (and wuestite inside ferrite/gas
 *       interfaces) without bound.
 *   R3  Oxygen uses the un-reduced flux j_O = -M_O grad mu_O, mu_O the
 *       variational derivative, M_O = D_O(phi) / psi_che''(x_O).
 *   R4  Species diffusivities D_i(phi) = (1 - h(phi_g)) D_i,solid + h(phi_g) D_i,gas.
 *   R5  Small-strain linear elasticity; eigenstrain eig0 W_f I + eps_p;
 *       periodic fluctuation u plus a free macroscopic strain Ebar whose mean
 *       stress is prescribed (-prestress I); plane strain in 2D.
 *   R6  Staggered coupling per step: elastic solve with eps_p^n as eigenstrain,
 *       then one radial return per cell on the cell-centre strain, then an
 *       explicit Euler step of all five fields with the returned stress.
 *   R7  Discretisation: cell-centred fields, 2d+1-point Laplacian, face fluxes
 *       with arithmetic face means, Q1 voxel elements with 2^d Gauss points
 *       and cell-constant moduli / eigenstrain, Jacobi-preconditioned CG
 *       stopped on ||r||_2 <= rtol ||b||_2.
 *   R8  Dirichlet cells: after each step x_H := xH_bc and x_H2O := 0, the
 *       removed water and the supplied hydrogen being counted.
 *
 * Pins (tests/test_oracle_*.py, no GPU): the printed CALPHAD coefficients,
 * derivative identities, the common tangent, the strain-coupled well count,
 * the tanh interface, exact discrete diffusion (DFT) of hydrogen and, in one
 * phase, of oxygen with its gradient-energy term, elasticity against an
 * independent Fourier solve and the Eshelby disk / sphere, free-energy
 * decrease, the O + H2O and H + 2 H2O balances, the lever rule, and J2
 * closed forms in shear and uniaxial strain.  The fully coupled step as a
 * whole has no closed form: beyond those pins its parity is unpinned, and
 * this file is the contract.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Parameter and state records (mirrored by ctypes in oracle/__init__.py).   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ndim, nx, ny, nz;
    double dt;
    double c_chem;      /* R theta / (V_mol E_s): scale of the CALPHAD polynomials */
    double w;           /* double-well height w_alpha (all phases)                  */
    double eps_phi;     /* gradient-energy coefficient epsilon_alpha (all phases)  */
    double kappa_O;     /* oxygen gradient-energy coefficient                       */
    double L;           /* phase mobility L_alpha                                   */
    double D_O_s, D_O_g, D_H_s, D_H_g, D_W_s, D_W_g;
    double k_for;       /* reaction constant                                        */
    double xH_bc;       /* hydrogen fraction held on Dirichlet cells                */
    double E_s, nu, E_g_ratio;
    double eig0;        /* linearised transformation strain (per unit h(phi_f))     */
    double sigma_Y, H_hard;
    double prestress;   /* prescribed mean stress = -prestress * I                  */
    double cg_rtol;
    int cg_maxit;
    int mechanics;      /* 0: no solve, coupling scalars zero                      */
    int plasticity;     /* 0: elastic                                              */
    int warm_start;     /* 0: zero initial guess, 1: previous solution            */
} or_params;

typedef struct {
    double *theta;                           /* N solid order parameter       */
    const double *phig;                      /* N fixed gas fraction          */
    double *xO, *xH, *xW;                    /* N each, x fastest             */
    double *u;                               /* N*ndim nodal fluctuation      */
    double *Ebar;                            /* 3 (2D) or 6 (3D), Voigt       */
    double *eps_p;                           /* N*4 (2D: xx,yy,zz,xy) or N*6  */
    double *alpha;                           /* N accumulated plastic strain  */
    const double *mob;                       /* N mobility factor             */
    const unsigned char *mask;               /* N Dirichlet flag              */
    double *trE, *devE2;                     /* N coupling scalars            */
    double *sigma;                           /* N*4 (2D) or N*6 stress        */
    double removedW, suppliedH;
    int cg_iters;
    double cg_relres;
} or_state;

/* ------------------------------------------------------------------------ */
/* Energy functions (Sec. 3.1).                                              */
/* ------------------------------------------------------------------------ */
double or_h(double x)   { return x * x * x * (6.0 * x * x - 15.0 * x + 10.0); }
double or_hp(double x)  { return 30.0 * x * x * (1.0 - x) * (1.0 - x); }
double or_m(double x)   { return x * x * (1.0 - x) * (1.0 - x); }           /* R1 */
double or_mp(double x)  { return 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x); }

/* alpha: 0 ferrite, 1 wuestite, 2 gas; scaled energies f = (V_mol/R theta) psi */
double or_f(int a, double x)
{
    if (a == 0) return 163.708 * x * x * x * x - 182.510 * x * x * x + 90.573 * x * x - 36.031 * x - 4.372;
    if (a == 1) return 173.263 * x * x - 213.460 * x + 41.953;
    return 1.0e3 * x * x;
}
double or_fp(int a, double x)
{
    if (a == 0) return 4.0 * 163.708 * x * x * x - 3.0 * 182.510 * x * x + 2.0 * 90.573 * x - 36.031;
    if (a == 1) return 2.0 * 173.263 * x - 213.460;
    return 2.0e3 * x;
}
double or_fpp(int a, double x)
{
    if (a == 0) return 12.0 * 163.708 * x * x - 6.0 * 182.510 * x + 2.0 * 90.573;
    if (a == 1) return 2.0 * 173.263;
    return 2.0e3;
}

/* Phase weights (R2): W_f, W_w, W_g from theta and the fixed gas fraction;
 * they play the role of h(phi_a) in (DenEneFreBul). */
static void weights(double th, double pg, double W[3])
{
    double hg = or_h(pg), ht = or_h(th);
    W[0] = (1.0 - hg) * ht;
    W[1] = (1.0 - hg) * (1.0 - ht);
    W[2] = hg;
}

/* Phase bulk / shear moduli from (E, nu). */
static void phase_moduli(const or_params *p, int a, double *K, double *G)
{
    double E = (a == 2) ? p->E_s * p->E_g_ratio : p->E_s;
    *K = E / (3.0 * (1.0 - 2.0 * p->nu));
    *G = E / (2.0 * (1.0 + p->nu));
}

/* Mixture moduli (ModElaEff, small-strain form: d_T dropped). */
static void cell_moduli(const or_params *p, double th, double pg, double *K, double *G)
{
    double hn[3], Ka, Ga;
    weights(th, pg, hn);
    *K = 0.0; *G = 0.0;
    for (int a = 0; a < 3; a++) {
        phase_moduli(p, a, &Ka, &Ga);
        *K += hn[a] * Ka;
        *G += hn[a] * Ga;
    }
}

/* ------------------------------------------------------------------------ */
/* Stable time step (reading: the paper integrates implicitly and states no   */
/* explicit limit).  Bounds for: species diffusion, the oxygen gradient       */
/* (fourth-order) term, the linear part of the phase equation, and the        */
/* reaction.  The caller takes 0.2 of it.                                     */
/* ------------------------------------------------------------------------ */
double or_dt_stable(const or_params *p)
{
    int d = p->ndim;
    double Dmax = p->D_O_s;
    double Ds[6] = { p->D_O_s, p->D_O_g, p->D_H_s, p->D_H_g, p->D_W_s, p->D_W_g };
    for (int i = 0; i < 6; i++) if (Ds[i] > Dmax) Dmax = Ds[i];
    double dt = 1.0e300;
    if (Dmax > 0.0) {
        double t = 1.0 / (2.0 * d * Dmax);
        if (t < dt) dt = t;
    }
    /* smallest curvature of the phase energies over [0,1]: the ferrite quartic
     * has its minimum second derivative where its third derivative vanishes. */
    double xm = (6.0 * 182.510) / (24.0 * 163.708);
    double fmin = or_fpp(0, xm);
    if (or_fpp(1, 0.0) < fmin) fmin = or_fpp(1, 0.0);
    if (p->kappa_O > 0.0 && p->c_chem > 0.0 && Dmax > 0.0) {
        double Mmax = Dmax / (p->c_chem * fmin);
        double t = 2.0 / (Mmax * p->kappa_O * (4.0 * d) * (4.0 * d));
        if (t < dt) dt = t;
    }
    if (p->L > 0.0) {
        /* theta equation (R2): gradient part L g eps (-Laplacian), symbol <= 4d;
         * double-well part <= 2 L g w; mobility factors <= 1.2 */
        double t = 1.0 / (1.2 * p->L * (2.0 * d * p->eps_phi + 2.0 * p->w));
        if (t < dt) dt = t;
    }
    if (p->k_for > 0.0) {
        double t = 1.0 / (p->k_for * (1.0 / 16.0) * (0.571 + 2.0 * p->xH_bc));
        if (t < dt) dt = t;
    }
    return dt;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers.                                                             */
/* ------------------------------------------------------------------------ */
static long ncell(const or_params *p) { return (long)p->nx * p->ny * (p->ndim == 3 ? p->nz : 1); }
static int nzz(const or_params *p) { return p->ndim == 3 ? p->nz : 1; }
static long idx(const or_params *p, int i, int j, int k)
{
    int nx = p->nx, ny = p->ny, nz = nzz(p);
    i = (i % nx + nx) % nx; j = (j % ny + ny) % ny; k = (k % nz + nz) % nz;
    return (long)i + (long)nx * ((long)j + (long)ny * k);
}
/* neighbour of cell c along axis ax by s = +-1 */
static long nbr(const or_params *p, long c, int ax, int s)
{
    int nx = p->nx, ny = p->ny;
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long)nx * ny));
    if (ax == 0) i += s; else if (ax == 1) j += s; else k += s;
    return idx(p, i, j, k);
}

static void laplacian(const or_params *p, const double *v, double *out)
{
    long N = ncell(p);
    for (long c = 0; c < N; c++) {
        double s = 0.0;
        for (int ax = 0; ax < p->ndim; ax++)
            s += v[nbr(p, c, ax, +1)] + v[nbr(p, c, ax, -1)] - 2.0 * v[c];
        out[c] = s;
    }
}

/* div(k grad v) with face value k_f = (k_c + k_n)/2 and face flux k_f (v_n - v_c) */
static void div_flux(const or_params *p, const double *k, const double *v, double *out)
{
    long N = ncell(p);
    for (long c = 0; c < N; c++) {
        double s = 0.0;
        for (int ax = 0; ax < p->ndim; ax++) {
            long cp = nbr(p, c, ax, +1), cm = nbr(p, c, ax, -1);
            s += 0.5 * (k[c] + k[cp]) * (v[cp] - v[c]);
            s -= 0.5 * (k[cm] + k[c]) * (v[c] - v[cm]);
        }
        out[c] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Q1 voxel finite elements (R5, R7).                                        */
/* Local node a has bits (ax, ay, az); element = cell (i,j,k) with nodes     */
/* (i+ax, j+ay, k+az).  Voigt order 2D: xx, yy, gxy; 3D: xx,yy,zz,gyz,gxz,gxy */
/* (engineering shears).  Plane strain in 2D.                                 */
/* ------------------------------------------------------------------------ */
static int nvoigt(const or_params *p) { return p->ndim == 2 ? 3 : 6; }
static int nnode_el(const or_params *p) { return p->ndim == 2 ? 4 : 8; }

/* derivative of local shape function a along axis k at local point xi[] */
static double dshape(int d, int a, int k, const double *xi)
{
    double v = 1.0;
    for (int l = 0; l < d; l++) {
        int bit = (a >> l) & 1;
        if (l == k) v *= bit ? 1.0 : -1.0;
        else v *= bit ? xi[l] : (1.0 - xi[l]);
    }
    return v;
}

static long el_node(const or_params *p, long e, int a)
{
    int nx = p->nx, ny = p->ny;
    int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long)nx * ny));
    return idx(p, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
}

/* Shape-function derivatives tabulated at a local point: dn[a][k]. */
typedef struct { double dn[8][3]; } shape_tab;

static void tabulate(int d, const double *xi, shape_tab *t)
{
    for (int a = 0; a < (1 << d); a++)
        for (int k = 0; k < d; k++) t->dn[a][k] = dshape(d, a, k, xi);
}

static void el_nodes(const or_params *p, long e, long *nodes)
{
    for (int a = 0; a < nnode_el(p); a++) nodes[a] = el_node(p, e, a);
}

/* strain (Voigt) at a tabulated point from the element's nodal displacements */
static void el_strain(const or_params *p, const long *nodes, const double *u, const shape_tab *t, double *eps)
{
    int d = p->ndim;
    double g[3][3] = { { 0 } };              /* g[i][k] = d u_i / d x_k */
    for (int a = 0; a < nnode_el(p); a++) {
        long n = nodes[a];
        for (int k = 0; k < d; k++)
            for (int i = 0; i < d; i++) g[i][k] += t->dn[a][k] * u[n * d + i];
    }
    if (d == 2) {
        eps[0] = g[0][0]; eps[1] = g[1][1]; eps[2] = g[0][1] + g[1][0];
    } else {
        eps[0] = g[0][0]; eps[1] = g[1][1]; eps[2] = g[2][2];
        eps[3] = g[1][2] + g[2][1]; eps[4] = g[0][2] + g[2][0]; eps[5] = g[0][1] + g[1][0];
    }
}

/* add wgt * B_a^T sigma into f for every local node a */
static void el_scatter(const or_params *p, const long *nodes, const shape_tab *t, const double *sig, double wgt, double *f)
{
    int d = p->ndim;
    for (int a = 0; a < nnode_el(p); a++) {
        long n = nodes[a];
        double dx = t->dn[a][0], dy = t->dn[a][1];
        if (d == 2) {
            f[n * 2 + 0] += wgt * (dx * sig[0] + dy * sig[2]);
            f[n * 2 + 1] += wgt * (dy * sig[1] + dx * sig[2]);
        } else {
            double dz = t->dn[a][2];
            f[n * 3 + 0] += wgt * (dx * sig[0] + dy * sig[5] + dz * sig[4]);
            f[n * 3 + 1] += wgt * (dy * sig[1] + dx * sig[5] + dz * sig[3]);
            f[n * 3 + 2] += wgt * (dz * sig[2] + dy * sig[3] + dx * sig[4]);
        }
    }
}

/* isotropic stiffness in Voigt form (plane strain in 2D: in-plane block) */
static void stress_voigt(int d, double lam, double mu, const double *eps, double *sig)
{
    if (d == 2) {
        double tr = eps[0] + eps[1];
        sig[0] = lam * tr + 2.0 * mu * eps[0];
        sig[1] = lam * tr + 2.0 * mu * eps[1];
        sig[2] = mu * eps[2];
    } else {
        double tr = eps[0] + eps[1] + eps[2];
        for (int i = 0; i < 3; i++) sig[i] = lam * tr + 2.0 * mu * eps[i];
        for (int i = 3; i < 6; i++) sig[i] = mu * eps[i];
    }
}

static void gauss_point(int d, int g, double *xi)
{
    const double a = 0.5 - 0.5 / sqrt(3.0), b = 0.5 + 0.5 / sqrt(3.0);
    for (int l = 0; l < d; l++) xi[l] = ((g >> l) & 1) ? b : a;
}

/* shape derivatives at the 2^d Gauss points */
static void gauss_tabs(int d, shape_tab *tabs)
{
    for (int g = 0; g < (1 << d); g++) {
        double xi[3];
        gauss_point(d, g, xi);
        tabulate(d, xi, &tabs[g]);
    }
}

/*
 * y = A x for the augmented unknown x = (u[N*d], E[nv]):
 *   A = sum_e int [B | I]^T D_e [B | I] dV      (energy of (RulFloDefLocAlt)-
 * driven small-strain elasticity with periodic fluctuation and mean strain).
 */
void or_mech_apply(const or_params *p, const double *lam, const double *mu, const double *x, double *y)
{
    long N = ncell(p);
    int d = p->ndim, nv = nvoigt(p), ng = 1 << d;
    long nu_ = N * d;
    const double *E = x + nu_;
    memset(y, 0, sizeof(double) * (nu_ + nv));
    double wgt = 1.0 / ng;
    shape_tab tabs[8];
    gauss_tabs(d, tabs);
    for (long e = 0; e < N; e++) {
        long nodes[8];
        el_nodes(p, e, nodes);
        for (int g = 0; g < ng; g++) {
            double eps[6], sig[6];
            el_strain(p, nodes, x, &tabs[g], eps);
            for (int k = 0; k < nv; k++) eps[k] += E[k];
            stress_voigt(d, lam[e], mu[e], eps, sig);
            el_scatter(p, nodes, &tabs[g], sig, wgt, y);
            for (int k = 0; k < nv; k++) y[nu_ + k] += wgt * sig[k];
        }
    }
}

/* Jacobi diagonal of A (computed from its definition: A e_i . e_i). */
void or_mech_diag(const or_params *p, const double *lam, const double *mu, double *dg)
{
    long N = ncell(p);
    int d = p->ndim, nv = nvoigt(p), ng = 1 << d;
    long nu_ = N * d;
    memset(dg, 0, sizeof(double) * (nu_ + nv));
    double wgt = 1.0 / ng;
    shape_tab tabs[8];
    gauss_tabs(d, tabs);
    for (long e = 0; e < N; e++) {
        long nodes[8];
        el_nodes(p, e, nodes);
        for (int g = 0; g < ng; g++) {
            for (int a = 0; a < nnode_el(p); a++) {
                long n = nodes[a];
                for (int i = 0; i < d; i++) {
                    /* strain of a unit displacement of node a, component i */
                    double eps[6] = { 0 }, sig[6];
                    double dn[3];
                    for (int k = 0; k < d; k++) dn[k] = tabs[g].dn[a][k];
                    if (d == 2) {
                        if (i == 0) { eps[0] = dn[0]; eps[2] = dn[1]; }
                        else { eps[1] = dn[1]; eps[2] = dn[0]; }
                    } else {
                        if (i == 0) { eps[0] = dn[0]; eps[5] = dn[1]; eps[4] = dn[2]; }
                        else if (i == 1) { eps[1] = dn[1]; eps[5] = dn[0]; eps[3] = dn[2]; }
                        else { eps[2] = dn[2]; eps[3] = dn[1]; eps[4] = dn[0]; }
                    }
                    stress_voigt(d, lam[e], mu[e], eps, sig);
                    double s = 0.0;
                    for (int k = 0; k < nv; k++) s += eps[k] * sig[k];
                    dg[n * d + i] += wgt * s;
                }
            }
            for (int k = 0; k < nv; k++) {
                double eps[6] = { 0 }, sig[6];
                eps[k] = 1.0;
                stress_voigt(d, lam[e], mu[e], eps, sig);
                dg[nu_ + k] += wgt * sig[k];
            }
        }
    }
}

/* Eigenstrain of a cell as a full symmetric tensor (R5), the linearised
 * transformation strain of (RulFloDefLocAlt) carried by ferrite:
 * eps* = eig0 W_f I + eps_p.  Returned as xx,yy,zz,yz,xz,xy (tensor comps). */
static double ferrite_weight(double th, double pg) { return (1.0 - or_h(pg)) * or_h(th); }

static void eigenstrain(const or_params *p, const or_state *s, long c, double es[6])
{
    double e0 = p->eig0 * ferrite_weight(s->theta[c], s->phig[c]);
    for (int i = 0; i < 6; i++) es[i] = 0.0;
    es[0] = es[1] = es[2] = e0;
    if (p->ndim == 2) {
        const double *ep = s->eps_p + c * 4;      /* xx, yy, zz, xy */
        es[0] += ep[0]; es[1] += ep[1]; es[2] += ep[2]; es[5] += ep[3];
    } else {
        const double *ep = s->eps_p + c * 6;      /* xx, yy, zz, yz, xz, xy */
        for (int i = 0; i < 6; i++) es[i] += ep[i];
    }
}

/* right-hand side b = sum_e int [B|I]^T (C_e : eps*_e) dV + V * Sigma_bar */
void or_mech_rhs(const or_params *p, const or_state *s, const double *lam, const double *mu, double *b)
{
    long N = ncell(p);
    int d = p->ndim, nv = nvoigt(p), ng = 1 << d;
    long nu_ = N * d;
    memset(b, 0, sizeof(double) * (nu_ + nv));
    double wgt = 1.0 / ng;
    shape_tab tabs[8];
    gauss_tabs(d, tabs);
    for (long e = 0; e < N; e++) {
        double es[6], sig[6];
        eigenstrain(p, s, e, es);
        double tr = es[0] + es[1] + es[2];
        /* C : eps* restricted to the Voigt components carried by the FE */
        if (d == 2) {
            sig[0] = lam[e] * tr + 2.0 * mu[e] * es[0];
            sig[1] = lam[e] * tr + 2.0 * mu[e] * es[1];
            sig[2] = 2.0 * mu[e] * es[5];
        } else {
            for (int i = 0; i < 3; i++) sig[i] = lam[e] * tr + 2.0 * mu[e] * es[i];
            for (int i = 3; i < 6; i++) sig[i] = 2.0 * mu[e] * es[i];
        }
        long nodes[8];
        el_nodes(p, e, nodes);
        for (int g = 0; g < ng; g++) {
            el_scatter(p, nodes, &tabs[g], sig, wgt, b);
            for (int k = 0; k < nv; k++) b[nu_ + k] += wgt * sig[k];
        }
    }
    /* prescribed mean stress -prestress * I on the normal components */
    for (int k = 0; k < d; k++) b[nu_ + k] += (double)N * (-p->prestress);
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Lame parameters per cell from the phase fields. */
void or_cell_lame(const or_params *p, const double *theta, const double *phig, double *lam, double *mu)
{
    long N = ncell(p);
    for (long c = 0; c < N; c++) {
        double K, G;
        cell_moduli(p, theta[c], phig[c], &K, &G);
        lam[c] = K - 2.0 * G / 3.0;
        mu[c] = G;
    }
}

/*
 * Jacobi-preconditioned CG (R7) on A x = b; x holds the initial guess and
 * receives the solution.  Returns the iteration count; *relres = ||r||/||b||.
 */
int or_pcg(const or_params *p, const double *lam, const double *mu, const double *b, double *x, double *relres)
{
    long N = ncell(p);
    long n = N * p->ndim + nvoigt(p);
    double *dg = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n), *pp = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    or_mech_diag(p, lam, mu, dg);
    double bnorm = sqrt(dot(n, b, b));
    int it = 0;
    if (bnorm == 0.0) {
        for (long i = 0; i < n; i++) x[i] = 0.0;
        *relres = 0.0;
        goto done;
    }
    or_mech_apply(p, lam, mu, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    double rn = sqrt(dot(n, r, r));
    *relres = rn / bnorm;
    if (rn <= p->cg_rtol * bnorm) goto done;
    for (long i = 0; i < n; i++) { z[i] = r[i] / dg[i]; pp[i] = z[i]; }
    double rz = dot(n, r, z);
    while (it < p->cg_maxit) {
        or_mech_apply(p, lam, mu, pp, q);
        double alpha = rz / dot(n, pp, q);
        for (long i = 0; i < n; i++) { x[i] += alpha * pp[i]; r[i] -= alpha * q[i]; }
        it++;
        rn = sqrt(dot(n, r, r));
        *relres = rn / bnorm;
        if (rn <= p->cg_rtol * bnorm) break;
        for (long i = 0; i < n; i++) z[i] = r[i] / dg[i];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < n; i++) pp[i] = z[i] + beta * pp[i];
    }
done:
    free(dg); free(r); free(z); free(pp); free(q);
    return it;
}

/*
 * Cell-centre strain (Voigt) of the current displacement plus Ebar; the
 * centre value equals the element average for Q1.
 */
static void centre_strain(const or_params *p, const or_state *s, long e, double *eps)
{
    double xi[3] = { 0.5, 0.5, 0.5 };
    shape_tab t;
    long nodes[8];
    tabulate(p->ndim, xi, &t);
    el_nodes(p, e, nodes);
    el_strain(p, nodes, s->u, &t, eps);
    for (int k = 0; k < nvoigt(p); k++) eps[k] += s->Ebar[k];
}

/*
 * Per-cell stress update with J2 radial return (PlaTwoJ), (RulFloPla),
 * small-strain analogue: yield |dev sigma| - sqrt(2/3)(sigma_Y + H a) <= 0,
 * associative flow along dev sigma / |dev sigma|, da = dlambda.
 * Writes eps_p, alpha, the stress and the coupling scalars
 * trE = tr eps_e and devE2 = |dev eps_e|^2 used by the phase equation.
 */
void or_return_map(const or_params *p, or_state *s)
{
    long N = ncell(p);
    int d = p->ndim;
    for (long c = 0; c < N; c++) {
        double ev[6], et[6];                  /* total strain, tensor comps */
        centre_strain(p, s, c, ev);
        if (d == 2) {
            et[0] = ev[0]; et[1] = ev[1]; et[2] = 0.0; et[3] = 0.0; et[4] = 0.0; et[5] = 0.5 * ev[2];
        } else {
            et[0] = ev[0]; et[1] = ev[1]; et[2] = ev[2];
            et[3] = 0.5 * ev[3]; et[4] = 0.5 * ev[4]; et[5] = 0.5 * ev[5];
        }
        double K, G;
        cell_moduli(p, s->theta[c], s->phig[c], &K, &G);
        double es[6], ee[6];
        eigenstrain(p, s, c, es);
        for (int i = 0; i < 6; i++) ee[i] = et[i] - es[i];
        double tr = ee[0] + ee[1] + ee[2];
        double dev[6];
        for (int i = 0; i < 6; i++) dev[i] = ee[i] - (i < 3 ? tr / 3.0 : 0.0);
        double n2 = dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]
                  + 2.0 * (dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
        if (p->plasticity) {
            double snorm = 2.0 * G * sqrt(n2);
            double ystress = sqrt(2.0 / 3.0) * (p->sigma_Y + p->H_hard * s->alpha[c]);
            double f = snorm - ystress;
            if (f > 0.0) {
                double dl = f / (2.0 * G + sqrt(2.0 / 3.0) * p->H_hard);
                double nrm = sqrt(n2);
                double dep[6];
                for (int i = 0; i < 6; i++) dep[i] = dl * dev[i] / nrm;
                if (d == 2) {
                    double *ep = s->eps_p + c * 4;
                    ep[0] += dep[0]; ep[1] += dep[1]; ep[2] += dep[2]; ep[3] += dep[5];
                } else {
                    double *ep = s->eps_p + c * 6;
                    for (int i = 0; i < 6; i++) ep[i] += dep[i];
                }
                s->alpha[c] += dl;
                for (int i = 0; i < 6; i++) { ee[i] -= dep[i]; dev[i] -= dep[i]; }
                tr = ee[0] + ee[1] + ee[2];
                n2 = dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]
                   + 2.0 * (dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
            }
        }
        s->trE[c] = tr;
        s->devE2[c] = n2;
        if (s->sigma) {
            double sg[6];
            for (int i = 0; i < 6; i++) sg[i] = 2.0 * G * dev[i] + (i < 3 ? K * tr : 0.0);
            if (d == 2) {
                double *o = s->sigma + c * 4;
                o[0] = sg[0]; o[1] = sg[1]; o[2] = sg[2]; o[3] = sg[5];
            } else {
                double *o = s->sigma + c * 6;
                for (int i = 0; i < 6; i++) o[i] = sg[i];
            }
        }
    }
}

/* Mechanics at the current state: solve, then return map (R6). */
int or_mechanics(const or_params *p, or_state *s)
{
    long N = ncell(p);
    int d = p->ndim, nv = nvoigt(p);
    long n = N * d + nv;
    if (!p->mechanics) {
        for (long c = 0; c < N; c++) { s->trE[c] = 0.0; s->devE2[c] = 0.0; }
        if (s->sigma) memset(s->sigma, 0, sizeof(double) * N * (d == 2 ? 4 : 6));
        s->cg_iters = 0; s->cg_relres = 0.0;
        return 0;
    }
    double *lam = malloc(sizeof(double) * N), *mu = malloc(sizeof(double) * N);
    double *b = malloc(sizeof(double) * n), *x = malloc(sizeof(double) * n);
    or_cell_lame(p, s->theta, s->phig, lam, mu);
    or_mech_rhs(p, s, lam, mu, b);
    if (p->warm_start) {
        memcpy(x, s->u, sizeof(double) * N * d);
        memcpy(x + N * d, s->Ebar, sizeof(double) * nv);
    } else {
        memset(x, 0, sizeof(double) * n);
    }
    double rel = 0.0;
    s->cg_iters = or_pcg(p, lam, mu, b, x, &rel);
    s->cg_relres = rel;
    memcpy(s->u, x, sizeof(double) * N * d);
    memcpy(s->Ebar, x + N * d, sizeof(double) * nv);
    or_return_map(p, s);
    free(lam); free(mu); free(b); free(x);
    return s->cg_iters;
}

/*
 * Local part of delta psi / delta theta (R2; the driving forces of
 * (FiePhaDenEneFreDerPar) restricted to the solid pair):
 *   (1 - h(phi_g)) h'(theta) (A_f - A_w) + 2 w m'(theta)
 *   - eig0 (1 - h(phi_g)) h'(theta) tr(sigma),
 * A_a = c f_a(x_O) + K_a t^2 / 2 + G_a s (small-strain phase elastic energy,
 * t = tr eps_e, s = |dev eps_e|^2), tr(sigma) = 3 K t; the last term is
 * -sigma : d(eps_star)/d(theta).
 */
static double theta_force(const or_params *p, double th, double pg, double xO, double t, double s2)
{
    double W[3];
    weights(th, pg, W);
    double A[3], Kmix = 0.0;
    for (int a = 0; a < 3; a++) {
        double Ka, Ga;
        phase_moduli(p, a, &Ka, &Ga);
        A[a] = p->c_chem * or_f(a, xO) + 0.5 * Ka * t * t + Ga * s2;
        Kmix += W[a] * Ka;
    }
    double solid = 1.0 - or_h(pg);
    double trsig = 3.0 * Kmix * t;
    return solid * or_hp(th) * (A[0] - A[1]) + 2.0 * p->w * or_mp(th)
         - p->eig0 * solid * or_hp(th) * trsig;
}

/* exported for derivative pins */
double or_theta_force(const or_params *p, double th, double pg, double xO, double t, double s2)
{
    return theta_force(p, th, pg, xO, t, s2);
}

/* local bulk + well energy density of one cell (for derivative pins and F) */
double or_local_energy(const or_params *p, double th, double pg, double xO, double t, double s2)
{
    double W[3];
    weights(th, pg, W);
    double e = 0.0;
    for (int a = 0; a < 3; a++) {
        double Ka, Ga;
        phase_moduli(p, a, &Ka, &Ga);
        e += W[a] * (p->c_chem * or_f(a, xO) + 0.5 * Ka * t * t + Ga * s2);
    }
    return e + 2.0 * p->w * or_m(th);
}

/*
 * Right-hand sides of the field relations (FieRelDRI) at the current state,
 * with the coupling scalars already in s->trE / devE2: rate[0..N) = d theta/dt,
 * rate[N..2N) = d x_O/dt, rate[2N..3N) = d x_H/dt, rate[3N..4N) = d x_H2O/dt.
 */
void or_rates(const or_params *p, const or_state *s, double *rate)
{
    long N = ncell(p);
    double *lt = malloc(sizeof(double) * N), *lx = malloc(sizeof(double) * N);
    double *mu = malloc(sizeof(double) * N), *MO = malloc(sizeof(double) * N);
    double *DH = malloc(sizeof(double) * N), *DW = malloc(sizeof(double) * N);
    double *dxo = malloc(sizeof(double) * N), *dxh = malloc(sizeof(double) * N), *dxw = malloc(sizeof(double) * N);
    laplacian(p, s->theta, lt);
    laplacian(p, s->xO, lx);
    for (long c = 0; c < N; c++) {
        double W[3];
        weights(s->theta[c], s->phig[c], W);
        double x = s->xO[c];
        double m1 = 0.0, m2 = 0.0;
        for (int a = 0; a < 3; a++) {
            m1 += W[a] * p->c_chem * or_fp(a, x);
            m2 += W[a] * p->c_chem * or_fpp(a, x);
        }
        mu[c] = m1 - p->kappa_O * lx[c];                 /* mu_O = delta psi / delta x_O */
        double hg = W[2];
        double DO = (1.0 - hg) * p->D_O_s + hg * p->D_O_g;
        MO[c] = (m2 != 0.0) ? DO / m2 : 0.0;             /* M_O = D_O / psi_che'' (R3) */
        DH[c] = (1.0 - hg) * p->D_H_s + hg * p->D_H_g;  /* R4 */
        DW[c] = (1.0 - hg) * p->D_W_s + hg * p->D_W_g;
    }
    div_flux(p, MO, mu, dxo);
    div_flux(p, DH, s->xH, dxh);
    div_flux(p, DW, s->xW, dxw);
    for (long c = 0; c < N; c++) {
        double th = s->theta[c], pg = s->phig[c];
        /* delta psi / delta theta = local force - 2 eps Lap(theta) */
        double dpsi = theta_force(p, th, pg, s->xO[c], s->trE[c], s->devE2[c]) - 2.0 * p->eps_phi * lt[c];
        double r = or_m(pg) * p->k_for * s->xO[c] * s->xH[c];   /* (EmpModRea), (forward-k) */
        if (s->xW[c] >= 1.0) r = 0.0;                            /* Sec. 4.3 */
        rate[c] = -0.5 * p->L * s->mob[c] * dpsi;
        rate[N + c] = dxo[c] - r;
        rate[2 * N + c] = dxh[c] - 2.0 * r;
        rate[3 * N + c] = dxw[c] + r;
    }
    free(lt); free(lx); free(mu); free(MO); free(DH); free(DW); free(dxo); free(dxh); free(dxw);
}

/*
 * Explicit Euler update of (theta, x_O, x_H, x_H2O) by the field relations
 * (FieRelDRI) with the coupling scalars already in s->trE / devE2, followed by
 * the Dirichlet reset (R8).
 */
void or_fields_update(const or_params *p, or_state *s)
{
    long N = ncell(p);
    double dt = p->dt;
    double *rate = malloc(sizeof(double) * 4 * N);
    or_rates(p, s, rate);
    for (long c = 0; c < N; c++) {
        s->theta[c] = s->theta[c] + dt * rate[c];
        s->xO[c] = s->xO[c] + dt * rate[N + c];
        s->xH[c] = s->xH[c] + dt * rate[2 * N + c];
        s->xW[c] = s->xW[c] + dt * rate[3 * N + c];
    }
    for (long c = 0; c < N; c++) {
        if (s->mask && s->mask[c]) {
            s->removedW += s->xW[c];
            s->suppliedH += p->xH_bc - s->xH[c];
            s->xH[c] = p->xH_bc;
            s->xW[c] = 0.0;
        }
    }
    free(rate);
}

/* One or more full coupled steps (R6).  Returns the last CG iteration count. */
int or_step(const or_params *p, or_state *s, int nsteps)
{
    int it = 0;
    for (int n = 0; n < nsteps; n++) {
        it = or_mechanics(p, s);
        or_fields_update(p, s);
    }
    return it;
}

/*
 * Discrete free energy: cell sum of bulk + well + elastic energy density,
 * plus face sums of eps |grad theta|^2 and (kappa/2)|grad x_O|^2
 * (DenEneFreBul), (DenEneFreInt), R2.
 */
double or_free_energy(const or_params *p, const or_state *s)
{
    long N = ncell(p);
    double F = 0.0;
    for (long c = 0; c < N; c++) {
        F += or_local_energy(p, s->theta[c], s->phig[c], s->xO[c], s->trE[c], s->devE2[c]);
        for (int ax = 0; ax < p->ndim; ax++) {
            long cp = nbr(p, c, ax, +1);
            double gt = s->theta[cp] - s->theta[c];
            double gx = s->xO[cp] - s->xO[c];
            F += p->eps_phi * gt * gt + 0.5 * p->kappa_O * gx * gx;
        }
    }
    return F;
}

/* plain sums used by the balance pins */
void or_sums(const or_params *p, const or_state *s, double *out3)
{
    long N = ncell(p);
    double a = 0.0, b = 0.0, c3 = 0.0;
    for (long c = 0; c < N; c++) { a += s->xO[c]; b += s->xH[c]; c3 += s->xW[c]; }
    out3[0] = a; out3[1] = b; out3[2] = c3;
}
