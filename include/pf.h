/*
 * pf.h -- C ABI of the GB300 (sm_103a) library that advances the
 * chemo-mechanical phase-field model of wuestite-to-iron reduction by
 * hydrogen (Bai, Mianroodi et al., arXiv 2111.11538).
 *
 * One call of pf_step advances every field by one explicit time step per
 * requested step:
 *   1. mechanics: small-strain elasticity with the transformation eigenstrain
 *      (Sec. 2.2, eq. RulFloDefLocAlt, linearised) and the plastic strain,
 *      solved for the periodic displacement and the mean strain by CG on
 *      Q1 voxel elements (Sec. 2.4, div P = 0), preconditioned by a
 *      geometric-multigrid V-cycle or the Jacobi diagonal (precond below);
 *   2. per-cell stress and J2 radial return (Sec. 2.3, eq. PlaTwoJ;
 *      Sec. 2.4, eq. RulFloPla);
 *   3. explicit Euler update of the solid order parameter and of the oxygen,
 *      hydrogen and water fractions with the reaction source terms
 *      (Sec. 2.4, eq. FieRelDRI; Sec. 2.3.1, eqs. EmpModRea, forward-k),
 *      then the reset of the supply (Dirichlet) cells (Sec. 4.3).
 * Gas fraction phi_g = 1 - phi_f - phi_w is held fixed; the solid is split by
 * the order parameter theta = phi_f / (phi_f + phi_w), which evolves.  This
 * is the library's reading of Sec. 2.2 and Sec. 2.4: the paper's two
 * Allen-Cahn relations for phi_f and phi_w, taken literally with phi_g
 * dependent and the absolute CALPHAD energies, create gas inside ferrite /
 * wuestite interfaces at the rate L h'(phi) (psi_f + psi_w); with phi_g held
 * and the weights W_f = (1 - h(phi_g)) h(theta), W_w = (1 - h(phi_g))
 * (1 - h(theta)), W_g = h(phi_g) in place of h(phi_a), every two-phase
 * interface keeps the paper's energies and the theta relation on a ferrite /
 * wuestite interface is the paper's phi_f relation minus its phi_w relation,
 * over two.
 *
 * Conventions
 *   - Grids are periodic, dx = 1, row-major with x fastest: index
 *     i + nx*(j + ny*k).  2D: nz is ignored (treated as 1).
 *   - Host arrays are always FP64.  PF_MIXED stores fields in FP32 on the
 *     device and converts on the way in and out.
 *   - Every function returns an int status (PF_OK on success) and never
 *     throws; pf_last_error(h) gives a text for the last failure.
 *   - The library owns all device memory it allocates; it never keeps a
 *     caller pointer after a call returns.
 *   - Calls on one handle must not overlap; different handles are
 *     independent.
 */
#ifndef PF_H
#define PF_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PF_OK = 0,
    PF_EINVAL = 1,      /* bad argument or configuration                       */
    PF_ENOMEM = 2,      /* device allocation failed                            */
    PF_ECUDA = 3,       /* a CUDA call failed                                  */
    PF_ENOTCONV = 4,    /* a CG solve hit cg_maxit; the step was still taken   */
    PF_ENONFINITE = 5,  /* a non-finite value appeared in the fields           */
    PF_ETIMEOUT = 6,    /* a bounded device-side wait gave up (no hang)        */
    PF_ESTATE = 7       /* call out of order (e.g. pf_step before set_fields)  */
};

enum { PF_FP64 = 0, PF_MIXED = 1 };            /* device storage / arithmetic */
enum { PF_WS_ZERO = 0, PF_WS_PREV = 1, PF_WS_LEARNED = 2, PF_WS_EXTRAP = 3, PF_WS_EXTRAP2 = 4 };   /* CG guess */
enum { PF_HOST = 0, PF_DEVICE = 1 };           /* where caller arrays live    */
enum { PF_PC_AUTO = 0, PF_PC_JACOBI = 1, PF_PC_MG = 2 };   /* CG preconditioner      */

/* Nondimensional model parameters (energy in units of the solid Young's
 * modulus, length in cells, time in 1/(L E_s)); see Sec. 3 / Table 1. */
typedef struct {
    double c_chem;      /* R theta / (V_mol E_s): scale of the CALPHAD energies (Sec. 3.1) */
    double w;           /* double-well height w_alpha                                   */
    double eps_phi;     /* gradient-energy coefficient epsilon_alpha                    */
    double kappa_O;     /* oxygen gradient-energy coefficient kappa_O                  */
    double L;           /* phase mobility L_alpha                                       */
    double D_O_s, D_O_g, D_H_s, D_H_g, D_W_s, D_W_g;   /* solid / gas diffusivities     */
    double k_for;       /* reaction constant k_for                                      */
    double xH_bc;       /* hydrogen fraction held on supply cells                       */
    double E_s, nu;     /* solid Young's modulus and Poisson ratio                      */
    double E_g_ratio;   /* gas / solid stiffness ratio                                  */
    double eig0;        /* linearised transformation strain of ferrite (e.g. -0.05)     */
    double sigma_Y;     /* initial yield stress                                         */
    double H_hard;      /* isotropic hardening modulus                                  */
    double prestress;   /* prescribed mean stress = -prestress * I                      */
} pf_params;

typedef struct {
    int ndim;           /* 2 (plane strain) or 3                                        */
    int nx, ny, nz;     /* grid size, each >= 2                                         */
    int precision;      /* PF_FP64 or PF_MIXED                                          */
    int mechanics;      /* 0: skip the solve (coupling terms zero)                      */
    int plasticity;     /* 0: elastic, 1: J2 radial return                              */
    int warm_start;     /* PF_WS_ZERO, PF_WS_PREV, PF_WS_LEARNED (see pf_attach_unet),
                           PF_WS_EXTRAP: 2 u_n - u_{n-1} (u and the mean strain) from the
                           third step after pf_set_fields on (before: PF_WS_PREV), or
                           PF_WS_EXTRAP2: 3 u_n - 3 u_{n-1} + u_{n-2} from the fourth
                           step on (before: the lower orders)                          */
    int cg_maxit;       /* CG iteration cap per step (> 0)                              */
    double cg_rtol;     /* stop when ||r||_2 <= cg_rtol ||b||_2                         */
    double dt;          /* time step; <= 0 selects 0.2 x the stable limit               */
    pf_params p;
    int pcg_tile;       /* node tile of the PCG sweep: 0 = the library's choice for the
                           grid size (measured per size class), 1 = 32x8 (2D) / 16x4x4
                           (3D), 2 = 32x16 / 32x4x2.  Results agree to rounding.        */
    int precond;        /* CG preconditioner: PF_PC_AUTO (the library's choice: PF_PC_MG
                           for grids whose sizes are all divisible by 4 and >= 32, else
                           Jacobi; one choice for a whole batch), PF_PC_JACOBI
                           (diagonal), or PF_PC_MG (one geometric multigrid V-cycle per
                           iteration, Chebyshev-smoothed, on grids halved while all
                           sizes stay even and the coarse grid keeps >= 8 nodes per
                           axis).  Both solve to the same cg_rtol; iteration counts
                           differ.                                                     */
    int fused_chunk;    /* planes per work item of the fused field update, which marches
                           along the slowest axis (z in 3D, y in 2D): 0 = the library's
                           choice (a cost model whose start-up weight is measured per
                           dimension), > 0 = that many planes.  Results are identical. */
} pf_config;

/* Field arrays, FP64, cell-major.  Any pointer may be NULL (skipped).
 *   phi_f, phi_w, x_O, x_H, x_H2O : N each
 *   u       : N*ndim, nodal periodic displacement, u[n*ndim + c]; node n is the
 *             lower corner of cell n
 *   Ebar    : 3 (2D: xx, yy, 2xy) or 6 (3D: xx, yy, zz, 2yz, 2xz, 2xy) mean strain
 *   eps_p   : N*4 (2D: xx, yy, zz, xy) or N*6 (3D: xx, yy, zz, yz, xz, xy)
 *   alpha   : N accumulated plastic strain
 *   sigma   : output only, N*4 / N*6 like eps_p (from the last step's return map)
 *   mobility: input only, N factor on L (grain scatter)
 *   dirichlet: input only, N bytes, 1 = supply cell
 *   theta   : N, the evolving solid order parameter, and
 *   phi_g   : N, the gas fraction the library holds fixed (the fields of
 *             Sec. 2.4 as the library advances them: theta, phi_g, x_O,
 *             x_H, x_H2O).  On output their values; on input, if given, they
 *             replace phi_f / (phi_f + phi_w) and 1 - phi_f - phi_w, which
 *             round, and which cannot recover theta in cells without solid
 *             (phi_g = 1), where theta still evolves and enters its
 *             neighbours' Laplacian.  A pf_get_fields of every field
 *             followed by pf_set_fields (plus mobility and dirichlet)
 *             restores the state exactly in FP64.
 * With PF_DEVICE every pointer is device memory holding the same FP64 layout. */
typedef struct {
    double *phi_f, *phi_w, *x_O, *x_H, *x_H2O;
    double *u, *Ebar, *eps_p, *alpha, *sigma;
    double *mobility;
    unsigned char *dirichlet;
    double *theta, *phi_g;
} pf_fields;

typedef struct {
    double sum_O, sum_H, sum_H2O;   /* FP64 sums over cells of x_O, x_H, x_H2O    */
    double removed_H2O;             /* water removed on supply cells, cumulative   */
    double supplied_H;              /* hydrogen added on supply cells, cumulative  */
    double sum_O_init;              /* sum of x_O at pf_set_fields                 */
    double reduction_degree;        /* 1 - sum_O / sum_O_init (Sec. 4.2.1)         */
    double cg_rel_residual;         /* last solve: ||r|| / ||b||                   */
    int cg_iters_last, cg_iters_max;/* last solve / max over the last pf_step call */
    long long cg_iters_total;       /* all solves since pf_set_fields              */
    long long steps;                /* steps taken since pf_set_fields             */
    double dt;                      /* time step of the last step (pf_step: cfg dt; pf_step_implicit: its own) */
    int status;                     /* sticky status of the last pf_step call      */
    int precond;                    /* preconditioner in use: PF_PC_JACOBI or PF_PC_MG */
    int mg_levels;                  /* levels of the multigrid hierarchy (0: Jacobi)   */
    double reduction_rate;          /* rate of the reduction degree over the last step,
                                       -(sum_O,n - sum_O,n-1) / (sum_O_init dt)
                                       (Sec. 4.2.1); 0 before the first step        */
} pf_diag;

typedef struct pf_handle pf_handle;

/* Allocate device state for one grid: the fields of the model (Sec. 2.4:
 * order parameter, gas fraction, the three species fractions; Sec. 2.3: the
 * plastic strain and hardening variable; the displacement of div P = 0) and
 * the solver's work arrays.  Validates cfg (PF_EINVAL), chooses dt
 * (pf_dt_stable x 0.2 when cfg->dt <= 0), allocates (PF_ENOMEM).  *out is set
 * to NULL on failure. */
int pf_create(const pf_config *cfg, pf_handle **out);

/* Copy in the state that the field relations of Sec. 2.4 evolve (the
 * initial conditions of Sec. 4: phases, species fractions, and the
 * mechanical state).  phi_f, phi_w, x_O, x_H, x_H2O are required; the rest
 * default to: theta = phi_f / (phi_f + phi_w) (0 without solid),
 * phi_g = 1 - phi_f - phi_w, u = 0,
 * Ebar = 0, eps_p = 0, alpha = 0, mobility = 1, dirichlet = 0.  Resets the
 * step counter and the diagnostics.  The extrapolation history of the CG
 * guess (PF_WS_EXTRAP, PF_WS_EXTRAP2) and, for PF_MIXED, the FP64 copy of
 * the displacement are reset too, unless u equals, bit for bit, the
 * handle's displacement as pf_get_fields exports it: a state round trip
 * through the host then continues the solver's trajectory (the guess only
 * sets where each solve starts; every solve still meets cfg->cg_rtol). */
int pf_set_fields(pf_handle *h, const pf_fields *f, int where);

/* Advance nsteps >= 0 steps on cudaStream (NULL: the handle's own stream),
 * blocking until they are done.  Returns PF_ENOTCONV if any CG solve stopped
 * at cg_maxit (the steps are still taken), PF_ENONFINITE if a non-finite
 * value appeared, PF_ETIMEOUT if a bounded device wait gave up.  With
 * per-kernel timing off, each step is replayed from a CUDA graph captured at
 * the first step after pf_create / pf_set_fields (direct launches if the
 * capture fails); the results are the same either way. */
int pf_step(pf_handle *h, int nsteps, void *cudaStream);

/* Backward-Euler steps of the field relations.  The paper integrates the
 * relations of Sec. 2.4 in time by backward Euler and solves each step by
 * Newton's method (Sec. 2.4, closing paragraph).  One step here: the
 * mechanics of pf_step at the current state (the solve and the J2 return,
 * whose coupling scalars tr eps_e, |dev eps_e|^2 are then held over the
 * step), then Newton's method on
 *     F(y) = y - y_n - dt R(y),   y = (theta, x_O, x_H, x_H2O),
 * R the right-hand sides of pf_step's update (the same fluxes, driving force
 * and reaction; the reaction switch at x_H2O >= 1 evaluated at the new
 * state), with x_H = x_H,bc and x_H2O = 0 held on supply cells at the new
 * time level; the water removed and the hydrogen supplied there are the
 * differences from what those cells' own relations would give, so the
 * balances of pf_get_diagnostics hold as for explicit steps.  Newton stops
 * when max |F| <= newton_tol, or when an update computed from a linear solve
 * that met gmres_rtol moves no entry by more than newton_tol * max(1, max |y|).
 * Each Newton iteration solves J delta = F by
 * restarted GMRES, matrix-free (each product J z is the directional
 * derivative of F along z, evaluated in forward mode), preconditioned on the right by pc_degree Chebyshev steps
 * (Jacobi-scaled) on each field's own block: theta's gradient term and the
 * species' diffusion with the phase-interpolated diffusivities.  Single-grid
 * handles with precision PF_FP64 only.  Blocking.
 * Returns PF_EINVAL (batch or mixed handle, invalid opts), PF_ESTATE (no
 * fields), PF_ENOTCONV (Newton did not meet its stopping rule within
 * newton_maxit: that step is not taken -- the fields stay at its start while
 * the mechanical state has advanced -- and the call stops; or a CG solve hit
 * cg_maxit), PF_ENONFINITE, PF_ETIMEOUT as pf_step.  stats may be NULL. */
typedef struct {
    double dt;          /* time step (> 0), free of the explicit limit              */
    double newton_tol;  /* Newton stopping tolerance (> 0), see above                */
    int newton_maxit;   /* Newton iterations per step (>= 1)                         */
    double gmres_rtol;  /* each linear solve to ||J delta - F|| <= gmres_rtol ||F||  */
    int gmres_restart;  /* Krylov vectors per GMRES cycle, 1 .. 60                   */
    int gmres_maxit;    /* GMRES iterations per Newton iteration (>= 1)              */
    int pc_degree;      /* Chebyshev steps of the block preconditioner, 0 (none) .. 64 */
    int pc_precision;   /* the preconditioner's arithmetic: PF_FP64, or PF_MIXED (FP32
                           coefficients and iterates, one fused kernel per Chebyshev
                           step; grids of fewer than 2^29 cells).  GMRES, the
                           Jacobian-vector products and F stay FP64 either way.   */
} pf_implicit_opts;

typedef struct {
    int newton_iters;          /* Newton iterations of the last step           */
    int newton_iters_total;    /* over all steps of the call                   */
    long long gmres_iters;     /* GMRES iterations over all steps of the call  */
    double residual;           /* max |F| at the end of the last step          */
} pf_implicit_stats;

int pf_step_implicit(pf_handle *h, int nsteps, const pf_implicit_opts *opts, pf_implicit_stats *stats,
                     void *cudaStream);

/* Finite-strain elastic equilibrium with the transformation stretch, for
 * given order parameter and gas fraction (Sec. 2.2: F_R = F_T F_P with
 * F_T = d_T^(1/3) I, d_T = 1 - W_f omega (RulFloDefLocAlt); the energy
 * d_T sum_a W_a phi_a(F_E), F_E = F F_R^-1, with the neo-Hooke phase energy
 * phi_a = K_a/4 (J_E^2 - 1 - 2 ln J_E) + G_a/2 (J_E^(-2/3) |F_E|^2 - 3)
 * (DenEneFreIntElaPha), K_a, G_a from cfg->p (E_s, nu, E_g_ratio); Sec. 2.4:
 * Div P = 0), with F_P = I.  The library's readings: P is the derivative of
 * that energy (half the printed stress); Q1 voxel elements with 2^d Gauss
 * points on the periodic grid of cfg (2D plane strain, F_33 = 1); F = Fbar +
 * grad u, Fbar symmetric, the symmetric part of the mean first Piola stress
 * prescribed (pbar, d x d row-major; NULL: -cfg->p.prestress I); u = 0 at
 * node 0.  Newton's method over opts->nload equal steps of omega, each
 * Newton system solved by conjugate gradients on the energy's Hessian
 * (products evaluated in forward mode, in FP64 or FP32 by opts->precision;
 * the CG scalars stay on the device and the host reads them every 16
 * iterations) with the small-strain diagonal as preconditioner; stops when
 * max |residual| (FP64) <= opts->newton_tol.
 *   theta, phi_g : host arrays of N cells (cell-major, x fastest)
 *   u            : out, host, N * ndim (u[n * ndim + c], node n = lower
 *                  corner of cell n)
 *   Fbar         : out, host, ndim * ndim row-major
 * Uses the current device; allocates and frees its own device memory;
 * blocking.  Returns PF_EINVAL (arguments), PF_ENOMEM, PF_ECUDA, PF_ENOTCONV
 * (Newton over newton_maxit in a load step; stats still filled);
 * pf_fs_last_error() gives the text.  Not part of the explicit step. */
typedef struct {
    int nload;          /* load steps of omega (>= 1)                    */
    int newton_maxit;   /* Newton iterations per load step (>= 1)        */
    double newton_tol;  /* max |residual| at convergence (> 0)           */
    int cg_maxit;       /* CG iterations per Newton system (>= 1)        */
    double cg_rtol;     /* CG relative residual per Newton system (0, 1) */
    int precision;      /* PF_FP64: Hessian-vector products in FP64;
                           PF_MIXED: in FP32 (the residual stays FP64, so
                           the solution is the same; CG then stops at
                           max(cg_rtol, 1e-5), an inexact Newton step)     */
} pf_fs_opts;

typedef struct {
    int newton_iters;   /* over all load steps                           */
    long long cg_iters; /* over all Newton systems                       */
    double residual;    /* max |residual| at the end                     */
    double hvp_ms;      /* device time of the Hessian-vector product
                           kernel (CUDA events around each launch)       */
    long long hvp_launches; /* its launches that did work              */
} pf_fs_stats;

int pf_finite_strain_solve(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                           const double *pbar, const pf_fs_opts *opts, double *u, double *Fbar,
                           pf_fs_stats *stats);

/* One staggered finite-strain mechanics step (the library's reading of the
 * paper's plastic flow, as for small strain): the equilibrium above with the
 * plastic deformation FP of every cell (F_E = d_T^(-1/3) F FP^-1), then, if
 * cfg->plasticity, one multiplicative J2 update per cell at its cell-centre
 * deformation (Sec. 2.3 PlaTwoJ, Sec. 2.4 RulFloPla: backward Euler with the
 * exponential map, FP_new = exp(dl N) FP, N = dev M / |dev M| at the end of
 * the step, |dev M| = sqrt(2/3) (sigma_Y + H_hard (epsP + dl)); M the Mandel
 * stress d_T (K/2 (det C_E - 1) I + G dev(det C_E^(-1/3) C_E)), the
 * derivative of the energy above), which keeps det FP = 1.
 *   FP   : in/out, host, N * 9 (3 x 3 row-major per cell; identity to start)
 *   epsP : in/out, host, N accumulated plastic strain
 * Other arguments and errors as pf_finite_strain_solve; PF_ENOTCONV also
 * when a cell's update does not converge (that cell keeps its FP). */
int pf_finite_strain_step(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                          const double *pbar, const pf_fs_opts *opts, double *u, double *Fbar, double *FP,
                          double *epsP, pf_fs_stats *stats);

/* The multiplicative J2 update above for n independent points (host arrays):
 * F (n * 9 total deformation gradients), FP (n * 9, in/out), epsP (n,
 * in/out), K, G, dT (n each: bulk and shear moduli, d_T), sigma_Y, H. */
int pf_fs_return_map(int n, const double *F, double *FP, double *epsP, const double *K, const double *G,
                     const double *dT, double sigma_Y, double H);

/* The elastic part of the order parameter's driving force per cell,
 * d psi / d theta at fixed deformation and plastic deformation (the
 * derivative of the energy above through W_f in d_T and through the
 * mixture moduli), at each cell-centre deformation of the state (u, Fbar) of
 * pf_finite_strain_solve / _step; FP may be NULL (identity).  force: out,
 * host, N.  The coupled explicit step adds -(L/2) mob times it to theta's
 * rate in place of the small-strain coupling. */
int pf_fs_elastic_force(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                        const double *u, const double *Fbar, const double *FP, double *force);

/* The same force as a small-strain coupling scalar: the solid phases share
 * their moduli, so d psi / d theta = -Omega (1 - h(phi_g)) h'(theta)
 * d psi / d d_T, and the field update's elastic term
 * -3 eig0 (1 - h(phi_g)) h'(theta) K_mix tr eps_e equals it for
 *   trE = Omega (d psi / d d_T) / (3 eig0 K_mix),
 *   K_mix = (1 - h(phi_g)) K_s + h(phi_g) K_g
 * (0 where K_mix = 0).  trE: out, host, N; hand it to pf_set_coupling (with
 * devE2 = NULL) on a mechanics = 0 handle to step the fields with the
 * finite-strain force.  PF_EINVAL also when cfg->p.eig0 == 0. */
int pf_fs_coupling(const pf_config *cfg, const double *theta, const double *phi_g, double omega,
                   const double *u, const double *Fbar, const double *FP, double *trE);
const char *pf_fs_last_error(void);

/* The coupling scalars of the field update (the elastic part of the order
 * parameter's driving force, Sec. 2.4 with the small-strain energy of
 * Sec. 2.2: tr eps_e and |dev eps_e|^2 per cell) supplied by the caller, for
 * handles created with mechanics = 0, whose steps then run the field update
 * alone with these values: for example the equivalent coupling of another
 * mechanics model (pf_fs_coupling).  trE, devE2: N values each, FP64, on the
 * host or the device (where); NULL sets zero.  They stay until the next call
 * or pf_set_fields (which zeroes them).  Blocking.  Returns PF_EINVAL
 * (batch handle, where), PF_ESTATE (mechanics on, no fields), PF_ECUDA. */
int pf_set_coupling(pf_handle *h, const double *trE, const double *devE2, int where);

/* Copy the current state (the fields of Sec. 2.4 and the mechanical state)
 * out into caller arrays (FP64); NULL members are skipped.  sigma is the
 * stress of the last return map (Sec. 2.3).  mobility / dirichlet are
 * ignored. */
int pf_get_fields(pf_handle *h, pf_fields *out, int where);

int pf_get_diagnostics(pf_handle *h, pf_diag *out);

/* Discrete free energy of the current state (FP64; cell bulk + well +
 * elastic energy, face gradient energies), Sec. 2.2. */
int pf_free_energy(pf_handle *h, double *out);

/* Stable explicit time step for cfg (host only, no GPU needed). */
double pf_dt_stable(const pf_config *cfg);

/* Per-kernel device timing (CUDA events on the launch stream) and launch
 * counts, for profiling.  Kernel classes of one step: */
enum { PF_K_SETUP = 0,    /* moduli and eigenstress per cell              */
       PF_K_CG = 1,       /* persistent PCG solve (one launch per step)   */
       PF_K_RETURN = 2,   /* stress and J2 return per cell                */
       PF_K_UPDATE = 3,   /* fused mu_O, M_O and explicit Euler update    */
       PF_K_WARM = 4,     /* learned warm start: inference and guess      */
       PF_K_NCLASS = 5 };

typedef struct {
    int enabled;
    long long launches;            /* all kernels launched by pf_step since reset */
    long long count[PF_K_NCLASS];  /* launches per class (timed only if enabled)  */
    double ms[PF_K_NCLASS];        /* summed device time per class, ms            */
    long long cg_iters;            /* CG iterations of the timed solves           */
    long long graph_steps;         /* steps replayed from a captured CUDA graph   */
} pf_profile;

/* Enable (on != 0) or disable event timing; either way the counters reset. */
int pf_profile_enable(pf_handle *h, int on);
int pf_profile_read(pf_handle *h, pf_profile *out);

/* ------------------------------------------------------------------------
 * Batches: many independent instances advanced by the same launches.
 *
 * Each instance is one simulation of the model above (the paper's
 * micrographs are independent particles and pores, Sec. 4.3); a batch steps
 * all of them with one launch per kernel class and step, the blocks of every
 * launch split between the instances.  Instances may differ in grid size,
 * parameters, CG tolerance and fields; they must share ndim, precision and
 * whether mechanics is on (PF_EINVAL otherwise).
 *
 * pf_batch_create: cfgs[0..n-1] as for pf_create; *out is a batch handle
 *   (NULL on failure; pf_last_error(NULL) names the failing instance).
 *   PF_EINVAL at the first pf_step if the instances need more co-resident CG
 *   blocks than the device holds (one per instance at least).
 * On a batch handle, pf_step advances every instance (all must have fields,
 *   else PF_ESTATE) and returns the worst status over the instances
 *   (PF_ETIMEOUT > PF_ENONFINITE > PF_ENOTCONV); pf_profile_*,
 *   pf_device_bytes (sum over instances), pf_last_error and pf_destroy work
 *   as for one instance.  pf_set_fields, pf_get_fields, pf_get_diagnostics
 *   and pf_free_energy return PF_EINVAL: use the pf_batch_ calls with the
 *   instance index i (0 <= i < n, PF_EINVAL otherwise), which have the
 *   semantics of their single-instance counterparts.
 * pf_batch_size: n for a batch handle, 1 for a single handle, 0 for NULL. */
int pf_batch_create(const pf_config *cfgs, int n, pf_handle **out);
int pf_batch_size(const pf_handle *h);
int pf_batch_set_fields(pf_handle *h, int i, const pf_fields *f, int where);
int pf_batch_get_fields(pf_handle *h, int i, pf_fields *out, int where);
int pf_batch_get_diagnostics(pf_handle *h, int i, pf_diag *out);

/* ------------------------------------------------------------------------
 * Learned warm start (PF_WS_LEARNED).  Attach a network (include/pf_unet.h;
 * 4 input channels, the grid's ndim outputs, each grid size divisible as
 * that header states, else PF_EINVAL) to a handle (every instance of a
 * batch).  Before each solve the network maps the cells' ferrite weight W_f,
 * gas weight W_g, prestress / |eig0| and ferrite-weight rate
 * (W_f - W_f,prev) / dt to y ~ (du/dt) / |eig0|, and the solve starts from
 *   u_prev + |eig0| dt y
 * (on the first step after pf_set_fields, which has no W_f,prev, from
 * u_prev).  The PCG still runs to cg_rtol, so results do not depend on the
 * network's accuracy.  Without a network PF_WS_LEARNED behaves as
 * PF_WS_PREV.  The network must stay alive while attached; net = NULL
 * detaches.  The inference runs inside pf_step (kernel class PF_K_WARM). */
struct pf_unet;
int pf_attach_unet(pf_handle *h, struct pf_unet *net);

/* Self-test of the bounded device-side wait that every PCG grid barrier
 * uses: one thread waits for a word that nothing updates, at most
 * spin_limit polls (1 .. 2^24, ~100 ns apart), and the kernel then returns
 * with PF_ETIMEOUT recorded -- the path a barrier takes when a peer block
 * never arrives.  Returns PF_ETIMEOUT when the wait timed out as designed
 * (the CUDA context stays usable), PF_EINVAL for a bad limit, PF_ECUDA /
 * PF_ENOMEM on CUDA failures. */
int pf_selftest_wait(long long spin_limit);

/* Device memory held by the handle, bytes. */
long long pf_device_bytes(const pf_handle *h);

const char *pf_last_error(const pf_handle *h);
void pf_destroy(pf_handle *h);

/* ------------------------------------------------------------------------
 * Field update that allocates no device memory.  (The paper has no
 * counterpart: this entry point exists for callers of the library.)
 *
 * For callers that cannot call cudaMalloc at the point of use: runtimes that
 * hand out a fixed device-memory budget once and forbid later allocations,
 * and hosts that must leave the process's allocator untouched.
 *
 * One explicit Euler step of the phase and species fields -- the part of
 * pf_step after the mechanics -- with the coupling scalars tr(eps_e) and
 * |dev eps_e|^2 given per cell (trE, devE2; NULL means zero, i.e. no
 * mechanics).  All pointers are DEVICE memory, FP64, laid out as in
 * pf_fields: `in` supplies phi_f, phi_w, x_O, x_H, x_H2O (required),
 * mobility and dirichlet (optional: 1 and 0); `out` receives phi_f, phi_w,
 * x_O, x_H, x_H2O (required; must not alias `in`).  dt is cfg->dt, or 0.2 x
 * pf_dt_stable(cfg) when cfg->dt <= 0; precision, mechanics and CG fields of
 * cfg are ignored (the update runs in FP64).  Work is queued on cudaStream
 * (NULL: the legacy default stream) and the call returns when it is done.
 *
 * Working arrays live in one fixed device array of the library (about
 * 8 * PF_STATIC_MAX_CELLS doubles plus about 0.2 MB; 4.5 MB), which every device
 * that loads the library keeps until the process exits.  Grids with more
 * than PF_STATIC_MAX_CELLS cells are rejected with PF_EINVAL.  The first call
 * on a device looks the array's device address up (cudaGetSymbolAddress)
 * and caches it for the life of the process; make that first call before
 * any stream capture, and do not use the library across a cudaDeviceReset
 * (the array moves to a new address in the new context).  Every call shares the
 * array and clears what must start at zero: calls whose GPU work overlaps
 * (other streams or host threads) race, so serialise them.
 * Returns PF_OK, PF_EINVAL, PF_ECUDA or PF_ENONFINITE; the text of the last
 * failure on this host thread is pf_static_last_error().
 * ------------------------------------------------------------------------ */
#define PF_STATIC_MAX_CELLS 65536
int pf_fields_update_static(const pf_config *cfg, const pf_fields *in, const double *trE,
                            const double *devE2, pf_fields *out, void *cudaStream);
const char *pf_static_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
