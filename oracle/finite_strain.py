"""Finite-strain elastic equilibrium with the transformation deformation
(test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import this module; it shares no code with the CUDA library.

Sec. 2.2 of the paper: the residual deformation F_R = F_T F_P with
F_T = d_T^(1/3) I and d_T = 1 - h(phi_f) Omega_f (RulFloDefLocAlt); the
elastic energy per reference volume psi_ela = d_T sum_a h(phi_a) phi_a(F_E)
with F_E = (grad chi) F_R^-1 (DenEneFreElaPha, DenEneFreBulEla); and the
neo-Hooke phase energy phi_a(F_E) = K_a/4 (J_E^2 - 1 - 2 ln J_E)
+ G_a/2 (|uni F_E|^2 - 3), uni A = A / det(A)^(1/3) (DenEneFreIntElaPha).
Mechanical equilibrium Div P = 0 (Sec. 2.4, FieRelDRI) is the stationarity
of the total elastic energy.

Readings (listed in the design notes as F1-F6):
  F1  The equilibrium is solved for a given plastic deformation F_P per
      cell (identity unless a plastic step has run, F8).
  F2  P = d psi_ela / d(grad chi), the derivative of the printed energy,
      whose linearisation at F = I has K_a and G_a as the bulk and shear
      moduli that Table 1 names.  The printed first Piola stress (StsRelMod)
      is twice this derivative; the energy is taken as the authority.
  F3  h(phi_a) -> the phase weights W_a of R2; d_T = 1 - W_f Omega.
  F4  2D is plane strain: F_33 = 1; 3D grids use 8-node hexahedra.
  F5  grad chi = Fbar + grad u on the periodic box; the mean deformation
      gradient Fbar is symmetric (no macroscopic rotation), and the
      symmetric part of the mean first Piola stress equals -prestress I.
  F6  Q1 voxel elements, 2^d Gauss points, nodes at cell corners (node
      i + nx (j + ny k) is the lower corner of cell (i, j, k)); the rigid
      translation is fixed by u = 0 at node 0.
  F7  The plastic flow dF_P/dt = L_P F_P (RulFloPla) is integrated by
      backward Euler with the exponential map, which keeps F_P isochoric
      (Sec. 2.2), with the flow direction taken at the end of the step;
      the Mandel stress follows F2 (half the printed StsRelMod form).
      ``return_map`` is the per-point update.
  F8  Plasticity is staggered as the small-strain step (R6): the
      equilibrium is solved with the plastic deformation of the step's
      start, then each cell takes one update on its cell-centre
      deformation (``Problem.mechanics_step``).
  F9  The elastic part of the order parameter's driving force is
      d psi_ela / d theta at fixed deformation and F_P, evaluated at each
      cell's centre deformation after the step's plastic update (as the
      small-strain coupling scalars, R6); ``CoupledSim`` is the explicit
      step with that force.
The solution is found by Newton's method on the residual (analytic P,
Jacobian by central differences, dense solve), with the transformation
applied in ``nload`` equal increments of Omega; it stops when the largest
residual entry is at most ``tol``.  Small grids only.

Pins (tests/test_oracle_finite_strain.py): P against central differences of
the energy, frame indifference, the small-strain moduli, the homogeneous
transformation and uniaxial-stress states against one-dimensional closed
forms (in 3D the transformation is exactly stress-free), the small-strain
oracle as Omega -> 0 in 2D and 3D; for the return map: det F_P = 1,
the yield condition after a plastic step, elastic unloading, objectivity,
the small-strain radial return as the strain vanishes, first-order
convergence along a shear path.
"""
import numpy as np

_GA, _GB = 0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)


def h(x):
    return x ** 3 * (6.0 * x * x - 15.0 * x + 10.0)


def weights(theta, phig):
    """W_f, W_w, W_g of R2 (each the shape of theta)."""
    hg, ht = h(phig), h(theta)
    return (1.0 - hg) * ht, (1.0 - hg) * (1.0 - ht), hg


def psi(F, K, G, dT, FPinv=None):
    """Elastic energy per reference volume at deformation gradient F
    (..., 3, 3), mixture moduli K, G (sum of W_a K_a, W_a G_a), d_T and the
    inverse plastic deformation (identity when None)."""
    s = dT ** (-1.0 / 3.0)
    FE = s[..., None, None] * F if np.ndim(s) else s * F
    if FPinv is not None:
        FE = FE @ FPinv
    JE = np.linalg.det(FE)
    I1 = np.einsum("...ij,...ij->...", FE, FE)
    return dT * (0.25 * K * (JE * JE - 1.0 - 2.0 * np.log(JE)) + 0.5 * G * (JE ** (-2.0 / 3.0) * I1 - 3.0))


def piola(F, K, G, dT, FPinv=None):
    """First Piola stress d psi / d F (F2), same shapes as psi:
    d_T s (d phi / d F_E) F_P^-T with F_E = s F F_P^-1, s = d_T^(-1/3)."""
    s = np.asarray(dT ** (-1.0 / 3.0))
    FE = s[..., None, None] * F
    if FPinv is not None:
        FE = FE @ FPinv
    JE = np.linalg.det(FE)
    I1 = np.einsum("...ij,...ij->...", FE, FE)
    FEiT = np.swapaxes(np.linalg.inv(FE), -1, -2)
    dphi = (0.5 * K * (JE * JE - 1.0))[..., None, None] * FEiT \
        + (G * JE ** (-2.0 / 3.0))[..., None, None] * (FE - (I1 / 3.0)[..., None, None] * FEiT)
    if FPinv is not None:
        dphi = dphi @ np.swapaxes(FPinv, -1, -2)
    return (dT * s)[..., None, None] * dphi


def _shape_grads(d, points):
    """dN[g, a, k]: derivative along x_k of local shape function a (bit l of
    a: offset along axis l) at each local point g of ``points`` (G, d)."""
    dN = np.zeros((len(points), 1 << d, d))
    for g, xi in enumerate(points):
        for a in range(1 << d):
            for k in range(d):
                v = 1.0
                for l in range(d):
                    bit = (a >> l) & 1
                    if l == k:
                        v *= 1.0 if bit else -1.0
                    else:
                        v *= xi[l] if bit else 1.0 - xi[l]
                dN[g, a, k] = v
    return dN


def _gauss(d):
    return [[_GB if (g >> l) & 1 else _GA for l in range(d)] for g in range(1 << d)]


class Problem:
    """Periodic box in 2D (plane strain, cell fields (ny, nx)) or 3D (cell
    fields (nz, ny, nx)): theta and phig per cell, phase moduli from (E_s,
    nu, E_g_ratio) as in the small-strain oracle, and the prescribed
    symmetric part of the mean first Piola stress: -prestress I, or
    ``pbar`` (d x d, symmetric) when given."""

    def __init__(self, theta, phig, prm, omega, prestress=0.0, pbar=None):
        self.shape = theta.shape
        self.d = d = len(self.shape)
        self.N = int(np.prod(self.shape))
        nu = prm["nu"]
        Es, Eg = prm["E_s"], prm["E_s"] * prm["E_g_ratio"]
        self.Ks, self.Gs = Es / (3 * (1 - 2 * nu)), Es / (2 * (1 + nu))
        self.Kg, self.Gg = Eg / (3 * (1 - 2 * nu)), Eg / (2 * (1 + nu))
        self.set_phases(theta, phig)
        self.omega = omega
        self.pbar = -prestress * np.eye(d) if pbar is None else np.asarray(pbar, float)
        self.dN = _shape_grads(d, _gauss(d))
        self.dNc = _shape_grads(d, [[0.5] * d])[0]
        self.w = 1.0 / (1 << d)
        # symmetric components of Fbar in z: the diagonal, then (1,2), (0,2), (0,1) in 3D / (0,1) in 2D
        self.sym = [(i, i) for i in range(d)] + ([(1, 2), (0, 2), (0, 1)] if d == 3 else [(0, 1)])
        self.FP = np.tile(np.eye(3), (self.N, 1, 1))      # per cell (F7, F8)
        self.epsP = np.zeros(self.N)
        self.sigma_Y, self.H = prm["sigma_Y"], prm["H_hard"]
        self.plastic = bool(prm.get("plasticity", 0))
        dims = self.shape[::-1]                           # nx, ny (, nz)
        cell = np.arange(self.N)
        coord = []
        for n in dims:
            cell, r = np.divmod(cell, n)
            coord.append(r)
        nodes = []
        for a in range(1 << d):
            idx, stride = 0, 1
            for l, n in enumerate(dims):
                idx = idx + stride * ((coord[l] + ((a >> l) & 1)) % n)
                stride *= n
            nodes.append(idx)
        self.nodes = np.stack(nodes, axis=1)

    def moduli(self, theta, phig):
        """Mixture K, G and the ferrite weight W_f of cells (F3)."""
        Wf, Ww, Wg = weights(theta, phig)
        return (Wf + Ww) * self.Ks + Wg * self.Kg, (Wf + Ww) * self.Gs + Wg * self.Gg, Wf

    def set_phases(self, theta, phig):
        self.theta = np.asarray(theta, float).ravel().copy()
        self.phig = np.asarray(phig, float).ravel().copy()
        self.K, self.G, self.Wf = self.moduli(self.theta, self.phig)

    def dT(self, omega):
        return 1.0 - self.Wf * omega

    def nz(self):
        """Number of unknowns: the fluctuation without node 0, then Fbar."""
        return self.d * (self.N - 1) + len(self.sym)

    def unpack(self, z):
        d, m = self.d, len(self.sym)
        u = np.zeros((self.N, d))
        u[1:] = z[:-m].reshape(-1, d)
        Fb = np.zeros((d, d))
        for v, (i, j) in zip(z[-m:], self.sym):
            Fb[i, j] = Fb[j, i] = v
        return u, Fb

    def _embed(self, Fd):
        F = np.zeros(Fd.shape[:-2] + (3, 3))
        F[..., :self.d, :self.d] = Fd
        if self.d == 2:
            F[..., 2, 2] = 1.0                            # F4
        return F

    def gradients(self, z):
        """Deformation gradients (N, 2^d, 3, 3) at every cell's Gauss points."""
        u, Fb = self.unpack(z)
        return self._embed(Fb[None, None] + np.einsum("eai,gak->egik", u[self.nodes], self.dN))

    def _fpinv(self):
        return np.linalg.inv(self.FP)[:, None]

    def energy(self, z, omega):
        F = self.gradients(z)
        e = psi(F, self.K[:, None], self.G[:, None], self.dT(omega)[:, None], self._fpinv())
        _, Fb = self.unpack(z)
        return self.w * e.sum() - self.N * np.sum(self.pbar * Fb)

    def residual(self, z, omega):
        """Gradient of the total energy with respect to z."""
        d = self.d
        F = self.gradients(z)
        P = piola(F, self.K[:, None], self.G[:, None], self.dT(omega)[:, None], self._fpinv())[..., :d, :d]
        fa = self.w * np.einsum("egik,gak->eai", P, self.dN)   # per element node
        fu = np.zeros((self.N, d))
        np.add.at(fu, self.nodes.ravel(), fa.reshape(-1, d))
        Ps = self.w * P.sum(axis=(0, 1)) - self.N * self.pbar
        rF = [Ps[i, i] if i == j else Ps[i, j] + Ps[j, i] for i, j in self.sym]
        return np.concatenate([fu[1:].ravel(), rF])

    def solve(self, tol=1e-11, nload=4, maxit=40, z0=None):
        """Equilibrium at self.omega; returns z (see unpack)."""
        n = self.nz()
        if z0 is None:
            z = np.zeros(n)
            m = n - len(self.sym)
            z[m:m + self.d] = 1.0                          # Fbar = I
        else:
            z = z0.copy()
        for step in range(1, nload + 1):
            om = self.omega * step / nload
            for it in range(maxit + 1):
                r = self.residual(z, om)
                if np.abs(r).max() <= tol:
                    break
                if it == maxit:
                    raise RuntimeError("finite-strain Newton did not converge (residual %.3e)" % np.abs(r).max())
                J = np.empty((n, n))
                for j in range(n):
                    hj = 1e-6
                    zp = z.copy()
                    zp[j] += hj
                    zm = z.copy()
                    zm[j] -= hj
                    J[:, j] = (self.residual(zp, om) - self.residual(zm, om)) / (2.0 * hj)
                z = z - np.linalg.solve(J, r)
        return z

    def mean_piola(self, z):
        F = self.gradients(z)
        P = piola(F, self.K[:, None], self.G[:, None], self.dT(self.omega)[:, None], self._fpinv())
        return P.mean(axis=(0, 1))

    def centre_gradients(self, z):
        """Deformation gradient (N, 3, 3) at every cell centre."""
        u, Fb = self.unpack(z)
        return self._embed(Fb[None] + np.einsum("eai,ak->eik", u[self.nodes], self.dNc))

    def mechanics_step(self, z0=None, nload=1, tol=1e-11):
        """One staggered mechanics step (reading F8, as R6 for small strain):
        the equilibrium with the plastic deformation of the step's start,
        then, with plasticity on, one multiplicative J2 update per cell on
        the cell-centre deformation.  Returns z."""
        z = self.solve(tol=tol, nload=nload, z0=z0)
        if not self.plastic:
            return z
        F = self.centre_gradients(z)
        dT = self.dT(self.omega)
        for c in range(self.N):
            self.FP[c], self.epsP[c], _, _ = return_map(F[c], self.FP[c], self.epsP[c], self.K[c], self.G[c],
                                                        dT[c], self.sigma_Y, self.H)
        return z


def mandel(C, K, G, dT):
    """Mandel stress of the elastic right Cauchy-Green tensor C (3 x 3):
    d_T (K/2 (det C - 1) I + G dev uni C), the F2 reading of (StsRelMod)."""
    J2 = np.linalg.det(C)
    u = C * J2 ** (-1.0 / 3.0)
    return dT * (0.5 * K * (J2 - 1.0) * np.eye(3) + G * (u - np.trace(u) / 3.0 * np.eye(3)))


def return_map(F, FP, epsP, K, G, dT, sigma_Y, H):
    """Multiplicative J2 update of one point (Sec. 2.3 PlaTwoJ; Sec. 2.4
    RulFloPla) for the total deformation gradient F (3 x 3), the plastic
    deformation FP and accumulated plastic strain epsP at the start of the
    step.  Backward Euler with the exponential map (reading F7):
        FP_new = exp(dl N) FP,  N = dev M_new / |dev M_new|,
        |dev M_new| = sqrt(2/3) (sigma_Y + H (epsP + dl)),  dl >= 0,
    which keeps det FP = 1.  With isotropic elasticity the update is
    coaxial with the trial C_E, so it is solved in its principal frame:
    elastic log stretches e = e_trial - dl n(e) and the yield condition,
    four equations by Newton with central-difference derivatives.
    Returns (FP_new, epsP_new, dl, M_new)."""
    s = dT ** (-1.0 / 3.0)
    FE = s * F @ np.linalg.inv(FP)
    C = FE.T @ FE
    M = mandel(C, K, G, dT)
    dev = M - np.trace(M) / 3.0 * np.eye(3)
    ry = np.sqrt(2.0 / 3.0)
    if np.linalg.norm(dev) - ry * (sigma_Y + H * epsP) <= 0.0:
        return FP.copy(), epsP, 0.0, M
    c, V = np.linalg.eigh(C)
    etr = 0.5 * np.log(c)

    def mand(e):
        cc = np.exp(2.0 * e)
        return np.diag(mandel(np.diag(cc), K, G, dT))

    def eqs(v):
        e, dl = v[:3], v[3]
        m = mand(e)
        dm = m - m.mean()
        nm = np.linalg.norm(dm)
        return np.concatenate([e - etr + dl * dm / nm, [nm - ry * (sigma_Y + H * (epsP + dl))]])

    v = np.concatenate([etr, [0.0]])
    for _ in range(60):
        r = eqs(v)
        if np.abs(r).max() <= 1e-14 * max(1.0, np.abs(mand(v[:3])).max()):
            break
        J = np.empty((4, 4))
        for j in range(4):
            h = 1e-7
            vp, vm = v.copy(), v.copy()
            vp[j] += h
            vm[j] -= h
            J[:, j] = (eqs(vp) - eqs(vm)) / (2.0 * h)
        v = v - np.linalg.solve(J, r)
    else:
        raise RuntimeError("finite-strain return map did not converge")
    e, dl = v[:3], v[3]
    m = mand(e)
    n = (m - m.mean()) / np.linalg.norm(m - m.mean())
    FPn = V @ np.diag(np.exp(dl * n)) @ V.T @ FP
    Mn = V @ np.diag(m) @ V.T
    return FPn, epsP + dl, dl, Mn


def elastic_force(pr, z, h=1e-6):
    """d psi_ela / d theta of every cell at fixed deformation and F_P
    (reading F9: at the cell-centre deformation, like the small-strain
    coupling scalars), by central differences of the cell's energy
    d_T(W_f) sum_a W_a phi_a(F_E) in theta."""
    F = pr.centre_gradients(z)
    FPinv = np.linalg.inv(pr.FP)

    def e(th):
        K, G, Wf = pr.moduli(th, pr.phig)
        return psi(F, K, G, 1.0 - Wf * pr.omega, FPinv)

    return (e(pr.theta + h) - e(pr.theta - h)) / (2.0 * h)


class CoupledSim:
    """Explicit coupled step with finite-strain mechanics (reading F9): the
    staggered elasto-plastic mechanics step of ``Problem`` at the current
    order parameter, then the explicit Euler update of the oracle
    (``oracle.Sim``: transport, reaction, chemical and double-well forces
    with its small-strain coupling scalars set to zero) with the elastic
    part of the theta force taken from the finite-strain energy, then the
    supply-cell reset of R8.  2D or 3D."""

    def __init__(self, fields, prm, omega, prestress=0.0, nload=4):
        import oracle
        self.sim = oracle.Sim(fields, dict(prm, mechanics=0))
        self.prm = prm
        sh = self.sim.shape
        self.pr = Problem(self.sim.f["theta"].reshape(sh), self.sim.f["phig"].reshape(sh), prm, omega,
                          prestress=prestress)
        self.z = None
        self.nload = nload

    def step(self, n=1):
        s, pr = self.sim, self.pr
        for _ in range(n):
            pr.set_phases(s.f["theta"], s.f["phig"])
            self.z = pr.mechanics_step(z0=self.z, nload=self.nload if self.z is None else 1)
            fel = elastic_force(pr, self.z).reshape(s.shape)
            s.f["trE"][:] = 0.0
            s.f["devE2"][:] = 0.0
            R = s.rates()
            dt = s.dt
            rth = R[0].reshape(s.shape) - 0.5 * self.prm["L"] * s.f["mob"] * fel
            s.f["theta"][:] = s.f["theta"] + dt * rth
            for i, k in ((1, "xO"), (2, "xH"), (3, "xW")):
                s.f[k][:] = s.f[k] + dt * R[i].reshape(s.shape)
            xH, xW = s.f["xH"].reshape(-1), s.f["xW"].reshape(-1)
            for c in np.nonzero(s.f["mask"].reshape(-1))[0]:       # R8, cell order
                s.s.removedW += float(xW[c])
                s.s.suppliedH += float(s.p.xH_bc - xH[c])
                xH[c] = s.p.xH_bc
                xW[c] = 0.0
