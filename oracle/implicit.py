"""Backward-Euler time step of the field relations (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import this module; it shares no code with the CUDA library.

The paper integrates its field relations (Sec. 2.4, FieRelDRI) and the
plastic flow in time by backward Euler and solves every step by a Newton
method (Sec. 2.4, closing paragraph).  This module is the plain definition
of that step on the build's discretisation:

    y_{n+1} = y_n + dt R(y_{n+1}),    y = (theta, x_O, x_H, x_H2O),

with R the right-hand sides of the explicit oracle (``or_rates`` in
oracle.c: the same fluxes, driving force and reaction), and these readings
where the paper leaves the details to its finite-element package:

  S1  Mechanics stays staggered as in the explicit step (R6): the elastic
      solve and the J2 return run once at y_n, and the coupling scalars
      tr eps_e, |dev eps_e|^2 are held over the step.  The radial return is
      itself the backward-Euler integration of the flow rule.
  S2  The reaction switch (no reaction where x_H2O >= 1, Sec. 4.3) is part
      of R and is evaluated at the new state.
  S3  Supply cells: x_H = xH_bc and x_H2O = 0 at the new time level are
      equations of the step.  The water removed there and the hydrogen
      supplied are the differences between what the cells' own
      backward-Euler relations would give, x_n + dt R(y_{n+1}), and the
      held values, so the two balances of the explicit step hold unchanged.

Newton's method with the Jacobian built column by column from central
differences of R and a dense linear solve; it stops when the largest
residual entry is at most ``tol``, or when an update moves no entry by more
than ``tol`` relative to the largest field value (the residual has then
reached its rounding floor: at the paper's diffusivities dt R carries
terms ~1e5 times the fields).  Dense means small grids only (4N x 4N,
N cells).

Pins (tests/test_oracle_implicit.py): exact DFT solutions in the linear
cases (hydrogen diffusion, single-phase oxygen with its gradient-energy
term) at time steps far above the explicit limit; the two balances with
reaction and supply cells; first-order convergence in dt; free-energy
decrease of the Allen-Cahn flow at large steps.
"""
import numpy as np

_KEYS = ("theta", "xO", "xH", "xW")


def _set_state(sim, y):
    N = sim.N
    for i, k in enumerate(_KEYS):
        sim.f[k].reshape(-1)[:] = y[i * N:(i + 1) * N]


def _rates(sim, y):
    _set_state(sim, y)
    return sim.rates().reshape(-1)


def _jacobian(sim, y, dt, fixed):
    """I - dt dR/dy by central differences; rows of held values are identity."""
    n = y.size
    A = np.empty((n, n))
    for j in range(n):
        h = 1e-6 * max(1.0, abs(y[j]))
        yp = y.copy()
        yp[j] += h
        ym = y.copy()
        ym[j] -= h
        A[:, j] = -dt * (_rates(sim, yp) - _rates(sim, ym)) / (2.0 * h)
    A[np.arange(n), np.arange(n)] += 1.0
    rows = np.nonzero(fixed)[0]
    A[rows, :] = 0.0
    A[rows, rows] = 1.0
    return A


def be_step(sim, dt, tol=1e-13, maxit=30):
    """Advance an ``oracle.Sim`` by one backward-Euler step of length dt.

    Returns the number of Newton iterations.  Raises RuntimeError (and
    leaves the fields at y_n) if neither stopping rule holds within
    ``maxit`` iterations.
    """
    sim.mechanics()                                   # S1: at y_n
    N = sim.N
    y0 = np.concatenate([sim.f[k].reshape(-1).copy() for k in _KEYS])
    mask = sim.f["mask"].reshape(-1).astype(bool)
    fixed = np.zeros(4 * N, dtype=bool)
    fixed[2 * N:3 * N] = mask
    fixed[3 * N:] = mask
    held = np.zeros(4 * N)
    held[2 * N:3 * N] = np.where(mask, sim.p.xH_bc, 0.0)

    def residual(y):
        F = y - y0 - dt * _rates(sim, y)
        F[fixed] = y[fixed] - held[fixed]
        return F

    y = y0.copy()
    y[fixed] = held[fixed]
    moved = np.inf
    for it in range(maxit + 1):
        F = residual(y)
        if np.abs(F).max() <= tol or moved <= tol * max(1.0, np.abs(y).max()):
            break
        if it == maxit:
            _set_state(sim, y0)
            raise RuntimeError("backward-Euler Newton iteration did not converge "
                               "(residual %.3e)" % np.abs(F).max())
        delta = np.linalg.solve(_jacobian(sim, y, dt, fixed), F)
        y = y - delta
        moved = np.abs(delta).max()
    R = _rates(sim, y)                                # S3: balances of the held cells
    w_free = y0[3 * N:] + dt * R[3 * N:]
    h_free = y0[2 * N:3 * N] + dt * R[2 * N:3 * N]
    sim.s.removedW += float(w_free[mask].sum())
    sim.s.suppliedH += float((sim.p.xH_bc - h_free[mask]).sum())
    _set_state(sim, y)
    return it
