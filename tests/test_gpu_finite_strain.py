"""GPU finite-strain elastic equilibrium (pf_finite_strain_solve) against
the finite-strain oracle (oracle/finite_strain.py, Problem.solve).

Sec. 2.2 of the paper: neo-Hooke elasticity of F_E = F F_R^-1 with the
transformation stretch d_T^(1/3), d_T = 1 - W_f Omega; Sec. 2.4: Div P = 0.
Both sides discretise the same energy on the same Q1 voxel elements with
2^d Gauss points and solve its stationarity by Newton's method over the
same load steps to max |residual| <= 1e-11 (the oracle with a dense
finite-difference Jacobian, the library matrix-free by conjugate
gradients), so u and Fbar agree to the Newton tolerance times the
problem's conditioning: 1e-8 relative to the largest displacement, 1e-10 on
Fbar.  The library's Hessian-vector products run in FP32 (PF_MIXED, the
default here) or FP64; the residual is FP64 either way.  With FP32
products Newton converges linearly (~1e-6 per step) and stops just under
its tolerance, where the oracle's exact Newton overshoots 1e-11 by orders;
the near-translation mode (u = 0 only at node 0) turns a 1e-11 residual
into ~2e-9 of u, so the library side solves to 1e-13 (FP64 residuals reach
it).
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import inputs, make_config, native, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


@pytest.fixture(scope="module")
def fs(orc):
    from oracle import finite_strain
    return finite_strain


def _opts(nload, tol=1e-13, precision=native.PF_MIXED):
    return native.pf_fs_opts(nload=nload, newton_maxit=40, newton_tol=tol, cg_maxit=20000, cg_rtol=1e-12,
                             precision=precision)


def _gpu(th, pg, prm, omega, nload, pbar=None, precision=native.PF_MIXED):
    cfg = make_config(th.shape, prm)
    rc, u, Fb, st = native.pf_finite_strain_solve(cfg, th.ravel(), pg.ravel(), omega, pbar,
                                                  _opts(nload, precision=precision))
    assert rc == native.PF_OK, native.lib().pf_fs_last_error()
    assert st.hvp_launches >= st.cg_iters and st.hvp_ms > 0.0
    return u, Fb, st


def _compare(fs, th, pg, prm, omega, nload, prestress=0.0, pbar=None, precision=native.PF_MIXED):
    pr = fs.Problem(th, pg, prm, omega, prestress=prestress, pbar=pbar)
    u0, F0 = pr.unpack(pr.solve(tol=1e-11, nload=nload))
    u, Fb, st = _gpu(th, pg, dict(prm, prestress=prestress), omega, nload, pbar, precision)
    scale = max(np.abs(u0).max(), 1e-12)
    assert np.abs(u - u0).max() < 1e-8 * scale, (np.abs(u - u0).max(), scale)
    assert np.abs(Fb - F0).max() < 1e-10, (Fb, F0)
    assert st.residual <= 1e-11 and st.newton_iters >= nload
    return u, Fb


@pytest.mark.parametrize("precision", [native.PF_MIXED, native.PF_FP64])
def test_finite_strain_2d_core_shell_matches_oracle(fs, precision):
    """Core-shell with gas cells and a 20 % volume change of ferrite,
    prestress 0.005, four load steps (plane strain)."""
    from oracle import split_phases
    f = inputs.core_shell((8, 8), 2.5, 1.0, delta=1.0)
    th, pg = split_phases(f["phi_f"], f["phi_w"])
    u, Fb = _compare(fs, th, pg, workloads.params(), 0.2, 4, prestress=0.005, precision=precision)
    assert Fb[0, 0] < 1.0 and np.abs(u).max() > 1e-3


def test_finite_strain_2d_sheared_box_matches_oracle(fs):
    """A prescribed mean shear stress (pbar with off-diagonal entries) on a
    ragged 7x5 grid."""
    rng = np.random.default_rng(3)
    th = np.clip(0.5 + 0.5 * rng.standard_normal((5, 7)), 0.0, 1.0)
    pg = np.zeros((5, 7))
    pbar = np.array([[0.0, 0.004], [0.004, -0.002]])
    _compare(fs, th, pg, workloads.params(), 0.1, 2, pbar=pbar)


@pytest.mark.parametrize("precision", [native.PF_MIXED, native.PF_FP64])
def test_finite_strain_3d_ball_matches_oracle(fs, precision):
    n = 4
    x = np.arange(n) + 0.5 - n / 2
    gz, gy, gx = np.meshgrid(x, x, x, indexing="ij")
    th = 0.5 * (1 - np.tanh((np.sqrt(gx ** 2 + gy ** 2 + gz ** 2) - 1.2) / 1.0))
    pg = np.zeros_like(th)
    pg[0, 0, :] = 1.0                      # a row of gas cells
    th[0, 0, :] = 0.0
    _compare(fs, th, pg, workloads.params(), 0.3, 3, precision=precision)


def test_finite_strain_3d_uniform_transformation_is_stress_free():
    """In 3D nothing constrains a uniform transformation: Fbar = d_T^(1/3) I
    exactly, u = 0 (d_T = 1 - Omega for uniform ferrite)."""
    th = np.ones((3, 4, 5))
    u, Fb, _ = _gpu(th, np.zeros_like(th), workloads.params(), 0.4, 2)
    assert np.abs(Fb - 0.6 ** (1 / 3) * np.eye(3)).max() < 1e-12
    assert np.abs(u).max() < 1e-12


def test_finite_strain_rejects_bad_arguments():
    th = np.ones((4, 4))
    cfg = make_config((4, 4), workloads.params())
    bad = native.pf_fs_opts(nload=0, newton_maxit=10, newton_tol=1e-10, cg_maxit=10, cg_rtol=1e-6)
    rc, _, _, _ = native.pf_finite_strain_solve(cfg, th.ravel(), th.ravel() * 0, 0.1, None, bad)
    assert rc == native.PF_EINVAL and b"pf_fs_opts" in native.lib().pf_fs_last_error()
    bad = native.pf_fs_opts(nload=1, newton_maxit=10, newton_tol=1e-10, cg_maxit=10, cg_rtol=1e-6, precision=2)
    rc, _, _, _ = native.pf_finite_strain_solve(cfg, th.ravel(), th.ravel() * 0, 0.1, None, bad)
    assert rc == native.PF_EINVAL and b"precision" in native.lib().pf_fs_last_error()


def test_return_map_matches_oracle(fs):
    """The multiplicative J2 update of independent points against the
    oracle's return_map (Sec. 2.3 PlaTwoJ, Sec. 2.4 RulFloPla): plastic and
    elastic points, first and second steps (FP from a previous update)."""
    rng = np.random.default_rng(7)
    n = 40
    F = np.empty((n, 3, 3))
    for i in range(n):
        g = (0.0005 if i % 3 == 0 else 0.02) * rng.standard_normal((3, 3))
        F[i] = np.eye(3) + g + g.T * 0.5
    K = np.full(n, 1.0 / (3 * 0.4))
    G = np.full(n, 1.0 / 2.6)
    dT = 1.0 - 0.2 * rng.random(n)
    sY, H = 0.004, 0.01
    FP = np.tile(np.eye(3), (n, 1, 1))
    ep = np.zeros(n)
    ref_FP, ref_ep = FP.copy(), ep.copy()
    for rnd in range(2):
        for i in range(n):
            ref_FP[i], ref_ep[i], _, _ = fs.return_map(F[i], ref_FP[i], ref_ep[i], K[i], G[i], dT[i], sY, H)
        rc = native.pf_fs_return_map(F, FP, ep, K, G, dT, sY, H)
        assert rc == native.PF_OK, native.lib().pf_fs_last_error()
        assert np.abs(FP - ref_FP).max() < 1e-11, (rnd, np.abs(FP - ref_FP).max())
        assert np.abs(ep - ref_ep).max() < 1e-11
        if rnd == 0:
            assert (ep > 0).sum() >= n // 2 and (ep == 0).sum() >= n // 4      # plastic and elastic points
        F = F @ (np.eye(3) + 0.01 * np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0]]))
    assert np.abs(np.linalg.det(FP) - 1.0).max() < 1e-12


@pytest.mark.parametrize("shape,precision", [((8, 8), native.PF_MIXED), ((4, 4, 4), native.PF_MIXED),
                                             ((4, 4, 4), native.PF_FP64)])
def test_finite_strain_plastic_steps_match_oracle(fs, shape, precision):
    """Two staggered elasto-plastic mechanics steps on a core-shell (the
    second with the plastic deformation of the first) against
    Problem.mechanics_step."""
    from oracle import split_phases
    r = 0.3 * min(shape)
    f = inputs.core_shell(shape, r, 0.15 * min(shape), delta=1.0)
    th, pg = split_phases(f["phi_f"], f["phi_w"])
    prm = workloads.params(plasticity=1, sigma_Y=0.002, H_hard=0.01)
    om = 0.2
    pr = fs.Problem(th, pg, prm, om)
    N = th.size
    FP = np.tile(np.eye(3), (N, 1, 1)).copy()
    ep = np.zeros(N)
    cfg = make_config(th.shape, prm)
    for k in range(2):
        u0, F0 = pr.unpack(pr.mechanics_step(nload=2))
        rc, u, Fb, st = native.pf_finite_strain_step(cfg, th.ravel(), pg.ravel(), om, None,
                                                     _opts(2, precision=precision), FP, ep)
        assert rc == native.PF_OK, native.lib().pf_fs_last_error()
        scale = max(np.abs(u0).max(), 1e-12)
        assert np.abs(u - u0).max() < 1e-8 * scale, (k, np.abs(u - u0).max(), scale)
        assert np.abs(Fb - F0).max() < 1e-10
        assert np.abs(FP - pr.FP).max() < 1e-9, (k, np.abs(FP - pr.FP).max())
        assert np.abs(ep - pr.epsP).max() < 1e-9
    assert pr.epsP.max() > 0.0 and (ep > 0).any()


def test_elastic_driving_force_matches_oracle(fs):
    """d psi / d theta at the cell centres (the coupled step's elastic force
    on the order parameter) after an elasto-plastic step, against the
    oracle's central differences (step 1e-6: agreement to 1e-7 relative)."""
    from oracle import split_phases
    f = inputs.core_shell((8, 8), 2.5, 1.0, delta=1.0)
    th, pg = split_phases(f["phi_f"], f["phi_w"])
    prm = workloads.params(plasticity=1, sigma_Y=0.002, H_hard=0.01)
    pr = fs.Problem(th, pg, prm, 0.2)
    z = pr.mechanics_step(nload=2)
    ref = fs.elastic_force(pr, z)
    u, Fb = pr.unpack(z)
    rc, g = native.pf_fs_elastic_force(make_config(th.shape, prm), th, pg, 0.2, u, Fb, pr.FP)
    assert rc == native.PF_OK, native.lib().pf_fs_last_error()
    assert np.abs(g - ref).max() < 1e-7 * np.abs(ref).max(), (np.abs(g - ref).max(), np.abs(ref).max())
    assert np.abs(ref).max() > 1e-4


def test_coupled_finite_strain_steps_match_oracle(fs):
    """Two explicit steps coupled to elasto-plastic finite-strain mechanics
    (FiniteStrainSimulation) against finite_strain.CoupledSim on a core-shell
    with gas and supply cells.  The oracle adds -(L/2) mob d psi/d theta
    (central differences, step 1e-6) to theta's rate; the library runs the
    mechanics-free field update with the equivalent coupling scalar
    (pf_fs_coupling, exact derivative along d_T).  The two forces differ by
    the difference quotient's error, ~1e-8 of the force, so each field's
    change over the steps agrees to 1e-6 of its size."""
    from paper_2111_11538_gb300 import FiniteStrainSimulation
    f = inputs.core_shell((8, 8), 2.5, 1.0, delta=1.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.002, H_hard=0.01)
    ref = fs.CoupledSim(f, prm, 0.2, nload=2)
    sim = FiniteStrainSimulation((8, 8), prm, 0.2, nload=2)
    sim.set_fields(f)
    keys = ("theta", "xO", "xH", "xW")
    f0 = {k: ref.sim.f[k].copy() for k in keys}
    for step in range(2):
        ref.step(1)
        sim.step(1)
        g = sim.get_fields(keys=keys)
        for k in keys:
            ch = np.abs(ref.sim.f[k] - f0[k]).max()
            assert np.abs(g[k] - ref.sim.f[k]).max() <= 1e-6 * ch + 1e-14, (step, k, np.abs(g[k] - ref.sim.f[k]).max(), ch)
        assert np.abs(sim.FP - ref.pr.FP).max() < 1e-9, (step, np.abs(sim.FP - ref.pr.FP).max())
        assert np.abs(sim.epsP - ref.pr.epsP).max() < 1e-9
    assert ref.pr.epsP.max() > 0.0
    d = sim.diagnostics()
    assert abs(d["removed_H2O"] - ref.sim.removedW) <= 1e-9 * max(ref.sim.removedW, 1e-12)
    # the elastic force matters: the same steps without it move theta by more
    # than the tolerance above
    bare = fs.CoupledSim(f, prm, 0.0, nload=1)
    bare.step(2)
    assert np.abs(bare.sim.f["theta"] - ref.sim.f["theta"]).max() > 1e-3 * np.abs(ref.sim.f["theta"] - f0["theta"]).max()
    sim.close()


def test_coupling_scalar_reproduces_the_elastic_force(fs):
    """pf_fs_coupling against pf_fs_elastic_force: the field update's elastic
    term -3 eig0 (1 - h(phi_g)) h'(theta) K_mix trE equals d psi / d theta."""
    from oracle import split_phases
    f = inputs.core_shell((8, 8), 2.5, 1.0, delta=1.0)
    th, pg = split_phases(f["phi_f"], f["phi_w"])
    prm = workloads.params(plasticity=1, sigma_Y=0.002, H_hard=0.01)
    pr = fs.Problem(th, pg, prm, 0.2)
    z = pr.mechanics_step(nload=2)
    u, Fb = pr.unpack(z)
    cfg = make_config(th.shape, prm)
    rc, g = native.pf_fs_elastic_force(cfg, th, pg, 0.2, u, Fb, pr.FP)
    assert rc == native.PF_OK
    rc, tE = native.pf_fs_coupling(cfg, th, pg, 0.2, u, Fb, pr.FP)
    assert rc == native.PF_OK, native.lib().pf_fs_last_error()
    t, hg = th.ravel(), pg.ravel() ** 3 * (pg.ravel() * (6 * pg.ravel() - 15) + 10)
    hp = 30 * t * t * (1 - t) ** 2
    E, nu = prm["E_s"], prm["nu"]
    Ks, Kg = E / (3 * (1 - 2 * nu)), E * prm["E_g_ratio"] / (3 * (1 - 2 * nu))
    Kmix = (1 - hg) * Ks + hg * Kg
    term = -3 * prm["eig0"] * (1 - hg) * hp * Kmix * tE
    assert np.abs(term - g).max() < 1e-12 * np.abs(g).max(), (np.abs(term - g).max(), np.abs(g).max())
    assert np.abs(g).max() > 1e-4
    rc, _ = native.pf_fs_coupling(make_config(th.shape, dict(prm, eig0=0.0)), th, pg, 0.2, u, Fb, pr.FP)
    assert rc == native.PF_EINVAL
