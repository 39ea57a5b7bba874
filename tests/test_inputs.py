"""The seeded input generators follow their stated recipes: the core-shell
geometry of Sec. 4.2, the porous stand-in for the micrograph of Sec. 4.3
(Voronoi grains with a mobility factor each, lognormal pores up to a
volume fraction, the outer supply layers) and the 64-instance batch."""
import numpy as np
import pytest

from paper_2111_11538_gb300 import inputs


def _common(f):
    pf, pw = f["phi_f"], f["phi_w"]
    pg = 1.0 - pf - pw
    assert pf.min() >= 0.0 and pw.min() >= 0.0 and pg.min() >= -1e-15
    assert np.allclose(f["xO"], inputs.X_W_INIT * pw + inputs.X_F_INIT * pf, rtol=0, atol=1e-15)
    assert np.allclose(f["xH"], inputs.XH_GAS * pg, rtol=0, atol=1e-15)
    assert np.all(f["xW"] == 0.0)
    assert f["mask"].dtype == np.uint8 and set(np.unique(f["mask"])) <= {0, 1}


@pytest.mark.parametrize("shape", [(64, 64), (24, 24, 24)])
def test_core_shell(shape):
    R, s, delta = 8.0, 3.0, 1.0
    f = inputs.core_shell(shape, R, s, delta=delta)
    _common(f)
    r = inputs._centre_dist(shape)
    core = r < R - 4 * delta
    shell = np.abs(r - (R + s / 2)) < 0.3
    gas = r > R + s + 4 * delta
    assert f["phi_w"][core].min() > 0.98
    assert f["phi_f"][shell].min() > 0.5
    assert (1.0 - f["phi_f"] - f["phi_w"])[gas].min() > 0.98
    assert np.array_equal(f["mask"] == 1, r > R + s + 2 * delta)
    assert np.all(f["mob"] == 1.0)


def test_porous_recipe():
    shape = (256, 256)
    f = inputs.porous(shape, 20, 0.2, 12.0, 0.5, seed=2)
    g = inputs.porous(shape, 20, 0.2, 12.0, 0.5, seed=2)
    for k in f:
        assert np.array_equal(f[k], g[k])                      # seeded
    _common(f)
    # mobility: one factor per grain, drawn from [0.8, 1.2]
    assert f["mob"].min() >= 0.8 and f["mob"].max() <= 1.2
    assert 1 < len(np.unique(f["mob"])) <= 20
    # supply mask: exactly the outer two layers of the box, all gas
    m = np.zeros(shape, bool)
    m[:2, :] = m[-2:, :] = m[:, :2] = m[:, -2:] = True
    assert np.array_equal(f["mask"] == 1, m)
    pg = 1.0 - f["phi_f"] - f["phi_w"]
    assert np.all(pg[m] == 1.0)
    # pore volume fraction: reached, and overshot by at most a few pores
    gas_inside = (pg[~m] > 0.5).mean()
    assert 0.17 < gas_inside < 0.3
    # iron rims: a diffuse ferrite layer around the pores (as wide as the
    # tanh profile, so it peaks near one half), wuestite in the grain bulk
    assert 0.4 < f["phi_f"].max() < 0.7 and f["phi_w"].max() > 0.99
    near = (pg > 0.05) & (pg < 0.95) & ~m
    assert f["phi_f"][near].mean() > 10 * f["phi_f"][pg < 1e-6].mean()


def test_porous_other_seed_differs():
    a = inputs.porous((64, 64), 6, 0.2, 6.0, 0.4, seed=3)
    b = inputs.porous((64, 64), 6, 0.2, 6.0, 0.4, seed=4)
    assert not np.array_equal(a["phi_f"], b["phi_f"])


def test_batch_instances_recipe():
    desc = inputs.batch_instances(64, 4)
    assert len(desc) == 64
    assert {d["n"] for d in desc} <= {128, 256, 512, 1024}
    assert len({d["n"] for d in desc}) == 4                   # every size class occurs
    assert all(0.05 <= d["pore_fraction"] <= 0.3 for d in desc)
    assert all(0.0 <= d["prestress"] <= 0.02 for d in desc)
    assert [d["seed"] for d in desc] == [4 * 1000 + i for i in range(64)]
    assert inputs.batch_instances(64, 4) == desc               # seeded
