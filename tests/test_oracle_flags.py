"""Pins of the oracle's alternative readings of paper-silent points (flags):
the inertial node update (c6), Ladd's term with the reference density (c8),
the mirrored partner density (c10) and drying by removal (c23).  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I


def test_mirror_partner_density_is_the_node_itself():
    """With the mirror reading the partner density across a cut or substrate
    link is the node's own: rho(2, 2, 2) = 222 for rho = x + 10y + 100z."""
    o = O.Oracle(5, 5, 5, wall=1, flags=O.Oracle.MIRROR)
    z, y, x = np.meshgrid(np.arange(5), np.arange(5), np.arange(5), indexing="ij")
    rho = (x + 10 * y + 100 * z).astype(np.float64)
    assert o.rho_interp(rho, 2, 2, 2) == 222.0 and o.rho_interp(rho, 2, 2, 1) == 122.0


@pytest.mark.parametrize("rho", [(1.0, 1.0), (0.55, 0.25)])
def test_ladd_reference_density(rho):
    """Ladd's term with rho_0 = 1: a uniform flow U shared by fluid and
    membrane is kept exactly when both densities are 1 (then rho_0 is the
    node's density); otherwise each population bounced back along -e_k
    differs from the equilibrium one by -2 w_k (1 - rho) e_k.U / c_s^2, so a
    cut node's streamed density moves by the sum of that over its cut links."""
    nx, ny, nz = 14, 13, 16
    o = O.Oracle(nx, ny, nz, wall=0, G=0.0, rep_dz=2.0, flags=O.Oracle.REF_RHO)
    X, F = I.icosphere(2, 4.0, (7.3, 6.9, 8.17))
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, I.MODE_FIXED)
    U = np.array([0.02, -0.01, 0.015])
    feq = [O.equilibrium(r, U) for r in rho]
    f = np.zeros((2, 19, nz, ny, nx))
    for c in range(2):
        f[c] = feq[c][:, None, None, None]
    o.set_populations(f)
    o.set_capsule_velocity(0, np.tile(U, (X.shape[0], 1)))
    o.step(1)
    g = o.populations()
    if rho == (1.0, 1.0):
        assert np.abs(g - f).max() < 1e-15
    else:
        mask, _, _ = o.cuts()
        e, w, _ = O.tables()
        r, _ = o.fields()
        checked = 0
        for zz, yy, xx in np.argwhere(mask != 0)[:20]:
            m = int(mask[zz, yy, xx])
            dev = sum(-6.0 * w[k] * (1.0 - rho[0]) * np.dot(e[k], U) for k in range(1, 19) if (m >> (k - 1)) & 1)
            assert r[0, zz, yy, xx] == pytest.approx(rho[0] + dev, rel=1e-12, abs=1e-15)
            checked += abs(dev) > 1e-6
        assert checked > 3


def test_inertial_node_update():
    """v(t+1) = v(t) + F_tot/m and x(t+1) = x(t) + v(t+1) for every node."""
    wl = I.tiny_film(mode=I.MODE_FREE)
    wl.flags = O.Oracle.INERTIAL
    o = O.Oracle.from_workload(wl)
    o.step(3)
    s0 = o.capsule_state(0)
    o.step(1)
    s1 = o.capsule_state(0)
    assert np.allclose(s1["V"], s0["V"] + s1["Ftot"] / 25.0, atol=1e-15)
    assert np.allclose(s1["X"] - s0["X"], s1["V"], atol=1e-14)
    assert np.abs(s0["V"]).max() > 0


def test_drying_by_removal():
    """The A inventory falls by dm per step and B keeps its mass (removal),
    so the total mass falls by dm."""
    wl = I.Workload("dry", 12, 10, 14, h_top=6.5, capsules=[], steps=1, seed=3, rep_dz=2.0)
    wl.flags = O.Oracle.REMOVE
    o = O.Oracle.from_workload(wl)
    o.step(2)
    m0 = o.total_mass()
    o.remove_mass(0.5)
    o.step(3)
    m1 = o.total_mass()
    assert m1[0] == pytest.approx(m0[0] - 1.5, rel=1e-12)
    assert m1[1] == pytest.approx(m0[1], rel=1e-12)
