"""Pins of the oracle's drying step (film lowered by turning component A into
component B; a reading, the paper fixes each film height per run): the A
inventory falls linearly by the requested amount while the total mass stays,
the conversion touches only A-majority nodes and moves mass in the rest-state
proportions, and a request larger than the available A converts all of it.
CPU only."""
import numpy as np

import oracle as O
from paper_2007_15405_gb300 import inputs as I


def film(nx=12, ny=10, nz=16, h_top=7.0):
    o = O.Oracle(nx, ny, nz, wall=1)
    jit = I.jitter((nz, ny, nx), 1e-3, seed=5)
    o.set_film(h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, jit)
    return o


def test_A_inventory_falls_linearly_total_conserved():
    o = film()
    m0 = o.total_mass()
    dm = 0.05
    o.remove_mass(dm)
    done = 0
    for n in (1, 4, 15):
        o.step(n)
        done += n
        m = o.total_mass()
        assert abs((m0[0] - m[0]) - done * dm) < 1e-10
        assert abs(m.sum() - m0.sum()) < 1e-10
    # off again: the inventory stays
    o.remove_mass(0.0)
    o.step(5)
    assert abs(o.total_mass()[0] - m[0]) < 1e-10


def test_conversion_only_at_A_majority_nodes_in_rest_proportions():
    _, w, _ = O.tables()
    a, b = film(), film()
    a.step(10); b.step(10)
    dm = 0.3
    a.remove_mass(dm)
    a.step(1); b.step(1)
    fa, fb = a.populations(), b.populations()
    rho, _ = b.fields()  # this step's densities (the same in both)
    sel = rho[0] > rho[1]
    sel[0] = False  # substrate plane
    eps = dm / rho[0][sel].sum()
    # B-majority and substrate nodes untouched, bit for bit
    assert np.array_equal(fa[:, :, ~sel], fb[:, :, ~sel])
    # A scaled by 1 - eps, B given w_i eps rho_A
    assert np.allclose(fa[0][:, sel], (1 - eps) * fb[0][:, sel], rtol=1e-14, atol=0)
    gain = fa[1][:, sel] - fb[1][:, sel]
    assert np.allclose(gain, w[:, None] * eps * rho[0][sel][None, :], rtol=1e-9, atol=1e-17)
    # per node, the mass is kept
    assert np.allclose(fa[:, :, sel].sum(axis=(0, 1)), fb[:, :, sel].sum(axis=(0, 1)), rtol=1e-14)


def test_request_beyond_the_inventory_converts_all_A():
    a, b = film(), film()
    a.remove_mass(1e9)
    a.step(1); b.step(1)
    rho, _ = b.fields()
    sel = rho[0] > rho[1]
    sel[0] = False
    fa = a.populations()
    assert np.all(fa[0][:, sel] == 0.0)
    assert abs(a.total_mass().sum() - b.total_mass().sum()) < 1e-10
    assert abs(a.total_mass()[0] - b.total_mass()[0] + rho[0][sel].sum()) < 1e-10
