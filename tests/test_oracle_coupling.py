"""Pins of the oracle's fluid-membrane coupling, film set-up, node update and
readouts (Sec. 3.1 coupling paragraphs, Eq. 9, Sec. 3.2, Sec. 4.1).  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I


def rest(rhoA, rhoB):
    _, w, _ = O.tables()
    return np.stack([w[:, None, None, None] * rhoA[None], w[:, None, None, None] * rhoB[None]])


def small_box(mode, wall=1, G=3.6, nx=14, ny=13, nz=16, R=4.0, level=2, rep_dz=2.0, centre=None):
    o = O.Oracle(nx, ny, nz, wall=wall, G=G, rep_dz=rep_dz)
    if centre is None:
        centre = (nx / 2 + 0.3, ny / 2 + 0.4, nz / 2 + 0.17)
    X, F = I.icosphere(level, R, centre)
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, mode)
    return o, X, F


def test_cut_links_bbox_equals_bruteforce():
    """Bounding-box enumeration finds exactly the links that a brute-force
    sweep of every link against every element finds (same element choice)."""
    o, _, _ = small_box(I.MODE_FREE)
    m, t, _ = o.cuts()
    mb, tb = o.cuts_bruteforce()
    assert (m == mb).all() and (t == tb).all()
    assert (m != 0).sum() > 100


def test_cut_links_separate_inside_from_outside():
    """Every cut link joins an interior and an exterior node, and the interior
    flags agree with the analytic sphere away from the surface."""
    o, X, F = small_box(I.MODE_FREE)
    m, t, ins = o.cuts()
    e, _, _ = O.tables()
    nz, ny, nx = m.shape
    for z, y, x in zip(*np.nonzero(m)):
        for k in range(1, 19):
            if m[z, y, x] >> (k - 1) & 1:
                z2, y2, x2 = (z + e[k, 2]) % nz, (y + e[k, 1]) % ny, (x + e[k, 0]) % nx
                assert ins[z, y, x] != ins[z2, y2, x2]
                assert m[z2, y2, x2] >> (O.tables()[2][k] - 1) & 1
    c = X.mean(0)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2)
    rin = np.linalg.norm(X - c, axis=1).min() * np.cos(np.deg2rad(20))
    assert ins[r < rin - 0.05].all() and not ins[r > 4.0 + 0.05].any()


def test_mass_conserved_with_fixed_capsule_and_wall():
    """Half-way bounce-back on the substrate and on a resting membrane moves no
    mass across: each component's mass is conserved to round-off."""
    wl = I.tiny_film(mode=I.MODE_FIXED)
    o = O.Oracle.from_workload(wl)
    m0 = o.total_mass()
    o.step(40)
    assert np.allclose(o.total_mass(), m0, rtol=2e-14)


def test_momentum_balance_fluid_plus_membrane():
    """No substrate, moving capsule, Shan-Chen on: what the fluid loses through
    bounce-back (with Ladd's term) and the decoupled Shan-Chen reactions is
    exactly what the membrane receives."""
    o, _, _ = small_box(I.MODE_FREE, wall=0)
    rng = np.random.default_rng(5)
    sh = (o.nz, o.ny, o.nx)
    o.set_film(6.5, 0.7, 0.04, 0.3, rng.uniform(-1e-2, 1e-2, size=(2,) + sh))
    p0, m0, _ = o.momentum()
    o.step(25)
    p1, m1, _ = o.momentum()
    assert np.abs(m1 - m0).max() > 1e-3  # real exchange happened
    # round-off of sums over ~3e3 nodes and 25 steps, relative to the exchange
    assert np.abs((p1 + m1) - (p0 + m0)).max() < 1e-12 * (1 + np.abs(m1 - m0).max()) * 5


def test_ladd_moving_wall_keeps_uniform_flow():
    """Half-way bounce-back with Ladd's term (Sec. 3.1): if fluid and membrane
    move with the same velocity U, bounced populations equal the equilibrium
    ones, f_ib = f_i - 2 w_i rho e_i.U / c_s^2 = f^eq_ib(rho, U), so the uniform
    flow is reproduced exactly by one step."""
    o, X, F = small_box(I.MODE_FIXED, wall=0, G=0.0)
    U = np.array([0.02, -0.01, 0.015])
    rho = (0.55, 0.25)
    feq = [O.equilibrium(r, U) for r in rho]
    f = np.zeros((2, 19, o.nz, o.ny, o.nx))
    for c in range(2):
        f[c] = feq[c][:, None, None, None]
    o.set_populations(f)
    o.set_capsule_velocity(0, np.tile(U, (X.shape[0], 1)))
    o.step(1)
    assert np.abs(o.populations() - f).max() < 1e-15


def test_two_step_average_of_exchanged_momentum():
    """Staggered-momentum fix (Sec. 3.1): the force applied in a step is half
    the momentum exchanged in it plus half that of the step before."""
    wl = I.tiny_film(mode=I.MODE_FIXED)
    o = O.Oracle.from_workload(wl)
    _, mem0, _ = o.momentum()
    o.step(1)
    _, mem1, _ = o.momentum()
    f1 = o.capsule_state(0)["force"]
    assert np.allclose(f1, 0.5 * (mem1 - mem0), atol=1e-14)
    o.step(1)
    _, mem2, _ = o.momentum()
    f2 = o.capsule_state(0)["force"]
    assert np.allclose(f2, 0.5 * (mem2 - mem0), atol=1e-14)


def test_free_node_update_is_first_order():
    """Eq. 9 with dt = 1: x(t+1) - x(t) = F_tot / m for every node."""
    wl = I.tiny_film(mode=I.MODE_FREE)
    o = O.Oracle.from_workload(wl)
    o.step(3)
    X0 = o.capsule_state(0)["X"]
    o.step(1)
    s = o.capsule_state(0)
    assert np.allclose(s["X"] - X0, s["Ftot"] / 25.0, atol=1e-15)
    assert np.allclose(s["V"], s["Ftot"] / 25.0, atol=1e-15)


def test_frozen_capsule_translates_rigidly_with_hertz_plane():
    """Frozen shape: every node moves by sum(F_tot)/(m n_v); the substrate
    Hertz force acts on nodes closer than delta0 to the repulsive plane."""
    nx, ny, nz = 14, 13, 16
    o = O.Oracle(nx, ny, nz, wall=1, rep_dz=2.0)
    R = 4.0
    X, F = I.icosphere(2, R, (7.3, 6.4, 0.5 + 2.0 + 1.0 + R))  # bottom inside the Hertz range
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, I.MODE_FROZEN)
    o.set_film(5.5, 0.7, 0.04, 0.3, None)
    o.step(2)
    X0 = o.capsule_state(0)["X"]
    o.step(1)
    s = o.capsule_state(0)
    d = s["X"] - X0
    assert np.allclose(d, d[0], atol=1e-15)
    assert np.allclose(d[0], s["Ftot"].sum(0) / (25.0 * X.shape[0]), atol=1e-15)
    Fint = s["Ftot"] - s["Fcpl"]
    dz = X0[:, 2] - 2.5
    hz = np.array([O.hertz(v) for v in dz])
    assert np.allclose(Fint[:, 2], hz, atol=1e-14) and hz.max() > 0.1
    assert np.abs(Fint[:, :2]).max() == 0.0


def test_film_initial_state():
    """Sec. 3.2: A majority 0.7 / minority 0.04 below the film top, reversed
    above, one mixed layer at 0.3, capsule interior B-majority; rest state."""
    wl = I.tiny_film(mode=I.MODE_FIXED)
    wl.jitter_amp = 0.0
    o = O.Oracle.from_workload(wl)
    f = o.populations()
    _, _, ins = o.cuts()
    rho = f.sum(1)
    zm = int(np.floor(wl.h_top + 0.5))
    out = ins == 0
    assert np.allclose(rho[0, 1:zm][out[1:zm]], 0.7) and np.allclose(rho[1, 1:zm][out[1:zm]], 0.04)
    assert np.allclose(rho[:, zm][:, out[zm]], 0.3)
    assert np.allclose(rho[0, zm + 1:][out[zm + 1:]], 0.04)
    assert np.allclose(rho[0][ins == 1], 0.04) and np.allclose(rho[1][ins == 1], 0.7)
    assert ins.sum() > 100
    assert np.all(rho[:, 0] == 0.0)


def test_meniscus_field_recovers_linear_interface():
    """Column film height: the zero of phi = rhoA - rhoB between the last
    positive and first non-positive node, exact for a linear phi."""
    nx, ny, nz = 5, 4, 12
    o = O.Oracle(nx, ny, nz, wall=1)
    h = 3.3 + 0.4 * np.arange(nx)[None, :] + 0.25 * np.arange(ny)[:, None]
    z = np.arange(nz)[:, None, None]
    phi = 0.1 * (h[None] - z)
    rho = np.stack([0.5 + phi / 2, 0.5 - phi / 2])
    got = o.meniscus_field(rho)
    assert np.allclose(got, h, atol=1e-13)


def sheet(nx, ny, zs, spacing=2.0, off=(0.3, 0.4)):
    """A flat triangulated sheet at height zs tiling one x-y period of the
    lattice (offset so that no link crosses it on an edge), counter-clockwise
    seen from +z."""
    xs = off[0] + spacing * np.arange(int(round(nx / spacing)) + 1)
    ys = off[1] + spacing * np.arange(int(round(ny / spacing)) + 1)
    X = np.array([[x, y, zs] for y in ys for x in xs])
    F, n = [], len(xs)
    for j in range(len(ys) - 1):
        for i in range(n - 1):
            a = j * n + i
            F += [[a, a + 1, a + n + 1], [a, a + n + 1, a + n]]
    return X, np.array(F)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_between_substrate_and_moving_sheet(tau):
    """A triangulated sheet at z = 6.5 moving with U along x between the
    substrate (wall at z = 0.5) and its periodic image (z = nz - 1/2): at
    steady state both gaps carry the linear Couette profile and the momentum
    exchanged with the sheet is the closed-form shear force of both gaps,
    -2 (rho_A + rho_B) nu U A / H with nu = c_s^2 (tau - 1/2) (Ladd's term
    and the momentum exchange of Sec. 3.1; half-way bounce-back is exact for a
    linear profile)."""
    nx, ny, nz, zs, H, U = 4, 4, 13, 6.5, 6.0, 0.01
    X, F = sheet(nx, ny, zs)
    o = O.Oracle(nx, ny, nz, wall=1, tau=(tau, tau), G=0.0, rep_dz=2.0)
    o.add_capsule(X, F, 0.0, 0.0, 0.0, 0.0, 25.0, I.MODE_FIXED)
    rA, rB = 1.0, 0.1
    f = rest(np.full((nz, ny, nx), rA), np.full((nz, ny, nx), rB))
    f[:, :, 0] = 0.0
    o.set_populations(f)
    V = np.tile([U, 0.0, 0.0], (X.shape[0], 1))
    for _ in range(3000):
        o.set_capsule_velocity(0, V)  # a fixed capsule's node velocities are reset each step
        o.step(1)
    _, u = o.fields()
    z = np.arange(1, nz)
    exact = np.where(z <= zs, (z - 0.5) / H, (nz - 0.5 - z) / H)
    assert np.abs(u[0, 1:] / U - exact[:, None, None]).max() < 1e-10
    assert np.abs(u[1:, 1:]).max() < 1e-12
    nu = (tau - 0.5) / 3.0
    F_exp = -2.0 * (rA + rB) * nu * U * nx * ny / H
    force = o.capsule_state(0)["force"]
    assert abs(force[0] / F_exp - 1.0) < 1e-10 and np.abs(force[1:]).max() < 1e-12
