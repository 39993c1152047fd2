"""Pins of the oracle's lattice Boltzmann part against what the paper and the
mathematics fix (Sec. 3.1, Eqs. 4, 5 and 10).  CPU only."""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def test_velocity_set_isotropy():
    """D3Q19 (Sec. 3.1): weights 1/3, 1/18, 1/36 give the lattice tensors of
    rank 0, 2 and 4 required for c_s^2 = 1/3."""
    e, w, op = O.tables()
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w[0], 1 / 3) and np.allclose(w[1:7], 1 / 18) and np.allclose(w[7:], 1 / 36)
    assert np.allclose((w[:, None] * e).sum(0), 0.0)
    M2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(M2, CS2 * np.eye(3), atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) * CS2 ** 2
    assert np.allclose(M4, iso, atol=1e-15)
    assert np.all(e[op] == -e)
    assert set(np.abs(e).sum(1)) == {0, 1, 2}


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.05, -0.02, 0.03), (-0.1, 0.07, 0.0)])
def test_equilibrium_moments(u):
    """Eq. 5: zeroth, first and second moments of f^eq are rho, rho u and
    rho (c_s^2 I + u u)."""
    e, w, _ = O.tables()
    rho = 0.83
    f = O.equilibrium(rho, np.array(u))
    u = np.array(u)
    assert np.isclose(f.sum(), rho, rtol=1e-14)
    assert np.allclose((f[:, None] * e).sum(0), rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, e, e)
    assert np.allclose(P, rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-14)


def rest_populations(rhoA, rhoB):
    """f_i = w_i rho for arrays rho [nz,ny,nx] (the rest state)."""
    _, w, _ = O.tables()
    return np.stack([w[:, None, None, None] * rhoA[None], w[:, None, None, None] * rhoB[None]])


def test_rest_state_is_fixed_point_with_wall():
    """Uniform densities at rest stay at rest: bounce-back with a wall at rest
    and the Shan-Chen force of a uniform field vanish."""
    nx, ny, nz = 6, 5, 8
    o = O.Oracle(nx, ny, nz, wall=1)
    rA = np.full((nz, ny, nx), 0.7); rB = np.full((nz, ny, nx), 0.04)
    rA[0] = rB[0] = 0.0
    f0 = rest_populations(rA, rB)
    o.set_populations(f0)
    o.step(10)
    f = o.populations()
    assert np.abs(f - f0).max() < 1e-15


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_shear_wave_decay(tau):
    """G = 0, periodic: u_x = U sin(k z) decays as exp(-nu k^2 t) with
    nu = c_s^2 (tau - 1/2) (second-order accurate; checked to 1%)."""
    nx, ny, nz = 2, 2, 32
    o = O.Oracle(nx, ny, nz, wall=0, tau=(tau, tau), G=0.0)
    k = 2 * np.pi / nz
    U = 1e-3
    f = np.zeros((2, 19, nz, ny, nx))
    for z in range(nz):
        feq = O.equilibrium(0.5, np.array([U * np.sin(k * z), 0.0, 0.0]))
        f[:, :, z] = feq[None, :, None, None]
    o.set_populations(f)
    o.step(50)
    a1 = _amp(o, k, nz)
    o.step(200)
    a2 = _amp(o, k, nz)
    nu = CS2 * (tau - 0.5)
    expect = np.exp(-nu * k * k * 200)
    assert abs(a2 / a1 - expect) / expect < 1e-2


def _amp(o, k, nz):
    _, u = o.fields()
    ux = u[0, :, 0, 0]
    z = np.arange(nz)
    return 2 * np.mean(ux * np.sin(k * z))


def test_shan_chen_force_stencil():
    """Eq. 10 on a field that varies along z only: the stencil sum
    sum_i w_i e_iz psi(z + e_iz) reduces to (psi(z+1) - psi(z-1))/6, so
    F^A_z = -G psi^A (psi^B(z+1) - psi^B(z-1))/6 and F_x = F_y = 0."""
    nx, ny, nz = 3, 4, 16
    G = 3.6
    o = O.Oracle(nx, ny, nz, wall=0, G=G)
    z = np.arange(nz)
    rB = 0.4 + 0.3 * np.sin(2 * np.pi * z / nz) ** 2
    rA = np.full(nz, 0.25)
    RA = np.broadcast_to(rA[:, None, None], (nz, ny, nx)).copy()
    RB = np.broadcast_to(rB[:, None, None], (nz, ny, nx)).copy()
    o.set_populations(rest_populations(RA, RB))
    F = o.sc_forces()
    psiA = 1 - np.exp(-rA); psiB = 1 - np.exp(-rB)
    expA = -G * psiA * (np.roll(psiB, -1) - np.roll(psiB, 1)) / 6.0
    expB = -G * psiB * (np.roll(psiA, -1) - np.roll(psiA, 1)) / 6.0
    assert np.allclose(F[0, 2, :, 1, 1], expA, atol=1e-15)
    assert np.allclose(F[1, 2, :, 1, 1], expB, atol=1e-15)
    assert np.abs(F[:, :2]).max() < 1e-15
    # action-reaction over the periodic box
    assert np.abs(F.sum(axis=(0, 2, 3, 4))).max() < 1e-13


def test_momentum_conserved_periodic_random():
    """No wall, no capsule, random densities: the pairwise Shan-Chen forces
    cancel, so total momentum is conserved to round-off while mass of each
    component is conserved exactly."""
    rng = np.random.default_rng(3)
    nx, ny, nz = 6, 5, 7
    o = O.Oracle(nx, ny, nz, wall=0, tau=(1.0, 0.7))
    rA = 0.3 + 0.3 * rng.random((nz, ny, nx)); rB = 0.3 + 0.3 * rng.random((nz, ny, nx))
    o.set_populations(rest_populations(rA, rB))
    m0 = o.total_mass()
    p0, _, _ = o.momentum()
    o.step(30)
    p1, _, _ = o.momentum()
    assert np.abs(p1 - p0).max() < 1e-12
    assert np.allclose(o.total_mass(), m0, rtol=1e-13)


@pytest.mark.slow
def test_phase_separation_and_laplace_law():
    """G = 3.6 separates the components (Sec. 3.2): a cylinder of A in B keeps
    majority/minority bulk densities, and the pressure jump obeys Laplace's law
    dp = gamma / R (cylinder) -- linear in 1/R through the origin.  Bulk pressure
    of the two-component Shan-Chen fluid: p = c_s^2 (rhoA + rhoB) + c_s^2 G psiA psiB."""
    ny = nz = 48
    res = []
    for R in (8.0, 11.0, 14.0):
        o = O.Oracle(1, ny, nz, wall=0)
        y, z = np.meshgrid(np.arange(ny), np.arange(nz), indexing="xy")
        r = np.sqrt((y - ny / 2 + 0.5) ** 2 + (z - nz / 2 + 0.5) ** 2).T
        inside = r < R
        rA = np.where(inside, 0.7, 0.04)[:, :, None].transpose(1, 0, 2).copy()
        rB = np.where(inside, 0.04, 0.7)[:, :, None].transpose(1, 0, 2).copy()
        o.set_populations(rest_populations(rA, rB))
        o.step(2500)
        rho, u = o.fields()
        psi = 1 - np.exp(-rho)
        p = CS2 * (rho[0] + rho[1]) + CS2 * 3.6 * psi[0] * psi[1]
        pin = p[nz // 2, ny // 2, 0]
        pout = p[0, 0, 0]
        res.append((R, pin - pout, rho[0, nz // 2, ny // 2, 0], rho[1, nz // 2, ny // 2, 0]))
        assert np.abs(u).max() < 5e-3  # spurious currents stay small
    R = np.array([r[0] for r in res]); dp = np.array([r[1] for r in res])
    # separated phases
    for _, _, a, b in res:
        assert a > 0.6 and b < 0.1
    # Laplace: dp * R constant (gamma) within 5 %
    gam = dp * R
    assert np.all(dp > 0)
    assert gam.std() / gam.mean() < 0.05


def test_flat_interface_symmetries_and_relaxation():
    """A slab of A in B in a periodic column (G = 3.6): the run keeps the
    set-up's symmetries -- exchanging the components with a half-period shift
    (G^AB = G^BA, equal tau) exactly, the reflection z -> 63 - z (the velocity
    set is symmetric, Eq. 10's stencil has no preferred direction) to
    round-off, uniformity in x and y exactly -- conserves each component's
    mass, separates the phases, and its velocities decay towards the static
    interface."""
    nx, ny, nz = 3, 3, 64
    o = O.Oracle(nx, ny, nz, wall=0)
    z = np.arange(nz)
    inA = (z >= 16) & (z < 48)
    ones = np.ones((nz, ny, nx))
    rA = np.where(inA, 0.7, 0.04)[:, None, None] * ones
    rB = np.where(inA, 0.04, 0.7)[:, None, None] * ones
    o.set_populations(rest_populations(rA, rB))
    m0 = o.total_mass()
    o.step(1000)
    u1 = np.abs(o.fields()[1]).max()
    o.step(1000)
    rho, u = o.fields()
    a, b = rho[0, :, 0, 0], rho[1, :, 0, 0]
    assert np.array_equal(a, np.roll(b, 32))
    assert np.abs(a - a[::-1]).max() < 1e-11
    assert np.array_equal(rho, np.broadcast_to(rho[:, :, :1, :1], rho.shape))
    assert np.allclose(o.total_mass(), m0, rtol=1e-13, atol=0)
    assert a[32] > 0.7 and a[0] < 0.04
    u2 = np.abs(u).max()
    assert u2 < u1 / 3 and u2 < 1e-4
