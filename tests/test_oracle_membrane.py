"""Pins of the oracle's membrane mechanics (Eqs. 6-8, 11) against closed forms,
finite differences and invariants.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300.inputs import icosphere


def fd_forces(X, X0, F, which, kw, stride=5, h=1e-6):
    fd = np.full(X.shape, np.nan)
    for v in range(0, X.shape[0], stride):
        for a in range(3):
            Xp = X.copy(); Xp[v, a] += h
            Xm = X.copy(); Xm[v, a] -= h
            ep = O.membrane(Xp, X0, F, which=which, **kw)[0].sum()
            em = O.membrane(Xm, X0, F, which=which, **kw)[0].sum()
            fd[v, a] = -(ep - em) / (2 * h)
    return fd


@pytest.fixture(scope="module")
def deformed():
    X0, F = icosphere(2, 4.0, (0.3, 0.2, 0.1))
    rng = np.random.default_rng(0)
    X = X0 * 1.05 + rng.normal(0, 0.05, X0.shape)
    return X0, X, F


@pytest.mark.parametrize("which,kw", [(1, dict(kS=0.01, C=2.0)), (2, dict(kB=0.01)),
                                      (4, dict(kV=0.5))])
def test_forces_are_negative_energy_gradient(deformed, which, kw):
    """Strain and volume forces by virtual work, bending by the functional
    derivative (Sec. 3.1): each is -dE/dx of its discrete energy."""
    X0, X, F = deformed
    E, Fo = O.membrane(X, X0, F, which=which, **kw)
    fd = fd_forces(X, X0, F, which, kw)
    sel = ~np.isnan(fd)
    assert np.abs(fd[sel] - Fo[sel]).max() < 1e-6 * np.abs(Fo).max()


@pytest.mark.parametrize("which,kw", [(1, dict(kS=0.01, C=2.0)), (2, dict(kB=0.01)),
                                      (4, dict(kV=0.5))])
def test_internal_forces_free_of_net_force_and_torque(deformed, which, kw):
    X0, X, F = deformed
    _, Fo = O.membrane(X, X0, F, which=which, **kw)
    scale = np.abs(Fo).max() * X.shape[0]
    assert np.abs(Fo.sum(0)).max() < 1e-12 * scale
    assert np.abs(np.cross(X, Fo).sum(0)).max() < 1e-11 * scale * 10


def test_skalak_zero_at_reference():
    X0, F = icosphere(2, 5.0)
    E, Fo = O.membrane(X0, X0, F, kS=0.1, C=3.0, which=1)
    assert abs(E[0]) < 1e-14 and np.abs(Fo).max() < 1e-13


@pytest.mark.parametrize("lam,C", [(1.1, 0.0), (0.93, 9.0), (1.3, 1.0)])
def test_skalak_isotropic_inflation_closed_form(lam, C):
    """Eq. 6 under uniform inflation by lam: lam1 = lam2 = lam on every element,
    I1 = 2 lam^2 - 2, I2 = lam^4 - 1, E = kS/4 A0 (I1^2 + 2 I1 - 2 I2 + C I2^2)."""
    kS = 0.02
    X0, F = icosphere(2, 5.0, (1.0, 2.0, 3.0))
    c = np.array([1.0, 2.0, 3.0])
    X = c + lam * (X0 - c)
    E, _ = O.membrane(X, X0, F, kS=kS, C=C, which=1)
    A0 = O.mesh_area(X0, F)
    I1 = 2 * lam ** 2 - 2; I2 = lam ** 4 - 1
    assert np.isclose(E[0], kS / 4 * A0 * (I1 ** 2 + 2 * I1 - 2 * I2 + C * I2 ** 2), rtol=1e-12)


def test_skalak_uniaxial_triangle_closed_form():
    """One flat element stretched by s along x: lam1 = s, lam2 = 1, so
    I1 = I2 = s^2 - 1 and E = kS/4 A0 (1 + C)(s^2 - 1)^2."""
    X0 = np.array([[0.0, 0.0, 0.0], [1.3, 0.1, 0.0], [0.4, 0.9, 0.0]])
    F = np.array([[0, 1, 2]], np.int32)
    s, kS, C = 1.2, 0.5, 2.5
    X = X0 * np.array([s, 1.0, 1.0])
    E, _ = O.membrane(X, X0, F, kS=kS, C=C, which=1)
    A0 = 0.5 * abs(np.cross(X0[1] - X0[0], X0[2] - X0[0])[2])
    assert np.isclose(E[0], kS / 4 * A0 * (1 + C) * (s * s - 1) ** 2, rtol=1e-13)


def test_helfrich_sphere_limit_and_scale_invariance():
    """Eq. 7 with H0 = 0 on a sphere: E = kB/2 (2/R)^2 4 pi R^2 = 8 pi kB,
    independent of R; the discrete energy converges to it with refinement."""
    errs = []
    for level in (2, 3, 4):
        X, F = icosphere(level, 10.0)
        E = O.membrane(X, X, F, kB=1.0, which=2)[0][1]
        errs.append(abs(E / (8 * np.pi) - 1))
        X2, _ = icosphere(level, 3.7)
        E2 = O.membrane(X2, X2, F, kB=1.0, which=2)[0][1]
        assert np.isclose(E, E2, rtol=1e-12)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-3
    # second-order convergence in the edge length (ratio ~4 per level)
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_volume_area_closed_forms():
    """Divergence-theorem volume is exact for a unit cube mesh and converges to
    4/3 pi R^3 (area to 4 pi R^2) on refined icospheres."""
    cube = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float) + 2.5
    Fc = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                   [1, 2, 6], [1, 6, 5], [2, 3, 7], [2, 7, 6], [3, 0, 4], [3, 4, 7]], np.int32)
    assert np.isclose(O.mesh_volume(cube, Fc), 1.0, rtol=1e-14)
    assert np.isclose(O.mesh_area(cube, Fc), 6.0, rtol=1e-14)
    prev = None
    for level in (2, 3, 4, 5):
        X, F = icosphere(level, 7.0, (1, 2, 3))
        ev = abs(O.mesh_volume(X, F) / (4 / 3 * np.pi * 343) - 1)
        ea = abs(O.mesh_area(X, F) / (4 * np.pi * 49) - 1)
        if prev:
            assert ev < prev[0] / 3.5 and ea < prev[1] / 3.5
        prev = (ev, ea)
    assert prev[0] < 1e-3


def test_volume_penalty_closed_form():
    """Eq. 8 on a sphere scaled by lam: E = kV/2 (V - V0)^2 / V0 with V = lam^3 V0;
    the force on each node is radial (dV/dx points outward)."""
    X0, F = icosphere(3, 6.0)
    lam, kV = 1.07, 0.3
    X = lam * X0
    V0 = O.mesh_volume(X0, F)
    E, Fo = O.membrane(X, X0, F, kV=kV, which=4)
    assert np.isclose(E[2], kV / 2 * (lam ** 3 - 1) ** 2 * V0, rtol=1e-12)
    radial = np.einsum("ij,ij->i", Fo, X) / (np.linalg.norm(Fo, axis=1) * np.linalg.norm(X, axis=1))
    assert np.all(radial < -0.99)  # inflated: pulled back inward


def test_hertz_closed_form():
    """Eq. 11 (reading: overlap delta0 - d): F = 1.5 (1.5 - d)^1.5 for d < 1.5, else 0."""
    for d in (0.0, 0.3, 1.0, 1.49):
        assert np.isclose(O.hertz(d), 1.5 * (1.5 - d) ** 1.5, rtol=1e-15)
    assert O.hertz(1.5) == 0.0 and O.hertz(2.0) == 0.0
