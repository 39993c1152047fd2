"""Pins of the oracle's diffuse-interface (immersed-boundary) coupling, a
variant of the cut-link bounce-back coupling that is not part of the paper:
Peskin's 4-point kernel, spreading and interpolation, and one coupled step
against fields derived by hand from the pinned membrane forces."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I


@pytest.mark.parametrize("x", [0.0, 0.13, 0.5, 0.77, 0.999])
def test_kernel_moments(x):
    """Shifts of the kernel sum to one, have zero first moment and squares
    summing to 3/8, at every offset (the kernel's defining properties)."""
    r = np.array([x + 1.0, x, x - 1.0, x - 2.0])
    phi = np.array([O.peskin(v) for v in r])
    assert abs(phi.sum() - 1.0) < 1e-14
    assert abs((r * phi).sum()) < 1e-14
    assert abs((phi ** 2).sum() - 3.0 / 8.0) < 1e-14
    assert O.peskin(2.0) == 0.0 and O.peskin(-2.5) == 0.0 and abs(O.peskin(0.0) - 0.5) < 1e-15


def ibm_box(nx=16, ny=14, nz=12, wall=0):
    return O.Oracle(nx, ny, nz, wall=wall, G=0.0, flags=O.Oracle.IBM)


def test_spread_conserves_force_and_its_moment():
    o = ibm_box()
    X = np.array([7.3, 6.85, 5.2])
    F = np.array([0.3, -0.7, 1.1])
    f = o.ibm_spread_point(X, F).reshape(3, o.nz, o.ny, o.nx)
    assert np.allclose(f.sum(axis=(1, 2, 3)), F, atol=1e-14)
    z, y, x = np.meshgrid(np.arange(o.nz), np.arange(o.ny), np.arange(o.nx), indexing="ij")
    pos = np.stack([x, y, z])
    for a in range(3):  # sum of x_a f_b = X_a F_b: the kernel's zero first moment
        assert np.allclose((pos[a] * f).sum(axis=(1, 2, 3)), X[a] * F, atol=1e-12)


def test_interpolation_is_exact_for_linear_fields_and_adjoint_to_spreading():
    o = ibm_box()
    X = np.array([8.4, 5.55, 6.1])
    z, y, x = np.meshgrid(np.arange(o.nz), np.arange(o.ny), np.arange(o.nx), indexing="ij")
    a0 = np.array([0.01, -0.02, 0.005])
    B = np.array([[1e-3, 2e-3, -1e-3], [0.0, -3e-3, 1e-3], [2e-3, 0.0, 4e-4]])
    u = np.stack([a0[i] + B[i, 0] * x + B[i, 1] * y + B[i, 2] * z for i in range(3)])
    assert np.allclose(o.ibm_interp_point(u, X), a0 + B @ X, atol=1e-14)
    rng = np.random.default_rng(3)
    ur = rng.standard_normal(3 * o.nx * o.ny * o.nz)
    F = rng.standard_normal(3)
    lhs = o.ibm_interp_point(ur, X) @ F
    rhs = ur @ o.ibm_spread_point(X, F)
    assert abs(lhs - rhs) < 1e-12


def capsule_in_quiescent_fluid(o, centre, wall, R=4.0, kB=1e-3):
    X, F = I.icosphere(2, R)
    X = np.asarray(X) + np.asarray(centre)
    o.add_capsule(X, F, 5e-3, 1.0, kB, 1.0, 1.0, 0)
    f = np.zeros((2, 19, o.nz, o.ny, o.nx))
    _, w, _ = O.tables()
    for i in range(19):
        f[:, i] = 0.5 * w[i]
    if wall:
        f[:, :, 0] = 0.0
    o.set_populations(f)
    return o.capsule_state(0)["X"], np.asarray(F)  # positions as stored (float32-rounded)


def test_uniform_flow_carries_the_capsule():
    """No wall, G = 0, a relaxed capsule (no bending) in a uniform flow: the
    nodes move by the flow velocity (the kernel's shifts sum to one)."""
    o = ibm_box(20, 20, 20)
    X0, F = capsule_in_quiescent_fluid(o, (10.3, 10.4, 10.17), 0, kB=0.0)
    U = np.array([0.01, -0.004, 0.002])
    f = np.zeros((2, 19, o.nz, o.ny, o.nx))
    for i in range(19):
        f[:, i] = 0.5 * O.equilibrium(1.0, U)[i]
    o.set_populations(f)
    o.step(1)
    X1 = o.capsule_state(0)["X"]
    assert np.allclose(X1 - X0, U, atol=1e-12)


def test_first_step_against_hand_fields():
    """Quiescent uniform fluid (both components 0.5, G = 0) with a substrate and
    a capsule whose bottom lies within the Hertz range of the repulsive plane:
    after one step the reported velocity is half the spread membrane force
    (elastic forces of the pinned membrane functions plus the plane's Hertz
    push) over the density, and every node has moved by that velocity
    interpolated at its position."""
    o = O.Oracle(24, 24, 24, wall=1, G=0.0, rep_dz=2.0, flags=O.Oracle.IBM)
    zrep = 0.5 + 2.0
    X0, F = capsule_in_quiescent_fluid(o, (12.3, 12.4, zrep + 4.0 + 1.0), 1)
    _, Fel = O.membrane(X0, X0, F, kS=5e-3, C=1.0, kB=1e-3, kV=1.0)
    d = X0[:, 2] - zrep
    Fh = np.zeros_like(X0)
    near = d < I.DELTA0
    assert near.any()
    Fh[near, 2] = I.XI * (I.DELTA0 - d[near]) ** 1.5  # Eq. 11, pinned in test_oracle_membrane
    fsp = np.zeros(3 * o.N)
    for v in range(X0.shape[0]):
        o.ibm_spread_point(X0[v], Fel[v] + Fh[v], fsp)
    o.step(1)
    rho, u = o.fields()
    fluid = np.zeros((o.nz, o.ny, o.nx), bool)
    fluid[1:] = True
    expect = 0.5 * fsp.reshape(3, o.nz, o.ny, o.nx) / 1.0
    assert np.allclose(rho.sum(0)[fluid], 1.0, atol=1e-14)
    assert np.abs(u[:, fluid] - expect[:, fluid]).max() < 1e-15 + 1e-12 * np.abs(expect).max()
    X1 = o.capsule_state(0)["X"]
    moved = np.array([o.ibm_interp_point(u, X0[v]) for v in range(X0.shape[0])])
    assert np.allclose(X1 - X0, moved, atol=1e-15)
    assert np.abs(moved).max() > 1e-7  # the capsule does move


def test_drying_with_the_diffuse_interface():
    """Drying composes with the diffuse-interface step: with a capsule in the
    film the A inventory still falls by exactly dm per step and the total mass
    stays (the spread force moves momentum, no mass)."""
    o = O.Oracle(14, 12, 18, wall=1, rep_dz=2.0, flags=O.Oracle.IBM)
    X, F = I.icosphere(2, 4.0, (7.3, 5.9, 9.17))
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, I.MODE_FREE)
    o.set_film(8.0, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, I.jitter((18, 12, 14), 1e-3, seed=2))
    m0 = o.total_mass()
    dm = 0.04
    o.remove_mass(dm)
    o.step(6)
    m = o.total_mass()
    assert abs((m0[0] - m[0]) - 6 * dm) < 1e-10
    assert abs(m.sum() - m0.sum()) < 1e-10


def test_flag_value_agrees_with_the_library_header_and_binding():
    """The diffuse-interface flag has one value in the C header, the Python
    binding and the oracle."""
    import os
    import re
    from paper_2007_15405_gb300 import capfilm as cfm
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "capfilm.h")).read()
    m = re.search(r"CF_IBM\s*=\s*(\d+)", hdr)
    assert m and int(m.group(1)) == cfm.IBM == O.Oracle.IBM


def test_diverged_membrane_is_reported():
    """A capsule placed below the repulsive plane (z = 10.5) meets Hertz forces
    of order Xi (delta0 - d)^1.5 with d ~ -5 and is thrown apart in one step;
    the oracle reports the diverged membrane instead of searching the
    exploded elements for cut links."""
    o = O.Oracle(14, 12, 18, wall=1, rep_dz=10.0, flags=O.Oracle.IBM)
    X, F = I.icosphere(2, 4.0, (7.3, 5.9, 9.17))
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, I.MODE_FREE)
    o.set_film(8.0, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, None)
    with pytest.raises(RuntimeError, match="16 lattice units"):
        o.step(4)


def _random_point_cases():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    return hyp, st


def test_spreading_and_interpolation_at_random_positions():
    """At any position, also across the periodic boundaries and next to the
    substrate: interpolation is the adjoint of spreading, spreading keeps the
    force where no stencil node is solid, and the weights of a point sum to
    one there (a constant field is interpolated exactly)."""
    hyp, st = _random_point_cases()
    o_per = ibm_box(9, 8, 7, wall=0)
    o_sub = ibm_box(9, 8, 7, wall=1)
    rng = np.random.default_rng(11)
    fields = {id(o): rng.standard_normal(3 * o.N) for o in (o_per, o_sub)}

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(st.floats(-3.0, 12.0), st.floats(-3.0, 11.0), st.floats(0.0, 7.0), st.booleans())
    def check(x, y, z, wall):
        o = o_sub if wall else o_per
        X = np.array([x, y, z])
        F = np.array([0.7, -1.3, 0.4])
        f = o.ibm_spread_point(X, F)
        u = fields[id(o)]
        assert abs(o.ibm_interp_point(u, X) @ F - u @ f) < 1e-11
        zs = [int(np.floor(z)) - 1 + k for k in range(4)]
        if not wall or all(zz % o.nz != 0 for zz in zs):
            assert np.allclose(f.reshape(3, -1).sum(axis=1), F, atol=1e-13)
            const = np.concatenate([np.full(o.N, c) for c in (0.3, -0.2, 0.1)])
            assert np.allclose(o.ibm_interp_point(const, X), [0.3, -0.2, 0.1], atol=1e-14)

    check()
