"""Pins of the oracle parts the earlier pins left open: the partner density
across cut and substrate links (Sec. 3.1, last paragraph; reading c10), the
node-node and node-plane Hertz forces (Eq. 11; reading c12), the meniscus
profile with its far-field height and rise Z (Sec. 4.1; reading c21) and the
lateral force (Eq. 3 sign; reading c22).  CPU only.

Expected values are worked out by hand for the stated inputs (the literals
below), or follow from symmetry or exact arithmetic of the construction.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I


def linear_rho(nx, ny, nz):
    """rho(x, y, z) = x + 10 y + 100 z, as [nz, ny, nx]."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (x + 10 * y + 100 * z).astype(np.float64)


def cut_one_link(o, x, y, z, k):
    """Cut structure with the single link (x, y, z) -> (x, y, z) + e_k cut."""
    e, _, op = O.tables()
    mask = np.zeros((o.nz, o.ny, o.nx), np.uint32)
    tri = np.full((o.nz, o.ny, o.nx, 18), -1, np.int32)
    x2, y2, z2 = (x + e[k, 0]) % o.nx, (y + e[k, 1]) % o.ny, (z + e[k, 2]) % o.nz
    mask[z, y, x] |= np.uint32(1 << (k - 1))
    mask[z2, y2, x2] |= np.uint32(1 << (op[k] - 1))
    tri[z, y, x, k - 1] = 0
    tri[z2, y2, x2, op[k] - 1] = 0
    return mask, tri


# ---------------------------------------------------------------- rho_interp
def test_rho_interp_across_one_cut_link():
    """Node (2, 2, 2) of a periodic 5^3 box, link +x cut, rho = x + 10y + 100z:
    the mean over the node and its 17 neighbours through uncut links.  The 18
    neighbours sum to 18 * 222 (offsets cancel); dropping (3, 2, 2) = 223 and
    adding the node itself gives 3995 over 18 values.  The far node sees the
    same link as -x: 18 * 223 - 222 + 223 = 4015 over 18."""
    o = O.Oracle(5, 5, 5, wall=0)
    rho = linear_rho(5, 5, 5)
    o.set_cuts(*cut_one_link(o, 2, 2, 2, 1))
    assert o.rho_interp(rho, 2, 2, 2) == pytest.approx(3995.0 / 18.0, rel=1e-15)
    assert o.rho_interp(rho, 3, 2, 2) == pytest.approx(4015.0 / 18.0, rel=1e-15)
    # a node with no cut link averages all 19 values: the node's own value
    assert o.rho_interp(rho, 2, 3, 2) == pytest.approx(232.0, rel=1e-15)


def test_rho_interp_next_to_the_substrate():
    """With the substrate (plane z = 0 solid), node (2, 2, 1) drops its five
    links with e_z = -1: 18 * 122 - (22 + 21 + 23 + 12 + 32) + 122 = 2208 over
    14 values; with link +y cut as well, (2, 3, 1) = 132 goes too: 2076 / 13.
    The top plane z = 4 drops the five links that wrap onto the substrate:
    8 * 422 + 5 * 322 + 422 = 5408 over 14."""
    o = O.Oracle(5, 5, 5, wall=1)
    rho = linear_rho(5, 5, 5)
    assert o.rho_interp(rho, 2, 2, 1) == pytest.approx(2208.0 / 14.0, rel=1e-15)
    assert o.rho_interp(rho, 2, 2, 4) == pytest.approx(5408.0 / 14.0, rel=1e-15)
    o.set_cuts(*cut_one_link(o, 2, 2, 1, 3))
    assert o.rho_interp(rho, 2, 2, 1) == pytest.approx(2076.0 / 13.0, rel=1e-15)


def test_uniform_state_is_a_fixed_point_with_capsule_and_substrate():
    """A uniform two-component rest state (inside and outside a resting
    capsule) above the substrate stays put: bounce-back returns the rest
    populations, every partner density equals the uniform one, so the
    Shan-Chen forces vanish and the exchanges of the two sides of every cut
    link cancel on the element."""
    nx, ny, nz = 14, 13, 16
    o = O.Oracle(nx, ny, nz, wall=1, rep_dz=2.0)
    X, F = I.icosphere(2, 4.0, (7.3, 6.4, 8.17))
    o.add_capsule(X, F, 5e-3, 1.0, 1e-3, 1.0, 25.0, I.MODE_FIXED)
    _, w, _ = O.tables()
    f = np.zeros((2, 19, nz, ny, nx))
    f[0] = w[:, None, None, None] * 0.55
    f[1] = w[:, None, None, None] * 0.3
    f[:, :, 0] = 0.0
    o.set_populations(f)
    o.step(3)
    assert np.abs(o.populations() - f).max() < 1e-15
    s = o.capsule_state(0)
    assert np.abs(s["force"]).max() < 1e-13 and np.abs(s["Fcpl"]).max() < 1e-15
    _, u = o.fields()
    assert np.abs(u).max() < 1e-15


# --------------------------------------------------------------------- Hertz
def tetra(tip, back, spread=1.5):
    """A tetrahedron with apex `tip` and its base three units behind it along
    x (back = -1 or +1 gives the side), faces oriented outward."""
    tip = np.asarray(tip, np.float64)
    base = tip + np.array([3.0 * back, 0.0, 0.0])
    X = np.array([tip,
                  base + [0.0, spread, 0.0],
                  base + [0.0, -0.5 * spread, 0.866 * spread],
                  base + [0.0, -0.5 * spread, -0.866 * spread]])
    F = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 1], [1, 3, 2]], np.int32)
    c = X.mean(0)
    for f in F:
        n = np.cross(X[f[1]] - X[f[0]], X[f[2]] - X[f[0]])
        if np.dot(n, X[f[0]] - c) < 0:
            f[[1, 2]] = f[[2, 1]]
    return X, F


def rest_box(o, rA=0.5, rB=0.3):
    _, w, _ = O.tables()
    f = np.zeros((2, 19, o.nz, o.ny, o.nx))
    f[0] = w[:, None, None, None] * rA
    f[1] = w[:, None, None, None] * rB
    o.set_populations(f)


@pytest.mark.parametrize("periodic", [False, True])
def test_hertz_node_pair_equal_and_opposite(periodic):
    """Two capsules whose apexes are 0.92736 apart (0.9, 0.2, 0.1), every
    other node pair farther than delta0: only the apexes feel Eq. 11, with
    Xi (delta0 - d)^1.5 = 1.5 * 0.57264^1.5 along the separation, away from
    each other, equal and opposite.  In the periodic case the second apex
    sits across the x boundary (its nearest image is 0.9 away)."""
    nx, ny, nz = 16, 12, 12
    o = O.Oracle(nx, ny, nz, wall=0, G=0.0)
    if periodic:
        ta, tb = (0.3, 6.0, 6.0), (nx - 0.6, 6.2, 6.1)
        sa, sb = 1, -1   # apex a points -x, towards b's image
    else:
        ta, tb = (6.0, 6.0, 6.0), (6.9, 6.2, 6.1)
        sa, sb = -1, 1
    Xa, Fa = tetra(ta, sa)
    Xb, Fb = tetra(tb, sb)
    o.add_capsule(Xa, Fa, 0.0, 0.0, 0.0, 0.0, 25.0, I.MODE_FIXED)
    o.add_capsule(Xb, Fb, 0.0, 0.0, 0.0, 0.0, 25.0, I.MODE_FIXED)
    rest_box(o)
    o.step(1)
    _, Ia = o.capsule_forces(0)
    _, Ib = o.capsule_forces(1)
    d = math.sqrt(0.9 ** 2 + 0.2 ** 2 + 0.1 ** 2)
    assert 1.5 * (1.5 - d) ** 1.5 == pytest.approx(0.6499975, rel=1e-6)   # worked by hand
    # the oracle starts from the single-precision node positions the GPU
    # stores: the separation of the float-rounded apexes (nearest image)
    sep = Xa[0].astype(np.float32).astype(np.float64) - Xb[0].astype(np.float32).astype(np.float64)
    sep[0] -= nx * np.floor(sep[0] / nx + 0.5)
    assert np.allclose(sep, [-0.9, -0.2, -0.1] if not periodic else [0.9, -0.2, -0.1], atol=1e-6)
    dd = np.linalg.norm(sep)
    mag = 1.5 * (1.5 - dd) ** 1.5
    assert np.allclose(Ia[0], mag * sep / dd, rtol=1e-12, atol=1e-15)
    assert np.allclose(Ib[0], -Ia[0], rtol=1e-15, atol=1e-15)
    assert np.abs(Ia[1:]).max() == 0.0 and np.abs(Ib[1:]).max() == 0.0
    # repulsive: apex a is pushed away from b
    assert (Ia[0][0] < 0) != periodic


def test_hertz_node_plane():
    """A node 0.5 above the repulsive plane (z_rep = 2.5) is pushed up by
    Xi (delta0 - 0.5)^1.5 = 1.5; nodes 2 or more above it feel nothing."""
    o = O.Oracle(12, 12, 14, wall=1, G=0.0, rep_dz=2.0)
    X = np.array([[6.0, 6.0, 3.0], [7.5, 6.0, 5.5], [5.25, 7.3, 5.5], [5.25, 4.7, 5.5]])
    F = np.array([[0, 2, 1], [0, 3, 2], [0, 1, 3], [1, 2, 3]], np.int32)
    c = X.mean(0)
    for f in F:
        n = np.cross(X[f[1]] - X[f[0]], X[f[2]] - X[f[0]])
        if np.dot(n, X[f[0]] - c) < 0:
            f[[1, 2]] = f[[2, 1]]
    o.add_capsule(X, F, 0.0, 0.0, 0.0, 0.0, 25.0, I.MODE_FIXED)
    rest_box(o)
    o.step(1)
    _, Fi = o.capsule_forces(0)
    assert Fi[0] == pytest.approx([0.0, 0.0, 1.5], abs=1e-15)
    assert np.abs(Fi[1:]).max() == 0.0


# ---------------------------------------------------------- meniscus profile
def cone_field(nx, ny, x0, y0, base=5.0, a=3.0, b=0.5):
    """h = base + max(0, a - b r), r the periodic distance to column (x0, y0)."""
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    dx = (x - x0 + nx / 2) % nx - nx / 2
    dy = (y - y0 + ny / 2) % ny - ny / 2
    return base + np.maximum(0.0, a - b * np.sqrt(dx * dx + dy * dy))


@pytest.mark.parametrize("dr", [1.0, 0.5])
def test_meniscus_profile_of_a_cone(dr):
    """A cone of height 3 and slope 1/2 on a flat film at 5, centred on the
    column nearest to the capsule: the far field is the flat film, the four
    rays see zeta(r) = max(0, 3 - r/2) exactly (linear between columns, kink
    on a column), Z = 3."""
    nx, ny = 40, 36
    h = cone_field(nx, ny, 12, 15)
    r, z, Z, hinf = O.meniscus_profile_of(h, [(12.2, 15.4)], 0, dr)
    assert hinf == 5.0
    assert len(r) == int(18 / dr)
    assert np.allclose(r, dr * np.arange(len(r)), rtol=0, atol=0)
    assert np.abs(z - np.maximum(0.0, 3.0 - 0.5 * r)).max() < 1e-14
    assert Z == 3.0


def test_meniscus_profile_skips_capsule_columns_and_second_capsule():
    """Columns inside the capsule (NaN, r <= 1.5) drop the samples that touch
    them; the far field is taken away from both capsules; a tilted ray
    average: +x rays see the cone, -x rays a cone of slope 1."""
    nx, ny = 40, 36
    h = cone_field(nx, ny, 12, 15)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    # the -x ray: a steeper cone (height 3, slope 1) on its side only
    left = (x < 12) & (y == 15)
    h[left] = 5.0 + np.maximum(0.0, 3.0 - 1.0 * (12 - x[left]))
    h[np.hypot(x - 12, y - 15) <= 1.5] = np.nan
    r, z, Z, hinf = O.meniscus_profile_of(h, [(12.2, 15.4), (31.6, 4.3)], 0, 0.5)
    assert hinf == 5.0
    assert np.isnan(z[:4]).all()          # r = 0, 0.5, 1, 1.5 touch a NaN column
    rv = r[4:]
    exp = (3 * np.maximum(0.0, 3.0 - 0.5 * rv) + np.maximum(0.0, 3.0 - rv)) / 4.0
    assert np.abs(z[4:] - exp).max() < 1e-14
    assert Z == pytest.approx((3 * 2.0 + 1.0) / 4.0, abs=1e-15)   # at r = 2


def test_meniscus_profile_of_context_matches_its_field():
    """The context's profile is the profile of its own height field and
    capsule centroids."""
    wl = I.tiny_film(mode=I.MODE_FIXED, steps=5)
    o = O.Oracle.from_workload(wl)
    o.step(5)
    h = o.meniscus_field()
    X = o.capsule_state(0)["X"]
    r0, z0, Z0, h0 = O.meniscus_profile_of(h, [X.mean(0)[:2]], 0, 1.0)
    r1, z1, Z1, h1 = o.meniscus_profile(0, 1.0)
    assert np.array_equal(r0, r1) and np.array_equal(np.isnan(z0), np.isnan(z1))
    ok = ~np.isnan(z0)
    assert np.array_equal(z0[ok], z1[ok]) and Z0 == Z1 and h0 == h1


# ------------------------------------------------------------- lateral force
def test_lateral_force_hand_values():
    """F = 1/2 (F_b - F_a) . e_ab: along x, along (0.6, 0.8), across the
    periodic x boundary (the nearest image of b lies at -x) and for
    coincident centroids."""
    Fa, Fb = [0.3, -0.1, 0.2], [-0.5, 0.4, 0.0]
    assert O.lateral_force_of(Fa, Fb, [10, 5], [20, 5], 32, 32) == pytest.approx(-0.4, rel=1e-15)
    assert O.lateral_force_of(Fa, Fb, [10, 5], [13, 9], 32, 32) == pytest.approx(-0.04, rel=1e-14)
    assert O.lateral_force_of(Fa, Fb, [2, 5], [29, 5], 32, 32) == pytest.approx(0.4, rel=1e-15)
    assert math.isnan(O.lateral_force_of(Fa, Fb, [2, 5], [2, 5], 32, 32))


def test_lateral_force_of_mirror_pair_is_antisymmetric():
    """Two fixed capsules placed mirror-symmetrically about x = nx/2 (off the
    lattice links) in a film without jitter: the x coupling forces are
    opposite (to the single-precision rounding of the node positions), the
    lateral force is F_b,x, and swapping a and b leaves it unchanged."""
    nx, ny, nz = 36, 16, 20
    caps = [I.CapsuleSpec(centre=(10.3, 8.4, 10.17), radius=4.0, level=2, mode=I.MODE_FIXED),
            I.CapsuleSpec(centre=(25.7, 8.4, 10.17), radius=4.0, level=2, mode=I.MODE_FIXED)]
    wl = I.Workload("mirror", nx, ny, nz, h_top=9.5, capsules=caps, steps=8, rep_dz=2.0,
                    jitter_amp=0.0)
    o = O.Oracle.from_workload(wl)
    o.step(8)
    Fa = o.capsule_state(0)["force"]; Fb = o.capsule_state(1)["force"]
    assert abs(Fa[0]) > 1e-6
    assert Fa[0] == pytest.approx(-Fb[0], rel=1e-4)
    L = o.lateral_force(0, 1)
    assert L == pytest.approx(0.5 * (Fb[0] - Fa[0]), rel=1e-12)
    assert L == pytest.approx(Fb[0], rel=1e-4)
    assert o.lateral_force(1, 0) == pytest.approx(L, rel=1e-12)
