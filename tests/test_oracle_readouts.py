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


# ---------------------------------------------------- cut-structure override
def sheet_oracle(zs, G=0.0, wet=0.0):
    """A flat triangulated sheet at height zs over a 6 x 6 periodic box (the
    vertices offset by (0.3, 0.4), so no link passes near an element edge)."""
    nx, ny, nz = 6, 6, 12
    xs = 0.3 + 2.0 * np.arange(4)
    ys = 0.4 + 2.0 * np.arange(4)
    X = np.array([[x, y, zs] for y in ys for x in xs])
    F = []
    for j in range(3):
        for i in range(3):
            a = j * 4 + i
            F += [[a, a + 1, a + 5], [a, a + 5, a + 4]]
    o = O.Oracle(nx, ny, nz, wall=0, G=G)
    o.add_capsule(X, np.array(F, np.int32), 0.0, 0.0, 0.0, 0.0, 25.0, I.MODE_FIXED, wet=wet)
    return o


def flip_link(mask, tri, x, y, z, k, nx, ny, nz, T=0):
    e, _, op = O.tables()
    m = mask.copy(); t = tri.copy()
    x2, y2, z2 = (x + e[k, 0]) % nx, (y + e[k, 1]) % ny, (z + e[k, 2]) % nz
    m[z, y, x] ^= np.uint32(1 << (k - 1))
    m[z2, y2, x2] ^= np.uint32(1 << (op[k] - 1))
    t[z, y, x, k - 1] = T
    t[z2, y2, x2, op[k] - 1] = T
    return m, t


def test_override_rejects_a_flip_far_from_a_tie():
    """The sheet at z = 6.5 crosses every link from z = 6 to 7 half-way,
    far from its edges: a structure that disagrees there is refused and the
    oracle's stays."""
    o = sheet_oracle(6.5)
    m, t, _ = o.cuts()
    assert m[6, 2, 2] >> 4 & 1                       # +z link of (2, 2, 6) cut
    assert o.override_cuts(m, t) == 0                # identical: nothing to do
    m2, t2 = flip_link(m, t, 2, 2, 6, 5, 6, 6, 12)
    assert o.override_cuts(m2, t2, 1e-4) == -2       # both link ends differ, no tie
    assert np.array_equal(o.cuts()[0], m)


def test_override_adopts_a_flip_at_a_tie():
    """The sheet 3e-5 above the plane z = 6: the link (2, 2, 5) -> +z ends
    within the margin of the element plane, so either decision is a tie: the
    oracle adopts the given structure (and its interior flags).  With a
    margin below the distance it does not."""
    o = sheet_oracle(6.00003)
    m, t, _ = o.cuts()
    assert not (m[5, 2, 2] >> 4 & 1) and (m[6, 2, 2] >> 4 & 1)
    m2, t2 = flip_link(m, t, 2, 2, 5, 5, 6, 6, 12)
    assert o.override_cuts(m2, t2, 1e-6) == -2
    assert o.override_cuts(m2, t2, 1e-4) == 2
    assert np.array_equal(o.cuts()[0], m2)


# ------------------------------------------------------------------ wetting
@pytest.mark.parametrize("wet", [0.0, 0.05, -0.05])
def test_wetting_offset_on_a_flat_sheet(wet):
    """A uniform state (rho_A = 0.5, rho_B = 0.3) around a flat sheet at
    z = 6.5: the partner densities across the sheet's cut links are the
    uniform ones plus the offset (A: +wet, B: -wet), every other neighbour
    term cancels, and the five cut links of a node below the sheet carry
    sum w e_z = 1/18 + 4/36 = 1/6.  So F^A_z = -G psi_A/6 (psi(rho_B - wet)
    - psi(rho_B)) and F^B_z = -G psi_B/6 (psi(rho_A + wet) - psi(rho_A)),
    with the opposite sign above the sheet and no lateral force: a positive
    offset draws A towards the sheet (A-philic), a negative one B, zero is
    neutral."""
    o = sheet_oracle(6.5, G=3.6, wet=wet)
    _, w, _ = O.tables()
    f = np.zeros((2, 19, o.nz, o.ny, o.nx))
    f[0] = w[:, None, None, None] * 0.5
    f[1] = w[:, None, None, None] * 0.3
    o.set_populations(f)
    F = o.sc_forces()
    psi = lambda r: 1.0 - math.exp(-r)
    fa = -3.6 * psi(0.5) / 6.0 * (psi(0.3 - wet) - psi(0.3))
    fb = -3.6 * psi(0.3) / 6.0 * (psi(0.5 + wet) - psi(0.5))
    assert np.allclose(F[0, 2, 6], fa, atol=1e-15) and np.allclose(F[1, 2, 6], fb, atol=1e-15)
    assert np.allclose(F[0, 2, 7], -fa, atol=1e-15) and np.allclose(F[1, 2, 7], -fb, atol=1e-15)
    assert np.abs(F[:, :2]).max() < 1e-15
    far = [z for z in range(o.nz) if z not in (6, 7)]
    assert np.abs(F[:, :, far]).max() < 1e-15
    if wet > 0:
        assert fa > 0 and fb < 0
    elif wet < 0:
        assert fa < 0 and fb > 0
