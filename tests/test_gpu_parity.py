"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (float32 storage and arithmetic against float64):
  densities      max |rho_gpu - rho_or| / max |rho_or|            < 1e-5
  velocities     max |u_gpu - u_or| / max |u_or|                    < TOL_U
  populations    max |f_gpu - f_or| / max |f_or|                    < 1e-5
  cut links      bit-exact masks, elements and interior flags
  capsule force  |F_gpu - F_or| / max(|F_or|)                       < 1e-3
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_RHO = 1e-5
TOL_U = 2e-4


@pytest.fixture(scope="module")
def cfm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_15405_gb300 import build
    build.build()
    from paper_2007_15405_gb300 import capfilm
    capfilm.load_library()
    return capfilm


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def compare_state(sim, orc, tol_u=TOL_U, check_pops=True):
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    e_rho = rel(rg, ro)
    e_u = rel(ug, uo)
    assert e_rho < TOL_RHO, f"rho rel err {e_rho:.3e}"
    assert e_u < tol_u, f"u rel err {e_u:.3e}"
    if check_pops:
        fg = sim.populations().astype(np.float64)
        fo = orc.populations()
        assert rel(fg, fo) < TOL_RHO, f"population rel err {rel(fg, fo):.3e}"
    return e_rho, e_u


def compare_cuts(sim, orc):
    mg, tg, ig = sim.cuts()
    mo, to, io = orc.cuts()
    assert (mg == mo).all(), f"{(mg != mo).sum()} nodes differ in cut masks"
    bits = ((mo[..., None] >> np.arange(18, dtype=np.uint32)) & 1).astype(bool)
    assert (tg[bits] == to[bits]).all()
    assert (ig == io).all()


def test_rest_state_and_mass_no_capsule(cfm):
    wl = I.Workload("rest", 40, 12, 10, h_top=4.5, capsules=[], steps=30)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    m0 = sim.total_mass()
    sim.step(30); orc.step(30)
    compare_state(sim, orc)
    assert np.allclose(sim.total_mass(), m0, rtol=1e-6)


def test_cut_links_match_oracle(cfm):
    for mode in (I.MODE_FIXED, I.MODE_FREE):
        wl = I.tiny_film(mode=mode)
        sim = cfm.Simulation.from_workload(wl)
        orc = O.Oracle.from_workload(wl)
        compare_cuts(sim, orc)


@pytest.mark.parametrize("mode", [I.MODE_FIXED, I.MODE_FREE, I.MODE_FROZEN])
def test_tiny_film_parity(cfm, mode):
    wl = I.tiny_film(mode=mode, steps=40)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    sg = sim.capsule_state(0); so = orc.capsule_state(0)
    assert np.abs(sg["X"] - so["X"]).max() < 1e-5
    Fg, Tg = sim.capsule_force(0)
    assert np.abs(Fg - so["force"]).max() < 1e-3 * np.abs(so["force"]).max() + 1e-7
    assert abs(sg["area"] / so["area"] - 1) < 1e-6 and abs(sg["volume"] / so["volume"] - 1) < 1e-6
    if mode != I.MODE_FIXED:
        compare_cuts(sim, orc)


@pytest.mark.parametrize("tau", [(0.8, 0.8), (0.75, 1.3)])
def test_tiny_film_parity_other_tau(cfm, tau):
    """tau != 1 takes the general collision (second pull, BGK relaxation of
    the pulled populations); tau = 1, in every other test, the equilibrium
    stored from the density pass's momentum."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=40)
    wl.tau = tau
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    # tau = 0.75 relaxes faster and the node trajectories drift more: 3.1e-5 measured
    assert np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max() < 1e-4
    compare_cuts(sim, orc)


def test_ragged_periodic_no_wall(cfm):
    """Lattice not a multiple of the tile, fully periodic (no substrate),
    capsule crossing the periodic x boundary."""
    nx, ny, nz = 37, 13, 15
    X, F = I.icosphere(2, 4.0, (nx - 1.3, 6.4, 7.17))
    wl = I.Workload("ragged", nx, ny, nz, h_top=6.5, steps=25, wall=0, seed=5,
                    capsules=[I.CapsuleSpec(centre=(nx - 1.3, 6.4, 7.17), radius=4.0, level=2,
                                            kS=5e-3, C=1.0, kB=1e-3, mode=I.MODE_FREE)])
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    compare_cuts(sim, orc)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)


@pytest.mark.parametrize("across", [False, True])
def test_two_capsules_hertz_contact(cfm, across):
    """Two capsules closer than the Hertz range interact (Eq. 11); also across
    the periodic x boundary."""
    nx, ny, nz = 32, 16, 20
    xa, xb = (10.3, 19.1) if not across else (4.3, 27.5)
    caps = [I.CapsuleSpec(centre=(xa, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE),
            I.CapsuleSpec(centre=(xb, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE)]
    wl = I.Workload("contact", nx, ny, nz, h_top=8.5, capsules=caps, steps=20, rep_dz=2.0)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    for k in range(2):
        assert np.abs(sim.capsule_state(k)["X"] - orc.capsule_state(k)["X"]).max() < 1e-5


@pytest.mark.slow
def test_hundred_capsules_in_contact(cfm):
    """100 free capsules (R = 4, level 2) on a 10 x 10 grid of spacing 8.8 in
    an 88 x 88 x 20 lattice: every capsule within the Hertz range of its four
    neighbours, across both periodic boundaries too.  Node positions and
    capsule forces against the oracle after 5 steps."""
    caps = [I.CapsuleSpec(centre=(4.3 + 8.8 * i, 4.4 + 8.8 * j, 10.17), radius=4.0, level=2, C=1.0,
                          mode=I.MODE_FREE) for j in range(10) for i in range(10)]
    wl = I.Workload("hundred", 88, 88, 20, h_top=8.5, capsules=caps, steps=5, rep_dz=2.0, seed=5)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    for k in range(0, 100, 7):
        assert np.abs(sim.capsule_state(k)["X"] - orc.capsule_state(k)["X"]).max() < 1e-5, k
        Fg, _ = sim.capsule_force(k)
        Fo = orc.capsule_state(k)["force"]
        assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max() + 1e-7, k


def test_meniscus_field_matches_oracle(cfm):
    wl = I.tiny_film(mode=I.MODE_FIXED, steps=30)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    hg = sim.meniscus_field(); ho = orc.meniscus_field()
    assert (np.isnan(hg) == np.isnan(ho)).all()
    ok = ~np.isnan(ho)
    assert np.abs(hg[ok] - ho[ok]).max() < 1e-3


@pytest.mark.slow
def test_single_capsule_film_1000_steps_fixed(cfm):
    """32x32x48 lattice, R=8 capsule through a 12-cell film, 1000 steps: the
    float32 populations stay within 1e-5 of the FP64 oracle (densities)."""
    wl = I.single_capsule_film(mode=I.MODE_FIXED, steps=1000)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    e_rho, e_u = compare_state(sim, orc, tol_u=1e-4)
    print(f"fixed: rho {e_rho:.2e} u {e_u:.2e}")
    Fg, _ = sim.capsule_force(0)
    Fo = orc.capsule_state(0)["force"]
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()
    compare_cuts(sim, orc)


# A free membrane crosses lattice nodes; its float32-force trajectory differs
# from the FP64 one by ~1e-6 after a few hundred steps, so a crossing can land
# one step apart in the two runs.  Each such event perturbs the densities near
# the node by ~3e-5 (relative) for a few tens of steps before it relaxes
# (measured step by step on this workload); the bounds below are 3x that.
TOL_RHO_FREE = 1e-4
TOL_U_FREE = 2e-3


@pytest.mark.slow
def test_single_capsule_film_1000_steps_free(cfm):
    wl = I.single_capsule_film(mode=I.MODE_FREE, steps=1000)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    rg, ug = sim.fields(); ro, uo = orc.fields()
    e_rho, e_u = rel(rg, ro), rel(ug, uo)
    print(f"free: rho {e_rho:.2e} u {e_u:.2e}")
    assert e_rho < TOL_RHO_FREE and e_u < TOL_U_FREE
    assert np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max() < 1e-3
    Fg, _ = sim.capsule_force(0)
    Fo = orc.capsule_state(0)["force"]
    assert np.abs(Fg - Fo).max() < 1e-2 * np.abs(Fo).max()


def step_with_cut_override(sim, orc, steps, margin=1e-4):
    """Step both paths one step at a time; where the cut links the GPU
    computed on its float node positions differ from the oracle's, every
    difference must be a near tie of the oracle's decision (within `margin`
    lattice units), and the oracle then takes the GPU's cut structure.
    Returns the number of adopted link-end differences."""
    adopted = 0
    for _ in range(steps):
        sim.step(1); orc.step(1)
        mg = sim.cut_mask()
        if (mg != orc.cut_mask()).any():
            mg, tg, _ = sim.cuts()
            n = orc.override_cuts(mg, tg, margin)
            assert n >= 0, f"{-n} cut-link differences are not near ties"
            adopted += n
    return adopted


@pytest.mark.slow
def test_single_capsule_film_1000_steps_free_parity(cfm):
    """The free capsule of the 1000-step film held to the float32 tolerances
    (1e-5 on densities and velocities): the membrane's float32-force
    trajectory differs from the FP64 one by ~1e-6, so a link whose crossing
    is a near tie can be decided differently; the oracle then takes the GPU's
    cut structure (every difference must be a tie within 1e-4 lattice units),
    and the two runs go on from the same cut links."""
    wl = I.single_capsule_film(mode=I.MODE_FREE, steps=1000)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    adopted = step_with_cut_override(sim, orc, wl.steps)
    rg, ug = sim.fields(); ro, uo = orc.fields()
    e_rho, e_u = rel(rg, ro), rel(ug, uo)
    print(f"free with cut override: rho {e_rho:.2e} u {e_u:.2e}, {adopted} link ends adopted")
    assert e_rho < TOL_RHO and e_u < 1e-5, (e_rho, e_u, adopted)
    assert np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max() < 1e-4
    Fg, _ = sim.capsule_force(0)
    Fo = orc.capsule_state(0)["force"]
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()


@pytest.mark.slow
def test_capsule_pair_full_size_lateral_force(cfm):
    """128x64x64 with two R=12 capsules at d = 3R, the benchmark workload's
    launch configuration, 60 steps: fields and the lateral force vs oracle."""
    wl = I.capsule_pair(steps=60)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc, check_pops=False)
    Fg = sim.lateral_force(0, 1)
    Fo = orc.lateral_force(0, 1)
    assert abs(Fg - Fo) <= 1e-2 * abs(Fo) + 1e-7, (Fg, Fo)


@pytest.mark.parametrize("level,radius", [(1, 6.0), (0, 5.0)])
def test_cut_links_coarse_mesh(cfm, level, radius):
    """Elements several lattice units long (level-1 and level-0 icospheres):
    the cut links match the oracle at set-up and after free motion."""
    c = (12.3, 11.6, 12.17)
    wl = I.Workload("coarse", 24, 24, 24, h_top=12.5, steps=10, seed=8,
                    capsules=[I.CapsuleSpec(centre=c, radius=radius, level=level, kS=5e-3, C=1.0,
                                            kB=1e-3, mode=I.MODE_FREE)], rep_dz=2.0)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    compare_cuts(sim, orc)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_cuts(sim, orc)
    compare_state(sim, orc)


def test_element_longer_than_16_units_is_rejected(cfm):
    """An element spanning more than 16 lattice units is reported as
    CF_EOVERFLOW instead of being searched."""
    c = (32.3, 32.4, 32.17)
    wl = I.Workload("huge", 64, 64, 64, h_top=30.5, steps=1,
                    capsules=[I.CapsuleSpec(centre=c, radius=20.0, level=0, mode=I.MODE_FIXED)])
    with pytest.raises(cfm.CapfilmError, match="16 lattice units"):
        sim = cfm.Simulation.from_workload(wl)
        sim.step(1)


def profile_case(steps=120):
    """40x40x28 lattice, one fixed R=6 capsule through the film: a meniscus
    with a few rays' worth of columns on every side."""
    cap = I.CapsuleSpec(centre=(20.3, 19.4, 0.5 + 2.0 + 1.5 + 6.0 + 0.17), radius=6.0, level=3,
                        mode=I.MODE_FIXED)
    return I.Workload("profile", 40, 40, 28, h_top=0.5 + 2.0 + 0.5 * 6.0, capsules=[cap], steps=steps,
                      rep_dz=2.0, seed=31)


@pytest.mark.parametrize("dr", [1.0, 0.5])
def test_meniscus_profile_and_height_match_oracle(cfm, dr):
    """cf_meniscus_profile (device kernel) against the oracle's profile of its
    own fields: same valid samples, zeta and Z within 1e-3 lattice units
    (the column heights interpolate the densities, which agree to 1e-5)."""
    wl = profile_case()
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    rg, zg, Zg = sim.meniscus_profile(0, dr)
    ro, zo, Zo, _ = orc.meniscus_profile(0, dr)
    assert np.array_equal(rg, ro)
    assert np.array_equal(np.isnan(zg), np.isnan(zo))
    ok = ~np.isnan(zo)
    assert ok.sum() > len(zo) // 2
    assert np.abs(zg[ok] - zo[ok]).max() < 1e-3
    assert abs(Zg - Zo) < 1e-3 and Zo > 0.1
    if dr == 1.0:
        assert sim.meniscus_height(0) == Zg


def test_lateral_force_matches_oracle_fixed_pair(cfm):
    """Two fixed capsules at d = 3R: cf_lateral_force against the oracle's
    lateral force (coupling forces of both capsules projected on the line of
    centres) after 150 steps, within 1%."""
    R = 5.0
    caps = [I.CapsuleSpec(centre=(16.3 - 1.5 * R, 12.4, 0.5 + 2.0 + 1.5 + R + 0.17), radius=R, level=2,
                          mode=I.MODE_FIXED),
            I.CapsuleSpec(centre=(16.3 + 1.5 * R, 12.4, 0.5 + 2.0 + 1.5 + R + 0.17), radius=R, level=2,
                          mode=I.MODE_FIXED)]
    wl = I.Workload("pair", 40, 24, 22, h_top=0.5 + 2.0 + 0.6 * R, capsules=caps, steps=150, rep_dz=2.0,
                    seed=17)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    Fg, Fo = sim.lateral_force(0, 1), orc.lateral_force(0, 1)
    assert abs(Fo) > 1e-6
    assert abs(Fg - Fo) <= 1e-2 * abs(Fo), (Fg, Fo)


@pytest.mark.parametrize("wet", [0.05, -0.05])
def test_wetting_offset_parity(cfm, wet):
    """Non-neutral wetting (Sec. 3.1, last paragraph): the offset of the
    interpolated densities across the membrane, with a free capsule, against
    the oracle at the parity tolerances."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=40)
    wl.capsules[0].wet = wet
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    assert np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max() < 1e-5
    Fg, _ = sim.capsule_force(0)
    Fo = orc.capsule_state(0)["force"]
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max() + 1e-7
    compare_cuts(sim, orc)


def test_wetting_offset_raises_or_lowers_the_meniscus(cfm):
    """A film-philic surface (offset > 0) pulls the film up the particle, a
    film-phobic one (< 0) lets it down: the rise Z orders with the offset."""
    Z = {}
    for wet in (-0.1, 0.0, 0.1):
        wl = profile_case(steps=600)
        wl.capsules[0].wet = wet
        sim = cfm.Simulation.from_workload(wl)
        sim.step(wl.steps)
        Z[wet] = sim.meniscus_height(0)
        sim.close()
    assert Z[-0.1] < Z[0.0] < Z[0.1], Z


def test_meniscus_fit_and_theory_force_match_oracle(cfm):
    """cf_meniscus_fit and cf_capillary_force against the oracle's fit and
    theory force: on a profile made from the model (exact recovery by both)
    and on a simulated profile (the same least-squares minimum)."""
    sp = pytest.importorskip("scipy.special")
    r = np.arange(0.0, 40.0, 0.5)
    z = 0.6 * sp.k0(0.09 * np.maximum(r, 1e-9))
    lib = cfm.meniscus_fit(r, z, rmin=4.0)
    ora = O.meniscus_fit(r, z, rmin=4.0)
    assert lib[3] == ora[3]
    assert lib[0] == pytest.approx(0.6, rel=1e-10) and lib[1] == pytest.approx(0.09, rel=1e-10)
    assert ora[0] == pytest.approx(lib[0], rel=1e-10) and ora[1] == pytest.approx(lib[1], rel=1e-10)
    wl = profile_case(steps=300)
    sim = cfm.Simulation.from_workload(wl)
    sim.step(wl.steps)
    rp, zp, _ = sim.meniscus_profile(0, 0.5)
    lib = cfm.meniscus_fit(rp, zp, rmin=8.0)
    ora = O.meniscus_fit(rp, zp, rmin=8.0)
    assert lib[3] == ora[3] and lib[3] > 10
    assert lib[0] == pytest.approx(ora[0], rel=1e-6) and lib[1] == pytest.approx(ora[1], rel=1e-6)
    for L in (25.0, 60.0):
        F1 = cfm.capillary_force(lib[1], 0.0488, lib[0], lib[0], L)
        F2 = O.capillary_force(lib[1], 0.0488, lib[0], lib[0], L)
        assert F1 == pytest.approx(F2, rel=1e-12)


@pytest.mark.parametrize("flag", ["INERTIAL", "LADD_REF_RHO", "PARTNER_MIRROR"])
def test_alternative_readings_parity(cfm, flag):
    """The alternative readings of paper-silent points (inertial node update,
    Ladd's term with the reference density, mirrored partner density), each
    selected by a flag of both the library and the oracle: free capsule, 40
    steps, the parity tolerances."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=40)
    wl.flags = getattr(cfm, flag)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    assert np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max() < 1e-5
    Fg, _ = sim.capsule_force(0)
    Fo = orc.capsule_state(0)["force"]
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max() + 1e-7
    compare_cuts(sim, orc)


def test_drying_by_removal_parity(cfm):
    """Drying by removal (flag): the A mass goes, B keeps its mass; fields
    against the oracle after 30 steps, and the mass budget."""
    wl = I.tiny_film(mode=I.MODE_FIXED, steps=30)
    wl.flags = cfm.DRY_REMOVE
    wl.dry_dm = 0.02
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    m0 = orc.total_mass()
    sim.step(wl.steps); orc.step(wl.steps)
    compare_state(sim, orc)
    mg, mo = sim.total_mass(), orc.total_mass()
    assert mo[0] == pytest.approx(m0[0] - 30 * 0.02, rel=1e-10)
    assert np.allclose(mg, mo, rtol=1e-5)


@pytest.mark.slow
def test_equilibrated_lateral_force_matches_oracle(cfm):
    """A reduced fixed pair (64 x 40 x 40, R = 6 level-3 capsules at d = 3R,
    film 0.4R) run until its lateral force is stationary (change over the
    last 1000 steps below 0.5%; the force relaxes by about 30% less per
    window, and is 0.6% per window at 6000 steps): the GPU's equilibrated
    force within 1% of the oracle's."""
    R = 6.0
    zc = I.z_rest(R) + 0.17
    caps = [I.CapsuleSpec(centre=(32.3 - 1.5 * R, 20.4, zc), radius=R, level=3, mode=I.MODE_FIXED),
            I.CapsuleSpec(centre=(32.3 + 1.5 * R, 20.4, zc), radius=R, level=3, mode=I.MODE_FIXED)]
    wl = I.Workload("pair eq", 64, 40, 40, h_top=0.5 + I.REP_DZ + 0.4 * R, capsules=caps, steps=10000, seed=23)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    fg, fo = [], []
    for _ in range(10):
        sim.step(1000); orc.step(1000)
        fg.append(sim.lateral_force(0, 1)); fo.append(orc.lateral_force(0, 1))
    print("lateral force gpu", fg, "oracle", fo)
    assert abs(fg[-1] - fg[-2]) < 5e-3 * abs(fg[-1])   # stationary
    assert fo[-1] < 0 and abs(fg[-1] - fo[-1]) <= 1e-2 * abs(fo[-1]), (fg[-1], fo[-1])
