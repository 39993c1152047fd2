"""Diffuse-interface (immersed-boundary) coupling on the GPU against the FP64
oracle, through the C ABI: Peskin-kernel spreading of the membrane forces,
the body force in the collision, the nodes moved with the interpolated fluid
velocity.  Tolerances are those of the cut-link parity tests (float32
storage and arithmetic against float64); the spread force is summed in
fixed point on the GPU (2^-40 per term), far below them."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_RHO = 1e-5
TOL_U = 2e-4
TOL_X = 1e-5


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


def run_pair(cfm, wl, steps=None):
    wl.flags = O.Oracle.IBM
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    n = wl.steps if steps is None else steps
    sim.step(n)
    orc.step(n)
    return sim, orc


def compare(sim, orc, ncaps, tol_u=TOL_U, tol_x=TOL_X):
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    assert rel(rg, ro) < TOL_RHO, f"rho rel err {rel(rg, ro):.3e}"
    assert rel(ug, uo) < tol_u, f"u rel err {rel(ug, uo):.3e}"
    fg = sim.populations().astype(np.float64)
    fo = orc.populations()
    assert rel(fg, fo) < TOL_RHO, f"population rel err {rel(fg, fo):.3e}"
    for k in range(ncaps):
        sg, so = sim.capsule_state(k), orc.capsule_state(k)
        dx = np.abs(sg["X"] - so["X"]).max()
        assert dx < tol_x, f"capsule {k}: node positions differ by {dx:.3e}"
        assert abs(sg["area"] / so["area"] - 1) < 1e-6 and abs(sg["volume"] / so["volume"] - 1) < 1e-6
        F, T = sim.capsule_force(k)  # no link is cut: no momentum exchange
        assert np.abs(F).max() == 0.0 and np.abs(T).max() == 0.0


def compare_inside(sim, orc):
    """The cut links of the moved membrane give the interior flags."""
    mg, _, ig = sim.cuts()
    mo, _, io = orc.cuts()
    assert (mg == mo).all(), f"{(mg != mo).sum()} nodes differ in cut masks"
    assert (ig == io).all()


@pytest.mark.parametrize("mode", [I.MODE_FREE, I.MODE_FIXED])
def test_ibm_tiny_film(cfm, mode):
    """A capsule through a film on the substrate: its stencils reach the
    substrate's solid plane (skipped) and both fluid components."""
    wl = I.tiny_film(mode=mode, steps=40)
    sim, orc = run_pair(cfm, wl)
    compare(sim, orc, 1)
    compare_inside(sim, orc)
    if mode == I.MODE_FREE:  # the membrane moved with the fluid
        X0 = wl.capsules[0].mesh()[0]
        assert np.abs(orc.capsule_state(0)["X"] - X0).max() > 1e-4


@pytest.mark.parametrize("tau", [(0.8, 0.8), (0.75, 1.3)])
def test_ibm_general_tau(cfm, tau):
    """tau != 1: the general collision (second pull, BGK of the pulled
    populations) adds the spread force the same way."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=30)
    wl.tau = tau
    sim, orc = run_pair(cfm, wl)
    compare(sim, orc, 1, tol_x=1e-4)


def test_ibm_periodic_ragged(cfm):
    """Fully periodic lattice that is no multiple of the tile, the capsule
    across the periodic x boundary: the stencils wrap in x."""
    nx, ny, nz = 37, 13, 15
    wl = I.Workload("ragged", nx, ny, nz, h_top=6.5, steps=25, wall=0, seed=5,
                    capsules=[I.CapsuleSpec(centre=(nx - 1.3, 6.4, 7.17), radius=4.0, level=2,
                                            kS=5e-3, C=1.0, kB=1e-3, mode=I.MODE_FREE)])
    sim, orc = run_pair(cfm, wl)
    compare(sim, orc, 1)
    compare_inside(sim, orc)


@pytest.mark.parametrize("across", [False, True])
def test_ibm_hertz_contact(cfm, across):
    """Two capsules within the Hertz range (Eq. 11): the contact forces are
    spread like the elastic ones, also across the periodic boundary."""
    nx, ny, nz = 32, 16, 20
    xa, xb = (10.3, 19.1) if not across else (4.3, 27.5)
    caps = [I.CapsuleSpec(centre=(xa, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE),
            I.CapsuleSpec(centre=(xb, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE)]
    wl = I.Workload("contact", nx, ny, nz, h_top=8.5, capsules=caps, steps=20, rep_dz=2.0)
    sim, orc = run_pair(cfm, wl)
    compare(sim, orc, 2)


def test_ibm_step_by_step_equals_graph(cfm):
    """Single steps and the captured step graph give the same bits, and two
    runs repeat bit for bit (the spread force is summed in fixed point)."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=12)
    wl.flags = O.Oracle.IBM
    a = cfm.Simulation.from_workload(wl)
    b = cfm.Simulation.from_workload(wl)
    c = cfm.Simulation.from_workload(wl)
    a.step(12)
    for _ in range(12):
        b.step(1)
    c.step(12)
    pa = a.populations()
    assert np.array_equal(pa, b.populations()) and np.array_equal(pa, c.populations())
    assert np.array_equal(a.capsule_state(0)["X"], b.capsule_state(0)["X"])
    assert np.array_equal(a.capsule_state(0)["X"], c.capsule_state(0)["X"])


def test_ibm_momentum_balance(cfm):
    """Fully periodic, no link cut: the Shan-Chen forces cancel over the
    lattice, the membrane's internal forces (Eqs. 6-8) sum to zero and the
    spreading weights of each node sum to one, so the fluid's total momentum
    stays at its start while the film's flow deforms and carries the capsule."""
    nx, ny, nz = 24, 20, 22
    wl = I.Workload("balance", nx, ny, nz, h_top=11.0, steps=150, wall=0, seed=3,
                    capsules=[I.CapsuleSpec(centre=(11.3, 9.8, 10.6), radius=5.0, level=2,
                                            kS=5e-3, C=1.0, kB=1e-3, mode=I.MODE_FREE)])
    wl.flags = O.Oracle.IBM
    sim = cfm.Simulation.from_workload(wl)
    e, _, _ = O.tables()
    f = sim.populations().astype(np.float64)
    p0 = np.einsum("cizyx,ia->a", f, e)
    X0 = sim.capsule_state(0)["X"]
    sim.step(wl.steps)
    f = sim.populations().astype(np.float64)
    p1 = np.einsum("cizyx,ia->a", f, e)
    assert np.abs(sim.capsule_state(0)["X"] - X0).max() > 1e-3
    assert np.abs(p1 - p0).max() < 1e-7 * f.sum()


@pytest.mark.slow
def test_ibm_hundred_capsules_in_contact(cfm):
    """100 free capsules on a 10 x 10 grid of spacing 8.8 in an 88 x 88 x 20
    lattice, each within the Hertz range of its four neighbours (also across
    both periodic boundaries), with contact-partner lists: node positions
    against the oracle after 5 steps."""
    caps = [I.CapsuleSpec(centre=(4.3 + 8.8 * i, 4.4 + 8.8 * j, 10.17), radius=4.0, level=2, C=1.0,
                          mode=I.MODE_FREE) for j in range(10) for i in range(10)]
    wl = I.Workload("hundred", 88, 88, 20, h_top=8.5, capsules=caps, steps=5, rep_dz=2.0, seed=5)
    sim, orc = run_pair(cfm, wl)
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    assert rel(rg, ro) < TOL_RHO and rel(ug, uo) < TOL_U
    for k in range(0, 100, 7):
        assert np.abs(sim.capsule_state(k)["X"] - orc.capsule_state(k)["X"]).max() < TOL_X, k


def test_ibm_drying(cfm):
    """Drying (A turned into B at A-majority nodes, Sec. 3.2 reading) with the
    diffuse-interface coupling, against the oracle."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=30)
    wl.dry_dm = 0.05
    sim, orc = run_pair(cfm, wl)
    compare(sim, orc, 1)
    mg, mo = sim.total_mass(), orc.total_mass()
    assert np.abs(mg - mo).max() < 1e-6 * mo.sum()


# 16-bit storage against the FP64 oracle: 3x the measured maxima of the
# cut-link coupling's 16-bit parity (tests/test_gpu_precision.py)
BOUNDS_16 = {1: dict(rho=2e-4, u=8e-3, X=1.2e-4), 2: dict(rho=1.2e-3, u=6e-2, X=5e-4)}


@pytest.mark.parametrize("prec", [1, 2])
def test_ibm_16bit_storage(cfm, prec):
    """FP16 / BF16 population storage with the diffuse-interface coupling."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=40)
    wl.flags = O.Oracle.IBM
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps)
    orc.step(wl.steps)
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    e = dict(rho=rel(rg, ro), u=rel(ug, uo),
             X=np.abs(sim.capsule_state(0)["X"] - orc.capsule_state(0)["X"]).max())
    for k, v in e.items():
        assert v < BOUNDS_16[prec][k], (k, v)


def test_ibm_restart_is_bit_identical(cfm, tmp_path):
    """A checkpoint of a diffuse-interface run (its cut links rebuilt for the
    saved positions) restarts into the same bits."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=1)
    wl.flags = O.Oracle.IBM
    a = cfm.Simulation.from_workload(wl)
    a.step(17)
    path = str(tmp_path / "ibm.bin")
    a.save(path)
    a.step(20)
    b = cfm.Simulation.from_workload(wl, set_film=False)
    b.load(path)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.capsule_state(0)["X"], b.capsule_state(0)["X"])
    assert (a.cuts()[0] == b.cuts()[0]).all()


def test_ibm_meniscus_readouts_between_steps(cfm):
    """Readouts rebuild the cut links for the positions of the moment; taken
    between steps they change nothing of the run, and the meniscus field
    equals the oracle's."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=30)
    wl.flags = O.Oracle.IBM
    a = cfm.Simulation.from_workload(wl)
    b = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    for _ in range(3):
        a.step(10)
        a.meniscus_field()
    b.step(30)
    orc.step(30)
    assert np.array_equal(a.populations(), b.populations())
    hg, ho = a.meniscus_field(), orc.meniscus_field()
    assert (np.isnan(hg) == np.isnan(ho)).all()
    ok = ~np.isnan(ho)
    assert np.abs(hg[ok] - ho[ok]).max() < 1e-3


def test_ibm_rejections(cfm):
    """Frozen capsules, the inertial reading and batches need the cut-link
    coupling."""
    wl = I.tiny_film(mode=I.MODE_FROZEN, steps=1)
    wl.flags = O.Oracle.IBM
    with pytest.raises(RuntimeError, match="frozen"):
        cfm.Simulation.from_workload(wl)
    wl = I.tiny_film(mode=I.MODE_FREE, steps=1)
    wl.flags = O.Oracle.IBM | O.Oracle.INERTIAL
    with pytest.raises(RuntimeError, match="CF_INERTIAL"):
        cfm.Simulation.from_workload(wl)
    wl.flags = O.Oracle.IBM
    sim = cfm.Simulation.from_workload(wl)
    with pytest.raises(RuntimeError, match="batch"):
        cfm.Batch([sim])
