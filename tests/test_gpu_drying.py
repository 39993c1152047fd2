"""Drying (A turned into B each step to lower the film) on the GPU against the
FP64 oracle: element-wise parity in float32, the A inventory falling by the
requested mass per step in every storage mode, reproducible runs, and the
mixed-precision drying film with four capsules (128x128x48) with the error
of every reported quantity stated.

Tolerances as in the other parity tests: float32 densities 1e-5 relative,
velocities 2e-4; 16-bit modes the bounds of the precision tests.  The A
inventory is read back in FP64 from float32 / 16-bit storage: relative 1e-5
of the inventory (float32), 1e-4 (16-bit)."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_RHO, TOL_U = 1e-5, 2e-4
# the precision tests' bounds, except the bfloat16 capsule force: on the
# four-capsule film its relative error (against forces that are still small
# 60 steps in) measured 2.0e-3 and 3.3e-3 in two runs with different rounding
# streams; 3x the larger
BOUNDS16 = {1: dict(rho=2e-4, u=8e-3, F=3e-4, X=1.2e-4),
            2: dict(rho=1.2e-3, u=6e-2, F=1e-2, X=5e-4)}


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


def errors(sim, orc, ncaps):
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    e = dict(rho=rel(rg, ro), u=rel(ug, uo), F=0.0, X=0.0)
    for c in range(ncaps):
        sg, so = sim.capsule_state(c), orc.capsule_state(c)
        Fg, _ = sim.capsule_force(c)
        e["F"] = max(e["F"], np.abs(Fg - so["force"]).max() / np.abs(so["force"]).max())
        e["X"] = max(e["X"], np.abs(sg["X"] - so["X"]).max())
    return e


@pytest.mark.parametrize("mode", [I.MODE_FIXED, I.MODE_FREE])
def test_drying_tiny_film_matches_oracle(cfm, mode):
    wl = I.tiny_film(mode=mode, steps=60)
    wl.dry_dm = 0.25
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    m0 = orc.total_mass()
    sim.step(wl.steps); orc.step(wl.steps)
    rg, ug = sim.fields()
    ro, uo = orc.fields()
    assert rel(rg, ro) < TOL_RHO, rel(rg, ro)
    assert rel(ug, uo) < TOL_U, rel(ug, uo)
    assert rel(sim.populations().astype(np.float64), orc.populations()) < TOL_RHO
    mo = orc.total_mass()
    if mode == I.MODE_FIXED:  # resting walls conserve mass: the oracle's linear law holds
        assert abs(m0[0] - mo[0] - wl.steps * wl.dry_dm) < 1e-9
    mg = sim.total_mass()
    assert abs(mg[0] - mo[0]) < 1e-5 * mo[0] and abs(mg.sum() - mo.sum()) < 1e-5 * mo.sum()


def test_drying_ragged_lattice_many_blocks(cfm):
    """No capsule, 40 x 14 x 24 with a wall: 2 x 4 x 23 density blocks feed the
    reduction, the x rows end in a ragged tail."""
    wl = I.Workload("dry ragged", 40, 14, 24, h_top=9.5, capsules=[], steps=50, dry_dm=0.8)
    sim = cfm.Simulation.from_workload(wl)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    rg, _ = sim.fields()
    ro, _ = orc.fields()
    assert rel(rg, ro) < TOL_RHO
    assert abs(sim.total_mass()[0] - orc.total_mass()[0]) < 1e-5 * orc.total_mass()[0]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_A_inventory_falls_linearly(cfm, prec):
    wl = I.Workload("dry mass", 48, 20, 24, h_top=10.5, capsules=[], steps=1, dry_dm=1.5)
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    m0 = sim.total_mass()
    tol = 1e-5 if prec == 0 else 1e-4
    done = 0
    for n in (1, 9, 190):
        sim.step(n)
        done += n
        m = sim.total_mass()
        assert abs((m0[0] - m[0]) - done * wl.dry_dm) < tol * m0[0], (done, m0[0] - m[0])
        assert abs(m.sum() - m0.sum()) < tol * m0.sum()
    sim.remove_mass(0.0)
    sim.step(20)
    assert abs(sim.total_mass()[0] - m[0]) < tol * m0[0]


@pytest.mark.parametrize("prec", [0, 1])
def test_drying_runs_are_reproducible(cfm, prec):
    """The drying sum is reduced in a fixed order: two runs give the same bits
    (fixed capsule, so no atomic force sum feeds back into the populations)."""
    wl = I.tiny_film(mode=I.MODE_FIXED, steps=30)
    wl.dry_dm = 0.25
    a = cfm.Simulation.from_workload(wl, precision=prec)
    b = cfm.Simulation.from_workload(wl, precision=prec)
    a.step(30); b.step(30)
    assert (a.populations() == b.populations()).all()


def test_drying_is_rejected_in_a_batch(cfm):
    wls = [I.tiny_film(mode=I.MODE_FIXED), I.tiny_film(mode=I.MODE_FIXED)]
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    sims[1].remove_mass(0.1)
    b = cfm.Batch(sims)
    with pytest.raises(cfm.CapfilmError):
        b.step(4)
    b.close()
    with pytest.raises(cfm.CapfilmError):
        sims[0].remove_mass(-1.0)


DRY_STEPS = 60


@pytest.mark.slow
def test_drying_film_four_capsules_against_oracle(cfm):
    """Mixed-precision drying film at 128 x 128 x 48, four free R=10 capsules on
    the seeded layout, float32, half and bfloat16 storage stepped one step at a
    time beside the FP64 oracle: errors of densities, velocities, capsule
    forces, node positions and the A inventory every 10 steps.  A moving
    membrane vertex that passes within rounding distance of a lattice node
    flips cut-link decisions, after which the states differ locally by the
    inside/outside density contrast; a mode is judged on its last comparison
    before its first flip (at least 20 steps in), and its flips are reported."""
    wl = I.drying_film(nx=128, ny=128, nz=48, n_caps=4, steps=50000)
    orc = O.Oracle.from_workload(wl)
    sims = {p: cfm.Simulation.from_workload(wl, precision=p) for p in (0, 1, 2)}
    last = {p: None for p in sims}
    flip = {p: None for p in sims}
    for n in range(1, DRY_STEPS + 1):
        orc.step(1)
        mo = orc.cut_mask()
        for p, sim in sims.items():
            if flip[p] is not None:
                continue
            sim.step(1)
            if (sim.cut_mask() != mo).any():
                flip[p] = n
                continue
            if n % 10 == 0:
                e = errors(sim, orc, len(wl.capsules))
                mg, mo_ = sim.total_mass(), orc.total_mass()
                e["massA"] = abs(mg[0] - mo_[0]) / mo_[0]
                last[p] = (n, e)
    print("first flip step", flip)
    print("errors at the last comparison", last)
    for p, (n, e) in last.items():
        assert n >= 20, (p, n)
        if p == 0:
            assert e["rho"] < TOL_RHO and e["u"] < TOL_U and e["F"] < 1e-3 and e["massA"] < 1e-5, e
        else:
            for k in ("rho", "u", "F", "X"):
                assert e[k] < BOUNDS16[p][k], (p, k, e[k])
            assert e["massA"] < 1e-4


@pytest.mark.slow
def test_drying_film_float32_through_flips_with_cut_override(cfm):
    """The float32 drying film held to the parity tolerances through its cut
    flips: stepped one step at a time beside the oracle, and where the cut
    links the GPU computed on its float positions differ from the oracle's,
    every difference must be a near tie of the oracle's decision (within 1e-4
    lattice units) and the oracle then takes the GPU's cut structure."""
    wl = I.drying_film(nx=128, ny=128, nz=48, n_caps=4, steps=50000)
    orc = O.Oracle.from_workload(wl)
    sim = cfm.Simulation.from_workload(wl)
    adopted = 0
    for _ in range(DRY_STEPS):
        sim.step(1); orc.step(1)
        if (sim.cut_mask() != orc.cut_mask()).any():
            mg, tg, _ = sim.cuts()
            n = orc.override_cuts(mg, tg, 1e-4)
            assert n >= 0, f"{-n} cut-link differences are not near ties"
            adopted += n
    e = errors(sim, orc, len(wl.capsules))
    mg, mo = sim.total_mass(), orc.total_mass()
    e["massA"] = abs(mg[0] - mo[0]) / mo[0]
    print(f"drying film float32 with cut override after {DRY_STEPS} steps: {e}, {adopted} link ends adopted")
    assert e["rho"] < TOL_RHO and e["u"] < 1e-4 and e["F"] < 1e-3 and e["X"] < 1e-5 and e["massA"] < 1e-5, e
