"""16-bit population storage (offsets from the rest equilibrium, stochastic
rounding, float32 arithmetic) against the FP64 oracle, with the error of every
reported quantity bounded.  The bounds are about 3x the largest errors measured
on GB300 over these workloads (40-step tiny film, 1000-step single capsule,
60-step capsule pair): half (11-bit significand, offsets scaled by 2^15)
resolves an offset to ~5e-4 of its size, bfloat16 (8-bit) to ~4e-3."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (rho, u, capsule force, node positions) relative / absolute bounds per mode
# measured maxima: half rho 5.6e-5, u 2.7e-3, F 7.8e-5, X 3.6e-5;
#                  bfloat16 rho 3.8e-4, u 2.0e-2, F 5.6e-4, X 1.5e-4
BOUNDS = {1: dict(rho=2e-4, u=8e-3, F=3e-4, X=1.2e-4),    # half offsets
          2: dict(rho=1.2e-3, u=6e-2, F=2e-3, X=5e-4)}     # bfloat16 offsets


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
    return np.abs(a - b).max() / np.abs(b).max()


def errors(sim, orc):
    rg, ug = sim.fields(); ro, uo = orc.fields()
    sg, so = sim.capsule_state(0), orc.capsule_state(0)
    Fg, _ = sim.capsule_force(0)
    return dict(rho=rel(rg, ro), u=rel(ug, uo),
                F=np.abs(Fg - so["force"]).max() / np.abs(so["force"]).max(),
                X=np.abs(sg["X"] - so["X"]).max())


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("mode", [I.MODE_FIXED, I.MODE_FREE])
def test_tiny_film_16bit(cfm, prec, mode):
    wl = I.tiny_film(mode=mode, steps=40)
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    e = errors(sim, orc)
    print(prec, mode, e)
    for k, v in e.items():
        assert v < BOUNDS[prec][k], (k, v)


@pytest.mark.parametrize("prec", [1, 2])
def test_tiny_film_16bit_other_tau(cfm, prec):
    """The general collision (tau != 1) with 16-bit storage."""
    wl = I.tiny_film(mode=I.MODE_FREE, steps=40)
    wl.tau = (0.8, 0.8)
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    e = errors(sim, orc)
    print(prec, e)
    for k, v in e.items():
        assert v < BOUNDS[prec][k], (k, v)


@pytest.mark.parametrize("prec", [1, 2])
def test_mass_16bit_no_capsule(cfm, prec):
    """The float rest population takes each node's mass balance after the
    offsets are rounded, so 16-bit storage changes the mass of a component
    only by float32 rounding, also at a Shan-Chen interface."""
    wl = I.Workload("rest16", 40, 12, 10, h_top=4.5, capsules=[], steps=200)
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    m0 = sim.total_mass()
    sim.step(200)
    assert np.allclose(sim.total_mass(), m0, rtol=1e-5)


def test_populations_decode_roundtrip(cfm):
    """The decoded 16-bit populations of the initial film equal the float32 ones
    to the offset resolution (rest state: offsets are exactly zero)."""
    wl = I.tiny_film(mode=I.MODE_FIXED)
    a = cfm.Simulation.from_workload(wl, precision=0).populations()
    for prec in (1, 2):
        b = cfm.Simulation.from_workload(wl, precision=prec).populations()
        assert np.abs(a - b).max() < 1e-6


def test_16bit_runs_are_deterministic(cfm):
    """The stochastic rounding is a hash of node, step and direction: two runs
    give the same bits (fixed capsule, so no atomic force sum feeds back into
    the populations)."""
    wl = I.tiny_film(mode=I.MODE_FIXED, steps=20)
    for prec in (1, 2):
        a = cfm.Simulation.from_workload(wl, precision=prec)
        b = cfm.Simulation.from_workload(wl, precision=prec)
        a.step(20); b.step(20)
        assert (a.populations() == b.populations()).all()


@pytest.mark.slow
@pytest.mark.parametrize("prec", [1, 2])
def test_single_capsule_film_1000_steps_16bit(cfm, prec):
    wl = I.single_capsule_film(mode=I.MODE_FIXED, steps=1000)
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    orc = O.Oracle.from_workload(wl)
    sim.step(wl.steps); orc.step(wl.steps)
    e = errors(sim, orc)
    print(prec, e)
    for k, v in e.items():
        assert v < BOUNDS[prec][k], (k, v)
