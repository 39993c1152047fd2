"""Runtime around the coupled step: checkpoint and restart, failure detection
(errors raised on the host: a non-finite initial state, an allocator that
fails), the meniscus-height and batch readouts, and the JSON-lines run log."""
import ctypes as C
import json

import numpy as np
import pytest

from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def state(sim):
    rho, u = sim.fields()
    out = dict(f=sim.populations(), rho=rho, u=u, mass=sim.total_mass())
    for c in range(len(sim.nv)):
        out[f"X{c}"] = sim.capsule_state(c)["X"]
        out[f"F{c}"] = sim.capsule_force(c)[0]
    return out


@pytest.mark.parametrize("prec,mode", [(0, I.MODE_FIXED), (1, I.MODE_FIXED), (2, None), (0, None)])
def test_restart_is_bit_identical(cfm, tmp_path, prec, mode):
    """Save after 33 steps (an odd count: the other buffer parity), run 24 more;
    a fresh context loading the file and running 24 steps ends in the same
    bits (fixed capsules or none: no atomic float sum feeds back).  The
    capsule force readout itself is an atomic float sum: equal to rounding."""
    if mode is None:
        wl = I.Workload("film", 40, 14, 24, h_top=9.5, capsules=[], steps=1, dry_dm=0.3)
    else:
        wl = I.tiny_film(mode=mode)
    a = cfm.Simulation.from_workload(wl, precision=prec)
    a.step(33)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(24)
    b = cfm.Simulation.from_workload(wl, precision=prec, set_film=False)
    b.load(path)
    b.step(24)
    sa, sb = state(a), state(b)
    for k in sa:
        if k.startswith("F"):
            assert np.abs(sa[k] - sb[k]).max() <= 1e-5 * np.abs(sa[k]).max(), k
        else:
            assert np.array_equal(sa[k], sb[k]), k


def test_restart_free_capsule_continues(cfm, tmp_path):
    """Free capsule: the restarted run repeats the original bit for bit (the
    momentum exchanged with each element is summed in fixed point, so no sum
    depends on the order its atomic contributions arrive in)."""
    wl = I.tiny_film(mode=I.MODE_FREE)
    a = cfm.Simulation.from_workload(wl)
    a.step(20)
    path = str(tmp_path / "free.bin")
    a.save(path)
    a.step(20)
    b = cfm.Simulation.from_workload(wl, set_film=False)
    b.load(path)
    b.step(20)
    sa, sb = state(a), state(b)
    for k in ("f", "rho", "X0"):
        assert np.array_equal(sa[k], sb[k]), k
    ma, mb = a.cuts()[0], b.cuts()[0]
    assert (ma == mb).all()


def test_free_runs_repeat_bit_for_bit(cfm):
    """Two runs of the same free two-capsule set-up (contact, moving cut
    links, momentum exchange) end in identical states."""
    caps = [I.CapsuleSpec(centre=(10.3, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE),
            I.CapsuleSpec(centre=(19.1, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FREE)]
    wl = I.Workload("contact", 32, 16, 20, h_top=8.5, capsules=caps, steps=60, rep_dz=2.0)
    runs = []
    for _ in range(2):
        s = cfm.Simulation.from_workload(wl)
        s.step(wl.steps)
        runs.append((s.populations(), s.capsule_state(0)["X"], s.capsule_state(1)["X"], s.capsule_force(0)[0]))
    for x, y in zip(*runs):
        assert np.array_equal(x, y)


def test_load_rejects_what_does_not_match(cfm, tmp_path):
    wl = I.tiny_film(mode=I.MODE_FIXED)
    a = cfm.Simulation.from_workload(wl)
    a.step(3)
    path = tmp_path / "ck.bin"
    a.save(str(path))
    other = cfm.Simulation.from_workload(I.tiny_film(nx=18, mode=I.MODE_FIXED))
    with pytest.raises(cfm.CapfilmError, match="does not match"):
        other.load(str(path))
    half = cfm.Simulation.from_workload(wl, precision=1)
    with pytest.raises(cfm.CapfilmError, match="does not match"):
        half.load(str(path))
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a checkpoint at all" * 4)
    with pytest.raises(cfm.CapfilmError, match="version"):
        a.load(str(junk))
    cut = tmp_path / "cut.bin"
    cut.write_bytes(path.read_bytes()[:200])
    b = cfm.Simulation.from_workload(wl)
    with pytest.raises(cfm.CapfilmError, match="truncated"):
        b.load(str(cut))
    with pytest.raises(cfm.CapfilmError, match="cf_set_film"):
        b.step(1)  # a partly loaded context must be set up again
    with pytest.raises(cfm.CapfilmError, match="cannot open"):
        a.load(str(tmp_path / "missing.bin"))


def test_non_finite_initial_state_is_reported(cfm):
    """A NaN planted in the host-prepared initial densities: the step's
    device-side check sets the status and the next synchronising call
    returns CF_EDIVERGED."""
    wl = I.tiny_film(mode=I.MODE_FIXED)
    sim = cfm.Simulation.from_workload(wl, set_film=False)
    rA = np.full((wl.nz, wl.ny, wl.nx), I.RHO_MAJ)
    rB = np.full((wl.nz, wl.ny, wl.nx), I.RHO_MIN)
    rA[7, 5, 3] = np.nan
    sim.set_densities(rA, rB)
    sim.step(3)
    with pytest.raises(cfm.CapfilmError, match="non-finite"):
        sim.sync()


def test_failing_allocator_reports_enomem_and_frees(cfm):
    """An allocator callback that fails on its fifth request: cf_create
    returns CF_ENOMEM and gives back every block it had obtained."""
    import torch
    L = cfm._lib
    live = {}
    calls = [0]

    def alloc(size, stream, user):
        calls[0] += 1
        if calls[0] >= 5:
            return None
        p = torch.cuda.caching_allocator_alloc(size)
        live[p] = size
        return p

    def free(ptr, stream, user):
        live.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a_fn, f_fn = cfm.ALLOC_FN(alloc), cfm.FREE_FN(free)
    al = cfm.Allocator(a_fn, f_fn, None)
    desc = cfm.LatticeDesc(16, 12, 20, 1, (C.c_double * 2)(1.0, 1.0), 3.6, 2.0, 1.5, 1.5, 0,
                           C.pointer(al), None, 0)
    h = C.c_void_p()
    rc = L.cf_create(C.byref(desc), C.byref(h))
    assert cfm.STATUS_NAMES[rc] == "CF_ENOMEM"
    torch.cuda.synchronize()
    assert calls[0] >= 5 and not live


def test_meniscus_height_is_the_profile_maximum(cfm):
    wl = I.tiny_film(mode=I.MODE_FIXED)
    sim = cfm.Simulation.from_workload(wl)
    sim.step(20)
    r, zeta, Z = sim.meniscus_profile(0)
    h = sim.meniscus_height(0)
    assert h == Z or (np.isnan(h) and np.isnan(Z))


def test_batch_lateral_forces_match_each_context(cfm):
    two = [I.CapsuleSpec(centre=(10.3, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FIXED),
           I.CapsuleSpec(centre=(21.3, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=I.MODE_FIXED)]
    wls = [I.Workload(f"pair {i}", 33 + 2 * i, 17, 21, h_top=8.5, capsules=two, steps=1, rep_dz=2.0, seed=3 + i)
           for i in range(3)]
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    b.step(10)
    F = b.lateral_forces(0, 1)
    assert np.array_equal(F, [s.lateral_force(0, 1) for s in sims])
    b.close()


def test_run_writes_one_json_line_per_readout(cfm, tmp_path):
    wl = I.tiny_film(mode=I.MODE_FIXED)
    sim = cfm.Simulation.from_workload(wl)
    log = tmp_path / "run.jsonl"
    recs = sim.run(25, 10, log=str(log))
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [r["step"] for r in lines] == [10, 20, 25] and lines == json.loads(json.dumps(recs))
    assert set(lines[0]) == {"step", "mlups", "mass", "force", "Z"}
    assert len(lines[-1]["force"]) == 1 and lines[-1]["mlups"] > 0


def test_add_capsules_at_once_equals_one_by_one(cfm):
    """cf_add_capsules builds the membrane once for many capsules; the state
    equals the one built capsule by capsule, and a bad descriptor adds none."""
    from paper_2007_15405_gb300.inputs import RHO_MAJ, RHO_MIN, RHO_MIX
    wl = I.many_capsules(n_caps=20, nx=120, ny=120, nz=40, radius=6.0, level=2, seed=3)
    specs = [(*c.mesh(), c.kS, c.C, c.kB, c.kV, c.mass, c.mode, 0.0) for c in wl.capsules]
    a = cfm.Simulation(wl.nx, wl.ny, wl.nz, wall=wl.wall, tau=wl.tau, G=wl.G, rep_dz=wl.rep_dz)
    assert a.add_capsules(specs) == list(range(20))
    b = cfm.Simulation(wl.nx, wl.ny, wl.nz, wall=wl.wall, tau=wl.tau, G=wl.G, rep_dz=wl.rep_dz)
    for sp in specs:
        b.add_capsule(*sp[:8], wet=sp[8])
    for s in (a, b):
        s.set_film(wl.h_top, RHO_MAJ, RHO_MIN, RHO_MIX, wl.jitter())
        s.step(12)
    assert np.array_equal(a.populations(), b.populations())
    for k in (0, 7, 19):
        assert np.array_equal(a.capsule_state(k)["X"], b.capsule_state(k)["X"])
    c = cfm.Simulation(wl.nx, wl.ny, wl.nz, wall=wl.wall, tau=wl.tau, G=wl.G, rep_dz=wl.rep_dz)
    bad = list(specs[:3])
    bad[1] = (*specs[1][:6], -1.0, *specs[1][7:])  # node mass must be positive
    with pytest.raises(cfm.CapfilmError, match="mass"):
        c.add_capsules(bad)
    assert c.add_capsules(specs[:2]) == [0, 1]
