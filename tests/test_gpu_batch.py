"""Batched stepping (cf_batch) against stepping the same lattices one by one,
and against the FP64 oracle.

A lattice stepped in a batch runs the same per-node arithmetic as alone, so
its populations agree with the lone run to float32 rounding (a different
inlining may fuse a multiply-add differently); membrane-free and fixed-capsule
lattices are compared at 1e-6, free capsules through the oracle tolerances.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-6     # batch vs lone run, relative
TOL_RHO = 1e-5      # vs the FP64 oracle (as in the single-lattice parity tests)
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


def mixed_workloads(mode=I.MODE_FIXED):
    """Lattices of different shapes: one capsule, none, two capsules."""
    two = [I.CapsuleSpec(centre=(10.3, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=mode),
           I.CapsuleSpec(centre=(21.3, 8.4, 10.17), radius=4.0, level=2, C=1.0, mode=mode)]
    return [I.tiny_film(mode=mode),
            I.Workload("film", 20, 16, 12, h_top=5.5, capsules=[], steps=1, seed=7),
            I.Workload("pair", 33, 17, 21, h_top=8.5, capsules=two, steps=1, rep_dz=2.0, seed=3)]


def run_batch(cfm, wls, steps, precision=0, config=None):
    sims = [cfm.Simulation.from_workload(w, precision=precision) for w in wls]
    b = cfm.Batch(sims)
    if config is not None:
        b.set_config(*config)
    b.step(steps)
    return b, sims


def run_alone(cfm, wls, steps, precision=0):
    out = []
    for w in wls:
        s = cfm.Simulation.from_workload(w, precision=precision)
        s.step(steps)
        out.append(s)
    return out


@pytest.mark.parametrize("config", [None, (0, 1), (3, 4), (5, 2)])
def test_batch_matches_lone_runs(cfm, config):
    """Fixed capsules and a capsule-free lattice, several launch shapes: the
    populations and cut links of every lattice equal its lone run."""
    wls = mixed_workloads()
    b, sims = run_batch(cfm, wls, 25, config=config)
    alone = run_alone(cfm, wls, 25)
    for s, a in zip(sims, alone):
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < TOL_SAME
        ms, ts, _ = s.cuts(); ma, ta, _ = a.cuts()
        assert (ms == ma).all() and (ts == ta).all()
        rs, us = s.fields(); ra, ua = a.fields()
        assert rel(rs, ra) < TOL_SAME
    b.close()


@pytest.mark.parametrize("groups", [2, 3])
def test_batch_groups_match_lone_runs(cfm, groups):
    """Pipeline groups (each group's lattice passes on a stream branch of its
    own): every lattice still equals its lone run, over an odd step count
    (graph replays and plain steps)."""
    wls = mixed_workloads()
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    b.set_groups(groups)
    assert b.config()["groups"] == groups
    b.step(25)
    alone = run_alone(cfm, wls, 25)
    for s, a in zip(sims, alone):
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < TOL_SAME
        rs, _ = s.fields(); ra, _ = a.fields()
        assert rel(rs, ra) < TOL_SAME
    b.close()


@pytest.mark.parametrize("config", [None, (4, 1)])
def test_batch_with_other_tau_matches_lone_runs(cfm, config):
    """One lattice with tau != 1: the batch takes the general collision for
    all of them, and every lattice still follows its lone run."""
    wls = mixed_workloads()
    wls[1].tau = (0.8, 0.9)
    b, sims = run_batch(cfm, wls, 25, config=config)
    alone = run_alone(cfm, wls, 25)
    for s, a, w in zip(sims, alone, wls):
        tol = TOL_SAME if w.tau != (1.0, 1.0) else 1e-5  # tau = 1 lattices: other summation order
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < tol
        rs, _ = s.fields(); ra, _ = a.fields()
        assert rel(rs, ra) < tol
    b.close()


def test_batch_free_capsules_vs_oracle(cfm):
    """Free capsules in a batch: every lattice against the FP64 oracle."""
    wls = mixed_workloads(mode=I.MODE_FREE)
    b, sims = run_batch(cfm, wls, 30)
    for s, w in zip(sims, wls):
        orc = O.Oracle.from_workload(w)
        orc.step(30)
        rg, ug = s.fields(); ro, uo = orc.fields()
        assert rel(rg, ro) < TOL_RHO and rel(ug, uo) < TOL_U, (w.name, rel(rg, ro), rel(ug, uo))
        for k in range(len(w.capsules)):
            assert np.abs(s.capsule_state(k)["X"] - orc.capsule_state(k)["X"]).max() < 1e-5
    b.close()


def test_batch_mixed_modes_and_many_lattices(cfm):
    """70 small lattices (more than one launch table of 64 lattices), with
    free, frozen and fixed capsules and capsule-free films mixed: the
    membrane and cut-link kernels of all lattices run batched, and every
    lattice follows its lone run (populations, cut links, node positions)."""
    modes = (I.MODE_FREE, I.MODE_FROZEN, I.MODE_FIXED)
    wls = []
    for i in range(70):
        if i % 7 == 3:
            wls.append(I.Workload("film", 14 + i % 3, 12, 12, h_top=5.5, capsules=[], steps=1, seed=i))
        else:
            wls.append(I.tiny_film(nx=16 + 2 * (i % 3), mode=modes[i % 3], seed=100 + i))
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    b.step(9)
    alone = run_alone(cfm, wls, 9)
    for s, a, w in zip(sims, alone, wls):
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < 1e-5, w.name
        ms, ts, _ = s.cuts(); ma, ta, _ = a.cuts()
        assert (ms == ma).all() and (ts == ta).all(), w.name
        if w.capsules:
            assert np.abs(s.capsule_state(0)["X"] - a.capsule_state(0)["X"]).max() < 1e-5
            Fs, _ = s.capsule_force(0); Fa, _ = a.capsule_force(0)
            assert np.abs(Fs - Fa).max() <= 1e-4 * np.abs(Fa).max() + 1e-8
    b.close()


def test_batch_then_alone_then_batch(cfm):
    """Contexts stay consistent when batch steps and lone steps alternate
    (odd step counts change every double-buffer parity)."""
    wls = mixed_workloads()
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    b.step(7)
    sims[1].step(3)
    b.step(5)
    ref = run_alone(cfm, wls, 12)
    ref[1].step(3)
    for s, a in zip(sims, ref):
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < TOL_SAME
    b.close()


def test_batch_autotune(cfm):
    """The autotuner returns one of the compiled shapes; the trial steps are
    real steps of every lattice."""
    wls = mixed_workloads()
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    cfg = b.autotune(steps=2)
    assert 0 <= cfg["tile"] < 6 and cfg["zchunk"] in (2, 4, 8) and cfg["ms_per_step"] > 0
    assert cfg["tile_x"] in (32, 64, 128) and cfg["tile_y"] in (2, 4, 8)
    assert cfg["groups"] in (1, 2)
    # 18 launch shapes with one group, then 2 groups (4 and 8 exceed the 3 lattices)
    done = (18 + 1) * (2 + 2)
    ref = run_alone(cfm, wls, done)
    for s, a in zip(sims, ref):
        assert rel(s.populations().astype(np.float64), a.populations().astype(np.float64)) < TOL_SAME
    b.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_16bit(cfm, prec):
    """16-bit storage in a batch follows its lone run (same stochastic
    rounding stream: node index and the lattice's own step counter)."""
    wls = mixed_workloads()
    b, sims = run_batch(cfm, wls, 20, precision=prec)
    alone = run_alone(cfm, wls, 20, precision=prec)
    for s, a in zip(sims, alone):
        rs, _ = s.fields(); ra, _ = a.fields()
        assert rel(rs, ra) < 1e-4
    b.close()


def test_batch_rejects_bad_input(cfm):
    wls = mixed_workloads()
    s0 = cfm.Simulation.from_workload(wls[0])
    s1 = cfm.Simulation.from_workload(wls[1], precision=1)
    with pytest.raises(cfm.CapfilmError, match="same precision"):
        cfm.Batch([s0, s1])
    with pytest.raises(cfm.CapfilmError, match="twice"):
        cfm.Batch([s0, s0])
    s2 = cfm.Simulation.from_workload(wls[1], set_film=False)
    with pytest.raises(cfm.CapfilmError, match="cf_set_film"):
        cfm.Batch([s0, s2])


@pytest.mark.slow
def test_sweep_of_64_lattices_sampled(cfm):
    """The full distance x softness sweep (64 lattices, 147k-819k nodes) in one
    batch, 10 steps: sampled lattices against their lone runs (free capsules:
    atomics sum the membrane forces in another order, so the comparison is at
    the free-run tolerances of the parity tests)."""
    wls = I.batched_sweep()
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    b = cfm.Batch(sims)
    b.set_config(1, 2)
    b.step(10)
    for i in (0, 21, 42, 63):
        a = cfm.Simulation.from_workload(wls[i])
        a.step(10)
        rs, us = sims[i].fields(); ra, ua = a.fields()
        assert rel(rs, ra) < 1e-5 and rel(us, ua) < 1e-3, (i, rel(rs, ra), rel(us, ua))
        fs = sims[i].lateral_force(0, 1); fa = a.lateral_force(0, 1)
        assert abs(fs - fa) <= 1e-3 * abs(fa) + 1e-9
        a.close()
    b.close()
