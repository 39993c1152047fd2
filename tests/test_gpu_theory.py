"""Physics checks of the coupled method against the theory of Sec. 2 (not
parity; the oracle pins the formulas themselves in test_oracle_theory.py).

- Film-height series (Sec. 4.1, capillary charge against film thickness):
  for a fixed rigid particle the fitted charge Q and the rise Z fall
  monotonically as the film rises towards the particle's centre.
- Rigid-pair lateral force (Sec. 4.1, force validation at h0 = 0.16R): two
  fixed particles at surface gaps 3, 4 and 5 R, meniscus run to stationarity,
  force within 15% of Eq. 13 with q and Q fitted on the single particle at
  the same film height and gamma from the oracle's Laplace test
  (tests/golden/gamma_G3.6.txt).  Measured: 0.998, 1.033, 1.101.
"""
import os

import numpy as np
import pytest

from paper_2007_15405_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
HERE = os.path.dirname(os.path.abspath(__file__))


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


def gamma():
    lines = open(os.path.join(HERE, "golden", "gamma_G3.6.txt")).read().split("\n")
    return float([l for l in lines if l and not l.startswith("#")][0])


def fit_single(cfm, sim, R, box):
    r, z, Z = sim.meniscus_profile(0, 1.0)
    Q, q, rms, m = cfm.meniscus_fit(r, z, rmin=R + 4.0, rmax=0.5 * box - 4.0)
    return Q, q, Z


def test_charge_and_rise_fall_with_film_height(cfm):
    R, box = 10.0, 128
    hs = (0.2, 0.5, 0.8)
    sims = [cfm.Simulation.from_workload(I.rigid_particle(h, R, nx=box, ny=box)) for h in hs]
    b = cfm.Batch(sims)
    b.step(40000)
    res = [fit_single(cfm, s, R, box) for s in sims]
    b.close()
    Q = [r[0] for r in res]
    Z = [r[2] for r in res]
    assert Q[0] > Q[1] > Q[2] > 0 and Z[0] > Z[1] > Z[2] > 0, (Q, Z)
    q = [r[1] for r in res]
    assert all(0.01 < v < 0.1 for v in q)


def test_rigid_pair_force_follows_eq13(cfm):
    R, box = 10.0, 160
    gaps = (3.0, 4.0, 5.0)
    single = cfm.Simulation.from_workload(I.rigid_particle(0.16, R, nx=box, ny=box))
    pairs = [cfm.Simulation.from_workload(I.rigid_pair(g, 0.16, R, ny=box)) for g in gaps]
    b = cfm.Batch([single] + pairs)
    hist = []
    for _ in range(12):
        b.step(10000)
        hist.append([s.lateral_force(0, 1) for s in pairs])
    Q, q, _ = fit_single(cfm, single, R, box)
    b.close()
    hist = np.array(hist)
    for k, g in enumerate(gaps):
        f = hist[-3:, k].mean()
        assert abs(hist[-1, k] - hist[-2, k]) < 0.01 * abs(f)  # stationary
        ft = cfm.capillary_force(q, gamma(), Q, Q, g * R + 2 * R)
        assert f < 0 and ft < 0
        assert abs(f / ft - 1.0) < 0.15, (g, f, ft)
