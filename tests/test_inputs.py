"""The seeded input generators (no arithmetic of the method): reproducible
draws, the layouts and ranges their docstrings promise.  CPU only."""
import math

import numpy as np

from paper_2007_15405_gb300 import inputs as I


def test_icosphere_counts_radius_and_orientation():
    for level, nv, nf in [(0, 12, 20), (2, 162, 320), (3, 642, 1280), (4, 2562, 5120)]:
        X, F = I.icosphere(level, 5.0, (1.0, 2.0, 3.0))
        assert X.shape == (nv, 3) and F.shape == (nf, 3)
        assert np.allclose(np.linalg.norm(X - [1.0, 2.0, 3.0], axis=1), 5.0)
        # outward orientation: (B - A) x (C - A) points away from the centre
        A, B, C = X[F[:, 0]], X[F[:, 1]], X[F[:, 2]]
        n = np.cross(B - A, C - A)
        assert (np.einsum("ij,ij->i", n, (A + B + C) / 3 - [1.0, 2.0, 3.0]) > 0).all()


def test_jitter_is_seeded_and_bounded():
    a = I.jitter((4, 5, 6), 1e-3, seed=3)
    b = I.jitter((4, 5, 6), 1e-3, seed=3)
    c = I.jitter((4, 5, 6), 1e-3, seed=4)
    assert a.shape == (2, 4, 5, 6) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.abs(a).max() <= 1e-3


def test_drying_film_layout():
    wl = I.drying_film()
    assert (wl.nx, wl.ny, wl.nz) == (256, 256, 96) and len(wl.capsules) == 16
    R = 10.0
    lo = R + I.DELTA0 + 1.0
    c = np.array([cap.centre for cap in wl.capsules])
    assert (c[:, 0] >= lo).all() and (c[:, 0] <= wl.nx - lo + 1).all()
    assert (c[:, 1] >= lo).all() and (c[:, 1] <= wl.ny - lo + 1).all()
    d = np.linalg.norm(c[:, None, :2] - c[None, :, :2], axis=-1) + np.eye(len(c)) * 1e9
    assert d.min() >= 2 * R + 2 * I.DELTA0 - 1e-9
    assert np.allclose(c[:, 2], I.z_rest(R) + 0.17)
    # the film falls from 0.6R to 0.2R over 50k steps: A excess of the lowered layer
    assert math.isclose(wl.dry_dm * 50000, 0.4 * R * 256 * 256 * (I.RHO_MAJ - I.RHO_MIN))
    assert math.isclose(wl.h_top, 0.5 + I.REP_DZ + 0.6 * R)
    again = I.drying_film()
    assert [cap.centre for cap in again.capsules] == [cap.centre for cap in wl.capsules]


def test_batched_sweep_sizes_and_moduli():
    wls = I.batched_sweep()
    assert len(wls) == 64
    nodes = [w.nodes for w in wls]
    assert min(nodes) == 64 * 48 * 48 and max(nodes) == 160 * 80 * 64
    rigid = [w for w in wls if w.capsules[0].mode == I.MODE_FROZEN]
    assert len(rigid) == 16
    for w in wls:
        a, b = w.capsules
        d = abs(b.centre[0] - a.centre[0]) / a.radius
        assert 2.2 - 1e-9 <= d <= 6.0 + 1e-9
        assert b.centre[0] + b.radius < w.nx and a.centre[0] - a.radius > 0
        assert a.radius == 10.0 and a.level == 4
        assert math.isclose(w.h_top, 0.5 + I.REP_DZ + 0.4 * a.radius)
    assert sum(nodes) == 26148864


def test_warm_dataset_ranges():
    wls = I.warm_dataset(40, seed=5)
    for w in wls:
        cap = w.capsules[0]
        assert 5.0 <= cap.radius <= 7.0 and 3e-3 <= cap.kS <= 1e-1 + 1e-12
        h = (w.h_top - 0.5 - I.REP_DZ) / cap.radius
        assert 0.3 <= h <= 0.9
        assert cap.radius + 4 <= cap.centre[0] - 0.3 <= w.nx - cap.radius - 4
    assert [w.capsules[0].centre for w in I.warm_dataset(40, seed=5)] == [w.capsules[0].centre for w in wls]


def test_many_capsules_layout():
    """The many-particle film: seeded random sequential addition with every
    periodic centre distance at least 2R + 2 delta0 + 1, bottoms where the
    substrate repulsion starts, bending modulus from beta = R^2 gamma / kB."""
    wl = I.many_capsules(100, 320, 320)
    again = I.many_capsules(100, 320, 320)
    other = I.many_capsules(100, 320, 320, seed=13)
    c = np.array([cap.centre for cap in wl.capsules])
    assert len(wl.capsules) == 100
    assert np.array_equal(c, np.array([cap.centre for cap in again.capsules]))
    assert not np.array_equal(c, np.array([cap.centre for cap in other.capsules]))
    R = wl.capsules[0].radius
    d = c[:, None, :2] - c[None, :, :2]
    d -= np.round(d / 320.0) * 320.0
    r = np.hypot(d[..., 0], d[..., 1]) + np.eye(len(c)) * 1e9
    assert r.min() >= 2 * R + 2 * I.DELTA0 + 1.0
    assert np.allclose(c[:, 2], I.z_rest(R) + c[0, 2] - I.z_rest(R))
    assert abs(c[0, 2] - R - I.DELTA0 - (0.5 + I.REP_DZ)) < 1.0  # bottom at the repulsion's reach
    assert all(abs(R * R * I.GAMMA_G36 / cap.kB - 25.0) < 1e-9 for cap in wl.capsules)
    assert abs(100 * np.pi * R * R / (320 * 320) - 0.307) < 1e-3


def test_pair_and_single_particle_workloads():
    """The two-particle and single-particle set-ups: centre distances, film
    heights above the repulsive plane, boxes and moduli as their recipes state."""
    rest = 0.5 + I.REP_DZ
    pair = I.capsule_pair()
    (a, b) = [np.array(c.centre) for c in pair.capsules]
    assert (pair.nx, pair.ny, pair.nz) == (128, 64, 64)
    assert abs(np.linalg.norm(b - a) - 3 * 12.0) < 1e-12 and a[2] == b[2]
    assert abs(pair.h_top - (rest + 0.6 * 12.0)) < 1e-12
    for gap in (3.0, 5.0, 7.0):
        rp = I.rigid_pair(gap)
        (a, b) = [np.array(c.centre) for c in rp.capsules]
        L = gap * 10.0 + 20.0
        assert abs(b[0] - a[0] - L) < 1e-12
        assert rp.nx % 8 == 0 and rp.nx >= 2 * L + 64
        assert all(c.mode == I.MODE_FIXED for c in rp.capsules)
        assert abs(rp.h_top - (rest + 0.16 * 10.0)) < 1e-12
    one = I.rigid_particle(0.4)
    assert len(one.capsules) == 1 and one.capsules[0].mode == I.MODE_FIXED
    assert abs(one.h_top - (rest + 4.0)) < 1e-12
    for beta in (10.0, 25.0, 50.0):
        ap = I.approach_pair(beta)
        (a, b) = [np.array(c.centre) for c in ap.capsules]
        assert abs(b[0] - a[0] - 40.0) < 1e-12  # surface gap 2R
        for c in ap.capsules:
            assert c.C == 9.0 and abs(100.0 * I.GAMMA_G36 / c.kB - beta) < 1e-9
