"""Pins of the oracle's theory functions (Sec. 2): the Bessel functions K_0,
K_1 (from their integral representation) against scipy's library routines,
the least-squares fit of the meniscus model zeta = Q K_0(q r) (Eq. 12) on
profiles generated from the model, and the lateral capillary force
F = -2 pi q gamma Q1 Q2 K_1(q L) (Eq. 13) with its Coulomb limit.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("scipy.special")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("x", [1e-3, 0.05, 0.5, 1.0, 3.7, 12.0, 60.0])
def test_bessel_k_matches_library(x):
    assert O.bessel_k(0, x) == pytest.approx(sp.k0(x), rel=1e-13)
    assert O.bessel_k(1, x) == pytest.approx(sp.k1(x), rel=1e-13)
    assert O.bessel_k(2, x) == pytest.approx(sp.kv(2, x), rel=1e-13)


def test_bessel_k_recurrence_and_limits():
    """K_2(x) = K_0(x) + 2 K_1(x) / x; K_0(x) ~ -ln(x/2) - 0.5772... for small
    x; K_1(x) ~ 1/x."""
    for x in (0.3, 2.0, 9.0):
        assert O.bessel_k(2, x) == pytest.approx(O.bessel_k(0, x) + 2 * O.bessel_k(1, x) / x, rel=1e-13)
    x = 1e-6
    assert O.bessel_k(0, x) == pytest.approx(-math.log(x / 2) - 0.5772156649015329, rel=1e-9)
    assert O.bessel_k(1, x) * x == pytest.approx(1.0, rel=1e-9)


@pytest.mark.parametrize("Q,q", [(0.7, 0.13), (-0.35, 0.05), (2.5, 0.4)])
def test_meniscus_fit_recovers_model_parameters(Q, q):
    """Profiles made from the model itself (sampled every 0.5 from r = 5 to
    40, with NaN samples and samples outside the window mixed in) return
    their Q and q to 1e-10 and a zero residual."""
    r = np.arange(0.0, 45.0, 0.5)
    z = np.where(r > 0, Q * sp.k0(q * np.maximum(r, 1e-9)), np.nan)
    z[7] = np.nan
    z[r > 40] = 123.0           # outside the window: must be ignored
    z[r < 5] = -7.0
    Qf, qf, rms, m = O.meniscus_fit(r, z, rmin=5.0, rmax=40.0)
    assert m == int((40 - 5) / 0.5) + 1 - (1 if 5.0 <= r[7] <= 40.0 else 0)
    assert Qf == pytest.approx(Q, rel=1e-10) and qf == pytest.approx(q, rel=1e-10)
    assert rms < 1e-12 * abs(Q)


def test_meniscus_fit_is_least_squares():
    """With noise the fit is the least-squares minimum: nudging q or Q either
    way raises the residual."""
    rng = np.random.default_rng(4)
    r = np.arange(6.0, 40.0, 1.0)
    z = 0.8 * sp.k0(0.11 * r) + rng.normal(0, 2e-3, r.size)
    Qf, qf, rms, m = O.meniscus_fit(r, z)

    def S(Q, q):
        return np.sum((z - Q * sp.k0(q * r)) ** 2)

    s0 = S(Qf, qf)
    assert rms == pytest.approx(math.sqrt(s0 / m), rel=1e-9)
    for dQ, dq in ((1e-4, 0), (-1e-4, 0), (0, 1e-5), (0, -1e-5)):
        assert S(Qf + dQ, qf + dq) > s0


def test_capillary_force_formula_and_limits():
    """F = -2 pi q gamma Q1 Q2 K_1(q L): attraction (F < 0) for charges of the
    same sign, symmetric in Q1 and Q2, and the Coulomb form -2 pi gamma Q1 Q2
    / L when q L << 1."""
    q, g, Q1, Q2, L = 0.12, 0.0488, 1.3, 0.9, 35.0
    F = O.capillary_force(q, g, Q1, Q2, L)
    assert F == pytest.approx(-2 * math.pi * q * g * Q1 * Q2 * sp.k1(q * L), rel=1e-13)
    assert F < 0 and O.capillary_force(q, g, Q2, Q1, L) == pytest.approx(F, rel=1e-15)
    assert O.capillary_force(q, g, -Q1, Q2, L) > 0
    qs = 1e-7
    assert O.capillary_force(qs, g, Q1, Q2, L) == pytest.approx(-2 * math.pi * g * Q1 * Q2 / L, rel=1e-8)


def test_surface_tension_golden_value():
    """gamma at G = 3.6 from the oracle's Laplace test (tests/golden/make_gamma.py):
    positive, and dp R of the three cylinders within 5% of it."""
    lines = open(os.path.join(HERE, "golden", "gamma_G3.6.txt")).read().split("\n")
    gamma = float([l for l in lines if l and not l.startswith("#")][0])
    dpR = [float(l.split("dp R = ")[1]) for l in lines if "dp R" in l]
    assert 0.04 < gamma < 0.06
    assert all(abs(v / gamma - 1) < 0.05 for v in dpR)
