"""The many-particle analysis (clusters and radial distribution of the
centroids, Sec. 4.7), on hand-made configurations.  CPU only."""
import numpy as np

from paper_2007_15405_gb300 import analysis as A


def test_clusters_of_a_chain_and_across_the_boundary():
    """Points 0-1-2 chained (spacing 2 < 2.5), 3 alone, 4 and 5 bonded across
    the periodic x boundary (distance 1.5): three clusters."""
    L = (20.0, 20.0)
    c = np.array([[1, 5, 0], [3, 5, 0], [5, 5, 0], [10, 10, 0], [0.5, 15, 0], [19.0, 15, 0]], float)
    lab = A.clusters(c, L, 2.5)
    assert lab.tolist() == [0, 0, 0, 1, 2, 2]
    assert A.cluster_stats(lab) == (3, 2.0, 3)
    assert A.clusters(c, L, 1.0).tolist() == [0, 1, 2, 3, 4, 5]


def test_rdf_of_an_ideal_gas_and_of_a_square_lattice():
    """Uniform random points: g(r) ~ 1; a square lattice of spacing a: the
    first peak at r = a holds 2 pairs per point (4 neighbours each) and
    nothing lies below a."""
    rng = np.random.default_rng(0)
    L = (100.0, 100.0)
    c = rng.uniform(0, 100, size=(4000, 3))
    r, g = A.rdf(c, L, 1.0, 30.0)
    assert abs(g[5:].mean() - 1.0) < 0.03
    a = 5.0
    xs = np.arange(0, 100, a)
    c = np.array([[x, y, 0.0] for x in xs for y in xs])
    r, g = A.rdf(c, L, 0.5, 7.0)
    n = len(c)
    assert g[r < a - 0.5].sum() == 0
    k = np.argmin(abs(r - (a + 0.25)))
    pairs = g[k] * n * (n - 1) / 2.0 * 2 * np.pi * r[k] * 0.5 / (L[0] * L[1])
    assert round(pairs) == 2 * n
