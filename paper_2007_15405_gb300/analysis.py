"""Analysis of many-particle runs (Sec. 4.7: aggregation of particles at the
film): clusters of touching particles and the radial distribution function
of the particle centres in the film plane.  Host-side post-processing of
readouts (capsule centroids); the stepping itself runs in the CUDA library.

clusters(c, L, cutoff): particles i, j are bonded when the periodic xy
distance of their centroids is below `cutoff`; clusters are the connected
components of the bond graph (union-find with path halving), returned as a
label per particle (labels 0, 1, ... in order of first appearance).

rdf(c, L, dr, rmax): g(r) of the xy centroids in a periodic box of sides L:
the histogram of pair distances in bins of width dr, divided by the count an
ideal gas of the same density would give in each annulus (n (n - 1) / 2 *
2 pi r dr / (Lx Ly) with r the bin centre).
"""
from __future__ import annotations

import numpy as np


def _pair_dist(c, L):
    d = c[:, None, :2] - c[None, :, :2]
    d -= np.asarray(L[:2], np.float64) * np.round(d / np.asarray(L[:2], np.float64))
    return np.sqrt((d ** 2).sum(-1))


def clusters(c, L, cutoff):
    """Cluster label per particle (see module doc)."""
    c = np.asarray(c, np.float64)
    n = len(c)
    parent = list(range(n))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    d = _pair_dist(c, L)
    for i in range(n):
        for j in range(i + 1, n):
            if d[i, j] < cutoff:
                ri, rj = find(i), find(j)
                if ri != rj:
                    parent[max(ri, rj)] = min(ri, rj)
    labels, out = {}, np.empty(n, np.int64)
    for i in range(n):
        r = find(i)
        if r not in labels:
            labels[r] = len(labels)
        out[i] = labels[r]
    return out


def cluster_stats(labels):
    """(number of clusters, mean cluster size, largest cluster size)."""
    sizes = np.bincount(labels)
    return int(len(sizes)), float(sizes.mean()), int(sizes.max())


def rdf(c, L, dr, rmax):
    """(bin centres, g(r)) of the xy centroids (see module doc)."""
    c = np.asarray(c, np.float64)
    n = len(c)
    d = _pair_dist(c, L)[np.triu_indices(n, 1)]
    edges = np.arange(0.0, rmax + dr, dr)
    h, _ = np.histogram(d, bins=edges)
    r = 0.5 * (edges[1:] + edges[:-1])
    ideal = n * (n - 1) / 2.0 * 2.0 * np.pi * r * dr / (L[0] * L[1])
    return r, h / ideal
