"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module holds no arithmetic of the method itself: it only builds meshes, random
density jitter and the workload descriptions (lattice sizes, film heights, capsule
placements and moduli) that both sides receive as plain arrays.

Workloads follow the simulation set-up of the paper (Sec. 3.2 "Simulation setup"):
two equal-density components with initial majority/minority densities 0.7/0.04 and
one mixed layer at 0.3, G = 3.6, node mass 25, Hertz range 1.5 and a repulsive plane
10 lattice units above the substrate.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# Physical constants of the set-up (Sec. 3.2).
RHO_MAJ = 0.7
RHO_MIN = 0.04
RHO_MIX = 0.3
G_SC = 3.6
NODE_MASS = 25.0
REP_DZ = 10.0  # repulsive plane offset above the substrate (Delta_z)
DELTA0 = 1.5   # Hertz cut-off
XI = 1.5       # Hertz strength

MODE_FREE = 0
MODE_FROZEN = 1
MODE_FIXED = 2


def icosphere(level: int, radius: float = 1.0,
              centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)) -> Tuple[np.ndarray, np.ndarray]:
    """Subdivided icosahedron projected on a sphere.

    Returns (nodes float64 [nv,3], faces int32 [nf,3]) with faces oriented
    counter-clockwise seen from outside (outward normals).  nv = 10*4**level + 2,
    nf = 20*4**level (level 3: 642/1280, level 4: 2562/5120).
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    X = np.array(verts, dtype=np.float64) * radius + np.asarray(centre, dtype=np.float64)
    F = np.array(faces, dtype=np.int32)
    # orient outward: the icosahedron list above is counter-clockwise from outside
    c = np.asarray(centre, dtype=np.float64)
    n = np.cross(X[F[:, 1]] - X[F[:, 0]], X[F[:, 2]] - X[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, X[F[:, 0]] - c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return X, F


def jitter(shape_zyx: Tuple[int, int, int], amplitude: float, seed: int) -> np.ndarray:
    """Uniform density jitter U(-a, a) for both components, float64 [2, nz, ny, nx]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape_zyx
    return rng.uniform(-amplitude, amplitude, size=(2, nz, ny, nx))


@dataclasses.dataclass
class CapsuleSpec:
    centre: Tuple[float, float, float]
    radius: float
    level: int
    kS: float = 5e-3
    C: float = 0.0
    kB: float = 1e-3
    kV: float = 1.0
    mass: float = NODE_MASS
    mode: int = MODE_FREE
    wet: float = 0.0  # wetting offset of the interpolated densities (0: neutral)

    def mesh(self):
        return icosphere(self.level, self.radius, self.centre)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    h_top: float
    capsules: List[CapsuleSpec]
    steps: int
    tau: Tuple[float, float] = (1.0, 1.0)
    G: float = G_SC
    wall: int = 1
    jitter_amp: float = 1e-3
    seed: int = 1234
    rep_dz: float = REP_DZ
    dry_dm: float = 0.0  # drying: A mass turned into B per step (0: off)
    flags: int = 0       # alternative readings of paper-silent points (cf_lattice_desc.flags)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def jitter(self) -> Optional[np.ndarray]:
        if self.jitter_amp == 0.0:
            return None
        return jitter((self.nz, self.ny, self.nx), self.jitter_amp, self.seed)


def z_rest(radius: float) -> float:
    """Capsule centre height with its bottom where the substrate repulsion starts
    (Sec. 4.2: the lower part of the particle sits at the boundary of the interaction)."""
    return 0.5 + REP_DZ + DELTA0 + radius


# Small generic offsets keep icosphere vertices off lattice links so that no
# link-triangle test is an exact tie.
_OFF = (0.3, 0.4, 0.17)


def single_capsule_film(mode: int = MODE_FREE, steps: int = 1000) -> Workload:
    """32x32x48 lattice, tau=1, substrate at z=0, A film 12 cells thick under B,
    one R=8 level-3 icosphere (642 nodes / 1280 faces), kS=5e-3, area-dilation
    ratio 1 (C=0), kB=1e-3, jitter +-1e-3, 1000 steps."""
    cap = CapsuleSpec(centre=(16 + _OFF[0], 16 + _OFF[1], z_rest(8.0) + _OFF[2]), radius=8.0,
                      level=3, kS=5e-3, C=0.0, kB=1e-3, mode=mode)
    return Workload("single-capsule film 32x32x48 R=8", 32, 32, 48, h_top=12.5,
                    capsules=[cap], steps=steps)


def capsule_pair(steps: int = 20000, mode: int = MODE_FREE, nx: int = 128, ny: int = 64,
                 nz: int = 64, radius: float = 12.0, level: int = 4) -> Workload:
    """Two R=12 level-4 capsules (2562 nodes each) at centre distance 3R in a
    128x64x64 lattice, film height 0.6R above the repulsive plane."""
    d = 3.0 * radius
    zc = z_rest(radius) + _OFF[2]
    cx = nx / 2 + _OFF[0]
    cy = ny / 2 + _OFF[1]
    caps = [CapsuleSpec(centre=(cx - d / 2, cy, zc), radius=radius, level=level, mode=mode),
            CapsuleSpec(centre=(cx + d / 2, cy, zc), radius=radius, level=level, mode=mode)]
    h_top = 0.5 + REP_DZ + 0.6 * radius
    return Workload(f"capsule pair {nx}x{ny}x{nz} R={radius:g} d=3R", nx, ny, nz, h_top=h_top,
                    capsules=caps, steps=steps)


def tiny_film(nx=16, ny=12, nz=20, radius=4.0, level=2, mode=MODE_FREE, steps=20,
              h_top=None, seed=99, rep_dz=2.0) -> Workload:
    """Small ragged lattice for oracle-vs-kernel element-wise parity (repulsive
    plane lowered to 2 lattice units so that the capsule fits)."""
    zc = 0.5 + rep_dz + DELTA0 + radius + _OFF[2]
    cap = CapsuleSpec(centre=(nx / 2 + _OFF[0], ny / 2 + _OFF[1], zc), radius=radius,
                      level=level, kS=5e-3, C=1.0, kB=1e-3, mode=mode)
    if h_top is None:
        h_top = zc - 0.3 * radius
    return Workload(f"tiny film {nx}x{ny}x{nz}", nx, ny, nz, h_top=h_top, capsules=[cap],
                    steps=steps, seed=seed, rep_dz=rep_dz)


def sweep_point(d_over_R: float, kS: Optional[float], nx: int, ny: int, nz: int,
                radius: float = 10.0, level: int = 4, steps: int = 20000, seed: int = 1234,
                h_frac: float = 0.4, mode: Optional[int] = None) -> Workload:
    """One lattice of a distance x softness sweep: two capsules of radius R at
    centre distance d = d_over_R * R along x, film h_frac R above the
    repulsive plane; kS None is the rigid limit (frozen shape).  mode, when
    given, overrides the capsules' mode (e.g. fixed capsules for force runs)."""
    d = d_over_R * radius
    zc = z_rest(radius) + _OFF[2]
    cx, cy = nx / 2 + _OFF[0], ny / 2 + _OFF[1]
    if mode is None:
        mode = MODE_FROZEN if kS is None else MODE_FREE
    k = 5e-3 if kS is None else kS
    caps = [CapsuleSpec(centre=(cx - d / 2, cy, zc), radius=radius, level=level, kS=k, mode=mode),
            CapsuleSpec(centre=(cx + d / 2, cy, zc), radius=radius, level=level, kS=k, mode=mode)]
    h_top = 0.5 + REP_DZ + h_frac * radius
    soft = "rigid" if kS is None else f"kS={kS:g}"
    return Workload(f"sweep {nx}x{ny}x{nz} d={d_over_R:.2f}R {soft}", nx, ny, nz, h_top=h_top,
                    capsules=caps, steps=steps, seed=seed)


def rigid_particle(h_frac: float, radius: float = 10.0, level: int = 4, nx: int = 128, ny: int = 128,
                   nz: int = 40, steps: int = 40000, seed: int = 4321) -> Workload:
    """One fixed rigid particle (Sec. 4.1: a level-4 icosphere of radius R,
    its bottom where the substrate repulsion starts) at the lattice centre,
    film h_frac R above the repulsive plane: the meniscus of one particle,
    for the fit of Eq. 12 and the film-height series of Q and Z."""
    cap = CapsuleSpec(centre=(nx / 2 + _OFF[0], ny / 2 + _OFF[1], z_rest(radius) + _OFF[2]), radius=radius,
                      level=level, mode=MODE_FIXED)
    return Workload(f"rigid particle {nx}x{ny}x{nz} h0={h_frac:g}R", nx, ny, nz,
                    h_top=0.5 + REP_DZ + h_frac * radius, capsules=[cap], steps=steps, seed=seed)


def rigid_pair(gap_over_R: float, h_frac: float = 0.16, radius: float = 10.0, level: int = 4,
               nx: Optional[int] = None, ny: int = 96, nz: int = 40, steps: int = 40000,
               seed: int = 4322) -> Workload:
    """Two fixed rigid particles (Sec. 4.1 force validation) with surface gap
    gap_over_R * R (centre distance L = gap + 2R) along x, film h_frac R
    above the repulsive plane (0.16R in the paper).  The box is 2L + 64 long
    (a multiple of 8) unless given, so the pair's periodic images stay
    farther than L + 64."""
    L = gap_over_R * radius + 2.0 * radius
    if nx is None:
        nx = 8 * int(math.ceil((2.0 * L + 64.0) / 8.0))
    zc = z_rest(radius) + _OFF[2]
    cx, cy = nx / 2 + _OFF[0], ny / 2 + _OFF[1]
    caps = [CapsuleSpec(centre=(cx - L / 2, cy, zc), radius=radius, level=level, mode=MODE_FIXED),
            CapsuleSpec(centre=(cx + L / 2, cy, zc), radius=radius, level=level, mode=MODE_FIXED)]
    return Workload(f"rigid pair {nx}x{ny}x{nz} gap={gap_over_R:g}R", nx, ny, nz,
                    h_top=0.5 + REP_DZ + h_frac * radius, capsules=caps, steps=steps, seed=seed)


SWEEP_MODULI = (1e-3, 1e-2, 1e-1, None)  # shear moduli and the rigid limit


def batched_sweep(n_dist: int = 16, moduli=SWEEP_MODULI, radius: float = 10.0, level: int = 4,
                  steps: int = 20000, h_frac: float = 0.4, mode: Optional[int] = None) -> List[Workload]:
    """Distance x softness sweep of independent lattices of uneven size: n_dist
    distances in [2.2R, 6R] times the moduli (64 lattices by default), two
    R = 10 level-4 capsules (2562 nodes each) per lattice, film 0.4R above the
    repulsive plane.  The lattice grows with the distance (x: 64..160) and
    with the modulus index (y: 48..80, z: 48..64), from 147k to 819k nodes
    (26.1M in all)."""
    out = []
    for i in range(n_dist):
        f = i / max(1, n_dist - 1)
        d_over_R = 2.2 + f * (6.0 - 2.2)
        nx = 64 + 8 * int(round(f * 12))
        for j, kS in enumerate(moduli):
            g = j / max(1, len(moduli) - 1)
            ny = 48 + 8 * int(round(g * 4))
            nz = 48 + 8 * int(round(g * 2))
            out.append(sweep_point(d_over_R, kS, nx, ny, nz, radius=radius, level=level,
                                   steps=steps, seed=1234 + 97 * i + j, h_frac=h_frac, mode=mode))
    return out


def drying_film(nx: int = 256, ny: int = 256, nz: int = 96, n_caps: int = 16, radius: float = 10.0,
                level: int = 4, seed: int = 7, steps: int = 50000, h_from: float = 0.6,
                h_to: float = 0.2) -> Workload:
    """Drying film: n_caps capsules of radius R (level-4 icospheres, 2562
    nodes each) at rest on the repulsive plane, on a seeded random layout
    (centres uniform in xy, at least R + delta0 + 1 from the box sides, centre
    distances at least 2R + 2 delta0; rejection sampling), in a film whose
    height is lowered linearly from h_from R to h_to R above the repulsive
    plane over `steps` steps.  The lowering is a steady conversion of A into B:
    per step, the A excess (rho_maj - rho_min) of the lowered layer over the
    whole nx x ny area, divided by the steps."""
    rng = np.random.default_rng(seed)
    lo = radius + DELTA0 + 1.0
    dmin = 2.0 * radius + 2.0 * DELTA0
    pts: List[Tuple[float, float]] = []
    tries = 0
    while len(pts) < n_caps:
        tries += 1
        if tries > 200000:
            raise ValueError(f"{n_caps} capsules of radius {radius} do not fit in {nx}x{ny}")
        p = (float(rng.uniform(lo, nx - lo)), float(rng.uniform(lo, ny - lo)))
        if all(math.hypot(p[0] - q[0], p[1] - q[1]) >= dmin for q in pts):
            pts.append(p)
    zc = z_rest(radius) + _OFF[2]
    caps = [CapsuleSpec(centre=(x + _OFF[0], y + _OFF[1], zc), radius=radius, level=level)
            for x, y in pts]
    h_top = 0.5 + REP_DZ + h_from * radius
    dm = (h_from - h_to) * radius * nx * ny * (RHO_MAJ - RHO_MIN) / steps
    return Workload(f"drying film {nx}x{ny}x{nz} {n_caps} capsules R={radius:g}", nx, ny, nz,
                    h_top=h_top, capsules=caps, steps=steps, seed=seed, dry_dm=dm)


def warm_dataset(n: int, seed: int = 0, nx: int = 48, ny: int = 32, nz: int = 32,
                 mode: int = MODE_FREE) -> List[Workload]:
    """Set-ups for the learned warm start: one capsule (R in [5, 7], level-3
    icosphere; free by default, or fixed: the rigid particles of Sec. 4.1) at a
    random position protruding through a film of random height (0.3R..0.9R
    above the repulsive plane), shear modulus log-uniform in [3e-3, 1e-1]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        R = float(rng.uniform(5.0, 7.0))
        cx = float(rng.uniform(R + 4, nx - R - 4)) + _OFF[0]
        cy = float(rng.uniform(R + 4, ny - R - 4)) + _OFF[1]
        zc = z_rest(R) + _OFF[2]
        kS = float(10 ** rng.uniform(math.log10(3e-3), -1))
        h_top = 0.5 + REP_DZ + float(rng.uniform(0.3, 0.9)) * R
        cap = CapsuleSpec(centre=(cx, cy, zc), radius=R, level=3, kS=kS, mode=mode)
        out.append(Workload(f"warm {i} R={R:.2f} kS={kS:.1e} h={h_top:.2f}", nx, ny, nz, h_top=h_top,
                            capsules=[cap], steps=1, seed=5000 + i))
    return out


def warm_pair_dataset(n: int, seed: int = 0, nx: int = 128, ny: int = 64, nz: int = 48, radius: float = 10.0,
                      level: int = 4, mode: int = MODE_FIXED) -> List[Workload]:
    """Set-ups of the sweep's generator for training the warm start: a
    capsule pair (R = 10 level-4 icospheres) at a centre distance uniform in
    [2.2R, 6R], a shear modulus log-uniform in [1e-3, 1e-1] or rigid (one
    set-up in four), a film uniform in [0.2R, 0.6R] above the repulsive plane,
    on one lattice shape (128 x 64 x 48: every lattice of a training batch has
    the same shape).  A rigid pair is given kS = 1 (far stiffer than the soft
    range, so its shape does not change and its modulus feature is distinct).
    mode: the capsules' mode (fixed for the equilibrated densities, free for
    the deformation)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d_over_R = float(rng.uniform(2.2, 6.0))
        rigid = rng.random() < 0.25
        kS = 1.0 if rigid else float(10 ** rng.uniform(-3.0, -1.0))
        h = float(rng.uniform(0.2, 0.6))
        w = sweep_point(d_over_R, kS, nx, ny, nz, radius=radius, level=level, seed=7000 + 31 * seed + i,
                        h_frac=h, mode=mode)
        w.name = f"warm pair {i} d={d_over_R:.2f}R kS={'rigid' if rigid else f'{kS:.1e}'} h0={h:.2f}R"
        out.append(w)
    return out


GAMMA_G36 = 0.048812802376  # surface tension at G = 3.6 (oracle Laplace test, tests/golden)


def approach_pair(beta: float, gap_over_R: float = 2.0, h_frac: float = 0.4, radius: float = 10.0,
                  level: int = 4, nx: int = 128, ny: int = 64, nz: int = 48, steps: int = 40000,
                  kS: float = 5e-3, seed: int = 4323) -> Workload:
    """Two free soft particles (Sec. 4.6, approach dynamics): spheres of
    radius R at surface gap gap_over_R * R along x in a film h_frac R above
    the repulsive plane, softness beta = R^2 gamma / kB (kB from beta and the
    surface tension at G = 3.6), Poisson ratio 0.9 (C = 9), shear modulus kS."""
    kB = radius * radius * GAMMA_G36 / beta
    L = gap_over_R * radius + 2.0 * radius
    zc = z_rest(radius) + _OFF[2]
    cx, cy = nx / 2 + _OFF[0], ny / 2 + _OFF[1]
    caps = [CapsuleSpec(centre=(cx - L / 2, cy, zc), radius=radius, level=level, kS=kS, C=9.0, kB=kB),
            CapsuleSpec(centre=(cx + L / 2, cy, zc), radius=radius, level=level, kS=kS, C=9.0, kB=kB)]
    return Workload(f"approach beta={beta:g} {nx}x{ny}x{nz}", nx, ny, nz, h_top=0.5 + REP_DZ + h_frac * radius,
                    capsules=caps, steps=steps, seed=seed)


def many_capsules(n_caps: int = 100, nx: int = 320, ny: int = 320, nz: int = 40, radius: float = 10.0,
                  level: int = 4, h_frac: float = 0.35, beta: float = 25.0, seed: int = 12,
                  steps: int = 20000, dmin: Optional[float] = None) -> Workload:
    """Many free soft particles in a film (Sec. 4.7, aggregation; the paper's
    run has 1730 particles of R = 10 on 1200 x 1200 x 40 at h0 = 0.35R, an
    area fraction of 0.38; 100 particles on 320 x 320 give 0.31): centres
    uniform in xy with centre distances at least dmin (default 2R + 2 delta0
    + 1; random sequential addition, periodic), bottoms where the substrate
    repulsion starts, softness beta = R^2 gamma / kB with Poisson ratio 0.9."""
    rng = np.random.default_rng(seed)
    if dmin is None:
        dmin = 2.0 * radius + 2.0 * DELTA0 + 1.0
    box = np.array([nx, ny], dtype=np.float64)
    pts = np.zeros((0, 2))
    tries = 0
    while len(pts) < n_caps:
        tries += 1
        if tries > 2000000:
            raise ValueError(f"{n_caps} capsules of radius {radius} do not fit in {nx}x{ny}")
        p = rng.uniform(0.0, 1.0, 2) * box
        d = pts - p
        d -= np.floor(d / box + 0.5) * box  # nearest periodic image
        if len(pts) == 0 or np.hypot(d[:, 0], d[:, 1]).min() >= dmin:
            pts = np.vstack([pts, p])
    kB = radius * radius * GAMMA_G36 / beta
    zc = z_rest(radius) + _OFF[2]
    caps = [CapsuleSpec(centre=(float(x), float(y), zc), radius=radius, level=level, kS=5e-3, C=9.0, kB=kB)
            for x, y in pts]
    return Workload(f"{n_caps} capsules {nx}x{ny}x{nz} beta={beta:g}", nx, ny, nz,
                    h_top=0.5 + REP_DZ + h_frac * radius, capsules=caps, steps=steps, seed=seed)
