"""ctypes binding of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import this
package.  It shares no code with the CUDA library (paper_2007_15405_gb300).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import build

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_up = C.POINTER(C.c_uint32)
_bp = C.POINTER(C.c_uint8)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_double]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_add_capsule.restype = C.c_int
        L.or_add_capsule.argtypes = [C.c_void_p, C.c_int, _dp, C.c_int, _ip, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
        L.or_set_film.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.or_set_populations.argtypes = [C.c_void_p, _dp]
        L.or_get_populations.argtypes = [C.c_void_p, _dp]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_remove_mass.argtypes = [C.c_void_p, C.c_double]
        L.or_fields.argtypes = [C.c_void_p, _dp, _dp]
        L.or_capsule_state.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_momentum.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.or_total_mass.argtypes = [C.c_void_p, _dp]
        L.or_cuts.argtypes = [C.c_void_p, _up, _ip, _bp]
        L.or_cuts_bruteforce.argtypes = [C.c_void_p, _up, _ip]
        L.or_meniscus_field.argtypes = [C.c_void_p, _dp, _dp]
        L.or_set_capsule_velocity.argtypes = [C.c_void_p, C.c_int, _dp]
        L.or_tables.argtypes = [_ip, _dp, _ip]
        L.or_equilibrium.argtypes = [C.c_double, _dp, _dp]
        L.or_sc_forces.argtypes = [C.c_void_p, _dp]
        L.or_membrane.argtypes = [C.c_int, _dp, _dp, C.c_int, _ip, C.c_double, C.c_double,
                                  C.c_double, C.c_double, _dp, _dp, C.c_int]
        L.or_mesh_volume.restype = C.c_double
        L.or_mesh_volume.argtypes = [_dp, _ip, C.c_int]
        L.or_mesh_area.restype = C.c_double
        L.or_mesh_area.argtypes = [_dp, _ip, C.c_int]
        L.or_hertz.restype = C.c_double
        L.or_hertz.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_rho_interp.restype = C.c_double
        L.or_rho_interp.argtypes = [C.c_void_p, _dp, C.c_int, C.c_int, C.c_int]
        L.or_set_cuts.argtypes = [C.c_void_p, _up, _ip]
        L.or_set_capsule_wetting.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_set_flags.argtypes = [C.c_void_p, C.c_int]
        L.or_bessel_k.restype = C.c_double
        L.or_bessel_k.argtypes = [C.c_int, C.c_double]
        L.or_meniscus_fit.restype = C.c_int
        L.or_meniscus_fit.argtypes = [_dp, _dp, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_capillary_force.restype = C.c_double
        L.or_capillary_force.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_override_cuts.restype = C.c_long
        L.or_override_cuts.argtypes = [C.c_void_p, _up, _ip, C.c_double]
        L.or_capsule_forces.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.or_meniscus_profile_of.restype = C.c_double
        L.or_meniscus_profile_of.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int,
                                             C.c_double, C.c_int, _dp, _dp, _dp]
        L.or_meniscus_profile.restype = C.c_double
        L.or_meniscus_profile.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, _dp, _dp, _dp]
        L.or_lateral_force_of.restype = C.c_double
        L.or_lateral_force_of.argtypes = [_dp, _dp, _dp, _dp, C.c_int, C.c_int]
        L.or_lateral_force.restype = C.c_double
        L.or_lateral_force.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.or_peskin.restype = C.c_double
        L.or_peskin.argtypes = [C.c_double]
        L.or_ibm_spread_point.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.or_ibm_interp_point.argtypes = [C.c_void_p, _dp, _dp, _dp]
        _lib = L
    return _lib


def peskin(r):
    """Peskin's 4-point kernel at offset r."""
    return lib().or_peskin(float(r))


def tables():
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    op = np.zeros(19, np.int32)
    lib().or_tables(_ptr(e, _ip), _ptr(w), _ptr(op, _ip))
    return e, w, op


def equilibrium(rho, u):
    f = np.zeros(19)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib().or_equilibrium(float(rho), _ptr(u), _ptr(f))
    return f


def membrane(X, Xref, F, kS=0.0, C=0.0, kB=0.0, kV=0.0, which=7):
    """Energies [skalak, helfrich, volume] and elastic node forces [nv,3]."""
    X = np.ascontiguousarray(X, np.float64)
    Xref = np.ascontiguousarray(Xref, np.float64)
    F = np.ascontiguousarray(F, np.int32)
    E = np.zeros(3)
    Fo = np.zeros_like(X)
    lib().or_membrane(X.shape[0], _ptr(X), _ptr(Xref), F.shape[0], _ptr(F, _ip), kS, C, kB, kV,
                      _ptr(E), _ptr(Fo), which)
    return E, Fo


def mesh_volume(X, F):
    X = np.ascontiguousarray(X, np.float64)
    F = np.ascontiguousarray(F, np.int32)
    return lib().or_mesh_volume(_ptr(X), _ptr(F, _ip), F.shape[0])


def mesh_area(X, F):
    X = np.ascontiguousarray(X, np.float64)
    F = np.ascontiguousarray(F, np.int32)
    return lib().or_mesh_area(_ptr(X), _ptr(F, _ip), F.shape[0])


def hertz(d, xi=1.5, delta0=1.5):
    return lib().or_hertz(xi, delta0, d)


def profile_samples(nx, ny, dr=1.0):
    """Samples of a meniscus profile: r_k = k dr for k < (min(nx, ny) // 2) / dr."""
    return int(np.floor((min(nx, ny) // 2) / dr + 1e-9))


def meniscus_profile_of(h, centres, cid, dr=1.0, nr=None):
    """Profile (r, zeta), rise Z and far-field height h_inf of capsule cid from a
    height field h [ny, nx] and the xy centroids [(cx, cy), ...] of all capsules."""
    h = np.ascontiguousarray(h, np.float64)
    ny, nx = h.shape
    c = np.asarray(centres, np.float64).reshape(-1, 2)
    cx = np.ascontiguousarray(c[:, 0]); cy = np.ascontiguousarray(c[:, 1])
    nr = profile_samples(nx, ny, dr) if nr is None else nr
    r = np.zeros(nr); z = np.zeros(nr); Z = np.zeros(1)
    hinf = lib().or_meniscus_profile_of(_ptr(h), nx, ny, len(cx), _ptr(cx), _ptr(cy), int(cid),
                                        float(dr), nr, _ptr(r), _ptr(z), _ptr(Z))
    return r, z, float(Z[0]), hinf


def lateral_force_of(Fa, Fb, ca, cb, nx, ny):
    """1/2 (F_b - F_a) . e_ab with e_ab the unit xy vector from centroid a to b."""
    a = [np.ascontiguousarray(v, np.float64) for v in (Fa, Fb, ca, cb)]
    return lib().or_lateral_force_of(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), int(nx), int(ny))


def bessel_k(nu, x):
    """K_nu(x) from its integral representation (nu = 0, 1, ...)."""
    return lib().or_bessel_k(int(nu), float(x))


def meniscus_fit(r, zeta, rmin=0.0, rmax=np.inf):
    """(Q, q, rms, samples) of the least-squares fit zeta = Q K_0(q r) over
    rmin <= r <= rmax (finite samples only)."""
    r = np.ascontiguousarray(r, np.float64)
    z = np.ascontiguousarray(zeta, np.float64)
    Q, q, rms = np.zeros(1), np.zeros(1), np.zeros(1)
    m = lib().or_meniscus_fit(_ptr(r), _ptr(z), len(r), float(rmin), float(min(rmax, 1e300)),
                              _ptr(Q), _ptr(q), _ptr(rms))
    return float(Q[0]), float(q[0]), float(rms[0]), m


def capillary_force(q, gamma, Q1, Q2, L):
    """-2 pi q gamma Q1 Q2 K_1(q L) (Eq. 13)."""
    return lib().or_capillary_force(float(q), float(gamma), float(Q1), float(Q2), float(L))


class Oracle:
    """One lattice with its capsules, stepped by the FP64 oracle."""

    # alternative readings of paper-silent points (or_set_flags)
    INERTIAL, REF_RHO, MIRROR, REMOVE, IBM = 1, 2, 4, 8, 16

    def __init__(self, nx, ny, nz, wall=1, tau=(1.0, 1.0), G=3.6, rep_dz=10.0, flags=0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self._h = lib().or_create(nx, ny, nz, wall, tau[0], tau[1], G, rep_dz)
        if flags:
            lib().or_set_flags(self._h, int(flags))
        self.nv = []

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def from_workload(cls, wl, set_film=True):
        o = cls(wl.nx, wl.ny, wl.nz, wall=wl.wall, tau=wl.tau, G=wl.G, rep_dz=wl.rep_dz,
                flags=getattr(wl, "flags", 0))
        for cap in wl.capsules:
            X, F = cap.mesh()
            o.add_capsule(X, F, cap.kS, cap.C, cap.kB, cap.kV, cap.mass, cap.mode,
                          wet=getattr(cap, "wet", 0.0))
        if set_film:
            from paper_2007_15405_gb300.inputs import RHO_MAJ, RHO_MIN, RHO_MIX
            o.set_film(wl.h_top, RHO_MAJ, RHO_MIN, RHO_MIX, wl.jitter())
        if getattr(wl, "dry_dm", 0.0) > 0.0:
            o.remove_mass(wl.dry_dm)
        return o

    def add_capsule(self, X, F, kS, C, kB, kV, mass, mode, wet=0.0):
        X = np.ascontiguousarray(X, np.float64)
        F = np.ascontiguousarray(F, np.int32)
        cid = lib().or_add_capsule(self._h, X.shape[0], _ptr(X), F.shape[0], _ptr(F, _ip), kS, C,
                                   kB, kV, mass, mode)
        if cid < 0:
            raise RuntimeError("oracle: capsule rejected (too many capsules, or an element spans more than "
                               "16 lattice units)")
        if wet:
            lib().or_set_capsule_wetting(self._h, cid, float(wet))
        self.nv.append(X.shape[0])
        return cid

    def set_film(self, h_top, rho_maj, rho_min, rho_mix, jit=None):
        j = None if jit is None else np.ascontiguousarray(jit, np.float64).reshape(-1)
        lib().or_set_film(self._h, h_top, rho_maj, rho_min, rho_mix, _ptr(j))

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        assert f.size == 38 * self.N
        lib().or_set_populations(self._h, _ptr(f))

    def populations(self):
        f = np.zeros((2, 19, self.nz, self.ny, self.nx))
        lib().or_get_populations(self._h, _ptr(f))
        return f

    def step(self, n=1):
        if lib().or_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle: a membrane element spans more than 16 lattice units or has a "
                               "non-finite vertex (diverged run)")

    def remove_mass(self, dmA):
        """Drying: turn dmA of component A into B each step (0 turns it off)."""
        lib().or_remove_mass(self._h, float(dmA))

    def fields(self):
        rho = np.zeros((2, self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        lib().or_fields(self._h, _ptr(rho), _ptr(u))
        return rho, u

    def capsule_state(self, cid):
        nv = self.nv[cid]
        X = np.zeros((nv, 3)); V = np.zeros((nv, 3)); Fc = np.zeros((nv, 3)); Ft = np.zeros((nv, 3))
        o = np.zeros(8)
        lib().or_capsule_state(self._h, cid, _ptr(X), _ptr(V), _ptr(Fc), _ptr(Ft), _ptr(o))
        return dict(X=X, V=V, Fcpl=Fc, Ftot=Ft, force=o[0:3].copy(), torque=o[3:6].copy(),
                    area=o[6], volume=o[7])

    def momentum(self):
        a, b, c = np.zeros(3), np.zeros(3), np.zeros(3)
        lib().or_momentum(self._h, _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def total_mass(self):
        m = np.zeros(2)
        lib().or_total_mass(self._h, _ptr(m))
        return m

    def cuts(self):
        mask = np.zeros((self.nz, self.ny, self.nx), np.uint32)
        tri = np.zeros((self.nz, self.ny, self.nx, 18), np.int32)
        inside = np.zeros((self.nz, self.ny, self.nx), np.uint8)
        lib().or_cuts(self._h, _ptr(mask, _up), _ptr(tri, _ip), _ptr(inside, _bp))
        return mask, tri, inside

    def cut_mask(self):
        mask = np.zeros((self.nz, self.ny, self.nx), np.uint32)
        lib().or_cuts(self._h, _ptr(mask, _up), None, None)
        return mask

    def cuts_bruteforce(self):
        mask = np.zeros((self.nz, self.ny, self.nx), np.uint32)
        tri = np.zeros((self.nz, self.ny, self.nx, 18), np.int32)
        lib().or_cuts_bruteforce(self._h, _ptr(mask, _up), _ptr(tri, _ip))
        return mask, tri

    def meniscus_field(self, rho=None):
        h = np.zeros((self.ny, self.nx))
        r = None if rho is None else np.ascontiguousarray(rho, np.float64)
        lib().or_meniscus_field(self._h, _ptr(r), _ptr(h))
        return h

    def set_capsule_velocity(self, cid, V):
        V = np.ascontiguousarray(V, np.float64)
        lib().or_set_capsule_velocity(self._h, cid, _ptr(V))

    def rho_interp(self, rho, x, y, z):
        """Partner density across a cut or substrate link at node (x, y, z) for
        the density field rho [nz, ny, nx] of one component."""
        r = np.ascontiguousarray(rho, np.float64)
        assert r.size == self.N
        return lib().or_rho_interp(self._h, _ptr(r), int(x), int(y), int(z))

    def set_cuts(self, mask, tri):
        """Replace the cut structure (mask [nz, ny, nx], elements [nz, ny, nx, 18])."""
        m = np.ascontiguousarray(mask, np.uint32)
        t = np.ascontiguousarray(tri, np.int32)
        lib().or_set_cuts(self._h, _ptr(m, _up), _ptr(t, _ip))

    def override_cuts(self, mask, tri, margin=1e-4):
        """Adopt a cut structure computed elsewhere where every difference is a
        near tie of the oracle's decision (returns the number of differing link
        ends), else keep the oracle's (returns minus the number of differences
        that are not near ties)."""
        m = np.ascontiguousarray(mask, np.uint32)
        t = np.ascontiguousarray(tri, np.int32)
        return lib().or_override_cuts(self._h, _ptr(m, _up), _ptr(t, _ip), float(margin))

    def capsule_forces(self, cid):
        """(elastic, interaction) node forces [nv, 3] of the last step."""
        nv = self.nv[cid]
        Fe = np.zeros((nv, 3)); Fi = np.zeros((nv, 3))
        lib().or_capsule_forces(self._h, cid, _ptr(Fe), _ptr(Fi))
        return Fe, Fi

    def meniscus_profile(self, cid, dr=1.0):
        """(r, zeta, Z, h_inf) of capsule cid on the last step's densities."""
        nr = profile_samples(self.nx, self.ny, dr)
        r = np.zeros(nr); z = np.zeros(nr); Z = np.zeros(1)
        hinf = lib().or_meniscus_profile(self._h, int(cid), float(dr), nr, _ptr(r), _ptr(z), _ptr(Z))
        return r, z, float(Z[0]), hinf

    def ibm_spread_point(self, X, F, f=None):
        """f [3][N] (float64) += the force F at X spread with Peskin's
        4-point kernel (diffuse-interface coupling)."""
        N = self.nx * self.ny * self.nz
        f = np.zeros(3 * N) if f is None else f
        X = np.ascontiguousarray(X, np.float64)
        F = np.ascontiguousarray(F, np.float64)
        lib().or_ibm_spread_point(self._h, _ptr(X), _ptr(F), _ptr(f))
        return f

    def ibm_interp_point(self, u, X):
        """The field u [3][N] interpolated at X with the same kernel."""
        u = np.ascontiguousarray(u, np.float64).reshape(-1)
        X = np.ascontiguousarray(X, np.float64)
        out = np.zeros(3)
        lib().or_ibm_interp_point(self._h, _ptr(u), _ptr(X), _ptr(out))
        return out

    def lateral_force(self, a, b):
        return lib().or_lateral_force(self._h, int(a), int(b))

    def sc_forces(self):
        F = np.zeros((2, 3, self.nz, self.ny, self.nx))
        lib().or_sc_forces(self._h, _ptr(F))
        return F
