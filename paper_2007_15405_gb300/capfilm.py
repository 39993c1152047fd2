"""Thin Python binding of the capfilm C ABI (include/capfilm.h).

Argument marshalling only: every step of the method runs in the CUDA library
libcapfilm.so built next to this file.  PyTorch supplies device memory (its
caching allocator, through the ABI's allocator callbacks) and the CUDA stream.
There is no CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcapfilm.so")

CF_OK = 0
STATUS_NAMES = {0: "CF_OK", 1: "CF_EINVAL", 2: "CF_ENOMEM", 3: "CF_ECUDA", 4: "CF_ESTATE",
                5: "CF_ENOTFOUND", 6: "CF_EDIVERGED", 7: "CF_EOVERFLOW"}

FREE, FROZEN, FIXED = 0, 1, 2
# alternative readings (cf_lattice_desc.flags)
INERTIAL, LADD_REF_RHO, PARTNER_MIRROR, DRY_REMOVE, IBM = 1, 2, 4, 8, 16
FP32, FP16_SHIFT, BF16_SHIFT = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("wall", C.c_int),
                ("tau", C.c_double * 2), ("G", C.c_double), ("rep_dz", C.c_double),
                ("xi", C.c_double), ("delta0", C.c_double), ("precision", C.c_int),
                ("allocator", C.POINTER(Allocator)), ("stream", C.c_void_p), ("flags", C.c_int)]


class CapsuleDesc(C.Structure):
    _fields_ = [("nv", C.c_int), ("nf", C.c_int), ("nodes", C.POINTER(C.c_double)),
                ("faces", C.POINTER(C.c_int)), ("kS", C.c_double), ("C", C.c_double),
                ("kB", C.c_double), ("kV", C.c_double), ("mass", C.c_double), ("mode", C.c_int),
                ("wet", C.c_double)]


class WarmPolicy(C.Structure):
    _fields_ = [("window", C.c_int), ("u_limit", C.c_double), ("grow", C.c_double), ("fallback", C.c_int)]


class CapfilmError(RuntimeError):
    pass


_lib = None
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


def _dptr(t):
    """Device pointer of a torch tensor (None stays NULL)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def load_library(path: Optional[str] = None):
    """Load libcapfilm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise CapfilmError(f"CUDA library not built: {path} is missing (run build())")
    L = C.CDLL(path)
    L.cf_last_error.restype = C.c_char_p
    sig = {
        "cf_create": [C.POINTER(LatticeDesc), C.POINTER(C.c_void_p)],
        "cf_destroy": [C.c_void_p],
        "cf_add_capsule": [C.c_void_p, C.POINTER(CapsuleDesc), C.POINTER(C.c_int)],
        "cf_add_capsules": [C.c_void_p, C.POINTER(CapsuleDesc), C.c_int, C.POINTER(C.c_int)],
        "cf_set_capsule_mode": [C.c_void_p, C.c_int, C.c_int],
        "cf_set_film": [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, _dp],
        "cf_step": [C.c_void_p, C.c_longlong],
        "cf_sync": [C.c_void_p],
        "cf_capsule_force": [C.c_void_p, C.c_int, _dp, _dp],
        "cf_lateral_force": [C.c_void_p, C.c_int, C.c_int, _dp],
        "cf_capsule_state": [C.c_void_p, C.c_int, _dp, _dp, _dp],
        "cf_fields": [C.c_void_p, _dp, _dp, C.POINTER(C.c_size_t)],
        "cf_populations": [C.c_void_p, _fp],
        "cf_total_mass": [C.c_void_p, _dp],
        "cf_meniscus_field": [C.c_void_p, _dp],
        "cf_meniscus_profile": [C.c_void_p, C.c_int, C.c_double, _dp, _dp, C.POINTER(C.c_size_t),
                                _dp],
        "cf_cuts": [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_int), C.POINTER(C.c_uint8)],
        "cf_launch_count": [C.c_void_p, C.POINTER(C.c_longlong)],
        "cf_time_phases": [C.c_void_p, C.c_longlong, _dp],
        "cf_lattice_step_static": [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                   _dp, C.c_double, C.c_void_p],
        "cf_set_densities": [C.c_void_p, _dp, _dp],
        "cf_remove_mass": [C.c_void_p, C.c_double],
        "cf_conv3d_forward": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                              C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
        "cf_conv3d_backward": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                               C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p],
        "cf_mse": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_double, C.c_void_p,
                   C.c_void_p, C.c_void_p],
        "cf_adam": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong,
                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p],
        "cf_to_bf16": [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p],
        "cf_from_bf16": [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p],
        "cf_batch_create": [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)],
        "cf_batch_destroy": [C.c_void_p],
        "cf_batch_step": [C.c_void_p, C.c_longlong],
        "cf_batch_time": [C.c_void_p, C.c_longlong, _dp],
        "cf_batch_time_phases": [C.c_void_p, C.c_longlong, _dp],
        "cf_batch_set_config": [C.c_void_p, C.c_int, C.c_int],
        "cf_batch_set_groups": [C.c_void_p, C.c_int],
        "cf_batch_config": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "cf_batch_autotune": [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int), _dp],
        "cf_batch_launch_count": [C.c_void_p, C.POINTER(C.c_longlong)],
        "cf_batch_lateral_forces": [C.c_void_p, C.c_int, C.c_int, _dp],
        "cf_save": [C.c_void_p, C.c_char_p],
        "cf_load": [C.c_void_p, C.c_char_p],
        "cf_meniscus_height": [C.c_void_p, C.c_int, _dp],
        "cf_warm_features": [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p],
        "cf_warm_apply": [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p],
        "cf_warm_target": [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p],
        "cf_field_check": [C.c_void_p, _dp],
        "cf_unet_conv": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                         C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_conv_tc": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                            C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_tc_error": [C.POINTER(C.c_uint)],
        "cf_unet_flip": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_wgrad": [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                          C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
        "cf_unet_relu_grad": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p],
        "cf_unet_loss": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                         C.c_double, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                         C.c_void_p, C.c_void_p],
        "cf_unet_pool": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_pool_bwd": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                             C.c_void_p],
        "cf_unet_upsample": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                             C.c_void_p],
        "cf_unet_upsample_bwd": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                 C.c_void_p],
        "cf_unet_concat": [C.c_longlong, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_split": [C.c_longlong, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
        "cf_unet_pack": [C.c_void_p, C.c_int, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p],
        "cf_unet_unpack": [C.c_void_p, C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_int, C.c_void_p,
                           C.c_void_p],
        "cf_meniscus_fit": [_dp, _dp, C.c_size_t, C.c_double, C.c_double, _dp],
        "cf_model_load": [C.c_char_p, C.POINTER(C.c_void_p)],
        "cf_model_destroy": [C.c_void_p],
        "cf_warmstart": [C.c_void_p, C.c_void_p, C.POINTER(WarmPolicy), C.c_double, C.c_double, C.c_double,
                         C.c_double, C.c_double, _dp, C.POINTER(C.c_int), C.POINTER(C.c_longlong)],
        "cf_capillary_force": [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _dp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    _lib = L
    return L


def exported_symbols():
    return ["cf_last_error", "cf_create", "cf_destroy", "cf_add_capsule", "cf_add_capsules", "cf_set_capsule_mode",
            "cf_set_film", "cf_step", "cf_sync", "cf_capsule_force", "cf_lateral_force",
            "cf_capsule_state", "cf_fields", "cf_populations", "cf_total_mass",
            "cf_meniscus_field", "cf_meniscus_profile", "cf_cuts", "cf_launch_count",
            "cf_time_phases", "cf_lattice_step_static", "cf_batch_create", "cf_batch_destroy",
            "cf_batch_step", "cf_batch_time", "cf_batch_time_phases", "cf_batch_set_config", "cf_batch_set_groups", "cf_batch_config",
            "cf_batch_autotune", "cf_batch_launch_count", "cf_set_densities", "cf_remove_mass", "cf_save", "cf_load", "cf_meniscus_height",
            "cf_batch_lateral_forces", "cf_warm_features", "cf_warm_apply", "cf_warm_target",
            "cf_field_check", "cf_conv3d_forward",
            "cf_conv3d_backward", "cf_mse", "cf_adam", "cf_to_bf16", "cf_from_bf16",
            "cf_meniscus_fit", "cf_capillary_force", "cf_model_load", "cf_model_destroy", "cf_warmstart",
            "cf_unet_conv", "cf_unet_conv_tc", "cf_unet_tc_error", "cf_unet_flip", "cf_unet_wgrad",
            "cf_unet_relu_grad", "cf_unet_loss", "cf_unet_pool", "cf_unet_pool_bwd", "cf_unet_upsample",
            "cf_unet_upsample_bwd", "cf_unet_concat", "cf_unet_split", "cf_unet_pack", "cf_unet_unpack"]


def _check(rc):
    if rc != CF_OK:
        msg = _lib.cf_last_error().decode()
        raise CapfilmError(f"{STATUS_NAMES.get(rc, rc)}: {msg}")


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def lattice_step_static(src_ptr, dst_ptr, nx, ny, nz, wall=1, tau=(1.0, 1.0), G=3.6,
                        stream_ptr=None):
    """One capsule-free lattice step on caller-owned device buffers (integer
    device addresses), with the library's fixed scratch: no allocation."""
    L = load_library()
    t = np.ascontiguousarray(tau, np.float64)
    _check(L.cf_lattice_step_static(C.c_void_p(src_ptr), C.c_void_p(dst_ptr), nx, ny, nz, wall,
                                    _ptr(t), G, C.c_void_p(stream_ptr) if stream_ptr else None))


def meniscus_fit(r, zeta, rmin=0.0, rmax=np.inf):
    """(Q, q, rms, samples) of zeta = Q K_0(q r) fitted over rmin <= r <= rmax
    (cf_meniscus_fit)."""
    L = load_library()
    r = np.ascontiguousarray(r, np.float64)
    z = np.ascontiguousarray(zeta, np.float64)
    out = np.zeros(4)
    _check(L.cf_meniscus_fit(_ptr(r), _ptr(z), len(r), float(rmin), float(min(rmax, 1e300)), _ptr(out)))
    return float(out[0]), float(out[1]), float(out[2]), int(out[3])


def capillary_force(q, gamma, Q1, Q2, L_):
    """-2 pi q gamma Q1 Q2 K_1(q L) (cf_capillary_force)."""
    L = load_library()
    F = np.zeros(1)
    _check(L.cf_capillary_force(float(q), float(gamma), float(Q1), float(Q2), float(L_), _ptr(F)))
    return float(F[0])


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, exposed as C callbacks."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(size, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), self.device, stream))
            except Exception:
                return None

        def _free(ptr, stream, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)
        self.struct = Allocator(self._alloc, self._free, None)


class Simulation:
    """One lattice with its capsules, stepped on the GPU by the CUDA library."""

    def __init__(self, nx, ny, nz, wall=1, tau=(1.0, 1.0), G=3.6, rep_dz=10.0, xi=1.5,
                 delta0=1.5, stream=None, use_torch_allocator=True, precision=FP32, flags=0):
        L = load_library()
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self._alloc = None
        alloc_ptr = None
        stream_handle = None
        self._stream = None
        if use_torch_allocator:
            import torch
            dev = torch.cuda.current_device()
            self._alloc = _TorchAllocator(dev)
            alloc_ptr = C.pointer(self._alloc.struct)
            s = stream if stream is not None else torch.cuda.current_stream()
            if s.cuda_stream == 0:
                # the library runs on a stream of its own; make it a torch
                # stream so that callers can order work and events after it
                s = torch.cuda.Stream()
            stream_handle = s.cuda_stream
            self._stream = s
        elif stream is not None:
            stream_handle = stream.cuda_stream
            self._stream = stream
        desc = LatticeDesc(nx, ny, nz, wall, (C.c_double * 2)(*tau), G, rep_dz, xi, delta0,
                           precision, alloc_ptr, stream_handle, int(flags))
        self._desc = desc
        h = C.c_void_p()
        _check(L.cf_create(C.byref(desc), C.byref(h)))
        self._h = h
        self.nv = []

    @classmethod
    def from_workload(cls, wl, set_film=True, **kw):
        kw.setdefault("flags", getattr(wl, "flags", 0))
        s = cls(wl.nx, wl.ny, wl.nz, wall=wl.wall, tau=wl.tau, G=wl.G, rep_dz=wl.rep_dz, **kw)
        if wl.capsules:
            meshes = [cap.mesh() for cap in wl.capsules]
            s.add_capsules([(X, F, cap.kS, cap.C, cap.kB, cap.kV, cap.mass, cap.mode, getattr(cap, "wet", 0.0))
                            for (X, F), cap in zip(meshes, wl.capsules)])
        if set_film:
            from .inputs import RHO_MAJ, RHO_MIN, RHO_MIX
            s.set_film(wl.h_top, RHO_MAJ, RHO_MIN, RHO_MIX, wl.jitter())
        if wl.dry_dm > 0.0:
            s.remove_mass(wl.dry_dm)
        return s

    def close(self):
        if getattr(self, "_h", None):
            _lib.cf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_capsules(self, specs):
        """Many capsules at once (cf_add_capsules): specs of (X, F, kS, C,
        kB, kV, mass, mode, wet); returns their ids."""
        keep, descs = [], (CapsuleDesc * len(specs))()
        for k, (X, F, kS, C_, kB, kV, mass, mode, wet) in enumerate(specs):
            X = np.ascontiguousarray(X, np.float64)
            F = np.ascontiguousarray(F, np.int32)
            keep.append((X, F))  # alive until the call returns
            descs[k] = CapsuleDesc(X.shape[0], F.shape[0], _ptr(X), F.ctypes.data_as(C.POINTER(C.c_int)),
                                   kS, C_, kB, kV, mass, mode, float(wet))
        ids = (C.c_int * len(specs))()
        _check(_lib.cf_add_capsules(self._h, descs, len(specs), ids))
        for X, _ in keep:
            self.nv.append(X.shape[0])
        return list(ids)

    def add_capsule(self, X, F, kS, C_, kB, kV, mass, mode, wet=0.0):
        X = np.ascontiguousarray(X, np.float64)
        F = np.ascontiguousarray(F, np.int32)
        d = CapsuleDesc(X.shape[0], F.shape[0], _ptr(X), F.ctypes.data_as(C.POINTER(C.c_int)),
                        kS, C_, kB, kV, mass, mode, float(wet))
        cid = C.c_int()
        _check(_lib.cf_add_capsule(self._h, C.byref(d), C.byref(cid)))
        self.nv.append(X.shape[0])
        return cid.value

    def set_capsule_mode(self, cid, mode):
        _check(_lib.cf_set_capsule_mode(self._h, cid, mode))

    def set_film(self, h_top, rho_maj, rho_min, rho_mix, jit=None):
        j = None if jit is None else np.ascontiguousarray(jit, np.float64).reshape(-1)
        _check(_lib.cf_set_film(self._h, h_top, rho_maj, rho_min, rho_mix, _ptr(j)))

    def step(self, n=1):
        _check(_lib.cf_step(self._h, int(n)))

    def set_densities(self, rhoA, rhoB):
        """Initial state at rest from density fields [nz][ny][nx] (cf_set_densities)."""
        a = np.ascontiguousarray(rhoA, dtype=np.float64).reshape(-1)
        b = np.ascontiguousarray(rhoB, dtype=np.float64).reshape(-1)
        assert a.size == self.N and b.size == self.N
        _check(_lib.cf_set_densities(self._h, _ptr(a), _ptr(b)))

    def remove_mass(self, dmA):
        """Drying: turn dmA of component A into B each step, 0 turns it off
        (cf_remove_mass)."""
        _check(_lib.cf_remove_mass(self._h, float(dmA)))

    @property
    def stream(self):
        """The torch stream every call of this simulation is enqueued on (None
        when the library created its own stream)."""
        return self._stream

    def sync(self):
        _check(_lib.cf_sync(self._h))

    def time_phases(self, n):
        """Mean device ms per step of (lattice passes, membrane, cut links, bounce
        records) over n steps."""
        ms = np.zeros(4)
        _check(_lib.cf_time_phases(self._h, int(n), _ptr(ms)))
        return ms

    def launches(self):
        n = C.c_longlong()
        _check(_lib.cf_launch_count(self._h, C.byref(n)))
        return n.value

    def warm_features(self, h_top, kS, x, mask=None):
        """Network inputs into device tensor x [4][N] and the fluid mask [N] (cf_warm_features)."""
        _check(_lib.cf_warm_features(self._h, float(h_top), float(kS), _dptr(x), _dptr(mask)))

    def warm_apply(self, h_top, rho_maj, rho_min, rho_mix, d):
        """State from predicted corrections d (device [2][N]) (cf_warm_apply)."""
        _check(_lib.cf_warm_apply(self._h, float(h_top), rho_maj, rho_min, rho_mix, _dptr(d)))

    def warm_target(self, h_top, rho_maj, rho_min, rho_mix, t):
        """Training target of the current state into device tensor t [2][N] (cf_warm_target)."""
        _check(_lib.cf_warm_target(self._h, float(h_top), rho_maj, rho_min, rho_mix, _dptr(t)))

    def field_check(self):
        """(all finite, smallest density, largest |u|, mean |rho - rho at the previous check|)
        of the last step's fields (cf_field_check)."""
        out = np.zeros(4)
        _check(_lib.cf_field_check(self._h, _ptr(out)))
        return out

    def save(self, path):
        """Checkpoint the state between two steps to a file (cf_save)."""
        _check(_lib.cf_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Restore a checkpoint into this simulation, set up like the saved one (cf_load)."""
        _check(_lib.cf_load(self._h, os.fsencode(path)))

    def meniscus_height(self, cid):
        """Largest rise zeta of capsule cid's meniscus profile (cf_meniscus_height)."""
        z = C.c_double()
        _check(_lib.cf_meniscus_height(self._h, int(cid), C.byref(z)))
        return z.value

    def run(self, steps, every, log=None):
        """Step `steps` times and read out every `every` steps: one record per
        readout (steps done in this call, MLUPS over the interval including the
        readout's synchronisation, total masses, per-capsule coupling forces,
        meniscus heights), appended as a JSON line to `log` (a path)
        when given.  Returns the records."""
        import json
        import time
        recs = []
        done = 0
        while done < steps:
            k = min(every, steps - done)
            t0 = time.perf_counter()
            self.step(k)
            self.sync()
            dt = time.perf_counter() - t0
            done += k
            forces = [self.capsule_force(c)[0].tolist() for c in range(len(self.nv))]
            zs = [self.meniscus_height(c) for c in range(len(self.nv))]
            rec = dict(step=done, mlups=self.N * k / dt / 1e6,
                       mass=self.total_mass().tolist(), force=forces, Z=zs)
            recs.append(rec)
            if log is not None:
                with open(log, "a") as f:
                    f.write(json.dumps(rec) + "\n")
        return recs

    def warmstart(self, model, h_top, kS, jitter=None, window=25, u_limit=0.1, grow=1.5, fallback=True):
        """The library's warm start (cf_warmstart): returns (kept, judging steps)."""
        from .inputs import RHO_MAJ, RHO_MIN, RHO_MIX
        pol = WarmPolicy(int(window), float(u_limit), float(grow), int(bool(fallback)))
        j = None if jitter is None else np.ascontiguousarray(jitter, np.float64).reshape(-1)
        used, steps = C.c_int(), C.c_longlong()
        _check(_lib.cf_warmstart(self._h, model._h, C.byref(pol), float(h_top), RHO_MAJ, RHO_MIN, RHO_MIX,
                                 float(kS), _ptr(j), C.byref(used), C.byref(steps)))
        return bool(used.value), int(steps.value)

    def capsule_force(self, cid):
        F = np.zeros(3); T = np.zeros(3)
        _check(_lib.cf_capsule_force(self._h, cid, _ptr(F), _ptr(T)))
        return F, T

    def lateral_force(self, a, b):
        F = np.zeros(1)
        _check(_lib.cf_lateral_force(self._h, a, b, _ptr(F)))
        return float(F[0])

    def capsule_state(self, cid):
        X = np.zeros((self.nv[cid], 3)); A = np.zeros(1); V = np.zeros(1)
        _check(_lib.cf_capsule_state(self._h, cid, _ptr(X), _ptr(A), _ptr(V)))
        return dict(X=X, area=float(A[0]), volume=float(V[0]))

    def fields(self):
        rho = np.zeros((2, self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        n = C.c_size_t(self.N)
        _check(_lib.cf_fields(self._h, _ptr(rho), _ptr(u), C.byref(n)))
        return rho, u

    def populations(self):
        f = np.zeros((2, 19, self.nz, self.ny, self.nx), np.float32)
        _check(_lib.cf_populations(self._h, _ptr(f, _fp)))
        return f

    def total_mass(self):
        m = np.zeros(2)
        _check(_lib.cf_total_mass(self._h, _ptr(m)))
        return m

    def meniscus_field(self):
        h = np.zeros((self.ny, self.nx))
        _check(_lib.cf_meniscus_field(self._h, _ptr(h)))
        return h

    def meniscus_profile(self, cid, dr=1.0):
        """(r, zeta, Z) of capsule cid's meniscus, sampled every dr (cf_meniscus_profile)."""
        n = C.c_size_t(0)
        _lib.cf_meniscus_profile(self._h, cid, float(dr), None, None, C.byref(n), None)
        r = np.zeros(n.value); z = np.zeros(n.value); Z = np.zeros(1)
        _check(_lib.cf_meniscus_profile(self._h, cid, float(dr), _ptr(r), _ptr(z), C.byref(n), _ptr(Z)))
        return r, z, float(Z[0])

    def cuts(self):
        mask = np.zeros((self.nz, self.ny, self.nx), np.uint32)
        tri = np.zeros((self.nz, self.ny, self.nx, 18), np.int32)
        ins = np.zeros((self.nz, self.ny, self.nx), np.uint8)
        _check(_lib.cf_cuts(self._h, mask.ctypes.data_as(C.POINTER(C.c_uint32)),
                            tri.ctypes.data_as(C.POINTER(C.c_int)),
                            ins.ctypes.data_as(C.POINTER(C.c_uint8))))
        return mask, tri, ins

    def cut_mask(self):
        """Cut bits per node [nz][ny][nx] (bit k-1: link to x + e_k cut) alone."""
        mask = np.zeros((self.nz, self.ny, self.nx), np.uint32)
        _check(_lib.cf_cuts(self._h, mask.ctypes.data_as(C.POINTER(C.c_uint32)), None, None))
        return mask


class Model:
    """The trained U-net loaded into the library (cf_model_load)."""

    def __init__(self, path):
        L = load_library()
        h = C.c_void_p()
        _check(L.cf_model_load(os.fsencode(path), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.cf_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many simulations stepped together (cf_batch): one persistent launch per
    lattice pass over all of them, their membrane phases as parallel branches.
    The simulations stay usable for readouts; close the batch before them."""

    def __init__(self, sims):
        L = load_library()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        h = C.c_void_p()
        _check(L.cf_batch_create(arr, len(self.sims), C.byref(h)))
        self._h = h

    def step(self, n):
        _check(_lib.cf_batch_step(self._h, int(n)))

    def time(self, n):
        """Device time (ms) of n steps."""
        ms = C.c_double()
        _check(_lib.cf_batch_time(self._h, int(n), C.byref(ms)))
        return ms.value

    def time_phases(self, n):
        """Mean device ms per step of (lattice passes, phase before them, phase
        after them) over n steps (cf_batch_time_phases)."""
        ms = np.zeros(3)
        _check(_lib.cf_batch_time_phases(self._h, int(n), _ptr(ms)))
        return ms

    def set_config(self, tile, zchunk):
        _check(_lib.cf_batch_set_config(self._h, int(tile), int(zchunk)))

    def set_groups(self, groups):
        """Pipeline groups of the batch (cf_batch_set_groups)."""
        _check(_lib.cf_batch_set_groups(self._h, int(groups)))

    def config(self):
        t, tx, ty, zc, g = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(_lib.cf_batch_config(self._h, C.byref(t), C.byref(tx), C.byref(ty), C.byref(zc), C.byref(g)))
        return dict(tile=t.value, tile_x=tx.value, tile_y=ty.value, zchunk=zc.value, groups=g.value)

    def autotune(self, steps=6):
        """Time the launch shapes and pipeline groups for `steps` steps each
        (real steps) and keep the fastest; returns the chosen configuration
        and its ms per step."""
        t, zc, g, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(_lib.cf_batch_autotune(self._h, int(steps), C.byref(t), C.byref(zc), C.byref(g), C.byref(ms)))
        d = self.config()
        d["ms_per_step"] = ms.value
        return d

    def launches(self):
        n = C.c_longlong()
        _check(_lib.cf_batch_launch_count(self._h, C.byref(n)))
        return n.value

    def lateral_forces(self, a=0, b=1):
        """Lateral force between capsules a and b of every simulation (cf_batch_lateral_forces)."""
        F = np.zeros(len(self.sims))
        _check(_lib.cf_batch_lateral_forces(self._h, int(a), int(b), _ptr(F)))
        return F

    def close(self):
        if getattr(self, "_h", None):
            _lib.cf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

