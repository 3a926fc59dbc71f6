"""FP64 CPU oracle of the explicit PDN impact step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the product package.  The
arithmetic lives in ``pdn_oracle.c`` (plain C, double precision, loops in the
order of the paper's Algorithms 1, 2, 4 and 5); this module only builds it,
loads it and marshals arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdn_oracle.c")
_LIB = os.path.join(_HERE, "libpdn_oracle.so")
_lock = threading.Lock()
_lib = None

NH = 7  # history fields per Gauss point


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction so that results do
    not depend on the host ISA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Material(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "rho", "E1", "E2", "E3", "nu12", "nu13", "nu23", "G12", "G13", "G23",
        "XT", "XC", "YT", "YC", "SL", "alpha0_deg",
        "GXT", "GXC", "GYT", "GYC", "GSL", "Sp", "Kp",
        "GIc", "GIIc", "tauI", "tauII", "eta", "KI", "spread")] + [("seed", C.c_uint64)]


class Options(C.Structure):
    _fields_ = [("damage_on", C.c_int32), ("plasticity_on", C.c_int32),
                ("max_release_iters", C.c_int32), ("n_threads", C.c_int32),
                ("phi", C.c_double), ("dt", C.c_double), ("dt_safety", C.c_double),
                ("gravity", C.c_double * 3)]


def material(d: dict) -> Material:
    m = Material()
    for name, _ in Material._fields_:
        setattr(m, name, int(d[name]) if name == "seed" else float(d[name]))
    return m


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.c_int64] * 4 + [dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int8), dp, C.c_int32, C.POINTER(C.c_uint8),
                                     C.POINTER(C.c_int32), C.POINTER(Material), C.POINTER(Options),
                                     C.c_int64]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_impactor.argtypes = [C.c_void_p, C.c_double, C.c_double, dp, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int64]
            L.orc_step.restype = C.c_int
            L.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp]
            L.orc_set_state.argtypes = [C.c_void_p, dp, dp]
            L.orc_install_state.argtypes = [C.c_void_p, dp, dp, dp, C.POINTER(C.c_uint8), dp, C.c_int64]
            L.orc_get_impactor.argtypes = [C.c_void_p, dp]
            L.orc_get_info.argtypes = [C.c_void_p, dp]
            L.orc_get_mass.argtypes = [C.c_void_p, dp]
            L.orc_get_active.argtypes = [C.c_void_p, C.POINTER(C.c_uint8), dp]
            L.orc_get_force_history.argtypes = [C.c_void_p, dp, C.c_int64]
            L.orc_get_force_history.restype = C.c_int64
            L.orc_get_history.argtypes = [C.c_void_p, dp, dp]
            L.orc_set_history.argtypes = [C.c_void_p, dp, dp]
            L.orc_get_strength_factors.argtypes = [C.c_void_p, dp]
            L.orc_get_lc.argtypes = [C.c_void_p, dp]
            L.orc_energies.argtypes = [C.c_void_p, dp]
            L.orc_internal_force.argtypes = [C.c_void_p, dp]
            L.orc_cdm_point.argtypes = [C.POINTER(Material), C.c_double, dp, dp, dp, dp, dp,
                                        C.c_int, C.c_int]
            L.orc_czm_point.argtypes = [C.POINTER(Material), dp, C.c_double, dp, dp]
            L.orc_hex8_force.argtypes = [C.POINTER(Material), C.c_double, C.c_double, dp, dp, dp,
                                         dp, dp, dp, C.c_int, C.c_int]
            L.orc_hex8_force.restype = C.c_double
            L.orc_coh8_force.argtypes = [C.POINTER(Material), dp, dp, dp, dp, dp]
            L.orc_hex8_volume.argtypes = [dp]
            L.orc_hex8_volume.restype = C.c_double
            L.orc_stiffness.argtypes = [C.POINTER(Material), dp]
            L.orc_strength_factor.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_double]
            L.orc_strength_factor.restype = C.c_double
            L.orc_damage_of_history.argtypes = [C.POINTER(Material), C.c_double, dp, dp, dp]
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# Point and element level functions (numpy in, numpy out).

def cdm_point(mat: dict, lc: float, eps, hist_in=None, sf=(1.0, 1.0, 1.0),
              damage_on=True, plasticity_on=True):
    """Algorithm 4 at one material point: ply-axis engineering strain
    [11,22,33,12,13,23] -> (stress, history)."""
    L = lib()
    m = material(mat)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    h = np.array([1, 1, 1, 1, 0, 0, 0], dtype=np.float64) if hist_in is None else \
        np.ascontiguousarray(hist_in, dtype=np.float64)
    s = np.ascontiguousarray(sf, dtype=np.float64)
    ho = np.zeros(NH)
    sig = np.zeros(6)
    L.orc_cdm_point(C.byref(m), lc, _p(s, C.c_double), _p(e, C.c_double), _p(h, C.c_double),
                    _p(ho, C.c_double), _p(sig, C.c_double), int(damage_on), int(plasticity_on))
    return sig, ho


def czm_point(mat: dict, delta, rD: float = 0.0):
    """Algorithm 5 at one interface point: local jump -> (traction, rD)."""
    L = lib()
    m = material(mat)
    dl = np.ascontiguousarray(delta, dtype=np.float64)
    tau = np.zeros(3)
    ro = np.zeros(1)
    L.orc_czm_point(C.byref(m), _p(dl, C.c_double), float(rD), _p(ro, C.c_double),
                    _p(tau, C.c_double))
    return tau, float(ro[0])


def hex8_force(mat: dict, X, u, angle_deg=0.0, lc=1.0, hist_in=None, sf=(1.0, 1.0, 1.0),
               damage_on=False, plasticity_on=False):
    """Internal force [8,3] of one hex8 (total Lagrangian, 2x2x2 Gauss);
    returns (f, hist_out [8,7], strain energy)."""
    L = lib()
    m = material(mat)
    Xa = np.ascontiguousarray(X, dtype=np.float64).reshape(8, 3)
    ua = np.ascontiguousarray(u, dtype=np.float64).reshape(8, 3)
    if hist_in is None:
        hist_in = np.tile(np.array([1, 1, 1, 1, 0, 0, 0], dtype=np.float64), (8, 1))
    hi = np.ascontiguousarray(hist_in, dtype=np.float64).reshape(8, NH)
    ho = np.zeros((8, NH))
    f = np.zeros((8, 3))
    s = np.ascontiguousarray(sf, dtype=np.float64)
    en = L.orc_hex8_force(C.byref(m), float(angle_deg), float(lc), _p(s, C.c_double),
                          _p(Xa, C.c_double), _p(ua, C.c_double), _p(hi, C.c_double),
                          _p(ho, C.c_double), _p(f, C.c_double), int(damage_on), int(plasticity_on))
    return f, ho, en


def coh8_force(mat: dict, X, u, rD_in=None):
    L = lib()
    m = material(mat)
    Xa = np.ascontiguousarray(X, dtype=np.float64).reshape(8, 3)
    ua = np.ascontiguousarray(u, dtype=np.float64).reshape(8, 3)
    ri = np.zeros(4) if rD_in is None else np.ascontiguousarray(rD_in, dtype=np.float64)
    ro = np.zeros(4)
    f = np.zeros((8, 3))
    L.orc_coh8_force(C.byref(m), _p(Xa, C.c_double), _p(ua, C.c_double), _p(ri, C.c_double),
                     _p(ro, C.c_double), _p(f, C.c_double))
    return f, ro


def hex8_volume(X) -> float:
    Xa = np.ascontiguousarray(X, dtype=np.float64).reshape(8, 3)
    return lib().orc_hex8_volume(_p(Xa, C.c_double))


def stiffness(mat: dict) -> np.ndarray:
    Cm = np.zeros((6, 6))
    m = material(mat)
    lib().orc_stiffness(C.byref(m), _p(Cm, C.c_double))
    return Cm


def strength_factor(seed: int, elem: int, k: int, spread: float) -> float:
    return lib().orc_strength_factor(seed, elem, k, spread)


def damage_of_history(mat: dict, lc: float, sf, h):
    m = material(mat)
    s = np.ascontiguousarray(sf, dtype=np.float64)
    ha = np.ascontiguousarray(h, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_damage_of_history(C.byref(m), lc, _p(s, C.c_double), _p(ha, C.c_double),
                                _p(out, C.c_double))
    return out


# ---------------------------------------------------------------------------
# Whole-model driver.

class Model:
    """The oracle solver for one plate and one striker."""

    def __init__(self, plate, mat: dict, damage_on=False, plasticity_on=False, phi=1.0,
                 dt=0.0, dt_safety=0.5, gravity=(0.0, 0.0, 0.0), max_release_iters=8,
                 n_threads=0, history_cap=1 << 20):
        L = lib()
        self.plate = plate
        self._keep = []
        X = np.ascontiguousarray(plate.X, dtype=np.float64)
        hexc = np.ascontiguousarray(plate.hex, dtype=np.int32)
        coh = np.ascontiguousarray(plate.coh, dtype=np.int32).reshape(-1, 8)
        ply = np.ascontiguousarray(plate.ply_of_hex, dtype=np.int8)
        ang = np.ascontiguousarray(plate.ply_angle_deg, dtype=np.float64)
        fixed = np.ascontiguousarray(plate.fixed, dtype=np.uint8)
        surf = np.ascontiguousarray(plate.surf, dtype=np.int32)
        self._mat = material(mat)
        o = Options()
        o.damage_on, o.plasticity_on = int(damage_on), int(plasticity_on)
        o.max_release_iters, o.n_threads = int(max_release_iters), int(n_threads)
        o.phi, o.dt, o.dt_safety = float(phi), float(dt), float(dt_safety)
        for i in range(3):
            o.gravity[i] = float(gravity[i])
        self._opt = o
        self.nn, self.nh, self.nc, self.ns = plate.n_nodes, plate.n_hex, plate.n_coh, plate.n_surf
        self.h = L.orc_create(self.nn, self.nh, self.nc, self.ns, _p(X, C.c_double),
                              _p(hexc, C.c_int32), _p(coh, C.c_int32), _p(ply, C.c_int8),
                              _p(ang, C.c_double), len(ang), _p(fixed, C.c_uint8),
                              _p(surf, C.c_int32), C.byref(self._mat), C.byref(o), history_cap)
        self.history_cap = history_cap

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_impactor(self, radius, mass, centre, velocity):
        c = np.array(centre, dtype=np.float64)
        w = np.array(velocity, dtype=np.float64)
        lib().orc_set_impactor(self.h, float(radius), float(mass), _p(c, C.c_double), _p(w, C.c_double))

    def step(self, n: int) -> int:
        return lib().orc_step(self.h, int(n))

    def state(self):
        d = np.zeros((3, self.nn))
        v = np.zeros((3, self.nn))
        a = np.zeros((3, self.nn))
        lib().orc_get_state(self.h, _p(d, C.c_double), _p(v, C.c_double), _p(a, C.c_double))
        return d, v, a

    def set_state(self, d, v):
        d = np.ascontiguousarray(d, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        lib().orc_set_state(self.h, _p(d, C.c_double), _p(v, C.c_double))

    def install_state(self, d, v, a, active, imp, step: int):
        """Continue from another solver's committed state of step ``step``:
        d, v, a [3, nn]; active [ns] contact set; imp = dict(centre,
        velocity, force, time) of the striker.  Nothing is recomputed."""
        d = np.ascontiguousarray(d, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        a = np.ascontiguousarray(a, dtype=np.float64)
        act = np.ascontiguousarray(active, dtype=np.uint8)
        im = np.concatenate([np.asarray(imp["centre"], dtype=np.float64), np.asarray(imp["velocity"], dtype=np.float64),
                             np.asarray(imp["force"], dtype=np.float64), [float(imp["time"])]])
        lib().orc_install_state(self.h, _p(d, C.c_double), _p(v, C.c_double), _p(a, C.c_double),
                                _p(act, C.c_uint8), _p(im, C.c_double), int(step))

    def impactor(self):
        out = np.zeros(10)
        lib().orc_get_impactor(self.h, _p(out, C.c_double))
        return dict(centre=out[0:3].copy(), velocity=out[3:6].copy(), force=out[6:9].copy(),
                    time=out[9])

    def info(self):
        out = np.zeros(8)
        lib().orc_get_info(self.h, _p(out, C.c_double))
        return dict(dt=out[0], dt_bulk=out[1], dt_coh=out[2], step=int(out[3]),
                    n_active=int(out[4]), n_repeats=int(out[5]), f_peak=out[6], status=int(out[7]))

    def mass(self):
        m = np.zeros(self.nn)
        lib().orc_get_mass(self.h, _p(m, C.c_double))
        return m

    def active(self):
        act = np.zeros(self.ns, dtype=np.uint8)
        lam = np.zeros(self.ns)
        lib().orc_get_active(self.h, _p(act, C.c_uint8), _p(lam, C.c_double))
        return act, lam

    def force_history(self):
        out = np.zeros(self.history_cap)
        n = lib().orc_get_force_history(self.h, _p(out, C.c_double), self.history_cap)
        return out[:n].copy()

    def history(self):
        h = np.zeros((self.nh, 8, NH))
        r = np.zeros((max(self.nc, 1), 4))
        lib().orc_get_history(self.h, _p(h, C.c_double), _p(r, C.c_double))
        return h, r[: self.nc]

    def set_history(self, hist, rD):
        h = np.ascontiguousarray(hist, dtype=np.float64)
        r = np.ascontiguousarray(rD, dtype=np.float64) if self.nc else np.zeros(4)
        lib().orc_set_history(self.h, _p(h, C.c_double), _p(r, C.c_double))

    def strength_factors(self):
        s = np.zeros((self.nh, 3))
        lib().orc_get_strength_factors(self.h, _p(s, C.c_double))
        return s

    def lc(self):
        s = np.zeros(self.nh)
        lib().orc_get_lc(self.h, _p(s, C.c_double))
        return s

    def energies(self):
        out = np.zeros(4)
        lib().orc_energies(self.h, _p(out, C.c_double))
        return dict(ke_plate=out[0], ke_striker=out[1], strain=out[2], interface=out[3])

    def internal_force(self):
        f = np.zeros((3, self.nn))
        lib().orc_internal_force(self.h, _p(f, C.c_double))
        return f


def model_for(workload, **kw) -> Model:
    """Oracle model of a pdn_inputs.Workload, striker installed."""
    M = Model(workload.plate, workload.material, damage_on=workload.damage_on,
              plasticity_on=workload.plasticity_on, phi=workload.phi,
              dt_safety=workload.dt_safety, gravity=workload.gravity, **kw)
    M.set_impactor(*workload.impactor())
    return M
