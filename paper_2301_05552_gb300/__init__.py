"""GB300-native explicit impact step with partial Dirichlet-Neumann contact.

Python binding of the C ABI declared in ``include/pdn.h`` (ctypes).  The
functions here carry the same names as the C entry points and only marshal
arguments: every step of the method runs in the CUDA kernels of
``lib/libpdn.so``.  There is no CPU fallback; a missing or unloadable library
raises.

Method: Guillamet et al., "Application of the partial Dirichlet-Neumann
contact algorithm to simulate low-velocity impact events on composite
structures", Composites Part A (2022), arXiv 2301.05552.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import _build

__all__ = [
    "PdnError", "lib", "build",
    "pdn_init_mesh", "pdn_set_impactor", "pdn_step", "pdn_contact_force", "pdn_damage_field",
    "pdn_get_state", "pdn_set_state", "pdn_get_contact", "pdn_get_history", "pdn_get_acceleration",
    "pdn_energies", "pdn_internal_force", "pdn_get_info", "pdn_profile_kernels", "pdn_destroy", "pdn_last_error", "Solver",
    "pdn_batch_init", "pdn_batch_plate", "pdn_batch_step", "pdn_batch_get_info",
    "pdn_batch_test_barrier_timeout", "pdn_batch_destroy", "pdn_batch_last_error",
    "pdn_sur_create", "pdn_sur_generate", "pdn_sur_train", "pdn_sur_forward", "pdn_sur_exact",
    "pdn_sur_gradient", "pdn_sur_get_params", "pdn_sur_set_params", "pdn_set_surrogate",
    "pdn_sur_destroy", "pdn_sur_last_error", "pdn_sur_get_data", "SUR_PARAMS", "SUR_SCALING",
    "pdn_mesh_multiply", "pdn_refined_get_info", "pdn_refined_get", "pdn_init_refined", "pdn_refined_destroy",
    "pdn_refined_last_error", "Refined",
    "PDN_FP64", "PDN_FP32_FORCE", "FIELDS", "KERNELS",
]

PDN_FP64 = 0
PDN_FP32_FORCE = 1
FIELDS = {"D1": 0, "D2": 1, "D6": 2, "DCOH": 3, "PLASTIC": 4}
KERNELS = ["contact", "hex", "coh", "gather", "tail"]
ERRORS = {-1: "PDN_E_ARG", -2: "PDN_E_CUDA", -3: "PDN_E_OOM", -4: "PDN_E_NONFINITE",
          -5: "PDN_E_RELEASE_LIMIT", -6: "PDN_E_TIMEOUT", -7: "PDN_E_UNSTABLE", -8: "PDN_E_STATE"}
EXPORTS = ["pdn_init_mesh", "pdn_set_impactor", "pdn_step", "pdn_contact_force", "pdn_damage_field",
           "pdn_get_state", "pdn_set_state", "pdn_get_contact", "pdn_get_history", "pdn_get_acceleration",
           "pdn_energies", "pdn_internal_force", "pdn_get_info", "pdn_profile_kernels", "pdn_destroy", "pdn_last_error", "pdn_internal_force_noalloc",
           "pdn_batch_init", "pdn_batch_plate", "pdn_batch_step", "pdn_batch_get_info",
           "pdn_batch_test_barrier_timeout", "pdn_batch_destroy", "pdn_batch_last_error",
           "pdn_sur_create", "pdn_sur_generate", "pdn_sur_train", "pdn_sur_forward", "pdn_sur_exact",
           "pdn_sur_gradient", "pdn_sur_get_params", "pdn_sur_set_params", "pdn_set_surrogate",
           "pdn_sur_destroy", "pdn_sur_last_error", "pdn_sur_get_data",
           "pdn_mesh_multiply", "pdn_refined_get_info", "pdn_refined_get", "pdn_init_refined",
           "pdn_refined_destroy", "pdn_refined_last_error"]
SUR_PARAMS = 9674
SUR_SCALING = 60


class PdnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_hex", C.c_int64), ("n_coh", C.c_int64), ("n_surf", C.c_int64),
                ("X", C.POINTER(C.c_double)), ("hex", C.POINTER(C.c_int32)), ("coh", C.POINTER(C.c_int32)),
                ("ply_of_hex", C.POINTER(C.c_int8)), ("ply_angle_deg", C.POINTER(C.c_double)),
                ("n_plies", C.c_int32), ("fixed", C.POINTER(C.c_uint8)), ("surf", C.POINTER(C.c_int32))]


class RefinedInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_hex", C.c_int64), ("n_coh", C.c_int64), ("n_surf", C.c_int64),
                ("n_edges", C.c_int64), ("n_faces", C.c_int64), ("levels", C.c_int32), ("pad", C.c_int32),
                ("device_ms", C.c_double)]


MATERIAL_KEYS = ("rho", "E1", "E2", "E3", "nu12", "nu13", "nu23", "G12", "G13", "G23",
                 "XT", "XC", "YT", "YC", "SL", "alpha0_deg", "GXT", "GXC", "GYT", "GYC", "GSL",
                 "Sp", "Kp", "GIc", "GIIc", "tauI", "tauII", "eta", "KI", "spread")


class Material(C.Structure):
    _fields_ = [(k, C.c_double) for k in MATERIAL_KEYS] + [("seed", C.c_uint64)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("damage_on", C.c_int32), ("plasticity_on", C.c_int32),
                ("max_release_iters", C.c_int32), ("phi", C.c_double), ("dt", C.c_double),
                ("dt_safety", C.c_double), ("gravity", C.c_double * 3), ("history_cap", C.c_int64),
                ("stream", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("dt", C.c_double), ("dt_bulk", C.c_double), ("dt_coh", C.c_double), ("time", C.c_double),
                ("f_peak", C.c_double), ("step", C.c_int64), ("n_active", C.c_int64), ("n_repeats", C.c_int64),
                ("n_nodes", C.c_int64), ("n_hex", C.c_int64), ("n_coh", C.c_int64), ("n_surf", C.c_int64),
                ("device_bytes", C.c_int64), ("status", C.c_int32), ("precision", C.c_int32),
                ("hex_variant", C.c_int32), ("sweep", C.c_int32), ("coh_pairs", C.c_int32),
                ("reserved", C.c_int32), ("tune_ms", C.c_double * 12)]


class BatchInfo(C.Structure):
    _fields_ = [("n_plates", C.c_int32), ("precision", C.c_int32), ("status", C.c_int32), ("tuned", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("tile_items", C.c_int32), ("reg_variant", C.c_int32),
                ("grid", C.c_int32), ("graph", C.c_int32), ("n_candidates", C.c_int32),
                ("n_tiles", C.c_int64 * 4), ("launches", C.c_int64), ("passes", C.c_int64),
                ("tune_ms", C.c_double * 16), ("tune_bps", C.c_int32 * 16), ("tune_tile", C.c_int32 * 16),
                ("tune_var", C.c_int32 * 16), ("dataflow", C.c_int32), ("pad", C.c_int32),
                ("tune_flow", C.c_int32 * 16)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    return _build.build(force=force)


def lib():
    """Load lib/libpdn.so (building it first if it is missing or stale); with
    the environment variable PDN_CHECKED=1, lib/libpdn_check.so, the build with
    the device bounds checks (PDN_CHECK)."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("PDN_CHECKED") == "1"
            path = _build.LIB_CHECK if checked else _build.LIB
            if _build._stale(path):
                _build.build(check=checked)
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run paper_2301_05552_gb300.build()")
            L = C.CDLL(path)
            vp, dp = C.c_void_p, C.POINTER(C.c_double)
            L.pdn_init_mesh.argtypes = [C.POINTER(vp), C.POINTER(MeshDesc), C.POINTER(Material), C.POINTER(Options)]
            L.pdn_set_impactor.argtypes = [vp, C.c_double, C.c_double, dp, dp]
            L.pdn_step.argtypes = [vp, C.c_int64]
            L.pdn_contact_force.argtypes = [vp, dp, dp, dp, C.c_int64]
            L.pdn_contact_force.restype = C.c_int64
            L.pdn_damage_field.argtypes = [vp, C.c_int32, C.c_void_p, C.c_int64, C.c_int32]
            L.pdn_get_state.argtypes = [vp, dp, dp, dp]
            L.pdn_set_state.argtypes = [vp, dp, dp]
            L.pdn_get_contact.argtypes = [vp, C.POINTER(C.c_uint8), dp]
            L.pdn_get_history.argtypes = [vp, vp, vp]
            L.pdn_get_acceleration.argtypes = [vp, dp]
            L.pdn_energies.argtypes = [vp, dp]
            L.pdn_internal_force.argtypes = [vp, dp]
            L.pdn_get_info.argtypes = [vp, C.POINTER(Info)]
            L.pdn_profile_kernels.argtypes = [vp, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_int64)]
            L.pdn_destroy.argtypes = [vp]
            L.pdn_destroy.restype = None
            L.pdn_last_error.argtypes = [vp]
            L.pdn_last_error.restype = C.c_char_p
            L.pdn_internal_force_noalloc.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp,
                                                     C.POINTER(Material), dp, C.c_int32, C.c_int32, C.c_int32,
                                                     C.c_int32, vp, vp]
            L.pdn_internal_force_noalloc.restype = C.c_int
            L.pdn_batch_init.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(MeshDesc), C.POINTER(Material),
                                         C.POINTER(Options)]
            L.pdn_batch_plate.argtypes = [vp, C.c_int32]
            L.pdn_batch_plate.restype = vp
            L.pdn_batch_step.argtypes = [vp, C.c_int64]
            L.pdn_batch_get_info.argtypes = [vp, C.POINTER(BatchInfo)]
            L.pdn_batch_test_barrier_timeout.argtypes = [vp, C.c_double]
            L.pdn_batch_destroy.argtypes = [vp]
            L.pdn_batch_destroy.restype = None
            L.pdn_batch_last_error.argtypes = [vp]
            L.pdn_batch_last_error.restype = C.c_char_p
            for name in ("pdn_batch_init", "pdn_batch_step", "pdn_batch_get_info", "pdn_batch_test_barrier_timeout"):
                getattr(L, name).restype = C.c_int
            fp = C.POINTER(C.c_float)
            L.pdn_sur_create.argtypes = [C.POINTER(vp), C.POINTER(Material), C.c_double, C.c_uint64, vp]
            L.pdn_sur_generate.argtypes = [vp, C.c_int64, C.c_int32, C.c_double, C.c_double, C.c_double,
                                           C.c_uint64, C.POINTER(C.c_int64)]
            L.pdn_sur_train.argtypes = [vp, C.c_int64, C.c_int32, C.c_double, C.c_uint64, dp]
            L.pdn_sur_get_data.argtypes = [vp, C.c_int64, C.c_int64, fp, fp]
            L.pdn_sur_get_data.restype = C.c_int
            L.pdn_sur_forward.argtypes = [vp, vp, vp, C.c_int64, C.c_int32]
            L.pdn_sur_exact.argtypes = [vp, vp, vp, C.c_int64, C.c_int32]
            L.pdn_sur_gradient.argtypes = [vp, fp, fp, C.c_int64, fp, dp]
            L.pdn_sur_get_params.argtypes = [vp, fp, fp]
            L.pdn_sur_set_params.argtypes = [vp, fp, fp]
            L.pdn_set_surrogate.argtypes = [vp, vp, C.c_double]
            L.pdn_sur_destroy.argtypes = [vp]
            L.pdn_sur_destroy.restype = None
            L.pdn_sur_last_error.argtypes = [vp]
            L.pdn_sur_last_error.restype = C.c_char_p
            for name in ("pdn_sur_create", "pdn_sur_generate", "pdn_sur_train", "pdn_sur_forward", "pdn_sur_exact",
                         "pdn_sur_gradient", "pdn_sur_get_params", "pdn_sur_set_params", "pdn_set_surrogate"):
                getattr(L, name).restype = C.c_int
            L.pdn_mesh_multiply.argtypes = [C.POINTER(vp), C.POINTER(MeshDesc), C.c_int32, vp]
            L.pdn_refined_get_info.argtypes = [vp, C.POINTER(RefinedInfo)]
            L.pdn_refined_get.argtypes = [vp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int8),
                                          C.POINTER(C.c_uint8), C.POINTER(C.c_int32)]
            L.pdn_init_refined.argtypes = [C.POINTER(vp), vp, C.POINTER(Material), C.POINTER(Options)]
            L.pdn_refined_destroy.argtypes = [vp]
            L.pdn_refined_destroy.restype = None
            L.pdn_refined_last_error.argtypes = [vp]
            L.pdn_refined_last_error.restype = C.c_char_p
            for name in ("pdn_mesh_multiply", "pdn_refined_get_info", "pdn_refined_get", "pdn_init_refined"):
                getattr(L, name).restype = C.c_int
            for name in ("pdn_set_impactor", "pdn_step", "pdn_damage_field", "pdn_get_state", "pdn_set_state",
                         "pdn_get_contact", "pdn_get_history", "pdn_get_acceleration", "pdn_energies",
                         "pdn_internal_force",
                         "pdn_get_info", "pdn_profile_kernels", "pdn_init_mesh"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _check(ctx, rc):
    if rc < 0:
        msg = lib().pdn_last_error(ctx.handle if ctx is not None else None)
        raise PdnError(int(rc), (msg or b"").decode())
    return rc


class Context:
    """A pdn_ctx handle (one plate + one striker on the current device)."""

    def __init__(self, handle, n_nodes, n_hex, n_coh, n_surf, stream, owner=None):
        self.handle = handle
        self.n_nodes, self.n_hex, self.n_coh, self.n_surf = n_nodes, n_hex, n_coh, n_surf
        self.stream = stream
        self.owner = owner  # a Batch owns the contexts of its plates

    def close(self):
        if self.handle and self.owner is None:
            lib().pdn_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
    except Exception:
        pass
    return None


def _mesh_desc(plate):
    """MeshDesc of a plate (any object with the fields of pdn_inputs.Plate:
    X [3,n], hex [n,8], coh [m,8], ply_of_hex, ply_angle_deg, fixed, surf)
    and the arrays it points into (keep them alive while it is used)."""
    keep = dict(
        X=np.ascontiguousarray(plate.X, dtype=np.float64),
        hex=np.ascontiguousarray(plate.hex, dtype=np.int32).reshape(-1, 8),
        coh=np.ascontiguousarray(plate.coh, dtype=np.int32).reshape(-1, 8),
        ply=np.ascontiguousarray(plate.ply_of_hex, dtype=np.int8),
        ang=np.ascontiguousarray(plate.ply_angle_deg, dtype=np.float64),
        fixed=np.ascontiguousarray(plate.fixed, dtype=np.uint8),
        surf=np.ascontiguousarray(plate.surf, dtype=np.int32),
    )
    m = MeshDesc()
    m.n_nodes = keep["X"].shape[1]
    m.n_hex = keep["hex"].shape[0]
    m.n_coh = keep["coh"].shape[0]
    m.n_surf = keep["surf"].shape[0]
    m.X = _ptr(keep["X"], C.c_double)
    m.hex = _ptr(keep["hex"], C.c_int32)
    m.coh = _ptr(keep["coh"], C.c_int32) if m.n_coh else None
    m.ply_of_hex = _ptr(keep["ply"], C.c_int8)
    m.ply_angle_deg = _ptr(keep["ang"], C.c_double)
    m.n_plies = keep["ang"].shape[0]
    m.fixed = _ptr(keep["fixed"], C.c_uint8)
    m.surf = _ptr(keep["surf"], C.c_int32) if m.n_surf else None
    return m, keep


def _material(material: dict) -> Material:
    mat = Material()
    for k in MATERIAL_KEYS:
        setattr(mat, k, float(material[k]))
    mat.seed = int(material["seed"])
    return mat


def _options(precision, damage_on, plasticity_on, max_release_iters, phi, dt, dt_safety, gravity,
             history_cap, stream) -> Options:
    o = Options()
    o.precision, o.damage_on, o.plasticity_on = int(precision), int(damage_on), int(plasticity_on)
    o.max_release_iters, o.phi, o.dt, o.dt_safety = int(max_release_iters), float(phi), float(dt), float(dt_safety)
    for i in range(3):
        o.gravity[i] = float(gravity[i])
    o.history_cap = int(history_cap)
    o.stream = stream
    return o


def pdn_init_mesh(plate, material: dict, precision: int = PDN_FP32_FORCE, damage_on: bool = True,
                  plasticity_on: bool = True, max_release_iters: int = 8, phi: float = 1.0, dt: float = 0.0,
                  dt_safety: float = 0.5, gravity=(0.0, 0.0, 0.0), history_cap: int = 1 << 20,
                  stream: Optional[int] = None) -> Context:
    """pdn_init_mesh: ``plate`` is any object with the fields of
    pdn_inputs.Plate (X [3,n], hex [n,8], coh [m,8], ply_of_hex, ply_angle_deg,
    fixed, surf)."""
    L = lib()
    m, keep = _mesh_desc(plate)
    mat = _material(material)
    if stream is None:
        stream = _current_stream()
    o = _options(precision, damage_on, plasticity_on, max_release_iters, phi, dt, dt_safety, gravity,
                 history_cap, stream)
    h = C.c_void_p()
    rc = L.pdn_init_mesh(C.byref(h), C.byref(m), C.byref(mat), C.byref(o))
    if rc < 0:
        raise PdnError(rc, (L.pdn_last_error(None) or b"").decode())
    return Context(h, m.n_nodes, m.n_hex, m.n_coh, m.n_surf, stream)


def pdn_set_impactor(ctx: Context, radius: float, mass: float, centre, velocity):
    c = np.ascontiguousarray(centre, dtype=np.float64)
    w = np.ascontiguousarray(velocity, dtype=np.float64)
    _check(ctx, lib().pdn_set_impactor(ctx.handle, float(radius), float(mass), _ptr(c, C.c_double),
                                       _ptr(w, C.c_double)))


def pdn_step(ctx: Context, nsteps: int):
    _check(ctx, lib().pdn_step(ctx.handle, int(nsteps)))


def pdn_contact_force(ctx: Context, cap: Optional[int] = None):
    """(f_now[3], f_peak, history[:n]) of the striker-plate contact force."""
    L = lib()
    f = np.zeros(3)
    pk = np.zeros(1)
    n_avail = _check(ctx, L.pdn_contact_force(ctx.handle, _ptr(f, C.c_double), _ptr(pk, C.c_double), None, 0))
    cap = n_avail if cap is None else min(cap, n_avail)
    hist = np.zeros(max(cap, 1))
    n = _check(ctx, L.pdn_contact_force(ctx.handle, None, None, _ptr(hist, C.c_double), cap)) if cap > 0 else 0
    return f, float(pk[0]), hist[:n]


def pdn_damage_field(ctx: Context, which, out=None):
    """Damage field as a float32 numpy array (host) or into a CUDA torch
    tensor ``out`` (device pointer path)."""
    w = FIELDS[which] if isinstance(which, str) else int(which)
    n = ctx.n_coh if w == FIELDS["DCOH"] else ctx.n_hex
    if out is not None and hasattr(out, "data_ptr"):
        _check(ctx, lib().pdn_damage_field(ctx.handle, w, C.c_void_p(out.data_ptr()), n, 1))
        return out
    a = np.zeros(n, dtype=np.float32)
    _check(ctx, lib().pdn_damage_field(ctx.handle, w, a.ctypes.data_as(C.c_void_p), n, 0))
    return a


def pdn_get_state(ctx: Context):
    d = np.zeros((3, ctx.n_nodes))
    v = np.zeros((3, ctx.n_nodes))
    imp = np.zeros(10)
    _check(ctx, lib().pdn_get_state(ctx.handle, _ptr(d, C.c_double), _ptr(v, C.c_double), _ptr(imp, C.c_double)))
    return d, v, dict(centre=imp[0:3].copy(), velocity=imp[3:6].copy(), force=imp[6:9].copy(), time=imp[9])


def pdn_set_state(ctx: Context, d, v):
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(3, ctx.n_nodes)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(3, ctx.n_nodes)
    _check(ctx, lib().pdn_set_state(ctx.handle, _ptr(d, C.c_double), _ptr(v, C.c_double)))


def pdn_get_contact(ctx: Context):
    act = np.zeros(max(ctx.n_surf, 1), dtype=np.uint8)
    lam = np.zeros(max(ctx.n_surf, 1))
    _check(ctx, lib().pdn_get_contact(ctx.handle, _ptr(act, C.c_uint8), _ptr(lam, C.c_double)))
    return act[: ctx.n_surf], lam[: ctx.n_surf]


def pdn_get_history(ctx: Context):
    """Committed history: (hist [7, 8, n_hex], rD [4, n_coh]) in the element
    precision (float32 for PDN_FP32_FORCE, float64 for PDN_FP64)."""
    dt = np.float64 if pdn_get_info(ctx)["precision"] == PDN_FP64 else np.float32
    h = np.zeros((7, 8, max(ctx.n_hex, 1)), dtype=dt)
    r = np.zeros((4, max(ctx.n_coh, 1)), dtype=dt)
    _check(ctx, lib().pdn_get_history(ctx.handle, h.ctypes.data_as(C.c_void_p), r.ctypes.data_as(C.c_void_p)))
    return h[:, :, : ctx.n_hex], r[:, : ctx.n_coh]


def pdn_get_acceleration(ctx: Context):
    """Acceleration of the committed step, [3, n_nodes] float64."""
    a = np.zeros((3, ctx.n_nodes))
    _check(ctx, lib().pdn_get_acceleration(ctx.handle, _ptr(a, C.c_double)))
    return a


def pdn_energies(ctx: Context) -> dict:
    """Energy ledger of the committed state (include/pdn.h), with the
    dissipated energy derived from it."""
    out = np.zeros(6)
    _check(ctx, lib().pdn_energies(ctx.handle, _ptr(out, C.c_double)))
    d = dict(ke_plate=out[0], ke_striker=out[1], stored_hex=out[2], stored_interface=out[3],
             work_gravity=out[4], e0_striker=out[5])
    d["dissipated"] = out[5] + out[4] - (out[0] + out[1] + out[2] + out[3])
    return d


def pdn_internal_force(ctx: Context):
    f = np.zeros((3, ctx.n_nodes))
    _check(ctx, lib().pdn_internal_force(ctx.handle, _ptr(f, C.c_double)))
    return f


def pdn_get_info(ctx: Context) -> dict:
    info = Info()
    _check(ctx, lib().pdn_get_info(ctx.handle, C.byref(info)))
    out = {k: getattr(info, k) for k, _ in Info._fields_ if k != "reserved"}
    out["tune_ms"] = list(info.tune_ms)
    return out


def pdn_profile_kernels(ctx: Context, nsteps: int):
    ms = (C.c_float * 5)()
    cnt = (C.c_int64 * 5)()
    _check(ctx, lib().pdn_profile_kernels(ctx.handle, int(nsteps), ms, cnt))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}


def pdn_destroy(ctx: Context):
    ctx.close()


def pdn_last_error(ctx: Optional[Context]) -> str:
    return (lib().pdn_last_error(ctx.handle if ctx is not None else None) or b"").decode()


def pdn_internal_force_noalloc(n_nodes: int, n_hex: int, hex_dev, ply_dev, X_dev, d_dev, history_dev,
                               row_dev, col_dev, material: dict, ply_angle_deg, precision: int,
                               damage_on: bool, plasticity_on: bool, f_out_dev, stream: Optional[int] = None):
    """pdn_internal_force_noalloc: every array argument is a CUDA tensor (or
    None for history); the library allocates nothing (its scratch is a fixed
    device array), see include/pdn.h."""
    mat = Material()
    for k in MATERIAL_KEYS:
        setattr(mat, k, float(material[k]))
    mat.seed = int(material["seed"])
    ang = np.ascontiguousarray(ply_angle_deg, dtype=np.float64)
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    if stream is None:
        stream = _current_stream()
    rc = lib().pdn_internal_force_noalloc(int(n_nodes), int(n_hex), ptr(hex_dev), ptr(ply_dev), ptr(X_dev),
                                          ptr(d_dev), ptr(history_dev), ptr(row_dev), ptr(col_dev), C.byref(mat),
                                          _ptr(ang, C.c_double), len(ang), int(precision), int(damage_on),
                                          int(plasticity_on), ptr(f_out_dev), stream)
    if rc < 0:
        raise PdnError(rc, (lib().pdn_last_error(None) or b"").decode())


class Batch:
    """A pdn_batch handle: plates[p] are its (non-owning) plate contexts."""

    def __init__(self, handle, plates, stream):
        self.handle = handle
        self.plates = plates
        self.stream = stream

    def close(self):
        if self.handle:
            for c in self.plates:
                c.handle = None
            lib().pdn_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(b, rc):
    if rc < 0:
        msg = lib().pdn_batch_last_error(b.handle if b is not None else None)
        raise PdnError(int(rc), (msg or b"").decode())
    return rc


def pdn_batch_init(plates, materials, precision: int = PDN_FP32_FORCE, damage_on: bool = True,
                   plasticity_on: bool = True, max_release_iters: int = 8, phi: float = 1.0, dt: float = 0.0,
                   dt_safety: float = 0.5, gravity=(0.0, 0.0, 0.0), history_cap: int = 1 << 20,
                   stream: Optional[int] = None) -> Batch:
    """pdn_batch_init: one plate per entry of ``plates`` (pdn_inputs.Plate
    fields) with material dict ``materials[p]``; the options are common."""
    L = lib()
    n = len(plates)
    descs = (MeshDesc * n)()
    mats = (Material * n)()
    keep = []
    for p, (pl, mt) in enumerate(zip(plates, materials)):
        m, k = _mesh_desc(pl)
        keep.append(k)
        descs[p] = m
        mats[p] = _material(mt)
    if stream is None:
        stream = _current_stream()
    o = _options(precision, damage_on, plasticity_on, max_release_iters, phi, dt, dt_safety, gravity,
                 history_cap, stream)
    h = C.c_void_p()
    rc = L.pdn_batch_init(C.byref(h), n, descs, mats, C.byref(o))
    if rc < 0:
        raise PdnError(rc, (L.pdn_batch_last_error(None) or b"").decode())
    b = Batch(h, [], stream)
    for p in range(n):
        ph = L.pdn_batch_plate(h, p)
        d = descs[p]
        b.plates.append(Context(C.c_void_p(ph), d.n_nodes, d.n_hex, d.n_coh, d.n_surf, stream, owner=b))
    return b


def pdn_batch_plate(b: Batch, p: int) -> Context:
    return b.plates[p]


def pdn_batch_step(b: Batch, nsteps: int):
    _bcheck(b, lib().pdn_batch_step(b.handle, int(nsteps)))


def pdn_batch_get_info(b: Batch) -> dict:
    info = BatchInfo()
    _bcheck(b, lib().pdn_batch_get_info(b.handle, C.byref(info)))
    out = {k: getattr(info, k) for k, _ in BatchInfo._fields_}
    nc = info.n_candidates
    out["n_tiles"] = list(info.n_tiles)
    out["candidates"] = [dict(ms=info.tune_ms[k], blocks_per_sm=info.tune_bps[k], tile_items=info.tune_tile[k],
                              reg_variant=info.tune_var[k], dataflow=info.tune_flow[k]) for k in range(nc)]
    for k in ("tune_ms", "tune_bps", "tune_tile", "tune_var", "tune_flow", "pad"):
        out.pop(k)
    return out


def pdn_batch_test_barrier_timeout(b: Batch, timeout_ms: float) -> int:
    """Returns the status code (PDN_E_TIMEOUT = -6 when the bounded wait ran
    out as designed); does not raise for that code."""
    rc = lib().pdn_batch_test_barrier_timeout(b.handle, float(timeout_ms))
    if rc < 0 and rc != -6:
        _bcheck(b, rc)
    return int(rc)


def pdn_batch_destroy(b: Batch):
    b.close()


def pdn_batch_last_error(b: Optional[Batch]) -> str:
    return (lib().pdn_batch_last_error(b.handle if b is not None else None) or b"").decode()


class Surrogate:
    """A pdn_surrogate handle (learned intralaminar law)."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().pdn_sur_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scheck(s, rc):
    if rc < 0:
        msg = lib().pdn_sur_last_error(s.handle if s is not None else None)
        raise PdnError(int(rc), (msg or b"").decode())
    return rc


def pdn_sur_create(material: dict, lc: float, seed: int = 0, stream: Optional[int] = None) -> Surrogate:
    L = lib()
    h = C.c_void_p()
    if stream is None:
        stream = _current_stream()
    rc = L.pdn_sur_create(C.byref(h), C.byref(_material(material)), float(lc), int(seed), stream)
    if rc < 0:
        raise PdnError(rc, (L.pdn_sur_last_error(None) or b"").decode())
    return Surrogate(h)


def pdn_sur_generate(s: Surrogate, n_paths: int, steps_per_path: int = 8, strain_max: float = 0.01,
                     cyclic_fraction: float = 0.4, onset_ratio: float = 0.9, seed: int = 0) -> int:
    n = C.c_int64()
    _scheck(s, lib().pdn_sur_generate(s.handle, int(n_paths), int(steps_per_path), float(strain_max),
                                      float(cyclic_fraction), float(onset_ratio), int(seed), C.byref(n)))
    return int(n.value)


def pdn_sur_get_data(s: Surrogate, offset: int, n: int):
    """Points [offset, offset+n) of the training set: (x[n,10], y[n,10]) raw."""
    x = np.zeros((int(n), 10), dtype=np.float32)
    y = np.zeros((int(n), 10), dtype=np.float32)
    _scheck(s, lib().pdn_sur_get_data(s.handle, int(offset), int(n), _ptr(x, C.c_float), _ptr(y, C.c_float)))
    return x, y


def pdn_sur_train(s: Surrogate, iters: int, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    loss = np.zeros(max(int(iters), 1))
    _scheck(s, lib().pdn_sur_train(s.handle, int(iters), int(batch), float(lr), int(seed), _ptr(loss, C.c_double)))
    return loss[: int(iters)]


def _points(s, fn, x):
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 10)
    y = np.zeros_like(x)
    _scheck(s, fn(s.handle, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p), x.shape[0], 0))
    return y


def pdn_sur_forward(s: Surrogate, x):
    """Network output for raw points x[n, 10] (strain 6, thresholds 4)."""
    return _points(s, lib().pdn_sur_forward, x)


def pdn_sur_exact(s: Surrogate, x):
    """Exact damage law (FP64 on the GPU) for the same points."""
    return _points(s, lib().pdn_sur_exact, x)


def pdn_sur_gradient(s: Surrogate, xn, tn):
    xn = np.ascontiguousarray(xn, dtype=np.float32).reshape(-1, 10)
    tn = np.ascontiguousarray(tn, dtype=np.float32).reshape(-1, 10)
    g = np.zeros(SUR_PARAMS, dtype=np.float32)
    loss = np.zeros(1)
    _scheck(s, lib().pdn_sur_gradient(s.handle, _ptr(xn, C.c_float), _ptr(tn, C.c_float), xn.shape[0],
                                      _ptr(g, C.c_float), _ptr(loss, C.c_double)))
    return g, float(loss[0])


def pdn_sur_get_params(s: Surrogate):
    p = np.zeros(SUR_PARAMS, dtype=np.float32)
    sc = np.zeros(SUR_SCALING, dtype=np.float32)
    _scheck(s, lib().pdn_sur_get_params(s.handle, _ptr(p, C.c_float), _ptr(sc, C.c_float)))
    return p, sc


def pdn_sur_set_params(s: Surrogate, params=None, scaling=None):
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    sc = None if scaling is None else np.ascontiguousarray(scaling, dtype=np.float32)
    _scheck(s, lib().pdn_sur_set_params(s.handle, _ptr(p, C.c_float), _ptr(sc, C.c_float)))


def pdn_set_surrogate(ctx: Context, s: Optional[Surrogate], onset_ratio: float = 0.9):
    _check(ctx, lib().pdn_set_surrogate(ctx.handle, s.handle if s is not None else None, float(onset_ratio)))


def pdn_sur_destroy(s: Surrogate):
    s.close()


def pdn_sur_last_error(s: Optional[Surrogate]) -> str:
    return (lib().pdn_sur_last_error(s.handle if s is not None else None) or b"").decode()


class Solver:
    """Convenience wrapper: one context for a pdn_inputs.Workload."""

    def __init__(self, workload, precision=None, **kw):
        prec = precision if precision is not None else (PDN_FP64 if workload.fp64 else PDN_FP32_FORCE)
        self.workload = workload
        self.ctx = pdn_init_mesh(workload.plate, workload.material, precision=prec,
                                 damage_on=workload.damage_on, plasticity_on=workload.plasticity_on,
                                 phi=workload.phi, dt_safety=workload.dt_safety, gravity=workload.gravity, **kw)
        pdn_set_impactor(self.ctx, *workload.impactor())

    def step(self, n):
        pdn_step(self.ctx, n)

    def info(self):
        return pdn_get_info(self.ctx)

    def state(self):
        return pdn_get_state(self.ctx)

    def force_history(self):
        return pdn_contact_force(self.ctx)[2]

    def close(self):
        self.ctx.close()


# ---------------------------------------------------------------------------
# Mesh multiplication on the device (include/pdn_mmu.h)

class Refined:
    """A pdn_refined handle: a divided mesh held in device memory."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().pdn_refined_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pdn_refined_last_error(r: Optional[Refined]) -> str:
    return (lib().pdn_refined_last_error(r.handle if r is not None else None) or b"").decode()


def _rcheck(r, rc):
    if rc < 0:
        raise PdnError(int(rc), pdn_refined_last_error(r))
    return rc


def pdn_mesh_multiply(plate, ndivi: int, stream: Optional[int] = None) -> Refined:
    """pdn_mesh_multiply: divide ``plate`` (pdn_inputs.Plate fields) ndivi
    times on the current device."""
    L = lib()
    m, keep = _mesh_desc(plate)
    if stream is None:
        stream = _current_stream()
    h = C.c_void_p()
    rc = L.pdn_mesh_multiply(C.byref(h), C.byref(m), int(ndivi), stream)
    if rc < 0:
        raise PdnError(rc, (L.pdn_refined_last_error(None) or b"").decode())
    return Refined(h)


def pdn_refined_get_info(r: Refined) -> dict:
    info = RefinedInfo()
    _rcheck(r, lib().pdn_refined_get_info(r.handle, C.byref(info)))
    return {k: getattr(info, k) for k, _ in RefinedInfo._fields_ if k != "pad"}


def pdn_refined_get(r: Refined) -> dict:
    """The divided mesh on the host: X [3, n], hex [n_hex, 8], coh [n_coh, 8],
    ply_of_hex, fixed, surf."""
    i = pdn_refined_get_info(r)
    X = np.empty((3, i["n_nodes"]), np.float64)
    hx = np.empty((i["n_hex"], 8), np.int32)
    ch = np.empty((i["n_coh"], 8), np.int32)
    ply = np.empty(i["n_hex"], np.int8)
    fx = np.empty(i["n_nodes"], np.uint8)
    sf = np.empty(i["n_surf"], np.int32)
    _rcheck(r, lib().pdn_refined_get(r.handle, _ptr(X, C.c_double), _ptr(hx, C.c_int32),
                                     _ptr(ch, C.c_int32) if ch.size else None, _ptr(ply, C.c_int8),
                                     _ptr(fx, C.c_uint8), _ptr(sf, C.c_int32) if sf.size else None))
    return dict(X=X, hex=hx, coh=ch, ply_of_hex=ply, fixed=fx, surf=sf)


def pdn_init_refined(r: Refined, material: dict, precision: int = PDN_FP32_FORCE, damage_on: bool = True,
                     plasticity_on: bool = True, max_release_iters: int = 8, phi: float = 1.0, dt: float = 0.0,
                     dt_safety: float = 0.5, gravity=(0.0, 0.0, 0.0), history_cap: int = 1 << 20,
                     stream: Optional[int] = None) -> Context:
    """pdn_init_refined: a solver context on the divided mesh."""
    L = lib()
    if stream is None:
        stream = _current_stream()
    o = _options(precision, damage_on, plasticity_on, max_release_iters, phi, dt, dt_safety, gravity,
                 history_cap, stream)
    mat = _material(material)
    h = C.c_void_p()
    rc = L.pdn_init_refined(C.byref(h), r.handle, C.byref(mat), C.byref(o))
    if rc < 0:
        raise PdnError(rc, (L.pdn_last_error(None) or b"").decode() or pdn_refined_last_error(r))
    i = pdn_refined_get_info(r)
    return Context(h, i["n_nodes"], i["n_hex"], i["n_coh"], i["n_surf"], stream)


def pdn_refined_destroy(r: Refined):
    r.close()
