"""ctypes declarations of the C ABI in include/pic.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

PIC_OK = 0
STATUS_NAMES = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA", -4: "PIC_ECOURANT",
                -5: "PIC_EOVERFLOW", -6: "PIC_ENONFINITE", -7: "PIC_ETIMEOUT", -8: "PIC_EUNSUPPORTED",
                -9: "PIC_ENOTBUILT"}
PIC_FP64_PLAIN, PIC_FP32_CELLOFF = 0, 1
PIC_BC_PERIODIC, PIC_BC_CONDUCT_ABSORB, PIC_BC_AXIAL = 0, 5, 20
PIC_COORDS_CARTESIAN, PIC_COORDS_CYLINDRICAL = 0, 1
PIC_E1, PIC_E2, PIC_E3, PIC_B1, PIC_B2, PIC_B3, PIC_J1, PIC_J2, PIC_J3, PIC_RHO = range(10)
FIELD_NAMES = {"E1": 0, "E2": 1, "E3": 2, "B1": 3, "B2": 4, "B3": 5, "J1": 6, "J2": 7, "J3": 8, "RHO": 9}
MAX_SMOOTH = 8

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t)


class PicAllocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class PicGrid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int * 3), ("xmin", C.c_double * 3), ("dx", C.c_double * 3),
                ("dt", C.c_double), ("bc", (C.c_int * 2) * 3), ("e0", C.c_double * 3), ("b0", C.c_double * 3),
                ("smooth_level", C.c_int * 3), ("smooth_w", ((C.c_double * 3) * MAX_SMOOTH) * 3),
                ("rho_bg", C.c_double), ("init_e_gauss_x1", C.c_int), ("precision", C.c_int),
                ("tile", C.c_int * 3), ("slack", C.c_double), ("sort_period", C.c_int),
                ("ctas_per_sm", C.c_int), ("move_window", C.c_int), ("deposit", C.c_int),
                ("window_start", C.c_double), ("coords", C.c_int)]


class PicSpecies(C.Structure):
    _fields_ = [("rqm", C.c_double), ("ppc", C.c_int * 3), ("uth", C.c_double * 3), ("ufl", C.c_double * 3),
                ("density", C.c_double), ("seed", C.c_ulonglong), ("n_explicit", C.c_longlong),
                ("x0", C.POINTER(C.c_double)), ("u0", C.POINTER(C.c_double)), ("q_explicit", C.c_double),
                ("np_max", C.c_longlong), ("track_ids", C.c_int), ("prof_n", C.c_int * 3),
                ("prof_x", C.POINTER(C.c_double) * 3), ("prof_f", C.POINTER(C.c_double) * 3), ("den_min", C.c_double),
                ("w0", C.POINTER(C.c_double))]


class PicLaser(C.Structure):
    _fields_ = [("vosc", C.c_double), ("rkkp", C.c_double), ("w0", C.c_double), ("rise", C.c_double),
                ("fall", C.c_double), ("length", C.c_double), ("start", C.c_double), ("pol", C.c_double),
                ("phase", C.c_double), ("offset", C.c_double * 2), ("wavetype", C.c_int), ("focus_on", C.c_int),
                ("focus", C.c_double), ("antenna", C.c_int)]


class PicTuneChoice(C.Structure):
    _fields_ = [("tile", C.c_int * 3), ("ctas_per_sm", C.c_int), ("sort_period", C.c_int),
                ("ms_per_step", C.c_double)]


class PicDiag(C.Structure):
    _fields_ = [("step", C.c_longlong), ("time", C.c_double), ("field_energy", C.c_double),
                ("kinetic_energy", C.c_double), ("total_charge", C.c_double), ("gauss_resid_max", C.c_double),
                ("rho_abs_max", C.c_double), ("rho_particles_abs_max", C.c_double),
                ("n_particles", C.c_longlong), ("error_flags", C.c_int)]


# every symbol include/pic.h declares, with its ctypes prototype
_P = C.c_void_p
PROTOTYPES = {
    "pic_init": (C.c_int, [C.POINTER(PicGrid), C.POINTER(PicSpecies), C.c_int, C.POINTER(PicAllocator), _P,
                           C.POINTER(_P)]),
    "pic_step": (C.c_int, [_P, C.c_int]),
    "pic_fields": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.c_int]),
    "pic_set_field": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.c_int]),
    "pic_particles": (C.c_int, [_P, C.c_int, _P, _P, C.c_longlong, C.POINTER(C.c_longlong), C.c_int]),
    "pic_particle_ids": (C.c_int, [_P, C.c_int, _P, C.c_longlong, C.POINTER(C.c_longlong), C.c_int]),
    "pic_particle_weights": (C.c_int, [_P, C.c_int, _P, C.c_longlong, C.POINTER(C.c_longlong), C.c_int]),
    "pic_tile_counts": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong), C.c_longlong, C.POINTER(C.c_longlong)]),
    "pic_diag": (C.c_int, [_P, C.POINTER(PicDiag)]),
    "pic_timing_enable": (C.c_int, [_P, C.c_int]),
    "pic_timing_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int, C.c_int]),
    "pic_destroy": (C.c_int, [_P]),
    "pic_last_error": (C.c_char_p, []),
    "pic_bin_tiles": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_longlong, _P, _P, _P, _P,
                                C.POINTER(PicAllocator), _P]),
    "pic_bin_tiles_noalloc": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_longlong, _P, _P, _P, _P, _P]),
    "pic_batch_init": (C.c_int, [C.c_int, C.POINTER(PicGrid), C.POINTER(PicSpecies), C.c_int, C.POINTER(PicAllocator),
                                 _P, C.POINTER(_P)]),
    "pic_batch_step": (C.c_int, [_P, C.c_int]),
    "pic_batch_sim": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "pic_batch_info": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "pic_batch_destroy": (C.c_int, [_P]),
    "pic_checkpoint_save": (C.c_int, [_P, C.c_char_p]),
    "pic_checkpoint_load": (C.c_int, [C.c_char_p, C.POINTER(PicAllocator), _P, C.POINTER(_P)]),
    "pic_laser_add": (C.c_int, [_P, C.POINTER(PicLaser)]),
    "pic_info": (C.c_int, [_P, C.POINTER(PicGrid), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "pic_autotune": (C.c_int, [C.POINTER(PicGrid), C.POINTER(PicSpecies), C.c_int, C.POINTER(PicAllocator), _P, C.c_int,
                               C.c_int, C.POINTER(PicTuneChoice), C.POINTER(PicTuneChoice), C.c_int,
                               C.POINTER(C.c_int)]),
    "pic_batch_autotune": (C.c_int, [C.c_int, C.POINTER(PicGrid), C.POINTER(PicSpecies), C.c_int,
                                     C.POINTER(PicAllocator), _P, C.c_int, C.c_int, C.POINTER(PicTuneChoice),
                                     C.POINTER(PicTuneChoice), C.c_int, C.POINTER(C.c_int)]),
}
BIN_NOALLOC_SCRATCH_BYTES = 16 << 20

_lock = threading.Lock()
_lib = None


class PicError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpicgb.so; raises if it is missing and cannot be built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libpicgb.so is not built ({path}); run __graft_entry__.build()")
                _build.build()
            L = C.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code: int, where: str):
    if code != PIC_OK:
        raise PicError(code, where, load().pic_last_error().decode())
