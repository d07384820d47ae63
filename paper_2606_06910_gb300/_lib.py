"""ctypes declaration of the C ABI in include/fdtd.h (argument marshalling only).

The library is built in-tree (``paper_2606_06910_gb300/_build/libfdtd.so``); a
missing or stale library is rebuilt with nvcc on first load.  There is no
fallback: if the library cannot be built or loaded, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

c_int, c_double, c_void_p, c_float, c_size_t = (ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.c_float, ctypes.c_size_t)

# fdtd_status
OK, EINVAL, ENOMEM, ECUDA, ESTATE, EUNSTABLE, EDIVERGED, ETIMEOUT, EUNSUPPORTED = range(9)
STATUS_NAMES = {0: "FDTD_OK", 1: "FDTD_EINVAL", 2: "FDTD_ENOMEM", 3: "FDTD_ECUDA", 4: "FDTD_ESTATE",
                5: "FDTD_EUNSTABLE", 6: "FDTD_EDIVERGED", 7: "FDTD_ETIMEOUT", 8: "FDTD_EUNSUPPORTED"}

# FDTD_NOALLOC_MISFIT_MAX: largest n of fdtd_misfit_noalloc
NOALLOC_MISFIT_MAX = 4096 * 65536

# fdtd_timing_class
TIMING_STEP, TIMING_ADJOINT = 0, 1

# fdtd_storage
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}

# fdtd_field
FIELDS = ["p", "vx", "vy", "vz", "psiv_x", "psiv_y", "psiv_z", "psip_x", "psip_y", "psip_z",
          "adj_p", "adj_vx", "adj_vy", "adj_vz", "adj_psiv_x", "adj_psiv_y", "adj_psiv_z",
          "adj_psip_x", "adj_psip_y", "adj_psip_z"]
FIELD_ID = {k: i for i, k in enumerate(FIELDS)}


class Desc(ctypes.Structure):
    """Mirror of fdtd_desc."""
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("nshots", c_int),
                ("h", c_double), ("dt", c_double), ("cpml_cells", c_int * 6),
                ("storage", c_int), ("tblock_k", c_int), ("nt_max", c_int), ("nrec_max", c_int),
                ("checkpoint_every", c_int), ("cpml_grad", c_int), ("cpml_local", c_int), ("stream", c_void_p)]


_SIGS = {
    "fdtd_abi_version": (c_int, []),
    "fdtd_status_string": (ctypes.c_char_p, [c_int]),
    "fdtd_workspace_bytes": (c_int, [ctypes.POINTER(Desc), ctypes.POINTER(c_size_t)]),
    "fdtd_create": (c_int, [ctypes.POINTER(Desc), c_void_p, c_size_t, ctypes.POINTER(c_void_p)]),
    "fdtd_destroy": (c_int, [c_void_p]),
    "fdtd_last_error": (ctypes.c_char_p, [c_void_p]),
    "fdtd_set_model": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fdtd_set_cpml": (c_int, [c_void_p, c_double, c_double, c_double, c_int, c_double]),
    "fdtd_set_cpml_ska": (c_int, [c_void_p, c_void_p]),
    "fdtd_set_anisotropy": (c_int, [c_void_p, c_void_p]),
    "fdtd_set_staggered": (c_int, [c_void_p, c_int]),
    "fdtd_set_cpml_local": (c_int, [c_void_p, c_void_p, c_double, c_double, c_double, c_int]),
    "fdtd_inject": (c_int, [c_void_p, ctypes.POINTER(c_int), c_void_p, c_int]),
    "fdtd_record": (c_int, [c_void_p, ctypes.POINTER(c_int), c_int, c_void_p]),
    "fdtd_step_n": (c_int, [c_void_p, c_int]),
    "fdtd_adjoint_step_n": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "fdtd_get_field": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "fdtd_set_field": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "fdtd_reset": (c_int, [c_void_p]),
    "fdtd_time": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "fdtd_sync": (c_int, [c_void_p]),
    "fdtd_set_time": (c_int, [c_void_p, c_int]),
    "fdtd_set_divergence_check": (c_int, [c_void_p, c_int, c_double]),
    "fdtd_energy": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "fdtd_misfit": (c_int, [c_void_p, c_void_p, c_int, c_void_p, ctypes.POINTER(c_double)]),
    "fdtd_misfit_noalloc": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_void_p,
                                    ctypes.POINTER(c_double), c_void_p]),
    "fdtd_set_velocity_scale": (c_int, [c_void_p, c_double]),
    "fdtd_exchange": (c_int, [c_void_p, c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "fdtd_set_timing": (c_int, [c_void_p, c_int]),
    "fdtd_timing": (c_int, [c_void_p, c_int, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "fdtd_cpml_grading": (c_int, [c_int, c_double, c_double, c_double, c_double, c_double, c_int, c_void_p]),
    "fdtd_mlp_fit_gradient": (c_int, [c_void_p, c_void_p, c_int, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "fdtd_cpml_ska_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fdtd_mlp_forward": (c_int, [c_void_p, c_void_p, c_int, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "fdtd_mlp_backward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_float, c_float,
                                  c_void_p, c_void_p]),
    "fdtd_adam_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_float, c_float,
                               c_float, c_float, c_void_p]),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libfdtd.so (building it first if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libfdtd.so not found at {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.fdtd_abi_version() != 2:
                raise RuntimeError("libfdtd ABI version mismatch")
            _lib = lib
        return _lib


def header_functions(path=None):
    """Names of the functions declared in include/fdtd.h."""
    path = path or os.path.join(_build.INCLUDE, "fdtd.h")
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", src)))


class FdtdError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
