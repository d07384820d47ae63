"""FP64 CPU oracle for the FDTD + CPML hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The CUDA library (``paper_2606_06910_gb300``) never imports, links or calls
this package, and this package never imports the library: the two share no
code.  The only module both sides use is ``paper_2606_06910_gb300.synth``,
which holds seeded input generators and none of the method's arithmetic.

Contents
--------
``oracle.oracle``   weights, CPML profiles, the time-stepping driver over the
                    C core, the explicit sparse-matrix second formulation,
                    the misfit gradient (adjoint) driver.
``oracle.mlp``      the learned-CPML network in NumPy FP64 (forward, backward,
                    Adam) and the (sigma, kappa, alpha) -> (b, a, 1/kappa) map.
``fdtd_oracle.c``   plain-loop FP64 time step and its transpose.

Parity status of every function is stated in its docstring; nothing here is
"parity unpinned" except where a docstring says so.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C core with gcc (plain IEEE FP64: no fast-math, no FMA
    contraction) and return the path of the shared library."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the oracle's C core."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.og_version.restype = ctypes.c_long
        if _lib.og_version() != 2:
            raise RuntimeError("oracle C core layout version mismatch")
    return _lib
