"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/fdtd.h declares, validates descriptors
and sizes workspaces without touching CUDA, and honours the host-side fault
hook."""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_2606_06910_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def _desc(**kw):
    d = _lib.Desc()
    d.nx, d.ny, d.nz, d.nshots = kw.get("nx", 64), kw.get("ny", 64), kw.get("nz", 64), kw.get("nshots", 1)
    d.h, d.dt = kw.get("h", 10.0), kw.get("dt", 2.5e-3)
    for i, c in enumerate(kw.get("cells", (10,) * 6)):
        d.cpml_cells[i] = c
    d.storage = kw.get("storage", 0)
    d.tblock_k = kw.get("tblock_k", 1)
    d.nt_max = kw.get("nt_max", 200)
    d.nrec_max = kw.get("nrec_max", 16)
    d.checkpoint_every = kw.get("checkpoint_every", 0)
    d.cpml_grad = kw.get("cpml_grad", 0)
    d.stream = None
    return d


def test_exports_every_declared_function(lib):
    names = _lib.header_functions()
    assert len(names) >= 24
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib._SIGS), set(names) ^ set(_lib._SIGS)


def test_abi_version_and_status_strings(lib):
    assert lib.fdtd_abi_version() == 2
    for s in range(9):
        assert lib.fdtd_status_string(s)
    assert lib.fdtd_status_string(99) == b"unknown status"


def _bytes(lib, d):
    n = ctypes.c_size_t(0)
    st = lib.fdtd_workspace_bytes(ctypes.byref(d), ctypes.byref(n))
    return st, n.value


def test_workspace_bytes_accounts_for_fields(lib):
    st, n = _bytes(lib, _desc())
    assert st == _lib.OK
    nxp = 64
    fields = 8 * 64 * 64 * nxp * 4                 # p, v double-buffered
    assert n >= fields + 64 * 64 * nxp * 4        # + dt K table
    st16, n16 = _bytes(lib, _desc(storage=1))
    assert st16 == _lib.OK and n16 < n            # 16-bit storage halves the fields
    st2, n2 = _bytes(lib, _desc(nshots=3))
    assert st2 == _lib.OK and n2 > 2.5 * fields
    # checkpointing adds checkpoints, tape, adjoint fields
    st3, n3 = _bytes(lib, _desc(checkpoint_every=50))
    assert st3 == _lib.OK and n3 > n + 4 * 64 ** 3 * 4 * 4


def test_memory_model_matches_tab14():
    # Tab. 14: p + 3 v + 6 psi fields in FP32 over the grid padded by 2r = 8
    # cells per side: 10 * (N + 16)^3 * 4 bytes (paper's accounting).
    for N, gib in [(320, 1.41), (544, 6.54), (800, 20.24)]:
        assert abs(10 * (N + 16) ** 3 * 4 / 2 ** 30 - gib) < 0.006


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(h=0.0), dict(dt=-1.0), dict(cells=(40, 40, 0, 0, 0, 0)), dict(storage=7),
    dict(tblock_k=3), dict(tblock_k=0), dict(tblock_k=8), dict(nt_max=0), dict(nshots=0), dict(nshots=2000), dict(nrec_max=-1),
    dict(checkpoint_every=-2), dict(cpml_grad=1),
])
def test_invalid_descriptors_rejected(lib, bad):
    st, _ = _bytes(lib, _desc(**bad))
    assert st == _lib.EINVAL


def test_temporal_blocking_needs_no_extra_workspace(lib):
    # k = 2, 4 run in the two ping-pong sets that single steps use
    st1, b1 = _bytes(lib, _desc(tblock_k=1))
    for k in (2, 4):
        st, b = _bytes(lib, _desc(tblock_k=k))
        assert st == _lib.OK and b == b1


def test_adjoint_needs_fp32(lib):
    st, _ = _bytes(lib, _desc(storage=1, checkpoint_every=10))
    assert st == _lib.EUNSUPPORTED


def test_create_rejects_small_workspace_without_touching_cuda(lib):
    d = _desc()
    ctx = ctypes.c_void_p()
    assert lib.fdtd_create(ctypes.byref(d), None, 0, ctypes.byref(ctx)) == _lib.ENOMEM
    assert not ctx.value


def test_fault_hook_alloc():
    # host-side failure injection: FDTD_FAULT=alloc makes create fail before any CUDA call
    code = ("import ctypes, sys; sys.path.insert(0, %r);"
            "from paper_2606_06910_gb300 import _lib;"
            "from tests.test_abi_host import _desc;"
            "lib = _lib.load(); d = _desc(); ctx = ctypes.c_void_p();"
            "print(lib.fdtd_create(ctypes.byref(d), ctypes.c_void_p(256), 1 << 40, ctypes.byref(ctx)))"
            % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    env = dict(os.environ, FDTD_FAULT="alloc")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == str(_lib.ENOMEM)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.fdtd_step_n(None, 1) == _lib.EINVAL
    assert lib.fdtd_destroy(None) == _lib.EINVAL
    assert lib.fdtd_last_error(None) == b"context is NULL"
    # the setters of the step's forms check their context before anything else
    assert lib.fdtd_set_staggered(None, 1) == _lib.EINVAL
    assert lib.fdtd_set_cpml_local(None, None, 1e-8, 5.0, 0.05, 3) == _lib.EINVAL
    assert lib.fdtd_set_anisotropy(None, None) == _lib.EINVAL
    assert lib.fdtd_set_model(None, None, None) == _lib.EINVAL
    assert lib.fdtd_adjoint_step_n(None, 0, None, None, None) == _lib.EINVAL


def test_noalloc_limit_matches_header():
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "fdtd.h")).read()
    m = re.search(r"#define FDTD_NOALLOC_MISFIT_MAX (\d+)LL", hdr)
    assert m and int(m.group(1)) == _lib.NOALLOC_MISFIT_MAX


@pytest.mark.parametrize("L,q,R,kmax,af", [(6, 3, 1e-8, 5.0, 0.05), (20, 2, 1e-5, 1.0, 0.0), (1, 3, 1e-3, 3.0, 0.1)])
def test_cpml_grading_matches_oracle_profile(lib, L, q, R, kmax, af):
    # the library's per-cell (sigma, kappa, alpha) against the oracle's low
    # face, node j = cell j (host computation, no GPU)
    from oracle import oracle as O
    h, c = 10.0, 2000.0
    out = (ctypes.c_double * (3 * L))()
    assert lib.fdtd_cpml_grading(L, h, c, R, kmax, af, q, out) == _lib.OK
    ska = [[out[3 * j + k] for k in range(3)] for j in range(L)]
    prof = O.axis_profile(3 * L + 4, L, L, h, 1e-3, c, R, q, kmax, af)
    for j in range(L):
        for k, name in enumerate(("sigma", "kappa", "alpha")):
            assert abs(ska[j][k] - prof[name][j]) <= 1e-12 * max(1.0, abs(prof[name][j])), (j, name)
    assert lib.fdtd_cpml_grading(0, h, c, R, kmax, af, q, out) == _lib.EINVAL
    assert lib.fdtd_cpml_grading(L, h, c, 2.0, kmax, af, q, out) == _lib.EINVAL
    assert lib.fdtd_cpml_grading(L, h, c, R, kmax, af, q, None) == _lib.EINVAL


def test_null_context_calls_fail_cleanly(lib):
    assert lib.fdtd_set_divergence_check(None, 1, 0.0) == _lib.EINVAL
    assert lib.fdtd_set_time(None, 3) == _lib.EINVAL
    assert lib.fdtd_set_velocity_scale(None, 1.0) == _lib.EINVAL
    assert lib.fdtd_set_timing(None, 1) == _lib.EINVAL
    assert lib.fdtd_exchange(None, None, None, None) == _lib.EINVAL
