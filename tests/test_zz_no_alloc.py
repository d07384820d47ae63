"""fdtd_misfit_noalloc, the data-misfit entry point for callers that cannot
allocate device memory (its scratch is a static device array), must give what
the context-based fdtd_misfit gives, call after call.

Kept in a file of its own that pytest collects last, so that a run stopping at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def test_noalloc_misfit_matches_context_misfit_twice():
    from paper_2606_06910_gb300.fdtd import Fdtd
    lib = _lib.load()
    shape, cells, h = (40, 36, 48), (6,) * 6, 10.0
    dt = 0.5 * h / 3000.0
    nt, nshots = 60, 2
    rec = synth.receiver_grid(shape, cells, 4, 5, 7)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_model(torch.full(shape, 3000.0, device="cuda"))
    sim.set_cpml(R=1e-6, c_ref=3000.0)
    wav = np.stack([synth.ricker(nt, dt, 20.0), synth.ricker(nt, dt, 25.0)]).astype(np.float32)
    sim.inject([[20, 18, 24], [15, 20, 30]], torch.from_numpy(wav).cuda())
    traces = sim.record(rec)
    sim.step(nt)
    sim.sync()
    rng = np.random.default_rng(0)
    dobs = torch.from_numpy((1e-3 * rng.standard_normal(tuple(traces.shape))).astype(np.float32)).cuda()
    ref_resid = torch.empty_like(traces)
    J_ref = sim.misfit(dobs, nt=nt, resid=ref_resid)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = traces.numel()
    for _ in range(2):
        resid = torch.full_like(traces, 7.0)
        out = ctypes.c_double(-1.0)
        st = lib.fdtd_misfit_noalloc(ctypes.c_void_p(traces.data_ptr()), ctypes.c_void_p(dobs.data_ptr()),
                                     ctypes.c_longlong(n), ctypes.c_void_p(resid.data_ptr()),
                                     ctypes.byref(out), stream)
        assert st == _lib.OK
        # FP64 sums of the same FP32 residuals in a different order
        assert abs(out.value - J_ref) <= 1e-12 * abs(J_ref), (out.value, J_ref)
        assert torch.equal(resid, ref_resid)


def test_noalloc_misfit_rejects_bad_sizes():
    lib = _lib.load()
    x = torch.zeros(8, device="cuda")
    out = ctypes.c_double(0.0)
    p = ctypes.c_void_p(x.data_ptr())
    for n in (0, -5, (1 << 28) + 1):
        assert lib.fdtd_misfit_noalloc(p, p, ctypes.c_longlong(n), None, ctypes.byref(out), None) == _lib.EINVAL
    assert lib.fdtd_misfit_noalloc(None, p, ctypes.c_longlong(8), None, ctypes.byref(out), None) == _lib.EINVAL


def _noalloc(lib, a, b, n, resid):
    out = ctypes.c_double(-1.0)
    st = lib.fdtd_misfit_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.c_longlong(n),
                                 ctypes.c_void_p(resid.data_ptr()) if resid is not None else None,
                                 ctypes.byref(out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out.value


def _fp64_half_sum_sq(a, b, chunk=1 << 26):
    """1/2 sum (a - b)^2 with the FP32 difference (the entry point's rounding)
    squared and summed in FP64, in chunks to bound the temporaries."""
    acc = 0.0
    for i in range(0, a.numel(), chunk):
        r = (a[i:i + chunk] - b[i:i + chunk]).double()
        acc += float((r * r).sum())
    return 0.5 * acc


@pytest.mark.parametrize("n", [3 * 65536 + 17, 65536, 65537])
def test_noalloc_misfit_several_partials(n):
    # more than one partial sum (the grid-stride kernel's blocks, then the
    # finishing block over them), with a ragged last block
    lib = _lib.load()
    g = torch.Generator(device="cuda").manual_seed(n)
    a = torch.randn(n, device="cuda", generator=g)
    b = torch.randn(n, device="cuda", generator=g)
    ref = _fp64_half_sum_sq(a, b)
    for _ in range(2):
        resid = torch.full_like(a, 7.0)
        st, J = _noalloc(lib, a, b, n, resid)
        assert st == _lib.OK
        assert abs(J - ref) <= 1e-12 * abs(ref), (J, ref)
        assert torch.equal(resid, a - b)


def test_noalloc_misfit_at_the_limit():
    # n = FDTD_NOALLOC_MISFIT_MAX: every one of the 4096 partial slots in use
    lib = _lib.load()
    n = _lib.NOALLOC_MISFIT_MAX
    g = torch.Generator(device="cuda").manual_seed(5)
    a = torch.rand(n, device="cuda", generator=g)
    b = torch.zeros(n, device="cuda")
    b[::3] = 0.5
    ref = _fp64_half_sum_sq(a, b)
    for _ in range(2):
        st, J = _noalloc(lib, a, b, n, None)
        assert st == _lib.OK
        assert abs(J - ref) <= 1e-11 * abs(ref), (J, ref)
    st, _ = _noalloc(lib, a, b, n + 1, None)
    assert st == _lib.EINVAL
    del a, b
    torch.cuda.empty_cache()
