"""Kernel timing (fdtd_set_timing / fdtd_timing): one CUDA event pair per
launch of the step kernel (single steps, and the band launches of temporal
blocking) and of the adjoint kernel; counts equal the launches made, times are
positive and bounded by the wall clock of the work, and timing leaves the
results unchanged."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import synth

pytestmark = pytest.mark.gpu


def _sim(**kw):
    from paper_2606_06910_gb300.fdtd import Fdtd
    shape, h = (72, 64, 80), 10.0
    dt = 0.5 * h / 3000.0
    sim = Fdtd(shape, h, dt, cpml_cells=8, nt_max=40, **kw)
    sim.set_model(torch.full(shape, 3000.0, device="cuda"))
    sim.set_cpml(R=1e-6, c_ref=3000.0)
    sim.inject([[30, 30, 40]], torch.from_numpy(synth.ricker(40, dt, 30.0).astype(np.float32)[None, :]).cuda())
    return sim


def test_step_launches_counted_and_timed():
    a, b = _sim(), _sim()
    b.set_timing(True)
    a.step(24)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(24)
    b.sync()
    wall_ms = (time.perf_counter() - t0) * 1e3
    ms, n = b.timing("step")
    assert n == 24 and 0.0 < ms <= wall_ms + 1.0
    assert b.timing("adjoint") == (0.0, 0)
    assert torch.equal(a.get("p"), b.get("p"))
    b.set_timing(True)   # clears the totals
    assert b.timing("step") == (0.0, 0)


def test_band_launches_counted():
    sim = _sim(tblock_k=2)
    sim.set_timing(True)
    sim.step(8)
    sim.sync()
    ms, n = sim.timing("step")
    # 4 blocks of 2 steps, each step launched once per z band
    assert n >= 8 and n % 8 == 0 and ms > 0.0


def test_adjoint_launches_counted():
    sim = _sim(checkpoint_every=10, nrec_max=4)
    sim.record(np.array([[10, 30, 40], [12, 20, 30], [40, 40, 40], [60, 10, 70]], np.int32))
    sim.step(20)
    resid = sim.traces.clone()
    grad = torch.zeros(sim.shape, device="cuda")
    sim.set_timing(True)
    sim.adjoint(20, resid, grad)
    sim.sync()
    ms, n = sim.timing("adjoint")
    assert n == 20 and ms > 0.0
    assert sim.timing("step")[1] == 20   # the recomputed forward steps
