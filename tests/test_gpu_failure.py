"""Failure detection on the GPU without a fault: a wait that nothing
completes.  With FDTD_FAULT=wait one CTA of the step kernel leaves one
pipeline stage without its copies; its bounded mbarrier wait gives up, the
kernel records ERR_TIMEOUT, drains the copies it has in flight and returns.
The host then reads FDTD_ETIMEOUT, and the context keeps working: after
fdtd_reset the same steps give the same bits as a fresh context."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, set_gpu_state, state_scales

pytestmark = pytest.mark.gpu


def _sim(shape, cells, h, dt, vel):
    from paper_2606_06910_gb300.fdtd import Fdtd
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=4)
    sim.set_model(vel)
    sim.set_cpml(R=1e-5, c_ref=2500.0)
    return sim


def test_bounded_wait_gives_up_and_the_context_recovers(monkeypatch):
    from paper_2606_06910_gb300 import _lib
    from paper_2606_06910_gb300.fdtd import FdtdError
    shape, cells, h, c = (40, 36, 44), (4, 5, 3, 4, 5, 4), 10.0, 2500.0
    dt = 0.5 * h / c
    vel = torch.from_numpy(synth.layered_model(shape, seed=1, vmin=1600.0, vmax=c)).cuda()
    state = synth.random_state(shape, cells, seed=31, **state_scales(h, dt))

    monkeypatch.delenv("FDTD_FAULT", raising=False)
    ref = _sim(shape, cells, h, dt, vel)
    set_gpu_state(ref, state)
    ref.step(3)
    ref.sync()
    want = {k: ref.get(k) for k in FIELDS}

    sim = _sim(shape, cells, h, dt, vel)
    set_gpu_state(sim, state)
    monkeypatch.setenv("FDTD_FAULT", "wait")
    t0 = time.perf_counter()
    sim.step(1)
    with pytest.raises(FdtdError) as ei:
        sim.sync()
    secs = time.perf_counter() - t0
    print(f"\n[failure] bounded wait gave up; step + sync took {secs:.2f} s")
    assert ei.value.status == _lib.ETIMEOUT
    assert secs < 60.0

    monkeypatch.delenv("FDTD_FAULT")
    sim.reset()
    set_gpu_state(sim, state)
    sim.step(3)
    sim.sync()
    for k in FIELDS:
        assert torch.equal(sim.get(k), want[k]), k
