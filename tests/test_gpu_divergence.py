"""Divergence detection (fdtd_set_divergence_check): an FP64 sum of p^2 over
every shot every M steps, flagged on the device and reported by the next
fdtd_sync as EDIVERGED.  The failure is made on the host side of the data (a
NaN written into the field, an energy limit set below the field's energy);
no GPU fault is involved."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _sim(check_every=0, limit=0.0):
    from paper_2606_06910_gb300.fdtd import Fdtd
    shape, h = (40, 36, 44), 10.0
    dt = 0.5 * h / 3000.0
    sim = Fdtd(shape, h, dt, nshots=2, cpml_cells=6, nt_max=30)
    sim.set_model(torch.full(shape, 3000.0, device="cuda"))
    sim.set_cpml(R=1e-6, c_ref=3000.0)
    wav = np.stack([synth.ricker(30, dt, 30.0), synth.ricker(30, dt, 25.0)]).astype(np.float32)
    sim.inject([[20, 18, 22], [10, 20, 30]], torch.from_numpy(wav).cuda())
    if check_every:
        sim.set_divergence_check(check_every, limit)
    return sim


def test_healthy_run_passes_and_is_unchanged():
    a, b = _sim(), _sim(check_every=5)
    a.step(30)
    b.step(30)
    a.sync()
    b.sync()
    for k in ("p", "vx", "psip_z"):
        for s in range(2):
            assert torch.equal(a.get(k, s), b.get(k, s))


def test_nan_in_the_field_is_reported_and_reset_clears_it():
    from paper_2606_06910_gb300._lib import FdtdError
    sim = _sim(check_every=1)
    sim.step(3)
    sim.sync()
    p = sim.get("p", 1)
    p[5, 7, 9] = math.nan
    sim.set("p", p, 1)
    sim.step(2)
    with pytest.raises(FdtdError) as e:
        sim.sync()
    assert e.value.status == _lib.EDIVERGED
    sim.reset()
    sim.step(4)
    sim.sync()


def test_energy_above_the_limit_is_reported():
    from paper_2606_06910_gb300._lib import FdtdError
    sim = _sim(check_every=4, limit=1e-30)
    sim.step(12)
    with pytest.raises(FdtdError) as e:
        sim.sync()
    assert e.value.status == _lib.EDIVERGED
