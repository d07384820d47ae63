"""Checkpoint / resume: a run stopped after some steps, its whole state read
out (fdtd_get_field), restored into a fresh context (fdtd_set_field) at the
same time index (fdtd_set_time) and continued, equals the uninterrupted run
bit for bit -- every field, both shots, and the traces of the continued
steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ["p", "vx", "vy", "vz", "psiv_x", "psiv_y", "psiv_z", "psip_x", "psip_y", "psip_z"]


def test_resume_equals_uninterrupted_run():
    from paper_2606_06910_gb300.fdtd import Fdtd
    shape, cells, h = (45, 38, 70), (6, 5, 4, 7, 8, 3), 10.0
    vel = synth.layered_model(shape, seed=21, vmin=1500.0, vmax=3200.0)
    dt = 0.5 * h / float(vel.max())
    nt, stop = 40, 17
    src = np.array([[20, 19, 35], [30, 10, 50]], np.int32)
    wav = np.stack([synth.ricker(nt, dt, 28.0), synth.ricker(nt, dt, 22.0)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 3, 4, 12)

    def make():
        sim = Fdtd(shape, h, dt, nshots=2, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
        sim.set_model(torch.from_numpy(vel).cuda())
        sim.set_cpml(R=1e-6, c_ref=float(vel.max()))
        sim.inject(src, torch.from_numpy(wav).cuda())
        return sim, sim.record(rec)

    a, tr_a = make()
    a.step(nt)
    a.sync()
    b, _ = make()
    b.step(stop)
    b.sync()
    saved = {(k, s): b.get(k, s).clone() for k in FIELDS for s in range(2)}
    c, tr_c = make()
    for (k, s), v in saved.items():
        c.set(k, v, s)
    c.set_time(stop)
    assert c.time == stop
    c.step(nt - stop)
    c.sync()
    for k in FIELDS:
        for s in range(2):
            assert torch.equal(c.get(k, s), a.get(k, s)), (k, s)
    assert torch.equal(tr_c[:, stop:], tr_a[:, stop:])
