"""Parity on the full run of the 512^3 layered workload (the benchmark's
headline configuration: 1000 steps, 20-cell CPML, R = 1e-8, 10 Hz Ricker 30
cells below the top face) against the FP64 oracle's result of the same run,
stored in tests/golden/layered512_full_run[_<form>].txt by
tests/golden/make_layered512_full_run.py (which calls only the oracle).
Traces at 72 receivers (every 10th step) and p at 128 sampled nodes after
the last step, within the FP32 bar: rel L2 <= 1e-4, max-abs rel <= 1e-3.
Forms: the plain step, the staggered grid at c dt / h = 0.4, the density
(c / 1500)^(1/4) and the local CPML grading; each form's golden run must be
stored."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import synth
from tests.parity_util import rel_errors

pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FORMS = ["plain", "staggered", "density", "local"]


def _golden_path(form):
    name = "layered512_full_run.txt" if form == "plain" else f"layered512_full_run_{form}.txt"
    return os.path.join(GOLDEN_DIR, name)


def _read_golden(form):
    rec, steps, traces, nodes, vals = [], [], [], [], []
    for line in open(_golden_path(form)):
        if line.startswith("R "):
            rec.append([int(v) for v in line.split()[1:4]])
        elif line.startswith("T "):
            parts = line.split()
            steps.append(int(parts[1]))
            traces.append([float(v) for v in parts[2:]])
        elif line.startswith("P "):
            parts = line.split()
            nodes.append(tuple(int(v) for v in parts[1:4]))
            vals.append(float(parts[4]))
    return (np.array(rec, np.int32), np.array(steps), np.array(traces), nodes, np.array(vals))


@pytest.mark.parametrize("form", FORMS)
def test_full_run_512_matches_oracle(form):
    from paper_2606_06910_gb300.fdtd import Fdtd
    rec, steps, tr_ref, nodes, p_ref = _read_golden(form)
    w = synth.preset("layered512")
    assert tr_ref.shape == (w.nt // 10, len(rec)) and len(nodes) == 128
    dt = 0.4 * w.h / w.vmax if form == "staggered" else w.dt
    vel = w.velocity()
    vt = torch.from_numpy(vel).cuda()
    sim = Fdtd(w.shape, w.h, dt, cpml_cells=w.cpml_cells, nt_max=w.nt, nrec_max=len(rec),
               cpml_local=form == "local")
    if form == "staggered":
        sim.set_staggered(True)
    rho = None
    if form == "density":
        rho = torch.from_numpy((vel / np.float32(1500.0)) ** np.float32(0.25)).cuda()
    sim.set_model(vt, rho)
    if form == "local":
        sim.set_cpml_local(vt, R=w.R)
    else:
        sim.set_cpml(R=w.R, c_ref=w.vmax)
    wav = synth.ricker(w.nt, dt, w.f0).astype(np.float32)[None, :]
    sim.inject(w.sources(), torch.from_numpy(wav).cuda())
    traces = sim.record(rec)
    sim.step(w.nt)
    sim.sync()
    got = traces[0].cpu().numpy()[steps]
    e2, em = rel_errors(got, tr_ref)
    print(f"\n[512^3 full run, {form}] traces: rel L2 {e2:.2e}, max-abs rel {em:.2e}")
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
    p = sim.get("p")
    p_got = np.array([float(p[n]) for n in nodes])
    e2, em = rel_errors(p_got, p_ref)
    print(f"[512^3 full run, {form}] p at 128 nodes: rel L2 {e2:.2e}, max-abs rel {em:.2e}")
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
