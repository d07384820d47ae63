"""Writes tests/golden/layered512_full_run[_<form>].txt: the FP64 oracle's
result of the full 512^3 layered workload (Sec. 3.1-3.2 step; 20-cell CPML
with R = 1e-8, 10 Hz Ricker source 30 cells below the top face, 1000 steps),
at 72 fixed receivers every 10th step and at 128 sampled nodes of p after the
last step.  Forms: plain (c_max dt / h = 0.5), staggered (the Yee form at
0.4), density (rho = (c / 1500)^(1/4) per node), local (the CPML graded from
the velocity at each slab node).  It calls only the oracle and the seeded
input generators; the GPU parity test reads the file.  Each form runs in
about an hour on 8 CPU threads and needs about 13 GB of memory.

    python tests/golden/make_layered512_full_run.py [plain|staggered|density|local]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2606_06910_gb300 import synth  # noqa: E402

EVERY = 10
FORMS = ("plain", "staggered", "density", "local")


def out_path(form):
    name = "layered512_full_run.txt" if form == "plain" else f"layered512_full_run_{form}.txt"
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), name)


def form_dt(w, form):
    """Time step of the form: the staggered limit is 0.4488, so it runs at 0.4."""
    return 0.4 * w.h / w.vmax if form == "staggered" else w.dt


def receivers_and_nodes(w):
    """The receiver set and the sampled nodes (also used by the test)."""
    cells = w.cpml_cells
    rec = synth.receiver_grid(w.shape, cells, 8, 8, cells[4])
    deep = np.array([[100, 256, 256], [256, 256, 256], [400, 128, 384], [480, 300, 200],
                     [256, 30, 256], [256, 256, 481], [505, 505, 505], [10, 10, 10]], np.int32)
    rec = np.concatenate([rec, deep]).astype(np.int32)
    rng = np.random.default_rng(2024)
    nodes = [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(112)]
    nodes += [(0, 0, 0), (511, 511, 511), (30, 256, 256), (31, 256, 256), (60, 200, 300), (19, 20, 21),
              (20, 19, 492), (491, 492, 19), (256, 256, 0), (256, 0, 256), (0, 256, 256), (300, 15, 16),
              (100, 16, 511), (17, 300, 63), (255, 63, 64), (40, 100, 100)]
    return rec, nodes


def main(form="plain"):
    assert form in FORMS, form
    OUT = out_path(form)
    w = synth.preset("layered512")
    rec, nodes = receivers_and_nodes(w)
    dt = form_dt(w, form)
    vel32 = w.velocity()
    vel = vel32.astype(np.float64)
    prof = O.make_profiles(w.shape, w.cpml_cells, w.h, dt, w.vmax, R=w.R)
    if form == "density":
        rho = ((vel32 / np.float32(1500.0)) ** np.float32(0.25)).astype(np.float64)   # the library's FP32 input
        g = O.Grid(rho * vel * vel, w.h, dt, prof, rho=rho)
    elif form == "local":
        g = O.Grid(vel * vel, w.h, dt, prof, local=O.local_profiles(vel, w.cpml_cells, w.h, dt, R=w.R))
    else:
        g = O.Grid(vel * vel, w.h, dt, prof, staggered=form == "staggered")
    del vel, vel32
    st = O.State(w.shape)
    src = tuple(int(v) for v in w.sources()[0])
    wav = synth.ricker(w.nt, dt, w.f0).astype(np.float32).astype(np.float64)
    t0 = time.time()
    traces = O.run(g, st, w.nt, 0, src, wav, rec)
    secs = time.time() - t0
    p = st["p"]
    with open(OUT + ".tmp", "w") as f:
        f.write("# FP64 oracle, full run of the 512^3 layered workload (Sec. 3.1 leapfrog, Sec. 3.2 CPML):\n")
        f.write(f"# form {form}; {w.nt} steps, dt = {dt!r}, h = {w.h}, 20-cell CPML, R = {w.R}, "
                f"c_ref = {w.vmax}, 10 Hz Ricker at {src}.\n")
        f.write(f"# Written by tests/golden/make_layered512_full_run.py ({secs:.0f} s).\n")
        f.write("# R z y x: receivers, in column order of the T lines\n")
        f.write(f"# T n v...: p at the receivers after step n (every {EVERY}th step)\n")
        f.write("# P z y x v: p at a sampled node after the last step\n")
        for r in rec:
            f.write(f"R {r[0]} {r[1]} {r[2]}\n")
        for n in range(EVERY - 1, w.nt, EVERY):
            f.write("T " + str(n) + " " + " ".join(f"{v:.17g}" for v in traces[n]) + "\n")
        for z, y, x in nodes:
            f.write(f"P {z} {y} {x} {p[z, y, x]:.17g}\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT} in {secs:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "plain")
