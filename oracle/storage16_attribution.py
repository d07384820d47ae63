"""Attribution of the 16-bit storage form's error to the stored fields.

    python -m oracle.storage16_attribution [--preset layered128] [--steps 250,375,500]

Runs the FP64 oracle on the precision form's accuracy instance (the 128^3
layered model, seed 3, 500 steps) with the storage rounding of the form
applied to one group of fields at a time (p; v; psi_v; psi_p; all), in FP16
(scale 2^10, velocities also by c_max) and BF16 (velocities by c_max), and
prints the relative L2 error of the pressure at each checkpoint and of the
receiver traces against the unrounded run.  A relative-L2 budget applies to
the sum of independent rounding noises, so the groups add in quadrature.

Test infrastructure: it calls only the oracle and the seeded input generator.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from oracle import oracle as O
from paper_2606_06910_gb300 import synth

GROUPS = {"p": 1, "v": 2, "psi_v": 4, "psi_p": 8, "all": 15}


def run(w, store, mask, checkpoints, sp, sv):
    vel = w.velocity().astype(np.float64)
    g = O.Grid(vel * vel, w.h, w.dt, O.make_profiles(w.shape, w.cpml_cells, w.h, w.dt, w.vmax, R=w.R),
               store=store, store_mask=mask, scale_p=sp, scale_v=sv)
    st = O.State(w.shape)
    src = tuple(w.sources()[0])
    wav = w.wavelet()[0].astype(np.float64)
    rec = synth.receiver_grid(w.shape, w.cpml_cells, 6, 6, w.cpml_cells[4])
    out, t, trs = {}, 0, []
    for c in checkpoints:
        trs.append(O.run(g, st, c - t, t, src, wav, rec))
        t = c
        out[c] = st["p"].copy()
    out["traces"] = np.concatenate(trs)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="layered128")
    ap.add_argument("--steps", default="250,375,500")
    ap.add_argument("--formats", default="f16,bf16")
    args = ap.parse_args()
    w = synth.preset(args.preset)
    cps = tuple(int(x) for x in args.steps.split(","))
    t0 = time.time()
    ref = run(w, None, 0, cps, 1.0, 1.0)
    rows = []
    for fmt in args.formats.split(","):
        sp = 1024.0 if fmt == "f16" else 1.0
        for name, mask in GROUPS.items():
            o = run(w, fmt, mask, cps, sp, float(w.vmax))
            e = {f"p_step{c}": float(np.linalg.norm(o[c] - ref[c]) / np.linalg.norm(ref[c])) for c in cps}
            e["traces"] = float(np.linalg.norm(o["traces"] - ref["traces"]) / np.linalg.norm(ref["traces"]))
            rows.append({"format": fmt, "rounded": name, **{k: float(f"{v:.3e}") for k, v in e.items()}})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"instance": f"{args.preset}, checkpoints {cps}", "threads": O.threads(),
                      "seconds": round(time.time() - t0, 1)}), flush=True)


if __name__ == "__main__":
    main()
