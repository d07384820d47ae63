"""The paper's 2D acoustic CPML demonstration (Sec. 5) on the library.

Domain 2 km x 2 km at dx = dz = 8 m (250 x 250 nodes; y has one node and no
layer, so delta_y vanishes), elliptic anisotropy c_x = 2600 m/s, c_z = 1800
m/s (model velocity c_z, axis factors ((c_x/c_z)^2, 1, 1)), a Ricker source
(1 - 2 a^2) exp(-a^2), a = pi f0 (t - t0), f0 = 30 Hz, at the centre, and a
10-cell layer on the four edges (or none).  The step is CFL 0.5 at c_x.
"""
from __future__ import annotations

import numpy as np
import torch

from . import synth
from .fdtd import Fdtd

N, H, CZ, CX, F0, L = 250, 8.0, 1800.0, 2600.0, 30.0, 10


def config():
    dt = 0.5 * H / CX
    return dict(shape=(N, 1, N), h=H, dt=dt, kr=(CX * CX / (CZ * CZ), 1.0, 1.0), f0=F0, L=L, cx=CX, cz=CZ,
                src=(N // 2, 0, N // 2), box=(L, N - L, 0, 1, L, N - L))


def anisotropic_2d(cpml: bool, nt: int, every: int, snap_at=None, device="cuda"):
    """Run the demonstration for nt steps; returns (sim, energies, config,
    snapshot): sum p^2 inside the layer every `every` steps, and p after
    `snap_at` steps (or None)."""
    cfg = config()
    shape, dt = cfg["shape"], cfg["dt"]
    cells = (L, L, 0, 0, L, L) if cpml else 0
    sim = Fdtd(shape, H, dt, cpml_cells=cells, nt_max=nt, device=device)
    sim.set_model(torch.full(shape, CZ, device=sim.device))
    sim.set_anisotropy(cfg["kr"])
    if cpml:
        sim.set_cpml(R=1e-5, c_ref=CX)
    wav = synth.ricker(nt, dt, F0).astype(np.float32)[None, :]
    cfg["wav"] = wav
    sim.inject(np.array([cfg["src"]], np.int32), torch.from_numpy(wav).to(sim.device))
    energies, snap = [], None
    for k in range(nt // every):
        sim.step(every)
        energies.append(sim.energy(0, cfg["box"]))
        if snap_at == (k + 1) * every:
            snap = sim.get("p").cpu().numpy()
    return sim, np.array(energies), cfg, snap
