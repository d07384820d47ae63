"""Shared helpers of the GPU parity tests: build the same seeded inputs for the
CUDA path and the FP64 oracle, and compare fields."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

FIELDS = ("p", "vx", "vy", "vz", "psiv_x", "psiv_y", "psiv_z", "psip_x", "psip_y", "psip_z")


def rel_errors(got, ref):
    """(relative L2, max-abs relative) of got against ref."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nref = np.sqrt(np.sum(ref * ref))
    mref = np.max(np.abs(ref))
    if nref == 0.0:
        return float(np.sqrt(np.sum(got * got))), float(np.max(np.abs(got)) if got.size else 0.0)
    return float(np.sqrt(np.sum((got - ref) ** 2)) / nref), float(np.max(np.abs(got - ref)) / mref)


def oracle_grid(vel, h, dt, cells, c_ref, R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3):
    vel = np.asarray(vel, dtype=np.float64)
    prof = O.make_profiles(vel.shape, cells, h, dt, c_ref, R=R, q=q, kappa_max=kappa_max,
                           alpha_frac=alpha_frac)
    return O.Grid(vel * vel, h, dt, prof)


def state_scales(h, dt):
    """Magnitudes that keep every term of the update comparable for random
    states: v ~ dt/h p, psi_v ~ p/h, psi_p ~ v/h."""
    return dict(p_scale=1.0, v_scale=dt / h, psiv_scale=1.0 / h, psip_scale=dt / h ** 2)


def gpu_fields(sim, shot=0):
    return {k: sim.get(k, shot).cpu().numpy() for k in FIELDS}


def set_gpu_state(sim, state, shot=0):
    import torch
    for k in FIELDS:
        sim.set(k, torch.from_numpy(np.ascontiguousarray(state[k], dtype=np.float32)).to(sim.device), shot)


def oracle_state(shape, state):
    st = O.State(shape)
    for k in FIELDS:
        st[k] = np.asarray(state[k], dtype=np.float64)
    return st


def subbox_point(full_state, vel, h, dt, cells, c_ref, point, radius, nsteps, R=1e-8, staggered=False, local=False):
    """Oracle values of every field at `point` after nsteps, computed on the
    sub-box of the given radius around it (exact when radius >= 8 nsteps: the
    step's dependence radius is 2r = 8 nodes per axis)."""
    nz, ny, nx = vel.shape
    z, y, x = point
    z0, z1 = max(0, z - radius), min(nz, z + radius + 1)
    y0, y1 = max(0, y - radius), min(ny, y + radius + 1)
    x0, x1 = max(0, x - radius), min(nx, x + radius + 1)
    prof_full = O.make_profiles(vel.shape, cells, h, dt, c_ref, R=R)
    sl = [(x0, x1), (y0, y1), (z0, z1)]
    prof = []
    for d in range(3):
        a, b = sl[d]
        prof.append({k: np.ascontiguousarray(prof_full[d][k][a:b])
                     for k in ("slab", "b", "a", "kinv", "bv", "av", "kinvv")})
    v = np.asarray(vel[z0:z1, y0:y1, x0:x1], dtype=np.float64)
    lp = O.local_profiles(v, cells, h, dt, R=R, full_shape=vel.shape, origin=(z0, y0, x0)) if local else None
    g = O.Grid(v * v, h, dt, prof, staggered=staggered, local=lp)
    st = O.State(v.shape)
    for k in FIELDS:
        st[k] = np.asarray(full_state[k][z0:z1, y0:y1, x0:x1], dtype=np.float64)
    O.run(g, st, nsteps)
    return {k: st[k][z - z0, y - y0, x - x0] for k in FIELDS}
