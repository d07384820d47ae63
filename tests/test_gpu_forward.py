"""Parity of the CUDA forward step (through the C ABI) with the FP64 oracle on
the same seeded inputs.  Tolerances: relative L2 <= 1e-4 and max-abs
relative <= 1e-3 on every field (FP32 storage)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import (FIELDS, gpu_fields, oracle_grid, oracle_state, rel_errors, set_gpu_state,
                               state_scales, subbox_point)

pytestmark = pytest.mark.gpu

RTOL_L2, RTOL_MAX = 1e-4, 1e-3


def _fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _check(name, got, ref, l2=RTOL_L2, mx=RTOL_MAX):
    e2, em = rel_errors(got, ref)
    assert e2 <= l2 and em <= mx, f"{name}: rel L2 {e2:.3e}, max-abs rel {em:.3e}"


def test_homogeneous_64_full_run_matches_oracle():
    """64^3, c = 2000 m/s, 15 Hz Ricker at the centre, 10 CPML cells, 200 steps."""
    Fdtd = _fdtd()
    w = synth.preset("homog64")
    vel = w.velocity()
    src = w.sources()
    wav = w.wavelet()
    rec = synth.receiver_grid(w.shape, w.cpml_cells, 4, 4, 12)
    sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, nt_max=w.nt, nrec_max=len(rec))
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=w.R, kappa_max=w.kappa_max, alpha_frac=w.alpha_frac, q=w.q, c_ref=w.c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    traces = sim.record(rec)
    sim.step(w.nt)
    sim.sync()
    got = gpu_fields(sim)

    g = oracle_grid(vel, w.h, w.dt, w.cpml_cells, w.c, R=w.R)
    st = O.State(w.shape)
    tr = O.run(g, st, w.nt, 0, tuple(src[0]), wav[0].astype(np.float64), rec)
    for k in FIELDS:
        _check(k, got[k], st[k])
    _check("traces", traces[0].cpu().numpy(), tr)


@pytest.mark.parametrize("shape,cells,zchunk", [
    ((11, 13, 17), (3, 2, 4, 3, 2, 5), None),
    ((70, 37, 150), (3, 5, 2, 4, 6, 1), None),
    ((70, 37, 150), (3, 5, 2, 4, 6, 1), "7"),
    ((40, 33, 70), (0, 0, 0, 0, 0, 0), "9"),
    ((24, 20, 64), (8, 8, 8, 8, 8, 8), None),
    # x layers reaching two tile columns on each side (launched before the others)
    ((20, 36, 200), (30, 33, 2, 3, 2, 2), None),
])
def test_ragged_grids_random_state_all_fields(shape, cells, zchunk, monkeypatch):
    """Random state on grids that span several tiles with ragged tails, unequal
    layers per face, z-chunk boundaries, no layer at all, and x layers wide enough
    that two tile columns per face carry them: 5 steps."""
    if zchunk:
        monkeypatch.setenv("FDTD_ZCHUNK", zchunk)
    Fdtd = _fdtd()
    h, c = 10.0, 2500.0
    rng = np.random.default_rng(3)
    vel = rng.uniform(1500.0, c, size=shape).astype(np.float32)
    dt = 0.5 * h / c
    state = synth.random_state(shape, cells, seed=11, **state_scales(h, dt))
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    set_gpu_state(sim, state)
    sim.step(5)
    sim.sync()
    got = gpu_fields(sim)
    g = oracle_grid(vel, h, dt, cells, c, R=1e-5)
    st = oracle_state(shape, state)
    O.run(g, st, 5)
    for k in FIELDS:
        if np.max(np.abs(st[k])) == 0.0:
            assert np.max(np.abs(got[k])) == 0.0, k
            continue
        _check(k, got[k], st[k])


def test_multi_shot_layered_with_receivers():
    Fdtd = _fdtd()
    shape, cells, h = (48, 40, 56), (6,) * 6, 10.0
    vel = synth.layered_model(shape, seed=4)
    dt = 0.5 * h / 4500.0
    nt, nshots = 120, 3
    src = synth.shot_positions(shape, cells, seed=5, nshots=nshots, z=8)
    wav = np.stack([synth.ricker(nt, dt, f) for f in (12.0, 15.0, 20.0)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 5, 6, 6)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-6, c_ref=4500.0)
    sim.inject(src, torch.from_numpy(wav).cuda())
    traces = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = oracle_grid(vel, h, dt, cells, 4500.0, R=1e-6)
    for s in range(nshots):
        st = O.State(shape)
        tr = O.run(g, st, nt, 0, tuple(src[s]), wav[s].astype(np.float64), rec)
        _check(f"shot {s} p", sim.get("p", s).cpu().numpy(), st["p"])
        _check(f"shot {s} traces", traces[s].cpu().numpy(), tr)


def test_full_size_512_sampled_parity():
    """512^3 layered model with 20-cell layers in the benchmark's launch
    configuration: random state, 2 steps, every field at sampled nodes (slab
    faces, edges, corners, interior) against the oracle on a sub-box around
    each node."""
    Fdtd = _fdtd()
    w = synth.preset("layered512")
    shape, cells = w.shape, w.cpml_cells
    vel = w.velocity()
    state = synth.random_state(shape, cells, seed=12, **state_scales(w.h, w.dt))
    sim = Fdtd(shape, w.h, w.dt, cpml_cells=cells, nt_max=4)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=w.R, c_ref=w.c_max)
    set_gpu_state(sim, state)
    nsteps = 2
    sim.step(nsteps)
    sim.sync()
    got = {k: sim.get(k).cpu().numpy() for k in FIELDS}
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (511, 511, 511), (0, 511, 255), (19, 20, 21), (20, 19, 492), (491, 492, 19),
           (256, 256, 256), (255, 63, 64), (300, 15, 16), (100, 16, 511), (17, 300, 63)]
    pts += [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(25)]
    pts += [tuple(int(v) for v in rng.integers(0, 24, 3)) for _ in range(6)]
    for p in pts:
        ref = subbox_point(state, vel, w.h, w.dt, cells, w.c_max, p, 8 * nsteps + 1, nsteps, R=w.R)
        for k in FIELDS:
            r = ref[k]
            gv = got[k][p]
            scale = max(np.max(np.abs(state[k])), 1e-30)
            assert abs(gv - r) <= 1e-5 * scale + 1e-5 * abs(r), (p, k, gv, r)


def test_errors_are_reported():
    from paper_2606_06910_gb300.fdtd import Fdtd, FdtdError
    from paper_2606_06910_gb300 import _lib
    shape = (16, 16, 16)
    sim = Fdtd(shape, 10.0, 4e-3, cpml_cells=4, nt_max=4)
    with pytest.raises(FdtdError) as e:
        sim.step(1)
    assert e.value.status == _lib.ESTATE
    vel = torch.full(shape, 2000.0, device="cuda")
    with pytest.raises(FdtdError) as e:
        sim.set_model(vel)            # c dt / h = 0.8 > 0.667
    assert e.value.status == _lib.EUNSTABLE
    sim2 = Fdtd(shape, 10.0, 2e-3, cpml_cells=4, nt_max=4)
    bad = vel.clone()
    bad[3, 3, 3] = -1.0
    with pytest.raises(FdtdError) as e:
        sim2.set_model(bad)
    assert e.value.status == _lib.EINVAL
    sim2.set_model(vel)
    with pytest.raises(FdtdError) as e:
        sim2.inject([[16, 0, 0]], torch.zeros((1, 4), device="cuda"))
    assert e.value.status == _lib.EINVAL


def test_field_roundtrip_and_slab_masking():
    Fdtd = _fdtd()
    shape, cells = (20, 18, 30), (3, 4, 5, 2, 1, 6)
    sim = Fdtd(shape, 10.0, 1e-3, cpml_cells=cells, nt_max=2)
    rng = np.random.default_rng(1)
    for k in FIELDS:
        a = rng.standard_normal(shape).astype(np.float32)
        sim.set(k, torch.from_numpy(a).cuda())
        b = sim.get(k).cpu().numpy()
        if k.startswith("psi"):
            d = "xyz".index(k[-1])
            n = shape[2 - d]
            m = synth.slab_mask(n, cells[2 * d], cells[2 * d + 1])
            shp = [1, 1, 1]
            shp[2 - d] = n
            expect = np.where(m.reshape(shp), a, 0.0)
        else:
            expect = a
        assert np.array_equal(b, expect), k


def test_energy_and_misfit_reductions_fp64():
    Fdtd = _fdtd()
    shape = (30, 20, 40)
    sim = Fdtd(shape, 10.0, 1e-3, cpml_cells=0, nt_max=6, nrec_max=5)
    rng = np.random.default_rng(2)
    p = rng.standard_normal(shape).astype(np.float32)
    sim.set("p", torch.from_numpy(p).cuda())
    e = sim.energy()
    assert abs(e - float(np.sum(p.astype(np.float64) ** 2))) <= 1e-12 * e
    box = (3, 17, 2, 9, 5, 33)
    eb = sim.energy(box=box)
    ref = float(np.sum(p[3:17, 2:9, 5:33].astype(np.float64) ** 2))
    assert abs(eb - ref) <= 1e-12 * ref
    sim.set_model(torch.full(shape, 2000.0, device="cuda"))
    rec = np.array([[5, 5, 5], [10, 3, 30], [29, 19, 39], [0, 0, 0], [15, 10, 20]])
    traces = sim.record(rec)
    sim.step(6)
    dobs = torch.from_numpy(rng.standard_normal((1, 6, 5)).astype(np.float32)).cuda()
    resid = torch.empty_like(dobs)
    J = sim.misfit(dobs, nt=4, resid=resid)
    t64 = traces.cpu().numpy().astype(np.float64)
    d64 = dobs.cpu().numpy().astype(np.float64)
    r = (t64 - d64)[:, :4]
    assert abs(J - 0.5 * float(np.sum(r * r))) <= 1e-6 * max(J, 1e-30)
    assert np.allclose(resid.cpu().numpy()[:, :4], (traces - dobs).cpu().numpy()[:, :4])
    assert np.all(resid.cpu().numpy()[:, 4:] == 0)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_interior_and_edge_chunkings_give_identical_state(monkeypatch, storage):
    """100 x 96 x 100, 24 shots: large enough that the default launch cuts z
    into one chunk per CPML end plus interior chunks (whose interior tiles run
    the kernel's interior form).  The state after 6 steps, with sources and
    receivers, equals bit for bit the one of uniform 7-plane chunks, where
    every CTA runs the general form; FP32 and FP16 storage."""
    Fdtd = _fdtd()
    shape, cells, nshots, n = (100, 96, 100), (4, 5, 4, 6, 5, 4), 24, 6
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    vel = synth.layered_model(shape, seed=4, vmin=1600.0, vmax=c, amp_cells=2.0)
    src = synth.shot_positions(shape, cells, 9, nshots, z=cells[4] + 2)
    wav = np.stack([synth.ricker(n, dt, 25.0) for _ in range(nshots)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 4, 4, 50)
    states = {s: synth.random_state(shape, cells, seed=70 + s, **state_scales(h, dt)) for s in (0, 11, 23)}
    out = []
    for zc in (None, "7"):
        if zc is None:
            monkeypatch.delenv("FDTD_ZCHUNK", raising=False)
        else:
            monkeypatch.setenv("FDTD_ZCHUNK", zc)
        sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, nrec_max=len(rec), storage=storage)
        sim.set_model(torch.from_numpy(vel).cuda())
        sim.set_cpml(R=1e-5, c_ref=c)
        sim.inject(src, torch.from_numpy(wav).cuda())
        tr = sim.record(rec)
        for s, st in states.items():
            set_gpu_state(sim, st, s)
        sim.step(n)
        sim.sync()
        out.append(({s: {f: sim.get(f, s) for f in FIELDS} for s in states}, tr.clone()))
        del sim
    for s in states:
        for f in FIELDS:
            assert torch.equal(out[0][0][s][f], out[1][0][s][f]), (s, f)
    assert torch.equal(out[0][1], out[1][1])
    assert float(out[0][1].abs().max()) > 0
