"""Domain decomposition with halo exchange (paper Sec. 3.3) through the C ABI
(fdtd_exchange): the grid split into parts, each part a context with ghost
layers of depth 8 s refreshed every s steps, must give the undivided grid's
state bit for bit -- the analogue of the paper's Tab. 9, where the enlarged
ghost region (s = 2, 4, 8) reproduces the standard exchange exactly.

The layouts are the paper's slab-z (1, 1, 4), block-xy (2, 2, 1) and
pencil-yz (1, 2, 2), plus a 2 x 2 x 2 split whose corners come from diagonal
neighbours; the grid is ragged, the layer unequal per face, one source sits
in a neighbour's ghost region and receivers fall in every part."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06910_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

SHAPE = (96, 84, 52)
CELLS = (5, 7, 6, 4, 8, 5)
FIELDS = ["p", "vx", "vy", "vz", "psiv_x", "psiv_y", "psiv_z", "psip_x", "psip_y", "psip_z"]


def _case(storage="f32", nsteps=23):
    h = 10.0
    vel = synth.layered_model(SHAPE, seed=11, vmin=1500.0, vmax=3500.0)
    dt = 0.5 * h / float(vel.max())
    # shot 0 next to the y = 42 / z = 48 interfaces (inside the neighbours'
    # ghost layers), shot 1 elsewhere
    src = np.array([[46, 40, 26], [20, 61, 17]], np.int32)
    wav = np.stack([synth.ricker(nsteps, dt, 30.0), synth.ricker(nsteps, dt, 24.0)]).astype(np.float32)
    z, y, x = np.meshgrid([10, 47, 48, 80], [9, 41, 42, 70], [8, 25, 26, 44], indexing="ij")
    rec = np.stack([z.ravel(), y.ravel(), x.ravel()], 1).astype(np.int32)
    return dict(vel=vel, h=h, dt=dt, src=src, wav=wav, rec=rec, nsteps=nsteps, storage=storage)


def _single(c):
    from paper_2606_06910_gb300.fdtd import Fdtd
    sim = Fdtd(SHAPE, c["h"], c["dt"], nshots=2, cpml_cells=CELLS, storage=c["storage"], nt_max=c["nsteps"],
               nrec_max=len(c["rec"]))
    sim.set_model(torch.from_numpy(c["vel"]).cuda())
    sim.set_cpml(R=1e-6, c_ref=float(c["vel"].max()))
    sim.inject(c["src"], torch.from_numpy(c["wav"]).cuda())
    tr = sim.record(c["rec"])
    sim.step(c["nsteps"])
    sim.sync()
    out = {(k, s): sim.get(k, s).clone() for k in FIELDS for s in range(2)}
    return out, tr.clone()


def _decomposed(c, parts, s):
    from paper_2606_06910_gb300.decomp import Decomposition
    dec = Decomposition(SHAPE, c["h"], c["dt"], parts=parts, s=s, nshots=2, cpml_cells=CELLS, storage=c["storage"],
                        nt_max=c["nsteps"], nrec_max=len(c["rec"]))
    dec.set_model(torch.from_numpy(c["vel"]).cuda())
    dec.set_cpml(R=1e-6)
    dec.inject(c["src"], torch.from_numpy(c["wav"]).cuda())
    tr = dec.record(c["rec"])
    dec.step(c["nsteps"])
    dec.sync()
    out = {(k, sh): dec.get(k, sh).clone() for k in FIELDS for sh in range(2)}
    nparts = len(dec.subs)
    dec.close()
    return out, tr.clone(), nparts


@pytest.fixture(scope="module")
def ref32():
    c = _case()
    return c, _single(c)


@pytest.mark.parametrize("parts,s", [((1, 2, 2), 1), ((1, 2, 2), 2), ((1, 2, 2), 4), ((1, 1, 4), 1),
                                     ((1, 1, 4), 2), ((2, 2, 1), 1), ((2, 2, 1), 2), ((2, 2, 2), 1)])
def test_decomposed_run_equals_single_grid(ref32, parts, s):
    c, (ref, tr_ref) = ref32
    out, tr, nparts = _decomposed(c, parts, s)
    assert nparts == parts[0] * parts[1] * parts[2]
    assert float(ref[("p", 0)].abs().max()) > 0 and float(ref[("psip_z", 1)].abs().max()) > 0
    for key in ref:
        assert torch.equal(out[key], ref[key]), (parts, s, key, float((out[key] - ref[key]).abs().max()))
    assert torch.equal(tr, tr_ref)


def test_decomposed_run_equals_single_grid_fp16():
    c = _case("f16")
    ref, tr_ref = _single(c)
    out, tr, _ = _decomposed(c, (1, 2, 2), 2)
    for key in ref:
        assert torch.equal(out[key], ref[key]), key
    assert torch.equal(tr, tr_ref)


@pytest.mark.parametrize("form", ["density", "staggered", "local"])
def test_decomposed_forms_equal_single_grid(form):
    # the step's forms keep their per-node tables in each part's box: the
    # density's dt / rho, the staggered half-node profiles, the local grading
    from paper_2606_06910_gb300.decomp import Decomposition
    from paper_2606_06910_gb300.fdtd import Fdtd
    c = _case()
    dt = 0.4 * c["h"] / float(c["vel"].max()) if form == "staggered" else c["dt"]
    vel = torch.from_numpy(c["vel"]).cuda()
    rho = (vel / 1500.0) ** 0.25 if form == "density" else None
    outs = []
    for kind in ("single", "parts"):
        if kind == "single":
            sim = Fdtd(SHAPE, c["h"], dt, nshots=2, cpml_cells=CELLS, nt_max=c["nsteps"], nrec_max=len(c["rec"]),
                       cpml_local=form == "local")
        else:
            sim = Decomposition(SHAPE, c["h"], dt, parts=(1, 2, 2), s=2, nshots=2, cpml_cells=CELLS,
                                nt_max=c["nsteps"], nrec_max=len(c["rec"]), cpml_local=form == "local")
        if form == "staggered":
            sim.set_staggered(True)
        sim.set_model(vel, rho)
        if form == "local":
            sim.set_cpml_local(vel, R=1e-6)
        else:
            sim.set_cpml(R=1e-6, c_ref=float(c["vel"].max()))
        sim.inject(c["src"], torch.from_numpy(c["wav"]).cuda())
        tr = sim.record(c["rec"])
        sim.step(c["nsteps"])
        sim.sync()
        outs.append(({(k, s): sim.get(k, s).clone() for k in FIELDS for s in range(2)}, tr.clone()))
        sim.close()
    (ref, tr_ref), (out, tr) = outs
    for key in ref:
        assert torch.equal(out[key], ref[key]), (form, key)
    assert torch.equal(tr, tr_ref)


def test_decomposed_large_grid_equals_single_grid():
    # a grid large enough that the parts' kernels and read-outs overlap on
    # their streams (ordering of steps, exchanges and read-outs by events)
    from paper_2606_06910_gb300.decomp import Decomposition
    from paper_2606_06910_gb300.fdtd import Fdtd
    shape, cells, h, nt = (224, 200, 176), (20, 20, 20, 20, 20, 20), 10.0, 12
    vel = torch.from_numpy(synth.layered_model(shape, seed=13)).cuda()
    dt = 0.5 * h / float(vel.max())
    wav = torch.from_numpy(synth.ricker(nt, dt, 40.0).astype(np.float32)[None, :]).cuda()
    src = [[60, 99, 90]]
    a = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt)
    b = Decomposition(shape, h, dt, parts=(2, 2, 2), s=2, cpml_cells=cells, nt_max=nt)
    for sim in (a, b):
        sim.set_model(vel)
        sim.set_cpml(R=1e-8, c_ref=float(vel.max()))
        sim.inject(src, wav)
        sim.step(nt)
    for k in FIELDS:
        assert torch.equal(b.get(k), a.get(k)), k
    b.close()


def test_exchange_validates_its_arguments():
    from paper_2606_06910_gb300.fdtd import Fdtd
    a = Fdtd((20, 20, 20), 10.0, 1e-3, nt_max=4)
    b = Fdtd((20, 20, 20), 10.0, 1e-3, nt_max=4)
    lib = _lib.load()
    box = (ctypes.c_int * 6)(0, 4, 0, 20, 0, 20)
    ok = (ctypes.c_int * 3)(16, 0, 0)
    bad = (ctypes.c_int * 3)(17, 0, 0)
    assert lib.fdtd_exchange(a.ctx, b.ctx, box, ok) == _lib.OK
    assert lib.fdtd_exchange(a.ctx, b.ctx, box, bad) == _lib.EINVAL
    assert lib.fdtd_exchange(a.ctx, a.ctx, box, ok) == _lib.EINVAL
    a.set_model(torch.full((20, 20, 20), 2000.0, device="cuda"))
    a.step(1)
    assert lib.fdtd_exchange(a.ctx, b.ctx, box, ok) == _lib.ESTATE
    a.sync()
    # 16-bit parts must store velocities at one scale
    c = Fdtd((20, 20, 20), 10.0, 1e-3, nt_max=4, storage="f16")
    d = Fdtd((20, 20, 20), 10.0, 1e-3, nt_max=4, storage="f16")
    c.set_model(torch.full((20, 20, 20), 2000.0, device="cuda"))
    d.set_model(torch.full((20, 20, 20), 2500.0, device="cuda"))
    assert lib.fdtd_exchange(c.ctx, d.ctx, box, ok) == _lib.EINVAL
    c.set_velocity_scale(2500.0)
    c.set_model(torch.full((20, 20, 20), 2000.0, device="cuda"))
    assert lib.fdtd_exchange(c.ctx, d.ctx, box, ok) == _lib.OK
    c.sync()
