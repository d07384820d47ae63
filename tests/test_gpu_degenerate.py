"""Degenerate grids through the C ABI against the FP64 oracle: lines along z
and x, a single z plane, axes whose every node lies in the CPML, z extents
below the stencil's reach, one tile with most of its nodes beyond the grid,
and the 16-bit, blocked, staggered, local-grading and adjoint paths on such
grids.  Random states (memory variables only inside their slabs) and a 1D
source run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, gpu_fields, oracle_grid, oracle_state, rel_errors, set_gpu_state, state_scales

pytestmark = pytest.mark.gpu

CASES = [
    ((60, 1, 1), (0, 0, 0, 0, 5, 5)),       # a line along z
    ((1, 1, 70), (6, 6, 0, 0, 0, 0)),       # a line along x
    ((1, 40, 37), (3, 4, 5, 2, 0, 0)),      # one z plane
    ((8, 6, 20), (3, 3, 3, 3, 4, 4)),       # every y and z node in a slab
    ((3, 9, 12), (2, 2, 1, 2, 1, 1)),       # nz below the reach of one step
    ((5, 33, 1), (0, 0, 4, 4, 2, 2)),       # one x node, two tiles along y
]


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _check_all(got, st, bar=(1e-4, 1e-3)):
    for k in FIELDS:
        if np.max(np.abs(st[k])) == 0.0:
            assert np.max(np.abs(got[k])) == 0.0, k
            continue
        e2, em = rel_errors(got[k], st[k])
        assert e2 <= bar[0] and em <= bar[1], (k, e2, em)


@pytest.mark.parametrize("shape,cells", CASES)
def test_degenerate_grid_random_state(shape, cells):
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(17)
    vel = rng.uniform(1500.0, c, size=shape).astype(np.float32)
    state = synth.random_state(shape, cells, seed=18, **state_scales(h, dt))
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    set_gpu_state(sim, state)
    sim.step(7)
    sim.sync()
    st = oracle_state(shape, state)
    O.run(oracle_grid(vel, h, dt, cells, c, R=1e-5), st, 7)
    _check_all(gpu_fields(sim), st)


def test_line_along_z_source_and_receivers():
    """A 1D run along z with a source, two shots and receivers on every
    tenth node: fields and traces over 200 steps."""
    Fdtd = _Fdtd()
    shape, cells, h, c, nt = (120, 1, 1), (0, 0, 0, 0, 10, 10), 10.0, 2000.0, 200
    dt = 0.5 * h / c
    vel = np.full(shape, c, np.float32)
    src = np.array([[40, 0, 0], [75, 0, 0]], np.int32)
    wav = np.stack([synth.ricker(nt, dt, 20.0), synth.ricker(nt, dt, 30.0)]).astype(np.float32)
    rec = np.array([[z, 0, 0] for z in range(0, 120, 10)], np.int32)
    sim = Fdtd(shape, h, dt, nshots=2, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = oracle_grid(vel, h, dt, cells, c, R=1e-5)
    for s in range(2):
        st = O.State(shape)
        tro = O.run(g, st, nt, 0, tuple(src[s]), wav[s].astype(np.float64), rec)
        _check_all(gpu_fields(sim, s), st)
        e2, em = rel_errors(tr[s].cpu().numpy(), tro)
        assert e2 <= 1e-4 and em <= 1e-3, (s, e2, em)


@pytest.mark.parametrize("shape,cells", [CASES[2], CASES[3]])
def test_degenerate_grid_fp16_within_budget(shape, cells):
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(19)
    vel = rng.uniform(1500.0, c, size=shape).astype(np.float32)
    state = synth.random_state(shape, cells, seed=20, **state_scales(h, dt))
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, storage="f16")
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    set_gpu_state(sim, state)
    sim.step(5)
    sim.sync()
    st = oracle_state(shape, state)
    O.run(oracle_grid(vel, h, dt, cells, c, R=1e-5), st, 5)
    e2, _ = rel_errors(sim.get("p").cpu().numpy(), st["p"])
    assert e2 <= 2e-2, e2


@pytest.mark.parametrize("shape,cells", [CASES[0], CASES[4]])
def test_degenerate_grid_blocked_equals_single_steps(shape, cells):
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(21)
    vel = torch.from_numpy(rng.uniform(1500.0, c, size=shape).astype(np.float32)).cuda()
    state = synth.random_state(shape, cells, seed=22, **state_scales(h, dt))
    out = []
    for k in (1, 2):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, tblock_k=k)
        sim.set_model(vel)
        sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(7)
        sim.sync()
        out.append({f: sim.get(f) for f in FIELDS})
    for f in FIELDS:
        assert torch.equal(out[0][f], out[1][f]), f


@pytest.mark.parametrize("shape,cells", CASES)
def test_degenerate_grid_staggered_and_local(shape, cells):
    """The staggered form and the local CPML grading on the same grids,
    random state, 7 steps, against the oracle's forms."""
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    rng = np.random.default_rng(23)
    vel = rng.uniform(1500.0, c, size=shape).astype(np.float32)
    vt = torch.from_numpy(vel).cuda()
    for form in ("staggered", "local"):
        dt = (0.4 if form == "staggered" else 0.5) * h / c
        state = synth.random_state(shape, cells, seed=24, **state_scales(h, dt))
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, cpml_local=form == "local")
        if form == "staggered":
            sim.set_staggered(True)
        sim.set_model(vt)
        if form == "local":
            sim.set_cpml_local(vt, R=1e-5)
        else:
            sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(7)
        sim.sync()
        v = vel.astype(np.float64)
        prof = O.make_profiles(shape, cells, h, dt, c if form == "staggered" else float(v.max()), R=1e-5)
        g = O.Grid(v * v, h, dt, prof, staggered=form == "staggered",
                   local=O.local_profiles(v, cells, h, dt, R=1e-5) if form == "local" else None)
        st = oracle_state(shape, state)
        O.run(g, st, 7)
        _check_all(gpu_fields(sim), st)


@pytest.mark.parametrize("shape,cells", [CASES[0], CASES[2], CASES[3], CASES[4]])
def test_degenerate_grid_adjoint_dot_product(shape, cells):
    """<F x, y> = <x, F^T y> through the library's adjoint on the degenerate
    grids (6 steps, checkpoints every 3)."""
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(25)
    vel = rng.uniform(1500.0, c, size=shape).astype(np.float32)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, checkpoint_every=3)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-4, c_ref=c)
    x = synth.random_state(shape, cells, seed=26, **state_scales(h, dt))
    y = synth.random_state(shape, cells, seed=27)
    for k in FIELDS:
        sim.set(k, torch.from_numpy(x[k]).cuda())
        sim.set("adj_" + k, torch.from_numpy(y[k]).cuda())
    sim.step(6)
    fx = {k: sim.get(k).cpu().numpy().astype(np.float64) for k in FIELDS}
    sim.adjoint(6)
    aty = {k: sim.get("adj_" + k).cpu().numpy().astype(np.float64) for k in FIELDS}
    lhs = sum(float(np.sum(fx[k] * y[k])) for k in FIELDS)
    rhs = sum(float(np.sum(x[k].astype(np.float64) * aty[k])) for k in FIELDS)
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)
