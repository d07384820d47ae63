"""The staggered (Yee) form through the C ABI against the FP64 oracle's
staggered form: p at the nodes, v_d at the half nodes, staggered radius-4
derivatives, velocity CPML at half-node depths.  Runs from rest with sources
and receivers on ragged multi-tile grids, random states on grids large enough
for the interior form and several z chunks (every chunking gives the same
bits), temporal blocking, anisotropy, sampled nodes of the 512^3 layered
workload, and the restrictions of the form."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, gpu_fields, rel_errors, set_gpu_state, state_scales, subbox_point

pytestmark = pytest.mark.gpu


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _grid(vel, h, dt, cells, c_ref, R, kr=(1.0, 1.0, 1.0)):
    prof = O.make_profiles(vel.shape, cells, h, dt, c_ref, R=R)
    v = vel.astype(np.float64)
    return O.Grid(v * v, h, dt, prof, kr=kr, staggered=True)


@pytest.mark.parametrize("shape,cells,nshots", [((41, 38, 45), (4, 5, 3, 6, 5, 4), 1),
                                                ((23, 70, 37), (3, 3, 4, 4, 2, 5), 2)])
def test_staggered_run_matches_oracle(shape, cells, nshots):
    """80 steps from rest, a Ricker source per shot and a receiver grid:
    every field and the traces within the FP32 bar (rel L2 1e-4, max-abs
    rel 1e-3)."""
    Fdtd = _Fdtd()
    h, c, nt = 10.0, 2600.0, 80
    dt = 0.4 * h / c
    vel = synth.layered_model(shape, seed=5, vmin=1700.0, vmax=c, amp_cells=2.0)
    src = synth.shot_positions(shape, cells, 6, nshots, z=cells[4] + 3)
    wav = np.stack([synth.ricker(nt, dt, 25.0 + 5 * s) for s in range(nshots)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 3, 4, cells[4] + 1)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_staggered(True)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = _grid(vel, h, dt, cells, c, 1e-5)
    for s in range(nshots):
        st = O.State(shape)
        tro = O.run(g, st, nt, 0, tuple(src[s]), wav[s].astype(np.float64), rec)
        got = gpu_fields(sim, s)
        for k in FIELDS:
            e2, em = rel_errors(got[k], st[k])
            assert e2 <= 1e-4 and em <= 1e-3, (s, k, e2, em)
        e2, em = rel_errors(tr[s].cpu().numpy(), tro)
        assert e2 <= 1e-4 and em <= 1e-3, (s, e2, em)


def test_staggered_differs_from_collocated():
    """The same inputs through the collocated form land far from the
    staggered oracle: the parity above tests the form, not a shared path."""
    Fdtd = _Fdtd()
    shape, cells, h, c, nt = (30, 34, 36), (4,) * 6, 10.0, 2500.0, 40
    dt = 0.4 * h / c
    vel = synth.layered_model(shape, seed=8, vmin=1700.0, vmax=c)
    src = np.array([[10, 17, 18]], np.int32)
    wav = synth.ricker(nt, dt, 30.0).astype(np.float32)[None, :]
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    sim.step(nt)
    sim.sync()
    st = O.State(shape)
    O.run(_grid(vel, h, dt, cells, c, 1e-5), st, nt, 0, tuple(src[0]), wav[0].astype(np.float64))
    e2, _ = rel_errors(sim.get("p").cpu().numpy(), st["p"])
    assert e2 > 1e-2, e2


def test_staggered_chunkings_identical_and_match_oracle(monkeypatch):
    """100 x 96 x 100 (interior CTAs), 4 shots, random state, 10 steps: the
    default chunking equals uniform 7-plane chunks bit for bit and shot 0
    matches the oracle."""
    Fdtd = _Fdtd()
    shape, cells, nshots, n = (100, 96, 100), (4, 5, 4, 6, 5, 4), 4, 10
    h, c = 10.0, 2500.0
    dt = 0.42 * h / c
    vel = synth.layered_model(shape, seed=4, vmin=1600.0, vmax=c, amp_cells=2.0)
    state = synth.random_state(shape, cells, seed=72, **state_scales(h, dt))
    out = []
    for zc in (None, "7"):
        if zc is None:
            monkeypatch.delenv("FDTD_ZCHUNK", raising=False)
        else:
            monkeypatch.setenv("FDTD_ZCHUNK", zc)
        sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n)
        sim.set_staggered(True)
        sim.set_model(torch.from_numpy(vel).cuda())
        sim.set_cpml(R=1e-5, c_ref=c)
        for s in range(nshots):
            set_gpu_state(sim, state, s)
        sim.step(n)
        sim.sync()
        out.append({k: sim.get(k, 0) for k in FIELDS})
        for s in range(1, nshots):
            for k in FIELDS:
                assert torch.equal(sim.get(k, s), out[-1][k]), (s, k)
        del sim
    for k in FIELDS:
        assert torch.equal(out[0][k], out[1][k]), k
    st = O.State(shape)
    for k in FIELDS:
        st[k] = state[k].astype(np.float64)
    O.run(_grid(vel, h, dt, cells, c, 1e-5), st, n)
    for k in FIELDS:
        e2, em = rel_errors(out[0][k].cpu().numpy(), st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)


@pytest.mark.parametrize("k", [2, 4])
def test_staggered_blocked_equals_single_steps(monkeypatch, k):
    monkeypatch.setenv("FDTD_TBAND", "8")
    Fdtd = _Fdtd()
    shape, cells, h, c = (45, 70, 75), (4, 5, 3, 6, 5, 4), 10.0, 2600.0
    dt = 0.4 * h / c
    vel = torch.from_numpy(synth.layered_model(shape, seed=3, vmin=1800.0, vmax=c)).cuda()
    state = synth.random_state(shape, cells, seed=19, **state_scales(h, dt))
    n = 2 * k + 3
    out = []
    for kk in (1, k):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=n, tblock_k=kk)
        sim.set_staggered(True)
        sim.set_model(vel)
        sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(n)
        sim.sync()
        out.append({f: sim.get(f) for f in FIELDS})
    for f in FIELDS:
        assert torch.equal(out[0][f], out[1][f]), f


def test_staggered_anisotropic_matches_oracle():
    Fdtd = _Fdtd()
    shape, cells = (40, 37, 45), (4, 5, 3, 6, 5, 4)
    kr = (1.6, 0.7, 1.0)
    h, c, nt = 8.0, 1800.0, 60
    dt = 0.35 * h / (c * math.sqrt(max(kr)))
    vel = synth.layered_model(shape, seed=12, vmin=1400.0, vmax=c, amp_cells=2.0)
    src = np.array([[cells[4] + 4, 18, 22]], np.int32)
    wav = synth.ricker(nt, dt, 30.0).astype(np.float32)[None, :]
    c_ref = c * math.sqrt(max(kr))
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt)
    sim.set_staggered(True)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_anisotropy(kr)
    sim.set_cpml(R=1e-5, c_ref=c_ref)
    sim.inject(src, torch.from_numpy(wav).cuda())
    sim.step(nt)
    sim.sync()
    st = O.State(shape)
    O.run(_grid(vel, h, dt, cells, c_ref, 1e-5, kr=kr), st, nt, 0, tuple(src[0]), wav[0].astype(np.float64))
    got = gpu_fields(sim)
    for k in FIELDS:
        e2, em = rel_errors(got[k], st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)


def test_staggered_full_size_512_sampled_parity():
    """512^3 layered model with 20-cell layers (the benchmark's grid and
    launch configuration, dt at CFL 0.4): random state, 2 steps, every field
    at sampled nodes against the oracle on a sub-box around each node."""
    Fdtd = _Fdtd()
    w = synth.preset("layered512")
    shape, cells = w.shape, w.cpml_cells
    dt = 0.4 * w.h / w.c_max
    vel = w.velocity()
    state = synth.random_state(shape, cells, seed=13, **state_scales(w.h, dt))
    sim = Fdtd(shape, w.h, dt, cpml_cells=cells, nt_max=4)
    sim.set_staggered(True)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=w.R, c_ref=w.c_max)
    set_gpu_state(sim, state)
    nsteps = 2
    sim.step(nsteps)
    sim.sync()
    got = {k: sim.get(k).cpu().numpy() for k in FIELDS}
    rng = np.random.default_rng(1)
    pts = [(0, 0, 0), (511, 511, 511), (0, 511, 255), (19, 20, 21), (20, 19, 492), (491, 492, 19),
           (256, 256, 256), (255, 63, 64), (300, 15, 16), (100, 16, 511), (17, 300, 63), (490, 490, 490)]
    pts += [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(20)]
    pts += [tuple(int(v) for v in rng.integers(488, 512, 3)) for _ in range(6)]
    for p in pts:
        ref = subbox_point(state, vel, w.h, dt, cells, w.c_max, p, 8 * nsteps + 1, nsteps, R=w.R,
                           staggered=True)
        for k in FIELDS:
            r = ref[k]
            gv = got[k][p]
            scale = max(np.max(np.abs(state[k])), 1e-30)
            assert abs(gv - r) <= 1e-5 * scale + 1e-5 * abs(r), (p, k, gv, r)


def test_staggered_restrictions():
    from paper_2606_06910_gb300 import _lib
    from paper_2606_06910_gb300.fdtd import FdtdError
    Fdtd = _Fdtd()
    shape, h, c = (16, 16, 16), 10.0, 2000.0
    vel = torch.full(shape, c, device="cuda")

    def status(fn):
        with pytest.raises(FdtdError) as ei:
            fn()
        return ei.value.status

    # CFL 0.5: stable collocated, unstable staggered (limit 0.44884)
    sim = Fdtd(shape, h, 0.5 * h / c, cpml_cells=3, nt_max=4, checkpoint_every=2)
    sim.set_model(vel)
    assert status(lambda: sim.set_staggered(True)) == _lib.EUNSTABLE
    sim = Fdtd(shape, h, 0.44 * h / c, cpml_cells=3, nt_max=4, checkpoint_every=2)
    sim.set_staggered(True)
    sim.set_model(vel)
    sim.set_cpml(R=1e-5, c_ref=c)
    assert status(lambda: sim.set_model(vel, torch.full(shape, 2.0, device="cuda"))) == _lib.EUNSUPPORTED
    assert status(lambda: sim.set_cpml_ska(torch.ones(3, 3, device="cuda"))) == _lib.EUNSUPPORTED
    sim.step(2)
    assert status(lambda: sim.set_staggered(False)) == _lib.ESTATE
    sim.adjoint(2)          # the transpose of the staggered step is provided
    sim.sync()
    sim.reset()
    sim.set_staggered(False)
    assert status(lambda: Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4, storage="f16").set_staggered(True)) \
        == _lib.EUNSUPPORTED


def test_staggered_profile_gradient_is_unsupported():
    from paper_2606_06910_gb300 import _lib
    from paper_2606_06910_gb300.fdtd import FdtdError
    Fdtd = _Fdtd()
    shape, h, c = (16, 16, 16), 10.0, 2000.0
    sim = Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4, checkpoint_every=2, cpml_grad=True)
    sim.set_staggered(True)
    sim.set_model(torch.full(shape, c, device="cuda"))
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.step(2)
    with pytest.raises(FdtdError) as ei:
        sim.adjoint(2, None, None, torch.zeros((3, 3, 16), device="cuda"))
    assert ei.value.status == _lib.EUNSUPPORTED


@pytest.mark.parametrize("shape,cells,zchunk,kr", [((37, 70, 75), (5, 6, 4, 7, 3, 5), 8, (1.0, 1.0, 1.0)),
                                                   ((60, 100, 100), (4, 4, 5, 3, 4, 4), 16, (1.0, 1.0, 1.0)),
                                                   ((37, 70, 75), (5, 6, 4, 7, 3, 5), 8, (1.4, 0.7, 1.1))])
def test_staggered_adjoint_state_and_gradient_match_oracle(monkeypatch, shape, cells, zchunk, kr):
    """The fused adjoint of the staggered step (D+ on lam_h, D- on lam_g,
    half-node velocity profiles) after 5 steps against the oracle's
    transpose, field by field, and dJ/dc, on multi-tile grids with ragged
    tails and two shots (interior CTAs on the 100 x 100 plane; anisotropy in
    one case)."""
    monkeypatch.setenv("FDTD_ZCHUNK", str(zchunk))
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.38 * h / (c * math.sqrt(max(kr)))
    n, C, nshots = 5, 3, 2
    rng = np.random.default_rng(51)
    vel = rng.uniform(1500, c, size=shape).astype(np.float32)
    c_ref = c * math.sqrt(max(kr))
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, checkpoint_every=C)
    sim.set_staggered(True)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_anisotropy(kr)
    sim.set_cpml(R=1e-4, c_ref=c_ref)
    g = _grid(vel, h, dt, cells, c_ref, 1e-4, kr=kr)
    refs = []
    for s in range(nshots):
        x = synth.random_state(shape, cells, seed=110 + s, **state_scales(h, dt))
        y = synth.random_state(shape, cells, seed=120 + s)
        for k in FIELDS:
            sim.set(k, torch.from_numpy(x[k]).cuda(), s)
            sim.set("adj_" + k, torch.from_numpy(y[k]).cuda(), s)
        fwd = O.State(shape)
        for k in FIELDS:
            fwd[k] = x[k].astype(np.float64)
        starts = []
        for _ in range(n):
            starts.append(fwd.copy())
            O.run(g, fwd, 1)
        adj = O.State(shape)
        for k in FIELDS:
            adj[k] = y[k].astype(np.float64)
        gK = np.zeros(shape)
        for k in range(n - 1, -1, -1):
            O.adjoint_step(g, starts[k], adj, gK)
        refs.append((adj, gK))
    sim.step(n)
    grad = torch.zeros(shape, device="cuda")
    sim.adjoint(n, None, grad)
    sim.sync()
    for s in range(nshots):
        for k in FIELDS:
            e2, em = rel_errors(sim.get("adj_" + k, s).cpu().numpy(), refs[s][0][k])
            assert e2 <= 1e-4 and em <= 1e-3, (s, k, e2, em)
    gref = (refs[0][1] + refs[1][1]) * 2.0 * vel.astype(np.float64)
    e2, em = rel_errors(grad.cpu().numpy(), gref)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
