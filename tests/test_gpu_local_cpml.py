"""Local-velocity CPML grading through the C ABI against the FP64 oracle:
b, a per slab node from the velocity at that node (heterogeneous media).
Runs from rest with sources and receivers on ragged multi-tile grids with a
strong velocity contrast (with and without a density), random states with
the interior form and two chunkings, temporal blocking, sampled nodes of the
512^3 layered workload, the reduction to the 1D grading in a homogeneous
model, and the restrictions."""
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


def _grid(vel, h, dt, cells, R, rho=None):
    v = vel.astype(np.float64)
    prof = O.make_profiles(vel.shape, cells, h, dt, float(v.max()), R=R)
    lp = O.local_profiles(v, cells, h, dt, R=R)
    if rho is None:
        return O.Grid(v * v, h, dt, prof, local=lp)
    r = rho.astype(np.float64)
    return O.Grid(r * v * v, h, dt, prof, rho=r, local=lp)


@pytest.mark.parametrize("shape,cells,nshots,with_rho", [((41, 38, 45), (4, 5, 3, 6, 5, 4), 1, False),
                                                         ((23, 70, 37), (3, 3, 4, 4, 2, 5), 2, False),
                                                         ((41, 38, 45), (4, 5, 3, 6, 5, 4), 1, True)])
def test_local_grading_run_matches_oracle(shape, cells, nshots, with_rho):
    """80 steps from rest in a 1500-4500 m/s layered model: every field and
    the traces within the FP32 bar (rel L2 1e-4, max-abs rel 1e-3)."""
    Fdtd = _Fdtd()
    h, nt = 10.0, 80
    vel = synth.layered_model(shape, seed=9, vmin=1500.0, vmax=4500.0, amp_cells=2.0)
    dt = 0.5 * h / float(vel.max())
    rho = (vel / 1500.0) ** 0.25 if with_rho else None
    src = synth.shot_positions(shape, cells, 10, nshots, z=cells[4] + 3)
    wav = np.stack([synth.ricker(nt, dt, 25.0 + 5 * s) for s in range(nshots)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 3, 4, cells[4] + 1)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=nt, nrec_max=len(rec), cpml_local=True)
    vt = torch.from_numpy(vel).cuda()
    sim.set_model(vt, torch.from_numpy(rho.astype(np.float32)).cuda() if with_rho else None)
    sim.set_cpml_local(vt, R=1e-5)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = _grid(vel, h, dt, cells, 1e-5, rho)
    for s in range(nshots):
        st = O.State(shape)
        tro = O.run(g, st, nt, 0, tuple(src[s]), wav[s].astype(np.float64), rec)
        got = gpu_fields(sim, s)
        for k in FIELDS:
            e2, em = rel_errors(got[k], st[k])
            assert e2 <= 1e-4 and em <= 1e-3, (s, k, e2, em)
        e2, em = rel_errors(tr[s].cpu().numpy(), tro)
        assert e2 <= 1e-4 and em <= 1e-3, (s, e2, em)


def test_local_grading_differs_from_the_1d_grading():
    """In the layered model the 1D grading (c_ref = c_max) lands measurably
    away from the local oracle in the memory variables: the parity above
    tests the per-node tables."""
    Fdtd = _Fdtd()
    shape, cells, h, nt = (30, 34, 36), (4,) * 6, 10.0, 60
    vel = synth.layered_model(shape, seed=9, vmin=1500.0, vmax=4500.0, amp_cells=2.0)
    dt = 0.5 * h / float(vel.max())
    src = np.array([[10, 17, 18]], np.int32)
    wav = synth.ricker(nt, dt, 25.0).astype(np.float32)[None, :]
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-5, c_ref=float(vel.max()))
    sim.inject(src, torch.from_numpy(wav).cuda())
    sim.step(nt)
    sim.sync()
    st = O.State(shape)
    O.run(_grid(vel, h, dt, cells, 1e-5), st, nt, 0, tuple(src[0]), wav[0].astype(np.float64))
    e2, _ = rel_errors(sim.get("psiv_x").cpu().numpy(), st["psiv_x"])
    assert e2 > 1e-2, e2


def test_homogeneous_local_grading_matches_the_1d_grading():
    Fdtd = _Fdtd()
    shape, cells, h, c = (37, 40, 45), (5, 6, 4, 7, 3, 5), 10.0, 2500.0
    dt = 0.5 * h / c
    vel = torch.full(shape, c, device="cuda")
    state = synth.random_state(shape, cells, seed=15, **state_scales(h, dt))
    out = []
    for local in (False, True):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, cpml_local=True)
        sim.set_model(vel)
        if local:
            sim.set_cpml_local(vel, R=1e-5)
        else:
            sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(8)
        sim.sync()
        out.append({k: sim.get(k).cpu().numpy() for k in FIELDS})
    for k in FIELDS:
        e2, em = rel_errors(out[1][k], out[0][k])
        assert e2 <= 1e-6 and em <= 1e-5, (k, e2, em)


def test_local_grading_chunkings_identical_and_match_oracle(monkeypatch):
    """100 x 96 x 100 (interior CTAs), 4 shots, random state, 10 steps: the
    default chunking equals uniform 7-plane chunks bit for bit, the shots
    agree, and shot 0 matches the oracle."""
    Fdtd = _Fdtd()
    shape, cells, nshots, n = (100, 96, 100), (4, 5, 4, 6, 5, 4), 4, 10
    h = 10.0
    vel = synth.layered_model(shape, seed=4, vmin=1500.0, vmax=4500.0, amp_cells=2.0)
    dt = 0.5 * h / float(vel.max())
    state = synth.random_state(shape, cells, seed=73, **state_scales(h, dt))
    vt = torch.from_numpy(vel).cuda()
    out = []
    for zc in (None, "7"):
        if zc is None:
            monkeypatch.delenv("FDTD_ZCHUNK", raising=False)
        else:
            monkeypatch.setenv("FDTD_ZCHUNK", zc)
        sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, cpml_local=True)
        sim.set_model(vt)
        sim.set_cpml_local(vt, R=1e-5)
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
    O.run(_grid(vel, h, dt, cells, 1e-5), st, n)
    for k in FIELDS:
        e2, em = rel_errors(out[0][k].cpu().numpy(), st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)


def test_local_grading_blocked_equals_single_steps(monkeypatch):
    monkeypatch.setenv("FDTD_TBAND", "8")
    Fdtd = _Fdtd()
    shape, cells, h = (45, 70, 75), (4, 5, 3, 6, 5, 4), 10.0
    vel = synth.layered_model(shape, seed=3, vmin=1500.0, vmax=4500.0)
    dt = 0.5 * h / float(vel.max())
    vt = torch.from_numpy(vel).cuda()
    state = synth.random_state(shape, cells, seed=21, **state_scales(h, dt))
    out = []
    for k in (1, 4):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=11, tblock_k=k, cpml_local=True)
        sim.set_model(vt)
        sim.set_cpml_local(vt, R=1e-5)
        set_gpu_state(sim, state)
        sim.step(11)
        sim.sync()
        out.append({f: sim.get(f) for f in FIELDS})
    for f in FIELDS:
        assert torch.equal(out[0][f], out[1][f]), f


def test_local_grading_full_size_512_sampled_parity():
    """512^3 layered model (1500-4500 m/s) with 20-cell layers graded from
    the local velocity, in the benchmark's launch configuration: random
    state, 2 steps, every field at sampled nodes against the oracle on a
    sub-box around each node (the sub-box keeps the full grid's depths)."""
    Fdtd = _Fdtd()
    w = synth.preset("layered512")
    shape, cells = w.shape, w.cpml_cells
    vel = w.velocity()
    vt = torch.from_numpy(vel).cuda()
    state = synth.random_state(shape, cells, seed=14, **state_scales(w.h, w.dt))
    sim = Fdtd(shape, w.h, w.dt, cpml_cells=cells, nt_max=4, cpml_local=True)
    sim.set_model(vt)
    sim.set_cpml_local(vt, R=w.R)
    set_gpu_state(sim, state)
    nsteps = 2
    sim.step(nsteps)
    sim.sync()
    got = {k: sim.get(k).cpu().numpy() for k in FIELDS}
    rng = np.random.default_rng(2)
    pts = [(0, 0, 0), (511, 511, 511), (0, 511, 255), (19, 20, 21), (20, 19, 492), (491, 492, 19),
           (256, 256, 256), (255, 63, 64), (300, 15, 16), (100, 16, 511), (17, 300, 63), (505, 3, 250)]
    pts += [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(18)]
    pts += [tuple(int(v) for v in rng.integers(0, 24, 3)) for _ in range(4)]
    pts += [tuple(int(v) for v in rng.integers(488, 512, 3)) for _ in range(4)]
    for p in pts:
        ref = subbox_point(state, vel, w.h, w.dt, cells, w.c_max, p, 8 * nsteps + 1, nsteps, R=w.R, local=True)
        for k in FIELDS:
            r = ref[k]
            gv = got[k][p]
            scale = max(np.max(np.abs(state[k])), 1e-30)
            assert abs(gv - r) <= 1e-5 * scale + 1e-5 * abs(r), (p, k, gv, r)


def test_local_grading_restrictions():
    from paper_2606_06910_gb300 import _lib
    from paper_2606_06910_gb300.fdtd import FdtdError
    Fdtd = _Fdtd()
    shape, h, c = (16, 16, 16), 10.0, 2000.0
    vel = torch.full(shape, c, device="cuda")

    def status(fn):
        with pytest.raises(FdtdError) as ei:
            fn()
        return ei.value.status

    plain = Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4)
    plain.set_model(vel)
    assert status(lambda: plain.set_cpml_local(vel)) == _lib.ESTATE
    sim = Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4, checkpoint_every=2, cpml_local=True, cpml_grad=True)
    assert status(lambda: sim.set_cpml_local(vel)) == _lib.ESTATE          # no model yet
    sim.set_model(vel)
    bad = vel.clone()
    bad[0, 5, 5] = -1.0
    assert status(lambda: sim.set_cpml_local(bad)) == _lib.EINVAL
    sim.set_cpml_local(vel, R=1e-5)
    assert status(lambda: sim.set_staggered(True)) == _lib.EUNSUPPORTED
    sim.step(2)
    gprof = torch.zeros((3, 3, 16), device="cuda")
    assert status(lambda: sim.adjoint(2, None, None, gprof)) == _lib.EUNSUPPORTED   # per axis and node index
    sim.adjoint(2)          # the transpose with per-node coefficients is provided
    sim.sync()
    st = Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4, cpml_local=True)
    st.set_staggered(True)
    st.set_model(vel)
    assert status(lambda: st.set_cpml_local(vel)) == _lib.EUNSUPPORTED
    f16 = Fdtd(shape, h, 0.4 * h / c, cpml_cells=3, nt_max=4, cpml_local=True, storage="f16")
    f16.set_model(vel)
    assert status(lambda: f16.set_cpml_local(vel)) == _lib.EUNSUPPORTED


@pytest.mark.parametrize("shape,cells,zchunk,with_rho", [((37, 70, 75), (5, 6, 4, 7, 3, 5), 8, False),
                                                         ((60, 100, 100), (4, 4, 5, 3, 4, 4), 16, False),
                                                         ((37, 70, 75), (5, 6, 4, 7, 3, 5), 8, True)])
def test_local_grading_adjoint_state_and_gradient_match_oracle(monkeypatch, shape, cells, zchunk, with_rho):
    """The fused adjoint with the per-node (b, a) of the local grading (and a
    density in one case) after 5 steps against the oracle's transpose, field
    by field, and dJ/dc at fixed coefficients, on multi-tile grids with
    ragged tails and two shots (interior CTAs on the 100 x 100 plane)."""
    monkeypatch.setenv("FDTD_ZCHUNK", str(zchunk))
    Fdtd = _Fdtd()
    h = 10.0
    n, C, nshots = 5, 3, 2
    vel = synth.layered_model(shape, seed=13, vmin=1500.0, vmax=4500.0, amp_cells=2.0)
    dt = 0.5 * h / float(vel.max())
    rho = ((vel / 1500.0) ** 0.25).astype(np.float32) if with_rho else None
    vt = torch.from_numpy(vel).cuda()
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, checkpoint_every=C, cpml_local=True)
    sim.set_model(vt, torch.from_numpy(rho).cuda() if with_rho else None)
    sim.set_cpml_local(vt, R=1e-4)
    g = _grid(vel, h, dt, cells, 1e-4, rho)
    refs = []
    for s in range(nshots):
        x = synth.random_state(shape, cells, seed=90 + s, **state_scales(h, dt))
        y = synth.random_state(shape, cells, seed=95 + s)
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
    r = rho.astype(np.float64) if with_rho else 1.0
    gref = (refs[0][1] + refs[1][1]) * 2.0 * r * vel.astype(np.float64)
    e2, em = rel_errors(grad.cpu().numpy(), gref)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
