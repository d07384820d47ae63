"""Elliptic anisotropy through the C ABI against the FP64 oracle, and the
paper's 2D CPML demonstration (Sec. 5): 2 km x 2 km at 8 m, c_x = 2600 and
c_z = 1800 m/s, a 30 Hz Ricker source at the centre, a 10-cell layer.  With
the layer the field energy (sum of p^2 inside the layer) falls by about two
orders of magnitude within 1.5 s and keeps falling (a 2D wave leaves a slowly
decaying tail behind its front); with none the waves stay trapped."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, gpu_fields, rel_errors, set_gpu_state, state_scales

pytestmark = pytest.mark.gpu

KR3 = (2600.0 ** 2 / 1800.0 ** 2, 0.7, 1.0)


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def test_anisotropic_run_matches_oracle():
    Fdtd = _Fdtd()
    shape, cells = (40, 37, 45), (4, 5, 3, 6, 5, 4)
    h, c, nt = 8.0, 1800.0, 60
    dt = 0.4 * h / (c * math.sqrt(max(KR3)))
    vel = synth.layered_model(shape, seed=12, vmin=1400.0, vmax=c, amp_cells=2.0)
    src = np.array([[cells[4] + 4, 18, 22]], np.int32)
    wav = synth.ricker(nt, dt, 30.0).astype(np.float32)[None, :]
    rec = synth.receiver_grid(shape, cells, 3, 3, cells[4] + 1)
    c_ref = c * math.sqrt(max(KR3))
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_anisotropy(KR3)
    sim.set_cpml(R=1e-5, c_ref=c_ref)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = O.Grid(vel.astype(np.float64) ** 2, h, dt, O.make_profiles(shape, cells, h, dt, c_ref, R=1e-5), kr=KR3)
    st = O.State(shape)
    tro = O.run(g, st, nt, 0, tuple(src[0]), wav[0].astype(np.float64), rec)
    got = gpu_fields(sim)
    for k in FIELDS:
        e2, em = rel_errors(got[k], st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)
    e2, em = rel_errors(tr[0].cpu().numpy(), tro)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)


def test_unit_factors_equal_default_bitwise():
    Fdtd = _Fdtd()
    shape, cells, h, c = (30, 33, 36), (3, 4, 2, 3, 4, 2), 10.0, 2500.0
    dt = 0.5 * h / c
    vel = torch.from_numpy(synth.layered_model(shape, seed=3, vmin=1600.0, vmax=c)).cuda()
    state = synth.random_state(shape, cells, seed=14, **state_scales(h, dt))
    out = []
    for kr in (None, (1.0, 1.0, 1.0)):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=6)
        sim.set_model(vel)
        if kr is not None:
            sim.set_anisotropy(kr)
        sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(6)
        sim.sync()
        out.append({k: sim.get(k) for k in FIELDS})
    for k in FIELDS:
        assert torch.equal(out[0][k], out[1][k]), k


def test_2d_demo_energy_decay_and_oracle():
    from paper_2606_06910_gb300 import demos
    nt, every = 1000, 20
    sim_c, e_c, cfg, snap = demos.anisotropic_2d(True, nt, every, snap_at=200)
    _, e_n, _, _ = demos.anisotropic_2d(False, nt, every)
    peak_c, peak_n = e_c.max(), e_n.max()
    print(f"\n[2d demo] final / peak energy: CPML {e_c[-1] / peak_c:.3e}, no CPML {e_n[-1] / peak_n:.3e}")
    assert e_c[-1] / peak_c < 2e-2           # absorbed
    assert e_n[-1] / peak_n > 0.5            # trapped without a layer
    assert (e_n[-1] / peak_n) / (e_c[-1] / peak_c) > 50
    # after the front has left (0.7 s) the energy keeps falling (sum p^2 is
    # not conserved, so small exchanges with the kinetic part are allowed)
    after = e_c[int(0.7 / (every * cfg["dt"])):]
    assert after.max() <= 1.01 * after[0] and after[-1] < 0.5 * after[0]
    # the CPML run against the oracle: the final field and the energy curve
    shape, h, dt, L = cfg["shape"], cfg["h"], cfg["dt"], cfg["L"]
    cells = (L, L, 0, 0, L, L)
    g = O.Grid(np.full(shape, cfg["cz"] ** 2), h, dt, O.make_profiles(shape, cells, h, dt, cfg["cx"], R=1e-5),
               kr=cfg["kr"])
    st = O.State(shape)
    src = cfg["src"]
    z0, z1, y0, y1, x0, x1 = cfg["box"]
    e_o, p200 = [], None
    for k in range(nt // every):
        O.run(g, st, every, k * every, src, cfg["wav"][0].astype(np.float64))
        e_o.append(float(np.sum(st["p"][z0:z1, y0:y1, x0:x1] ** 2)))
        if (k + 1) * every == 200:
            p200 = st["p"].copy()
    e_o = np.array(e_o)
    # the wavefield in flight: the FP32 bar
    e2, em = rel_errors(snap, p200)
    print(f"[2d demo] p at 200 steps: rel L2 {e2:.2e}, max-abs rel {em:.2e}")
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
    # after absorption the field is a small residual: compared to the peak field
    sim_c.sync()
    d = np.max(np.abs(sim_c.get("p").cpu().numpy() - st["p"]))
    assert d <= 1e-5 * np.max(np.abs(p200)), (d, np.max(np.abs(p200)))
    assert np.max(np.abs(e_c - e_o) / e_o.max()) <= 1e-5


def test_anisotropy_errors():
    from paper_2606_06910_gb300 import _lib
    from paper_2606_06910_gb300.fdtd import FdtdError
    Fdtd = _Fdtd()
    shape = (16, 16, 16)
    h, c = 10.0, 2000.0
    sim = Fdtd(shape, h, 0.6 * h / c, cpml_cells=3, nt_max=4, checkpoint_every=2)
    sim.set_model(torch.full(shape, c, device="cuda"))
    with pytest.raises(FdtdError) as ei:
        sim.set_anisotropy((3.0, 1.0, 1.0))     # CFL 0.6 > 2 / (sqrt(5) 1.7307)
    assert ei.value.status == _lib.EUNSTABLE
    with pytest.raises(FdtdError) as ei:
        sim.set_anisotropy((1.0, 0.0, 1.0))
    assert ei.value.status == _lib.EINVAL
    sim.set_anisotropy((1.2, 1.0, 0.8))
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.step(4)
    sim.adjoint(4)          # the transpose of the anisotropic step is provided
    sim.sync()


@pytest.mark.parametrize("shape,cells,zchunk,kr", [
    ((37, 70, 75), (5, 6, 4, 7, 3, 5), 8, (1.7, 0.6, 1.2)),
    ((60, 100, 100), (4, 4, 5, 3, 4, 4), 16, (0.8, 1.4, 2.0)),
])
def test_anisotropic_adjoint_state_and_gradient_match_oracle(monkeypatch, shape, cells, zchunk, kr):
    """The fused adjoint of the anisotropic step after 5 steps against the
    oracle's transpose, field by field, and dJ/dc, on 3 x 3 and 4 x 4 tiles
    with ragged tails, six unequal layers and two shots (the 100 x 100 plane
    with 16-plane chunks has CTAs that run the interior form)."""
    monkeypatch.setenv("FDTD_ZCHUNK", str(zchunk))
    Fdtd = _Fdtd()
    h, c = 10.0, 2000.0
    dt = 0.35 * h / (c * math.sqrt(max(kr)))
    n, C, nshots = 5, 3, 2
    rng = np.random.default_rng(33)
    vel = rng.uniform(1500, c, size=shape).astype(np.float32)
    c_ref = c * math.sqrt(max(kr))
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, checkpoint_every=C)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_anisotropy(kr)
    sim.set_cpml(R=1e-4, c_ref=c_ref)
    g = O.Grid(vel.astype(np.float64) ** 2, h, dt, O.make_profiles(shape, cells, h, dt, c_ref, R=1e-4), kr=kr)
    refs = []
    for s in range(nshots):
        x = synth.random_state(shape, cells, seed=50 + s, **state_scales(h, dt))
        y = synth.random_state(shape, cells, seed=60 + s)
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


def test_anisotropic_cpml_profile_gradient_matches_oracle():
    """dJ/d(b, a, 1/kappa) per axis and node (the node-per-thread adjoint
    kernels) for an anisotropic misfit against the oracle."""
    Fdtd = _Fdtd()
    shape, cells, h, nt, C = (20, 18, 22), (3, 4, 2, 3, 4, 2), 10.0, 40, 15
    kr = (1.6, 0.7, 1.1)
    c_true = synth.layered_model(shape, seed=9, vmin=1800.0, vmax=2600.0, amp_cells=2.0)
    c0 = synth.gaussian_smooth(c_true, 2.0)
    dt = 0.4 * h / (2600.0 * math.sqrt(max(kr)))
    c_ref = 2600.0 * math.sqrt(max(kr))
    src = synth.shot_positions(shape, cells, 10, 1, z=cells[4] + 2)
    rec = synth.receiver_grid(shape, cells, 3, 3, cells[4] + 1)
    wav = synth.ricker(nt, dt, 35.0).astype(np.float32)[None, :]
    prof = O.make_profiles(shape, cells, h, dt, c_ref, R=1e-5)
    gt = O.Grid(c_true.astype(np.float64) ** 2, h, dt, prof, kr=kr)
    dobs = O.forward_traces(gt, nt, tuple(src[0]), wav[0].astype(np.float64), rec)[None].astype(np.float32)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec), checkpoint_every=C, cpml_grad=True)
    sim.set_model(torch.from_numpy(c0).cuda())
    sim.set_anisotropy(kr)
    sim.set_cpml(R=1e-5, c_ref=c_ref)
    sim.inject(src, torch.from_numpy(wav).cuda())
    sim.record(rec)
    sim.step(nt)
    d = torch.from_numpy(dobs).cuda()
    resid = torch.empty_like(d)
    sim.misfit(d, nt=nt, resid=resid)
    grad = torch.zeros(shape, device="cuda")
    gprof = torch.zeros((3, 3, max(shape)), device="cuda")
    sim.adjoint(nt, resid, grad, gprof)
    sim.sync()
    g0 = O.Grid(c0.astype(np.float64) ** 2, h, dt, prof, kr=kr)
    _, gK, gpo, _ = O.misfit_gradient(g0, nt, tuple(src[0]), wav[0].astype(np.float64), rec,
                                      dobs[0].astype(np.float64), checkpoint_every=C, want_profiles=True)
    gp = gprof.cpu().numpy()
    for dd in range(3):
        for coef in range(3):
            e2, em = rel_errors(gp[dd, coef], gpo[dd, coef])
            assert e2 <= 1e-3 and em <= 1e-3, (dd, coef, e2, em)
    e2, em = rel_errors(grad.cpu().numpy(), gK * 2.0 * c0.astype(np.float64))
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
