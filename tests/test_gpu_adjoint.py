"""The CUDA discrete adjoint (fdtd_adjoint_step_n, checkpoint + recompute)
against the FP64 oracle's gradient, the dot-product identity and finite
differences.  Gradient tolerance (FP32 path): relative L2 <= 1e-4 and
max-abs relative <= 1e-3, as for the forward fields."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, rel_errors, state_scales

pytestmark = pytest.mark.gpu

ADJ = ["adj_" + k for k in FIELDS]


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _rand_state(shape, cells, seed, h, dt):
    return synth.random_state(shape, cells, seed=seed, **state_scales(h, dt))


def test_dot_product_identity_fp32():
    """<F x, y> = <x, F^T y> for F = 7 steps with unequal CPML layers; the
    adjoint is applied by the library from checkpoints (C = 3)."""
    Fdtd = _Fdtd()
    shape, cells, h, c = (20, 18, 22), (3, 4, 2, 3, 4, 2), 10.0, 2500.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(4)
    vel = rng.uniform(1500, c, size=shape).astype(np.float32)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8, checkpoint_every=3)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-4, c_ref=c)
    x = _rand_state(shape, cells, 5, h, dt)
    y = synth.random_state(shape, cells, seed=6)
    for k in FIELDS:
        sim.set(k, torch.from_numpy(x[k]).cuda())
        sim.set("adj_" + k, torch.from_numpy(y[k]).cuda())
    n = 7
    sim.step(n)
    fx = {k: sim.get(k).cpu().numpy().astype(np.float64) for k in FIELDS}
    sim.adjoint(n)
    aty = {k: sim.get("adj_" + k).cpu().numpy().astype(np.float64) for k in FIELDS}
    lhs = sum(float(np.sum(fx[k] * y[k])) for k in FIELDS)
    rhs = sum(float(np.sum(x[k].astype(np.float64) * aty[k])) for k in FIELDS)
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _gradient_case(shape=(24, 22, 26), cells=(4,) * 6, nt=60, C=20, nshots=2, seed=7):
    h = 10.0
    c_true = synth.layered_model(shape, seed=seed, vmin=1800.0, vmax=2600.0, amp_cells=2.0)
    c0 = synth.gaussian_smooth(c_true, 2.0)
    dt = 0.5 * h / 2600.0
    src = synth.shot_positions(shape, cells, seed + 1, nshots, z=cells[4] + 2)
    rec = synth.receiver_grid(shape, cells, 3, 3, cells[4] + 1)
    wav = np.stack([synth.ricker(nt, dt, 35.0 + 5 * s) for s in range(nshots)]).astype(np.float32)
    # observed data: the oracle's traces in the true model (an input to both sides)
    gt = O.Grid(c_true.astype(np.float64) ** 2, h, dt, O.make_profiles(shape, cells, h, dt, 2600.0, R=1e-5))
    dobs = np.stack([O.forward_traces(gt, nt, tuple(src[s]), wav[s].astype(np.float64), rec)
                     for s in range(nshots)]).astype(np.float32)
    return dict(shape=shape, cells=cells, nt=nt, C=C, nshots=nshots, h=h, dt=dt, c0=c0, src=src, rec=rec,
                wav=wav, dobs=dobs)


def _gpu_gradient(case, cpml_grad=False):
    Fdtd = _Fdtd()
    k = case
    sim = Fdtd(k["shape"], k["h"], k["dt"], nshots=k["nshots"], cpml_cells=k["cells"], nt_max=k["nt"],
               nrec_max=len(k["rec"]), checkpoint_every=k["C"], cpml_grad=cpml_grad)
    sim.set_model(torch.from_numpy(k["c0"]).cuda())
    sim.set_cpml(R=1e-5, c_ref=2600.0)
    sim.inject(k["src"], torch.from_numpy(k["wav"]).cuda())
    sim.record(k["rec"])
    sim.step(k["nt"])
    dobs = torch.from_numpy(k["dobs"]).cuda()
    resid = torch.empty_like(dobs)
    J = sim.misfit(dobs, nt=k["nt"], resid=resid)
    grad = torch.zeros(k["shape"], device="cuda")
    gprof = torch.zeros((3, 3, max(k["shape"])), device="cuda") if cpml_grad else None
    sim.adjoint(k["nt"], resid, grad, gprof)
    sim.sync()
    return J, grad.cpu().numpy(), (gprof.cpu().numpy() if cpml_grad else None)


def _oracle_gradient(case, want_profiles=False):
    k = case
    g = O.Grid(k["c0"].astype(np.float64) ** 2, k["h"], k["dt"],
               O.make_profiles(k["shape"], k["cells"], k["h"], k["dt"], 2600.0, R=1e-5))
    J, gK, gp = 0.0, np.zeros(k["shape"]), np.zeros((3, 3, max(k["shape"])))
    for s in range(k["nshots"]):
        Js, gKs, gps, _ = O.misfit_gradient(g, k["nt"], tuple(k["src"][s]), k["wav"][s].astype(np.float64),
                                            k["rec"], k["dobs"][s].astype(np.float64), checkpoint_every=k["C"],
                                            want_profiles=want_profiles)
        J += Js
        gK += gKs
        if want_profiles:
            gp += gps
    # dJ/dc = dJ/dK * 2 rho c (rho = 1)
    return J, gK * 2.0 * k["c0"].astype(np.float64), gp


def test_velocity_gradient_matches_oracle():
    case = _gradient_case()
    J, g, _ = _gpu_gradient(case)
    Jo, go, _ = _oracle_gradient(case)
    assert abs(J - Jo) <= 1e-4 * Jo
    e2, em = rel_errors(g, go)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)


def test_cpml_profile_gradient_matches_oracle():
    case = _gradient_case(shape=(20, 18, 22), cells=(3, 4, 2, 3, 4, 2), nt=40, C=15, nshots=1, seed=9)
    _, _, gp = _gpu_gradient(case, cpml_grad=True)
    _, _, gpo = _oracle_gradient(case, want_profiles=True)
    for d in range(3):
        for coef in range(3):
            e2, em = rel_errors(gp[d, coef], gpo[d, coef])
            assert e2 <= 1e-3 and em <= 1e-3, (d, coef, e2, em)


def test_gradient_finite_differences_48():
    """48^3 layered instance of the gradient workload: central differences of
    the misfit (FP32 forward, FP64 reduction) at sampled nodes."""
    Fdtd = _Fdtd()
    w = synth.preset("adjoint48")
    shape, cells, nt = w.shape, w.cpml_cells, w.nt
    c_true = w.velocity()
    c0 = synth.gaussian_smooth(c_true, w.extra["smooth_sigma"])
    src = w.sources()
    rec = synth.receiver_grid(shape, cells, *w.extra["receivers"], z=cells[4])
    wav = np.tile(synth.ricker(nt, w.dt, 25.0)[None, :], (w.nshots, 1)).astype(np.float32)
    sim = Fdtd(shape, w.h, w.dt, nshots=w.nshots, cpml_cells=cells, nt_max=nt, nrec_max=len(rec),
               checkpoint_every=w.extra["checkpoint_every"])
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sim.inject(src, torch.from_numpy(wav).cuda())
    sim.record(rec)
    # observed data in the true model (the oracle's, cast to FP32)
    gt = O.Grid(c_true.astype(np.float64) ** 2, w.h, w.dt, O.make_profiles(shape, cells, w.h, w.dt, w.vmax, R=w.R))
    dobs = torch.from_numpy(np.stack([O.forward_traces(gt, nt, tuple(src[s]), wav[s].astype(np.float64), rec)
                                      for s in range(w.nshots)]).astype(np.float32)).cuda()

    def J_of(c):
        sim.reset()
        sim.set_model(torch.from_numpy(c).cuda())
        sim.step(nt)
        return sim.misfit(dobs, nt=nt)

    J0 = J_of(c0)
    resid = torch.empty_like(dobs)
    sim.misfit(dobs, nt=nt, resid=resid)
    grad = torch.zeros(shape, device="cuda")
    sim.adjoint(nt, resid, grad)
    g = grad.cpu().numpy()
    sim.reset()
    # nodes where the gradient is large (near sources / receivers)
    flat = np.argsort(np.abs(g).ravel())[::-1]
    nodes = [np.unravel_index(i, shape) for i in flat[:200:40]]
    for node in nodes:
        eps = 2e-3 * float(c0[node])
        cp, cm = c0.copy(), c0.copy()
        cp[node] += eps
        cm[node] -= eps
        fd = (J_of(cp) - J_of(cm)) / (2 * eps)
        assert abs(fd - g[node]) <= 0.02 * abs(g[node]) + 1e-3 * np.max(np.abs(g)), (node, fd, g[node], J0)


def test_autograd_function_matches_direct_adjoint():
    from paper_2606_06910_gb300.fdtd import FdtdFn
    Fdtd = _Fdtd()
    case = _gradient_case(shape=(22, 20, 24), nt=40, C=10, nshots=2, seed=11)
    k = case
    sim = Fdtd(k["shape"], k["h"], k["dt"], nshots=k["nshots"], cpml_cells=k["cells"], nt_max=k["nt"],
               nrec_max=len(k["rec"]), checkpoint_every=k["C"])
    sim.set_cpml(R=1e-5, c_ref=2600.0)
    sim.inject(k["src"], torch.from_numpy(k["wav"]).cuda())
    sim.record(k["rec"])
    vel = torch.from_numpy(k["c0"]).cuda().requires_grad_(True)
    dobs = torch.from_numpy(k["dobs"]).cuda()
    traces = FdtdFn.apply(vel, sim, k["nt"])
    loss = 0.5 * ((traces - dobs) ** 2).sum()
    loss.backward()
    J, g, _ = _gpu_gradient(case)
    assert abs(float(loss) - J) <= 1e-5 * J
    assert np.allclose(vel.grad.cpu().numpy(), g, rtol=1e-5, atol=1e-6 * np.max(np.abs(g)))


@pytest.mark.parametrize("shape,cells,zchunk", [
    ((37, 70, 75), (5, 6, 4, 7, 3, 5), None),
    ((37, 70, 75), (5, 6, 4, 7, 3, 5), 8),
    ((60, 100, 100), (4, 4, 5, 3, 4, 4), 16),
])
def test_adjoint_state_matches_oracle_multi_tile(monkeypatch, shape, cells, zchunk):
    """Adjoint state and dJ/dc after 5 steps against the oracle's transpose,
    field by field, on grids of 3 x 3 and 4 x 4 tiles with ragged x and y
    tails, six unequal layers and two shots; z in chunks of 8 (ragged last
    chunk), of 16, or the default chunking.  On the 100 x 100 plane with
    16-plane chunks some CTAs lie 8 nodes clear of every slab and edge and
    run the kernel's interior form."""
    if zchunk is not None:
        monkeypatch.setenv("FDTD_ZCHUNK", str(zchunk))
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    n, C, nshots = 5, 3, 2
    rng = np.random.default_rng(21)
    vel = rng.uniform(1500, c, size=shape).astype(np.float32)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, checkpoint_every=C)
    sim.set_model(torch.from_numpy(vel).cuda())
    sim.set_cpml(R=1e-4, c_ref=c)
    g = O.Grid(vel.astype(np.float64) ** 2, h, dt, O.make_profiles(shape, cells, h, dt, c, R=1e-4))
    refs = []
    for s in range(nshots):
        x = _rand_state(shape, cells, 30 + s, h, dt)
        y = synth.random_state(shape, cells, seed=40 + s)
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


def test_dot_product_identity_full_size_256x16():
    """The adjoint workload's grid and launch configuration (256^3, 20-cell
    layers, 16 shots): <F x, y> = <x, F^T y> over 6 steps with checkpoints
    every 3, for random x and y of every shot, generated on the device from a
    seeded generator; the sums are taken in FP64."""
    Fdtd = _Fdtd()
    w = synth.preset("adjoint256")
    shape, cells, nshots, n = w.shape, w.cpml_cells, w.nshots, 6
    sim = Fdtd(shape, w.h, w.dt, nshots=nshots, cpml_cells=cells, nt_max=8, checkpoint_every=3)
    sim.set_model(torch.from_numpy(w.velocity()).cuda())
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sc = state_scales(w.h, w.dt)
    scale = {"p": sc["p_scale"], "vx": sc["v_scale"], "vy": sc["v_scale"], "vz": sc["v_scale"]}
    gen = torch.Generator(device="cuda").manual_seed(2024)
    x, y = {}, {}
    for s in range(nshots):
        for k in FIELDS:
            f = scale.get(k, sc["psiv_scale"] if k.startswith("psiv") else sc["psip_scale"])
            sim.set(k, f * torch.randn(shape, device="cuda", generator=gen), s)
            sim.set("adj_" + k, torch.randn(shape, device="cuda", generator=gen), s)
            x[s, k] = sim.get(k, s).double()      # as stored (memory variables only in their slabs)
            y[s, k] = sim.get("adj_" + k, s).double()
    sim.step(n)
    lhs = sum(float(torch.sum(sim.get(k, s).double() * y[s, k])) for s in range(nshots) for k in FIELDS)
    del y
    sim.adjoint(n)
    rhs = sum(float(torch.sum(x[s, k] * sim.get("adj_" + k, s).double())) for s in range(nshots) for k in FIELDS)
    print(f"\n[adjoint 256^3 x 16] <Fx, y> = {lhs:.10e}, <x, F^T y> = {rhs:.10e}")
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)
