"""Variable density (density per node, collocated with p and v) through the C
ABI against the FP64 oracle; density 1 everywhere against the constant-density
form bit for bit; the chunkings with the interior form; 16-bit storage."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, gpu_fields, oracle_grid, rel_errors, set_gpu_state, state_scales

pytestmark = pytest.mark.gpu


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _density(shape, seed):
    """A smooth seeded density field between about 0.8 and 2.6 with two
    layer-like jumps (the layered generator's interfaces)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    base = synth.layered_model(shape, seed=seed, n_layers=3, vmin=1.0, vmax=2.2, amp_cells=2.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wob = 0.25 * np.sin(2 * np.pi * (x / nx + rng.uniform())) * np.cos(2 * np.pi * (y / ny + rng.uniform()))
    return (base + wob + 0.3 * np.sin(2 * np.pi * z / nz)).astype(np.float32)


def _oracle_grid(vel, rho, h, dt, cells, c_ref, R):
    prof = O.make_profiles(vel.shape, cells, h, dt, c_ref, R=R)
    v = vel.astype(np.float64)
    r = rho.astype(np.float64)
    return O.Grid(r * v * v, h, dt, prof, rho=r)


@pytest.mark.parametrize("shape,cells", [((41, 38, 45), (4, 5, 3, 6, 5, 4)), ((23, 70, 37), (3, 3, 4, 4, 2, 5))])
def test_variable_density_run_matches_oracle(shape, cells):
    """60 steps from rest with a source and receivers; every field and the
    traces within the FP32 tolerance (rel L2 1e-4, max-abs rel 1e-3)."""
    Fdtd = _Fdtd()
    h, c, nt = 10.0, 2600.0, 60
    dt = 0.5 * h / c
    vel = synth.layered_model(shape, seed=5, vmin=1700.0, vmax=c, amp_cells=2.0)
    rho = _density(shape, 6)
    src = np.array([[cells[4] + 3, shape[1] // 2, shape[2] // 2]], np.int32)
    wav = synth.ricker(nt, dt, 30.0).astype(np.float32)[None, :]
    rec = synth.receiver_grid(shape, cells, 3, 4, cells[4] + 1)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec))
    sim.set_model(torch.from_numpy(vel).cuda(), torch.from_numpy(rho).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = _oracle_grid(vel, rho, h, dt, cells, c, 1e-5)
    st = O.State(shape)
    tro = O.run(g, st, nt, 0, tuple(src[0]), wav[0].astype(np.float64), rec)
    got = gpu_fields(sim)
    for k in FIELDS:
        e2, em = rel_errors(got[k], st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)
    e2, em = rel_errors(tr[0].cpu().numpy(), tro)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)


def test_unit_density_equals_constant_density_bitwise():
    """A density array of ones runs the variable-density form with factors
    equal to the constant form's, so every field matches bit for bit."""
    Fdtd = _Fdtd()
    shape, cells, h, c = (37, 70, 75), (5, 6, 4, 7, 3, 5), 10.0, 2500.0
    dt = 0.5 * h / c
    vel = torch.from_numpy(synth.layered_model(shape, seed=2, vmin=1600.0, vmax=c)).cuda()
    state = synth.random_state(shape, cells, seed=9, **state_scales(h, dt))
    out = []
    for rho in (None, torch.ones(shape, device="cuda")):
        sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=8)
        sim.set_model(vel, rho)
        sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state)
        sim.step(8)
        sim.sync()
        out.append({k: sim.get(k) for k in FIELDS})
    for k in FIELDS:
        assert torch.equal(out[0][k], out[1][k]), k


def test_variable_density_chunkings_identical_and_match_oracle(monkeypatch):
    """100 x 96 x 100, 24 shots (large enough for the interior form): the
    default chunking equals uniform 7-plane chunks bit for bit, and shot 0
    matches the oracle after 12 steps from a random state."""
    Fdtd = _Fdtd()
    shape, cells, nshots, n = (100, 96, 100), (4, 5, 4, 6, 5, 4), 24, 12
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    vel = synth.layered_model(shape, seed=4, vmin=1600.0, vmax=c, amp_cells=2.0)
    rho = _density(shape, 8)
    state = synth.random_state(shape, cells, seed=71, **state_scales(h, dt))
    out = []
    for zc in (None, "7"):
        if zc is None:
            monkeypatch.delenv("FDTD_ZCHUNK", raising=False)
        else:
            monkeypatch.setenv("FDTD_ZCHUNK", zc)
        sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n)
        sim.set_model(torch.from_numpy(vel).cuda(), torch.from_numpy(rho).cuda())
        sim.set_cpml(R=1e-5, c_ref=c)
        set_gpu_state(sim, state, 0)
        sim.step(n)
        sim.sync()
        out.append({k: sim.get(k, 0) for k in FIELDS})
        del sim
    for k in FIELDS:
        assert torch.equal(out[0][k], out[1][k]), k
    g = _oracle_grid(vel, rho, h, dt, cells, c, 1e-5)
    st = O.State(shape)
    for k in FIELDS:
        st[k] = state[k].astype(np.float64)
    O.run(g, st, n)
    for k in FIELDS:
        e2, em = rel_errors(out[0][k].cpu().numpy(), st[k])
        assert e2 <= 1e-4 and em <= 1e-3, (k, e2, em)


def test_variable_density_fp16_storage_within_budget():
    """FP16 storage with a density, 120 steps of a source run against the
    oracle: relative L2 of p and traces within the 16-bit budget 2e-2."""
    Fdtd = _Fdtd()
    shape, cells, h, c, nt = (48, 52, 56), (6, 6, 6, 6, 6, 6), 10.0, 2600.0, 120
    dt = 0.5 * h / c
    vel = synth.layered_model(shape, seed=3, vmin=1700.0, vmax=c, amp_cells=2.0)
    rho = _density(shape, 4)
    src = np.array([[12, 26, 28]], np.int32)
    wav = synth.ricker(nt, dt, 25.0).astype(np.float32)[None, :]
    rec = synth.receiver_grid(shape, cells, 4, 4, 8)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec), storage="f16")
    sim.set_model(torch.from_numpy(vel).cuda(), torch.from_numpy(rho).cuda())
    sim.set_cpml(R=1e-5, c_ref=c)
    sim.inject(src, torch.from_numpy(wav).cuda())
    tr = sim.record(rec)
    sim.step(nt)
    sim.sync()
    g = _oracle_grid(vel, rho, h, dt, cells, c, 1e-5)
    st = O.State(shape)
    tro = O.run(g, st, nt, 0, tuple(src[0]), wav[0].astype(np.float64), rec)
    e_p, _ = rel_errors(sim.get("p").cpu().numpy(), st["p"])
    e_t, _ = rel_errors(tr[0].cpu().numpy(), tro)
    print(f"\n[density fp16] rel L2 p {e_p:.3e}, traces {e_t:.3e}")
    assert e_p <= 2e-2 and e_t <= 2e-2


def test_nonpositive_density_is_rejected():
    from paper_2606_06910_gb300.fdtd import FdtdError
    from paper_2606_06910_gb300 import _lib
    Fdtd = _Fdtd()
    shape = (16, 16, 16)
    sim = Fdtd(shape, 10.0, 1e-3, cpml_cells=3, nt_max=4, checkpoint_every=2)
    with pytest.raises(FdtdError) as ei:
        sim.set_model(torch.full(shape, 2000.0, device="cuda"), torch.zeros(shape, device="cuda"))
    assert ei.value.status == _lib.EINVAL


@pytest.mark.parametrize("shape,cells,zchunk", [((37, 70, 75), (5, 6, 4, 7, 3, 5), 8),
                                                ((60, 100, 100), (4, 4, 5, 3, 4, 4), 16)])
def test_density_adjoint_state_and_gradient_match_oracle(monkeypatch, shape, cells, zchunk):
    """The fused adjoint with a density (-dt/rho per node in the velocity
    transpose) after 5 steps against the oracle's transpose, field by field,
    and dJ/dc = 2 rho c dJ/dK, on 3 x 3 and 4 x 4 tiles with ragged tails,
    six unequal layers and two shots (the 100 x 100 plane with 16-plane
    chunks has CTAs that run the interior form)."""
    monkeypatch.setenv("FDTD_ZCHUNK", str(zchunk))
    Fdtd = _Fdtd()
    h, c = 10.0, 2500.0
    dt = 0.5 * h / c
    n, C, nshots = 5, 3, 2
    rng = np.random.default_rng(41)
    vel = rng.uniform(1500, c, size=shape).astype(np.float32)
    rho = _density(shape, 12)
    sim = Fdtd(shape, h, dt, nshots=nshots, cpml_cells=cells, nt_max=n, checkpoint_every=C)
    sim.set_model(torch.from_numpy(vel).cuda(), torch.from_numpy(rho).cuda())
    sim.set_cpml(R=1e-4, c_ref=c)
    g = _oracle_grid(vel, rho, h, dt, cells, c, 1e-4)
    refs = []
    for s in range(nshots):
        x = synth.random_state(shape, cells, seed=70 + s, **state_scales(h, dt))
        y = synth.random_state(shape, cells, seed=80 + s)
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
    gref = (refs[0][1] + refs[1][1]) * 2.0 * rho.astype(np.float64) * vel.astype(np.float64)
    e2, em = rel_errors(grad.cpu().numpy(), gref)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)


def test_density_cpml_profile_gradient_and_misfit_gradient_match_oracle():
    """A source run with a density: dJ/dc and dJ/d(b, a, 1/kappa) (the
    node-per-thread adjoint kernels) against the oracle's misfit gradient."""
    Fdtd = _Fdtd()
    shape, cells, h, nt, C = (20, 18, 22), (3, 4, 2, 3, 4, 2), 10.0, 40, 15
    c_true = synth.layered_model(shape, seed=9, vmin=1800.0, vmax=2600.0, amp_cells=2.0)
    c0 = synth.gaussian_smooth(c_true, 2.0)
    rho = _density(shape, 14)
    dt = 0.5 * h / 2600.0
    src = synth.shot_positions(shape, cells, 10, 1, z=cells[4] + 2)
    rec = synth.receiver_grid(shape, cells, 3, 3, cells[4] + 1)
    wav = synth.ricker(nt, dt, 35.0).astype(np.float32)[None, :]
    gt = _oracle_grid(c_true, rho, h, dt, cells, 2600.0, 1e-5)
    dobs = O.forward_traces(gt, nt, tuple(src[0]), wav[0].astype(np.float64), rec)[None].astype(np.float32)
    sim = Fdtd(shape, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec), checkpoint_every=C, cpml_grad=True)
    sim.set_model(torch.from_numpy(c0).cuda(), torch.from_numpy(rho).cuda())
    sim.set_cpml(R=1e-5, c_ref=2600.0)
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
    g0 = _oracle_grid(c0, rho, h, dt, cells, 2600.0, 1e-5)
    _, gK, gpo, _ = O.misfit_gradient(g0, nt, tuple(src[0]), wav[0].astype(np.float64), rec,
                                      dobs[0].astype(np.float64), checkpoint_every=C, want_profiles=True)
    gp = gprof.cpu().numpy()
    for dd in range(3):
        for coef in range(3):
            e2, em = rel_errors(gp[dd, coef], gpo[dd, coef])
            assert e2 <= 1e-3 and em <= 1e-3, (dd, coef, e2, em)
    e2, em = rel_errors(grad.cpu().numpy(), gK * 2.0 * rho.astype(np.float64) * c0.astype(np.float64))
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)
