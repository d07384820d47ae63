"""Temporal blocking (tblock_k = 2, 4): blocks of k steps over z bands give
the same state, node for node, as single steps, and hence the oracle's
result; checkpoints taken during blocked stepping feed the same adjoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2606_06910_gb300 import synth
from tests.parity_util import FIELDS, oracle_grid, rel_errors, state_scales

pytestmark = pytest.mark.gpu

ALL = FIELDS


def _Fdtd():
    from paper_2606_06910_gb300.fdtd import Fdtd
    return Fdtd


def _case(shape, cells, nshots, nt, seed):
    h, c = 10.0, 2600.0
    dt = 0.5 * h / c
    vel = synth.layered_model(shape, seed=seed, vmin=1800.0, vmax=c, amp_cells=2.0)
    src = synth.shot_positions(shape, cells, seed + 1, nshots, z=cells[4] + 3)
    wav = np.stack([synth.ricker(nt, dt, 20.0 + 5 * s) for s in range(nshots)]).astype(np.float32)
    rec = synth.receiver_grid(shape, cells, 5, 4, cells[4] + 1)
    # one receiver deep in the grid, so that traces cross band boundaries
    rec = np.concatenate([rec, [[shape[0] - cells[5] - 2, shape[1] // 2, shape[2] // 2]]]).astype(np.int32)
    return dict(shape=shape, cells=cells, nshots=nshots, nt=nt, h=h, dt=dt, c=c, vel=vel, src=src, wav=wav,
                rec=rec)


def _run(k, case, n, state=None, **kw):
    Fdtd = _Fdtd()
    sim = Fdtd(case["shape"], case["h"], case["dt"], nshots=case["nshots"], cpml_cells=case["cells"],
               nt_max=case["nt"], nrec_max=len(case["rec"]), tblock_k=k, **kw)
    sim.set_model(torch.from_numpy(case["vel"]).cuda())
    sim.set_cpml(R=1e-5, c_ref=case["c"])
    sim.inject(case["src"], torch.from_numpy(case["wav"]).cuda())
    traces = sim.record(case["rec"])
    if state is not None:
        for s in range(case["nshots"]):
            for f in FIELDS:
                sim.set(f, torch.from_numpy(state[s][f]).cuda(), s)
    return sim, traces


@pytest.mark.parametrize("k,band,storage", [(2, "8", "f32"), (4, "8", "f32"), (2, None, "f32"), (4, "11", "f32"),
                                            (2, "8", "bf16")])
def test_blocked_steps_equal_single_steps_bitwise(monkeypatch, k, band, storage):
    """45 x 70 x 75 (3 x 3 tiles with ragged tails; bands of 8 with a 13-plane
    last band, or of 11, or the default 48, which is one band here), unequal
    CPML layers, two shots with sources and receivers, a random initial
    state, and a step count that leaves single steps after the last whole
    block; FP32 and BF16 storage."""
    if band is not None:
        monkeypatch.setenv("FDTD_TBAND", band)
    case = _case((45, 70, 75), (4, 5, 3, 6, 5, 4), nshots=2, nt=24, seed=3)
    sc = state_scales(case["h"], case["dt"])
    state = [synth.random_state(case["shape"], case["cells"], seed=50 + s, **sc) for s in range(2)]
    n = 2 * k + 3
    ref, tr_ref = _run(1, case, n, state, storage=storage)
    ref.step(n)
    ref.sync()
    sim, tr = _run(k, case, n, state, storage=storage)
    sim.step(n)
    sim.sync()
    assert sim.time == n
    for s in range(2):
        for f in ALL:
            a, b = sim.get(f, s), ref.get(f, s)
            assert torch.equal(a, b), (k, s, f, float((a - b).abs().max()))
    assert torch.equal(tr, tr_ref)


def test_blocked_run_matches_oracle(monkeypatch):
    """k = 2 over 40 steps from rest against the FP64 oracle (fields and
    traces of shot 0), bands of 8 planes."""
    monkeypatch.setenv("FDTD_TBAND", "8")
    case = _case((41, 36, 40), (4, 4, 4, 4, 4, 4), nshots=1, nt=40, seed=7)
    sim, tr = _run(2, case, 40)
    sim.step(40)
    sim.sync()
    g = oracle_grid(case["vel"], case["h"], case["dt"], case["cells"], case["c"], R=1e-5)
    st = O.State(case["shape"])
    tro = O.run(g, st, 40, 0, tuple(case["src"][0]), case["wav"][0].astype(np.float64), case["rec"])
    for f in ALL:
        e2, em = rel_errors(sim.get(f).cpu().numpy(), st[f])
        assert e2 <= 1e-4 and em <= 1e-3, (f, e2, em)
    e2, em = rel_errors(tr[0].cpu().numpy(), tro)
    assert e2 <= 1e-4 and em <= 1e-3, (e2, em)


def test_blocked_forward_gives_the_same_checkpoints_and_gradient(monkeypatch):
    """k = 4 with checkpoints every 6 steps (blocks that would straddle a
    checkpoint run as single steps): the adjoint gradient equals the one of
    a k = 1 context bit for bit."""
    monkeypatch.setenv("FDTD_TBAND", "8")
    case = _case((34, 30, 36), (3, 3, 3, 3, 3, 3), nshots=2, nt=23, seed=11)
    grads = []
    for k in (1, 4):
        sim, tr = _run(k, case, case["nt"], checkpoint_every=6)
        sim.step(case["nt"])
        resid = tr.clone()
        grad = torch.zeros(case["shape"], device="cuda")
        sim.adjoint(case["nt"], resid, grad)
        sim.sync()
        grads.append(grad)
    assert float(grads[0].abs().max()) > 0
    assert torch.equal(grads[0], grads[1])
