"""Pins of the oracle's misfit gradient (transposed step run backwards with
checkpoint + recompute) by central finite differences of the FP64 misfit and
by the dot-product identity.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


def _setup(seed=0, shape=(16, 15, 14), L=(3, 3, 4, 2, 3, 3), nt=60):
    h = 10.0
    rng = np.random.default_rng(seed)
    c_true = rng.uniform(1800, 2600, size=shape)
    c0 = np.full(shape, 2200.0)
    dt = 0.5 * h / 2600.0
    prof = O.make_profiles(shape, L, h, dt, 2600.0, R=1e-5)
    src = (shape[0] // 2, shape[1] // 2, shape[2] // 2)
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[4, 4, 5], [5, 10, 9], [11, 6, 4], [3, 11, 10], [12, 12, 11], [8, 3, 8]])
    dobs = O.forward_traces(O.Grid(c_true ** 2, h, dt, prof), nt, src, wav, rec)
    return h, dt, prof, src, wav, rec, dobs, c0, nt


def test_gradient_wrt_K_matches_central_differences():
    h, dt, prof, src, wav, rec, dobs, c0, nt = _setup()
    K0 = c0 ** 2
    J, gK, _, _ = O.misfit_gradient(O.Grid(K0, h, dt, prof), nt, src, wav, rec, dobs,
                                    checkpoint_every=13)
    rng = np.random.default_rng(1)
    nodes = [tuple(rng.integers(0, s) for s in K0.shape) for _ in range(6)]
    nodes += [(8, 7, 7), (0, 0, 0), (15, 14, 13)]   # near source, corners (slabs)
    for node in nodes:
        eps = 1e-4 * K0[node]
        Kp, Km = K0.copy(), K0.copy()
        Kp[node] += eps
        Km[node] -= eps
        Jp, _ = O.misfit(O.Grid(Kp, h, dt, prof), nt, src, wav, rec, dobs)
        Jm, _ = O.misfit(O.Grid(Km, h, dt, prof), nt, src, wav, rec, dobs)
        fd = (Jp - Jm) / (2 * eps)
        scale = np.max(np.abs(gK))
        assert abs(gK[node] - fd) <= 1e-6 * scale + 1e-5 * abs(fd), (node, gK[node], fd)


def test_gradient_independent_of_checkpoint_interval():
    h, dt, prof, src, wav, rec, dobs, c0, nt = _setup(seed=2, nt=40)
    g = O.Grid(c0 ** 2, h, dt, prof)
    J1, g1, p1, _ = O.misfit_gradient(g, nt, src, wav, rec, dobs, checkpoint_every=1,
                                      want_profiles=True)
    J2, g2, p2, _ = O.misfit_gradient(g, nt, src, wav, rec, dobs, checkpoint_every=17,
                                      want_profiles=True)
    assert J1 == J2
    assert np.array_equal(g1, g2)
    assert np.array_equal(p1, p2)


@pytest.mark.parametrize("coef", [0, 1, 2])
def test_gradient_wrt_cpml_profiles_matches_central_differences(coef):
    """dJ/d(b, a, 1/kappa) per axis and node index: the learned-CPML training
    signal.  b and a are shared by psi_v and psi_p (collocated nodes)."""
    h, dt, prof, src, wav, rec, dobs, c0, nt = _setup(seed=3, nt=50)
    K0 = c0 ** 2
    g = O.Grid(K0, h, dt, prof)
    _, _, gp, _ = O.misfit_gradient(g, nt, src, wav, rec, dobs, checkpoint_every=10,
                                    want_profiles=True)
    key = ("b", "a", "kinv")[coef]
    scale = np.max(np.abs(gp[:, coef, :]))
    checked = 0
    for d in range(3):
        pr = prof[d]
        for i in np.nonzero(pr["slab"])[0][:3]:
            base = pr[key][i]
            eps = 1e-5 * max(abs(base), 1e-3)
            vals = []
            for sgn in (1, -1):
                pp = [dict(q) for q in prof]
                pp[d] = dict(pp[d])
                arr = pp[d][key].copy()
                arr[i] = base + sgn * eps
                pp[d][key] = arr
                Jv, _ = O.misfit(O.Grid(K0, h, dt, pp), nt, src, wav, rec, dobs)
                vals.append(Jv)
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(gp[d, coef, i] - fd) <= 1e-6 * scale + 1e-4 * abs(fd), (d, i, gp[d, coef, i], fd)
            checked += 1
    assert checked == 9


def test_dot_product_identity_several_steps():
    """<F x, y> = <x, F^T y> for F = n full steps (no source), F^T = n
    transposed steps: relative mismatch at FP64 rounding."""
    shape = (10, 11, 12)
    L = (2, 3, 3, 2, 2, 3)
    h, c = 10.0, 2000.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(9)
    K = rng.uniform(1500, 2500, size=shape) ** 2
    g = O.Grid(K, h, dt, O.make_profiles(shape, L, h, dt, c, R=1e-5))
    xs = synth.random_state(shape, L, seed=21, v_scale=dt / h, psiv_scale=1 / h,
                            psip_scale=dt / h ** 2, dtype=np.float64)
    ys = synth.random_state(shape, L, seed=22, dtype=np.float64)
    x = O.State(shape)
    for k, v in xs.items():
        x[k] = v
    y = O.State(shape)
    for k, v in ys.items():
        y[k] = v
    fx = x.copy()
    O.run(g, fx, 6)
    aty = y.copy()
    for _ in range(6):
        O.adjoint_step(g, O.State(shape), aty)
    lhs = float(np.dot(fx.as_vector(), y.as_vector()))
    rhs = float(np.dot(x.as_vector(), aty.as_vector()))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
