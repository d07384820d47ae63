"""Pins of the learned-CPML network oracle: closed forms, finite differences of
every derivative, the Adam first step.  CPU only."""
import math

import numpy as np

from oracle import mlp as M
from oracle import oracle as O


def test_parameter_count():
    assert M.NPARAM == 4 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 4675


def test_zero_weights_give_softplus_of_zero():
    theta = np.zeros(M.NPARAM)
    X = np.random.default_rng(0).standard_normal((5, 4))
    out, _ = M.forward(theta, X, 700.0, 30.0)
    ln2 = math.log(2.0)
    assert np.allclose(out[:, 0], 700.0 * ln2, rtol=1e-15)
    assert np.allclose(out[:, 1], 1.0 + ln2, rtol=1e-15)
    assert np.allclose(out[:, 2], 30.0 * ln2, rtol=1e-15)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = M.init_params(3)
    X = rng.standard_normal((7, 4))
    wout = rng.standard_normal((7, 3))
    s_sc, a_sc = 500.0, 20.0

    def J(t):
        out, _ = M.forward(t, X, s_sc, a_sc)
        return float(np.sum(wout * out))

    _, cache = M.forward(theta, X, s_sc, a_sc)
    g = M.backward(theta, cache, wout, s_sc, a_sc)
    idx = rng.choice(M.NPARAM, size=40, replace=False)
    idx = np.concatenate([idx, [0, 255, 256 + 63, 4675 - 1, 4675 - 4]])
    for i in idx:
        e = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += e
        tm[i] -= e
        fd = (J(tp) - J(tm)) / (2 * e)
        assert abs(fd - g[i]) <= 1e-6 * (abs(fd) + np.max(np.abs(g)) * 1e-3), (i, fd, g[i])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(50)
    grad = rng.standard_normal(50)
    lr, eps = 1e-2, 1e-8
    t1, m, v = M.adam_step(theta, grad, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    # bias-corrected moments of the first step are g and g^2
    assert np.allclose(t1, theta - lr * grad / (np.abs(grad) + eps), rtol=1e-14, atol=1e-16)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad * grad)


def test_coefficient_jacobian_values_and_derivatives():
    dt = 1.1e-3
    ska = np.array([[800.0, 4.0, 5.0], [120.0, 1.3, 40.0], [3.0, 1.0, 0.5]])
    b, a, kinv, J = M.coefficient_jacobian(ska[:, 0], ska[:, 1], ska[:, 2], dt)
    b0, a0, k0 = O.cpml_coefficients(ska[:, 0], ska[:, 1], ska[:, 2], dt)
    assert np.allclose(b, b0, rtol=1e-15) and np.allclose(a, a0, rtol=1e-14) and np.allclose(kinv, k0)
    for m in range(3):
        e = 1e-6 * np.maximum(np.abs(ska[:, m]), 1e-3)
        sp, sm = ska.copy(), ska.copy()
        sp[:, m] += e
        sm[:, m] -= e
        cp = np.stack(M.coefficient_jacobian(sp[:, 0], sp[:, 1], sp[:, 2], dt)[:3], -1)
        cm = np.stack(M.coefficient_jacobian(sm[:, 0], sm[:, 1], sm[:, 2], dt)[:3], -1)
        fd = (cp - cm) / (2 * e[:, None])
        assert np.allclose(J[:, :, m], fd, rtol=1e-6, atol=1e-12), m


def test_learned_misfit_gradient_matches_central_differences():
    """End to end: network -> (sigma, kappa, alpha) -> (b, a, 1/kappa) ->
    FDTD + CPML -> misfit, differentiated through the transposed steps."""
    from paper_2606_06910_gb300 import synth
    shape, L, h, c = (14, 14, 14), 3, 10.0, 2000.0
    dt = 0.5 * h / c
    nt = 40
    K = np.full(shape, c * c)
    feats = M.features(L, 6, 20.0, h, c, dt)
    s_sc, a_sc = c / h, 2 * math.pi * 20.0
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[7, 7, 4], [7, 4, 7], [4, 7, 7]])
    ref = np.zeros((nt, 3))                       # "no reflection" target
    shots = [((7, 7, 7), wav, rec, ref)]
    theta = M.init_params(5)
    J, g, _ = M.learned_misfit_gradient(theta, shape, L, dt, h, K, feats, s_sc, a_sc, shots, nt)

    def Jof(t):
        ska, _ = M.forward(t, feats, s_sc, a_sc)
        prof = M.learned_profiles(shape, L, ska, dt)
        return sum(O.misfit(O.Grid(K, h, dt, prof), nt, s, w, r, d)[0] for s, w, r, d in shots)

    assert abs(Jof(theta) - J) <= 1e-14 * abs(J)
    rng = np.random.default_rng(0)
    for i in list(rng.choice(M.NPARAM, 6, replace=False)) + [M.NPARAM - 1, M.NPARAM - 3]:
        e = 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[i] += e
        tm[i] -= e
        fd = (Jof(tp) - Jof(tm)) / (2 * e)
        assert abs(fd - g[i]) <= 1e-5 * (abs(fd) + 1e-3 * np.max(np.abs(g))), (i, fd, g[i])
