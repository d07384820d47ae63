"""Pins of the oracle's elliptic anisotropy (the acoustic system of the
paper's 2D CPML demonstration, Sec. 5: axis velocities c_x = 2600 and
c_z = 1800 m/s).  The pressure update weights the derivative along axis d by
kr_d = (c_d / c)^2, so a plane standing wave obeys the discrete dispersion
relation sin(omega dt / 2) = (c dt / 2) sqrt(sum_d kr_d Dhat_d^2 / h^2), and
the energy 1/2 sum_d kr_d rho |v_d|^2 + 1/2 sum p p' / K is conserved.
CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_06910_gb300 import synth

KR = (2600.0 ** 2 / 1800.0 ** 2, 0.7, 1.0)


@pytest.mark.parametrize("m", [(1, 2, 3), (2, 1, 1)])
def test_anisotropic_dispersion_relation_exact(m):
    shape = (12, 10, 16)
    h, c, rho = 8.0, 1800.0, 1.3
    dt = 0.3 * h / c
    K = rho * c * c * np.ones(shape)
    st, phi, _ = O.standing_wave_state(shape, m, h, dt, rho)
    nz, ny, nx = shape
    th = [2 * np.pi * m[2] / nx, 2 * np.pi * m[1] / ny, 2 * np.pi * m[0] / nz]
    lam2 = sum(kr * (O.symbol(t) / h) ** 2 for kr, t in zip(KR, th))
    g = O.Grid(K, h, dt, rho=rho, periodic=True, kr=KR)
    nsteps = 41
    O.run(g, st, nsteps)
    omega_h = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2))
    err = np.max(np.abs(st["p"] - phi * math.cos(omega_h * nsteps * dt)))
    assert err < 1e-12, err
    # the isotropic relation is visibly off for the same run
    lam2_iso = sum((O.symbol(t) / h) ** 2 for t in th)
    omega_iso = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2_iso))
    assert np.max(np.abs(st["p"] - phi * math.cos(omega_iso * nsteps * dt))) > 1e-3


def test_anisotropic_energy_conserved():
    rng = np.random.default_rng(5)
    shape = (11, 12, 13)
    h, rho = 8.0, 1.0
    c = rng.uniform(1500, 1800, size=shape)
    K = rho * c * c
    dt = 0.3 * h / (c.max() * math.sqrt(max(KR)))
    g = O.Grid(K, h, dt, rho=rho, periodic=True, kr=KR)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    energies, plain = [], []
    g_iso = O.Grid(K, h, dt, rho=rho, periodic=True)
    for _ in range(25):
        p_n = st["p"].copy()
        O.run(g, st, 1)
        v = [st["vx"], st["vy"], st["vz"]]
        energies.append(O.staggered_energy(g, p_n, st["p"], v))
        plain.append(O.staggered_energy(g_iso, p_n, st["p"], v))
    e, ep = np.array(energies), np.array(plain)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) < 1e-12
    # without the kr weights the quantity is not invariant
    assert np.max(np.abs(ep - ep[0])) / abs(ep[0]) > 1e-4


def test_unit_factors_equal_isotropic_grid():
    rng = np.random.default_rng(2)
    shape = (9, 8, 10)
    h, c = 10.0, 2000.0
    dt = 0.5 * h / c
    prof = O.make_profiles(shape, (2, 3, 2, 2, 3, 2), h, dt, c, R=1e-5)
    K = np.full(shape, c * c)
    p0 = rng.standard_normal(shape)
    out = []
    for kr in (None, (1.0, 1.0, 1.0)):
        st = O.State(shape)
        st["p"] = p0
        g = O.Grid(K, h, dt, prof) if kr is None else O.Grid(K, h, dt, prof, kr=kr)
        O.run(g, st, 6)
        out.append(st)
    for k in O.FIELDS:
        assert np.array_equal(out[0][k], out[1][k]), k


def _aniso_adjoint_case(kr_adj=None):
    shape = (10, 11, 12)
    L = (2, 3, 3, 2, 2, 3)
    h, c = 10.0, 2000.0
    kr = (1.7, 0.6, 1.2)
    dt = 0.35 * h / (c * np.sqrt(max(kr)))
    rng = np.random.default_rng(19)
    K = rng.uniform(1500, 2500, size=shape) ** 2
    prof = O.make_profiles(shape, L, h, dt, c * np.sqrt(max(kr)), R=1e-5)
    g = O.Grid(K, h, dt, prof, kr=kr)
    ga = g if kr_adj is None else O.Grid(K, h, dt, prof, kr=kr_adj)
    xs = synth.random_state(shape, L, seed=23, v_scale=dt / h, psiv_scale=1 / h,
                            psip_scale=dt / h ** 2, dtype=np.float64)
    ys = synth.random_state(shape, L, seed=24, dtype=np.float64)
    x = O.State(shape)
    y = O.State(shape)
    for k in O.FIELDS:
        x[k] = xs[k]
        y[k] = ys[k]
    fx = x.copy()
    O.run(g, fx, 6)
    aty = y.copy()
    for _ in range(6):
        O.adjoint_step(ga, O.State(shape), aty)
    lhs = float(np.dot(fx.as_vector(), y.as_vector()))
    rhs = float(np.dot(x.as_vector(), aty.as_vector()))
    return lhs, rhs


def test_anisotropic_dot_product_identity():
    """<F x, y> = <x, F^T y> over 6 anisotropic steps with unequal CPML
    layers: the transpose weights axis d's bracket by kr_d, also through the
    memory variables."""
    lhs, rhs = _aniso_adjoint_case()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_anisotropic_dot_product_detects_unweighted_transpose():
    """The same identity with the isotropic transpose fails: the pin sees a
    missing kr weight."""
    lhs, rhs = _aniso_adjoint_case(kr_adj=(1.0, 1.0, 1.0))
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


def test_anisotropic_gradient_matches_central_differences():
    """dJ/dK of the anisotropic misfit against central differences of the
    FP64 misfit at random nodes, in the slabs and near the source."""
    shape, L, h = (14, 13, 15), (3, 3, 2, 3, 3, 2), 10.0
    kr = (1.5, 0.8, 1.0)
    rng = np.random.default_rng(4)
    c_true = rng.uniform(1800, 2600, size=shape)
    c0 = np.full(shape, 2200.0)
    dt = 0.4 * h / (2600.0 * np.sqrt(max(kr)))
    prof = O.make_profiles(shape, L, h, dt, 2600.0 * np.sqrt(max(kr)), R=1e-5)
    nt = 50
    src = (7, 6, 7)
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[4, 4, 5], [5, 9, 9], [10, 6, 4], [3, 10, 11], [11, 9, 10]])
    dobs = O.forward_traces(O.Grid(c_true ** 2, h, dt, prof, kr=kr), nt, src, wav, rec)
    K0 = c0 ** 2
    _, gK, _, _ = O.misfit_gradient(O.Grid(K0, h, dt, prof, kr=kr), nt, src, wav, rec, dobs, checkpoint_every=9)
    nodes = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(5)] + [(7, 6, 8), (0, 0, 0), (13, 12, 14)]
    scale = np.max(np.abs(gK))
    for node in nodes:
        eps = 1e-4 * K0[node]
        Kp, Km = K0.copy(), K0.copy()
        Kp[node] += eps
        Km[node] -= eps
        Jp, _ = O.misfit(O.Grid(Kp, h, dt, prof, kr=kr), nt, src, wav, rec, dobs)
        Jm, _ = O.misfit(O.Grid(Km, h, dt, prof, kr=kr), nt, src, wav, rec, dobs)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(gK[node] - fd) <= 1e-6 * scale + 1e-5 * abs(fd), (node, gK[node], fd)
