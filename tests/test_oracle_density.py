"""Pins of the oracle's variable-density form (density per node, collocated
with p and v; the velocity update at a node uses dt / rho of that node and
K = rho c^2 enters the pressure update).  The paper fixes rho only through
p_t = -K div v, v_t = -(1/rho) grad p (Sec. 3.1); these tests check the
oracle against what that system implies: the discrete energy
1/2 sum rho |v|^2 + 1/2 sum p p' / K is conserved, a plane wave meets a
density step with the impedance reflection and transmission coefficients,
and the transpose stays a transpose.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


@pytest.mark.parametrize("periodic", [True, False])
def test_energy_conserved_with_variable_density(periodic):
    rng = np.random.default_rng(17)
    shape = (11, 12, 13)
    h = 5.0
    rho = rng.uniform(0.6, 3.0, size=shape)
    c = rng.uniform(1500, 3000, size=shape)
    K = rho * c * c
    dt = 0.5 * h / c.max()
    g = O.Grid(K, h, dt, rho=rho, periodic=periodic)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    for ax in "xyz":
        st["v" + ax] = rng.standard_normal(shape) * dt / h
    energies = []
    for _ in range(25):
        p_n = st["p"].copy()
        O.run(g, st, 1)
        energies.append(O.staggered_energy(g, p_n, st["p"], [st["vx"], st["vy"], st["vz"]]))
    e = np.array(energies)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) < 1e-12


def test_energy_pin_detects_density_in_the_wrong_place():
    """The same run with the density used as 1/rho (a plausible slip) does
    not conserve the energy the pin measures."""
    rng = np.random.default_rng(17)
    shape = (11, 12, 13)
    h = 5.0
    rho = rng.uniform(0.6, 3.0, size=shape)
    c = rng.uniform(1500, 3000, size=shape)
    dt = 0.5 * h / c.max()
    g_wrong = O.Grid(rho * c * c, h, dt, rho=1.0 / rho, periodic=True)
    g_right = O.Grid(rho * c * c, h, dt, rho=rho, periodic=True)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    energies = []
    for _ in range(25):
        p_n = st["p"].copy()
        O.run(g_wrong, st, 1)
        energies.append(O.staggered_energy(g_right, p_n, st["p"], [st["vx"], st["vy"], st["vz"]]))
    e = np.array(energies)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) > 1e-3


def test_constant_density_array_equals_scalar_density():
    rng = np.random.default_rng(3)
    shape = (9, 8, 10)
    h, c, rho = 10.0, 2000.0, 1.7
    dt = 0.5 * h / c
    prof = O.make_profiles(shape, (2, 3, 2, 2, 3, 2), h, dt, c, R=1e-5)
    K = np.full(shape, rho * c * c)
    states = []
    for r in (rho, np.full(shape, rho)):
        st = O.State(shape)
        st["p"] = rng.standard_normal(shape) if not states else states[0][1]
        init = st["p"].copy()
        O.run(O.Grid(K, h, dt, prof, rho=r), st, 7)
        states.append((st, init))
    for k in O.FIELDS:
        assert np.array_equal(states[0][0][k], states[1][0][k]), k


@pytest.mark.parametrize("rho2", [3.0, 1.0 / 3.0])
def test_plane_wave_at_a_density_step_matches_impedance_coefficients(rho2):
    """A right-going Gaussian plane wave (uniform in x, y on a periodic grid)
    meets a step from rho1 = 1 to rho2 at equal velocity.  The reflected and
    transmitted pressure peaks match R = (Z2 - Z1) / (Z2 + Z1) and
    T = 2 Z2 / (Z1 + Z2), Z = rho c, to within 1% of the incident peak."""
    nz, h, c = 1200, 10.0, 2000.0
    shape = (nz, 2, 2)
    cfl = 0.4
    dt = cfl * h / c
    z = np.arange(nz, dtype=np.float64)
    zi, z0, w = 600, 300, 12.0
    rho = np.where(z >= zi, rho2, 1.0)[:, None, None] * np.ones(shape)
    K = rho * c * c
    g = O.Grid(K, h, dt, rho=rho, periodic=True)
    st = O.State(shape)
    f = lambda s: np.exp(-((s - z0) / w) ** 2)
    st["p"] = f(z)[:, None, None] * np.ones(shape)
    # v_z at t = -dt/2 of the right-going wave p = f(z - c t), v = p / (rho c)
    st["vz"] = (f(z + 0.5 * cfl) / (1.0 * c))[:, None, None] * np.ones(shape)
    nsteps = int(round(450 / cfl))   # the wave travels 450 cells
    O.run(g, st, nsteps)
    p = st["p"][:, 0, 0]
    Z1, Z2 = 1.0 * c, rho2 * c
    R, T = (Z2 - Z1) / (Z2 + Z1), 2 * Z2 / (Z1 + Z2)
    refl = p[350:560]
    trans = p[650:850]
    r_num = refl[np.argmax(np.abs(refl))]
    t_num = trans[np.argmax(np.abs(trans))]
    assert abs(r_num - R) < 0.01, (r_num, R)
    assert abs(t_num - T) < 0.01, (t_num, T)
    # the reflected peak sits where a wave at speed c puts it
    assert abs(350 + int(np.argmax(np.abs(refl))) - (zi - 150)) <= 2


def test_dot_product_identity_with_variable_density():
    shape = (10, 11, 12)
    L = (2, 3, 3, 2, 2, 3)
    h, c = 10.0, 2000.0
    dt = 0.5 * h / c
    rng = np.random.default_rng(29)
    rho = rng.uniform(0.7, 2.5, size=shape)
    K = rho * rng.uniform(1500, 2500, size=shape) ** 2
    g = O.Grid(K, h, dt, O.make_profiles(shape, L, h, dt, c, R=1e-5), rho=rho)
    xs = synth.random_state(shape, L, seed=31, v_scale=dt / h, psiv_scale=1 / h,
                            psip_scale=dt / h ** 2, dtype=np.float64)
    ys = synth.random_state(shape, L, seed=32, dtype=np.float64)
    x = O.State(shape)
    for k, v in xs.items():
        x[k] = v
    y = O.State(shape)
    for k, v in ys.items():
        y[k] = v
    fx = x.copy()
    O.run(g, fx, 5)
    aty = y.copy()
    for _ in range(5):
        O.adjoint_step(g, O.State(shape), aty)
    lhs = float(np.dot(fx.as_vector(), y.as_vector()))
    rhs = float(np.dot(x.as_vector(), aty.as_vector()))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradient_wrt_K_with_density_matches_central_differences():
    """dJ/dK of a source run with a per-node density (the transpose's
    velocity stage uses dt / rho of each node) against central differences
    of the FP64 misfit."""
    shape, L, h = (14, 13, 15), (3, 3, 2, 3, 3, 2), 10.0
    rng = np.random.default_rng(6)
    rho = rng.uniform(0.8, 2.4, size=shape)
    c_true = rng.uniform(1800, 2600, size=shape)
    c0 = np.full(shape, 2200.0)
    dt = 0.5 * h / 2600.0
    prof = O.make_profiles(shape, L, h, dt, 2600.0, R=1e-5)
    nt = 50
    src = (7, 6, 7)
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[4, 4, 5], [5, 9, 9], [10, 6, 4], [3, 10, 11], [11, 9, 10]])
    dobs = O.forward_traces(O.Grid(rho * c_true ** 2, h, dt, prof, rho=rho), nt, src, wav, rec)
    K0 = rho * c0 ** 2
    _, gK, _, _ = O.misfit_gradient(O.Grid(K0, h, dt, prof, rho=rho), nt, src, wav, rec, dobs, checkpoint_every=9)
    nodes = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(5)] + [(7, 6, 8), (0, 0, 0), (13, 12, 14)]
    scale = np.max(np.abs(gK))
    for node in nodes:
        eps = 1e-4 * K0[node]
        Kp, Km = K0.copy(), K0.copy()
        Kp[node] += eps
        Km[node] -= eps
        Jp, _ = O.misfit(O.Grid(Kp, h, dt, prof, rho=rho), nt, src, wav, rec, dobs)
        Jm, _ = O.misfit(O.Grid(Km, h, dt, prof, rho=rho), nt, src, wav, rec, dobs)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(gK[node] - fd) <= 1e-6 * scale + 1e-5 * abs(fd), (node, gK[node], fd)
