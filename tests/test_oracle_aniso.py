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
