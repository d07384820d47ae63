"""Pins of the FP64 oracle's interior scheme (derivative, leapfrog) against
what the paper and the mathematics fix.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_first_derivative_weights_are_exact_rationals():
    # Degree-8 exactness fixes the antisymmetric radius-4 weights uniquely.
    a = O.first_derivative_weights(4)
    assert a == [Fraction(4, 5), Fraction(-1, 5), Fraction(4, 105), Fraction(-1, 280)]
    # exactness conditions, stated independently: sum_l 2 a_l l^(2k-1) = [k == 1]
    for k in range(1, 5):
        s = sum(2 * a[l - 1] * Fraction(l) ** (2 * k - 1) for l in range(1, 5))
        assert s == (1 if k == 1 else 0)


def _derivative_via_oracle(f, axis, h):
    """delta_axis f through the C core: one velocity stage with dt = -1,
    rho = 1, v = 0 and no CPML leaves v_axis = delta_axis p."""
    shape = f.shape
    g = O.Grid(np.ones(shape), h, -1.0)
    st = O.State(shape)
    st["p"] = f
    O.velocity_stage(g, st)
    return st["v" + "xyz"[axis]]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_oracle_derivative_exact_for_polynomials_up_to_degree_8(axis):
    shape = (21, 22, 23)
    h = 0.37
    n = shape[2 - axis]
    coord = (np.arange(n) - n / 2.0) * h
    for k in range(0, 10):
        prof = coord ** k
        if axis == 0:
            f = np.broadcast_to(prof[None, None, :], shape).copy()
        elif axis == 1:
            f = np.broadcast_to(prof[None, :, None], shape).copy()
        else:
            f = np.broadcast_to(prof[:, None, None], shape).copy()
        d = _derivative_via_oracle(f, axis, h)
        exact1d = k * coord ** (k - 1) if k > 0 else np.zeros(n)
        inner = slice(4, n - 4)
        if axis == 0:
            got = d[5, 5, inner]
        elif axis == 1:
            got = d[5, inner, 5]
        else:
            got = d[inner, 5, 5]
        err = np.max(np.abs(got - exact1d[inner])) / max(1.0, np.max(np.abs(exact1d[inner])))
        if k <= 8:
            assert err < 1e-11, (k, err)
        else:
            assert err > 1e-6, (k, err)   # degree 9 is not differentiated exactly
        # the other two derivatives of a function of one coordinate vanish
        for other in range(3):
            if other != axis:
                dd = _derivative_via_oracle(f, other, h)
                sl = [slice(4, s - 4) for s in shape]
                assert np.max(np.abs(dd[tuple(sl)])) <= 1e-9 * max(1.0, np.max(np.abs(f)))


def test_tab6_spatial_convergence_reproduced():
    rows = _golden("tab6_spatial_convergence.txt")
    for order, N, l2, linf in rows:
        if N > 240:
            continue
        got_l2, got_inf = O.laplacian_convergence_error(int(order), int(N), m=4)
        # printed to 4 significant digits; the N = 240, order 8 row is at the
        # level of FP64 rounding of the paper's own run (printed L2 and Linf
        # differ by 1%), so it gets a looser bound
        tol = 2e-3 if not (order == 8 and N == 240) else 2e-2
        assert abs(got_l2 - l2) / l2 < tol, (order, N, got_l2, l2)
        assert abs(got_inf - linf) / linf < tol, (order, N, got_inf, linf)


def test_stability_limit_value():
    # (c dt / 2h) sqrt(3) max D-hat <= 1 for the collocated leapfrog
    assert abs(O.stability_limit() - 0.66722) < 1e-4


@pytest.mark.parametrize("rho", [1.0, 2.0])
def test_discrete_dispersion_relation_exact(rho):
    """p^n = phi cos(omega_h n dt) with sin(omega_h dt / 2) = (c dt / 2) sqrt(sum_d Dhat_d^2 / h^2):
    the fully discrete standing wave, to FP64 rounding."""
    shape = (12, 10, 16)
    h, c = 7.0, 1300.0
    dt = 0.4 * h / c
    K = rho * c * c * np.ones(shape)
    st, phi, lam2 = O.standing_wave_state(shape, (1, 2, 3), h, dt, rho)
    g = O.Grid(K, h, dt, rho=rho, periodic=True)
    nsteps = 57
    O.run(g, st, nsteps)
    omega_h = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2))
    expect = phi * math.cos(omega_h * nsteps * dt)
    err = np.max(np.abs(st["p"] - expect))
    assert err < 1e-12, err


def test_dispersion_pin_detects_a_wrong_weight():
    # a planted mistake in the oracle's weights must break the dispersion pin
    shape = (12, 10, 16)
    h, c, rho = 7.0, 1300.0, 1.0
    dt = 0.4 * h / c
    st, phi, lam2 = O.standing_wave_state(shape, (1, 2, 3), h, dt, rho)
    bad = list(O.WEIGHTS)
    bad[2] *= 1.01
    g = O.Grid(rho * c * c * np.ones(shape), h, dt, rho=rho, periodic=True, weights=bad)
    O.run(g, st, 57)
    omega_h = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2))
    assert np.max(np.abs(st["p"] - phi * math.cos(omega_h * 57 * dt))) > 1e-6


def test_tab7_time_convergence_rate():
    """Leapfrog time error against the continuous standing wave (m = 1,
    c = 1, unit periodic cube, T = 0.2): observed rate 2.00 (Tab. 7)."""
    rows = _golden("tab7_time_convergence.txt")
    N, m, c, T = 32, 1, 1.0, 0.2
    h = 1.0 / N
    x = np.arange(N) * h
    s, co = np.sin(2 * np.pi * m * x), np.cos(2 * np.pi * m * x)
    phi = s[:, None, None] * s[None, :, None] * s[None, None, :]
    omega = 2 * np.pi * m * math.sqrt(3.0) * c
    errs = []
    for dt, _, _ in rows:
        st = O.State((N, N, N))
        st["p"] = phi
        # v(-dt/2) of the continuous solution: v = -grad(phi) sin(omega t) / omega
        k = 2 * np.pi * m
        amp = math.sin(omega * dt / 2) / omega * k
        st["vx"] = amp * s[:, None, None] * s[None, :, None] * co[None, None, :]
        st["vy"] = amp * s[:, None, None] * co[None, :, None] * s[None, None, :]
        st["vz"] = amp * co[:, None, None] * s[None, :, None] * s[None, None, :]
        g = O.Grid(np.full((N, N, N), c * c), h, dt, periodic=True)
        nsteps = int(round(T / dt))
        O.run(g, st, nsteps)
        ex = phi * math.cos(omega * nsteps * dt)
        errs.append(np.sqrt(np.sum((st["p"] - ex) ** 2) / np.sum(ex ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert abs(r - 2.0) < 0.02, rates
    # same order of magnitude as the printed values (T and N unprinted)
    for e, (_, ref, _) in zip(errs, rows):
        assert 0.3 < e / ref < 3.0, (e, ref)


@pytest.mark.parametrize("periodic", [True, False])
def test_energy_conserved_without_cpml(periodic):
    """E^{n+1/2} = 1/2 sum rho |v^{n+1/2}|^2 + 1/2 sum p^n p^{n+1}/K is
    invariant when delta is skew-adjoint (periodic, or zero values beyond the
    grid) and there is no CPML and no source."""
    rng = np.random.default_rng(7)
    shape = (11, 13, 12)
    h, rho = 5.0, 1.5
    c = rng.uniform(1500, 3000, size=shape)
    K = rho * c * c
    dt = 0.5 * h / c.max()
    g = O.Grid(K, h, dt, rho=rho, periodic=periodic)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    for ax in "xyz":
        st["v" + ax] = rng.standard_normal(shape) * dt / (rho * h)
    energies = []
    for _ in range(25):
        p_n = st["p"].copy()
        O.run(g, st, 1)
        energies.append(O.staggered_energy(g, p_n, st["p"], [st["vx"], st["vy"], st["vz"]]))
    e = np.array(energies)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) < 1e-12
