"""Pins of the oracle's staggered (Yee) form of Sec. 3.1: p at the nodes, v_d
at the half nodes i + 1/2 along d, the eighth-order staggered first
derivative (weights 1225/1024, -245/3072, 49/5120, -5/7168 for the offsets
1/2, 3/2, 5/2, 7/2) from p to v and back.  The checks rest on what the
mathematics fixes: exact differentiation of polynomials up to degree 7 at the
right half node, the fully discrete dispersion relation of a standing wave,
conservation of the discrete energy (the backward operator is minus the
transpose of the forward one, also next to a boundary), the stability limit
and its closed form at theta = pi, and absorption by the CPML at half-node
depths.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


def test_staggered_weights_are_the_textbook_values():
    assert O.staggered_weights(4) == [Fraction(1225, 1024), Fraction(-245, 3072),
                                      Fraction(49, 5120), Fraction(-5, 7168)]
    # second order: the plain half-node difference
    assert O.staggered_weights(1) == [Fraction(1)]
    # fourth order: 9/8, -1/24
    assert O.staggered_weights(2) == [Fraction(9, 8), Fraction(-1, 24)]


def _poly_grid(shape, h, dt):
    return O.Grid(np.full(shape, 2000.0 ** 2), h, dt, staggered=True)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("deg", [1, 4, 7])
def test_forward_operator_differentiates_polynomials_at_the_half_node(axis, deg):
    """v' = v - dt/rho D+ p with p = x^deg along one axis: away from the
    boundary D+ p at index i is deg (i + 1/2)^(deg-1) h^(deg-1), exactly up to
    rounding for deg <= 7."""
    shape, h, dt = (20, 21, 22), 1.0, 1e-3
    g = _poly_grid(shape, h, dt)
    st = O.State(shape)
    n = shape[2 - axis]
    s = np.arange(n, dtype=np.float64) - n / 2
    pr = s ** deg
    st["p"] = pr.reshape([-1 if k == 2 - axis else 1 for k in range(3)]) * np.ones(shape)
    O.velocity_stage(g, st)
    v = st["v" + "xyz"[axis]]
    got = -v / dt
    got = np.moveaxis(got, 2 - axis, 0)[:, 3, 3]
    expect = deg * (s + 0.5) ** (deg - 1)
    sl = slice(4, n - 4)
    assert np.max(np.abs(got[sl] - expect[sl])) <= 1e-9 * np.max(np.abs(expect[sl])), axis
    # the centred difference (the collocated form) misses this: a half-node slip shows
    wrong = deg * s ** (deg - 1)
    assert deg == 1 or np.max(np.abs(got[sl] - wrong[sl])) > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("deg", [1, 4, 7])
def test_backward_operator_differentiates_polynomials_at_the_node(axis, deg):
    """The pressure bracket of v_d = (x at the half node)^deg is
    deg i^(deg-1) at node i (the backward staggered derivative)."""
    shape, h, dt = (20, 21, 22), 1.0, 1e-3
    g = _poly_grid(shape, h, dt)
    st = O.State(shape)
    n = shape[2 - axis]
    s = np.arange(n, dtype=np.float64) - n / 2
    vr = (s + 0.5) ** deg
    st["v" + "xyz"[axis]] = vr.reshape([-1 if k == 2 - axis else 1 for k in range(3)]) * np.ones(shape)
    br = O.pressure_stage(g, st, want_bracket=True)
    got = np.moveaxis(br, 2 - axis, 0)[:, 3, 3]
    expect = deg * s ** (deg - 1)
    sl = slice(4, n - 4)
    assert np.max(np.abs(got[sl] - expect[sl])) <= 1e-9 * max(1.0, np.max(np.abs(expect[sl])))


@pytest.mark.parametrize("rho", [1.0, 2.0])
def test_staggered_dispersion_relation_exact(rho):
    """p^n = phi cos(omega_h n dt) with sin(omega_h dt / 2) = (c dt / 2)
    sqrt(sum_d S-hat_d^2 / h^2), S-hat(theta) = 2 sum_l c_l sin((l - 1/2) theta):
    the fully discrete staggered standing wave, to FP64 rounding."""
    shape = (12, 10, 16)
    h, c = 7.0, 1300.0
    dt = 0.4 * h / c
    st, phi, lam2 = O.standing_wave_state(shape, (1, 2, 3), h, dt, rho, staggered=True)
    g = O.Grid(rho * c * c * np.ones(shape), h, dt, rho=rho, periodic=True, staggered=True)
    O.run(g, st, 57)
    omega_h = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2))
    assert np.max(np.abs(st["p"] - phi * math.cos(omega_h * 57 * dt))) < 1e-12


def test_staggered_dispersion_pin_detects_wrong_weight_or_collocated_state():
    shape = (12, 10, 16)
    h, c, rho = 7.0, 1300.0, 1.0
    dt = 0.4 * h / c
    # a planted weight slip in the oracle
    st, phi, lam2 = O.standing_wave_state(shape, (1, 2, 3), h, dt, rho, staggered=True)
    bad = list(O.STAGGERED_WEIGHTS)
    bad[1] *= 1.01
    g = O.Grid(rho * c * c * np.ones(shape), h, dt, rho=rho, periodic=True, staggered=True, weights=bad)
    O.run(g, st, 57)
    omega_h = 2.0 / dt * math.asin(0.5 * c * dt * math.sqrt(lam2))
    assert np.max(np.abs(st["p"] - phi * math.cos(omega_h * 57 * dt))) > 1e-6
    # the collocated operators on the staggered standing wave
    st, phi, lam2 = O.standing_wave_state(shape, (1, 2, 3), h, dt, rho, staggered=True)
    g = O.Grid(rho * c * c * np.ones(shape), h, dt, rho=rho, periodic=True,
               weights=O.STAGGERED_WEIGHTS)
    O.run(g, st, 57)
    assert np.max(np.abs(st["p"] - phi * math.cos(omega_h * 57 * dt))) > 1e-3


@pytest.mark.parametrize("periodic", [True, False])
def test_staggered_energy_conserved(periodic):
    """Zero values beyond the grid make the backward operator minus the
    transpose of the forward one, so 1/2 sum rho |v|^2 + 1/2 sum p p' / K
    stays constant, with a variable density and anisotropy too."""
    rng = np.random.default_rng(23)
    shape = (11, 12, 13)
    h = 5.0
    rho = rng.uniform(0.6, 3.0, size=shape)
    c = rng.uniform(1500, 3000, size=shape)
    kr = (1.4, 0.8, 1.0)
    dt = 0.35 * h / (c.max() * math.sqrt(max(kr)))
    g = O.Grid(rho * c * c, h, dt, rho=rho, periodic=periodic, kr=kr, staggered=True)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    for ax in "xyz":
        st["v" + ax] = rng.standard_normal(shape) * dt / h
    e = []
    for _ in range(30):
        p_n = st["p"].copy()
        O.run(g, st, 1)
        e.append(O.staggered_energy(g, p_n, st["p"], [st["vx"], st["vy"], st["vz"]]))
    e = np.array(e)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) < 1e-12


def test_stability_limit_closed_form_and_growth():
    """The staggered symbol peaks at theta = pi, S-hat(pi) = 2 sum_l |c_l|,
    so the limit is 1 / (sqrt(3) sum_l |c_l|) = 0.44884; below it a random
    state stays bounded, 3% above it grows without bound."""
    w = O.staggered_weights(4)
    closed = 1.0 / (math.sqrt(3.0) * float(sum(abs(x) for x in w)))
    lim = O.stability_limit(staggered=True)
    assert abs(lim - closed) < 1e-9
    assert abs(lim - 0.4488424) < 1e-7
    shape, h, c = (8, 8, 8), 10.0, 2000.0
    rng = np.random.default_rng(5)
    out = []
    for f in (0.99, 1.03):
        dt = f * lim * h / c
        g = O.Grid(np.full(shape, c * c), h, dt, periodic=True, staggered=True)
        st = O.State(shape)
        st["p"] = rng.standard_normal(shape)
        a0 = np.max(np.abs(st["p"]))
        O.run(g, st, 400)
        out.append(np.max(np.abs(st["p"])) / a0)
    assert out[0] < 10.0 and out[1] > 1e6, out


def test_half_node_profiles_interpolate_and_mirror():
    """The velocity profile depths lie half way between the node depths on
    the low face, mirror the low face on the high face (v index i <-> n-2-i, but for the innermost),
    and give every coefficient the same form as the nodes' (b in (0, 1],
    a <= 0, 1/kappa in [1/kappa_max, 1])."""
    n, L, h, dt, c = 40, 9, 10.0, 1e-3, 2500.0
    pr = O.axis_profile(n, L, L, h, dt, c, R=1e-5)
    rv, rp = pr["rho_v"], pr["rho"]
    assert np.allclose(rv[:L], 0.5 * (rp[:L] + np.append(rp[1:L], 0.0)))
    assert np.allclose(rv[:L - 1], rv[n - 2 - np.arange(L - 1)])
    # the one half node the high slab leaves out (depth 1/(2L), sigma = sigma_max / (8 L^3))
    assert rv[n - 1 - L] == 0.0 and pr["slab"][n - 1 - L] == 0
    assert rv[n - 1] == 1.0
    sl = pr["slab"] == 1
    assert np.all((pr["bv"][sl] > 0) & (pr["bv"][sl] <= 1) & (pr["av"][sl] <= 0))
    assert np.all((pr["kinvv"][sl] >= 1 / 5.0 - 1e-12) & (pr["kinvv"][sl] <= 1.0))
    # the layer's outermost velocity sits deeper than its innermost
    assert pr["bv"][0] < pr["bv"][L - 1] and pr["bv"][n - 1] < pr["bv"][n - L]


def test_staggered_cpml_absorbs_a_point_source():
    """A Ricker source in a 44^3 box with a 10-cell layer on every face: once
    the pulse has left, the energy inside is below 1e-4 of its peak; with no
    layer the waves stay (ratio above 0.05, at least 1000 times more)."""
    shape, L, h, c = (44, 44, 44), 10, 10.0, 2000.0
    dt = 0.4 * h / c
    nt = 330
    wav = synth.ricker(nt, dt, 25.0)
    src = (22, 22, 22)
    ratios = []
    for cells in ((L,) * 6, (0,) * 6):
        prof = O.make_profiles(shape, cells, h, dt, c, R=1e-5)
        g = O.Grid(np.full(shape, c * c), h, dt, prof, staggered=True)
        st = O.State(shape)
        e = []
        for k in range(nt // 10):
            p_n = st["p"].copy()
            O.run(g, st, 10, 10 * k, src, wav)
            inner = (slice(L, -L),) * 3
            e.append(float(np.sum(st["p"][inner] ** 2) + np.sum(p_n[inner] ** 2)))
        e = np.array(e)
        ratios.append(e[-1] / e.max())
    assert ratios[0] < 1e-4 and ratios[1] > 0.05 and ratios[1] / ratios[0] > 1e3, ratios


def _stag_dot(adj_grid_kwargs=None):
    rng = np.random.default_rng(31)
    shape, L, h = (10, 11, 12), (2, 3, 3, 2, 2, 3), 10.0
    rho = rng.uniform(0.8, 2.2, size=shape)
    c = rng.uniform(1500.0, 2500.0, size=shape)
    kr = (1.3, 0.8, 1.0)
    dt = 0.35 * h / (c.max() * np.sqrt(max(kr)))
    prof = O.make_profiles(shape, L, h, dt, c.max() * np.sqrt(max(kr)), R=1e-5)
    g = O.Grid(rho * c * c, h, dt, prof, rho=rho, kr=kr, staggered=True)
    ga = g if adj_grid_kwargs is None else O.Grid(rho * c * c, h, dt, prof, rho=rho, kr=kr, **adj_grid_kwargs)
    xs = synth.random_state(shape, L, seed=32, v_scale=dt / h, psiv_scale=1 / h, psip_scale=dt / h ** 2,
                            dtype=np.float64)
    ys = synth.random_state(shape, L, seed=33, dtype=np.float64)
    x, y = O.State(shape), O.State(shape)
    for k in O.FIELDS:
        x[k] = xs[k]
        y[k] = ys[k]
    fx = x.copy()
    O.run(g, fx, 6)
    aty = y.copy()
    for _ in range(6):
        O.adjoint_step(ga, O.State(shape), aty)
    return float(np.dot(fx.as_vector(), y.as_vector())), float(np.dot(x.as_vector(), aty.as_vector()))


def test_staggered_transpose_dot_product():
    """<F x, y> = <x, F^T y> over 6 staggered steps with unequal CPML layers
    (half-node velocity profiles), a density and anisotropy."""
    lhs, rhs = _stag_dot()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_staggered_dot_product_detects_the_collocated_transpose():
    lhs, rhs = _stag_dot(dict(weights=O.STAGGERED_WEIGHTS))   # centred operators, staggered weights
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


def test_staggered_gradient_matches_central_differences():
    shape, L, h = (14, 13, 15), (3, 3, 2, 3, 3, 2), 10.0
    rng = np.random.default_rng(12)
    c_true = rng.uniform(1800, 2600, size=shape)
    c0 = np.full(shape, 2200.0)
    dt = 0.4 * h / 2600.0
    prof = O.make_profiles(shape, L, h, dt, 2600.0, R=1e-5)
    nt = 50
    src = (7, 6, 7)
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[4, 4, 5], [5, 9, 9], [10, 6, 4], [3, 10, 11], [11, 9, 10]])
    dobs = O.forward_traces(O.Grid(c_true ** 2, h, dt, prof, staggered=True), nt, src, wav, rec)
    K0 = c0 ** 2
    _, gK, _, _ = O.misfit_gradient(O.Grid(K0, h, dt, prof, staggered=True), nt, src, wav, rec, dobs,
                                    checkpoint_every=9)
    nodes = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(5)] + [(7, 6, 8), (0, 0, 0), (13, 12, 14)]
    scale = np.max(np.abs(gK))
    for node in nodes:
        eps = 1e-4 * K0[node]
        Kp, Km = K0.copy(), K0.copy()
        Kp[node] += eps
        Km[node] -= eps
        Jp, _ = O.misfit(O.Grid(Kp, h, dt, prof, staggered=True), nt, src, wav, rec, dobs)
        Jm, _ = O.misfit(O.Grid(Km, h, dt, prof, staggered=True), nt, src, wav, rec, dobs)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(gK[node] - fd) <= 1e-6 * scale + 1e-5 * abs(fd), (node, gK[node], fd)
