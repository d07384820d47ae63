"""Pins of the oracle's CPML (Sec. 3.2, Tab. 2, Tab. 8) and of the whole step
(symmetry, explicit-matrix second formulation).  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


def test_sigma_max_gives_target_reflection_for_continuous_layer():
    # normal incidence on the continuous graded layer: R = exp(-2/c int_0^{Lh} sigma)
    for L, h, c, R, q in [(20, 10.0, 4500.0, 1e-8, 3), (10, 10.0, 2000.0, 1e-5, 3), (6, 5.0, 3000.0, 1e-3, 2)]:
        smax = O.sigma_max(L, h, c, R, q)
        integral, _ = integrate.quad(lambda s: smax * (s / (L * h)) ** q, 0.0, L * h)
        assert abs(math.exp(-2.0 * integral / c) / R - 1.0) < 1e-10


def test_recursive_coefficient_a_is_the_kernel_integrated_over_one_step():
    # the CFS-PML convolution kernel -(sigma/kappa^2) exp(-(sigma/kappa + alpha) t)
    # integrated over [0, dt] is the a of the recursion; b is its decay over dt
    dt = 1.1e-3
    for sigma, kappa, alpha in [(828.9, 5.0, 0.0), (300.0, 1.7, 20.0), (5.0, 1.0, 41.4)]:
        b, a, kinv = O.cpml_coefficients(sigma, kappa, alpha, dt)
        rate = sigma / kappa + alpha
        kern, _ = integrate.quad(lambda t: -(sigma / kappa ** 2) * math.exp(-rate * t), 0.0, dt)
        assert abs(a - kern) <= 1e-12 * abs(kern)
        assert abs(b - math.exp(-rate * dt)) < 1e-15
        assert abs(kinv * kappa - 1.0) < 1e-15


def test_profile_grading_shape():
    n, L, h, dt, c, R = 40, 8, 10.0, 1e-3, 3000.0, 1e-8
    pr = O.axis_profile(n, L, L, h, dt, c, R)
    smax = O.sigma_max(L, h, c, R)
    assert pr["slab"].sum() == 2 * L and pr["slab"][L] == 0 and pr["slab"][n - 1 - L] == 0
    # outermost node: rho = 1, full damping and stretching, no frequency shift
    for i in (0, n - 1):
        assert pr["rho"][i] == 1.0
        assert abs(pr["sigma"][i] - smax) < 1e-9 * smax
        assert abs(pr["kappa"][i] - 5.0) < 1e-12
        assert abs(pr["alpha"][i]) < 1e-12
    # innermost slab node: rho = 1/L
    assert abs(pr["rho"][L - 1] - 1.0 / L) < 1e-15
    assert abs(pr["alpha"][L - 1] - 0.05 * smax * (1 - 1.0 / L)) < 1e-9
    # mirror symmetry of the two faces
    for k in ("b", "a", "kinv", "sigma"):
        assert np.allclose(pr[k], pr[k][::-1], rtol=0, atol=0)
    # monotone grading into the layer
    assert np.all(np.diff(pr["sigma"][:L]) < 0)


def _grid_with_cpml(shape, L, h=10.0, c=2000.0, R=1e-5, cfl=0.5, K=None):
    dt = cfl * h / c
    prof = O.make_profiles(shape, L, h, dt, c, R=R)
    if K is None:
        K = np.full(shape, c * c)
    return O.Grid(K, h, dt, prof), dt


def test_sigma_zero_reduces_to_interior_update_bitwise():
    """sigma = 0, kappa = 1 (R = 1, kappa_max = 1): the CPML code path leaves
    the update identical to the plain interior update (Sec. 3.2)."""
    shape = (14, 15, 16)
    h, c = 10.0, 2000.0
    dt = 0.5 * h / c
    L = (3, 4, 2, 5, 4, 3)
    prof = O.make_profiles(shape, L, h, dt, c, R=1.0, kappa_max=1.0, alpha_frac=0.0)
    g1 = O.Grid(np.full(shape, c * c), h, dt, prof)
    g0 = O.Grid(np.full(shape, c * c), h, dt, None)
    init = synth.random_state(shape, (0,) * 6, seed=3, dtype=np.float64)
    s1, s0 = O.State(shape), O.State(shape)
    for k in ("p", "vx", "vy", "vz"):
        s1[k] = init[k]
        s0[k] = init[k]
    O.run(g1, s1, 7)
    O.run(g0, s0, 7)
    for k in ("p", "vx", "vy", "vz"):
        assert np.array_equal(s1[k], s0[k])


def test_psi_recursion_equals_explicit_convolution():
    """psi^n = sum_m a b^(n-m) delta f^m at every slab node (Sec. 3.2: the
    single memory variable carries the whole convolution)."""
    shape = (12, 13, 14)
    L = (3, 3, 4, 2, 3, 3)
    g, dt = _grid_with_cpml(shape, L)
    rng = np.random.default_rng(5)
    st = O.State(shape)
    st["p"] = rng.standard_normal(shape)
    hist = []
    nsteps = 9
    for _ in range(nsteps):
        hist.append(st["p"].copy())
        O.run(g, st, 1)
    # independent derivative: slicing with zero padding
    w = O.WEIGHTS

    def dz(f, axis):
        pad = [(0, 0)] * 3
        pad[axis] = (4, 4)
        fp = np.pad(f, pad)
        n = f.shape[axis]
        out = np.zeros_like(f)
        for l in range(1, 5):
            sl_p = [slice(None)] * 3
            sl_m = [slice(None)] * 3
            sl_p[axis] = slice(4 + l, 4 + l + n)
            sl_m[axis] = slice(4 - l, 4 - l + n)
            out += w[l - 1] * (fp[tuple(sl_p)] - fp[tuple(sl_m)])
        return out / g.h

    for d, ax in enumerate("xyz"):
        arr_axis = 2 - d
        pr = g.profiles[d]
        conv = np.zeros(shape)
        bshape = [1, 1, 1]
        bshape[arr_axis] = -1
        b = pr["b"].reshape(bshape)
        a = pr["a"].reshape(bshape)
        sl = pr["slab"].reshape(bshape).astype(bool)
        for m in range(nsteps):
            conv += a * b ** (nsteps - 1 - m) * dz(hist[m], arr_axis)
        conv = np.where(sl, conv, 0.0)
        assert np.allclose(st["psiv_" + ax], conv, rtol=1e-12, atol=1e-12 * np.max(np.abs(conv))), ax


def test_octahedral_symmetry_centred_source():
    """Odd cube, homogeneous medium, equal layers on all faces, source at the
    centre: p is invariant under the 48 axis permutations and reflections."""
    n, L = 25, 5
    shape = (n, n, n)
    g, dt = _grid_with_cpml(shape, (L,) * 6)
    st = O.State(shape)
    wav = synth.ricker(40, dt, 25.0)
    O.run(g, st, 40, 0, (n // 2,) * 3, wav)
    p = st["p"]
    scale = np.max(np.abs(p))
    assert scale > 0
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product([False, True], repeat=3):
            q = np.transpose(p, perm)
            for ax, f in enumerate(flips):
                if f:
                    q = np.flip(q, axis=ax)
            assert np.max(np.abs(q - p)) <= 1e-12 * scale


def test_symmetry_pin_detects_a_wrong_y_profile():
    # planted mistake: a y-profile off by a little breaks the symmetry pin
    n, L = 25, 5
    shape = (n, n, n)
    g, dt = _grid_with_cpml(shape, (L,) * 6)
    g.profiles[1]["a"] *= 1.001
    g = O.Grid(g.K, g.h, g.dt, g.profiles)
    st = O.State(shape)
    O.run(g, st, 40, 0, (n // 2,) * 3, synth.ricker(40, dt, 25.0))
    p = st["p"]
    assert np.max(np.abs(np.transpose(p, (1, 0, 2)) - p)) > 1e-9 * np.max(np.abs(p))


def _reflection_ratios(layers, nsteps=90, core=30, f0=10.0):
    """Reflected-to-incident ratio for layers of L cells: receivers 11 cells
    from a centred source (4 cells inside the core edge) compared with the same
    core embedded in a grid large enough that nothing returns within nsteps.
    Ratio = max |p_L - p_big| / max |p_big| over the receivers and steps."""
    h, c = 10.0, 2000.0
    dt = 0.5 * h / c
    wav = synth.ricker(nsteps, dt, f0)
    off = 11
    nb = core + 2 * 50
    cb = nb // 2
    rec_rel = np.array([[0, 0, off], [0, off, 0], [off, 0, 0]])
    gb = O.Grid(np.full((nb,) * 3, c * c), h, dt, None)
    tb = O.run(gb, O.State(gb.shape), nsteps, 0, (cb,) * 3, wav, rec_rel + cb)
    out = []
    for L in layers:
        n = core + 2 * L
        cs = n // 2
        gs = O.Grid(np.full((n,) * 3, c * c), h, dt,
                    O.make_profiles((n,) * 3, (L,) * 6, h, dt, c, R=1e-8))
        ts = O.run(gs, O.State(gs.shape), nsteps, 0, (cs,) * 3, wav, rec_rel + cs)
        out.append(np.max(np.abs(ts - tb)) / np.max(np.abs(tb)))
    return out


@pytest.mark.slow
def test_cpml_reflection_falls_with_layer_thickness():
    """Tab. 8 trend: the reflected/incident ratio falls monotonically with the
    number of CPML cells, from O(1) for a bare zero wall, by roughly an order
    of magnitude per 4 cells (the paper: about 12x per 4 cells from 8 to 16)."""
    ratios = _reflection_ratios((0, 4, 8, 12, 16))
    assert ratios[0] > 0.3, ratios
    for a, b in zip(ratios, ratios[1:]):
        assert b < a, ratios
    for a, b in zip(ratios[1:], ratios[2:]):
        assert b < a / 4.0, ratios


def test_explicit_matrix_matches_c_step():
    """Second formulation (whole step as a sparse matrix assembled from the
    operators) against the C loops, on a tiny grid with unequal faces,
    heterogeneous K and rho != 1."""
    shape = (7, 9, 10)
    L = (2, 3, 1, 2, 3, 2)
    rng = np.random.default_rng(11)
    h, rho = 10.0, 1.3
    c = rng.uniform(1500, 3000, size=shape)
    dt = 0.5 * h / c.max()
    prof = O.make_profiles(shape, L, h, dt, 3000.0, R=1e-4)
    for periodic in (False, True):
        g = O.Grid(rho * c * c, h, dt, prof, rho=rho, periodic=periodic)
        M = O.explicit_step_matrix(g)
        st = O.State(shape)
        init = synth.random_state(shape, L, seed=2, v_scale=dt / h, psiv_scale=1 / h,
                                  psip_scale=dt / h ** 2, dtype=np.float64)
        for k, v in init.items():
            st[k] = v
        u0 = st.as_vector()
        O.run(g, st, 1)
        u1 = st.as_vector()
        ref = M @ u0
        assert np.max(np.abs(u1 - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_explicit_matrix_transpose_matches_adjoint_step():
    shape = (7, 8, 9)
    L = (2, 2, 3, 1, 2, 3)
    rng = np.random.default_rng(12)
    h, rho = 10.0, 1.1
    c = rng.uniform(1500, 3000, size=shape)
    dt = 0.5 * h / c.max()
    prof = O.make_profiles(shape, L, h, dt, 3000.0, R=1e-4)
    g = O.Grid(rho * c * c, h, dt, prof, rho=rho)
    M = O.explicit_step_matrix(g)
    ystate = O.State(shape)
    init = synth.random_state(shape, L, seed=4, dtype=np.float64)
    for k, v in init.items():
        ystate[k] = v
    y = ystate.as_vector()
    fwd = O.State(shape)          # forward state does not enter the state adjoint
    adj = ystate.copy()
    O.adjoint_step(g, fwd, adj)
    ref = M.T @ y
    assert np.max(np.abs(adj.as_vector() - ref)) <= 1e-13 * np.max(np.abs(ref))
