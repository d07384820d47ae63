"""Pins of the oracle's local-velocity CPML grading (heterogeneous media, the
extension Sec. 7 names): at a node of a d-slab sigma_max uses the velocity of
that node, sigma_max(c) = -(q+1) c ln(R) / (2 L h), so the layer's
continuous normal-incidence round trip exp(-2 int sigma / c ds) is R for
every column whatever its velocity.  The checks: the reduction to the 1D
grading for a homogeneous model (bit for bit), the round trip per column on
unequal faces, the monotone shape of the coefficients, and absorption with
long-time stability in a strongly layered model.  CPU only."""
import math

import numpy as np

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


def test_homogeneous_model_reduces_to_the_1d_grading_bitwise():
    shape, cells, h, c = (18, 20, 22), (3, 4, 2, 5, 4, 3), 10.0, 2300.0
    dt = 0.5 * h / c
    vel = np.full(shape, c)
    prof = O.make_profiles(shape, cells, h, dt, c, R=1e-6)
    lp = O.local_profiles(vel, cells, h, dt, R=1e-6)
    for d in range(3):
        shp = [1, 1, 1]
        shp[2 - d] = shape[2 - d]
        assert np.array_equal(lp[d]["b"], np.broadcast_to(prof[d]["b"].reshape(shp), shape)), d
        assert np.array_equal(lp[d]["a"], np.broadcast_to(prof[d]["a"].reshape(shp), shape)), d
    rng = np.random.default_rng(4)
    out = []
    for local in (None, lp):
        st = O.State(shape)
        st["p"] = rng.standard_normal(shape) if not out else out[0][1]
        init = st["p"].copy()
        O.run(O.Grid(vel ** 2, h, dt, prof, local=local), st, 6)
        out.append((st, init))
    for k in O.FIELDS:
        assert np.array_equal(out[0][0][k], out[1][0][k]), k


def test_round_trip_is_R_for_every_column():
    """The outermost node of each face has normalised depth 1, so sigma there
    is sigma_max(c) and -2 sigma_max(c) L h / ((q + 1) c) must equal ln R for
    the face's own L and the node's own c (unequal faces, random velocities)."""
    rng = np.random.default_rng(8)
    shape, cells, h, R, q = (14, 15, 16), (3, 5, 2, 4, 6, 2), 7.5, 1e-7, 3
    vel = rng.uniform(1400.0, 5200.0, size=shape)
    lp = O.local_profiles(vel, cells, h, 1e-3, R=R, q=q)
    nz, ny, nx = shape
    faces = [(0, (slice(None), slice(None), 0), cells[0]), (0, (slice(None), slice(None), nx - 1), cells[1]),
             (1, (slice(None), 0, slice(None)), cells[2]), (1, (slice(None), ny - 1, slice(None)), cells[3]),
             (2, (0, slice(None), slice(None)), cells[4]), (2, (nz - 1, slice(None), slice(None)), cells[5])]
    for d, sl, L in faces:
        s = lp[d]["sigma"][sl]
        c = vel[sl]
        lnR = -2.0 * s * L * h / ((q + 1) * c)
        assert np.allclose(lnR, math.log(R), rtol=1e-12, atol=0), (d, L)


def test_local_coefficients_shape():
    """b in (0, 1], a <= 0 inside the slabs, zero outside; along a column
    into a face (velocity constant along it) b falls towards the outside; at
    equal depth a faster node is damped harder."""
    shape, cells, h = (24, 6, 30), (8, 8, 0, 0, 6, 6), 10.0
    dt = 1e-3
    vel = synth.layered_model(shape, seed=3, vmin=1500.0, vmax=4500.0, amp_cells=1.0).astype(np.float64)
    vel = np.repeat(vel[:, :, :1], shape[2], axis=2)     # layers constant along x
    lp = O.local_profiles(vel, cells, h, dt, R=1e-8)
    b, a = lp[0]["b"], lp[0]["a"]
    inx = np.zeros(shape[2], bool)
    inx[:8] = inx[-8:] = True
    assert np.all((b[:, :, inx] > 0) & (b[:, :, inx] <= 1) & (a[:, :, inx] <= 0))
    assert np.all(b[:, :, ~inx] == 0) and np.all(a[:, :, ~inx] == 0)
    assert np.all(np.diff(b[:, :, :8], axis=2) > 0)        # less damping going inwards
    z_slow, z_fast = int(np.argmin(vel[:, 0, 0])), int(np.argmax(vel[:, 0, 0]))
    assert b[z_fast, 0, 0] < b[z_slow, 0, 0]


def test_layered_model_absorbs_and_stays_stable():
    """A 2D section (ny = 1) of a 1500-4500 m/s layered model with 10-cell
    layers on the x and z faces graded from the local velocity: the field
    energy falls below 1e-3 of its peak and stays bounded over a long run."""
    nz, nx, h, L = 90, 90, 10.0, 10
    shape, cells = (nz, 1, nx), (L, L, 0, 0, L, L)
    vel = synth.layered_model(shape, seed=6, vmin=1500.0, vmax=4500.0, amp_cells=2.0).astype(np.float64)
    dt = 0.5 * h / vel.max()
    prof = O.make_profiles(shape, cells, h, dt, vel.max(), R=1e-5)
    g = O.Grid(vel ** 2, h, dt, prof, local=O.local_profiles(vel, cells, h, dt, R=1e-5))
    st = O.State(shape)
    nt = 3000
    wav = synth.ricker(nt, dt, 12.0)
    e = []
    for k in range(nt // 50):
        O.run(g, st, 50, 50 * k, (45, 0, 45), wav)
        e.append(float(np.sum(st["p"][L:-L, :, L:-L] ** 2)))
    e = np.array(e)
    assert e[-1] < 1e-3 * e.max(), e[-1] / e.max()
    assert np.all(np.isfinite(e)) and e[-10:].max() < 2e-3 * e.max()


def test_each_node_uses_its_own_coefficients():
    """One velocity stage from psi = 0 leaves psi_v,d = a_d(node) delta_d p,
    with delta_d p read off a run without a layer; a second stage with p = 0
    (no new derivative) multiplies psi_v,d by b_d(node).  Random velocities
    make every node's pair different, so a coefficient taken from another
    node or axis shows."""
    rng = np.random.default_rng(12)
    shape, cells, h = (12, 13, 14), (3, 4, 2, 3, 4, 2), 10.0
    vel = rng.uniform(1500.0, 4000.0, size=shape)
    dt = 0.5 * h / vel.max()
    prof = O.make_profiles(shape, cells, h, dt, vel.max(), R=1e-6)
    lp = O.local_profiles(vel, cells, h, dt, R=1e-6)
    p0 = rng.standard_normal(shape)
    free = O.State(shape)
    free["p"] = p0
    O.velocity_stage(O.Grid(vel ** 2, h, dt), free)
    st = O.State(shape)
    st["p"] = p0
    g = O.Grid(vel ** 2, h, dt, prof, local=lp)
    O.velocity_stage(g, st)
    nz, ny, nx = shape
    for d, ax in enumerate("xyz"):
        delta = -free["v" + ax] / dt
        n = (nx, ny, nz)[d]
        shp = [1, 1, 1]
        shp[2 - d] = n
        slab = np.broadcast_to(prof[d]["slab"].reshape(shp).astype(bool), shape)
        expect = np.where(slab, lp[d]["a"] * delta, 0.0)
        assert np.max(np.abs(st["psiv_" + ax] - expect)) <= 1e-12 * np.max(np.abs(expect)), ax
    psi1 = {ax: st["psiv_" + ax].copy() for ax in "xyz"}
    st["p"] = np.zeros(shape)
    O.velocity_stage(g, st)
    for d, ax in enumerate("xyz"):
        assert np.max(np.abs(st["psiv_" + ax] - lp[d]["b"] * psi1[ax])) <= 1e-14 * np.max(np.abs(psi1[ax])), ax


def test_pressure_stage_uses_each_nodes_coefficients():
    """The same check for psi_p: with v only along axis d the pressure
    bracket of a run without a layer is delta_d v_d, and one pressure stage
    from psi = 0 leaves psi_p,d = a_d(node) delta_d v_d."""
    rng = np.random.default_rng(13)
    shape, cells, h = (12, 13, 14), (3, 4, 2, 3, 4, 2), 10.0
    vel = rng.uniform(1500.0, 4000.0, size=shape)
    dt = 0.5 * h / vel.max()
    prof = O.make_profiles(shape, cells, h, dt, vel.max(), R=1e-6)
    lp = O.local_profiles(vel, cells, h, dt, R=1e-6)
    nz, ny, nx = shape
    for d, ax in enumerate("xyz"):
        v0 = rng.standard_normal(shape)
        free = O.State(shape)
        free["v" + ax] = v0
        delta = O.pressure_stage(O.Grid(vel ** 2, h, dt), free, want_bracket=True)
        st = O.State(shape)
        st["v" + ax] = v0
        O.pressure_stage(O.Grid(vel ** 2, h, dt, prof, local=lp), st)
        n = (nx, ny, nz)[d]
        shp = [1, 1, 1]
        shp[2 - d] = n
        slab = np.broadcast_to(prof[d]["slab"].reshape(shp).astype(bool), shape)
        expect = np.where(slab, lp[d]["a"] * delta, 0.0)
        assert np.max(np.abs(st["psip_" + ax] - expect)) <= 1e-12 * np.max(np.abs(expect)), ax


def test_sub_box_profiles_equal_the_full_grids():
    """local_profiles on a box of a larger grid (its origin given) equals the
    box cut out of the full grid's profiles."""
    rng = np.random.default_rng(3)
    shape, cells, h = (20, 22, 24), (4, 5, 3, 6, 5, 4), 10.0
    vel = rng.uniform(1500.0, 4000.0, size=shape)
    full = O.local_profiles(vel, cells, h, 1e-3, R=1e-6)
    for o, e in (((0, 0, 0), (9, 10, 11)), ((11, 7, 13), (20, 22, 24)), ((3, 4, 5), (17, 18, 19))):
        box = tuple(slice(a, b) for a, b in zip(o, e))
        part = O.local_profiles(vel[box], cells, h, 1e-3, R=1e-6, full_shape=shape, origin=o)
        for d in range(3):
            for k in ("b", "a", "sigma"):
                assert np.array_equal(part[d][k], full[d][k][box]), (o, d, k)


def test_transpose_with_local_grading_dot_product():
    """<F x, y> = <x, F^T y> over 6 steps with per-node (b, a) from a random
    velocity field: the transpose takes each node's own coefficients."""
    rng = np.random.default_rng(25)
    shape, L, h = (10, 11, 12), (2, 3, 3, 2, 2, 3), 10.0
    vel = rng.uniform(1500.0, 4000.0, size=shape)
    dt = 0.5 * h / vel.max()
    prof = O.make_profiles(shape, L, h, dt, vel.max(), R=1e-5)
    g = O.Grid(vel ** 2, h, dt, prof, local=O.local_profiles(vel, L, h, dt, R=1e-5))
    xs = synth.random_state(shape, L, seed=26, v_scale=dt / h, psiv_scale=1 / h, psip_scale=dt / h ** 2,
                            dtype=np.float64)
    ys = synth.random_state(shape, L, seed=27, dtype=np.float64)
    x, y = O.State(shape), O.State(shape)
    for k in O.FIELDS:
        x[k] = xs[k]
        y[k] = ys[k]
    fx = x.copy()
    O.run(g, fx, 6)
    aty = y.copy()
    for _ in range(6):
        O.adjoint_step(g, O.State(shape), aty)
    lhs = float(np.dot(fx.as_vector(), y.as_vector()))
    rhs = float(np.dot(x.as_vector(), aty.as_vector()))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the 1D-profile transpose on the same run does not satisfy it
    g1 = O.Grid(vel ** 2, h, dt, prof)
    aty1 = y.copy()
    for _ in range(6):
        O.adjoint_step(g1, O.State(shape), aty1)
    rhs1 = float(np.dot(x.as_vector(), aty1.as_vector()))
    assert abs(lhs - rhs1) > 1e-6 * abs(lhs)


def test_gradient_with_local_grading_matches_central_differences():
    """dJ/dK with the local grading held fixed (the coefficients computed
    once from the starting model) against central differences."""
    shape, L, h = (14, 13, 15), (3, 3, 2, 3, 3, 2), 10.0
    rng = np.random.default_rng(8)
    c_true = rng.uniform(1800, 3600, size=shape)
    c0 = rng.uniform(2000, 3400, size=shape)
    dt = 0.5 * h / 3600.0
    prof = O.make_profiles(shape, L, h, dt, 3600.0, R=1e-5)
    loc = O.local_profiles(c0, L, h, dt, R=1e-5)
    nt = 50
    src = (7, 6, 7)
    wav = synth.ricker(nt, dt, 40.0)
    rec = np.array([[4, 4, 5], [5, 9, 9], [10, 6, 4], [3, 10, 11], [11, 9, 10]])
    dobs = O.forward_traces(O.Grid(c_true ** 2, h, dt, prof, local=loc), nt, src, wav, rec)
    K0 = c0 ** 2
    _, gK, _, _ = O.misfit_gradient(O.Grid(K0, h, dt, prof, local=loc), nt, src, wav, rec, dobs, checkpoint_every=9)
    nodes = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(5)] + [(7, 6, 8), (0, 0, 0), (13, 12, 14)]
    scale = np.max(np.abs(gK))
    for node in nodes:
        eps = 1e-4 * K0[node]
        Kp, Km = K0.copy(), K0.copy()
        Kp[node] += eps
        Km[node] -= eps
        Jp, _ = O.misfit(O.Grid(Kp, h, dt, prof, local=loc), nt, src, wav, rec, dobs)
        Jm, _ = O.misfit(O.Grid(Km, h, dt, prof, local=loc), nt, src, wav, rec, dobs)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(gK[node] - fd) <= 1e-6 * scale + 1e-5 * abs(fd), (node, gK[node], fd)
