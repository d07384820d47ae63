"""Pins of the oracle's source injection and receiver sampling order.

Reading of the paper (it prints only the wavelet, Sec. 4.2): the pressure
source adds w[n] to p after the pressure update of step n, and the receivers
then sample p.  The symmetry, dispersion and energy pins run without a
source, so they cannot see this order; the cases below fix it by hand, from
a zero state with one impulse w[0] = 1:

  step 0: v stays 0, p stays 0, then p[s] = w[0]      -> trace[0] at s is w[0],
                                                          at s + e_x it is 0;
  step 1: v_x(s + m) = -dt/rho (1/h) sum_l a_l (p(s+m+l) - p(s+m-l)),
          i.e. v_x(s + m) = +dt a_m w0 / h, v_x(s - m) = -dt a_m w0 / h (m = 1..4);
          the pressure at s + e_x then loses dt K D_x v_x(s + 1) with
          D_x v_x(s + 1) = (dt w0 / h^2) 2 sum_{l=1..3} a_l a_{l+1}
          (D_y v_y and D_z v_z vanish off the source's lines), and at s
          p(s) = w0 (1 - 6 K dt^2 / h^2 sum_l a_l^2).

Planted copies of the run loop (injecting before the velocity stage,
sampling before the injection, sampling before the pressure stage), built from
the oracle's own stage functions, must fail these pins.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O

SHAPE = (17, 15, 19)
H, DT, K = 10.0, 1.0e-3, 2500.0 ** 2
SRC = (8, 7, 9)
A = [float(x) for x in O.first_derivative_weights(4)]


def _grid():
    return O.Grid(np.full(SHAPE, K), H, DT)


def _receivers():
    z, y, x = SRC
    return np.array([[z, y, x], [z, y, x + 1], [z, y + 1, x], [z + 1, y, x], [z, y + 1, x + 1]], dtype=np.int64)


def _wavelet(n):
    w = np.zeros(n)
    w[0] = 1.0
    return w


def _by_hand():
    """Expected traces of the two steps at the receivers of _receivers()."""
    w0 = 1.0
    s_neigh = 2.0 * sum(A[l] * A[l + 1] for l in range(3))
    s_self = sum(a * a for a in A)
    at_s = w0 * (1.0 - 6.0 * K * DT * DT / (H * H) * s_self)
    at_nb = -K * DT * DT / (H * H) * s_neigh * w0
    # step 0: only the source node; step 1: the three axis neighbours are
    # equal by symmetry of the isotropic stencil, the diagonal one stays 0
    return np.array([[w0, 0.0, 0.0, 0.0, 0.0], [at_s, at_nb, at_nb, at_nb, 0.0]])


def _run_loop(order, nsteps=2):
    """A Python copy of the oracle's run loop from its stage functions, with
    the stages in the given order ('v', 'p', 'inject', 'sample')."""
    g = _grid()
    st = O.State(SHAPE)
    rec = _receivers()
    w = _wavelet(nsteps)
    out = np.zeros((nsteps, len(rec)))
    for n in range(nsteps):
        for stage in order:
            if stage == "v":
                O.velocity_stage(g, st)
            elif stage == "p":
                O.pressure_stage(g, st)
            elif stage == "inject":
                p = st["p"]
                p[SRC] += w[n]
                st["p"] = p
            else:
                out[n] = [st["p"][tuple(r)] for r in rec]
    return out


def _matches_by_hand(tr):
    ref = _by_hand()
    if tr[0, 0] != ref[0, 0] or np.any(tr[0, 1:] != 0.0):
        return False
    return np.allclose(tr[1], ref[1], rtol=1e-12, atol=1e-15)


def test_oracle_run_injects_after_pressure_then_samples():
    tr = O.run(_grid(), O.State(SHAPE), 2, 0, SRC, _wavelet(2), _receivers())
    ref = _by_hand()
    # step 0: the receiver at the source reads w[0] exactly, the others 0
    assert tr[0, 0] == 1.0
    assert np.all(tr[0, 1:] == 0.0)
    # step 1: one impulse through one velocity and one pressure stage
    np.testing.assert_allclose(tr[1], ref[1], rtol=1e-12, atol=1e-15)
    assert _matches_by_hand(tr)


def test_python_copy_of_the_loop_equals_oracle_run():
    tr = O.run(_grid(), O.State(SHAPE), 2, 0, SRC, _wavelet(2), _receivers())
    np.testing.assert_array_equal(_run_loop(("v", "p", "inject", "sample")), tr)


@pytest.mark.parametrize("order", [
    ("inject", "v", "p", "sample"),     # source before the velocity stage
    ("v", "p", "sample", "inject"),     # receivers before the source
    ("v", "sample", "p", "inject"),     # receivers before the pressure stage
])
def test_planted_orders_fail_the_pin(order):
    assert not _matches_by_hand(_run_loop(order))
