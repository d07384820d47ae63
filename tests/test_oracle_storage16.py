"""Pins of the oracle's 16-bit storage emulation (the precision form: FP16 /
BF16 storage of p, v and the memory variables, arithmetic at full precision).

The emulation rounds every stored value to nearest, ties to even, in the
storage format.  It is pinned by:
  - the rounding itself against numpy's float16 and torch's bfloat16
    conversions (independent implementations of the IEEE / bfloat16 rounding);
  - the reduction to the FP64 oracle, bit for bit, when nothing is rounded;
  - the error of a run against the FP64 oracle scaling with the unit roundoff
    of the format: BF16 (8-bit significand) about 2^3 times FP16 (11 bits);
  - the size of the error not depending on a power-of-two storage scale.
CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_06910_gb300 import synth


def test_round16_matches_numpy_float16():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4000) * np.exp(rng.uniform(-18, 11, 4000))
    x = x[np.abs(x) < 65504.0]
    got = np.array([O.round16(v, "f16") for v in x])
    np.testing.assert_array_equal(got, x.astype(np.float16).astype(np.float64))
    # ties go to the even neighbour
    assert O.round16(1 + 2 ** -11, "f16") == 1.0
    assert O.round16(1 + 3 * 2 ** -11, "f16") == 1 + 2 ** -9


def test_round16_matches_torch_bfloat16():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(4000) * np.exp(rng.uniform(-60, 60, 4000))).astype(np.float32).astype(np.float64)
    got = np.array([O.round16(v, "bf16") for v in x])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(got, ref)
    assert O.round16(1 + 2 ** -8, "bf16") == 1.0
    assert O.round16(1 + 3 * 2 ** -8, "bf16") == 1 + 2 ** -6


def _instance():
    shape, cells, h = (40, 36, 44), (8, 8, 8, 8, 8, 8), 10.0
    vel = synth.layered_model(shape, seed=7).astype(np.float64)
    dt = 0.5 * h / vel.max()
    prof = O.make_profiles(shape, cells, h, dt, vel.max(), R=1e-6)
    src = (14, 18, 22)
    wav = synth.ricker(120, dt, 25.0)
    rec = synth.receiver_grid(shape, cells, 3, 3, 10)
    return shape, vel, h, dt, prof, src, wav, rec


def _run(store=None, mask=15, sp=1.0, sv=1.0, nsteps=120):
    shape, vel, h, dt, prof, src, wav, rec = _instance()
    g = O.Grid(vel * vel, h, dt, prof, store=store, store_mask=mask, scale_p=sp, scale_v=sv)
    st = O.State(shape)
    tr = O.run(g, st, nsteps, 0, src, wav, rec)
    return st, tr


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_no_rounding_reduces_to_the_fp64_oracle():
    ref, tr_ref = _run()
    for store, mask in (("f16", 0), ("bf16", 0)):
        st, tr = _run(store, mask)
        for k in O.FIELDS:
            np.testing.assert_array_equal(st[k], ref[k])
        np.testing.assert_array_equal(tr, tr_ref)


def test_error_scales_with_the_unit_roundoff():
    ref, tr_ref = _run()
    vmax = float(_instance()[1].max())
    st16, _ = _run("f16", 15, 1024.0, vmax)
    stbf, _ = _run("bf16", 15, 1.0, vmax)
    e16, ebf = _rel(st16["p"], ref["p"]), _rel(stbf["p"], ref["p"])
    # nonzero, small, and about 8x apart (2^-11 against 2^-8 relative spacing)
    assert 1e-6 < e16 < 1e-2
    assert 4.0 < ebf / e16 < 16.0, (e16, ebf)
    # every rounded field is on the format's grid after the scale
    assert all(O.round16(v * 1024.0, "f16") == v * 1024.0 for v in st16["p"].ravel()[::97])
    sv = 1024.0 * vmax   # not a power of two: the round trip through the scale is within an FP64 ulp
    assert all(abs(O.round16(v * sv, "f16") - v * sv) <= 1e-12 * abs(v * sv) for v in st16["vx"].ravel()[::97])


def test_error_size_does_not_depend_on_the_scale():
    # a power-of-two scale moves values relative to FP16's subnormal range
    # only, so the size of the rounding error stays the same; the noise itself
    # differs from scale to scale (one rounding decided differently spreads),
    # so only its size is compared
    ref, _ = _run()
    errs = [_rel(_run("f16", 15, sp, 4096.0)[0]["p"], ref["p"]) for sp in (1.0, 1024.0, 4096.0)]
    assert max(errs) < 1.5 * min(errs), errs


def test_planted_rounding_of_the_used_velocity_is_caught():
    # planted mistake: rounding v before the pressure update uses it (the
    # form keeps the new velocity unrounded in registers for that update) must
    # change the run; the emulation rounds v only once the step is done
    shape, vel, h, dt, prof, src, wav, rec = _instance()
    g = O.Grid(vel * vel, h, dt, prof, store="f16", scale_p=1024.0, scale_v=float(vel.max()))
    good = O.State(shape)
    O.run(g, good, 40, 0, src, wav, rec)
    planted = O.State(shape)
    for n in range(40):
        O.velocity_stage(g, planted)
        sv = 1024.0 * vel.max()
        for k in ("vx", "vy", "vz"):
            planted[k] = (planted[k] * sv).astype(np.float16).astype(np.float64) / sv
        O.pressure_stage(g, planted)
        p = planted["p"]
        if n < wav.size:
            p[src] += wav[n]
        planted["p"] = p
        O.store_state(g, planted)
    assert not np.array_equal(planted["p"], good["p"])
