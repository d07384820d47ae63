"""The seeded input generators follow the recipe they state (the layered model,
the Ricker wavelet of Sec. 4.2, shot and receiver layouts, random states and
the workload presets), and hold no method arithmetic: they import neither the
library nor the oracle.  CPU only."""
import math
import pathlib

import numpy as np
import pytest

from paper_2606_06910_gb300 import synth


def test_generators_import_neither_library_nor_oracle():
    src = pathlib.Path(synth.__file__).read_text()
    for bad in ("import oracle", "from oracle", "_lib", "fdtd", "ctypes"):
        assert bad not in src, bad


def test_ricker_peak_zero_crossings_and_first_sample():
    f0, dt = 15.0, 1e-4
    t0 = 1.2 / f0
    w = synth.ricker(4000, dt, f0)
    n0 = int(round(t0 / dt))
    assert w[n0] == pytest.approx(1.0, abs=1e-6) and np.argmax(w) == n0
    # zero crossings at a^2 = 1/2, i.e. t0 +- 1 / (pi f0 sqrt 2)
    tz = 1.0 / (math.pi * f0 * math.sqrt(2.0))
    for t in (t0 - tz, t0 + tz):
        a = math.pi * f0 * (t - t0)
        assert abs((1 - 2 * a * a) * math.exp(-a * a)) < 1e-12
        n = int(t / dt)
        assert w[n] * w[n + 1] <= 0.0
    # the delay puts the first sample near -1.85e-5 of the peak
    assert w[0] == pytest.approx((1 - 2 * (1.2 * math.pi) ** 2) * math.exp(-(1.2 * math.pi) ** 2), rel=1e-12)
    assert -2e-5 < w[0] < -1.7e-5
    # zero mean over the whole pulse (the Ricker wavelet has no DC part)
    assert abs(w.sum() * dt) < 1e-6
    assert np.allclose(synth.ricker(50, 1e-3, 10.0, amplitude=3.0), 3.0 * synth.ricker(50, 1e-3, 10.0))


def test_layered_model_recipe():
    shape = (120, 40, 56)
    v = synth.layered_model(shape, seed=5)
    levels = np.linspace(1500.0, 4500.0, 10).astype(np.float32)
    assert v.dtype == np.float32 and v.shape == shape
    assert set(np.unique(v)) <= set(levels) and len(np.unique(v)) == 10
    assert np.all(v[0] == 1500.0) and np.all(v[-1] == 4500.0)
    # velocity never decreases with depth in any column
    assert np.all(np.diff(v, axis=0) >= 0)
    # each interface lies within amp_cells of its mean depth (i + 1) nz / 10
    for i in range(9):
        depth = np.argmax(v > levels[i], axis=0)     # first node below interface i
        mean = (i + 1) * shape[0] / 10
        assert np.all(depth >= math.floor(mean - 5)) and np.all(depth <= math.ceil(mean + 5) + 1)
    assert np.array_equal(v, synth.layered_model(shape, seed=5))
    assert not np.array_equal(v, synth.layered_model(shape, seed=6))


def test_layouts_stay_in_the_interior():
    shape, L = (60, 70, 80), (5, 7, 6, 4, 8, 9)
    rec = synth.receiver_grid(shape, L, 6, 5, 8)
    assert rec.shape == (30, 3) and rec.dtype == np.int32 and np.all(rec[:, 0] == 8)
    assert rec[:, 1].min() == L[2] and rec[:, 1].max() == shape[1] - 1 - L[3]
    assert rec[:, 2].min() == L[0] and rec[:, 2].max() == shape[2] - 1 - L[1]
    assert len({tuple(r) for r in rec}) == 30
    src = synth.shot_positions(shape, L, seed=3, nshots=50, z=12)
    assert np.all(src[:, 0] == 12)
    assert np.all((src[:, 1] >= L[2]) & (src[:, 1] < shape[1] - L[3]))
    assert np.all((src[:, 2] >= L[0]) & (src[:, 2] < shape[2] - L[1]))
    assert np.array_equal(src, synth.shot_positions(shape, L, seed=3, nshots=50, z=12))
    n, Lc = 96, 12
    pos, th, faces = synth.angled_sources(n, Lc, 40, seed=1)
    assert np.all((pos >= Lc + 6) & (pos <= n - 1 - Lc - 6))
    assert np.all((th >= 0.0) & (th <= 80.0)) and set(faces) <= set(synth.FACE_ORDER)
    fr = synth.face_receivers(n, Lc, 4)
    assert fr.shape == (6 * 16, 3) and np.all((fr >= Lc + 2) & (fr <= n - 1 - Lc - 2))
    f = synth.frequency_groups((5.0, 30.0), 5, seed=2)
    edges = np.linspace(5.0, 30.0, 6)
    assert all(edges[k] <= f[k] <= edges[k + 1] for k in range(5))


def test_random_state_memory_variables_only_in_their_slabs():
    shape, L = (20, 24, 28), (3, 4, 2, 5, 1, 6)
    st = synth.random_state(shape, L, seed=9, p_scale=2.0, psiv_scale=0.5)
    assert abs(float(st["p"].std()) - 2.0) < 0.1 and abs(float(st["vx"].std()) - 1.0) < 0.05
    masks = {"x": synth.slab_mask(shape[2], L[0], L[1])[None, None, :],
             "y": synth.slab_mask(shape[1], L[2], L[3])[None, :, None],
             "z": synth.slab_mask(shape[0], L[4], L[5])[:, None, None]}
    for kind in ("psiv", "psip"):
        for ax, m in masks.items():
            a = st[f"{kind}_{ax}"]
            m = np.broadcast_to(m, shape)
            assert np.all(a[~m] == 0.0) and np.all(a[m] != 0.0), (kind, ax)


def test_presets_match_the_benchmark_configurations():
    w = synth.preset("homog64")
    assert w.shape == (64,) * 3 and w.cpml_cells == (10,) * 6 and w.dt == pytest.approx(2.5e-3)
    assert np.array_equal(w.sources(), [[32, 32, 32]])
    w = synth.preset("layered512")
    assert w.shape == (512,) * 3 and w.cpml_cells == (20,) * 6 and w.R == 1e-8 and w.nt == 1000
    assert w.dt == pytest.approx(0.5 * 10.0 / 4500.0) and w.f0 == 10.0
    assert w.sources()[0, 0] == 30
    w = synth.preset("layered1024")
    assert w.shape == (1024,) * 3 and w.nt == 500
    w = synth.preset("adjoint256")
    assert w.nshots == 16 and w.extra["checkpoint_every"] == 50 and w.extra["receivers"] == (128, 128)
    assert w.wavelet(800).shape == (16, 800)
    with pytest.raises(KeyError):
        synth.preset("nope")
