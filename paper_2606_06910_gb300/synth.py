"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
FP64 oracle.

This module generates inputs only (velocity models, wavelets, source and
receiver layouts, random states, workload presets).  It holds none of the
method's arithmetic: no derivative, no CPML coefficient, no time step.  It
imports nothing from the CUDA library or from the oracle.

The paper's workloads are synthetic grids (Sec. 4 and Sec. 6, Tab. 10); the
layered model, shot and receiver layouts below are this package's recipe for
the presets, since the paper prints none of them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FACE_ORDER = ("x_lo", "x_hi", "y_lo", "y_hi", "z_lo", "z_hi")


def ricker(nt: int, dt: float, f0: float, t0: float | None = None, amplitude: float = 1.0):
    """Ricker wavelet s(t) = (1 - 2 a^2) exp(-a^2), a = pi f0 (t - t0), sampled
    at t = n dt (Sec. 4.2).  The paper gives no delay; t0 defaults to 1.2/f0 so
    the first sample is ~1e-5 of the peak."""
    if t0 is None:
        t0 = 1.2 / f0
    t = np.arange(nt, dtype=np.float64) * dt
    a = math.pi * f0 * (t - t0)
    return amplitude * (1.0 - 2.0 * a * a) * np.exp(-a * a)


def _smooth_field(rng, ny, nx, n_modes=8):
    """Sum of n_modes random low-wavenumber cosines over the (y, x) plane,
    scaled so that max |xi| = 1."""
    y = np.arange(ny)[:, None] / max(ny, 1)
    x = np.arange(nx)[None, :] / max(nx, 1)
    xi = np.zeros((ny, nx))
    for _ in range(n_modes):
        ky, kx = rng.integers(0, 4, size=2)
        ph = rng.uniform(0, 2 * math.pi)
        amp = rng.uniform(0.5, 1.0)
        xi += amp * np.cos(2 * math.pi * (ky * y + kx * x) + ph)
    m = np.max(np.abs(xi))
    return xi / m if m > 0 else xi


def layered_model(shape, seed: int, n_layers: int = 10, vmin: float = 1500.0,
                  vmax: float = 4500.0, amp_cells: float = 5.0, n_modes: int = 8,
                  dtype=np.float32):
    """Velocity model [nz, ny, nx]: n_layers layers whose velocities rise
    linearly from vmin (top) to vmax (bottom); the mean interfaces are equally
    spaced in z and each interface i is displaced by amp_cells * xi_i(y, x),
    xi_i a smooth seeded field with max |xi_i| = 1 (NumPy PCG64 seed)."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    vel_layers = np.linspace(vmin, vmax, n_layers)
    depth = np.zeros((n_layers - 1, ny, nx))
    for i in range(n_layers - 1):
        mean = (i + 1) * nz / n_layers
        depth[i] = mean + amp_cells * _smooth_field(rng, ny, nx, n_modes)
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    layer = np.zeros(shape, dtype=np.int32)
    for i in range(n_layers - 1):
        layer += (z >= depth[i][None, :, :]).astype(np.int32)
    return vel_layers[layer].astype(dtype)


def homogeneous_model(shape, c: float, dtype=np.float32):
    return np.full(shape, c, dtype=dtype)


def gaussian_smooth(vel, sigma_cells: float, dtype=np.float32):
    """Gaussian-smoothed copy of a model (starting model of the gradient
    workload), edges handled by nearest-value extension."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(np.asarray(vel, dtype=np.float64), sigma=sigma_cells,
                           mode="nearest").astype(dtype)


def uniform_interior_xy(rng, shape, L, count: int):
    """count (y, x) positions drawn uniformly in the CPML-free interior."""
    nz, ny, nx = shape
    ys = rng.integers(L[2], ny - L[3], size=count)
    xs = rng.integers(L[0], nx - L[1], size=count)
    return ys, xs


def shot_positions(shape, L, seed: int, nshots: int, z: int):
    """nshots sources (z, y, x) at depth z, (y, x) seeded uniform in the interior."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ys, xs = uniform_interior_xy(rng, shape, L, nshots)
    return np.stack([np.full(nshots, z), ys, xs], axis=1).astype(np.int32)


def receiver_grid(shape, L, nry: int, nrx: int, z: int):
    """nry x nrx receivers evenly spaced (rounded linspace) over the interior
    (y, x) range, on depth z.  Returns int32 [nry*nrx, 3] of (z, y, x)."""
    nz, ny, nx = shape
    ys = np.round(np.linspace(L[2], ny - 1 - L[3], nry)).astype(np.int32)
    xs = np.round(np.linspace(L[0], nx - 1 - L[1], nrx)).astype(np.int32)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([np.full(yy.size, z, np.int32), yy.ravel(), xx.ravel()], axis=1)


def slab_mask(n: int, lo: int, hi: int):
    m = np.zeros(n, dtype=bool)
    m[:lo] = True
    if hi > 0:
        m[n - hi:] = True
    return m


def random_state(shape, L, seed: int, p_scale=1.0, v_scale=1.0, psiv_scale=1.0,
                 psip_scale=1.0, dtype=np.float32):
    """Seeded random wavefield state for parity tests: p, vx, vy, vz standard
    normal times their scale; each memory variable psi_{v,d}, psi_{p,d}
    standard normal times its scale inside the d-slabs and zero elsewhere.
    Returns a dict of arrays [nz, ny, nx]."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    out["p"] = (p_scale * rng.standard_normal(shape)).astype(dtype)
    for ax in "xyz":
        out["v" + ax] = (v_scale * rng.standard_normal(shape)).astype(dtype)
    masks = [slab_mask(nx, L[0], L[1])[None, None, :],
             slab_mask(ny, L[2], L[3])[None, :, None],
             slab_mask(nz, L[4], L[5])[:, None, None]]
    for kind, sc in (("psiv", psiv_scale), ("psip", psip_scale)):
        for d, ax in enumerate("xyz"):
            a = sc * rng.standard_normal(shape)
            out[f"{kind}_{ax}"] = np.where(masks[d], a, 0.0).astype(dtype)
    return out


# ----------------------------------------------------------------------------
# Workload presets
# ----------------------------------------------------------------------------


@dataclass
class Workload:
    """One synthetic workload: grid, material recipe, CPML, source and steps."""
    name: str
    shape: tuple
    h: float
    nt: int
    f0: float
    cpml_cells: tuple
    R: float
    kappa_max: float = 5.0
    alpha_frac: float = 0.05
    q: int = 3
    model: str = "homogeneous"      # or "layered"
    c: float = 2000.0               # homogeneous velocity
    seed: int = 0
    cfl: float = 0.5
    vmax: float = 4500.0
    nshots: int = 1
    src_depth: int | None = None    # None: grid centre
    extra: dict = field(default_factory=dict)

    @property
    def c_max(self) -> float:
        return self.c if self.model == "homogeneous" else self.vmax

    @property
    def dt(self) -> float:
        """dt from c_max dt / h = cfl."""
        return self.cfl * self.h / self.c_max

    def velocity(self, shape=None, dtype=np.float32):
        shape = tuple(shape or self.shape)
        if self.model == "homogeneous":
            return homogeneous_model(shape, self.c, dtype)
        return layered_model(shape, self.seed, vmax=self.vmax, dtype=dtype)

    def sources(self, shape=None):
        shape = tuple(shape or self.shape)
        nz, ny, nx = shape
        if self.src_depth is None:
            return np.array([[nz // 2, ny // 2, nx // 2]] * self.nshots, dtype=np.int32)
        return shot_positions(shape, self.cpml_cells, self.seed + 1000, self.nshots,
                              self.src_depth)

    def wavelet(self, nt=None):
        w = ricker(nt or self.nt, self.dt, self.f0)
        return np.tile(w[None, :], (self.nshots, 1)).astype(np.float32)


def preset(name: str) -> Workload:
    """Named workloads (sizes from the five benchmark configurations)."""
    if name == "homog64":
        # 64^3, c = 2000 m/s, dx = 10 m, CFL 0.5, 15 Hz Ricker at the centre,
        # 10 CPML cells per face, cubic grading, R = 1e-5, 200 steps.
        return Workload("homog64", (64, 64, 64), 10.0, 200, 15.0, (10,) * 6, 1e-5,
                        model="homogeneous", c=2000.0)
    if name == "layered512":
        # 512^3 layered 1500-4500 m/s (seed 2), dx = 10 m, 20 CPML cells,
        # R = 1e-8, 10 Hz Ricker 30 cells below the top face, 1000 steps.
        return Workload("layered512", (512, 512, 512), 10.0, 1000, 10.0, (20,) * 6, 1e-8,
                        model="layered", seed=2, src_depth=30)
    if name == "layered256":
        # smaller grid of the same recipe (profiling captures, quick runs)
        return Workload("layered256", (256, 256, 256), 10.0, 1000, 10.0, (20,) * 6, 1e-8,
                        model="layered", seed=2, src_depth=30)
    if name == "layered1024":
        return Workload("layered1024", (1024, 1024, 1024), 10.0, 500, 10.0, (20,) * 6, 1e-8,
                        model="layered", seed=3, src_depth=30)
    if name == "layered128":
        # accuracy instance of the 1024^3 precision workload (same generator, seed 3)
        return Workload("layered128", (128, 128, 128), 10.0, 500, 10.0, (20,) * 6, 1e-8,
                        model="layered", seed=3, src_depth=30)
    if name == "adjoint256":
        return Workload("adjoint256", (256, 256, 256), 10.0, 800, 10.0, (20,) * 6, 1e-8,
                        model="layered", seed=4, nshots=16, src_depth=20,
                        extra=dict(checkpoint_every=50, receivers=(128, 128), smooth_sigma=8.0))
    if name == "adjoint48":
        return Workload("adjoint48", (48, 48, 48), 10.0, 200, 10.0, (8,) * 6, 1e-8,
                        model="layered", seed=4, nshots=2, src_depth=8,
                        extra=dict(checkpoint_every=50, receivers=(8, 8), smooth_sigma=3.0))
    raise KeyError(name)
