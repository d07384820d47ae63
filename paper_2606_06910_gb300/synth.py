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


def face_receivers(n: int, L: int, k: int, inset: int = 2) -> np.ndarray:
    """k x k receivers on each of the six planes `inset` nodes inside the
    inner edge of an L-cell layer on a cube of n nodes, over the interior
    extent of that plane.  Returns int32 [6 k^2, 3] of (z, y, x)."""
    lo, hi = L + inset, n - 1 - L - inset
    span = np.round(np.linspace(lo, hi, k)).astype(np.int32)
    a, b = np.meshgrid(span, span, indexing="ij")
    a, b = a.ravel(), b.ravel()
    out = []
    for plane in (lo, hi):
        out.append(np.stack([np.full_like(a, plane), a, b], 1))   # z faces
        out.append(np.stack([a, np.full_like(a, plane), b], 1))   # y faces
        out.append(np.stack([a, b, np.full_like(a, plane)], 1))   # x faces
    return np.concatenate(out).astype(np.int32)


def angled_sources(n: int, L: int, nshots: int, seed: int, angles=(0.0, 80.0), inset: int = 2,
                   d_max: int = 40, clearance: int = 6):
    """Point sources for CPML reflection tasks on a cube of n nodes with an
    L-cell layer: shot s draws a face, an incidence angle theta in `angles`
    (degrees) and an azimuth, and sits at normal distance d from the face's
    receiver plane (face_receivers) with lateral offset d tan(theta) from the
    plane's centre, so that its wave meets the middle of that face at theta;
    d is as large as fits (at most d_max) with the source at least
    `clearance` nodes clear of the layer.  Returns (int32 [nshots, 3] of
    (z, y, x), the angles in degrees, the faces in FACE_ORDER order)."""
    rng = np.random.default_rng(seed)
    lo_src, hi_src = L + clearance, n - 1 - L - clearance
    plane = {0: L + inset, 1: n - 1 - L - inset}
    centre = (n - 1) / 2.0
    half = centre - lo_src
    out, th, fc = [], [], []
    for _ in range(nshots):
        face = int(rng.integers(6))
        theta = float(rng.uniform(*angles))
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        t = math.tan(math.radians(theta))
        d = float(d_max) if t * d_max <= half else half / t
        d = max(d, float(lo_src - plane[0]) + 1.0)
        axis, side = face // 2, face % 2
        normal = plane[side] + (d if side == 0 else -d)
        lat = (centre + d * t * math.cos(phi), centre + d * t * math.sin(phi))
        pos = [0.0, 0.0, 0.0]                   # (x, y, z)
        pos[axis] = normal
        others = [a for a in range(3) if a != axis]
        pos[others[0]], pos[others[1]] = lat
        zyx = [int(np.clip(round(pos[2 - i]), lo_src, hi_src)) for i in range(3)]
        out.append(zyx)
        th.append(theta)
        fc.append(FACE_ORDER[face])
    return np.array(out, dtype=np.int32), np.array(th), fc


def frequency_groups(freqs, nfreq: int, seed: int):
    """nfreq dominant frequencies, one drawn uniformly (seeded) from each of
    nfreq equal sub-ranges of freqs = (f_lo, f_hi)."""
    rng = np.random.default_rng(seed)
    edges = np.linspace(freqs[0], freqs[1], nfreq + 1)
    return [float(rng.uniform(edges[k], edges[k + 1])) for k in range(nfreq)]


def mlp_init_params(seed: int, scale1=0.5, scale2=0.2, scale3=0.1) -> np.ndarray:
    """Seeded initial weights of the 4 -> 64 -> 64 -> 3 network (normal,
    fixed scales) and zero biases, flattened as W1, b1, W2, b2, W3, b3;
    float64."""
    rng = np.random.default_rng(seed)
    W1 = scale1 * rng.standard_normal((64, 4))
    W2 = scale2 * rng.standard_normal((64, 64))
    W3 = scale3 * rng.standard_normal((3, 64))
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(3)])


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
