"""FP64 oracle for the radius-4 acoustic FDTD + CPML path (test infrastructure).

Every function states the passage of the paper it follows.  Where the paper is
silent the reading used is named in the docstring; the same readings are
listed in the repository's design notes.

Conventions
-----------
* Fields are float64 arrays shaped ``[nz, ny, nx]`` (x fastest).
* Axis numbering 0 = x, 1 = y, 2 = z.
* CPML cells per face are given as ``L = (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi)``;
  the cells lie inside the grid (the grid extent includes the layer).
"""
from __future__ import annotations

import ctypes
import math
from fractions import Fraction

import numpy as np

from . import lib as _clib

# ----------------------------------------------------------------------------
# Finite-difference weights (Sec. 3.1; the paper does not print a_l)
# ----------------------------------------------------------------------------


def fd_weights(offsets, m: int):
    """Exact rational weights c_j with sum_j c_j f(x + j h) = h^m f^(m)(x) + O(h^{len}).

    Solves the Vandermonde system sum_j c_j j^k = m! delta_{k,m},
    k = 0..len(offsets)-1, in exact rationals (Gauss-Jordan on Fractions).
    Pinned by: the Tab. 6 spatial-convergence values (second derivative,
    orders 2/4/8) and exact differentiation of polynomials (first derivative).
    """
    offs = [Fraction(o) for o in offsets]
    n = len(offs)
    A = [[o ** k for o in offs] + [Fraction(math.factorial(m) if k == m else 0)]
         for k in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return [A[k][n] for k in range(n)]


def first_derivative_weights(r: int = 4):
    """a_1..a_r of the centred first derivative of order 2r (Sec. 3.1).

    Reading: the paper's centred operator (f_{i+l} - f_{i-l}) with the unique
    weights that make it exact for polynomials of degree <= 2r.  For r = 4 this
    gives 4/5, -1/5, 4/105, -1/280.
    """
    c = fd_weights(range(-r, r + 1), 1)
    return [c[r + l] for l in range(1, r + 1)]


def second_derivative_weights(r: int):
    """c_0..c_r of the standard (2r+1)-point second derivative (Tab. 6 helper)."""
    c = fd_weights(range(-r, r + 1), 2)
    return [c[r + l] for l in range(0, r + 1)]


WEIGHTS = [float(x) for x in first_derivative_weights(4)]


def staggered_weights(r: int = 4):
    """c_1..c_r of the staggered first derivative (the Yee reading of Sec. 3.1):
    (f(x + (l - 1/2) h) - f(x - (l - 1/2) h)) with the unique weights exact for
    polynomials of degree <= 2r - 1.  For r = 4: 1225/1024, -245/3072, 49/5120,
    -5/7168."""
    offs = [Fraction(2 * k - 1, 2) for k in range(-r + 1, r + 1)]   # -7/2 .. 7/2
    c = fd_weights(offs, 1)
    return [c[r - 1 + l] for l in range(1, r + 1)]


STAGGERED_WEIGHTS = [float(x) for x in staggered_weights(4)]


# ----------------------------------------------------------------------------
# CPML profiles (Sec. 3.2, Tab. 2)
# ----------------------------------------------------------------------------


def cpml_coefficients(sigma, kappa, alpha, dt):
    """Recursive coefficients of Sec. 3.2:
    b = exp(-(sigma/kappa + alpha) dt),  a = sigma (b - 1) / (kappa (sigma + kappa alpha)).
    Where sigma = 0 the memory variable receives nothing (a = 0)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    b = np.exp(-(sigma / kappa + alpha) * dt)
    den = kappa * (sigma + kappa * alpha)
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.where(sigma > 0, sigma * (b - 1.0) / np.where(den == 0, 1.0, den), 0.0)
    return b, a, 1.0 / kappa


def sigma_max(L: int, h: float, c_ref: float, R: float, q: int = 3) -> float:
    """sigma_max = -(q+1) c_ref ln(R) / (2 L h).

    Reading of Sec. 3.2 / Tab. 2: the printed -4 log(R)/(2 L h) carries no
    velocity and has units of 1/m; a reference velocity c_ref restores 1/s, and
    4 = q + 1 for the cubic grading.  With this value the continuous layer's
    normal-incidence round trip exp(-2 int_0^{Lh} sigma(s)/c ds) equals R
    exactly (pinned in tests)."""
    if L <= 0:
        return 0.0
    return -(q + 1) * c_ref * math.log(R) / (2.0 * L * h)


def axis_profile(n: int, L_lo: int, L_hi: int, h: float, dt: float, c_ref: float,
                 R: float = 1e-8, q: int = 3, kappa_max: float = 5.0,
                 alpha_frac: float = 0.05):
    """Per-node CPML profile along one axis of n nodes (Sec. 3.2, Tab. 2).

    Normalised depth (reading): rho(i) = (L_lo - i)/L_lo for i < L_lo (the
    outermost node has rho = 1), mirrored on the high face:
    rho(n-1-i) = (L_hi - i)/L_hi for i < L_hi.  Then
    sigma = sigma_max rho^q, kappa = 1 + (kappa_max - 1) rho^q,
    alpha = alpha_frac sigma_max (1 - rho); b, a from cpml_coefficients.
    Returns dict with slab (uint8), rho, sigma, kappa, alpha, b, a, kinv.
    Outside the slabs: slab = 0, kinv = 1, b = a = 0 (unused).

    Also bv, av, kinvv: the same profile at the half nodes i + 1/2 where the
    staggered (Yee) form keeps v (reading: the velocity memory variables use
    the slab index set of p, with depth (L_lo - i - 1/2)/L_lo on the low face
    and (i + 1/2 - (n - 1 - L_hi))/L_hi, clamped to 1, on the high face; the
    half node just inside the high slab, depth 1/(2 L_hi), is left out).
    """
    rho = np.zeros(n)
    slab = np.zeros(n, dtype=np.uint8)
    smax = np.zeros(n)
    for i in range(n):
        if i < L_lo:
            rho[i] = (L_lo - i) / L_lo
            slab[i] = 1
            smax[i] = sigma_max(L_lo, h, c_ref, R, q)
        elif i >= n - L_hi:
            rho[i] = (i - (n - 1 - L_hi)) / L_hi
            slab[i] = 1
            smax[i] = sigma_max(L_hi, h, c_ref, R, q)
    sigma = smax * rho ** q
    kappa = 1.0 + (kappa_max - 1.0) * rho ** q
    alpha = alpha_frac * smax * (1.0 - rho)
    b, a, kinv = cpml_coefficients(sigma, kappa, alpha, dt)
    b = np.where(slab == 1, b, 0.0)
    a = np.where(slab == 1, a, 0.0)
    kinv = np.where(slab == 1, kinv, 1.0)
    rv = np.zeros(n)
    for i in range(n):
        if i < L_lo:
            rv[i] = (L_lo - i - 0.5) / L_lo
        elif i >= n - L_hi:
            rv[i] = min(1.0, (i + 0.5 - (n - 1 - L_hi)) / L_hi)
    bv, av, kinvv = cpml_coefficients(smax * rv ** q, 1.0 + (kappa_max - 1.0) * rv ** q,
                                      alpha_frac * smax * (1.0 - rv), dt)
    bv = np.where(slab == 1, bv, 0.0)
    av = np.where(slab == 1, av, 0.0)
    kinvv = np.where(slab == 1, kinvv, 1.0)
    return dict(slab=slab, rho=rho, sigma=sigma, kappa=kappa, alpha=alpha, b=b, a=a, kinv=kinv,
                rho_v=rv, bv=bv, av=av, kinvv=kinvv)


def make_profiles(shape, L, h, dt, c_ref, R=1e-8, q=3, kappa_max=5.0, alpha_frac=0.05):
    """Profiles for the three axes of a grid shaped (nz, ny, nx); L as in the
    module docstring.  Each axis has its own profile (Sec. 3.2)."""
    nz, ny, nx = shape
    ns = (nx, ny, nz)
    return [axis_profile(ns[d], L[2 * d], L[2 * d + 1], h, dt, c_ref, R, q, kappa_max, alpha_frac)
            for d in range(3)]


def local_profiles(vel, L, h, dt, R=1e-8, q=3, kappa_max=5.0, alpha_frac=0.05, full_shape=None, origin=(0, 0, 0)):
    """Local-velocity grading (the heterogeneous-media extension named in
    Sec. 7): at every node of a d-slab, sigma_max takes the velocity c of
    that node in place of the one reference velocity, so sigma = sigma_max(c)
    rho_d^q and alpha = alpha_frac sigma_max(c) (1 - rho_d), with the node's
    normalised depth rho_d along d; kappa does not depend on c.
    Returns [x, y, z] dicts with b, a, sigma as [nz][ny][nx] arrays (0
    outside the d-slabs); 1/kappa stays the 1D profile of make_profiles.
    full_shape / origin: vel is the box of a larger grid starting at origin
    (z, y, x); depths then follow the larger grid's faces."""
    vel = np.asarray(vel, dtype=np.float64)
    nz, ny, nx = vel.shape
    ns = (nx, ny, nz)
    fz, fy, fx = vel.shape if full_shape is None else full_shape
    fns = (fx, fy, fz)
    org = (origin[2], origin[1], origin[0])
    out = []
    for d in range(3):
        lo, hi = L[2 * d], L[2 * d + 1]
        pr = axis_profile(fns[d], lo, hi, h, dt, 1.0, R, q, kappa_max, alpha_frac)
        sl = slice(org[d], org[d] + ns[d])
        shp = [1, 1, 1]
        shp[2 - d] = ns[d]
        depth = pr["rho"][sl].reshape(shp)
        slab = pr["slab"][sl].reshape(shp).astype(bool)
        Lnode = np.where(np.arange(fns[d]) < lo, lo, hi)[sl].reshape(shp)
        with np.errstate(divide="ignore", invalid="ignore"):
            smax = np.where(slab, -(q + 1) * vel * math.log(R) / (2.0 * np.maximum(Lnode, 1) * h), 0.0)
        sigma = smax * depth ** q
        kappa = 1.0 + (kappa_max - 1.0) * depth ** q
        alpha = alpha_frac * smax * (1.0 - depth)
        b, a, _ = cpml_coefficients(sigma, np.broadcast_to(kappa, vel.shape), alpha, dt)
        slab3 = np.broadcast_to(slab, vel.shape)
        out.append(dict(b=np.ascontiguousarray(np.where(slab3, b, 0.0)),
                        a=np.ascontiguousarray(np.where(slab3, a, 0.0)),
                        sigma=np.ascontiguousarray(np.where(slab3, sigma, 0.0))))
    return out


def no_cpml_profiles(shape):
    """Profiles with no slab anywhere (plain interior update everywhere)."""
    nz, ny, nx = shape
    out = []
    for n in (nx, ny, nz):
        out.append(dict(slab=np.zeros(n, np.uint8), b=np.zeros(n), a=np.zeros(n),
                        kinv=np.ones(n), bv=np.zeros(n), av=np.zeros(n), kinvv=np.ones(n)))
    return out


# ----------------------------------------------------------------------------
# ctypes view of the C core
# ----------------------------------------------------------------------------

_P3 = ctypes.c_void_p * 3


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_long), ("ny", ctypes.c_long), ("nz", ctypes.c_long),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("rho", ctypes.c_double),
                ("w", ctypes.c_double * 4), ("periodic", ctypes.c_int),
                ("K", ctypes.c_void_p), ("b", _P3), ("a", _P3), ("kinv", _P3),
                ("slab", _P3), ("rho_n", ctypes.c_void_p), ("kr", ctypes.c_double * 3),
                ("staggered", ctypes.c_int), ("bv", _P3), ("av", _P3), ("kinvv", _P3),
                ("bn", _P3), ("an", _P3), ("store_bits", ctypes.c_int), ("store_mask", ctypes.c_int),
                ("scale_p", ctypes.c_double), ("scale_v", ctypes.c_double)]


class _State(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p), ("v", _P3), ("psiv", _P3), ("psip", _P3)]


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


FIELDS = ("p", "vx", "vy", "vz", "psiv_x", "psiv_y", "psiv_z", "psip_x", "psip_y", "psip_z")


class State:
    """Wavefield state: p, v_d, psi_{v,d}, psi_{p,d} as full-volume FP64 arrays
    (the memory variables are zero outside their slab and never touched there)."""

    def __init__(self, shape):
        self.shape = tuple(shape)
        self.arrays = {k: np.zeros(self.shape) for k in FIELDS}

    def __getitem__(self, k):
        return self.arrays[k]

    def __setitem__(self, k, val):
        self.arrays[k][...] = val

    def copy(self):
        s = State(self.shape)
        for k in FIELDS:
            s.arrays[k][...] = self.arrays[k]
        return s

    def as_vector(self):
        return np.concatenate([self.arrays[k].ravel() for k in FIELDS])

    @classmethod
    def from_vector(cls, shape, vec):
        s = cls(shape)
        n = int(np.prod(shape))
        for i, k in enumerate(FIELDS):
            s.arrays[k][...] = vec[i * n:(i + 1) * n].reshape(shape)
        return s

    def _c(self):
        st = _State()
        st.p = _ptr(self.arrays["p"])
        for d, ax in enumerate("xyz"):
            st.v[d] = _ptr(self.arrays["v" + ax])
            st.psiv[d] = _ptr(self.arrays["psiv_" + ax])
            st.psip[d] = _ptr(self.arrays["psip_" + ax])
        return st


class Grid:
    """Grid, material and CPML description for the oracle.

    kr: elliptic anisotropy, (x, y, z) factors of the modulus in the
    pressure update, p' = p - dt K sum_d kr_d [...]_d; the axis velocities are
    c sqrt(kr_d) (the 2D demo of Sec. 5 has c_x = 2600, c_z = 1800 m/s).
    K: bulk modulus K = rho c^2 per node (Sec. 3.1); rho: the density, a
    constant or an array [nz][ny][nx] of per-node values (variable density,
    collocated with p and v: the velocity update at a node uses dt / rho of
    that node).
    local: per-node (b, a) of each axis from local_profiles (local-velocity
    grading; the 1D slab flags and 1/kappa still come from profiles).
    staggered: the Yee reading of Sec. 3.1 (v_d at half nodes i + 1/2 along
    d, forward differences p -> v and backward v -> p with the staggered
    weights; the CPML of v uses the half-node profiles bv, av, kinvv).
    Reading (Sec. 3.1 "normalized form"): physical units with rho given
    (1 in every workload here), velocity update scaled by dt/rho, pressure
    update by dt K, and each coefficient multiplies the whole CPML bracket.
    """

    def __init__(self, K, h, dt, profiles=None, rho=1.0, periodic=False, weights=None, kr=(1.0, 1.0, 1.0),
                 staggered=False, local=None, store=None, store_mask=15, scale_p=1.0, scale_v=1.0):
        self.K = np.ascontiguousarray(K, dtype=np.float64)
        self.shape = self.K.shape
        self.h, self.dt = float(h), float(dt)
        if np.ndim(rho) == 0:
            self.rho, self.rho_n = float(rho), None
        else:
            self.rho = 1.0
            self.rho_n = np.ascontiguousarray(rho, dtype=np.float64)
            assert self.rho_n.shape == self.K.shape
        self.periodic = bool(periodic)
        self.kr = tuple(float(r) for r in kr)   # (x, y, z): axis moduli kr_d K
        self.staggered = bool(staggered)
        self.local = None
        if local is not None:
            assert not self.staggered, "local grading: collocated form only"
            self.local = [dict(b=np.ascontiguousarray(lp["b"], dtype=np.float64),
                               a=np.ascontiguousarray(lp["a"], dtype=np.float64)) for lp in local]
            for lp in self.local:
                assert lp["b"].shape == self.shape and lp["a"].shape == self.shape
        if weights is None:
            weights = STAGGERED_WEIGHTS if self.staggered else WEIGHTS
        self.weights = list(weights)
        if profiles is None:
            profiles = no_cpml_profiles(self.shape)
        self.profiles = []
        for pr in profiles:
            self.profiles.append(dict(
                slab=np.ascontiguousarray(pr["slab"], dtype=np.uint8),
                b=np.ascontiguousarray(pr["b"], dtype=np.float64),
                a=np.ascontiguousarray(pr["a"], dtype=np.float64),
                kinv=np.ascontiguousarray(pr["kinv"], dtype=np.float64),
                bv=np.ascontiguousarray(pr.get("bv", pr["b"]), dtype=np.float64),
                av=np.ascontiguousarray(pr.get("av", pr["a"]), dtype=np.float64),
                kinvv=np.ascontiguousarray(pr.get("kinvv", pr["kinv"]), dtype=np.float64)))
        # the 16-bit storage form: FP64 arithmetic, stored fields rounded to
        # FP16 / BF16 (bits of the significand 11 / 8) after scaling as the
        # form stores them (see fdtd_oracle.c: og_store)
        assert store in (None, "f16", "bf16")
        self.store_bits = {None: 0, "f16": 11, "bf16": 8}[store]
        self.store_mask = int(store_mask)
        self.scale_p, self.scale_v = float(scale_p), float(scale_v)
        self._cg = self._make_c()

    def _make_c(self):
        g = _Grid()
        g.nz, g.ny, g.nx = self.shape
        g.h, g.dt, g.rho = self.h, self.dt, self.rho
        for i in range(4):
            g.w[i] = self.weights[i]
        g.periodic = 1 if self.periodic else 0
        g.K = _ptr(self.K)
        for d in range(3):
            pr = self.profiles[d]
            g.b[d] = _ptr(pr["b"])
            g.a[d] = _ptr(pr["a"])
            g.kinv[d] = _ptr(pr["kinv"])
            g.slab[d] = _ptr(pr["slab"])
            g.bv[d] = _ptr(pr["bv"])
            g.av[d] = _ptr(pr["av"])
            g.kinvv[d] = _ptr(pr["kinvv"])
        g.staggered = 1 if self.staggered else 0
        for d in range(3):
            g.bn[d] = _ptr(self.local[d]["b"]) if self.local is not None else None
            g.an[d] = _ptr(self.local[d]["a"]) if self.local is not None else None
        g.rho_n = _ptr(self.rho_n) if self.rho_n is not None else None
        for d in range(3):
            g.kr[d] = self.kr[d]
        g.store_bits, g.store_mask = self.store_bits, self.store_mask
        g.scale_p, g.scale_v = self.scale_p, self.scale_v
        return g


def store_state(grid: Grid, st: State):
    """Round p and v as the 16-bit storage form writes them back at the end
    of a step (no-op without ``store``)."""
    _clib().og_store_state(ctypes.byref(grid._cg), ctypes.byref(st._c()))


def round16(x: float, fmt: str) -> float:
    """x rounded to nearest, ties to even, in FP16 or BF16 (as a double)."""
    f = _clib().og_round16
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_double, ctypes.c_int]
    return float(f(float(x), 11 if fmt == "f16" else 8))


def threads() -> int:
    """OpenMP threads the C core's loops use."""
    f = _clib().og_threads
    f.restype = ctypes.c_long
    return int(f())


def velocity_stage(grid: Grid, st: State):
    """Velocity half step (Sec. 3.1 leapfrog, Sec. 3.2 CPML velocity update)."""
    c = st._c()
    _clib().og_velocity_stage(ctypes.byref(grid._cg), ctypes.byref(c))


def pressure_stage(grid: Grid, st: State, want_bracket=False):
    """Pressure step (Sec. 3.1, Sec. 3.2 CPML pressure update).  Optionally
    returns the bracket sum_d[(1/kappa_d) delta_d v_d + psi_{p,d}] per node."""
    c = st._c()
    s = np.zeros(grid.shape) if want_bracket else None
    _clib().og_pressure_stage(ctypes.byref(grid._cg), ctypes.byref(c),
                              _ptr(s) if s is not None else None)
    return s


def run(grid: Grid, st: State, nsteps: int, n0: int = 0, src=None, wavelet=None, rec=None):
    """Advance ``nsteps`` full steps from time index n0 (state modified in place).

    After the pressure update of step n the wavelet sample w[n] is added at the
    source node (reading: additive pressure source, amplitude as given), and
    every receiver records p.  src: (z, y, x) or None; rec: int array [nrec, 3].
    Returns traces [nsteps, nrec] (FP64)."""
    src_arr = np.array(src if src is not None else (-1, -1, -1), dtype=np.int64)
    if wavelet is None:
        wav = np.zeros(1)
        nt_w = 0
    else:
        wav = np.ascontiguousarray(wavelet, dtype=np.float64)
        nt_w = wav.size
    rec_arr = np.ascontiguousarray(np.zeros((0, 3)) if rec is None else rec, dtype=np.int64)
    nrec = rec_arr.shape[0]
    traces = np.zeros((nsteps, max(nrec, 1)))
    c = st._c()
    _clib().og_run(ctypes.byref(grid._cg), ctypes.byref(c), ctypes.c_long(n0),
                   ctypes.c_long(nsteps), _ptr(src_arr), _ptr(wav), ctypes.c_long(nt_w),
                   ctypes.c_long(nrec), _ptr(rec_arr) if nrec else None, _ptr(traces))
    return traces[:, :nrec]


def adjoint_step(grid: Grid, fwd: State, adj: State, gradK=None, gprof=None):
    """Transpose of one full step (see fdtd_oracle.c:og_adjoint_step).

    fwd: forward state at the start of the step.  adj: adjoint of the state at
    the end of the step (receiver residuals already added), replaced by the
    adjoint at the start.  gradK: [nz,ny,nx] accumulator of dJ/dK.
    gprof: [3, 3, nmax] accumulator of dJ/d(b, a, kinv) per axis and node
    (collocated form with 1D profiles only).  The staggered form transposes
    its own operators and half-node velocity profiles; the local grading's
    per-node (b, a) are transposed too."""
    assert gprof is None or (grid.local is None and not grid.staggered), \
        "adjoint_step: gprof is per axis and node index of the node profiles"
    nmax = max(grid.shape)
    fc = fwd._c()
    ac = adj._c()
    _clib().og_adjoint_step(ctypes.byref(grid._cg), ctypes.byref(fc), ctypes.byref(ac),
                            _ptr(gradK) if gradK is not None else None,
                            _ptr(gprof) if gprof is not None else None,
                            ctypes.c_long(nmax))


# ----------------------------------------------------------------------------
# Misfit and its gradient (data-misfit adjoint, checkpoint + recompute)
# ----------------------------------------------------------------------------


def forward_traces(grid: Grid, nt: int, src, wavelet, rec):
    """Traces [nt, nrec] of one shot from a zero initial state (reading: all
    fields and memory variables start at zero)."""
    st = State(grid.shape)
    return run(grid, st, nt, 0, src, wavelet, rec)


def misfit(grid: Grid, nt, src, wavelet, rec, dobs):
    """J = 1/2 sum_{n,r} (trace[n,r] - dobs[n,r])^2 for one shot."""
    tr = forward_traces(grid, nt, src, wavelet, rec)
    return 0.5 * float(np.sum((tr - dobs) ** 2)), tr


def misfit_gradient(grid: Grid, nt, src, wavelet, rec, dobs, checkpoint_every=10,
                    want_profiles=False):
    """J and dJ/dK (and optionally dJ/d(b, a, kinv) per axis and node) for one
    shot, by the transposed step run backwards in time.

    The forward run keeps a full state copy every ``checkpoint_every`` steps;
    each segment is recomputed from its checkpoint (newest first) before its
    steps are transposed.  Pinned by central finite differences of ``misfit``.
    Returns (J, gradK, gprof or None, traces)."""
    rec = np.asarray(rec, dtype=np.int64)
    C = int(checkpoint_every)
    st = State(grid.shape)
    ckpts = {}
    traces = np.zeros((nt, rec.shape[0]))
    for n in range(nt):
        if n % C == 0:
            ckpts[n] = st.copy()
        traces[n] = run(grid, st, 1, n, src, wavelet, rec)[0]
    resid = traces - dobs
    J = 0.5 * float(np.sum(resid ** 2))

    gradK = np.zeros(grid.shape)
    gprof = np.zeros((3, 3, max(grid.shape))) if want_profiles else None
    adj = State(grid.shape)
    seg_starts = sorted(ckpts.keys(), reverse=True)
    for s0 in seg_starts:
        s1 = min(s0 + C, nt)
        seg = []
        cur = ckpts[s0].copy()
        for n in range(s0, s1):
            seg.append(cur.copy())
            run(grid, cur, 1, n, src, wavelet, None)
        for n in range(s1 - 1, s0 - 1, -1):
            for r in range(rec.shape[0]):
                z, y, x = rec[r]
                adj["p"][z, y, x] += resid[n, r]
            adjoint_step(grid, seg[n - s0], adj, gradK, gprof)
    return J, gradK, gprof, traces


# ----------------------------------------------------------------------------
# Second, independent formulation: the step as an explicit sparse matrix
# ----------------------------------------------------------------------------


def explicit_step_matrix(grid: Grid):
    """The full step u^{n} -> u^{n+1} (no source) as a scipy.sparse matrix on
    the state vector [p, vx, vy, vz, psiv_x..z, psip_x..z] (each block
    nz*ny*nx, x fastest), assembled from the operators of Sec. 3.1-3.2:

      psiv_d' = B_d psiv_d + A_d D_d p
      v_d'    = v_d - dt/rho (Kv_d D_d p + S_d psiv_d')
      psip_d' = B_d psip_d + A_d D_d v_d'
      p'      = p - dt diag(K) sum_d (Kv_d D_d v_d' + S_d psip_d')

    with D_d = 1D difference matrix (zero or periodic ends) kron'd into 3D,
    S_d = slab indicator, B_d = b inside the slab and identity outside,
    A_d = a inside the slab, Kv_d = 1/kappa inside the slab and 1 outside.
    Used only on tiny grids.  Independent of the C loops."""
    import scipy.sparse as sp

    nz, ny, nx = grid.shape
    N = nx * ny * nz
    w = grid.weights

    def d1(n):
        rows, cols, vals = [], [], []
        for i in range(n):
            for l in range(1, 5):
                for sgn in (1, -1):
                    j = i + sgn * l
                    if grid.periodic:
                        j %= n
                    elif j < 0 or j >= n:
                        continue
                    rows.append(i)
                    cols.append(j)
                    vals.append(sgn * w[l - 1] / grid.h)
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    Iz, Iy, Ix = sp.identity(nz), sp.identity(ny), sp.identity(nx)
    D = [sp.kron(Iz, sp.kron(Iy, d1(nx))), sp.kron(Iz, sp.kron(d1(ny), Ix)),
         sp.kron(d1(nz), sp.kron(Iy, Ix))]

    def per_node(vec1d, axis):
        if axis == 0:
            full = np.broadcast_to(vec1d[None, None, :], (nz, ny, nx))
        elif axis == 1:
            full = np.broadcast_to(vec1d[None, :, None], (nz, ny, nx))
        else:
            full = np.broadcast_to(vec1d[:, None, None], (nz, ny, nx))
        return np.ascontiguousarray(full).ravel()

    S, B, A, Kv = [], [], [], []
    for d in range(3):
        pr = grid.profiles[d]
        s = per_node(pr["slab"].astype(np.float64), d)
        S.append(sp.diags(s))
        B.append(sp.diags(np.where(s > 0, per_node(pr["b"], d), 1.0)))
        A.append(sp.diags(s * per_node(pr["a"], d)))
        Kv.append(sp.diags(np.where(s > 0, per_node(pr["kinv"], d), 1.0)))
    I = sp.identity(N)
    dtr = grid.dt / grid.rho
    Kd = sp.diags(grid.K.ravel())

    # velocity stage: rows [p, v, psiv, psip] in terms of the incoming state
    blocks_v = [[None] * 10 for _ in range(10)]
    blocks_v[0][0] = I
    for d in range(3):
        # psiv_d'
        blocks_v[4 + d][4 + d] = B[d]
        blocks_v[4 + d][0] = A[d] @ D[d]
        # v_d' = v_d - dtr (Kv D p + S (B psiv + A D p))
        blocks_v[1 + d][1 + d] = I
        blocks_v[1 + d][0] = -dtr * (Kv[d] @ D[d] + S[d] @ A[d] @ D[d])
        blocks_v[1 + d][4 + d] = -dtr * (S[d] @ B[d])
        blocks_v[7 + d][7 + d] = I
    Mv = sp.bmat(blocks_v, format="csr")

    blocks_p = [[None] * 10 for _ in range(10)]
    blocks_p[0][0] = I
    for d in range(3):
        blocks_p[1 + d][1 + d] = I
        blocks_p[4 + d][4 + d] = I
        blocks_p[7 + d][7 + d] = B[d]
        blocks_p[7 + d][1 + d] = A[d] @ D[d]
        # p' = p - dt K sum_d (Kv D v + S (B psip + A D v))
        blocks_p[0][1 + d] = -grid.dt * Kd @ (Kv[d] @ D[d] + S[d] @ A[d] @ D[d])
        blocks_p[0][7 + d] = -grid.dt * Kd @ (S[d] @ B[d])
    Mp = sp.bmat(blocks_p, format="csr")
    return Mp @ Mv


# ----------------------------------------------------------------------------
# Verification helpers (Sec. 4.1, Tab. 6 / Tab. 7; dispersion; energy)
# ----------------------------------------------------------------------------


def laplacian_convergence_error(order: int, N: int, m: int = 4):
    """Relative L2 and Linf error of the standard (order+1)-point
    second-derivative Laplacian applied to the standing wave
    sin(2 pi m x) sin(2 pi m y) sin(2 pi m z) on the periodic N^3 grid of [0,1)^3
    (Sec. 4.1, Tab. 6).  Applies the stencil to the 3D array."""
    r = order // 2
    c = [float(x) for x in second_derivative_weights(r)]
    h = 1.0 / N
    x = np.arange(N) * h
    s = np.sin(2 * np.pi * m * x)
    u = s[:, None, None] * s[None, :, None] * s[None, None, :]
    lap = 3 * c[0] * u
    for ax in range(3):
        for l in range(1, r + 1):
            lap += c[l] * (np.roll(u, l, axis=ax) + np.roll(u, -l, axis=ax))
    lap /= h * h
    exact = -3 * (2 * np.pi * m) ** 2 * u
    err = lap - exact
    rel_l2 = np.sqrt(np.sum(err ** 2) / np.sum(exact ** 2))
    rel_inf = np.max(np.abs(err)) / np.max(np.abs(exact))
    return rel_l2, rel_inf


def symbol(theta, weights=None):
    """D-hat(theta) = 2 sum_l a_l sin(l theta): the Fourier symbol (times h) of
    the centred first derivative acting on sin(theta i) -> D-hat cos(theta i)."""
    w = WEIGHTS if weights is None else weights
    return 2.0 * sum(w[l] * np.sin((l + 1) * theta) for l in range(len(w)))


def staggered_symbol(theta, weights=None):
    """S-hat(theta) = 2 sum_l c_l sin((l - 1/2) theta): the staggered first
    derivative maps sin(theta i) at the nodes to (S-hat/h) cos(theta (i + 1/2))
    at the half nodes, and cos at the half nodes back to -(S-hat/h) sin."""
    w = STAGGERED_WEIGHTS if weights is None else weights
    return 2.0 * sum(w[l] * np.sin((l + 0.5) * theta) for l in range(len(w)))


def stability_limit(weights=None, staggered=False):
    """Largest c dt / h for which the 3D leapfrog is stable:
    (c dt / 2h) sqrt(3) max D-hat <= 1 (collocated), S-hat in the staggered form."""
    th = np.linspace(0.0, np.pi, 400001)
    sym = staggered_symbol(th, weights) if staggered else symbol(th, weights)
    return 2.0 / (math.sqrt(3.0) * float(np.max(sym)))


def standing_wave_state(shape, m, h, dt, rho, weights=None, staggered=False):
    """Initial (p^0, v^{-1/2}) on a periodic grid for which the leapfrog gives
    p^n = phi cos(omega_h n dt) exactly, phi = prod_d sin(theta_d i_d),
    theta_d = 2 pi m_d / n_d, with v^{-1/2} = (dt / (2 rho)) D phi written in
    closed form through the symbol (D sin = (D-hat/h) cos).  staggered: v_d
    sits at i_d + 1/2, so its cosine is taken there and S-hat replaces D-hat."""
    nz, ny, nx = shape
    mz, my, mx = m
    th = [2 * np.pi * mx / nx, 2 * np.pi * my / ny, 2 * np.pi * mz / nz]
    ix, iy, iz = np.arange(nx), np.arange(ny), np.arange(nz)
    sx, sy, sz = np.sin(th[0] * ix), np.sin(th[1] * iy), np.sin(th[2] * iz)
    half = 0.5 if staggered else 0.0
    cx, cy, cz = np.cos(th[0] * (ix + half)), np.cos(th[1] * (iy + half)), np.cos(th[2] * (iz + half))
    phi = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    sym = staggered_symbol if staggered else symbol
    Dh = [sym(t, weights) / h for t in th]
    st = State(shape)
    st["p"] = phi
    st["vx"] = dt / (2 * rho) * Dh[0] * sz[:, None, None] * sy[None, :, None] * cx[None, None, :]
    st["vy"] = dt / (2 * rho) * Dh[1] * sz[:, None, None] * cy[None, :, None] * sx[None, None, :]
    st["vz"] = dt / (2 * rho) * Dh[2] * cz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    lam2 = sum(d * d for d in Dh)
    return st, phi, lam2


def staggered_energy(grid: Grid, p_n, p_np1, v_half):
    """E^{n+1/2} = 1/2 sum_d kr_d rho |v_d^{n+1/2}|^2 + 1/2 sum p^n p^{n+1} / K,
    the discrete energy conserved by the leapfrog when D is skew-adjoint
    (kr: the grid's anisotropy factors, 1 when isotropic)."""
    rho = grid.rho if grid.rho_n is None else grid.rho_n
    ek = 0.5 * sum(kr * float(np.sum(rho * v * v)) for kr, v in zip(grid.kr, v_half))
    ep = 0.5 * float(np.sum(p_n * p_np1 / grid.K))
    return ek + ep
