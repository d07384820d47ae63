"""Learned CPML: a 4 -> 64 -> 64 -> 3 network that emits the grading of a thin
layer (sigma, kappa, alpha per layer cell), trained through the library's
discrete adjoint on reflected energy.

Downstream of (sigma, kappa, alpha) everything is the CPML of paper Sec. 3.2
(b = exp(-(sigma/kappa + alpha) dt), a = sigma (b - 1) / (kappa (sigma + kappa
alpha)), 1/kappa); the polynomial (Roden-Gedney) grading of Sec. 3.2 / Tab. 2
is the fallback and the starting point.  All arithmetic runs in the library's
kernels: network forward/backward and Adam (fdtd_mlp_*, fdtd_adam_step),
coefficient map and its chain rule (fdtd_set_cpml_ska, fdtd_cpml_ska_backward),
forward and adjoint wave propagation.  This module only marshals tensors.

Features of layer cell j (j = 0 outermost of L cells):
    [rho_j = (L - j)/L, L / L_ref, f0 h / c, c dt / h]
Outputs: sigma = sigma_scale softplus(o0), kappa = 1 + softplus(o1),
alpha = alpha_scale softplus(o2), sigma_scale = c / h, alpha_scale = pi f0.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import FdtdError

NPARAM = 4 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3
ACT = 2 * 64 + 3


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def init_params(seed: int, scale1=0.5, scale2=0.2, scale3=0.1) -> np.ndarray:
    """Seeded initial weights (normal, fixed scales), zero biases; float64."""
    rng = np.random.default_rng(seed)
    W1 = scale1 * rng.standard_normal((64, 4))
    W2 = scale2 * rng.standard_normal((64, 64))
    W3 = scale3 * rng.standard_normal((3, 64))
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(3)])


def features(L: int, L_ref: int, f0: float, h: float, c: float, dt: float) -> np.ndarray:
    j = np.arange(L)
    return np.stack([(L - j) / L, np.full(L, L / L_ref), np.full(L, f0 * h / c), np.full(L, c * dt / h)],
                    axis=1)


def roden_gedney_ska(L: int, h: float, c_ref: float, R: float = 1e-8, q: int = 3, kappa_max: float = 5.0,
                     alpha_frac: float = 0.05) -> np.ndarray:
    """Per-cell (sigma, kappa, alpha) of the polynomial grading of Sec. 3.2
    (sigma_max = -(q+1) c_ref ln R / (2 L h)), cell j at depth rho = (L-j)/L."""
    j = np.arange(L)
    rho = (L - j) / L
    smax = -(q + 1) * c_ref * math.log(R) / (2.0 * L * h)
    return np.stack([smax * rho ** q, 1.0 + (kappa_max - 1.0) * rho ** q, alpha_frac * smax * (1.0 - rho)],
                    axis=1)


class Network:
    """Parameters and Adam state on the device, with the library's kernels."""

    def __init__(self, theta: np.ndarray, device, stream=None):
        self.lib = _lib.load()
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.theta = torch.tensor(np.asarray(theta, np.float32), device=self.device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.t = 0

    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def forward(self, X: torch.Tensor, sigma_scale: float, alpha_scale: float):
        n = X.shape[0]
        out = torch.empty((n, 3), dtype=torch.float32, device=self.device)
        act = torch.empty((n, ACT), dtype=torch.float32, device=self.device)
        st = self.lib.fdtd_mlp_forward(_p(self.theta), _p(X), n, float(sigma_scale), float(alpha_scale),
                                       _p(out), _p(act), self._s())
        if st != _lib.OK:
            raise FdtdError(st, "fdtd_mlp_forward")
        return out, act

    def backward(self, X, act, gout, sigma_scale: float, alpha_scale: float):
        g = torch.empty_like(self.theta)
        st = self.lib.fdtd_mlp_backward(_p(self.theta), _p(X), X.shape[0], _p(act), _p(gout.contiguous()),
                                        float(sigma_scale), float(alpha_scale), _p(g), self._s())
        if st != _lib.OK:
            raise FdtdError(st, "fdtd_mlp_backward")
        return g

    def adam(self, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        st = self.lib.fdtd_adam_step(_p(self.theta), _p(grad), _p(self.m), _p(self.v), NPARAM, self.t,
                                     float(lr), float(beta1), float(beta2), float(eps), self._s())
        if st != _lib.OK:
            raise FdtdError(st, "fdtd_adam_step")


class LearnedCPML:
    """A learned grading for a layer of L cells on every face of `sim` (an
    Fdtd created with cpml_cells = L, checkpoint_every > 0 and cpml_grad)."""

    def __init__(self, L: int, h: float, dt: float, c: float, f0: float, L_ref: int = 20, seed: int = 0,
                 device="cuda", theta: np.ndarray | None = None):
        self.L, self.h, self.dt, self.c, self.f0, self.L_ref = L, h, dt, c, f0, L_ref
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.net = Network(init_params(seed) if theta is None else theta, self.device)
        self.sigma_scale = c / h
        self.alpha_scale = math.pi * f0
        self.set_frequency(f0)

    def set_frequency(self, f0: float):
        self.f0 = f0
        self.alpha_scale = math.pi * f0
        self.X = torch.tensor(features(self.L, self.L_ref, f0, self.h, self.c, self.dt).astype(np.float32),
                              device=self.device)

    def ska(self):
        out, act = self.net.forward(self.X, self.sigma_scale, self.alpha_scale)
        return out, act

    def fit_profile(self, target_ska: np.ndarray, iters=400, lr=3e-3):
        """Fit the network to a given grading (e.g. the polynomial one) by
        minimising sum over cells of ((sigma - s*)/sigma_scale)^2 +
        (kappa - k*)^2 + ((alpha - a*)/alpha_scale)^2 with the library's
        backward and Adam kernels."""
        tgt = torch.tensor(np.asarray(target_ska, np.float32), device=self.device)
        w = torch.tensor([1.0 / self.sigma_scale ** 2, 1.0, 1.0 / self.alpha_scale ** 2], device=self.device)
        for _ in range(iters):
            out, act = self.ska()
            gout = 2.0 * (out - tgt) * w
            g = self.net.backward(self.X, act, gout, self.sigma_scale, self.alpha_scale)
            self.net.adam(g, lr)
        out, _ = self.ska()
        return float((((out - tgt) ** 2) * w).sum())

    def gradient(self, sim, ref_traces: torch.Tensor, nt: int):
        """J (reflected energy at the receivers: 1/2 sum (traces - ref)^2) and
        dJ/dtheta for the current parameters, through one forward and one
        adjoint run of `sim` (whose source and receivers are set)."""
        out, act = self.ska()
        sim.reset()
        sim.set_cpml_ska(out)
        sim.step(nt)
        resid = torch.empty_like(ref_traces)
        J = sim.misfit(ref_traces, nt=nt, resid=resid)
        gprof = torch.zeros((3, 3, max(sim.shape)), dtype=torch.float32, device=self.device)
        sim.adjoint(nt, resid, None, gprof)
        gska = sim.ska_backward(out, gprof)
        g = self.net.backward(self.X, act, gska, self.sigma_scale, self.alpha_scale)
        sim.reset()
        return J, g, out

    def train_step(self, sim, ref_traces, nt, lr=2e-3):
        J, g, out = self.gradient(sim, ref_traces, nt)
        self.net.adam(g, lr)
        return J


def _face_receivers(n: int, L: int, k: int, inset: int = 2) -> np.ndarray:
    """k x k receivers on each of the six planes `inset` nodes inside the
    layer (one plane per face), over the interior extent of that plane."""
    lo, hi = L + inset, n - 1 - L - inset
    span = np.round(np.linspace(L + inset, n - 1 - L - inset, k)).astype(np.int32)
    a, b = np.meshgrid(span, span, indexing="ij")
    a, b = a.ravel(), b.ravel()
    out = []
    for plane in (lo, hi):
        out.append(np.stack([np.full_like(a, plane), a, b], 1))   # z faces
        out.append(np.stack([a, np.full_like(a, plane), b], 1))   # y faces
        out.append(np.stack([a, b, np.full_like(a, plane)], 1))   # x faces
    return np.concatenate(out).astype(np.int32)


def reflection_task(n=96, L=6, nshots=8, seed=0, nt=220, f0=15.0, c=2000.0, h=10.0, margin=40,
                    ref_cells=20, device="cuda"):
    """Training and evaluation data of the learned layer, generated by the
    solver itself: point sources at seeded interior positions (so that the
    waves meet the faces at angles from normal to grazing), receivers on
    planes just inside the layer on all six faces, and reference traces from
    the same interior embedded in a grid `margin` nodes larger per side (its
    own 20-cell polynomial layer far away), where nothing returns to the
    receivers within the window.  The misfit against the reference is the
    energy reflected by the thin layer."""
    from .fdtd import Fdtd
    from .synth import ricker
    dt = 0.5 * h / c
    rng = np.random.default_rng(seed)
    lo, hi = L + 6, n - L - 6
    src = {k: rng.integers(lo, hi, size=(nshots, 3)).astype(np.int32) for k in ("train", "eval")}
    rec = _face_receivers(n, L, 5)
    wav = np.tile(ricker(nt, dt, f0)[None, :], (nshots, 1)).astype(np.float32)
    nb = n + 2 * margin
    big = Fdtd((nb,) * 3, h, dt, nshots=nshots, cpml_cells=ref_cells, nt_max=nt, nrec_max=len(rec), device=device)
    big.set_model(torch.full((nb,) * 3, c, device=device))
    big.set_cpml(R=1e-8, c_ref=c)
    big.record(rec + margin)
    refs = {}
    for k in ("train", "eval"):
        big.reset()
        big.inject(src[k] + margin, torch.from_numpy(wav).to(device))
        big.step(nt)
        refs[k] = big.traces.clone()
    big.close()
    return dict(n=n, L=L, nshots=nshots, nt=nt, f0=f0, c=c, h=h, dt=dt, src=src, rec=rec, wav=wav, ref=refs,
                device=device)


def _reflection(sim, task, which):
    sim.reset()
    sim.inject(task["src"][which], torch.from_numpy(task["wav"]).to(task["device"]))
    sim.step(task["nt"])
    ref = task["ref"][which]
    num = float(((sim.traces - ref) ** 2).sum())
    den = float((ref ** 2).sum())
    return math.sqrt(num / den)


def train_learned_cpml(task, iters=60, lr=5e-3, seed=0, checkpoint_every=25, fit_iters=400):
    """Fit the network to the polynomial grading of the same thickness (the
    fallback), then train it through the adjoint on the reflection task.
    Returns reflection ratios ||traces - ref|| / ||ref|| on held-out shots for
    the polynomial and the learned layer, the training misfits, and the
    learned (sigma, kappa, alpha)."""
    from .fdtd import Fdtd
    n, L, nt, dev = task["n"], task["L"], task["nt"], task["device"]
    shape = (n,) * 3
    sim = Fdtd(shape, task["h"], task["dt"], nshots=task["nshots"], cpml_cells=L, nt_max=nt,
               nrec_max=len(task["rec"]), checkpoint_every=checkpoint_every, cpml_grad=True, device=dev)
    sim.set_model(torch.full(shape, task["c"], device=dev))
    sim.record(task["rec"])
    # polynomial grading of the same thickness (paper Tab. 2 parameters)
    sim.set_cpml(R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3, c_ref=task["c"])
    poly_eval = _reflection(sim, task, "eval")
    model = LearnedCPML(L, task["h"], task["dt"], task["c"], task["f0"], seed=seed, device=dev)
    fit_err = model.fit_profile(roden_gedney_ska(L, task["h"], task["c"]), iters=fit_iters)
    sim.reset()
    sim.inject(task["src"]["train"], torch.from_numpy(task["wav"]).to(dev))
    Js = []
    for _ in range(iters):
        Js.append(model.train_step(sim, task["ref"]["train"], nt, lr=lr))
    ska, _ = model.ska()
    sim.set_cpml_ska(ska)
    learned_eval = _reflection(sim, task, "eval")
    sim.close()
    return dict(poly_eval=poly_eval, learned_eval=learned_eval, J_first=Js[0], J_last=Js[-1], J=Js,
                fit_err=fit_err, ska=ska.cpu().numpy(), model=model)


__all__ = ["LearnedCPML", "Network", "features", "roden_gedney_ska", "init_params", "NPARAM", "reflection_task",
           "train_learned_cpml"]
