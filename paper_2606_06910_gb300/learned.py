"""Learned CPML: a 4 -> 64 -> 64 -> 3 network that emits the grading of a thin
layer (sigma, kappa, alpha per layer cell), trained through the library's
discrete adjoint on reflected energy.

Downstream of (sigma, kappa, alpha) everything is the CPML of paper Sec. 3.2
(b = exp(-(sigma/kappa + alpha) dt), a = sigma (b - 1) / (kappa (sigma + kappa
alpha)), 1/kappa); the polynomial (Roden-Gedney) grading of Sec. 3.2 / Tab. 2
is the fallback and the starting point.  All arithmetic runs in the library:
the polynomial grading (fdtd_cpml_grading), network forward/backward, the
pre-fit loss gradient and Adam (fdtd_mlp_*, fdtd_adam_step), coefficient map
and its chain rule (fdtd_set_cpml_ska, fdtd_cpml_ska_backward), forward and
adjoint wave propagation, and the misfits (fdtd_misfit, fdtd_misfit_noalloc).
This module builds the input features and marshals tensors.

Features of layer cell j (j = 0 outermost of L cells), for a layer graded
against the reference velocity c at time step dt and dominant frequency f0:
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
from .synth import angled_sources, face_receivers, frequency_groups, mlp_init_params, ricker

NPARAM = 4 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3
ACT = 2 * 64 + 3


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def features(L: int, L_ref: int, f0: float, h: float, c: float, dt: float) -> np.ndarray:
    """Network inputs of the L cells (see the module docstring)."""
    j = np.arange(L)
    return np.stack([(L - j) / L, np.full(L, L / L_ref), np.full(L, f0 * h / c), np.full(L, c * dt / h)],
                    axis=1)


def polynomial_ska(L: int, h: float, c_ref: float, R: float = 1e-8, q: int = 3, kappa_max: float = 5.0,
                   alpha_frac: float = 0.05) -> np.ndarray:
    """Per-cell (sigma, kappa, alpha) [L, 3] of the polynomial grading of
    Sec. 3.2 / Tab. 2, from the library (fdtd_cpml_grading)."""
    lib = _lib.load()
    out = (ctypes.c_double * (3 * L))()
    st = lib.fdtd_cpml_grading(int(L), float(h), float(c_ref), float(R), float(kappa_max), float(alpha_frac),
                               int(q), out)
    if st != _lib.OK:
        raise FdtdError(st, "fdtd_cpml_grading")
    return np.frombuffer(out, dtype=np.float64).reshape(L, 3).copy()


def misfit_flat(a: torch.Tensor, b: torch.Tensor) -> float:
    """1/2 sum (a - b)^2 in FP64 on the device (fdtd_misfit_noalloc)."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    st = lib.fdtd_misfit_noalloc(_p(a), _p(b), ctypes.c_longlong(a.numel()), None, ctypes.byref(out),
                                 ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream))
    if st != _lib.OK:
        raise FdtdError(st, "fdtd_misfit_noalloc")
    return out.value


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
        self.net = Network(mlp_init_params(seed) if theta is None else theta, self.device)
        self.set_conditions(c, dt, f0)

    def set_conditions(self, c: float, dt: float, f0: float):
        """Reference velocity, time step and dominant frequency the layer is
        graded for (the network's inputs and output scales)."""
        self.c, self.dt = float(c), float(dt)
        self.sigma_scale = self.c / self.h
        self.set_frequency(f0)

    def set_frequency(self, f0: float):
        self.f0 = float(f0)
        self.alpha_scale = math.pi * self.f0
        self.X = torch.tensor(features(self.L, self.L_ref, self.f0, self.h, self.c, self.dt).astype(np.float32),
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
        gout = torch.empty_like(tgt)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        lib, s = self.net.lib, self.net._s()
        for _ in range(iters):
            out, act = self.ska()
            st = lib.fdtd_mlp_fit_gradient(_p(out), _p(tgt), self.L, float(self.sigma_scale), float(self.alpha_scale),
                                           _p(gout), _p(loss), s)
            if st != _lib.OK:
                raise FdtdError(st, "fdtd_mlp_fit_gradient")
            g = self.net.backward(self.X, act, gout, self.sigma_scale, self.alpha_scale)
            self.net.adam(g, lr)
        out, _ = self.ska()
        st = lib.fdtd_mlp_fit_gradient(_p(out), _p(tgt), self.L, float(self.sigma_scale), float(self.alpha_scale),
                                       _p(gout), _p(loss), s)
        if st != _lib.OK:
            raise FdtdError(st, "fdtd_mlp_fit_gradient")
        return float(loss.item())

    def gradient(self, sim, ref_traces: torch.Tensor, nt: int, weight: float = 1.0):
        """J (reflected energy at the receivers: weight * 1/2 sum (traces -
        ref)^2 over the first nt steps) and dJ/dtheta for the current
        parameters, through one forward and one adjoint run of `sim` (whose
        source and receivers are set)."""
        out, act = self.ska()
        sim.reset()
        sim.set_cpml_ska(out)
        sim.step(nt)
        resid = torch.empty_like(ref_traces)
        J = weight * sim.misfit(ref_traces, nt=nt, resid=resid)
        if weight != 1.0:
            resid.mul_(weight)
        gprof = torch.zeros((3, 3, max(sim.shape)), dtype=torch.float32, device=self.device)
        sim.adjoint(nt, resid, None, gprof)
        gska = sim.ska_backward(out, gprof)
        g = self.net.backward(self.X, act, gska, self.sigma_scale, self.alpha_scale)
        sim.reset()
        return J, g, out

    def train_step(self, sim, ref_traces, nt, lr=2e-3, weight=1.0):
        J, g, out = self.gradient(sim, ref_traces, nt, weight)
        self.net.adam(g, lr)
        return J


def reflection_task(n=96, L=6, nshots=8, seed=3, freqs=(5.0, 30.0), nfreq=4, angles=(0.0, 80.0), c=2000.0,
                    h=10.0, margin=48, ref_cells=20, nt=None, device="cuda"):
    """Training and evaluation data of the learned layer, generated by the
    solver itself on an n^3 homogeneous grid:
      - nfreq frequency groups, f0 drawn (seeded, one per equal sub-range)
        from `freqs`; each group has its own Ricker wavelet and window
        nt = (2.4 / f0 + 0.3 s) / dt unless given;
      - per group, training and held-out shots whose sources meet a seeded
        face at seeded incidence angles in `angles` (synth.angled_sources);
      - receivers on the six planes 2 nodes inside the layer
        (synth.face_receivers, 5 x 5 per face);
      - reference traces from the same interior embedded in a grid `margin`
        nodes larger per side (its own ref_cells-cell polynomial layer far
        away), where nothing returns to the receivers within the window.
    The misfit against the reference is the energy the thin layer reflects."""
    from .fdtd import Fdtd
    dt = 0.5 * h / c
    f0s = frequency_groups(freqs, nfreq, seed)
    rec = face_receivers(n, L, 5)
    groups = []
    for k, f0 in enumerate(f0s):
        ntk = int(nt) if nt else int(math.ceil((2.4 / f0 + 0.3) / dt))
        src, th = {}, {}
        for j, which in enumerate(("train", "eval")):
            src[which], th[which], _ = angled_sources(n, L, nshots, seed * 1000 + 2 * k + j, angles)
        wav = np.tile(ricker(ntk, dt, f0)[None, :], (nshots, 1)).astype(np.float32)
        groups.append(dict(f0=f0, nt=ntk, src=src, angles=th, wav=wav))
    nt_max = max(g["nt"] for g in groups)
    nb = n + 2 * margin
    big = Fdtd((nb,) * 3, h, dt, nshots=nshots, cpml_cells=ref_cells, nt_max=nt_max, nrec_max=len(rec), device=device)
    big.set_model(torch.full((nb,) * 3, c, device=device))
    big.set_cpml(R=1e-8, c_ref=c)
    big.record(rec + margin)
    zeros = None
    for g in groups:
        g["ref"], g["ref_energy"] = {}, {}
        for which in ("train", "eval"):
            big.reset()
            big.inject(g["src"][which] + margin, torch.from_numpy(g["wav"]).to(device))
            big.step(g["nt"])
            big.sync()
            ref = torch.zeros_like(big.traces)
            ref[:, :g["nt"]] = big.traces[:, :g["nt"]]
            if zeros is None:
                zeros = torch.zeros_like(ref)
            g["ref"][which] = ref
            g["ref_energy"][which] = misfit_flat(ref, zeros)
    big.close()
    return dict(n=n, L=L, nshots=nshots, c=c, h=h, dt=dt, rec=rec, groups=groups, nt_max=nt_max, device=device,
                freqs=tuple(freqs), angles=tuple(angles))


def _reflection(sim, task, g, which):
    """||traces - ref|| / ||ref|| of one group's shots (library misfits)."""
    sim.reset()
    sim.inject(g["src"][which], torch.from_numpy(g["wav"]).to(task["device"]))
    sim.step(g["nt"])
    J = sim.misfit(g["ref"][which], nt=g["nt"])
    return math.sqrt(J / g["ref_energy"][which])


def train_learned_cpml(task, iters=48, lr=5e-3, seed=0, checkpoint_every=25, fit_iters=400):
    """Fit the network to the polynomial grading of the same thickness (the
    fallback), then train it through the adjoint on the reflection task,
    cycling through the frequency groups (the network's frequency input
    changes from step to step); each group's misfit is weighted by the
    inverse of its reference energy, so every group counts as its squared
    reflection ratio.  Returns per group the reflection ratios ||traces -
    ref|| / ||ref|| on held-out shots for the polynomial and the learned
    layer, the training misfits and the model."""
    from .fdtd import Fdtd
    n, L, dev = task["n"], task["L"], task["device"]
    shape = (n,) * 3
    sim = Fdtd(shape, task["h"], task["dt"], nshots=task["nshots"], cpml_cells=L, nt_max=task["nt_max"],
               nrec_max=len(task["rec"]), checkpoint_every=checkpoint_every, cpml_grad=True, device=dev)
    sim.set_model(torch.full(shape, task["c"], device=dev))
    sim.record(task["rec"])
    # polynomial grading of the same thickness (paper Tab. 2 parameters)
    sim.set_cpml(R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3, c_ref=task["c"])
    groups = task["groups"]
    poly = [_reflection(sim, task, g, "eval") for g in groups]
    model = LearnedCPML(L, task["h"], task["dt"], task["c"], groups[0]["f0"], seed=seed, device=dev)
    fit_err = model.fit_profile(polynomial_ska(L, task["h"], task["c"]), iters=fit_iters)
    Js = []
    for it in range(iters):
        g = groups[it % len(groups)]
        model.set_frequency(g["f0"])
        sim.inject(g["src"]["train"], torch.from_numpy(g["wav"]).to(dev))
        Js.append(model.train_step(sim, g["ref"]["train"], g["nt"], lr=lr, weight=1.0 / g["ref_energy"]["train"]))
    learned = []
    for g in groups:
        model.set_frequency(g["f0"])
        ska, _ = model.ska()
        sim.set_cpml_ska(ska)
        learned.append(_reflection(sim, task, g, "eval"))
    sim.close()
    ng = len(groups)
    return dict(f0=[g["f0"] for g in groups], poly_eval=poly, learned_eval=learned,
                J_first=float(np.mean(Js[:ng])), J_last=float(np.mean(Js[-ng:])), J=Js, fit_err=fit_err,
                model=model)


__all__ = ["LearnedCPML", "Network", "features", "polynomial_ska", "NPARAM", "reflection_task", "train_learned_cpml",
           "misfit_flat"]
