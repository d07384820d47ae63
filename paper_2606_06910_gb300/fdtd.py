"""Python binding of libfdtd (include/fdtd.h): the ``Fdtd`` simulator and the
``FdtdFn`` autograd function.

Everything here is argument marshalling around the C ABI: PyTorch supplies the
device memory (one workspace tensor per simulator, plus the caller's inputs
and outputs) and the stream; every step of the method runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import FIELD_ID, STORAGE, Desc, FdtdError


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, shape, device, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32 or not t.is_contiguous() or t.device != device:
        raise ValueError(f"{name} must be a contiguous float32 tensor on {device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _cells6(cpml_cells):
    if isinstance(cpml_cells, int):
        return (cpml_cells,) * 6
    cells = tuple(int(c) for c in cpml_cells)
    if len(cells) != 6:
        raise ValueError("cpml_cells must be an int or 6 values (-x,+x,-y,+y,-z,+z)")
    return cells


class Fdtd:
    """One context of the library: a grid of nshots wavefields sharing a model.

    shape = (nz, ny, nx); the CPML cells (int or per face -x,+x,-y,+y,-z,+z)
    lie inside the grid.  ``storage`` is "f32", "f16" or "bf16".
    """

    def __init__(self, shape, h, dt, *, nshots=1, cpml_cells=0, storage="f32", nt_max=1,
                 nrec_max=0, checkpoint_every=0, cpml_grad=False, tblock_k=1, cpml_local=False, device=None,
                 stream=None):
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        if self.device.type != "cuda":
            raise ValueError("Fdtd runs on a CUDA device only")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.nshots = int(nshots)
        self.nt_max = int(nt_max)
        self.storage = storage
        self.h, self.dt = float(h), float(dt)
        self.cells = _cells6(cpml_cells)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        d = Desc()
        d.nx, d.ny, d.nz, d.nshots = nx, ny, nz, self.nshots
        d.h, d.dt = self.h, self.dt
        for i, c in enumerate(self.cells):
            d.cpml_cells[i] = c
        d.storage = STORAGE[storage]
        d.tblock_k = int(tblock_k)
        self.tblock_k = int(tblock_k)
        d.nt_max = self.nt_max
        d.nrec_max = int(nrec_max)
        d.checkpoint_every = int(checkpoint_every)
        d.cpml_grad = 1 if cpml_grad else 0
        d.cpml_local = 1 if cpml_local else 0
        d.stream = ctypes.c_void_p(stream.cuda_stream)
        self._desc = d
        nbytes = ctypes.c_size_t(0)
        self._check(self.lib.fdtd_workspace_bytes(ctypes.byref(d), ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.fdtd_create(ctypes.byref(d), ctypes.c_void_p(self._ws_ptr),
                                      ctypes.c_size_t(self.workspace_bytes), ctypes.byref(ctx))
        self._check(st)
        self.ctx = ctx
        self.traces = None
        self.nrec = 0

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fdtd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        if status != _lib.OK:
            msg = ""
            if getattr(self, "ctx", None):
                msg = (self.lib.fdtd_last_error(self.ctx) or b"").decode()
            raise FdtdError(status, msg)

    # -- set-up --------------------------------------------------------------
    def set_model(self, vel: torch.Tensor, rho: torch.Tensor | None = None):
        """Velocity [m/s] and, optionally, density per node (both [nz, ny, nx])."""
        _need(vel, self.shape, self.device, "vel")
        if rho is not None:
            _need(rho, self.shape, self.device, "rho")
        self._check(self.lib.fdtd_set_model(self.ctx, _ptr(vel), _ptr(rho)))

    def set_cpml(self, R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3, c_ref=None):
        self._check(self.lib.fdtd_set_cpml(self.ctx, float(R), float(kappa_max), float(alpha_frac),
                                           int(q), float(c_ref) if c_ref is not None else -1.0))

    def set_anisotropy(self, kr):
        """Elliptic anisotropy: axis moduli kr_d K for (x, y, z); the wave
        speed along axis d is c sqrt(kr_d)."""
        arr = (ctypes.c_double * 3)(*[float(v) for v in kr])
        self._check(self.lib.fdtd_set_anisotropy(self.ctx, ctypes.cast(arr, ctypes.c_void_p)))

    def set_cpml_local(self, vel: torch.Tensor, R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3):
        """Local-velocity grading: sigma_max from the velocity at each slab
        node (needs cpml_local=True at construction and set_model first)."""
        _need(vel, self.shape, self.device, "vel")
        self._check(self.lib.fdtd_set_cpml_local(self.ctx, _ptr(vel), float(R), float(kappa_max),
                                                 float(alpha_frac), int(q)))

    def set_staggered(self, on: bool = True):
        """Staggered (Yee) form: v_d at the half nodes i + 1/2, staggered
        radius-4 derivatives; FP32 storage and constant density.  adjoint()
        transposes it (grad_cpml is not provided for it)."""
        self._check(self.lib.fdtd_set_staggered(self.ctx, 1 if on else 0))

    def set_cpml_ska(self, ska: torch.Tensor):
        _need(ska, (self.cells[0], 3), self.device, "ska")
        self._check(self.lib.fdtd_set_cpml_ska(self.ctx, _ptr(ska)))

    def inject(self, src_zyx, wavelet: torch.Tensor):
        src = np.ascontiguousarray(np.asarray(src_zyx, dtype=np.int32).reshape(self.nshots, 3))
        _need(wavelet, None, self.device, "wavelet")
        if wavelet.dim() != 2 or wavelet.shape[0] != self.nshots:
            raise ValueError("wavelet must be [nshots, nt]")
        self._wavelet = wavelet
        self._check(self.lib.fdtd_inject(self.ctx, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         _ptr(wavelet), int(wavelet.shape[1])))

    def record(self, rec_zyx):
        rec = np.ascontiguousarray(np.asarray(rec_zyx, dtype=np.int32).reshape(-1, 3))
        nrec = rec.shape[0]
        self.traces = torch.zeros((self.nshots, self.nt_max, max(nrec, 1)), dtype=torch.float32,
                                  device=self.device)[:, :, :nrec].contiguous()
        self._check(self.lib.fdtd_record(self.ctx, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nrec,
                                         _ptr(self.traces)))
        self.nrec = nrec
        return self.traces

    # -- stepping ----------------------------------------------------------
    def step(self, n=1):
        self._check(self.lib.fdtd_step_n(self.ctx, int(n)))

    def adjoint(self, n, resid=None, grad_vel=None, grad_cpml=None):
        """The discrete adjoint of the last n (= current time) steps from the
        checkpoints: resid [nshots, nt_max, nrec] is injected at the
        receivers; grad_vel [nz, ny, nx] receives += dJ/dc summed over shots;
        grad_cpml [3, 3, max(shape)] receives += dJ/d(b, a, 1/kappa) (needs
        cpml_grad=True; collocated form with the 1D grading only)."""
        if resid is not None:
            _need(resid, (self.nshots, self.nt_max, self.nrec), self.device, "resid")
        if grad_vel is not None:
            _need(grad_vel, self.shape, self.device, "grad_vel")
        if grad_cpml is not None:
            _need(grad_cpml, (3, 3, max(self.shape)), self.device, "grad_cpml")
        self._check(self.lib.fdtd_adjoint_step_n(self.ctx, int(n), _ptr(resid), _ptr(grad_vel),
                                                 _ptr(grad_cpml)))

    def reset(self):
        self._check(self.lib.fdtd_reset(self.ctx))

    @property
    def time(self) -> int:
        t = ctypes.c_int(0)
        self._check(self.lib.fdtd_time(self.ctx, ctypes.byref(t)))
        return t.value

    def sync(self):
        self._check(self.lib.fdtd_sync(self.ctx))

    def set_divergence_check(self, every: int, limit: float = 0.0):
        """Every `every` steps, flag a non-finite sum of p^2 (or one above
        `limit` if > 0); sync() then raises EDIVERGED.  0 turns it off."""
        self._check(self.lib.fdtd_set_divergence_check(self.ctx, int(every), float(limit)))

    def set_time(self, t: int):
        """Time index to continue from (resume after set() of every field)."""
        self._check(self.lib.fdtd_set_time(self.ctx, int(t)))

    def set_velocity_scale(self, scale: float):
        """Stored velocity = scale * v with 16-bit storage (0: the model's
        maximum velocity); takes effect at the next set_model."""
        self._check(self.lib.fdtd_set_velocity_scale(self.ctx, float(scale)))

    # -- kernel timing (CUDA events around each launch, in the library) -------
    def set_timing(self, on: bool = True):
        self._check(self.lib.fdtd_set_timing(self.ctx, 1 if on else 0))

    def timing(self, kernel: str = "step"):
        """(milliseconds, launches) of the step or adjoint kernels since
        set_timing(True)."""
        ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
        k = {"step": _lib.TIMING_STEP, "adjoint": _lib.TIMING_ADJOINT}[kernel]
        self._check(self.lib.fdtd_timing(self.ctx, k, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # -- fields ------------------------------------------------------------
    def get(self, which: str, shot=0, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        _need(out, self.shape, self.device, "out")
        self._check(self.lib.fdtd_get_field(self.ctx, FIELD_ID[which], int(shot), _ptr(out)))
        return out

    def set(self, which: str, value: torch.Tensor, shot=0):
        _need(value, self.shape, self.device, "value")
        self._check(self.lib.fdtd_set_field(self.ctx, FIELD_ID[which], int(shot), _ptr(value)))

    # -- reductions (FP64 on the device) --------------------------------------
    def energy(self, shot=0, box=None) -> float:
        nz, ny, nx = self.shape
        b = (0, nz, 0, ny, 0, nx) if box is None else tuple(int(v) for v in box)
        arr = (ctypes.c_int * 6)(*b)
        out = ctypes.c_double(0.0)
        self._check(self.lib.fdtd_energy(self.ctx, int(shot), arr, ctypes.byref(out)))
        return out.value

    def misfit(self, dobs: torch.Tensor, nt=None, resid: torch.Tensor | None = None) -> float:
        _need(dobs, (self.nshots, self.nt_max, self.nrec), self.device, "dobs")
        if resid is not None:
            _need(resid, (self.nshots, self.nt_max, self.nrec), self.device, "resid")
        out = ctypes.c_double(0.0)
        self._check(self.lib.fdtd_misfit(self.ctx, _ptr(dobs), int(self.nt_max if nt is None else nt),
                                         _ptr(resid), ctypes.byref(out)))
        return out.value

    def ska_backward(self, ska: torch.Tensor, grad_cpml: torch.Tensor) -> torch.Tensor:
        gska = torch.empty_like(ska)
        self._check(self.lib.fdtd_cpml_ska_backward(self.ctx, _ptr(ska), _ptr(grad_cpml), _ptr(gska)))
        return gska


class FdtdFn(torch.autograd.Function):
    """traces = F(vel): a full forward run of ``sim`` (from a zero state) with
    the velocity model ``vel``; backward runs the library's discrete adjoint
    (checkpoint + recompute) and returns dJ/dvel.  The CPML coefficients must
    be set with an explicit c_ref so that they do not depend on vel."""

    @staticmethod
    def forward(ctx, vel, sim: Fdtd, nt: int):
        sim.reset()
        sim.set_model(vel.detach().contiguous())
        sim.step(nt)
        ctx.sim, ctx.nt = sim, nt
        ctx.shape = vel.shape
        return sim.traces[:, :nt].clone()

    @staticmethod
    def backward(ctx, grad_traces):
        sim = ctx.sim
        resid = torch.zeros((sim.nshots, sim.nt_max, sim.nrec), dtype=torch.float32, device=sim.device)
        resid[:, :ctx.nt] = grad_traces
        grad_vel = torch.zeros(ctx.shape, dtype=torch.float32, device=sim.device)
        sim.adjoint(ctx.nt, resid.contiguous(), grad_vel)
        sim.reset()
        return grad_vel, None, None


__all__ = ["Fdtd", "FdtdFn", "FdtdError"]
